// probe_kernels.cu -- throughput probe of the fused multiply-add pipes.
//
// The on-chip FTCS kernels are bound by the FP64 pipe (FP64 runs: three DFMA
// per update) or by the FP32 FMA pipe (FP32 runs).  Their roofline is the rate
// at which one GB300 retires those instructions; this probe measures it: every
// thread advances independent chains a <- fma(a, b, c), so nothing but the
// pipe limits the rate.  The caller times one launch with CUDA events.
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "heat1d.h"
#include "impl.h"

namespace {

template <typename real, int kChains>
__global__ void fma_rate_kernel(int64_t iters, real b, real c, real* out) {
  real a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = static_cast<real>(threadIdx.x + j) * static_cast<real>(1e-3);
#pragma unroll 4
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
  }
  real s = static_cast<real>(0);
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  out[static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x] = s;
}

// The FTCS update's own instruction pattern: kPts points per thread in two
// register arrays, each step a = fma(r, fma(one, fma(-2, a_i, a_{i+1}), a_{i-1}),
// a_i) on a ring of the thread's points (no shuffles, no memory): the three
// fused multiply-adds per point of the stencil kernels, with the same
// operand dependencies.
template <typename real, int kPts>
__global__ void stencil_rate_kernel(int64_t iters, real r, real one, real* out) {
  real x[kPts], y[kPts];
#pragma unroll
  for (int j = 0; j < kPts; ++j) x[j] = static_cast<real>(threadIdx.x + 3 * j) * static_cast<real>(1e-3);
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kPts; ++j)
      y[j] = fma(r, fma(one, fma(static_cast<real>(-2), x[j], x[(j + 1) % kPts]), x[(j + kPts - 1) % kPts]), x[j]);
#pragma unroll
    for (int j = 0; j < kPts; ++j)
      x[j] = fma(r, fma(one, fma(static_cast<real>(-2), y[j], y[(j + 1) % kPts]), y[(j + kPts - 1) % kPts]), y[j]);
  }
  real s = static_cast<real>(0);
#pragma unroll
  for (int j = 0; j < kPts; ++j) s += x[j];
  out[static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int heat1d_probe_fma(int dtype, int chains, int64_t iters, int64_t blocks, int threads, void* out,
                                void* stream, int64_t* fma_per_launch) {
  if (dtype != HEAT1D_F32 && dtype != HEAT1D_F64) {
    heat1d_impl::set_last_error("heat1d_probe_fma: dtype must be HEAT1D_F32 or HEAT1D_F64");
    return HEAT1D_ERR_INVAL;
  }
  if (chains != 4 && chains != 8 && chains != 16 && chains != -8 && chains != -16) {
    heat1d_impl::set_last_error("heat1d_probe_fma: chains must be 4, 8, 16, -8 or -16");
    return HEAT1D_ERR_INVAL;
  }
  if (iters < 1 || blocks < 1 || blocks > (1 << 20) || threads < 32 || threads > 1024 || threads % 32 || !out) {
    heat1d_impl::set_last_error("heat1d_probe_fma: bad launch shape or null output");
    return HEAT1D_ERR_INVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const dim3 grid(static_cast<unsigned>(blocks)), block(threads);
  // b < 1 and c small keep every chain finite (it converges to c / (1 - b)).
  if (dtype == HEAT1D_F64) {
    double* o = static_cast<double*>(out);
    if (chains == -8) stencil_rate_kernel<double, 8><<<grid, block, 0, st>>>(iters, 0.25, 1.0, o);
    if (chains == -16) stencil_rate_kernel<double, 16><<<grid, block, 0, st>>>(iters, 0.25, 1.0, o);
    if (chains == 4) fma_rate_kernel<double, 4><<<grid, block, 0, st>>>(iters, 0.999999, 1e-6, o);
    if (chains == 8) fma_rate_kernel<double, 8><<<grid, block, 0, st>>>(iters, 0.999999, 1e-6, o);
    if (chains == 16) fma_rate_kernel<double, 16><<<grid, block, 0, st>>>(iters, 0.999999, 1e-6, o);
  } else {
    float* o = static_cast<float*>(out);
    if (chains == -8) stencil_rate_kernel<float, 8><<<grid, block, 0, st>>>(iters, 0.25f, 1.0f, o);
    if (chains == -16) stencil_rate_kernel<float, 16><<<grid, block, 0, st>>>(iters, 0.25f, 1.0f, o);
    if (chains == 4) fma_rate_kernel<float, 4><<<grid, block, 0, st>>>(iters, 0.999f, 1e-3f, o);
    if (chains == 8) fma_rate_kernel<float, 8><<<grid, block, 0, st>>>(iters, 0.999f, 1e-3f, o);
    if (chains == 16) fma_rate_kernel<float, 16><<<grid, block, 0, st>>>(iters, 0.999f, 1e-3f, o);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    heat1d_impl::set_last_error(std::string("heat1d_probe_fma: ") + cudaGetErrorString(e));
    return HEAT1D_ERR_CUDA;
  }
  // a stencil step is 3 fused multiply-adds per point, two steps per iteration
  if (fma_per_launch) *fma_per_launch = blocks * threads * iters * (chains > 0 ? chains : -chains * 6);
  return HEAT1D_OK;
}
