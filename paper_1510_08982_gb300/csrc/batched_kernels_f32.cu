// batched_kernels_f32.cu -- the batched launch's FP32 instances (the kernel
// is in batched_impl.cuh; compiled apart from the FP64 instances so that the
// two build in parallel).
#include "batched_impl.cuh"

namespace heat1d_impl {

int launch_batched_f32(const BatchRun& a, int E, int threads, int grid, cudaStream_t st) {
  switch (E) {
    case 4: return launch_batched_t<float, 4>(a, threads, grid, st);
    case 8: return launch_batched_t<float, 8>(a, threads, grid, st);
    case 16: return launch_batched_t<float, 16>(a, threads, grid, st);
    case 32: return launch_batched_t<float, 32>(a, threads, grid, st);
    default: return HEAT1D_ERR_INVAL;
  }
}

int max_resident_batched_f32(int E, int threads) {
  switch (E) {
    case 4: return resident_batched_t<float, 4>(threads);
    case 8: return resident_batched_t<float, 8>(threads);
    case 16: return resident_batched_t<float, 16>(threads);
    case 32: return resident_batched_t<float, 32>(threads);
    default: return 0;
  }
}

}  // namespace heat1d_impl
