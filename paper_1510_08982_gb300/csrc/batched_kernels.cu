// batched_kernels.cu -- the batched launch's FP64 instances and the dispatch
// over precision and tile shape (the kernel itself is in batched_impl.cuh; the
// FP32 instances are compiled in batched_kernels_f32.cu, in parallel).
#include "batched_impl.cuh"

namespace heat1d_impl {

int launch_batched(const BatchRun& a, int dtype, int E, int threads, int grid, cudaStream_t st) {
  if (dtype != HEAT1D_F64) return launch_batched_f32(a, E, threads, grid, st);
  switch (E) {
    case 4: return launch_batched_t<double, 4>(a, threads, grid, st);
    case 8: return launch_batched_t<double, 8>(a, threads, grid, st);
    case 16: return launch_batched_t<double, 16>(a, threads, grid, st);
    default: return HEAT1D_ERR_INVAL;
  }
}

int max_resident_batched(int dtype, int E, int threads) {
  if (dtype != HEAT1D_F64) return max_resident_batched_f32(E, threads);
  switch (E) {
    case 4: return resident_batched_t<double, 4>(threads);
    case 8: return resident_batched_t<double, 8>(threads);
    case 16: return resident_batched_t<double, 16>(threads);
    default: return 0;
  }
}

}  // namespace heat1d_impl
