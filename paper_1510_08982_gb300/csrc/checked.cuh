// checked.cuh -- the bounds-checked build.
//
// Compiled with HEAT1D_CHECKED defined, the kernels compare every global
// index they compute for their buffers (state, snapshots, traces, edge
// buffers, rings, strips, edge histories) with the buffer's extent before the
// access.  An index outside it skips the access and records
// HEAT1D_ERR_BOUNDS in the run's status word; nothing traps, and the host
// reports the status after the run.  In the normal build the checks are
// compile-time `true` and cost nothing.
#pragma once

#include <cstdint>

#include "common.cuh"

namespace heat1d_dev {

#ifdef HEAT1D_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

// 0 <= i < n; in the checked build a false result records HEAT1D_ERR_BOUNDS.
__device__ __forceinline__ bool index_ok(int* status, int64_t i, int64_t n) {
  if constexpr (!kChecked) {
    return true;
  } else {
    if (i >= 0 && i < n) return true;
    raise_status(status, HEAT1D_ERR_BOUNDS);
    return false;
  }
}

}  // namespace heat1d_dev
