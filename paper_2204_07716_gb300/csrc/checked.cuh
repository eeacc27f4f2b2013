// The checked build (-DFKREG_CHECKED): range checks on the index arithmetic
// of the main kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace fk {

// ---- the checked build (-DFKREG_CHECKED) ------------------------------------
// Index arithmetic of the main kernels is range-checked before the access it
// guards: a failed check skips the access, sets kErrBounds in the plan's
// error word and records the first failing site and index there (read by
// fkreg_sync_status).  No check traps.  In the normal build in_range is the
// constant true and the compiler drops the checks.
#ifdef FKREG_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

enum CheckSite {
  kSiteSortScatter = 1,  // scatter position of a radix pass
  kSiteSortHist = 2,     // tile histogram of the next pass
  kSiteSortCoords = 3,   // sorted coordinates of the last pass
  kSiteSpreadTile = 4,   // shared-memory tile cell of the spreading
  kSiteSpreadFlush = 5,  // fine-grid cell of the tile flush
  kSiteInterpWindow = 6, // staged-window cell of the 2-D interpolation
  kSiteInterpField = 7,  // field-grid cell read from global memory
  kSiteSolveField = 8,   // lattice cell of the grid solve
  kSiteDirectBins = 9,   // bin range of the direct sums
  kSiteSelfTest = 15     // fkreg_checked_selftest
};

__device__ __forceinline__ bool in_range(int* errw, int site, int64_t i, int64_t n) {
  if constexpr (!kChecked) {
    return true;
  } else {
    const bool ok = i >= 0 && i < n;
    if (!ok && errw) {
      atomicOr(errw, kErrBounds);
      if (atomicCAS(errw + 1, 0, site) == 0) {
        errw[2] = int(uint32_t(uint64_t(i) & 0xffffffffu));
        errw[3] = int(uint32_t(uint64_t(i) >> 32));
      }
    }
    return ok;
  }
}

}  // namespace fk
