// Entry points of the checked build (fkreg_checked_build, fkreg_check_selftest).
#include <cuda_runtime.h>

#include "checked.cuh"
#include "internal.h"

namespace fk {
namespace {

// One checked store at index 20 of a logical array of 16 ints that starts at
// errw + 16: the store, if it were not skipped, would land on errw[36],
// inside the 64-int error-word region.
__global__ void check_selftest_kernel(int* errw) {
  if (threadIdx.x == 0 && in_range(errw, kSiteSelfTest, 20, 16)) errw[16 + 20] = 1;
}

}  // namespace
}  // namespace fk

extern "C" int fkreg_checked_build(void) { return fk::kChecked ? 1 : 0; }

extern "C" fkreg_status fkreg_check_selftest(fkreg_plan P, void* stream) {
  if (!P || !P->ws) return FKREG_ERR_INVALID_ARG;
  fk::check_selftest_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(P->geo.errw);
  return cudaGetLastError() == cudaSuccess ? FKREG_OK : FKREG_ERR_CUDA;
}
