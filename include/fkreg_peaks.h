/*
 * fkreg_peaks.h - measured SM-side peaks of the current GPU.
 *
 * The paper has no counterpart: this is measurement tooling.  The spreading
 * and interpolation kernels of the smoother do w^d multiply-adds per sample
 * and field against a few bytes of HBM traffic, so their roofline is set by
 * the SM (FP32 FMA issue, shared-memory delivery, atomics), not by HBM.  This
 * call measures those rates on the device in use, with CUDA events on the
 * given stream, so the reported fractions rest on measured denominators.
 *
 * The call allocates nothing: the caller hands a device scratch buffer
 * (scratch_bytes >= FKREG_PEAKS_SCRATCH_BYTES) that the global-atomic test
 * overwrites.  It synchronises the stream several times (about a second in
 * all) and changes no device setting (clocks are read, never set).
 *
 *   sm_count            cudaDevAttrMultiProcessorCount
 *   sm_mhz              SM clock during the FP32 test: clock64() cycles of the
 *                       blocks / their event-timed duration
 *   fp32_tflops         scalar FFMA (2 flop per lane) over 8 independent chains
 *   fp32x2_tflops       packed FFMA2 (4 flop per lane)
 *   tf32_mma_tflops     warp-level TF32 tensor products (mma.sync m16n8k8,
 *                       FP32 accumulation; 2 x 16 x 8 x 8 flop each)
 *   smem_load_gbs[k]    shared-memory loads of 4, 8, 16 bytes per lane at
 *                       consecutive addresses (no bank conflicts), bytes
 *                       delivered to the lanes per second
 *   smem_bcast16_gbs    16-byte shared loads with every lane of a warp at one
 *                       address, bytes delivered to the lanes per second
 *   smem_atomic_gops    32-bit integer atomicAdd on shared memory, one address
 *                       per lane, operations per second (units of 1e9)
 *   gmem_atomic_gops    FP32 atomicAdd on global memory (an L2-resident
 *                       4 MB span), one address per lane, 1e9 ops per second
 * Returns FKREG_ERR_INVALID_ARG for a NULL out or a small scratch,
 * FKREG_ERR_CUDA if a CUDA call fails.
 */
#ifndef FKREG_PEAKS_H
#define FKREG_PEAKS_H

#include <stddef.h>

#include "fkreg.h"

#ifdef __cplusplus
extern "C" {
#endif

#define FKREG_PEAKS_SCRATCH_BYTES ((size_t)4 << 20)

typedef struct {
  int sm_count;
  double sm_mhz;
  double fp32_tflops;
  double fp32x2_tflops;
  double tf32_mma_tflops;
  double smem_load_gbs[3];
  double smem_bcast16_gbs;
  double smem_atomic_gops;
  double gmem_atomic_gops;
} fkreg_peaks;

fkreg_status fkreg_measure_peaks(fkreg_peaks* out, void* scratch_dev, size_t scratch_bytes,
                                 void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FKREG_PEAKS_H */
