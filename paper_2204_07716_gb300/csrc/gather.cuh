// Per-sample window geometry and the warp-cooperative gather of interleaved
// fields, shared by the interpolation and backward kernels.
#pragma once

#include <cuda_runtime.h>

#include "device_common.cuh"
#include "internal.h"

namespace fk {

// ---- per-sample window geometry ---------------------------------------------
template <typename T, int D>
struct SampleWin {
  int i0, i1, i2;   // first cell of the window per axis (unwrapped)
  T wl0, wl1;       // lane-distributed 1-D kernel values (axis l / w, tap l % w)
};

template <typename T, int D>
__device__ __forceinline__ SampleWin<T, D> sample_window(const GeoDev& g, int w, T beta, T halfw,
                                                         T ih0, T ih1, T ih2, T x0, T x1, T x2,
                                                         int lane) {
  SampleWin<T, D> sw;
  T off0, off1 = T(0), off2 = T(0);
  {
    const T u = x0 * ih0;
    const T f = ceil(u - halfw);
    sw.i0 = int(f);
    off0 = f - u;
  }
  sw.i1 = 0;
  sw.i2 = 0;
  if (D > 1) {
    const T u = x1 * ih1;
    const T f = ceil(u - halfw);
    sw.i1 = int(f);
    off1 = f - u;
  }
  if (D > 2) {
    const T u = x2 * ih2;
    const T f = ceil(u - halfw);
    sw.i2 = int(f);
    off2 = f - u;
  }
  const int ax = lane / w, t = lane % w;
  sw.wl0 = ax < D ? phi<T>(g.skind, w, beta, sel3<T>(ax, off0, off1, off2) + T(t)) : T(0);
  const int l2 = lane + 32, ax2 = l2 / w, t2 = l2 % w;
  sw.wl1 = ax2 < D ? phi<T>(g.skind, w, beta, sel3<T>(ax2, off0, off1, off2) + T(t2)) : T(0);
  return sw;
}

// Gather fields [f_first, f_first + fcount) of one sample from the global
// field grid (periodic wrap).  Lanes cover the fields.
template <typename T, int D, int W, int NCH>
__device__ __forceinline__ void gather_global(const T* __restrict__ fld, int64_t rec, int f_first,
                                              int fcount, int lane, const SampleWin<T, D>& sw,
                                              int w, int nf0, int nf1, int nf2, T* cellw,
                                              T acc[NCH]) {
#pragma unroll
  for (int ch = 0; ch < NCH; ++ch) acc[ch] = T(0);
  const T* fb = fld + f_first + lane;
  if constexpr (W > 0) {
    T wa[D][W];
#pragma unroll
    for (int d = 0; d < D; ++d)
#pragma unroll
      for (int t = 0; t < W; ++t) {
        const int l = d * W + t;
        wa[d][t] = l < 32 ? __shfl_sync(0xffffffffu, sw.wl0, l) : __shfl_sync(0xffffffffu, sw.wl1, l - 32);
      }
    const int ilast = D == 1 ? sw.i0 : (D == 2 ? sw.i1 : sw.i2);
    const int nlast = D == 1 ? nf0 : (D == 2 ? nf1 : nf2);
    int64_t clf[W];
#pragma unroll
    for (int t = 0; t < W; ++t) clf[t] = wrap_idx(ilast + t, nlast) * rec;
    if (D == 1) {
#pragma unroll
      for (int t0 = 0; t0 < W; ++t0) {
        const T* q = fb + clf[t0];
        const T v = wa[0][t0];
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch)
          if (lane + ch * 32 < fcount) acc[ch] += __ldg(q + ch * 32) * v;
      }
    } else if (D == 2) {
#pragma unroll
      for (int t0 = 0; t0 < W; ++t0) {
        const T* rowp = fb + wrap_idx(sw.i0 + t0, nf0) * nf1 * rec;
        const T w0 = wa[0][t0];
#pragma unroll
        for (int t1 = 0; t1 < W; ++t1) {
          const T* q = rowp + clf[t1];
          const T v = w0 * wa[D - 1][t1];
#pragma unroll
          for (int ch = 0; ch < NCH; ++ch)
            if (lane + ch * 32 < fcount) acc[ch] += __ldg(q + ch * 32) * v;
        }
      }
    } else {
#pragma unroll 1
      for (int t0 = 0; t0 < W; ++t0) {
        const int64_t r0 = wrap_idx(sw.i0 + t0, nf0) * nf1;
#pragma unroll
        for (int t1 = 0; t1 < W; ++t1) {
          const T* rowp = fb + (r0 + wrap_idx(sw.i1 + t1, nf1)) * nf2 * rec;
          const T w01 = wa[0][t0] * wa[1 % D][t1];
#pragma unroll
          for (int t2 = 0; t2 < W; ++t2) {
            const T* q = rowp + clf[t2];
            const T v = w01 * wa[D - 1][t2];
#pragma unroll
            for (int ch = 0; ch < NCH; ++ch)
              if (lane + ch * 32 < fcount) acc[ch] += __ldg(q + ch * 32) * v;
          }
        }
      }
    }
  } else {
    // runtime width: tensor-product cell weights through shared memory
    int ncw = 1;
    for (int j = 0; j < D; ++j) ncw *= w;
    for (int c0 = 0; c0 < ncw; c0 += 32) {
      const int c = c0 + lane;
      int rem = c < ncw ? c : 0;
      T v = T(1);
      for (int d = D - 1; d >= 0; --d) {
        const int t = rem % w;
        rem /= w;
        const int l = d * w + t;
        const T a0 = __shfl_sync(0xffffffffu, sw.wl0, l & 31);
        const T a1 = __shfl_sync(0xffffffffu, sw.wl1, l & 31);
        v *= (l < 32) ? a0 : a1;
      }
      if (c < ncw) cellw[c] = v;
    }
    __syncwarp();
    for (int c = 0; c < ncw; ++c) {
      int rem = c;
      int64_t cell = 0, mult = 1;
      for (int d = D - 1; d >= 0; --d) {
        const int t = rem % w;
        rem /= w;
        const int id = d == 0 ? sw.i0 : (d == 1 ? sw.i1 : sw.i2);
        const int nfd = d == 0 ? nf0 : (d == 1 ? nf1 : nf2);
        cell += wrap_idx(id + t, nfd) * mult;
        mult *= nfd;
      }
      const T* q = fb + cell * rec;
      const T v = cellw[c];
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch)
        if (lane + ch * 32 < fcount) acc[ch] += q[ch * 32] * v;
    }
    __syncwarp();
  }
}

}  // namespace fk
