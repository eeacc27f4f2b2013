// Type-2 interpolation back to the samples, the at-sample solve, and the
// DF / GCV reductions.
//
// Every sorted sample gathers the fields of one bandwidth from that
// bandwidth's fine grid with the spreading kernel (the uniform-to-non-uniform
// NUFFT that Sec. 1.1 mentions), solves the system of eq. 3 at q = x_i, and
// contributes to
//   rss_r      = sum_i (y_ri - mhat_r(x_i))^2                 (numerator of eq. 22)
//   wSw_p      = sum_i w_pi (S w_p)_i,  ww_p = sum_i w_pi^2   (Sec. 2.1)
//   tr_exact   = K_H(0) sum_i [S(x_i)^-1]_11                  (diagonal of S_h)
// Block partials are summed in a fixed order, so results are deterministic.
//
// Fields are stored interleaved per fine-grid cell ([cell][rec], rec >= F2
// a multiple of 4), so a warp gathers one sample at a time with its lanes
// spread over the fields: every load of the 32 lanes is one contiguous run.
// A warp walks a group of 32 consecutive sorted samples, parks each sample's
// field values in shared memory, and then each lane takes one sample for the
// FP64 solve and the reductions.  Fields go in passes of pass_f; pass 0 holds
// the s-fields.
//
// Two kernels share that structure.  The TMA kernel takes one spreading
// sub-problem (samples of one bin) at a time, copies the bin's window of the
// field grid (all fields) into shared memory with bulk asynchronous copies
// completing on an mbarrier, and gathers from there.  The global kernel
// gathers straight from the (cache-resident) field grid and serves 3-D and
// windows that do not fit shared memory.
#include <cuda_runtime.h>

#include <algorithm>

#include "device_common.cuh"
#include "gather.cuh"
#include "interp_common.cuh"
#include "internal.h"

namespace fk {

namespace {

constexpr int kI2Warps = 16;   // global kernel: warps per block (upper bound)
constexpr int kTWarps = 16;    // TMA kernel: warps per block (upper bound)
constexpr int kMaxWRun = 32;   // runtime-width fallback

// Gather from a window staged in shared memory: win[(l0 * e1 + l1) * rec + f],
// (l0, l1) = (i0 - o0, i1 - o1) already checked to lie inside the window.
template <typename T, int D, int W, int NCH>
__device__ __forceinline__ void gather_smem(const T* win, int rec, int e1, int l0, int l1,
                                            int f_first, int fcount, int lane,
                                            const SampleWin<T, D>& sw, T acc[NCH]) {
  static_assert(D <= 2 && W > 0, "shared-memory gather serves 1-D and 2-D with a fixed width");
#pragma unroll
  for (int ch = 0; ch < NCH; ++ch) acc[ch] = T(0);
  T wa[D][W];
#pragma unroll
  for (int d = 0; d < D; ++d)
#pragma unroll
    for (int t = 0; t < W; ++t) {
      const int l = d * W + t;
      wa[d][t] = l < 32 ? __shfl_sync(0xffffffffu, sw.wl0, l) : __shfl_sync(0xffffffffu, sw.wl1, l - 32);
    }
  const T* fb = win + f_first + lane;
  if (D == 1) {
    const T* q0 = fb + l0 * rec;
#pragma unroll
    for (int t0 = 0; t0 < W; ++t0) {
      const T v = wa[0][t0];
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch)
        if (lane + ch * 32 < fcount) acc[ch] += q0[t0 * rec + ch * 32] * v;
    }
  } else {
#pragma unroll
    for (int t0 = 0; t0 < W; ++t0) {
      const T* rowp = fb + ((l0 + t0) * e1 + l1) * rec;
      const T w0 = wa[0][t0];
#pragma unroll
      for (int t1 = 0; t1 < W; ++t1) {
        const T v = w0 * wa[D - 1][t1];
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch)
          if (lane + ch * 32 < fcount) acc[ch] += rowp[t1 * rec + ch * 32] * v;
      }
    }
  }
}

// Two samples at once from a staged window, FP32, every field in one pass
// (F2 <= 64): lane l accumulates fields 2l and 2l+1 with 8-byte shared loads,
// and the two samples' independent chains hide each other's latency.
template <int D, int W>
__device__ __forceinline__ void gather_smem_pair(const float* win, int rec, int e1, int la0,
                                                 int la1, int lb0, int lb1, int lane, bool active,
                                                 const SampleWin<float, D>& swa,
                                                 const SampleWin<float, D>& swb, float2& acca,
                                                 float2& accb) {
  float wa[D][W], wb[D][W];
#pragma unroll
  for (int d = 0; d < D; ++d)
#pragma unroll
    for (int t = 0; t < W; ++t) {
      const int l = d * W + t;
      wa[d][t] = l < 32 ? __shfl_sync(0xffffffffu, swa.wl0, l) : __shfl_sync(0xffffffffu, swa.wl1, l - 32);
      wb[d][t] = l < 32 ? __shfl_sync(0xffffffffu, swb.wl0, l) : __shfl_sync(0xffffffffu, swb.wl1, l - 32);
    }
  acca = make_float2(0.f, 0.f);
  accb = make_float2(0.f, 0.f);
  if (!active) return;
  const float* fa = win + 2 * lane;
  if (D == 1) {
#pragma unroll
    for (int t0 = 0; t0 < W; ++t0) {
      const float2 va = *reinterpret_cast<const float2*>(fa + (la0 + t0) * rec);
      const float2 vb = *reinterpret_cast<const float2*>(fa + (lb0 + t0) * rec);
      acca.x += va.x * wa[0][t0];
      acca.y += va.y * wa[0][t0];
      accb.x += vb.x * wb[0][t0];
      accb.y += vb.y * wb[0][t0];
    }
  } else {
#pragma unroll
    for (int t0 = 0; t0 < W; ++t0) {
      const float* ra = fa + ((la0 + t0) * e1 + la1) * rec;
      const float* rb = fa + ((lb0 + t0) * e1 + lb1) * rec;
      float2 ra2 = make_float2(0.f, 0.f), rb2 = make_float2(0.f, 0.f);
#pragma unroll
      for (int t1 = 0; t1 < W; ++t1) {
        const float2 va = *reinterpret_cast<const float2*>(ra + t1 * rec);
        const float2 vb = *reinterpret_cast<const float2*>(rb + t1 * rec);
        ra2.x += va.x * wa[D - 1][t1];
        ra2.y += va.y * wa[D - 1][t1];
        rb2.x += vb.x * wb[D - 1][t1];
        rb2.y += vb.y * wb[D - 1][t1];
      }
      acca.x += ra2.x * wa[0][t0];
      acca.y += ra2.y * wa[0][t0];
      accb.x += rb2.x * wb[0][t0];
      accb.y += rb2.y * wb[0][t0];
    }
  }
}

// Gather-only mode: the pass's field values of this lane's sample go to
// V[f][s] (sorted sample order; consecutive lanes write consecutive samples).
template <typename T>
__device__ __forceinline__ void store_fields(T* __restrict__ V, const T* my, int f_first,
                                             int fcount, bool valid, int64_t s, int64_t n) {
  if (!valid) return;
  for (int f = 0; f < fcount; ++f) V[int64_t(f_first + f) * n + s] = my[f];
}

// ---- kernel 1: gathers from the global field grid ---------------------------
template <typename T, int D, int W, int NCH>
__global__ void __launch_bounds__(kI2Warps * 32)
interp_kernel(GeoDev g, MonoTab mono, const BwDev* __restrict__ bwt, int b, int order, int64_t n,
              const T* __restrict__ xs, const T* __restrict__ str, const uint32_t* __restrict__ perm,
              const T* __restrict__ fld, int rec, int F2, int pass_f, int n_rhs_real, int n_probes,
              int cplx, int n_rhs_out, T* __restrict__ mhat_at_x, int nacc, int nbw,
              double* __restrict__ part, T* __restrict__ vout) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = int(blockDim.x >> 5);
  const int w = W > 0 ? W : g.w;
  int ncw = 1;
  for (int j = 0; j < D; ++j) ncw *= w;
  if (W > 0) ncw = 0;
  const int bstride = pass_f + 1;
  double* red_all = reinterpret_cast<double*>(smem_raw);
  double* red = red_all + warp * nacc;
  T* cellw = reinterpret_cast<T*>(red_all + nwarps * nacc) + warp * ncw;
  T* buf = reinterpret_cast<T*>(red_all + nwarps * nacc) + nwarps * ncw + warp * 32 * bstride;
  for (int a = lane; a < nacc; a += 32) red[a] = 0.0;
  __syncwarp();
  const BwDev& B = bwt[b];
  const int nf0 = int(B.nf[0]), nf1 = D > 1 ? int(B.nf[1]) : 1, nf2 = D > 2 ? int(B.nf[2]) : 1;
  const T ih0 = T(B.inv_h[0]), ih1 = T(D > 1 ? B.inv_h[1] : 1.0), ih2 = T(D > 2 ? B.inv_h[2] : 1.0);
  const T beta = T(g.beta);
  const T halfw = T(0.5) * T(w);
  GroupCtx c{mono.n, mono.nt, mono.nt, n_rhs_real + n_probes, n_rhs_real, n_probes, cplx,
             n_rhs_out, nacc, order, b};
  T tsc[kMaxP];
#pragma unroll
  for (int k = 0; k < kMaxP; ++k) tsc[k] = (k < c.p) ? T(1.0 / tscale(mono, k, B.sigma)) : T(0);
  const T k0t = T(B.k0);
  const double isg[3] = {1.0 / B.sigma[0], 1.0 / B.sigma[1], 1.0 / B.sigma[2]};
  // each block walks one contiguous run of sample groups (neighbouring bins)
  const int64_t ngroups = (n + 31) / 32;
  const int64_t per_block = (ngroups + gridDim.x - 1) / gridDim.x;
  const int64_t g_begin = int64_t(blockIdx.x) * per_block;
  const int64_t g_end = min(ngroups, g_begin + per_block);
  for (int64_t grp = g_begin + warp; grp < g_end; grp += nwarps) {
    const int64_t s0 = grp * 32;
    const int cnt = int(min(int64_t(32), n - s0));
    const int64_t s = s0 + lane;
    const bool valid = lane < cnt;
    T af[kMaxP] = {T(0), T(0), T(0), T(0)};
    int q_done = 0, f_first = 0;
    for (int pass = 0; f_first < F2; ++pass) {
      const int q_in = vout ? 0
                            : (pass == 0 ? min(c.nq, (pass_f - c.ns) / c.nt)
                                         : min(c.nq - q_done, pass_f / c.nt));
      const int f_last =
          vout ? min(F2, f_first + pass_f) : (pass == 0 ? c.ns : f_first) + q_in * c.nt;
      const int fcount = f_last - f_first;
      T xn0 = xs[s0], xn1 = D > 1 ? xs[n + s0] : T(0), xn2 = D > 2 ? xs[2 * n + s0] : T(0);
      for (int j = 0; j < cnt; ++j) {
        const T x0 = xn0, x1 = xn1, x2 = xn2;
        if (j + 1 < cnt) {  // prefetch the next sample's coordinates
          xn0 = xs[s0 + j + 1];
          if (D > 1) xn1 = xs[n + s0 + j + 1];
          if (D > 2) xn2 = xs[2 * n + s0 + j + 1];
        }
        const SampleWin<T, D> sw =
            sample_window<T, D>(g, w, beta, halfw, ih0, ih1, ih2, x0, x1, x2, lane);
        T acc[NCH];
        gather_global<T, D, W, NCH>(fld, rec, f_first, fcount, lane, sw, w, nf0, nf1, nf2, cellw, acc);
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch)
          if (lane + ch * 32 < fcount) buf[j * bstride + lane + ch * 32] = acc[ch];
        __syncwarp();
      }
      if (vout)
        store_fields<T>(vout, buf + lane * bstride, f_first, fcount, valid, s, n);
      else
        finish_pass<T>(c, mono, B, buf + lane * bstride, pass, q_done, q_in, lane, valid, n,
                       str + n + s, n, valid ? perm[s] : 0u, mhat_at_x, tsc, af, red, k0t, isg);
      __syncwarp();
      q_done += q_in;
      f_first = f_last;
    }
  }
  __syncthreads();
  for (int a = threadIdx.x; a < nacc; a += blockDim.x) {
    double t = 0.0;
    for (int wv = 0; wv < nwarps; ++wv) t += red_get<T>(red_all, wv * nacc + a);
    part[(int64_t(blockIdx.x) * nbw + b) * nacc + a] = t;
  }
}

// ---- kernel 2: bin windows staged in shared memory by bulk copies ----------
// One block takes spreading sub-problems (samples of one bin) in turn.  The
// bin's window of the field grid, [wm0][wm1][rec] cells x fields, is copied
// row by row with cp.async.bulk (periodic wrap splits a row in two), the
// copies complete on an mbarrier, and the warps gather from shared memory.
// The wait is bounded: if it gives up, the block raises the timeout bit of
// the error word, waits once more (bounded) for its copies, and exits.
template <typename T, int D, int W, int NCH>
__global__ void __launch_bounds__(kTWarps * 32)
interp_tma_kernel(GeoDev g, MonoTab mono, const BwDev* __restrict__ bwt, int b, int order,
                  int64_t n, const T* __restrict__ xs, const T* __restrict__ str,
                  const uint32_t* __restrict__ perm, const T* __restrict__ fld, int rec, int F2,
                  int pass_f, int n_rhs_real, int n_probes, int cplx, int n_rhs_out,
                  T* __restrict__ mhat_at_x, int nacc, int nbw, double* __restrict__ part,
                  const uint32_t* __restrict__ sub_bin, const uint32_t* __restrict__ sub_first,
                  const uint32_t* __restrict__ bin_start, const uint32_t* __restrict__ sub_total,
                  int wm0, int wm1, int lo_slack, int bstride_in, int* __restrict__ errw,
                  T* __restrict__ vout) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t mbar;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = int(blockDim.x >> 5);
  const int bstride = bstride_in;
  const size_t win_bytes = (size_t(wm0) * wm1 * rec * sizeof(T) + 127) / 128 * 128;
  T* win = reinterpret_cast<T*>(smem_raw);
  double* red_all = reinterpret_cast<double*>(smem_raw + win_bytes);
  double* red = red_all + warp * nacc;
  T* buf = reinterpret_cast<T*>(red_all + nwarps * nacc) + warp * 32 * bstride;
  for (int a = lane; a < nacc; a += 32) red[a] = 0.0;
  if (threadIdx.x == 0) {
    mbar_init(&mbar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  const BwDev& B = bwt[b];
  const int nf0 = int(B.nf[0]), nf1 = D > 1 ? int(B.nf[1]) : 1;
  const T ih0 = T(B.inv_h[0]), ih1 = T(D > 1 ? B.inv_h[1] : 1.0);
  const double r0 = double(B.nf[0]) / double(g.nf[0]);
  const double r1 = D > 1 ? double(B.nf[1]) / double(g.nf[1]) : 1.0;
  const T beta = T(g.beta);
  const T halfw = T(0.5) * T(W);
  GroupCtx c{mono.n, mono.nt, mono.nt, n_rhs_real + n_probes, n_rhs_real, n_probes, cplx,
             n_rhs_out, nacc, order, b};
  T tsc[kMaxP];
#pragma unroll
  for (int k = 0; k < kMaxP; ++k) tsc[k] = (k < c.p) ? T(1.0 / tscale(mono, k, B.sigma)) : T(0);
  const T k0t = T(B.k0);
  const double isg[3] = {1.0 / B.sigma[0], 1.0 / B.sigma[1], 1.0 / B.sigma[2]};
  uint32_t parity = 0;
  const uint32_t nsub = *sub_total;
  bool failed = false;
  for (uint32_t k = blockIdx.x; k < nsub; k += gridDim.x) {
    const uint32_t bin = sub_bin[k];
    const uint32_t first = sub_first[k];
    const uint32_t last = min(first + uint32_t(kSubMax), bin_start[bin + 1]);
    const int64_t bj0 = D > 1 ? int64_t(bin) / g.nbins[1] : int64_t(bin);
    const int64_t bj1 = D > 1 ? int64_t(bin) % g.nbins[1] : 0;
    const int o0 = int(floor(double(bj0 * g.tile[0]) * r0)) - g.pad - lo_slack;
    const int o1 = D > 1 ? int(floor(double(bj1 * g.tile[1]) * r1)) - g.pad - lo_slack : 0;
    if (threadIdx.x == 0)
      issue_window_copies<T, D>(fld, rec, nf0, nf1, o0, o1, wm0, wm1, wm1 * rec, win, &mbar);
    bool ok = false;
    for (uint32_t it = 0; it < g.wait_limit && !ok; ++it) ok = mbar_try_wait(&mbar, parity);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) atomicOr(errw, 2);
      bool late = false;
      for (uint32_t it = 0; it < kMaxSpin && !late; ++it) late = mbar_try_wait(&mbar, parity);
      failed = true;
      break;
    }
    parity ^= 1u;
    const int ngr = int((last - first + 31) / 32);
    for (int gi = warp; gi < ngr; gi += nwarps) {
      const int64_t s0 = int64_t(first) + int64_t(gi) * 32;
      const int cnt = int(min(int64_t(32), int64_t(last) - s0));
      const int64_t s = s0 + lane;
      const bool valid = lane < cnt;
      T af[kMaxP] = {T(0), T(0), T(0), T(0)};
      int q_done = 0, f_first = 0;
      for (int pass = 0; f_first < F2; ++pass) {
        const int q_in = vout ? 0
                              : (pass == 0 ? min(c.nq, (pass_f - c.ns) / c.nt)
                                           : min(c.nq - q_done, pass_f / c.nt));
        const int f_last =
            vout ? min(F2, f_first + pass_f) : (pass == 0 ? c.ns : f_first) + q_in * c.nt;
        const int fcount = f_last - f_first;
        bool paired = false;
        if constexpr (sizeof(T) == 4) {
          // every field in one pass: two samples at a time, 8-byte loads
          if (F2 <= 64 && fcount == F2) {
            paired = true;
            for (int j = 0; j < cnt; j += 2) {
              const int jb = j + 1 < cnt ? j + 1 : j;
              const T xa0 = xs[s0 + j], xa1 = D > 1 ? xs[n + s0 + j] : T(0);
              const T xb0 = xs[s0 + jb], xb1 = D > 1 ? xs[n + s0 + jb] : T(0);
              const SampleWin<T, D> swa =
                  sample_window<T, D>(g, W, beta, halfw, ih0, ih1, T(1), xa0, xa1, T(0), lane);
              const SampleWin<T, D> swb =
                  sample_window<T, D>(g, W, beta, halfw, ih0, ih1, T(1), xb0, xb1, T(0), lane);
              const int la0 = swa.i0 - o0, la1 = D > 1 ? swa.i1 - o1 : 0;
              const int lb0 = swb.i0 - o0, lb1 = D > 1 ? swb.i1 - o1 : 0;
              const bool in_a = la0 >= 0 && la0 + W <= wm0 && (D == 1 || (la1 >= 0 && la1 + W <= wm1));
              const bool in_b = lb0 >= 0 && lb0 + W <= wm0 && (D == 1 || (lb1 >= 0 && lb1 + W <= wm1));
              if (in_a && in_b) {
                float2 acca, accb;
                gather_smem_pair<D, W>(reinterpret_cast<const float*>(win), rec, D > 1 ? wm1 : 1,
                                       la0, la1, lb0, lb1, lane, 2 * lane < rec, swa, swb, acca,
                                       accb);
                T* oa = buf + j * bstride + 2 * lane;
                T* ob = buf + jb * bstride + 2 * lane;
                if (2 * lane < fcount) oa[0] = acca.x;
                if (2 * lane + 1 < fcount) oa[1] = acca.y;
                if (jb != j) {
                  if (2 * lane < fcount) ob[0] = accb.x;
                  if (2 * lane + 1 < fcount) ob[1] = accb.y;
                }
              } else {
                auto one = [&](const SampleWin<T, D>& sw, int l0, int l1, bool in, int jj) {
                  T acc[NCH];
                  if (in)
                    gather_smem<T, D, W, NCH>(win, rec, D > 1 ? wm1 : 1, l0, l1, f_first, fcount,
                                              lane, sw, acc);
                  else
                    gather_global<T, D, W, NCH>(fld, rec, f_first, fcount, lane, sw, W, nf0, nf1, 1,
                                                nullptr, acc);
#pragma unroll
                  for (int ch = 0; ch < NCH; ++ch)
                    if (lane + ch * 32 < fcount) buf[jj * bstride + lane + ch * 32] = acc[ch];
                };
                one(swa, la0, la1, in_a, j);
                if (jb != j) one(swb, lb0, lb1, in_b, jb);
              }
              __syncwarp();
            }
          }
        }
        T xn0 = xs[s0], xn1 = D > 1 ? xs[n + s0] : T(0);
        for (int j = 0; j < (paired ? 0 : cnt); ++j) {
          const T x0 = xn0, x1 = xn1;
          if (j + 1 < cnt) {
            xn0 = xs[s0 + j + 1];
            if (D > 1) xn1 = xs[n + s0 + j + 1];
          }
          const SampleWin<T, D> sw =
              sample_window<T, D>(g, W, beta, halfw, ih0, ih1, T(1), x0, x1, T(0), lane);
          const int l0 = sw.i0 - o0, l1 = D > 1 ? sw.i1 - o1 : 0;
          const bool inside =
              l0 >= 0 && l0 + W <= wm0 && (D == 1 || (l1 >= 0 && l1 + W <= wm1));
          T acc[NCH];
          if (inside)
            gather_smem<T, D, W, NCH>(win, rec, D > 1 ? wm1 : 1, l0, l1, f_first, fcount, lane, sw,
                                      acc);
          else
            gather_global<T, D, W, NCH>(fld, rec, f_first, fcount, lane, sw, W, nf0, nf1, 1,
                                        nullptr, acc);
#pragma unroll
          for (int ch = 0; ch < NCH; ++ch)
            if (lane + ch * 32 < fcount) buf[j * bstride + lane + ch * 32] = acc[ch];
          __syncwarp();
        }
        if (vout)
          store_fields<T>(vout, buf + lane * bstride, f_first, fcount, valid, s, n);
        else
          finish_pass<T>(c, mono, B, buf + lane * bstride, pass, q_done, q_in, lane, valid, n,
                         str + n + s, n, valid ? perm[s] : 0u, mhat_at_x, tsc, af, red, k0t, isg);
        __syncwarp();
        q_done += q_in;
        f_first = f_last;
      }
    }
    __syncthreads();  // every read of this window is done before the next copies
  }
  if (failed) return;
  __syncthreads();
  for (int a = threadIdx.x; a < nacc; a += blockDim.x) {
    double t = 0.0;
    for (int wv = 0; wv < nwarps; ++wv) t += red_get<T>(red_all, wv * nacc + a);
    part[(int64_t(blockIdx.x) * nbw + b) * nacc + a] = t;
  }
}

// ---- kernel 3: one lane per sample over a staged window (FP32, fixed W) ----
// Same sub-problem loop and window staging as kernel 2, but each lane takes
// one sample of the group and walks the window cells and the float4 quads
// of the fields itself: every shared load is 16 bytes, every lane does useful
// multiply-adds, and because sorted samples that share a window are adjacent
// most loads of a warp are broadcasts of a few addresses.  The lane's field
// values go to its own row of the staging buffer (or straight to V in the
// gather-only mode) and phase B follows as in the other kernels.
template <int D, int W, int NQ>
__global__ void __launch_bounds__(kLWarps * 32)
interp_lane_kernel(GeoDev g, MonoTab mono, const BwDev* __restrict__ bwt, int b, int order,
                   int64_t n, const float* __restrict__ xs, const float* __restrict__ str,
                   const uint32_t* __restrict__ perm, const float* __restrict__ fld, int rec,
                   int F2, int pass_f, int n_rhs_real, int n_probes, int cplx, int n_rhs_out,
                   float* __restrict__ mhat_at_x, int nacc, int nbw, double* __restrict__ part,
                   const uint32_t* __restrict__ sub_bin, const uint32_t* __restrict__ sub_first,
                   const uint32_t* __restrict__ bin_start, const uint32_t* __restrict__ sub_total,
                   int wm0, int wm1, int pitch, int lo_slack, int bstride, int cst,
                   int* __restrict__ errw, float* __restrict__ vout) {
  using T = float;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t mbar;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = int(blockDim.x >> 5);
  const size_t win_bytes = (size_t(D > 1 ? wm0 : 1) * pitch * sizeof(T) + 127) / 128 * 128;
  T* win = reinterpret_cast<T*>(smem_raw);
  double* red_all = reinterpret_cast<double*>(smem_raw + win_bytes);
  double* red = red_all + warp * nacc;
  T* my = reinterpret_cast<T*>(red_all + nwarps * nacc) + (warp * 32 + lane) * bstride;
  // this lane's strengths (responses, probes) of its sample, copied ahead
  T* cvs = reinterpret_cast<T*>(red_all + nwarps * nacc) + nwarps * 32 * bstride +
           (warp * 32 + lane) * cst;
  for (int a = lane; a < nacc; a += 32) red[a] = 0.0;
  if (threadIdx.x == 0) {
    mbar_init(&mbar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  const BwDev& B = bwt[b];
  const int nf0 = int(B.nf[0]), nf1 = D > 1 ? int(B.nf[1]) : 1;
  const T ih0 = T(B.inv_h[0]), ih1 = T(D > 1 ? B.inv_h[1] : 1.0);
  const double r0 = double(B.nf[0]) / double(g.nf[0]);
  const double r1 = D > 1 ? double(B.nf[1]) / double(g.nf[1]) : 1.0;
  const T beta = T(g.beta);
  const T halfw = T(0.5) * T(W);
  const int skind = g.skind;
  GroupCtx c{mono.n, mono.nt, mono.nt, n_rhs_real + n_probes, n_rhs_real, n_probes, cplx,
             n_rhs_out, nacc, order, b};
  T tsc[kMaxP];
#pragma unroll
  for (int k = 0; k < kMaxP; ++k) tsc[k] = (k < c.p) ? T(1.0 / tscale(mono, k, B.sigma)) : T(0);
  const T k0t = T(B.k0);
  const double isg[3] = {1.0 / B.sigma[0], 1.0 / B.sigma[1], 1.0 / B.sigma[2]};
  uint32_t parity = 0;
  const uint32_t nsub = *sub_total;
  bool failed = false;
  for (uint32_t k = blockIdx.x; k < nsub; k += gridDim.x) {
    const uint32_t bin = sub_bin[k];
    const uint32_t first = sub_first[k];
    const uint32_t last = min(first + uint32_t(kSubMax), bin_start[bin + 1]);
    const int64_t bj0 = D > 1 ? int64_t(bin) / g.nbins[1] : int64_t(bin);
    const int64_t bj1 = D > 1 ? int64_t(bin) % g.nbins[1] : 0;
    const int o0 = int(floor(double(bj0 * g.tile[0]) * r0)) - g.pad - lo_slack;
    const int o1 = D > 1 ? int(floor(double(bj1 * g.tile[1]) * r1)) - g.pad - lo_slack : 0;
    if (threadIdx.x == 0)
      issue_window_copies<T, D>(fld, rec, nf0, nf1, o0, o1, wm0, wm1, pitch, win, &mbar);
    bool ok = false;
    for (uint32_t it = 0; it < g.wait_limit && !ok; ++it) ok = mbar_try_wait(&mbar, parity);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) atomicOr(errw, 2);
      bool late = false;
      for (uint32_t it = 0; it < kMaxSpin && !late; ++it) late = mbar_try_wait(&mbar, parity);
      failed = true;
      break;
    }
    parity ^= 1u;
    const int ngr = int((last - first + 31) / 32);
    // coordinates of this lane's sample, one group ahead
    T xn0 = T(0), xn1 = T(0);
    if (warp < ngr) {
      const int64_t sn = min(int64_t(first) + int64_t(warp) * 32 + lane, int64_t(last) - 1);
      xn0 = xs[sn];
      if (D > 1) xn1 = xs[n + sn];
    }
    for (int gi = warp; gi < ngr; gi += nwarps) {
      const int64_t s0 = int64_t(first) + int64_t(gi) * 32;
      const int cnt = int(min(int64_t(32), int64_t(last) - s0));
      const int64_t s = s0 + lane;
      const bool valid = lane < cnt;
      const T x0 = xn0, x1 = xn1;
      if (gi + nwarps < ngr) {
        const int64_t sn =
            min(int64_t(first) + int64_t(gi + nwarps) * 32 + lane, int64_t(last) - 1);
        xn0 = xs[sn];
        if (D > 1) xn1 = xs[n + sn];
      }
      uint32_t orig = 0u;
      if (!vout && valid) {
        orig = perm[s];
        for (int q = 0; q < c.nq; ++q) cp_async4(cvs + q, str + int64_t(1 + q) * n + s);
      }
      // window of this lane's sample (same rounding as the bin rule)
      const T u0 = __fmul_rn(x0, ih0);
      const T fo0 = ceilf(__fsub_rn(u0, halfw));
      const int i0 = int(fo0);
      const T off0 = fo0 - u0;
      int i1 = 0;
      T off1 = T(0);
      if (D > 1) {
        const T u1 = __fmul_rn(x1, ih1);
        const T fo1 = ceilf(__fsub_rn(u1, halfw));
        i1 = int(fo1);
        off1 = fo1 - u1;
      }
      const int l0 = i0 - o0, l1 = D > 1 ? i1 - o1 : 0;
      const bool inside = l0 >= 0 && l0 + W <= wm0 && (D == 1 || (l1 >= 0 && l1 + W <= wm1));
      T pl[W];  // kernel values along the last axis
#pragma unroll
      for (int t = 0; t < W; ++t) pl[t] = phi<T>(skind, W, beta, (D > 1 ? off1 : off0) + T(t));
      T af[kMaxP] = {T(0), T(0), T(0), T(0)};
      int q_done = 0, f_first = 0;
      for (int pass = 0; f_first < F2; ++pass) {
        const int q_in = vout ? 0
                              : (pass == 0 ? min(c.nq, (pass_f - c.ns) / c.nt)
                                           : min(c.nq - q_done, pass_f / c.nt));
        const int f_last =
            vout ? min(F2, f_first + pass_f) : (pass == 0 ? c.ns : f_first) + q_in * c.nt;
        const int qa = f_first >> 2, nq = ((f_last + 3) >> 2) - qa;
        float4 acc[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (inside)
          lane_gather_smem<D, W, NQ>(win + size_t(l0) * (D > 1 ? pitch : rec) + l1 * rec + 4 * qa,
                                     rec, pitch, nq, skind, beta, off0, pl, acc);
        if (__any_sync(0xffffffffu, valid && !inside)) {
          if (valid && !inside)
            lane_gather_global<D, W, NQ>(fld, rec, qa, nq, i0, i1, nf0, nf1, skind, beta, off0, pl,
                                         acc);
        }
        if (vout) {
          if (valid)
#pragma unroll
            for (int q = 0; q < NQ; ++q)
#pragma unroll
              for (int cc = 0; cc < 4; ++cc) {
                const int f = 4 * (qa + q) + cc;
                if (q < nq && f >= f_first && f < f_last) vout[int64_t(f) * n + s] = quad_comp(acc[q], cc);
              }
        } else {
#pragma unroll
          for (int q = 0; q < NQ; ++q)
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
              const int f = 4 * (qa + q) + cc;
              if (q < nq && f >= f_first && f < f_last) my[f - f_first] = quad_comp(acc[q], cc);
            }
          if (pass == 0) cp_async_wait_all();
          finish_pass<T>(c, mono, B, my, pass, q_done, q_in, lane, valid, n, cvs + q_done, 1,
                         orig, mhat_at_x, tsc, af, red, k0t, isg);
        }
        q_done += q_in;
        f_first = f_last;
      }
    }
    __syncthreads();  // every read of this window is done before the next copies
  }
  if (failed) return;
  __syncthreads();
  for (int a = threadIdx.x; a < nacc; a += blockDim.x) {
    double t = 0.0;
    for (int wv = 0; wv < nwarps; ++wv) t += red_get<T>(red_all, wv * nacc + a);
    part[(int64_t(blockIdx.x) * nbw + b) * nacc + a] = t;
  }
}

// sum block partials in a fixed order: sums[b][a]; one block per output
__global__ void reduce_partials(const double* __restrict__ part, int64_t nblk, int nbw, int nacc,
                                double* __restrict__ sums) {
  __shared__ double sh[256];
  const int o = blockIdx.x;
  double t = 0.0;
  for (int64_t k = threadIdx.x; k < nblk; k += blockDim.x) t += part[k * nbw * nacc + o];
  sh[threadIdx.x] = t;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[o] = sh[0];
}

__global__ void finalize_kernel(const double* __restrict__ sums, int nbw, int nacc, int n_rhs_real,
                                int n_probes, int cplx, int64_t n, int use_exact,
                                double* __restrict__ rss, double* __restrict__ trace,
                                double* __restrict__ gcv) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbw) return;
  const double* sb = sums + int64_t(b) * nacc;
  double girard = 0.0, hutch = 0.0;
  for (int p = 0; p < n_probes; ++p) {
    const double wsw = sb[n_rhs_real + p], ww = sb[n_rhs_real + n_probes + p];
    girard += wsw / ww;
    hutch += wsw;
  }
  if (n_probes > 0) {
    girard = double(n) * girard / n_probes;
    hutch = hutch / n_probes;
  } else {
    girard = hutch = __longlong_as_double(0x7ff8000000000000LL);
  }
  const double exact = sb[nacc - 1];
  if (trace) {
    trace[b * 3 + 0] = girard;
    trace[b * 3 + 1] = hutch;
    trace[b * 3 + 2] = exact;
  }
  const int mult = cplx ? 2 : 1;
  const int n_rhs = n_rhs_real / mult;
  const double tr = use_exact ? exact : girard;
  for (int r = 0; r < n_rhs; ++r) {
    double v = 0.0;
    for (int pt = 0; pt < mult; ++pt) v += sb[r * mult + pt];
    if (rss) rss[b * n_rhs + r] = v;
    if (gcv) {
      const double den = 1.0 - tr / double(n);
      gcv[b * n_rhs + r] = (v / double(n)) / (den * den);
    }
  }
}

template <typename T>
inline int record_stride(int F2) {
  return t2_record_stride(F2);
}

template <int D, int NQ>
cudaError_t launch_lane(fkreg_plan_s* P, int b, int n_rhs_real, int n_probes, void* mhat_at_x,
                        cudaStream_t st, int nacc, int F2, float* vout, int rec, int pass_f,
                        int bstride, int cst, int wm0, int wm1, int pitch, int slack, int nw,
                        size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(interp_lane_kernel<D, 7, NQ>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  interp_lane_kernel<D, 7, NQ><<<unsigned(P->nblk_interp), nw * 32, smem, st>>>(
      P->geo, P->mono, wsp<BwDev>(P, P->r_bw), b, P->order, P->n, wsp<float>(P, P->r_xs),
      wsp<float>(P, P->r_str), perm_ptr(P), wsp<float>(P, P->r_t2field), rec, F2, pass_f,
      n_rhs_real, n_probes, P->o.y_complex, P->nrhs, static_cast<float*>(mhat_at_x), nacc, P->nbw,
      wsp<double>(P, P->r_part), wsp<uint32_t>(P, P->r_subbin), wsp<uint32_t>(P, P->r_subfirst),
      wsp<uint32_t>(P, P->r_binstart), wsp<uint32_t>(P, P->r_substart) + P->nbins_total, wm0, wm1,
      pitch, slack, bstride, cst, wsp<int>(P, P->r_err), vout);
  P->launches += 1;
  return cudaGetLastError();
}

template <typename T, int D, int W, int NCH>
cudaError_t launch_interp_w(fkreg_plan_s* P, int b, int n_rhs_real, int n_probes, void* mhat_at_x,
                            cudaStream_t st, int nacc, int F2, T* vout) {
  constexpr int pass_f = 32 * NCH;
  const int rec = record_stride<T>(F2);
  const unsigned blocks = unsigned(P->nblk_interp);
  if constexpr (sizeof(T) == 4 && W == 7 && D <= 2) {
    // lane-per-sample kernel: every field in one pass up to 64 fields, else
    // passes of 60 (any 60 consecutive fields span at most 16 quads)
    const BwDev& B = P->bw[b];
    const int wm0 = tma_window(P->geo, B, 0);
    const int wm1 = D > 1 ? tma_window(P->geo, B, 1) : 1;
    // window rows one quad apart in bank space (2-D)
    const int pitch = D > 1 ? wm1 * rec + 4 : wm0 * rec;
    const size_t win = (size_t(D > 1 ? wm0 : 1) * pitch * sizeof(T) + 127) / 128 * 128;
    const int slack = std::max(tma_slack(P->geo, B, 0), D > 1 ? tma_slack(P->geo, B, 1) : 0);
    const int pf = F2 <= 64 ? F2 : 60;
    const int bstride = pf | 1;
    const int cst = (n_rhs_real + n_probes) | 1;
    const size_t per_warp = sizeof(T) * 32 * (bstride + cst) + sizeof(double) * nacc;
    const size_t budget = 220 * 1024;
    const int nw = win < budget ? int(std::min<size_t>(kTWarps, (budget - win) / per_warp)) : 0;
    const size_t smem = win + per_warp * size_t(nw);
    const bool fits = wm0 <= B.nf[0] && (D == 1 || wm1 <= B.nf[1]) && nw >= 4;
    if (fits) {
      const int nqn = F2 <= 64 ? (F2 + 3) / 4 : 16;
      float* vo = reinterpret_cast<float*>(vout);
#define FK_L(Q) \
  return launch_lane<D, Q>(P, b, n_rhs_real, n_probes, mhat_at_x, st, nacc, F2, vo, rec, pf, bstride, cst, wm0, wm1, pitch, slack, nw, smem)
      if (nqn <= 1) FK_L(1);
      if (nqn <= 2) FK_L(2);
      if (nqn <= 3) FK_L(3);
      if (nqn <= 4) FK_L(4);
      if (nqn <= 6) FK_L(6);
      if (nqn <= 8) FK_L(8);
      if (nqn <= 10) FK_L(10);
      if (nqn <= 12) FK_L(12);
      FK_L(16);
#undef FK_L
    }
  }
  const size_t buf_warp = sizeof(T) * 32 * (pass_f + 1) + sizeof(double) * nacc;
  if constexpr (D <= 2 && W > 0) {
    const BwDev& B = P->bw[b];
    const int wm0 = tma_window(P->geo, B, 0);
    const int wm1 = D > 1 ? tma_window(P->geo, B, 1) : 1;
    const size_t win = (size_t(wm0) * wm1 * rec * sizeof(T) + 127) / 128 * 128;
    const int slack = std::max(tma_slack(P->geo, B, 0), D > 1 ? tma_slack(P->geo, B, 1) : 0);
    // staging stride: the record when every field fits one pass, odd for
    // conflict-free column reads
    const int span = F2 <= pass_f ? F2 : pass_f;
    const int bstride = span | 1;
    const size_t per_warp = sizeof(T) * 32 * bstride + sizeof(double) * nacc;
    const size_t budget = 220 * 1024;
    const int nw = win < budget ? int(std::min<size_t>(kTWarps, (budget - win) / per_warp)) : 0;
    const size_t smem = win + per_warp * size_t(nw);
    const bool fits = wm0 <= B.nf[0] && (D == 1 || wm1 <= B.nf[1]) && nw >= 4;
    if (fits) {
      cudaError_t e = cudaFuncSetAttribute(interp_tma_kernel<T, D, W, NCH>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      if (e != cudaSuccess) return e;
      interp_tma_kernel<T, D, W, NCH><<<blocks, nw * 32, smem, st>>>(
          P->geo, P->mono, wsp<BwDev>(P, P->r_bw), b, P->order, P->n, wsp<T>(P, P->r_xs),
          wsp<T>(P, P->r_str), perm_ptr(P), wsp<T>(P, P->r_t2field), rec, F2, pass_f, n_rhs_real,
          n_probes, P->o.y_complex, P->nrhs, static_cast<T*>(mhat_at_x), nacc, P->nbw,
          wsp<double>(P, P->r_part), wsp<uint32_t>(P, P->r_subbin), wsp<uint32_t>(P, P->r_subfirst),
          wsp<uint32_t>(P, P->r_binstart), wsp<uint32_t>(P, P->r_substart) + P->nbins_total, wm0,
          wm1, slack, bstride, wsp<int>(P, P->r_err), vout);
      P->launches += 1;
      return cudaGetLastError();
    }
  }
  int ncw = 1;
  for (int j = 0; j < D; ++j) ncw *= P->geo.w;
  if (W > 0) ncw = 0;
  // warps per block: as many as fit (up to kI2Warps) in the shared-memory budget
  const size_t per_warp = buf_warp + sizeof(T) * ncw;
  const int nwarps = int(std::min<size_t>(kI2Warps, (200 * 1024) / per_warp));
  if (nwarps < 1) return cudaErrorInvalidConfiguration;
  const size_t smem = per_warp * nwarps;
  cudaError_t e = cudaFuncSetAttribute(interp_kernel<T, D, W, NCH>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  interp_kernel<T, D, W, NCH><<<blocks, nwarps * 32, smem, st>>>(
      P->geo, P->mono, wsp<BwDev>(P, P->r_bw), b, P->order, P->n, wsp<T>(P, P->r_xs),
      wsp<T>(P, P->r_str), perm_ptr(P), wsp<T>(P, P->r_t2field), rec, F2, pass_f, n_rhs_real,
      n_probes, P->o.y_complex, P->nrhs, static_cast<T*>(mhat_at_x), nacc, P->nbw,
      wsp<double>(P, P->r_part), vout);
  P->launches += 1;
  return cudaGetLastError();
}

template <typename T, int D, int NCH>
cudaError_t launch_interp_d(fkreg_plan_s* P, int b, int n_rhs_real, int n_probes, void* mhat_at_x,
                            cudaStream_t st, int nacc, int F2, T* vout = nullptr) {
  const int w = P->geo.w;
#define FK_W(WW) \
  return launch_interp_w<T, D, WW, NCH>(P, b, n_rhs_real, n_probes, mhat_at_x, st, nacc, F2, vout)
  if (w == 7) FK_W(7);
  if constexpr (sizeof(T) == 8 && D < 3) {
    if (w == 10) FK_W(10);
    if (w == 13) FK_W(13);
  }
  FK_W(0);
#undef FK_W
}

template <typename T>
cudaError_t launch_interp(fkreg_plan_s* P, int b, int n_rhs_str, int n_probes, void* mhat_at_x,
                          cudaStream_t st) {
  const int n_rhs_real = n_rhs_str;
  const int nacc = n_rhs_real + 2 * n_probes + 1;
  if (nacc > kMaxAcc) return cudaErrorInvalidValue;
  const int F2 = P->ns + (n_rhs_real + n_probes) * P->nt;
  if (P->d * P->geo.w > 64 || P->geo.w > kMaxWRun) return cudaErrorInvalidValue;
  if (sizeof(T) == 4) {
    bool used = false;
    cudaError_t e =
        run_interp_direct(P, b, n_rhs_real, n_probes, mhat_at_x, st, nacc, F2, nullptr, &used);
    if (used || e != cudaSuccess) return e;
    e = run_interp_global_lane(P, b, n_rhs_real, n_probes, mhat_at_x, st, nacc, F2, nullptr, &used);
    if (used || e != cudaSuccess) return e;
  }
  // fields per pass: 64 (float) or 32 (double)
  const bool two = sizeof(T) == 4 && F2 > 32;
  if (two) {
    if (P->d == 1) return launch_interp_d<T, 1, 2>(P, b, n_rhs_real, n_probes, mhat_at_x, st, nacc, F2);
    if (P->d == 2) return launch_interp_d<T, 2, 2>(P, b, n_rhs_real, n_probes, mhat_at_x, st, nacc, F2);
    return launch_interp_d<T, 3, 2>(P, b, n_rhs_real, n_probes, mhat_at_x, st, nacc, F2);
  }
  if (P->d == 1) return launch_interp_d<T, 1, 1>(P, b, n_rhs_real, n_probes, mhat_at_x, st, nacc, F2);
  if (P->d == 2) return launch_interp_d<T, 2, 1>(P, b, n_rhs_real, n_probes, mhat_at_x, st, nacc, F2);
  return launch_interp_d<T, 3, 1>(P, b, n_rhs_real, n_probes, mhat_at_x, st, nacc, F2);
}

// Gather-only: F fields of bandwidth b's type-2 grid at every sorted sample
// into V[f][n], through the same kernels (and window staging) as above.
template <typename T>
cudaError_t launch_gather(fkreg_plan_s* P, int b, int F, T* V, cudaStream_t st) {
  if (P->n == 0) return cudaSuccess;
  if (P->d * P->geo.w > 64 || P->geo.w > kMaxWRun) return cudaErrorInvalidValue;
  if (sizeof(T) == 4) {
    bool used = false;
    cudaError_t e = run_interp_direct(P, b, 0, 0, nullptr, st, 0, F, V, &used);
    if (used || e != cudaSuccess) return e;
    e = run_interp_global_lane(P, b, 0, 0, nullptr, st, 0, F, V, &used);
    if (used || e != cudaSuccess) return e;
  }
  if (sizeof(T) == 4 && F > 32) {
    if (P->d == 1) return launch_interp_d<T, 1, 2>(P, b, 0, 0, nullptr, st, 0, F, V);
    if (P->d == 2) return launch_interp_d<T, 2, 2>(P, b, 0, 0, nullptr, st, 0, F, V);
    return launch_interp_d<T, 3, 2>(P, b, 0, 0, nullptr, st, 0, F, V);
  }
  if (P->d == 1) return launch_interp_d<T, 1, 1>(P, b, 0, 0, nullptr, st, 0, F, V);
  if (P->d == 2) return launch_interp_d<T, 2, 1>(P, b, 0, 0, nullptr, st, 0, F, V);
  return launch_interp_d<T, 3, 1>(P, b, 0, 0, nullptr, st, 0, F, V);
}

}  // namespace

cudaError_t run_gather_fields(fkreg_plan_s* P, int b, int F, void* V, cudaStream_t st) {
  return P->prec == FKREG_F32 ? launch_gather<float>(P, b, F, static_cast<float*>(V), st)
                              : launch_gather<double>(P, b, F, static_cast<double*>(V), st);
}

cudaError_t run_interp(fkreg_plan_s* P, int b, int n_rhs_str, int n_probes, const void*,
                       void* mhat_at_x, cudaStream_t st) {
  if (P->direct) return run_direct_interp(P, b, n_rhs_str, n_probes, mhat_at_x, st);
  return P->prec == FKREG_F32 ? launch_interp<float>(P, b, n_rhs_str, n_probes, mhat_at_x, st)
                              : launch_interp<double>(P, b, n_rhs_str, n_probes, mhat_at_x, st);
}

// Sum the partials of the last interpolation passes and derive DF and GCV.
cudaError_t run_finalize(fkreg_plan_s* P, int n_probes, const fkreg_outputs* out, cudaStream_t st) {
  const int nacc = P->nrhs_real + 2 * n_probes + 1;
  double* sums = wsp<double>(P, P->r_part) + P->nblk_interp * int64_t(P->nbw) * P->nacc;
  const int64_t nblk = P->nblk_interp;
  const int tot = P->nbw * nacc;
  reduce_partials<<<tot, 256, 0, st>>>(wsp<double>(P, P->r_part), nblk, P->nbw, nacc, sums);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  finalize_kernel<<<(P->nbw + 63) / 64, 64, 0, st>>>(
      sums, P->nbw, nacc, P->nrhs_real, n_probes, P->o.y_complex, P->n,
      (P->o.flags & FKREG_GCV_EXACT_TRACE) ? 1 : 0, out ? out->rss : nullptr,
      out ? out->trace : nullptr, out ? out->gcv : nullptr);
  P->launches += 2;
  return cudaGetLastError();
}

// Field record stride of the type-2 grids for F2 fields: a multiple of 4 so
// every cell record starts on a 16-byte boundary for the bulk copies, with an
// odd number of 16-byte quads so neighbouring cells start on different
// shared-memory banks.
int t2_record_stride(int F2) {
  const int r = (F2 + 3) / 4 * 4;
  return (r / 4) % 2 == 0 ? r + 4 : r;
}

}  // namespace fk
