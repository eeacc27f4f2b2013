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
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "internal.h"

namespace fk {

namespace {

constexpr int kI2Warps = 4;
constexpr int kMaxAcc = 512;
constexpr int kMaxCh = 4;     // 32-field chunks per pass (pass_f <= 128)
constexpr int kMaxWRun = 32;  // runtime-width fallback

// Fields are stored interleaved per fine-grid cell ([cell][F2]), so a warp
// gathers one sample at a time with its lanes spread over the fields: every
// load of the 32 lanes is one contiguous run.  A warp walks a group of 32
// consecutive sorted samples (one bin, nearby cells, cache-resident), parks
// each sample's field values in shared memory, and then each lane takes one
// sample for the FP64 solve and the reductions.  Fields go in passes of
// pass_f so the staging buffer stays small; pass 0 holds the s-fields.
// W > 0 fixes the spreading width at compile time (unrolled window, weights
// in registers); W == 0 is the runtime-width fallback.
template <typename T, int D, int W>
__global__ void __launch_bounds__(kI2Warps * 32)
interp_kernel(GeoDev g, MonoTab mono, const BwDev* __restrict__ bwt, int b, int order, int64_t n,
              const T* __restrict__ xs, const T* __restrict__ str, const uint32_t* __restrict__ perm,
              const T* __restrict__ fld, int F2, int pass_f, int n_rhs_real, int n_probes, int cplx,
              int n_rhs_out, T* __restrict__ mhat_at_x, int nacc, int nbw, double* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int w = W > 0 ? W : g.w;
  int ncw = 1;
  for (int j = 0; j < D; ++j) ncw *= w;
  if (W > 0) ncw = 0;
  const int bstride = pass_f + 1;
  double* red_all = reinterpret_cast<double*>(smem_raw);
  double* red = red_all + warp * nacc;
  T* cellw = reinterpret_cast<T*>(red_all + kI2Warps * nacc) + warp * ncw;
  T* buf = reinterpret_cast<T*>(red_all + kI2Warps * nacc) + kI2Warps * ncw + warp * 32 * bstride;
  for (int a = lane; a < nacc; a += 32) red[a] = 0.0;
  __syncwarp();
  const BwDev& B = bwt[b];
  const int nf0 = int(B.nf[0]), nf1 = D > 1 ? int(B.nf[1]) : 1, nf2 = D > 2 ? int(B.nf[2]) : 1;
  const T ih0 = T(B.inv_h[0]), ih1 = T(D > 1 ? B.inv_h[1] : 1.0), ih2 = T(D > 2 ? B.inv_h[2] : 1.0);
  const T beta = T(g.beta);
  const T halfw = T(0.5) * T(w);
  const int ns = mono.n, nt = mono.nt, p = nt;
  const int nq = n_rhs_real + n_probes;
  T tsc[kMaxP];
  for (int k = 0; k < kMaxP; ++k) tsc[k] = (k < p) ? T(1.0 / tscale(mono, k, B.sigma)) : T(0);
  const int64_t ngroups = (n + 31) / 32;
  const int64_t gstride = int64_t(gridDim.x) * kI2Warps;
  for (int64_t grp = int64_t(blockIdx.x) * kI2Warps + warp; grp < ngroups; grp += gstride) {
    const int64_t s0 = grp * 32;
    const int cnt = int(min(int64_t(32), n - s0));
    const int64_t s = s0 + lane;
    const bool valid = lane < cnt;
    T af[kMaxP] = {T(0), T(0), T(0), T(0)};
    int q_done = 0, f_first = 0;
    for (int pass = 0; f_first < F2; ++pass) {
      const int q_in = pass == 0 ? min(nq, (pass_f - ns) / nt) : min(nq - q_done, pass_f / nt);
      const int f_last = (pass == 0 ? ns : f_first) + q_in * nt;
      const int fcount = f_last - f_first;
      const int nch = (fcount + 31) / 32;
      // ---- phase A: warp-cooperative gather, one sample at a time ----
      T xn0 = xs[s0], xn1 = D > 1 ? xs[n + s0] : T(0), xn2 = D > 2 ? xs[2 * n + s0] : T(0);
      for (int j = 0; j < cnt; ++j) {
        const T x0 = xn0, x1 = xn1, x2 = xn2;
        if (j + 1 < cnt) {  // prefetch the next sample's coordinates
          xn0 = xs[s0 + j + 1];
          if (D > 1) xn1 = xs[n + s0 + j + 1];
          if (D > 2) xn2 = xs[2 * n + s0 + j + 1];
        }
        int i0, i1 = 0, i2 = 0;
        T off0, off1 = T(0), off2 = T(0);
        {
          const T u = x0 * ih0;
          const T f = ceil(u - halfw);
          i0 = int(f);
          off0 = f - u;
        }
        if (D > 1) {
          const T u = x1 * ih1;
          const T f = ceil(u - halfw);
          i1 = int(f);
          off1 = f - u;
        }
        if (D > 2) {
          const T u = x2 * ih2;
          const T f = ceil(u - halfw);
          i2 = int(f);
          off2 = f - u;
        }
        // 1-D kernel values: lane l holds axis l / w, tap l % w (two rounds)
        T wl0, wl1;
        {
          const int ax = lane / w, t = lane % w;
          wl0 = ax < D ? phi<T>(g.skind, w, beta, sel3<T>(ax, off0, off1, off2) + T(t)) : T(0);
          const int l2 = lane + 32, ax2 = l2 / w, t2 = l2 % w;
          wl1 = ax2 < D ? phi<T>(g.skind, w, beta, sel3<T>(ax2, off0, off1, off2) + T(t2)) : T(0);
        }
        T acc[kMaxCh];
#pragma unroll
        for (int ch = 0; ch < kMaxCh; ++ch) acc[ch] = T(0);
        const T* fb = fld + f_first + lane;
        if constexpr (W > 0) {
          T wa[D][W > 0 ? W : 1];
#pragma unroll
          for (int d = 0; d < D; ++d)
#pragma unroll
            for (int t = 0; t < W; ++t) {
              const int l = d * W + t;
              wa[d][t] = l < 32 ? __shfl_sync(0xffffffffu, wl0, l) : __shfl_sync(0xffffffffu, wl1, l - 32);
            }
          int cl[W > 0 ? W : 1];
#pragma unroll
          for (int t = 0; t < W; ++t) cl[t] = int(wrap_idx(D == 1 ? i0 + t : (D == 2 ? i1 + t : i2 + t),
                                                          D == 1 ? nf0 : (D == 2 ? nf1 : nf2)));
          if (D == 1) {
#pragma unroll
            for (int t0 = 0; t0 < W; ++t0) {
              const T* q = fb + int64_t(cl[t0]) * F2;
              const T v = wa[0][t0];
#pragma unroll
              for (int ch = 0; ch < kMaxCh; ++ch)
                if (ch < nch && lane + ch * 32 < fcount) acc[ch] += __ldg(q + ch * 32) * v;
            }
          } else if (D == 2) {
#pragma unroll
            for (int t0 = 0; t0 < W; ++t0) {
              const int row = int(wrap_idx(i0 + t0, nf0)) * nf1;
              const T w0 = wa[0][t0];
#pragma unroll
              for (int t1 = 0; t1 < W; ++t1) {
                const T* q = fb + int64_t(row + cl[t1]) * F2;
                const T v = w0 * wa[D - 1][t1];
#pragma unroll
                for (int ch = 0; ch < kMaxCh; ++ch)
                  if (ch < nch && lane + ch * 32 < fcount) acc[ch] += __ldg(q + ch * 32) * v;
              }
            }
          } else {
#pragma unroll 1
            for (int t0 = 0; t0 < W; ++t0) {
              const int r0 = int(wrap_idx(i0 + t0, nf0)) * nf1;
#pragma unroll
              for (int t1 = 0; t1 < W; ++t1) {
                const int r1 = (r0 + int(wrap_idx(i1 + t1, nf1))) * nf2;
                const T w01 = wa[0][t0] * wa[1 % D][t1];
#pragma unroll
                for (int t2 = 0; t2 < W; ++t2) {
                  const T* q = fb + int64_t(r1 + cl[t2]) * F2;
                  const T v = w01 * wa[D - 1][t2];
#pragma unroll
                  for (int ch = 0; ch < kMaxCh; ++ch)
                    if (ch < nch && lane + ch * 32 < fcount) acc[ch] += __ldg(q + ch * 32) * v;
                }
              }
            }
          }
        } else {
          // runtime width: tensor-product cell weights through shared memory
          for (int c0 = 0; c0 < ncw; c0 += 32) {
            const int c = c0 + lane;
            int rem = c < ncw ? c : 0;
            T v = T(1);
            for (int d = D - 1; d >= 0; --d) {
              const int t = rem % w;
              rem /= w;
              const int l = d * w + t;
              const T a0 = __shfl_sync(0xffffffffu, wl0, l & 31);
              const T a1 = __shfl_sync(0xffffffffu, wl1, l & 31);
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
              const int id = d == 0 ? i0 : (d == 1 ? i1 : i2);
              const int nfd = d == 0 ? nf0 : (d == 1 ? nf1 : nf2);
              cell += wrap_idx(id + t, nfd) * mult;
              mult *= nfd;
            }
            const T* q = fb + cell * F2;
            const T v = cellw[c];
#pragma unroll
            for (int ch = 0; ch < kMaxCh; ++ch)
              if (ch < nch && lane + ch * 32 < fcount) acc[ch] += q[ch * 32] * v;
          }
        }
#pragma unroll
        for (int ch = 0; ch < kMaxCh; ++ch)
          if (ch < nch && lane + ch * 32 < fcount) buf[j * bstride + lane + ch * 32] = acc[ch];
        __syncwarp();
      }
      // ---- phase B: one lane per sample ----
      const T* my = buf + lane * bstride;
      if (pass == 0) {
        double a[kMaxP] = {0, 0, 0, 0};
        bool ok = false;
        if (valid) {
          double sv[kMaxMono];
          for (int k = 0; k < ns; ++k) sv[k] = double(my[k]);
          if (order == 0) {
            ok = sv[0] > 0.0;
            a[0] = ok ? 1.0 / sv[0] : 0.0;
          } else {
            ok = lpr_weights_fast(mono, p, sv, B.sigma, a);
          }
        }
        for (int k = 0; k < p; ++k) af[k] = ok ? T(a[k]) * tsc[k] : T(0);
        const double tv = warp_sum_t<double>((valid && ok) ? B.k0 * a[0] : 0.0);
        if (lane == 0) red[nacc - 1] += tv;
      }
      const int fq0 = pass == 0 ? ns : 0;
      const uint32_t orig = valid ? perm[s] : 0u;
      for (int qq = 0; qq < q_in; ++qq) {
        const int q = q_done + qq;
        T mh = T(0);
        for (int k = 0; k < p; ++k) mh += af[k] * my[fq0 + qq * nt + k];
        const T c = valid ? str[int64_t(1 + q) * n + s] : T(0);
        if (q < n_rhs_real) {
          const T r = valid ? c - mh : T(0);
          const T v = warp_sum_t<T>(r * r);
          if (lane == 0) red[q] += double(v);
          if (valid && mhat_at_x) {
            const int mult = cplx ? 2 : 1;
            const int rr = q / mult, pt = q % mult;
            mhat_at_x[((int64_t(b) * n_rhs_out + rr) * n + orig) * mult + pt] = mh;
          }
        } else {
          const int pp = q - n_rhs_real;
          const T v1 = warp_sum_t<T>(valid ? c * mh : T(0));
          const T v2 = warp_sum_t<T>(valid ? c * c : T(0));
          if (lane == 0) {
            red[n_rhs_real + pp] += double(v1);
            red[n_rhs_real + n_probes + pp] += double(v2);
          }
        }
      }
      __syncwarp();
      q_done += q_in;
      f_first = f_last;
    }
  }
  __syncthreads();
  for (int a = threadIdx.x; a < nacc; a += blockDim.x) {
    double t = 0.0;
    for (int wv = 0; wv < kI2Warps; ++wv) t += red_all[wv * nacc + a];
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

template <typename T, int D, int W>
cudaError_t launch_interp_w(fkreg_plan_s* P, int b, int n_rhs_real, int n_probes, void* mhat_at_x,
                            cudaStream_t st, unsigned blocks, int nacc, int F2, int pass_f) {
  int ncw = 1;
  for (int j = 0; j < D; ++j) ncw *= P->geo.w;
  if (W > 0) ncw = 0;
  const size_t smem = sizeof(double) * kI2Warps * nacc + sizeof(T) * kI2Warps * ncw +
                      sizeof(T) * kI2Warps * 32 * (pass_f + 1);
  if (smem > 220 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(interp_kernel<T, D, W>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  interp_kernel<T, D, W><<<blocks, kI2Warps * 32, smem, st>>>(
      P->geo, P->mono, wsp<BwDev>(P, P->r_bw), b, P->order, P->n, wsp<T>(P, P->r_xs),
      wsp<T>(P, P->r_str), perm_ptr(P), wsp<T>(P, P->r_t2field), F2, pass_f, n_rhs_real, n_probes,
      P->o.y_complex, P->nrhs, static_cast<T*>(mhat_at_x), nacc, P->nbw, wsp<double>(P, P->r_part));
  P->launches += 1;
  return cudaGetLastError();
}

template <typename T, int D>
cudaError_t launch_interp_d(fkreg_plan_s* P, int b, int n_rhs_real, int n_probes, void* mhat_at_x,
                            cudaStream_t st, unsigned blocks, int nacc, int F2, int pass_f) {
  const int w = P->geo.w;
#define FK_W(WW) \
  return launch_interp_w<T, D, WW>(P, b, n_rhs_real, n_probes, mhat_at_x, st, blocks, nacc, F2, pass_f)
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
  const int64_t groups = (P->n + 31) / 32;
  const unsigned blocks =
      unsigned(std::min<int64_t>((groups + kI2Warps - 1) / kI2Warps, P->nblk_interp));
  const int nacc = n_rhs_real + 2 * n_probes + 1;
  if (nacc > kMaxAcc) return cudaErrorInvalidValue;
  if (blocks == 0) return cudaSuccess;
  const int F2 = P->ns + (n_rhs_real + n_probes) * P->nt;
  int pass_f = (int(sizeof(T)) == 4) ? 128 : 64;
  pass_f = std::min(pass_f, ((F2 + 31) / 32) * 32);
  pass_f = std::max(pass_f, P->ns + P->nt);
  if (P->d * P->geo.w > 64 || P->geo.w > kMaxWRun) return cudaErrorInvalidValue;
  switch (P->d) {
    case 1: return launch_interp_d<T, 1>(P, b, n_rhs_real, n_probes, mhat_at_x, st, blocks, nacc, F2, pass_f);
    case 2: return launch_interp_d<T, 2>(P, b, n_rhs_real, n_probes, mhat_at_x, st, blocks, nacc, F2, pass_f);
    default: return launch_interp_d<T, 3>(P, b, n_rhs_real, n_probes, mhat_at_x, st, blocks, nacc, F2, pass_f);
  }
}

}  // namespace

cudaError_t run_interp(fkreg_plan_s* P, int b, int n_rhs_str, int n_probes, const void*,
                       void* mhat_at_x, cudaStream_t st) {
  return P->prec == FKREG_F32 ? launch_interp<float>(P, b, n_rhs_str, n_probes, mhat_at_x, st)
                              : launch_interp<double>(P, b, n_rhs_str, n_probes, mhat_at_x, st);
}

// Sum the partials of the last interpolation passes and derive DF and GCV.
cudaError_t run_finalize(fkreg_plan_s* P, int n_probes, const fkreg_outputs* out, cudaStream_t st) {
  const int nacc = P->nrhs_real + 2 * n_probes + 1;
  double* sums = wsp<double>(P, P->r_part) + P->nblk_interp * int64_t(P->nbw) * P->nacc;
  const int64_t groups = (P->n + 31) / 32;
  const int64_t nblk = std::min<int64_t>((groups + kI2Warps - 1) / kI2Warps, P->nblk_interp);
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

}  // namespace fk
