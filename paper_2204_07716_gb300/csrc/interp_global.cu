// Type-2 interpolation with one lane per sample straight from the field
// grid (FP32, width 7): the form for windows that do not fit shared memory,
// chiefly 3-D (a 16^3-cell bin window of 34 fields is 2 MB).  See interp.cu
// for the method.  Each lane walks its own sample's w^d cells and loads four
// fields per 16-byte load from the (L2-resident where it fits) grid of cell
// records; sorted samples that share cells hit the same lines.  Phase B reads
// the fields from registers (system known at compile time: Nadaraya-Watson);
// the strengths of the group are copied ahead with cp.async.
#include <cuda_runtime.h>

#include <algorithm>

#include "device_common.cuh"
#include "interp_common.cuh"
#include "internal.h"

namespace fk {

namespace {

constexpr int kGWarps = 8;  // warps per block

template <int D, int W, int NQ, bool GONLY>
__global__ void __launch_bounds__(kGWarps * 32, 1)
interp_global_lane_kernel(GeoDev g, const BwDev* __restrict__ bwt, int b, int64_t n,
                          const float* __restrict__ xs, const float* __restrict__ str,
                          const uint32_t* __restrict__ perm, const float* __restrict__ fld,
                          int rec, int F2, int n_rhs_real, int n_probes, int cplx, int n_rhs_out,
                          float* __restrict__ mhat_at_x, int nacc, int nbw,
                          double* __restrict__ part, int cst, float* __restrict__ vout) {
  using T = float;
  constexpr int QMAX = GONLY ? 0 : 4 * NQ - 1;  // NW: one s-field, one t-field per response
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* red_all = reinterpret_cast<double*>(smem_raw);
  double* red = red_all + warp * nacc;
  T* cvs = reinterpret_cast<T*>(red_all + kGWarps * nacc) + (warp * 32 + lane) * cst;
  for (int a = lane; a < nacc; a += 32) red[a] = 0.0;
  __syncwarp();
  const BwDev& B = bwt[b];
  const int nf0 = int(B.nf[0]), nf1 = D > 1 ? int(B.nf[1]) : 1, nf2 = D > 2 ? int(B.nf[2]) : 1;
  const T ih[3] = {T(B.inv_h[0]), T(D > 1 ? B.inv_h[1] : 1.0), T(D > 2 ? B.inv_h[2] : 1.0)};
  const T beta = T(g.beta);
  const T halfw = T(0.5) * T(W);
  const int skind = g.skind;
  const int nq = n_rhs_real + n_probes;
  const T k0t = T(B.k0);
  const int nqd = (F2 + 3) >> 2;
  const int64_t ngroups = (n + 31) / 32;
  for (int64_t grp = int64_t(blockIdx.x) * kGWarps + warp; grp < ngroups;
       grp += int64_t(gridDim.x) * kGWarps) {
    const int64_t s0 = grp * 32;
    const int64_t s = s0 + lane;
    const bool valid = s < n;
    const int64_t sl = valid ? s : s0;
    uint32_t orig = 0u;
    if (!GONLY && valid) {
      orig = perm[s];
      for (int q = 0; q < nq; ++q) cp_async4(cvs + q, str + int64_t(1 + q) * n + s);
    }
    int i[3] = {0, 0, 0};
    T off[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const T u = __fmul_rn(xs[int64_t(j) * n + sl], ih[j]);
      const T fo = ceilf(__fsub_rn(u, halfw));
      i[j] = int(fo);
      off[j] = fo - u;
    }
    // wrapped cell indices and kernel values of the inner axes
    T pl[W], pm[W];
    int cl[W], cm[W];
#pragma unroll
    for (int t = 0; t < W; ++t) {
      pl[t] = phi<T>(skind, W, beta, off[D - 1] + T(t));
      cl[t] = int(wrap_idx(i[D - 1] + t, D == 1 ? nf0 : (D == 2 ? nf1 : nf2)));
      pm[t] = D == 3 ? phi<T>(skind, W, beta, off[1] + T(t)) : T(1);
      cm[t] = D == 3 ? int(wrap_idx(i[1] + t, nf1)) : 0;
    }
    float4 acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 1
    for (int t0 = 0; t0 < (D == 1 ? 1 : W); ++t0) {
      const T w0 = D == 1 ? T(1) : phi<T>(skind, W, beta, off[0] + T(t0));
      const int64_t r0 = D == 1 ? 0 : wrap_idx(i[0] + t0, nf0);
#pragma unroll 1
      for (int t1 = 0; t1 < (D == 3 ? W : 1); ++t1) {
        const T w01 = w0 * pm[t1];
        int64_t rb;
        if (D == 1) rb = 0;
        else if (D == 2) rb = r0 * nf1;
        else rb = (r0 * nf1 + cm[t1]) * int64_t(nf2);
#pragma unroll
        for (int t2 = 0; t2 < W; ++t2) {
          if (!in_range(g.errw, kSiteInterpField, rb + cl[t2], int64_t(nf0) * nf1 * nf2)) continue;
          const float* cell = fld + (rb + cl[t2]) * rec;
          const T wgt = w01 * pl[t2];
#pragma unroll
          for (int q = 0; q < NQ; ++q)
            if (q < nqd) {
              const float4 v = __ldg(reinterpret_cast<const float4*>(cell + 4 * q));
              quad_fma(acc[q], wgt, v);
            }
        }
      }
    }
    if (GONLY) {
      if (valid)
#pragma unroll
        for (int q = 0; q < NQ; ++q)
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) {
            const int f = 4 * q + cc;
            if (f < F2) vout[int64_t(f) * n + s] = quad_comp(acc[q], cc);
          }
      continue;
    }
    // phase B (Nadaraya-Watson): mhat = t / s
    cp_async_wait_all();
    const T s0v = acc[0].x;
    const bool okv = valid && s0v > T(0);
    const T a0 = okv ? T(1) / s0v : T(0);
    {
      const T tv = warp_sum_t<T>(okv ? k0t * a0 : T(0));
      if (lane == 0) red_add<T>(red, nacc - 1, tv);
    }
#pragma unroll
    for (int q = 0; q < QMAX; ++q) {
      if (q >= nq) break;
      const int f = 1 + q;
      const T mh = a0 * quad_comp(acc[f >> 2], f & 3);
      const T cv = valid ? cvs[q] : T(0);
      if (q < n_rhs_real) {
        const T r = valid ? cv - mh : T(0);
        const T v = warp_sum_t<T>(r * r);
        if (lane == 0) red_add<T>(red, q, v);
        if (valid && mhat_at_x) {
          const int mult = cplx ? 2 : 1;
          const int rr = q / mult, pt = q % mult;
          mhat_at_x[((int64_t(b) * n_rhs_out + rr) * n + orig) * mult + pt] = mh;
        }
      } else {
        const int pp = q - n_rhs_real;
        const T v1 = warp_sum_t<T>(valid ? cv * mh : T(0));
        const T v2 = warp_sum_t<T>(valid ? cv * cv : T(0));
        if (lane == 0) {
          red_add<T>(red, n_rhs_real + pp, v1);
          red_add<T>(red, n_rhs_real + n_probes + pp, v2);
        }
      }
    }
    __syncwarp();  // the cp.async rows are rewritten by the next group
  }
  __syncthreads();
  for (int a = threadIdx.x; a < nacc; a += blockDim.x) {
    double t = 0.0;
    for (int wv = 0; wv < kGWarps; ++wv) t += red_get<T>(red_all, wv * nacc + a);
    part[(int64_t(blockIdx.x) * nbw + b) * nacc + a] = t;
  }
}

template <int D, int NQ, bool GONLY>
cudaError_t launch_global_k(fkreg_plan_s* P, int b, int n_rhs_real, int n_probes,
                            void* mhat_at_x, cudaStream_t st, int nacc, int F2, float* vout,
                            int rec, int cst, size_t smem) {
  auto kern = interp_global_lane_kernel<D, 7, NQ, GONLY>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  kern<<<unsigned(P->nblk_interp), kGWarps * 32, smem, st>>>(
      P->geo, wsp<BwDev>(P, P->r_bw), b, P->n, wsp<float>(P, P->r_xs), wsp<float>(P, P->r_str),
      perm_ptr(P), wsp<float>(P, P->r_t2field), rec, F2, n_rhs_real, n_probes, P->o.y_complex,
      P->nrhs, static_cast<float*>(mhat_at_x), nacc, P->nbw, wsp<double>(P, P->r_part), cst,
      vout);
  P->launches += 1;
  return cudaGetLastError();
}

template <int D, bool GONLY>
cudaError_t launch_global_q(fkreg_plan_s* P, int b, int n_rhs_real, int n_probes,
                            void* mhat_at_x, cudaStream_t st, int nacc, int F2, float* vout,
                            int rec, int cst, size_t smem) {
  const int nqn = (F2 + 3) / 4;
#define FK_Q(Q)                                                                               \
  return launch_global_k<D, Q, GONLY>(P, b, n_rhs_real, n_probes, mhat_at_x, st, nacc, F2, \
                                      vout, rec, cst, smem)
  if (nqn <= 4) FK_Q(4);
  if (nqn <= 8) FK_Q(8);
  if (nqn <= 10) FK_Q(10);
  if (nqn <= 12) FK_Q(12);
  FK_Q(16);
#undef FK_Q
}

}  // namespace

// Launch the lane-per-sample global kernel if it applies (FP32, width 7,
// 3-D Nadaraya-Watson or 3-D gather-only, F2 <= 64); *launched says
// whether it ran.
cudaError_t run_interp_global_lane(fkreg_plan_s* P, int b, int n_rhs_real, int n_probes,
                                   void* mhat_at_x, cudaStream_t st, int nacc, int F2,
                                   void* vout, bool* launched) {
  *launched = false;
  if (P->prec != FKREG_F32 || P->geo.w != 7 || P->d != 3 || F2 > 64 || P->n == 0)
    return cudaSuccess;
  if (!vout && P->order != 0) return cudaSuccess;
  const int rec = t2_record_stride(F2);
  const int cst = vout ? 1 : ((n_rhs_real + n_probes) | 1);
  const size_t smem = sizeof(double) * size_t(kGWarps) * nacc +
                      sizeof(float) * size_t(kGWarps) * 32 * cst;
  float* vo = static_cast<float*>(vout);
  *launched = true;
  if (vout) return launch_global_q<3, true>(P, b, 0, 0, nullptr, st, 0, F2, vo, rec, cst, smem);
  return launch_global_q<3, false>(P, b, n_rhs_real, n_probes, mhat_at_x, st, nacc, F2, nullptr,
                                   rec, cst, smem);
}

}  // namespace fk
