// Direct-sum path for the compact regression kernels (Table 1: uniform,
// Epanechnikov, triangle, biweight, triweight).  Their Fourier transforms
// decay only algebraically, so the NUFFT's truncation cannot be controlled by
// a tolerance; instead the moment sums of eq. 9 are summed exactly over the
// samples inside each point's support (an ellipsoid |H^(-1/2) z| <= 1), found
// through the bins of the sort.  This file computes the grid fields; the
// grid solve (solve.cu) and the at-sample pass (interp.cu) follow as for the
// Gaussian path.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "interp_common.cuh"
#include "internal.h"

namespace fk {

namespace {

constexpr int kDirectMaxFields = 64;

// warp per (grid point m, bandwidth bw_first + bb), eight per block:
// fields [bb][fgrid][Mtot]
template <typename T, int D, int ORD, int FMAX>
__global__ void __launch_bounds__(256)
direct_grid_kernel(GeoDev g, const BwDev* __restrict__ bwt, int bw_first, int bw_count,
                   int64_t Mtot, int64_t n, const T* __restrict__ xs, const T* __restrict__ str,
                   int str_first, int nstr, const uint32_t* __restrict__ bin_start, int fgrid,
                   T* __restrict__ field) {
  constexpr int QB = direct_queue_bytes<T, D>();
  __shared__ __align__(16) unsigned char qsm[8 * QB];
  const int lane = threadIdx.x & 31;
  const int64_t gid = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (gid >= Mtot * bw_count) return;
  const int64_t m = gid % Mtot;
  const int bb = int(gid / Mtot);
  const BwDev& B = bwt[bw_first + bb];
  double q[3] = {0.0, 0.0, 0.0};
  int64_t rem = m;
  for (int a = D - 1; a >= 0; --a) {
    const int64_t idx = rem % g.M[a];
    rem /= g.M[a];
    q[a] = double(idx) * (g.hi[a] - g.lo[a]) / double(g.M[a] - 1);
  }
  T o0, o1;
  direct_warp_sums<T, D, ORD, FMAX>(g, B, n, xs, str, str_first, nstr, bin_start, q, lane,
                                    qsm + (threadIdx.x >> 5) * QB, o0, o1);
  T* fb = field + int64_t(bb) * fgrid * Mtot + m;
  if (lane < fgrid) fb[int64_t(lane) * Mtot] = o0;
  if (lane + 32 < fgrid) fb[int64_t(lane + 32) * Mtot] = o1;
}

template <typename T, int D, int ORD, int FMAX>
cudaError_t launch_direct_grid(fkreg_plan_s* P, int str_first, int nstr, int bw_first,
                               int bw_count, int64_t Mtot, int fgrid, cudaStream_t st) {
  constexpr int NS = mono_count(D, 2 * ORD), NT = mono_count(D, ORD);
  if constexpr (FMAX < kDirectMaxFields) {
    if (fgrid > FMAX)
      return launch_direct_grid<T, D, ORD, 2 * FMAX>(P, str_first, nstr, bw_first, bw_count,
                                                     Mtot, fgrid, st);
  }
  if constexpr ((FMAX - NS) / NT < 1) {
    return cudaErrorInvalidValue;
  } else {
    const unsigned blocks = unsigned((Mtot * bw_count + 7) / 8);
    direct_grid_kernel<T, D, ORD, FMAX><<<blocks, 256, 0, st>>>(
        P->geo, wsp<BwDev>(P, P->r_bw), bw_first, bw_count, Mtot, P->n, wsp<T>(P, P->r_xs),
        wsp<T>(P, P->r_str), str_first, nstr, wsp<uint32_t>(P, P->r_binstart), fgrid,
        wsp<T>(P, P->r_gfield));
    return cudaSuccess;
  }
}

template <typename T>
cudaError_t dispatch_direct_grid(fkreg_plan_s* P, int str_first, int nstr, int bw_first,
                                 int bw_count, int64_t Mtot, int fgrid, cudaStream_t st) {
#define FK_DG(DD, OO)                                                                         \
  if (P->d == DD && P->order == OO)                                                           \
    return launch_direct_grid<T, DD, OO, 16>(P, str_first, nstr, bw_first, bw_count, Mtot, \
                                             fgrid, st);
  FK_DG(1, 0) FK_DG(1, 1) FK_DG(1, 2) FK_DG(2, 0) FK_DG(2, 1) FK_DG(2, 2) FK_DG(3, 0) FK_DG(3, 1)
#undef FK_DG
  return cudaErrorInvalidValue;
}

// ---- at-sample pass of the direct path (compact kernels) --------------------
// Warp per 32 consecutive sorted samples: the warp sums the support of each
// of the 32 samples in turn (direct_warp_sums: lanes over the candidates),
// the reduced fields land in that sample's staging row, and phase B follows
// lane per sample as in the other kernels (one pass, F2 <= 64).
template <typename T, int D, int ORD, int FMAX>
__global__ void __launch_bounds__(256)
direct_interp_kernel(GeoDev g, MonoTab mono, const BwDev* __restrict__ bwt, int b, int order,
                     int64_t n, const T* __restrict__ xs, const T* __restrict__ str,
                     const uint32_t* __restrict__ perm, const uint32_t* __restrict__ bin_start,
                     int F2, int n_rhs_real, int n_probes, int cplx, int n_rhs_out,
                     T* __restrict__ mhat_at_x, int nacc, int nbw, double* __restrict__ part,
                     int bstride) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = int(blockDim.x >> 5);
  double* red_all = reinterpret_cast<double*>(smem_raw);
  double* red = red_all + warp * nacc;
  T* rows = reinterpret_cast<T*>(red_all + nwarps * nacc) + warp * 32 * bstride;
  T* my = rows + lane * bstride;
  unsigned char* qmem = smem_raw + sizeof(double) * nwarps * nacc +
                        sizeof(T) * nwarps * 32 * bstride + warp * direct_queue_bytes<T, D>();
  for (int a = lane; a < nacc; a += 32) red[a] = 0.0;
  __syncwarp();
  const BwDev& B = bwt[b];
  GroupCtx c{mono.n, mono.nt, mono.nt, n_rhs_real + n_probes, n_rhs_real, n_probes, cplx,
             n_rhs_out, nacc, order, b};
  T tsc[kMaxP];
#pragma unroll
  for (int k = 0; k < kMaxP; ++k) tsc[k] = (k < c.p) ? T(1.0 / tscale(mono, k, B.sigma)) : T(0);
  const T k0t = T(B.k0);
  const double isg[3] = {1.0 / B.sigma[0], 1.0 / B.sigma[1], 1.0 / B.sigma[2]};
  const int64_t ngroups = (n + 31) / 32;
  for (int64_t grp = int64_t(blockIdx.x) * nwarps + warp; grp < ngroups;
       grp += int64_t(gridDim.x) * nwarps) {
    const int64_t s = grp * 32 + lane;
    const bool valid = s < n;
    const int64_t sl = valid ? s : grp * 32;
    const int kmax = int(n - grp * 32 < 32 ? n - grp * 32 : 32);
    for (int k = 0; k < kmax; ++k) {
      const int64_t sk = grp * 32 + k;
      double q[3] = {0.0, 0.0, 0.0};
#pragma unroll
      for (int j = 0; j < D; ++j) q[j] = double(xs[int64_t(j) * n + sk]);
      T o0, o1;
      direct_warp_sums<T, D, ORD, FMAX>(g, B, n, xs, str, 1, c.nq, bin_start, q, lane, qmem, o0,
                                        o1);
      T* rk = rows + k * bstride;
      if (lane < F2) rk[lane] = o0;
      if (lane + 32 < F2) rk[lane + 32] = o1;
    }
    __syncwarp();
    T af[kMaxP] = {T(0), T(0), T(0), T(0)};
    finish_pass<T>(c, mono, B, my, 0, 0, c.nq, lane, valid, n, str + n + sl, n,
                   valid ? perm[s] : 0u, mhat_at_x, tsc, af, red, k0t, isg);
    __syncwarp();
  }
  __syncthreads();
  for (int a = threadIdx.x; a < nacc; a += blockDim.x) {
    double t = 0.0;
    for (int wv = 0; wv < nwarps; ++wv) t += red_get<T>(red_all, wv * nacc + a);
    part[(int64_t(blockIdx.x) * nbw + b) * nacc + a] = t;
  }
}

}  // namespace

cudaError_t run_direct_grid(fkreg_plan_s* P, int str_first, int nstr, int bw_first,
                            int bw_count, cudaStream_t st) {
  int64_t Mtot = 1;
  for (int a = 0; a < 3; ++a) Mtot *= P->geo.M[a];
  const int fgrid = P->ns + nstr * P->nt;
  if (fgrid > kDirectMaxFields) return cudaErrorInvalidValue;
  if (Mtot * bw_count == 0) return cudaSuccess;
  const cudaError_t e =
      P->prec == FKREG_F32
          ? dispatch_direct_grid<float>(P, str_first, nstr, bw_first, bw_count, Mtot, fgrid, st)
          : dispatch_direct_grid<double>(P, str_first, nstr, bw_first, bw_count, Mtot, fgrid,
                                         st);
  if (e != cudaSuccess) return e;
  P->launches += 1;
  return cudaGetLastError();
}

template <typename T, int D, int ORD, int FMAX>
cudaError_t launch_direct_interp(fkreg_plan_s* P, int b, int F2, int n_rhs_str, int n_probes,
                                 void* mhat_at_x, int nacc, int bstride, size_t smem,
                                 cudaStream_t st) {
  constexpr int NS = mono_count(D, 2 * ORD), NT = mono_count(D, ORD);
  if constexpr (FMAX < 64) {
    if (F2 > FMAX) return launch_direct_interp<T, D, ORD, 2 * FMAX>(
        P, b, F2, n_rhs_str, n_probes, mhat_at_x, nacc, bstride, smem, st);
  }
  if constexpr ((FMAX - NS) / NT < 1) {
    return cudaErrorInvalidValue;
  } else {
    const size_t sm = smem + 8 * direct_queue_bytes<T, D>();
    cudaError_t e = cudaFuncSetAttribute(direct_interp_kernel<T, D, ORD, FMAX>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
    if (e != cudaSuccess) return e;
    direct_interp_kernel<T, D, ORD, FMAX><<<unsigned(P->nblk_interp), 256, sm, st>>>(
        P->geo, P->mono, wsp<BwDev>(P, P->r_bw), b, P->order, P->n, wsp<T>(P, P->r_xs),
        wsp<T>(P, P->r_str), perm_ptr(P), wsp<uint32_t>(P, P->r_binstart), F2, n_rhs_str,
        n_probes, P->o.y_complex, P->nrhs, static_cast<T*>(mhat_at_x), nacc, P->nbw,
        wsp<double>(P, P->r_part), bstride);
    return cudaSuccess;
  }
}

template <typename T>
cudaError_t dispatch_direct_interp(fkreg_plan_s* P, int b, int F2, int n_rhs_str, int n_probes,
                                   void* mhat_at_x, int nacc, int bstride, size_t smem,
                                   cudaStream_t st) {
#define FK_DI(DD, OO)                                                                      \
  if (P->d == DD && P->order == OO)                                                        \
    return launch_direct_interp<T, DD, OO, 16>(P, b, F2, n_rhs_str, n_probes, mhat_at_x, \
                                               nacc, bstride, smem, st);
  FK_DI(1, 0) FK_DI(1, 1) FK_DI(1, 2) FK_DI(2, 0) FK_DI(2, 1) FK_DI(2, 2) FK_DI(3, 0) FK_DI(3, 1)
#undef FK_DI
  return cudaErrorInvalidValue;
}

cudaError_t run_direct_interp(fkreg_plan_s* P, int b, int n_rhs_str, int n_probes,
                              void* mhat_at_x, cudaStream_t st) {
  if (P->n == 0) return cudaSuccess;
  const int nacc = n_rhs_str + 2 * n_probes + 1;
  const int F2 = P->ns + (n_rhs_str + n_probes) * P->nt;
  if (F2 > 64 || nacc > kMaxAcc) return cudaErrorInvalidValue;
  const int bstride = F2 | 1;
  const size_t smem = sizeof(double) * 8 * nacc + P->tsize * 8 * 32 * bstride;
  const cudaError_t e =
      P->prec == FKREG_F32
          ? dispatch_direct_interp<float>(P, b, F2, n_rhs_str, n_probes, mhat_at_x, nacc,
                                          bstride, smem, st)
          : dispatch_direct_interp<double>(P, b, F2, n_rhs_str, n_probes, mhat_at_x, nacc,
                                           bstride, smem, st);
  if (e != cudaSuccess) return e;
  P->launches += 1;
  return cudaGetLastError();
}

}  // namespace fk
