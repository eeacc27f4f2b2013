// Direct-sum path for the compact regression kernels (Table 1: uniform,
// Epanechnikov, triangle, biweight, triweight).  Their Fourier transforms
// decay only algebraically, so the NUFFT's truncation cannot be controlled by
// a tolerance; instead the moment sums of eq. 9 are summed exactly over the
// samples inside each point's support (an ellipsoid |H^(-1/2) z| <= 1), found
// through the bins of the sort.  This file holds both passes: the grid
// fields (warp per grid point) and the at-sample pass with its phase B (lane
// per sample); the grid solve (solve.cu) and the reductions follow as for
// the Gaussian path.
#include <cuda_runtime.h>

#include <algorithm>

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
      return launch_direct_grid<T, D, ORD, FMAX == 16 ? 40 : 64>(P, str_first, nstr, bw_first, bw_count,
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
// Record stride (in T) of one staged candidate: coordinates at [0, D),
// strengths at [4, 4 + nstr), in an odd number of 4-element chunks so that
// the 32 lanes' scalar stores into their records spread over 8 banks.
template <typename T, int D, int ORD, int FMAX>
__host__ __device__ constexpr int direct_rec_stride() {
  return 4 * ((1 + ((FMAX - mono_count(D, 2 * ORD)) / mono_count(D, ORD) + 3) / 4) | 1);
}

// Lane per sorted sample.  The 32 consecutive samples of a warp lie in one
// or two bins, so their supports nearly coincide: the warp walks the bins
// covering the union of the supports, stages 32 candidates at a time
// (coordinates and strengths, coalesced loads) in shared memory, and every
// lane tests each staged candidate against its own sample's support and adds
// it to its fields in registers.  The candidates are read from global memory
// once per warp, not once per sample.  Phase B follows as in the other
// at-sample kernels (one pass, F2 <= 64).
template <typename T, int D, int ORD, int FMAX>
__global__ void __launch_bounds__(256)
direct_interp_kernel(GeoDev g, MonoTab mono, const BwDev* __restrict__ bwt, int b, int order,
                     int64_t n, const T* __restrict__ xs, const T* __restrict__ str,
                     const uint32_t* __restrict__ perm, const uint32_t* __restrict__ bin_start,
                     int F2, int n_rhs_real, int n_probes, int cplx, int n_rhs_out,
                     T* __restrict__ mhat_at_x, int nacc, int nbw, double* __restrict__ part,
                     int bstride, int64_t nblk_rows) {
  constexpr int NS = mono_count(D, 2 * ORD), NT = mono_count(D, ORD);
  constexpr int QMAX = (FMAX - NS) / NT;
  constexpr int QC = (QMAX + 3) / 4;     // strength chunks of four
  constexpr int ACC = NS + 4 * QC * NT;  // fields incl. the last chunk's padding
  constexpr int RS = direct_rec_stride<T, D, ORD, FMAX>();
  static_assert(RS >= 4 + 4 * QC && RS % 4 == 0, "record layout");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = int(blockDim.x >> 5);
  double* red_all = reinterpret_cast<double*>(smem_raw);
  double* red = red_all + warp * nacc;
  // candidate records first (16-byte aligned), then the staging rows
  T* recs = reinterpret_cast<T*>(red_all + ((nwarps * nacc + 1) & ~1)) + warp * 32 * RS;
  T* my = reinterpret_cast<T*>(red_all + ((nwarps * nacc + 1) & ~1)) + nwarps * 32 * RS +
          (warp * 32 + lane) * bstride;
  for (int a = lane; a < nacc; a += 32) red[a] = 0.0;
  const BwDev& B = bwt[b];
  GroupCtx c{mono.n, mono.nt, mono.nt, n_rhs_real + n_probes, n_rhs_real, n_probes, cplx,
             n_rhs_out, nacc, order, b};
  const int nstr = c.nq;
  for (int a = 4 + nstr; a < RS; ++a) recs[lane * RS + a] = T(0);
  __syncwarp();
  T tsc[kMaxP];
#pragma unroll
  for (int k = 0; k < kMaxP; ++k) tsc[k] = (k < c.p) ? T(1.0 / tscale(mono, k, B.sigma)) : T(0);
  const T k0t = T(B.k0);
  const double isg[3] = {1.0 / B.sigma[0], 1.0 / B.sigma[1], 1.0 / B.sigma[2]};
  T hi[D][D];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int e = 0; e < D; ++e) hi[a][e] = T(B.Hinv[a * 3 + e]);
  const T ks = T(B.kscale), kr2 = T(B.kr2);
  const int kern = g.kern;
  const int64_t ngroups = (n + 31) / 32;
  for (int64_t grp = int64_t(blockIdx.x) * nwarps + warp; grp < ngroups;
       grp += int64_t(gridDim.x) * nwarps) {
    const int64_t s = grp * 32 + lane;
    const bool valid = s < n;
    const int64_t sl = valid ? s : grp * 32;
    T qv[D];
#pragma unroll
    for (int j = 0; j < D; ++j) qv[j] = xs[int64_t(j) * n + sl];
    // bins covering the union of the warp's supports
    DirectRows<D> rows;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      T mn = qv[j], mx = qv[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      }
      rows.mn[j] = float(mn);
      rows.mx[j] = float(mx);
    }
    rows.box(g, B);
    T acc[ACC];                    // FP64 plans: every field
    float2 accs[(NS + 1) / 2];     // FP32 plans: s-fields in pairs
    float2 acct[2 * QC][NT];       // FP32 plans: t-fields of strengths (2h, 2h + 1)
#pragma unroll
    for (int f = 0; f < ACC; ++f) acc[f] = T(0);
#pragma unroll
    for (int f = 0; f < (NS + 1) / 2; ++f) accs[f] = make_float2(0.f, 0.f);
#pragma unroll
    for (int h = 0; h < 2 * QC; ++h)
#pragma unroll
      for (int k = 0; k < NT; ++k) acct[h][k] = make_float2(0.f, 0.f);
    const int o0 = rows.rows0(), o1 = rows.rows1();
    for (int r0 = 0; r0 < o0; ++r0)
      for (int r1 = 0; r1 < o1; ++r1) {
        int64_t first, last;  // bins [first, last] are adjacent in sorted order
        if (!rows.row(g, r0, r1, first, last)) continue;
        if (!in_range(g.errw, kSiteDirectBins, first, last + 1) ||
            !in_range(g.errw, kSiteDirectBins, last, g.nbins[0] * g.nbins[1] * g.nbins[2]))
          continue;
        const uint32_t i1 = bin_start[last + 1];
        for (uint32_t base = bin_start[first]; base < i1; base += 32) {
          const uint32_t i = base + uint32_t(lane);
          __syncwarp();  // the previous batch's records are no longer read
          if (i < i1) {
            T* rw = recs + lane * RS;
#pragma unroll
            for (int j = 0; j < D; ++j) rw[j] = xs[int64_t(j) * n + i];
#pragma unroll
            for (int r = 0; r < QMAX; ++r)
              if (r < nstr) rw[4 + r] = str[int64_t(1 + r) * n + i];
          }
          __syncwarp();
          const int cnt = int(i1 - base < 32u ? i1 - base : 32u);
          for (int cc = 0; cc < cnt; ++cc) {
            const T* rc = recs + cc * RS;
            T z[D];
#pragma unroll
            for (int j = 0; j < D; ++j) z[j] = rc[j] - qv[j];
            T u2 = T(0);
#pragma unroll
            for (int a = 0; a < D; ++a) {
              T ra = T(0);
#pragma unroll
              for (int e = 0; e < D; ++e) ra += hi[a][e] * z[e];
              u2 += z[a] * ra;
            }
            if (u2 <= T(1)) {
              const T wgt = ks * compact_k<T>(kern, u2, kr2);
              T mo[NS];
              mono_build<T, D, 2 * ORD>(mo, z);
              if constexpr (sizeof(T) == 4) {
                // packed FP32: two fields per instruction, each rounded as a
                // scalar fma
                const float2 w2 = make_float2(wgt, wgt);
#pragma unroll
                for (int f = 0; f < (NS + 1) / 2; ++f)
                  accs[f] = __ffma2_rn(w2, make_float2(mo[2 * f], 2 * f + 1 < NS ? mo[2 * f + 1] : 0.f),
                                       accs[f]);
#pragma unroll
                for (int v = 0; v < QC; ++v)
                  if (4 * v < nstr) {  // four strengths at a time (zero past nstr)
                    const float4 t4 = reinterpret_cast<const float4*>(rc + 4)[v];
                    const float2 c01 = __fmul2_rn(w2, make_float2(t4.x, t4.y));
                    const float2 c23 = __fmul2_rn(w2, make_float2(t4.z, t4.w));
#pragma unroll
                    for (int k = 0; k < NT; ++k) {
                      const float2 m2 = make_float2(mo[k], mo[k]);
                      acct[2 * v][k] = __ffma2_rn(c01, m2, acct[2 * v][k]);
                      acct[2 * v + 1][k] = __ffma2_rn(c23, m2, acct[2 * v + 1][k]);
                    }
                  }
              } else {
#pragma unroll
                for (int f = 0; f < NS; ++f) acc[f] += wgt * mo[f];
#pragma unroll
                for (int v = 0; v < QC; ++v)
                  if (4 * v < nstr) {  // four strengths at a time (zero past nstr)
                    const double2 ta = reinterpret_cast<const double2*>(rc + 4)[2 * v];
                    const double2 tb = reinterpret_cast<const double2*>(rc + 4)[2 * v + 1];
                    const T sv[4] = {T(ta.x), T(ta.y), T(tb.x), T(tb.y)};
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                      const T cw = wgt * sv[u];
#pragma unroll
                      for (int k = 0; k < NT; ++k) acc[NS + (4 * v + u) * NT + k] += cw * mo[k];
                    }
                  }
              }
            }
          }
        }
      }
    if constexpr (sizeof(T) == 4) {
#pragma unroll
      for (int f = 0; f < NS; ++f) my[f] = (f & 1) ? accs[f >> 1].y : accs[f >> 1].x;
#pragma unroll
      for (int r = 0; r < 4 * QC; ++r)
        if (r < nstr)
#pragma unroll
          for (int k = 0; k < NT; ++k)
            my[NS + r * NT + k] = (r & 1) ? acct[r >> 1][k].y : acct[r >> 1][k].x;
    } else {
#pragma unroll
      for (int f = 0; f < ACC; ++f)
        if (f < F2) my[f] = acc[f];
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
    // partial rows of the block indices this one-wave grid does not launch
    for (int64_t r = int64_t(blockIdx.x) + gridDim.x; r < nblk_rows; r += gridDim.x)
      part[(r * nbw + b) * nacc + a] = 0.0;
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
    if (F2 > FMAX) return launch_direct_interp<T, D, ORD, FMAX == 16 ? 40 : 64>(
        P, b, F2, n_rhs_str, n_probes, mhat_at_x, nacc, bstride, smem, st);
  }
  if constexpr ((FMAX - NS) / NT < 1) {
    return cudaErrorInvalidValue;
  } else {
    const size_t sm = smem + 8 + 8 * 32 * sizeof(T) * direct_rec_stride<T, D, ORD, FMAX>();
    cudaError_t e = cudaFuncSetAttribute(direct_interp_kernel<T, D, ORD, FMAX>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
    if (e != cudaSuccess) return e;
    // one wave of resident blocks; each warp strides over the sample groups
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, direct_interp_kernel<T, D, ORD, FMAX>, 256, sm);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
      return e;
    int64_t blocks = int64_t(per_sm < 1 ? 1 : per_sm) * nsm;
    const int64_t ngroups = (P->n + 31) / 32;
    blocks = std::min<int64_t>(blocks, std::min<int64_t>(P->nblk_interp, (ngroups + 7) / 8));
    direct_interp_kernel<T, D, ORD, FMAX><<<unsigned(blocks), 256, sm, st>>>(
        P->geo, P->mono, wsp<BwDev>(P, P->r_bw), b, P->order, P->n, wsp<T>(P, P->r_xs),
        wsp<T>(P, P->r_str), perm_ptr(P), wsp<uint32_t>(P, P->r_binstart), F2, n_rhs_str,
        n_probes, P->o.y_complex, P->nrhs, static_cast<T*>(mhat_at_x), nacc, P->nbw,
        wsp<double>(P, P->r_part), bstride, P->nblk_interp);
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
