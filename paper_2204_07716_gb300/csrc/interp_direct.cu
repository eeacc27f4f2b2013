// Type-2 interpolation, persistent form (FP32, width 7, 1-D / 2-D, every
// field in one pass): see interp.cu for the method.  For every field in one
// pass (F2 <= 64) and a compile-time system (order, dimension) a sample's
// fields end in its lane's registers and phase B reads them there, so no
// staging rows are needed and two bin windows fit shared memory.  One block
// per SM walks its sub-problems in turn; while it gathers from one window the
// bulk copies fill the other.  In 2-D a warp whose 32 samples' windows lie
// in a small union (rows padded to 8 at most 16, at most 24 columns) gathers
// on the tensor cores (mma_union_gather: split-TF32 products over the
// union); other warps, and 1-D plans, gather lane per sample with packed FP32
// FMAs.  The gather-only form (GONLY) writes V[f][s] for the backward instead
// of phase B.
#include <cuda_runtime.h>

#include <algorithm>

#include "device_common.cuh"
#include "interp_common.cuh"
#include "internal.h"

namespace fk {

namespace {

// Warps per block: 16 for the 1-D lane-per-sample kernel; 12 in 2-D, where
// the tensor-core gather's fragments need the registers that a 384-thread
// block leaves each thread.
template <int D>
constexpr int direct_warps() { return D == 2 ? 12 : kLWarps; }

template <int D, int W, int NQ, int ORD, bool GONLY>
__global__ void __launch_bounds__(direct_warps<D>() * 32, 1)
interp_direct_kernel(GeoDev g, const BwDev* __restrict__ bwt, int b, int64_t n,
                     const float* __restrict__ xs, const float* __restrict__ str,
                     const uint32_t* __restrict__ perm, const float* __restrict__ fld, int rec,
                     int F2, int n_rhs_real, int n_probes, int cplx, int n_rhs_out,
                     float* __restrict__ mhat_at_x, int nacc, int nbw, int64_t nblk_rows,
                     double* __restrict__ part, const uint32_t* __restrict__ sub_bin,
                     const uint32_t* __restrict__ sub_first, const uint32_t* __restrict__ bin_start,
                     const uint32_t* __restrict__ sub_total, int wm0, int wm1, int pitch,
                     int lo_slack, int win_floats, int* __restrict__ errw,
                     float* __restrict__ vout) {
  using T = float;
  constexpr int NS = ORD == 0 ? 1 : (D == 1 ? 3 : 6);   // s-fields
  constexpr int NT = ORD == 0 ? 1 : D + 1;              // t-fields per response (= p)
  constexpr int QMAX = GONLY ? 0 : (4 * NQ - NS) / NT;  // responses + probes held
  constexpr bool MMA = D == 2;                          // tensor-core union gather
  constexpr int NTL = NQ / 2;                           // its n-tiles of 8 fields
  constexpr int SROW = MMA ? mma_stage_row(NQ) : 0;     // its transpose row (floats)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t mbar[2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = int(blockDim.x >> 5);
  T* wins = reinterpret_cast<T*>(smem_raw);
  // layout: two windows, the warps' transpose rows [nwarps][8][SROW], the
  // warps' reduction accumulators [nwarps][nacc]
  float* stg = wins + 2 * size_t(win_floats) + size_t(warp) * 8 * SROW;
  double* red_all = reinterpret_cast<double*>(wins + 2 * size_t(win_floats) +
                                              size_t(nwarps) * 8 * SROW);
  double* red = red_all + warp * nacc;
  // Work sharing: sub-problem k (of the block's sequence it = 0, 1, ...) sits
  // in buffer it % 2.  Warps claim its groups of 32 samples from s_claim and
  // move on to the next sub-problem when none is left; the last warp to leave
  // a sub-problem refills its buffer with the sub-problem two ahead.  So warps
  // never wait for each other at a block barrier, and are at most one
  // sub-problem apart.
  __shared__ int s_claim[2], s_left[2], s_issued[2], s_failed;
  for (int a = lane; a < nacc; a += 32) red[a] = 0.0;
  if (threadIdx.x == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    fence_mbar_init();
    s_claim[0] = s_claim[1] = 0;
    s_left[0] = s_left[1] = 0;
    s_issued[0] = s_issued[1] = 0;
    s_failed = 0;
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
  const int nq = n_rhs_real + n_probes;
  // scaling of the t-fields: 1, 1/sigma_j
  T dsc[3] = {T(1), T(1.0 / B.sigma[0]), T(D > 1 ? 1.0 / B.sigma[1] : 1.0)};
  const T k0t = T(B.k0);
  const uint32_t nsub = *sub_total;
  auto window_of = [&](uint32_t k, int& o0, int& o1) {
    const uint32_t bin = sub_bin[k];
    const int64_t bj0 = D > 1 ? int64_t(bin) / g.nbins[1] : int64_t(bin);
    const int64_t bj1 = D > 1 ? int64_t(bin) % g.nbins[1] : 0;
    o0 = int(floor(double(bj0 * g.tile[0]) * r0)) - g.pad - lo_slack;
    o1 = D > 1 ? int(floor(double(bj1 * g.tile[1]) * r1)) - g.pad - lo_slack : 0;
  };
  if (threadIdx.x == 0) {
    for (int j = 0; j < 2; ++j) {
      const uint32_t kj = blockIdx.x + uint32_t(j) * gridDim.x;
      if (kj < nsub) {
        int a0, a1;
        window_of(kj, a0, a1);
        s_issued[j] = 1;
        issue_window_copies<T, D>(fld, rec, nf0, nf1, a0, a1, wm0, wm1, pitch,
                                  wins + size_t(j) * win_floats, &mbar[j]);
      }
    }
  }
  // per-lane running sums (hi + lo) of the slots of phase B (see below)
  constexpr int NCH = GONLY ? 1 : (2 * QMAX + 1 + 31) / 32;
  float rs_hi[NCH], rs_lo[NCH];
#pragma unroll
  for (int ch = 0; ch < NCH; ++ch) rs_hi[ch] = rs_lo[ch] = 0.f;
  volatile int* failed_flag = &s_failed;
  for (int it = 0;; ++it) {
    const uint32_t k = blockIdx.x + uint32_t(it) * gridDim.x;
    if (k >= nsub || *failed_flag) break;
    const int cur = it & 1;
    const uint32_t parity = uint32_t(it >> 1) & 1u;
    bool ok = false;
    for (uint32_t i = 0; i < g.wait_limit && !ok; ++i) ok = mbar_try_wait(&mbar[cur], parity);
    if (!__all_sync(0xffffffffu, ok)) {
      if (lane == 0) {
        atomicOr(errw, 2);
        *failed_flag = 1;
      }
      break;
    }
    const T* win = wins + size_t(cur) * win_floats;
    int o0, o1;
    window_of(k, o0, o1);
    const uint32_t first = sub_first[k];
    const uint32_t last = min(first + uint32_t(kSubMax), bin_start[sub_bin[k] + 1]);
    const int ngr = int((last - first + 31) / 32);
    // groups are claimed one ahead: the next group's coordinates load while
    // this one is processed
    auto claim = [&]() {
      int v = 0;
      if (lane == 0) v = atomicAdd(&s_claim[cur], 1);
      return __shfl_sync(0xffffffffu, v, 0);
    };
    auto coords = [&](int gq, T& c0v, T& c1v) {
      const int64_t sq = min(int64_t(first) + int64_t(gq) * 32 + lane, int64_t(last) - 1);
      c0v = xs[sq];
      c1v = D > 1 ? xs[n + sq] : T(0);
    };
    int gnext = claim();
    T xn0 = T(0), xn1 = T(0);
    if (gnext < ngr) coords(gnext, xn0, xn1);
    while (gnext < ngr) {
      const int gi = gnext;
      const T x0 = xn0, x1 = xn1;
      gnext = claim();
      if (gnext < ngr) coords(gnext, xn0, xn1);
      const int64_t s0 = int64_t(first) + int64_t(gi) * 32;
      const int cnt = int(min(int64_t(32), int64_t(last) - s0));
      const int64_t s = s0 + lane;
      const bool valid = lane < cnt;
      const T u0 = __fmul_rn(x0, ih0);
      const T fo0 = ceilf(__fsub_rn(u0, halfw));
      const int i0 = int(fo0);
      const T off0 = fo0 - u0;
      int i1 = 0;
      T off1 = T(0), u1 = T(0);
      if (D > 1) {
        u1 = __fmul_rn(x1, ih1);
        const T fo1 = ceilf(__fsub_rn(u1, halfw));
        i1 = int(fo1);
        off1 = fo1 - u1;
      }
      const int l0 = i0 - o0, l1 = D > 1 ? i1 - o1 : 0;
      const bool inside = l0 >= 0 && l0 + W <= wm0 && (D == 1 || (l1 >= 0 && l1 + W <= wm1));
      const int nqd = (F2 + 3) >> 2;
      float4 acc[NQ];
      // the union of the warp's windows (rows padded to a multiple of 8)
      bool use_mma = false;
      int ur0 = 0, unrb = 0, uc0 = 0, uncol = 0;
      if constexpr (MMA) {
        if (__all_sync(0xffffffffu, !valid || inside)) {
          const int lo0 = __reduce_min_sync(0xffffffffu, valid ? l0 : INT_MAX);
          const int hi0 = __reduce_max_sync(0xffffffffu, valid ? l0 : INT_MIN) + W;
          const int lo1 = __reduce_min_sync(0xffffffffu, valid ? l1 : INT_MAX);
          const int hi1 = __reduce_max_sync(0xffffffffu, valid ? l1 : INT_MIN) + W;
          const int rows = (hi0 - lo0 + 7) & ~7;
          if (rows <= kMmaMaxRows && rows <= wm0 && hi1 - lo1 <= kMmaMaxCols) {
            use_mma = true;
            unrb = rows >> 3;
            ur0 = min(lo0, wm0 - rows);
            uc0 = lo1;
            uncol = hi1 - lo1;
            if constexpr (kChecked)  // the union inside the staged window
              use_mma = in_range(errw, kSiteInterpWindow, ur0, wm0 - rows + 1) &&
                        in_range(errw, kSiteInterpWindow, uc0, wm1 - uncol + 1);
          }
        }
      }
      // strengths and original index (phase B), issued before the transpose
      // of the tensor-core path so their latency overlaps it
      uint32_t orig = 0u;
      T cv[QMAX > 0 ? QMAX : 1];
      auto load_strengths = [&]() {
        if (!GONLY) {
          orig = valid ? perm[s] : 0u;
#pragma unroll
          for (int q = 0; q < QMAX; ++q)
            cv[q] = (valid && q < nq) ? str[int64_t(1 + q) * n + s] : T(0);
        }
      };
      if (use_mma) {
        const T zr = valid ? T(o0 + ur0) - u0 : T(1e4f);
        const T zc = valid ? T(o1 + uc0) - u1 : T(1e4f);
        float dfr[2][NTL][4];
        mma_union_products<W, NTL>(win, rec, pitch, ur0, unrb, uc0, uncol, lane, zr, zc, skind,
                                   beta, dfr);
        load_strengths();
        mma_union_transpose<NTL, NQ, SROW>(dfr, lane, stg, acc);
      } else {
        load_strengths();
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        T pl[W];
#pragma unroll
        for (int t = 0; t < W; ++t) pl[t] = phi<T>(skind, W, beta, (D > 1 ? off1 : off0) + T(t));
        const int64_t last_read = (D > 1 ? int64_t(l0 + W - 1) * pitch + int64_t(l1 + W - 1) * rec
                                         : int64_t(l0 + W - 1) * rec) + 4 * nqd - 1;
        if (inside && in_range(errw, kSiteInterpWindow, last_read, win_floats))
          lane_gather_smem<D, W, NQ>(win + size_t(l0) * (D > 1 ? pitch : rec) + l1 * rec, rec,
                                     pitch, nqd, skind, beta, off0, pl, acc);
        if (__any_sync(0xffffffffu, valid && !inside)) {
          if (valid && !inside)
            lane_gather_global<D, W, NQ>(fld, rec, 0, nqd, i0, i1, nf0, nf1, skind, beta, off0, pl,
                                         acc);
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
      // phase B: the system of eq. 3 at x_i from the s-fields in registers
      float a[kMaxP] = {0.f, 0.f, 0.f, 0.f};
      bool okv = false;
      if (valid) {
        float sv[6];
#pragma unroll
        for (int k2 = 0; k2 < 6; ++k2) sv[k2] = k2 < NS ? quad_comp(acc[k2 >> 2], k2 & 3) : 0.f;
        okv = lpr_weights_f32(NT, sv, dsc, a);
      }
      T af[NT];
#pragma unroll
      for (int k2 = 0; k2 < NT; ++k2) af[k2] = okv ? a[k2] * dsc[k2 < 3 ? k2 : 0] : T(0);
      // this sample's terms of the sums of eq. 22 and Sec. 2.1, by slot:
      // [0, QMAX) the squared residual (responses) or w_p S w_p (probes),
      // [QMAX, 2 QMAX) w_p w_p (probes), 2 QMAX the exact-trace term
      float vals[32 * NCH];
#pragma unroll
      for (int j = 0; j < 32 * NCH; ++j) vals[j] = 0.f;
      vals[2 * QMAX] = okv ? k0t * a[0] : T(0);
#pragma unroll
      for (int q = 0; q < QMAX; ++q) {
        if (q >= nq) break;
        T mh = T(0);
#pragma unroll
        for (int k2 = 0; k2 < NT; ++k2) {
          const int f = NS + q * NT + k2;
          mh += af[k2] * quad_comp(acc[f >> 2], f & 3);
        }
        if (q < n_rhs_real) {
          const T r = valid ? cv[q] - mh : T(0);
          vals[q] = r * r;
          if (valid && mhat_at_x) {
            const int mult = cplx ? 2 : 1;
            const int rr = q / mult, pt = q % mult;
            mhat_at_x[((int64_t(b) * n_rhs_out + rr) * n + orig) * mult + pt] = mh;
          }
        } else {
          vals[q] = valid ? cv[q] * mh : T(0);
          vals[QMAX + q] = valid ? cv[q] * cv[q] : T(0);
        }
      }
      // the warp's totals, one slot per lane, added to the lane's
      // compensated running sums
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) {
        float part32[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) part32[j] = vals[32 * ch + j];
        const float t = warp_transpose_sum(part32, lane);
        float e;
        rs_hi[ch] = two_sum(rs_hi[ch], t, e);
        rs_lo[ch] += e;
      }
    }
    // this warp leaves sub-problem k; the last to leave refills the buffer
    __syncwarp();
    if (lane == 0) {
      __threadfence_block();
      if (atomicAdd(&s_left[cur], 1) == nwarps - 1) {
        s_claim[cur] = 0;
        s_left[cur] = 0;
        const uint32_t k2 = k + 2 * gridDim.x;
        if (k2 < nsub && !*failed_flag) {
          int a0, a1;
          window_of(k2, a0, a1);
          s_issued[cur] += 1;
          __threadfence_block();
          issue_window_copies<T, D>(fld, rec, nf0, nf1, a0, a1, wm0, wm1, pitch,
                                    wins + size_t(cur) * win_floats, &mbar[cur]);
        }
      }
    }
  }
  // slot j -> accumulator of the partial-sum layout: responses' RSS and the
  // probes' w S w at j, the probes' w w at n_rhs_real + n_probes + p, the
  // exact-trace term at nacc - 1
  if (!GONLY) {
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) {
      const int j = 32 * ch + lane;
      int a = -1;
      if (j < nq) a = j;
      else if (j >= QMAX && j < QMAX + nq && j - QMAX >= n_rhs_real) a = n_probes + j - QMAX;
      else if (j == 2 * QMAX) a = nacc - 1;
      if (a >= 0) reinterpret_cast<float2*>(red)[a] = make_float2(rs_hi[ch], rs_lo[ch]);
    }
  }
  __syncthreads();
  if (*failed_flag) {
    // wait (bounded) for the copies still in flight before leaving
    if (threadIdx.x == 0)
      for (int j = 0; j < 2; ++j)
        if (s_issued[j] > 0) {
          const uint32_t pj = uint32_t(s_issued[j] - 1) & 1u;
          bool late = false;
          for (uint32_t i = 0; i < kMaxSpin && !late; ++i) late = mbar_try_wait(&mbar[j], pj);
        }
    return;
  }
  for (int a = threadIdx.x; a < nacc; a += blockDim.x) {
    double t = 0.0;
    for (int wv = 0; wv < nwarps; ++wv) t += red_get<T>(red_all, wv * nacc + a);
    part[(int64_t(blockIdx.x) * nbw + b) * nacc + a] = t;
    // partial rows of the block indices this persistent grid does not launch
    for (int64_t r = int64_t(blockIdx.x) + gridDim.x; r < nblk_rows; r += gridDim.x)
      part[(r * nbw + b) * nacc + a] = 0.0;
  }
}


template <int D, int NQ, int ORD, bool GONLY>
cudaError_t launch_direct_k(fkreg_plan_s* P, int b, int n_rhs_real, int n_probes,
                            void* mhat_at_x, cudaStream_t st, int nacc, int F2, float* vout,
                            int rec, int wm0, int wm1, int pitch, int slack, int win_floats,
                            int nw, size_t smem, unsigned grid) {
  auto kern = interp_direct_kernel<D, 7, NQ, ORD, GONLY>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  kern<<<grid, nw * 32, smem, st>>>(
      P->geo, wsp<BwDev>(P, P->r_bw), b, P->n, wsp<float>(P, P->r_xs), wsp<float>(P, P->r_str),
      perm_ptr(P), wsp<float>(P, P->r_t2field), rec, F2, n_rhs_real, n_probes, P->o.y_complex,
      P->nrhs, static_cast<float*>(mhat_at_x), nacc, P->nbw, P->nblk_interp,
      wsp<double>(P, P->r_part), wsp<uint32_t>(P, P->r_subbin), wsp<uint32_t>(P, P->r_subfirst),
      wsp<uint32_t>(P, P->r_binstart), wsp<uint32_t>(P, P->r_substart) + P->nbins_total, wm0, wm1,
      pitch, slack, win_floats, wsp<int>(P, P->r_err), vout);
  P->launches += 1;
  return cudaGetLastError();
}

template <int D, int ORD, bool GONLY>
cudaError_t launch_direct_q(fkreg_plan_s* P, int b, int n_rhs_real, int n_probes,
                            void* mhat_at_x, cudaStream_t st, int nacc, int F2, float* vout,
                            int rec, int wm0, int wm1, int pitch, int slack, int win_floats,
                            int nw, size_t smem, unsigned grid) {
#define FK_Q(Q)                                                                                  \
  return launch_direct_k<D, Q, ORD, GONLY>(P, b, n_rhs_real, n_probes, mhat_at_x, st, nacc, F2, \
                                           vout, rec, wm0, wm1, pitch, slack, win_floats, nw,     \
                                           smem, grid)
  switch (interp_quads(F2)) {
    case 2: FK_Q(2);
    case 4: FK_Q(4);
    case 6: FK_Q(6);
    case 8: FK_Q(8);
    case 10: FK_Q(10);
    case 12: FK_Q(12);
    default: FK_Q(16);
  }
#undef FK_Q
}

}  // namespace

// Launch the persistent kernel if it applies (FP32, width 7, 1-D / 2-D,
// F2 <= 64, two windows fit shared memory); *launched says whether it ran.
cudaError_t run_interp_direct(fkreg_plan_s* P, int b, int n_rhs_real, int n_probes,
                              void* mhat_at_x, cudaStream_t st, int nacc, int F2, void* vout,
                              bool* launched) {
  *launched = false;
  const int D = P->d;
  if (P->prec != FKREG_F32 || P->geo.w != 7 || D > 2 || F2 > 64 || P->n == 0) return cudaSuccess;
  if (!vout && P->order > 1) return cudaSuccess;
  const BwDev& B = P->bw[b];
  const int rec = t2_record_stride(F2);
  const int wm0 = tma_window(P->geo, B, 0);
  const int wm1 = D > 1 ? tma_window(P->geo, B, 1) : 1;
  if (wm0 > B.nf[0] || (D > 1 && wm1 > B.nf[1])) return cudaSuccess;
  const int nq = interp_quads(F2);
  // 2-D rows end in a pad that keeps the pitch at 8 (mod 32) floats, so the
  // eight rows of a tensor-core k-step start in distinct bank groups, and
  // that holds the fields up to 4 nq a union-gather lane reads in a row's
  // last cell
  int pitch = wm0 * rec;
  if (D > 1) {
    int pad = std::max(4, 4 * nq - rec);
    while ((wm1 * rec + pad) % 32 != 8) pad += 4;
    pitch = wm1 * rec + pad;
  }
  const int win_floats = ((D > 1 ? wm0 : 1) * pitch + 31) / 32 * 32;
  const int slack = std::max(tma_slack(P->geo, B, 0), D > 1 ? tma_slack(P->geo, B, 1) : 0);
  const size_t budget = 225 * 1024;
  const size_t wins = 2 * sizeof(float) * size_t(win_floats);
  const size_t per_warp =
      sizeof(double) * nacc + (D > 1 ? sizeof(float) * 8 * size_t(mma_stage_row(nq)) : 0);
  if (wins + per_warp * 8 > budget) return cudaSuccess;
  const int nw = int(std::min<size_t>(D > 1 ? direct_warps<2>() : direct_warps<1>(),
                                      (budget - wins) / std::max<size_t>(per_warp, 1)));
  const size_t smem = wins + per_warp * size_t(nw);
  const unsigned grid = unsigned(std::min<int64_t>(P->sm_count, std::max<int64_t>(1, P->nsub_max)));
  float* vo = static_cast<float*>(vout);
  *launched = true;
#define FK_A(DD, OO, GG)                                                                        \
  return launch_direct_q<DD, OO, GG>(P, b, n_rhs_real, n_probes, mhat_at_x, st, nacc, F2, vo,  \
                                     rec, wm0, wm1, pitch, slack, win_floats, nw, smem, grid)
  if (vout) {
    if (D == 1) FK_A(1, 0, true);
    FK_A(2, 0, true);
  }
  if (D == 1) {
    if (P->order == 0) FK_A(1, 0, false);
    FK_A(1, 1, false);
  }
  if (P->order == 0) FK_A(2, 0, false);
  FK_A(2, 1, false);
#undef FK_A
}

}  // namespace fk
