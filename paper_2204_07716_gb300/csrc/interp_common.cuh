// Device helpers shared by the at-sample kernels (interp.cu,
// interp_direct.cu, interp_global.cu and the compact-kernel pass of
// direct.cu): bulk-copy / mbarrier / cp.async primitives, the bin window
// staging, the lane-per-sample gathers, the per-warp reduction accumulators
// and phase B (finish_pass: the at-sample solve and the DF / RSS sums).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "device_common.cuh"
#include "internal.h"

namespace fk {

namespace {

constexpr int kMaxAcc = 512;  // bound on the reduced sums of one at-sample launch

// Bounded mbarrier waits: a staged-window wait polls GeoDev::wait_limit
// times (kMaxSpin unless fkreg_set_wait_limit changed it) before the kernel
// records a timeout; the wait for copies still in flight before an early
// exit always polls kMaxSpin times.
constexpr uint32_t kMaxSpin = 1u << 22;
constexpr int kLWarps = 16;              // lane-per-sample kernels: warps per block (upper bound)
constexpr int kMmaMaxRows = 16;          // tensor-core union gather: union rows (padded to 8)
constexpr int kMmaMaxCols = 24;          // and columns at most

// Transpose row (floats) of the union gather for NQ quads of fields: 4 NQ
// rounded to an odd number of 16-byte quads (eight lanes reading eight rows
// then hit distinct banks).
__host__ __device__ constexpr int mma_stage_row(int nq) { return 4 * nq + ((nq & 1) ? 0 : 4); }

// Quads of fields (4 floats) the persistent kernel keeps per sample for F2
// fields: the compile-time sizes it is instantiated for.
inline int interp_quads(int F2) {
  const int nqn = (F2 + 3) / 4;
  for (int q : {2, 4, 6, 8, 10, 12}) if (nqn <= q) return q;
  return 16;
}

// ---- bulk-copy / mbarrier primitives (inline PTX) --------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return uint32_t(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* m, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* m, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(m)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* m, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(m)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* m) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(m))
      : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Transposed warp sum: v[j] (j < 32) are this lane's values of 32 sums; on
// return lane L holds the warp total of sum L.  Five exchange levels, each
// halving the values a lane keeps: 31 shuffles for 32 sums instead of 5 per
// sum.
__device__ __forceinline__ float warp_transpose_sum(float (&v)[32], int lane) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int k = 0; k < o; ++k) {
      const float send = up ? v[k] : v[k + o];
      const float keep = up ? v[k + o] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0];
}

// Per-warp accumulators of the reductions (written by lane 0).  FP64 runs
// accumulate in double; FP32 runs keep an unevaluated sum hi + lo of two
// floats in the same 8 bytes (two_sum), which keeps the FP64 pipe (a small
// fraction of the FP32 rate on this part) out of the per-sample path.
template <typename T>
__device__ __forceinline__ void red_add(double* red, int a, T v) {
  if constexpr (sizeof(T) == 4) {
    float2* r2 = reinterpret_cast<float2*>(red) + a;
    float2 x = *r2;
    float e;
    x.x = two_sum(x.x, v, e);
    x.y += e;
    *r2 = x;
  } else {
    red[a] += v;
  }
}
template <typename T>
__device__ __forceinline__ double red_get(const double* red, int a) {
  if constexpr (sizeof(T) == 4) {
    const float2 x = reinterpret_cast<const float2*>(red)[a];
    return double(x.x) + double(x.y);
  } else {
    return red[a];
  }
}

// Issue the bulk copies of one bin window (thread 0): rows of the window
// [wm0][wm1][rec] (1-D: one row of wm0 cells) from the periodic field grid,
// row r landing at win + r * pitch, a row that wraps split in two, all
// completing on one mbarrier.
template <typename T, int D>
__device__ __forceinline__ void issue_window_copies(const T* __restrict__ fld, int rec, int nf0,
                                                    int nf1, int o0, int o1, int wm0, int wm1,
                                                    int pitch, T* win, uint64_t* mbar) {
  fence_proxy_async();  // earlier reads of the window come before the new copies
  mbar_expect_tx(mbar, uint32_t(size_t(wm0) * wm1 * rec * sizeof(T)));
  for (int r = 0; r < (D > 1 ? wm0 : 1); ++r) {
    // axis of the contiguous segment: axis 1 in 2-D, axis 0 in 1-D
    const int oseg = D > 1 ? o1 : o0;
    const int nseg = D > 1 ? nf1 : nf0;
    const int eseg = D > 1 ? wm1 : wm0;
    const int64_t rowbase = D > 1 ? wrap_idx(o0 + r, nf0) * int64_t(nf1) : 0;
    const int start = int(wrap_idx(oseg, nseg));
    const int len = min(eseg, nseg - start);
    T* dst = win + size_t(r) * pitch;
    bulk_g2s(dst, fld + (rowbase + start) * rec, uint32_t(size_t(len) * rec * sizeof(T)), mbar);
    if (len < eseg)
      bulk_g2s(dst + size_t(len) * rec, fld + rowbase * rec,
               uint32_t(size_t(eseg - len) * rec * sizeof(T)), mbar);
  }
}

// ---- lane-per-sample gathers (FP32, fixed width) ----------------------------
// acc += w * v on four fields with two packed FP32 FMAs (one issue slot per
// pair of fields; per-component results equal fmaf).
__device__ __forceinline__ void quad_fma(float4& acc, float w, const float4& v) {
  const float2 w2 = make_float2(w, w);
  const float2 lo = __ffma2_rn(w2, make_float2(v.x, v.y), make_float2(acc.x, acc.y));
  const float2 hi = __ffma2_rn(w2, make_float2(v.z, v.w), make_float2(acc.z, acc.w));
  acc = make_float4(lo.x, lo.y, hi.x, hi.y);
}

template <int D, int W, int NQ>
__device__ __forceinline__ void lane_gather_smem(const float* base, int rec, int pitch, int nq,
                                                 int skind, float beta, float off0,
                                                 const float (&pl)[W], float4 (&acc)[NQ]) {
  if (D == 1) {
#pragma unroll
    for (int t = 0; t < W; ++t) {
      const float wgt = pl[t];
      const float* cell = base + t * rec;
#pragma unroll
      for (int q = 0; q < NQ; ++q)
        if (q < nq) {
          const float4 v = *reinterpret_cast<const float4*>(cell + 4 * q);
          quad_fma(acc[q], wgt, v);
        }
    }
  } else {
#pragma unroll 1
    for (int t0 = 0; t0 < W; ++t0) {
      const float w0 = phi<float>(skind, W, beta, off0 + float(t0));
      const float* row = base + t0 * pitch;
#pragma unroll
      for (int t1 = 0; t1 < W; ++t1) {
        const float wgt = w0 * pl[t1];
        const float* cell = row + t1 * rec;
#pragma unroll
        for (int q = 0; q < NQ; ++q)
          if (q < nq) {
            const float4 v = *reinterpret_cast<const float4*>(cell + 4 * q);
            quad_fma(acc[q], wgt, v);
          }
      }
    }
  }
}

// The same from the global field grid (periodic wrap), for the rare sample
// whose window leaves the staged one.
template <int D, int W, int NQ>
__device__ __forceinline__ void lane_gather_global(const float* __restrict__ fld, int rec, int qa,
                                                int nq, int i0, int i1, int nf0, int nf1,
                                                int skind, float beta, float off0,
                                                const float (&pl)[W], float4 (&acc)[NQ]) {
#pragma unroll 1
  for (int t0 = 0; t0 < (D == 1 ? 1 : W); ++t0) {
    const float w0 = D == 1 ? 1.f : phi<float>(skind, W, beta, off0 + float(t0));
    const int64_t r = D == 1 ? 0 : wrap_idx(i0 + t0, nf0) * int64_t(nf1);
#pragma unroll
    for (int t1 = 0; t1 < W; ++t1) {
      const int64_t c = D == 1 ? wrap_idx(i0 + t1, nf0) : r + wrap_idx(i1 + t1, nf1);
      const float wgt = w0 * pl[t1];
      const float* cell = fld + c * rec + 4 * qa;
#pragma unroll
      for (int q = 0; q < NQ; ++q)
        if (q < nq) {
          const float4 v = __ldg(reinterpret_cast<const float4*>(cell + 4 * q));
          quad_fma(acc[q], wgt, v);
        }
    }
  }
}

// ---- warp-union gather on the tensor cores (2-D, FP32 fields) -----------
// The 32 sorted samples of a warp share most of their w x w windows.  Over
// the union of the windows (rows padded to a multiple of 8) the warp forms
//   V[s][f] = sum_c A[s][c] G[c][f],   A[s][c] = phi(z_s0 + r) phi(z_s1 + col)
// (A is 0 outside sample s's own window, since phi vanishes there) as
// mma.m16n8k8 products: M = 32 samples (two m-tiles), N = fields in tiles of
// 8, one k-step per union column of 8 rows.  FP32 accuracy comes from the
// three-term split x = hi + lo of both operands into TF32
// (lo*hi + hi*lo + hi*hi): hi is x cut to TF32 (11 significant bits, two
// instructions where rounding takes three), lo = x - hi exactly, and the
// tensor core reads lo's top 19 bits; the dropped lo*lo term and the two
// cuts of lo are each below 2^-20 of the product, 3 * 2^-20 in all.
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  // hi: x with its 13 low mantissa bits cleared (the tensor cores read no
  // more of a TF32 operand); lo = x - hi is exact, |lo| < 2^-10 |x|, and the
  // tensor cores drop its own low 13 bits, an error below 2^-20 |x|
  hi = __float_as_uint(x) & 0xFFFFE000u;
  lo = __float_as_uint(x - __uint_as_float(hi));
}
// d += a * b for one m16n8k8 tile; a, b hold TF32 operands.  Fragment
// layout (g = lane / 4, t = lane % 4): a = A[g][t], A[g+8][t], A[g][t+4],
// A[g+8][t+4]; b = B[t][g], B[t+4][g]; d = D[g][2t], D[g][2t+1],
// D[g+8][2t], D[g+8][2t+1].
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, "
      "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// win: the staged window; the union is rows [r0, r0 + 8 nrb) x columns
// [c0, c0 + ncol) of it (inside the window).  zr / zc: this lane's z of the
// union's first row / column (a large value for a lane without a sample).
// Fields f < 8 NTL are read from each cell (the caller keeps that inside the
// staged rows).  d[mt][nt] receives the D fragments of m-tile mt (samples
// 16 mt .. 16 mt + 15) and n-tile nt (fields 8 nt .. 8 nt + 7).
template <int W, int NTL>
__device__ __forceinline__ void mma_union_products(const float* win, int rec, int pitch, int r0,
                                                   int nrb, int c0, int ncol, int lane, float zr,
                                                   float zc, int skind, float beta,
                                                   float (&d)[2][NTL][4]) {
  const int g = lane >> 2, tq = lane & 3;
  // The A rows of this lane are samples g + 8 j (j = 0..3), the same for the
  // four lanes of a quad.  Their row weights differ per lane (rows tq and
  // tq + 4); their column weights do not, so lane tq of the quad evaluates
  // sample g + 8 tq's and the quad exchanges them.
  float zrs[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) zrs[j] = __shfl_sync(0xffffffffu, zr, g + 8 * j);
  const float zc_q = __shfl_sync(0xffffffffu, zc, g + 8 * tq);
  const int qbase = lane & ~3;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < NTL; ++nt)
#pragma unroll
      for (int k = 0; k < 4; ++k) d[mt][nt][k] = 0.f;
  const float* base = win + size_t(r0 + tq) * pitch + size_t(c0) * rec + g;
#pragma unroll 1
  for (int rb = 0; rb < nrb; ++rb) {
    // row weights of rows 8 rb + tq and 8 rb + tq + 4 for the four samples
    float wra[4], wrb[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      wra[j] = phi<float>(skind, W, beta, zrs[j] + float(8 * rb + tq));
      wrb[j] = phi<float>(skind, W, beta, zrs[j] + float(8 * rb + tq + 4));
    }
    const float* rowp = base + size_t(8 * rb) * pitch;
    // software pipeline: the next column's weight and field values are
    // fetched while this column's products run
    float wc_next = phi<float>(skind, W, beta, zc_q);
    float bn[NTL][2];
#pragma unroll
    for (int nt = 0; nt < NTL; ++nt) {
      bn[nt][0] = rowp[8 * nt];
      bn[nt][1] = rowp[size_t(4) * pitch + 8 * nt];
    }
#pragma unroll 1
    for (int c = 0; c < ncol; ++c) {
      const float wc_own = wc_next;
      float bv[NTL][2];
#pragma unroll
      for (int nt = 0; nt < NTL; ++nt) {
        bv[nt][0] = bn[nt][0];
        bv[nt][1] = bn[nt][1];
      }
      if (c + 1 < ncol) {
        wc_next = phi<float>(skind, W, beta, zc_q + float(c + 1));
        const float* cpn = rowp + size_t(c + 1) * rec;
#pragma unroll
        for (int nt = 0; nt < NTL; ++nt) {
          bn[nt][0] = cpn[8 * nt];
          bn[nt][1] = cpn[size_t(4) * pitch + 8 * nt];
        }
      }
      uint32_t ah[2][4], al[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const float wc0 = __shfl_sync(0xffffffffu, wc_own, qbase + 2 * mt);
        const float wc1 = __shfl_sync(0xffffffffu, wc_own, qbase + 2 * mt + 1);
        split_tf32(wra[2 * mt] * wc0, ah[mt][0], al[mt][0]);
        split_tf32(wra[2 * mt + 1] * wc1, ah[mt][1], al[mt][1]);
        split_tf32(wrb[2 * mt] * wc0, ah[mt][2], al[mt][2]);
        split_tf32(wrb[2 * mt + 1] * wc1, ah[mt][3], al[mt][3]);
      }
      // n-tiles in pairs: four independent tiles between the three products
      // of one tile
#pragma unroll
      for (int np = 0; np < NTL; np += 2) {
        constexpr int kP = 2;
        uint32_t bh[kP][2], bl[kP][2];
#pragma unroll
        for (int u = 0; u < kP; ++u)
          if (np + u < NTL) {
            split_tf32(bv[np + u][0], bh[u][0], bl[u][0]);
            split_tf32(bv[np + u][1], bh[u][1], bl[u][1]);
          }
#pragma unroll
        for (int u = 0; u < kP; ++u)
          if (np + u < NTL)
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) mma_tf32(d[mt][np + u], al[mt], bh[u][0], bh[u][1]);
#pragma unroll
        for (int u = 0; u < kP; ++u)
          if (np + u < NTL)
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) mma_tf32(d[mt][np + u], ah[mt], bl[u][0], bl[u][1]);
#pragma unroll
        for (int u = 0; u < kP; ++u)
          if (np + u < NTL)
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) mma_tf32(d[mt][np + u], ah[mt], bh[u][0], bh[u][1]);
      }
    }
  }
}

// The D fragments to one sample per lane, through shared memory one group of
// 8 samples at a time (group k = 2 mt + h holds samples 16 mt + 8 h + g,
// lanes 8k .. 8k + 7): stg is this warp's [8][SROW] floats; lane s ends with
// its own sample's fields in acc[q] = fields 4q .. 4q + 3.
template <int NTL, int NQ, int SROW>
__device__ __forceinline__ void mma_union_transpose(const float (&d)[2][NTL][4], int lane,
                                                    float* stg, float4 (&acc)[NQ]) {
  static_assert(2 * NTL <= NQ, "fields of the n-tiles must fit the accumulators");
  const int g = lane >> 2, tq = lane & 3;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int mt = k >> 1, h = k & 1;
#pragma unroll
    for (int nt = 0; nt < NTL; ++nt)
      *reinterpret_cast<float2*>(stg + g * SROW + 8 * nt + 2 * tq) =
          make_float2(d[mt][nt][2 * h], d[mt][nt][2 * h + 1]);
    __syncwarp();
    // group 0: every lane reads (acc holds no value while the products run,
    // and lanes of later groups overwrite theirs); later groups: only the
    // group's lanes read
    if (k == 0 || (lane >> 3) == k) {
#pragma unroll
      for (int q = 0; q < 2 * NTL; ++q)
        acc[q] = *reinterpret_cast<const float4*>(stg + (lane & 7) * SROW + 4 * q);
    }
    __syncwarp();
  }
#pragma unroll
  for (int q = 2 * NTL; q < NQ; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
}

__device__ __forceinline__ float quad_comp(const float4& v, int c) {
  return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
}

// Window extent of a bin on bandwidth b's fine grid (cells, per axis): covers
// every window of a sample in the bin with one cell of slack on each side.
// On the spreading grid itself (r = 1) the window is exact: origin
// b T - pad, extent T + w + 1.  Other grids get one more cell of slack on each
// side for the rounding of the rescaled coordinates (a sample whose window
// still falls outside is gathered from global memory).
inline int tma_slack(const GeoDev& g, const BwDev& B, int j) { return B.nf[j] == g.nf[j] ? 0 : 1; }
inline int tma_window(const GeoDev& g, const BwDev& B, int j) {
  const double r = double(B.nf[j]) / double(g.nf[j]);
  return int(std::ceil(double(g.tile[j]) * r)) + g.w + 1 + 2 * tma_slack(g, B, j);
}

// Per-group epilogue state shared by the at-sample kernels.
struct GroupCtx {
  int ns, nt, p, nq, n_rhs_real, n_probes, cplx, n_rhs_out, nacc, order, b;
};

// Phase B of one pass: lane = sample (valid when lane < cnt).  Solves on pass 0,
// then forms mhat for this pass's responses / probes and accumulates.  FP32
// runs solve p <= 3 with the compensated FP32 closed forms, everything else
// goes through FP64.
template <typename T>
__device__ __forceinline__ void finish_pass(const GroupCtx& c, const MonoTab& mono, const BwDev& B,
                                            const T* my, int pass, int q_done, int q_in, int lane,
                                            bool valid, int64_t n, const T* cvp, int64_t cstride,
                                            uint32_t orig, T* __restrict__ mhat_at_x,
                                            const T* tsc, T af[kMaxP], double* red, T k0,
                                            const double* isg) {
  if (pass == 0) {
    bool ok = false;
    T a0 = T(0);
    if (sizeof(T) == 4 && c.p <= 3 && c.order <= 1) {
      float a[kMaxP] = {0.f, 0.f, 0.f, 0.f};
      float dsc[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) dsc[k] = float(tsc[k]);
      if (valid) {
        float sv[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) sv[k] = k < c.ns ? float(my[k]) : 0.f;
        ok = lpr_weights_f32(c.p, sv, dsc, a);
      }
#pragma unroll
      for (int k = 0; k < kMaxP; ++k) af[k] = (ok && k < c.p) ? T(a[k]) * tsc[k] : T(0);
      a0 = ok ? T(a[0]) : T(0);
    } else {
      double a[kMaxP] = {0, 0, 0, 0};
      if (valid) {
        double sv[kMaxMono];
#pragma unroll
        for (int k = 0; k < kMaxMono; ++k) sv[k] = k < c.ns ? double(my[k]) : 0.0;
        if (c.order == 0) {
          ok = sv[0] > 0.0;
          a[0] = ok ? 1.0 / sv[0] : 0.0;
        } else {
          ok = lpr_weights_fast(mono, c.p, sv, B.sigma, isg, a);
        }
      }
#pragma unroll
      for (int k = 0; k < kMaxP; ++k) af[k] = (ok && k < c.p) ? T(a[k]) * tsc[k] : T(0);
      a0 = ok ? T(a[0]) : T(0);
    }
    const T tv = warp_sum_t<T>(valid ? k0 * a0 : T(0));
    if (lane == 0) red_add<T>(red, c.nacc - 1, tv);
  }
  const int fq0 = pass == 0 ? c.ns : 0;
  for (int qq = 0; qq < q_in; ++qq) {
    const int q = q_done + qq;
    T mh = T(0);
#pragma unroll
    for (int k = 0; k < kMaxP; ++k)
      if (k < c.p) mh += af[k] * my[fq0 + qq * c.nt + k];
    const T cv = valid ? cvp[int64_t(q) * cstride] : T(0);
    if (q < c.n_rhs_real) {
      const T r = valid ? cv - mh : T(0);
      const T v = warp_sum_t<T>(r * r);
      if (lane == 0) red_add<T>(red, q, v);
      if (valid && mhat_at_x) {
        const int mult = c.cplx ? 2 : 1;
        const int rr = q / mult, pt = q % mult;
        mhat_at_x[((int64_t(c.b) * c.n_rhs_out + rr) * n + orig) * mult + pt] = mh;
      }
    } else {
      const int pp = q - c.n_rhs_real;
      const T v1 = warp_sum_t<T>(valid ? cv * mh : T(0));
      const T v2 = warp_sum_t<T>(valid ? cv * cv : T(0));
      if (lane == 0) {
        red_add<T>(red, c.n_rhs_real + pp, v1);
        red_add<T>(red, c.n_rhs_real + c.n_probes + pp, v2);
      }
    }
  }
}

}  // namespace

}  // namespace fk
