// Device helpers shared by the spreading, interpolation, direct-sum and
// solve kernels.
#pragma once

#include <cuda_runtime.h>

#include "checked.cuh"
#include "internal.h"

namespace fk {

__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

template <typename T>
__device__ __forceinline__ T inv_h_of(const GeoDev& g, int j);
template <>
__device__ __forceinline__ float inv_h_of<float>(const GeoDev& g, int j) { return g.inv_h_f[j]; }
template <>
__device__ __forceinline__ double inv_h_of<double>(const GeoDev& g, int j) { return g.inv_h[j]; }

// Spreading kernel phi at offset z (fine cells): exponential of semicircle
// exp(beta (sqrt(1 - (2z/w)^2) - 1)) on |z| <= w/2, or the truncated Gaussian
// exp(-beta z^2) of eq. 17.
template <typename T>
__device__ __forceinline__ T phi(int kind, int w, T beta, T z) {
  if (kind == FKREG_SPREAD_ES) {
    const T t = z * (T(2) / T(w));
    const T a = T(1) - t * t;
    return a > T(0) ? exp(beta * (sqrt(a) - T(1))) : T(0);
  }
  return (fabs(z) <= T(0.5) * T(w)) ? exp(-beta * z * z) : T(0);
}

// FP32: the same kernels from the hardware reciprocal square root and base-2
// exponential (rsqrtf, exp2f), with exp(x) = 2^(x log2 e).  sqrt(a) is taken
// as s = a rsqrt(a) plus one Newton step on the exact residual a - s^2
// (fmaf), which brings s to within about one unit in the last place, as a
// correctly rounded square root would be; the exponent beta log2e (s - 1) is
// one fused multiply-add.  The error of the value, relative, stays near
// beta 2^-23 at the centre (the amplification of the rounding of s that the
// formula itself has) and far below the FP32 tolerance of the transform.
template <>
__device__ __forceinline__ float phi<float>(int kind, int w, float beta, float z) {
  constexpr float kLog2e = 1.4426950408889634f;
  const float bl = beta * kLog2e;
  if (kind == FKREG_SPREAD_ES) {
    const float t = z * (2.f / float(w));
    const float a = fmaf(-t, t, 1.f);
    if (!(a > 0.f)) return 0.f;
    const float r = rsqrtf(a);
    float s = a * r;
    s = fmaf(0.5f * r, fmaf(-s, s, a), s);
    return exp2f(fmaf(s, bl, -bl));
  }
  return (fabsf(z) <= 0.5f * float(w)) ? exp2f(-bl * z * z) : 0.f;
}

// Compact radial profile k(|u|^2) of the regression kernels (unit ball;
// normalisation in BwDev::kscale): uniform, Epanechnikov, triangle,
// biweight, triweight, and the Gaussian cut at Mahalanobis radius R
// (u = z / R in the bandwidth's metric, k = exp(-R^2 |u|^2 / 2), r2 = R^2).
template <typename T>
__device__ __forceinline__ T compact_k(int kern, T u2, T r2) {
  if (!(u2 <= T(1))) return T(0);
  const T e = T(1) - u2;
  switch (kern) {
    case FKREG_KERNEL_UNIFORM: return T(1);
    case FKREG_KERNEL_EPANECHNIKOV: return e;
    case FKREG_KERNEL_TRIANGLE: return T(1) - sqrt(u2);
    case FKREG_KERNEL_BIWEIGHT: return e * e;
    case FKREG_KERNEL_GAUSSIAN_DIRECT: return exp(T(-0.5) * r2 * u2);
    default: return e * e * e;
  }
}

// Compile-time chain of the monomials of degree <= DEG in d = D variables, in
// the graded order the plan's monomial table uses (degree by degree, index
// multisets in lexicographic order): monomial f > 0 is monomial parent[f]
// times coordinate axis[f].  The monomials of degree <= l are a prefix.
struct MonoChain {
  int n;
  int parent[kMaxMono];
  int axis[kMaxMono];
};

__host__ __device__ constexpr MonoChain make_mono_chain(int D, int DEG) {
  MonoChain c{0, {}, {}};
  int e[kMaxMono][3] = {};
  for (int k = 0; k <= DEG; ++k) {
    int idx[4] = {0, 0, 0, 0};
    for (;;) {
      const int m = c.n;
      for (int j = 0; j < 3; ++j) e[m][j] = 0;
      for (int j = 0; j < k; ++j) e[m][idx[j]] += 1;
      c.parent[m] = 0;
      c.axis[m] = 0;
      if (k > 0) {
        const int ax = idx[k - 1];
        c.axis[m] = ax;
        for (int r = 0; r < m; ++r) {
          bool same = true;
          for (int j = 0; j < 3; ++j)
            if (e[r][j] != e[m][j] - (j == ax ? 1 : 0)) same = false;
          if (same) {
            c.parent[m] = r;
            break;
          }
        }
      }
      c.n = m + 1;
      int p = k - 1;
      while (p >= 0 && idx[p] == D - 1) --p;
      if (p < 0) break;
      idx[p] += 1;
      for (int j = p + 1; j < k; ++j) idx[j] = idx[p];
    }
  }
  return c;
}

__host__ __device__ constexpr int mono_count(int D, int DEG) { return make_mono_chain(D, DEG).n; }

template <typename T, int D, int DEG, int F = 0>
__device__ __forceinline__ void mono_build(T* mo, const T* z) {
  if constexpr (F < mono_count(D, DEG)) {
    if constexpr (F == 0) {
      mo[0] = T(1);
    } else {
      constexpr int pf = make_mono_chain(D, DEG).parent[F];
      constexpr int af = make_mono_chain(D, DEG).axis[F];
      mo[F] = mo[pf] * z[af];
    }
    mono_build<T, D, DEG, F + 1>(mo, z);
  }
}

// Candidate bins of a support query for points whose coordinates (relative
// to lo) span [mn_j, mx_j] on each axis.  box(): the bins of the leading axes
// and the full range of the last axis; row(): one row of leading-axis bins,
// i.e. a run of bins adjacent along the last axis (one contiguous range of
// the sort).  With a diagonal H the row's last-axis range is cut to the
// section of the support ellipsoid nearest to the points: a sample whose
// leading coordinates lie at distances dx_j from [mn_j, mx_j] can be inside
// the support only within sigma_d sqrt(1 - sum (dx_j / sigma_j)^2) of
// [mn_d, mx_d].  The bin arithmetic is FP32 (floor(floor(u) / t) =
// floor(u / t) for the tile t); every range is widened by 1e-3 sigma and by
// a rounding margin in bins, so that no sample inside a support is dropped.
template <int D>
struct DirectRows {
  int blo[3], bhi[3];
  float mn[3], mx[3], sg[3], isg[3], ibw[3], wb[3], mb[3];
  bool diag;

  __device__ __forceinline__ void box(const GeoDev& g, const BwDev& B) {
    diag = true;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int c = 0; c < D; ++c)
        if (a != c && B.Hinv[a * 3 + c] != 0.0) diag = false;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      blo[j] = 0;
      bhi[j] = 0;
    }
#pragma unroll
    for (int j = 0; j < D; ++j) {
      sg[j] = float(B.sigma[j]);
      isg[j] = float(1.0 / B.sigma[j]);
      ibw[j] = float(g.inv_h[j] / double(g.tile[j]));
      wb[j] = float(double(g.tile[j]) / g.inv_h[j]);
      mb[j] = 1e-3f + 2e-7f * float(g.nbins[j]);
      const float hw = sg[j] * 1.001f;
      const int nb = int(g.nbins[j]);
      int b0 = int(floorf((mn[j] - hw) * ibw[j] - mb[j]));
      int b1 = int(floorf((mx[j] + hw) * ibw[j] + mb[j]));
      blo[j] = b0 < 0 ? 0 : (b0 > nb - 1 ? nb - 1 : b0);
      bhi[j] = b1 < 0 ? 0 : (b1 > nb - 1 ? nb - 1 : b1);
    }
  }
  __device__ __forceinline__ int rows0() const { return D > 1 ? bhi[0] - blo[0] + 1 : 1; }
  __device__ __forceinline__ int rows1() const { return D > 2 ? bhi[1] - blo[1] + 1 : 1; }

  // bins [first, last] of row (r0, r1); false when the row is empty
  __device__ __forceinline__ bool row(const GeoDev& g, int r0, int r1, int64_t& first,
                                      int64_t& last) const {
    int lo = blo[D - 1], hi = bhi[D - 1];
    if (D > 1 && diag) {
      const int b[2] = {blo[0] + r0, blo[1] + r1};
      float rem = 1.f;
#pragma unroll
      for (int j = 0; j < D - 1; ++j) {
        const float a = float(b[j]) * wb[j], e = a + wb[j];
        float dx = fmaxf(a - mx[j], mn[j] - e) - 1e-3f * sg[j];
        dx = dx > 0.f ? dx : 0.f;
        const float t = dx * isg[j];
        rem -= t * t;
      }
      if (rem < 0.f) return false;
      const float hw = sg[D - 1] * (sqrtf(rem) + 1e-3f);
      const int c0 = int(floorf((mn[D - 1] - hw) * ibw[D - 1] - mb[D - 1]));
      const int c1 = int(floorf((mx[D - 1] + hw) * ibw[D - 1] + mb[D - 1]));
      lo = c0 > lo ? c0 : lo;
      hi = c1 < hi ? c1 : hi;
      if (lo > hi) return false;
    }
    if (D == 1) {
      first = lo;
      last = hi;
    } else if (D == 2) {
      first = int64_t(blo[0] + r0) * g.nbins[1] + lo;
      last = first + (hi - lo);
    } else {
      first = (int64_t(blo[0] + r0) * g.nbins[1] + blo[1] + r1) * g.nbins[2] + lo;
      last = first + (hi - lo);
    }
    return true;
  }
};

// Shared memory of one warp's candidate queue in direct_warp_sums: 64
// entries of (z[0..D), weight) in T, then 64 sample indices.
template <typename T, int D>
__host__ __device__ constexpr int direct_queue_bytes() {
  return 64 * (D + 1) * int(sizeof(T)) + 64 * 4;
}

// Warp-cooperative moment sums of one evaluation point q (coordinates
// relative to lo) over the binned samples inside its kernel support: the
// lanes stride over the sample ranges of the support's bins (bins adjacent
// along the last axis are one contiguous range of the sort) and test each
// candidate; the ones inside the support are compacted into a per-warp queue
// in shared memory (qmem, direct_queue_bytes), and each time 32 are queued
// every lane adds one of them to all fields in registers, so that the
// monomial and strength work runs on full warps.  The fields are reduced
// across the warp at the end: field f is returned to lane f mod 32 (out0 for
// f < 32, out1 above): [0, NS) the s-fields, NS + r NT + k the t-fields of
// strength str_first + r.  NS and NT are the monomial counts of degrees 2*ORD
// and ORD; FMAX >= NS + nstr NT bounds the fields.  Sums are in the plan
// precision T.
template <typename T, int D, int ORD, int FMAX>
__device__ __forceinline__ void direct_warp_sums(const GeoDev& g, const BwDev& B, int64_t n,
                                                 const T* __restrict__ xs,
                                                 const T* __restrict__ str, int str_first,
                                                 int nstr, const uint32_t* __restrict__ bin_start,
                                                 const double* q, int lane, unsigned char* qmem,
                                                 T& out0, T& out1) {
  constexpr int NS = mono_count(D, 2 * ORD), NT = mono_count(D, ORD);
  constexpr int QMAX = (FMAX - NS) / NT;
  static_assert(QMAX >= 1 && FMAX <= 64, "field bucket");
  T* qv = reinterpret_cast<T*>(qmem);                                   // [D + 1][64]
  uint32_t* qi = reinterpret_cast<uint32_t*>(qmem + 64 * (D + 1) * sizeof(T));  // [64]
  DirectRows<D> rows;
#pragma unroll
  for (int j = 0; j < D; ++j) rows.mn[j] = rows.mx[j] = float(q[j]);
  rows.box(g, B);
  T qt[D], hi[D][D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    qt[a] = T(q[a]);
#pragma unroll
    for (int c = 0; c < D; ++c) hi[a][c] = T(B.Hinv[a * 3 + c]);
  }
  const T ks = T(B.kscale), kr2 = T(B.kr2);
  const int kern = g.kern;
  T acc[FMAX];
#pragma unroll
  for (int f = 0; f < FMAX; ++f) acc[f] = T(0);
  // one queued candidate per lane (lane < cnt) into every field
  auto consume = [&](int cnt) {
    if (lane < cnt) {
      T z[D];
#pragma unroll
      for (int j = 0; j < D; ++j) z[j] = qv[j * 64 + lane];
      const T wgt = qv[D * 64 + lane];
      const int64_t i = qi[lane];
      T mo[NS];
      mono_build<T, D, 2 * ORD>(mo, z);
#pragma unroll
      for (int f = 0; f < NS; ++f) acc[f] += wgt * mo[f];
#pragma unroll
      for (int r = 0; r < QMAX; ++r)
        if (r < nstr) {
          const T cw = wgt * str[int64_t(str_first + r) * n + i];
#pragma unroll
          for (int k = 0; k < NT; ++k) acc[NS + r * NT + k] += cw * mo[k];
        }
    }
  };
  int qn = 0;  // queued candidates (warp-uniform)
  const unsigned below = (1u << lane) - 1u;
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
        T z[D];
        bool in = false;
        T wgt = T(0);
        if (i < i1) {
#pragma unroll
          for (int j = 0; j < D; ++j) z[j] = xs[int64_t(j) * n + i] - qt[j];
          T u2 = T(0);
#pragma unroll
          for (int a = 0; a < D; ++a) {
            T ra = T(0);
#pragma unroll
            for (int c = 0; c < D; ++c) ra += hi[a][c] * z[c];
            u2 += z[a] * ra;
          }
          in = u2 <= T(1);
          if (in) wgt = ks * compact_k<T>(kern, u2, kr2);
        }
        const unsigned m = __ballot_sync(0xffffffffu, in);
        if (in) {
          const int slot = qn + __popc(m & below);
#pragma unroll
          for (int j = 0; j < D; ++j) qv[j * 64 + slot] = z[j];
          qv[D * 64 + slot] = wgt;
          qi[slot] = i;
        }
        qn += __popc(m);
        if (qn >= 32) {
          __syncwarp();
          consume(32);
          __syncwarp();
          if (lane < qn - 32) {  // move the overflow to the front of the queue
#pragma unroll
            for (int j = 0; j <= D; ++j) qv[j * 64 + lane] = qv[j * 64 + 32 + lane];
            qi[lane] = qi[32 + lane];
          }
          qn -= 32;
          __syncwarp();
        }
      }
    }
  __syncwarp();
  consume(qn);
  __syncwarp();
  out0 = T(0);
  out1 = T(0);
  const int nf = NS + nstr * NT;
#pragma unroll
  for (int f = 0; f < FMAX; ++f) {
    if (f < nf) {
      T v = acc[f];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == (f & 31)) {
        if (f < 32)
          out0 = v;
        else
          out1 = v;
      }
    }
  }
}

template <typename T>
__device__ __forceinline__ T sel3(int ax, T a, T b, T c) {
  return ax == 0 ? a : (ax == 1 ? b : c);
}

__device__ __forceinline__ int64_t wrap_idx(int64_t m, int64_t nf) {
  return m < 0 ? m + nf : (m >= nf ? m - nf : m);
}

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Solve S a = e_1 (p x p, FP64, partial pivoting). Returns false if singular.
__device__ __forceinline__ bool solve_e1(int p, double S[kMaxP][kMaxP], double a[kMaxP]) {
  double r[kMaxP];
  for (int i = 0; i < p; ++i) r[i] = (i == 0) ? 1.0 : 0.0;
  for (int c = 0; c < p; ++c) {
    int piv = c;
    for (int i = c + 1; i < p; ++i)
      if (fabs(S[i][c]) > fabs(S[piv][c])) piv = i;
    if (!(fabs(S[piv][c]) > 0.0)) return false;
    if (piv != c) {
      for (int j = 0; j < p; ++j) {
        double t = S[c][j];
        S[c][j] = S[piv][j];
        S[piv][j] = t;
      }
      double t = r[c];
      r[c] = r[piv];
      r[piv] = t;
    }
    for (int i = c + 1; i < p; ++i) {
      const double f = S[i][c] / S[c][c];
      for (int j = c; j < p; ++j) S[i][j] -= f * S[c][j];
      r[i] -= f * r[c];
    }
  }
  for (int i = p - 1; i >= 0; --i) {
    double v = r[i];
    for (int j = i + 1; j < p; ++j) v -= S[i][j] * a[j];
    a[i] = v / S[i][i];
  }
  return isfinite(a[0]);
}

__device__ __forceinline__ int mono_index(const MonoTab& m, int nm, int e0, int e1, int e2) {
  for (int k = 0; k < nm; ++k)
    if (m.e[k][0] == e0 && m.e[k][1] == e1 && m.e[k][2] == e2) return k;
  return 0;
}

// sigma^g for the t-field monomial a
__device__ __forceinline__ double tscale(const MonoTab& mono, int a, const double* sigma) {
  double sc = 1.0;
  for (int j = 0; j < 3; ++j)
    for (int r = 0; r < mono.e[a][j]; ++r) sc *= sigma[j];
  return sc;
}

// Scaled normal matrix S~_ab = s_(a+b) / sigma^(a+b) from the s-fields, and
// a = S~^-1 e_1 (the intercept is unchanged by the scaling), by elimination.
__device__ __forceinline__ bool lpr_weights(const MonoTab& mono, int p, const double* s,
                                            const double* sigma, double a[kMaxP]) {
  double S[kMaxP][kMaxP];
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < p; ++j) {
      const int e0 = mono.e[i][0] + mono.e[j][0];
      const int e1 = mono.e[i][1] + mono.e[j][1];
      const int e2 = mono.e[i][2] + mono.e[j][2];
      const int k = mono_index(mono, mono.n, e0, e1, e2);
      double sc = 1.0;
      for (int r = 0; r < e0; ++r) sc *= sigma[0];
      for (int r = 0; r < e1; ++r) sc *= sigma[1];
      for (int r = 0; r < e2; ++r) sc *= sigma[2];
      S[i][j] = s[k] / sc;
    }
  return solve_e1(p, S, a);
}

// Same result with closed forms for Nadaraya-Watson and local linear in 1-D
// and 2-D (one division); isg = 1 / sigma.  Other systems (local linear in
// 3-D, local quadratic) go through elimination.
__device__ __forceinline__ bool lpr_weights_fast(const MonoTab& mono, int p, const double* s,
                                                 const double* sigma, const double* isg,
                                                 double a[kMaxP]) {
  if (p == 1) {
    a[0] = 1.0 / s[0];
    return s[0] > 0.0;
  }
  if (p == 2 && mono.n == 3) {  // 1-D local linear
    const double s01 = s[1] * isg[0], s11 = s[2] * (isg[0] * isg[0]);
    const double det = s[0] * s11 - s01 * s01;
    if (!(det > 0.0)) return false;
    const double inv = 1.0 / det;
    a[0] = s11 * inv;
    a[1] = -s01 * inv;
    return isfinite(a[0]);
  }
  if (p == 3 && mono.n == 6) {  // 2-D local linear, s-fields 1, z1, z2, z1z1, z1z2, z2z2
    const double h0 = isg[0], h1 = isg[1];
    const double s00 = s[0], s01 = s[1] * h0, s02 = s[2] * h1;
    const double s11 = s[3] * (h0 * h0), s12 = s[4] * (h0 * h1), s22 = s[5] * (h1 * h1);
    const double c0 = s11 * s22 - s12 * s12;
    const double c1 = s12 * s02 - s01 * s22;
    const double c2 = s01 * s12 - s11 * s02;
    const double det = s00 * c0 + s01 * c1 + s02 * c2;
    if (!(det > 0.0)) return false;
    const double inv = 1.0 / det;
    a[0] = c0 * inv;
    a[1] = c1 * inv;
    a[2] = c2 * inv;
    return isfinite(a[0]);
  }
  return lpr_weights(mono, p, s, sigma, a);
}

// ---- compensated FP32 arithmetic for the at-sample solves ------------------
// two_sum: s + e == a + b exactly (Knuth's branch-free sum).
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}

// a b - c d by Kahan's algorithm: the rounding error of c d is recovered
// exactly with an FMA, so the result is within two units of rounding of the
// exact value even under cancellation (Jeannerod, Louvet, Muller 2013).
__device__ __forceinline__ float dop(float a, float b, float c, float d) {
  const float w = __fmul_rn(c, d);
  const float e = fmaf(-c, d, w);
  const float f = fmaf(a, b, -w);
  return __fadd_rn(f, e);
}

// a = S~^-1 e_1 for p <= 3 from FP32 s-fields, S~_jk = D_j D_k s_(j+k) with
// D = (1, dsc[1], dsc[2]) the scaling the t-fields get.  Cofactors come from
// dop and the determinant from a compensated dot product (Ogita, Rump, Oishi
// 2005), so the solve adds rounding errors of a few units of FP32 whatever
// the cancellation in the cofactor expansion; the FP32 field values carry
// the NUFFT tolerance, which dominates.
__device__ __forceinline__ bool lpr_weights_f32(int p, const float* s, const float* dsc,
                                                float a[kMaxP]) {
  if (p == 1) {
    a[0] = 1.0f / s[0];
    return s[0] > 0.f;
  }
  if (p == 2) {  // 1-D local linear
    const float h0 = dsc[1];
    const float s01 = s[1] * h0, s11 = s[2] * (h0 * h0);
    const float det = dop(s[0], s11, s01, s01);
    if (!(det > 0.f)) return false;
    const float inv = 1.0f / det;
    a[0] = s11 * inv;
    a[1] = -s01 * inv;
    return isfinite(a[0]);
  }
  // 2-D local linear, s-fields 1, z1, z2, z1z1, z1z2, z2z2
  const float h0 = dsc[1], h1 = dsc[2];
  const float s00 = s[0], s01 = s[1] * h0, s02 = s[2] * h1;
  const float s11 = s[3] * (h0 * h0), s12 = s[4] * (h0 * h1), s22 = s[5] * (h1 * h1);
  const float c0 = dop(s11, s22, s12, s12);
  const float c1 = dop(s12, s02, s01, s22);
  const float c2 = dop(s01, s12, s11, s02);
  const float p0 = __fmul_rn(s00, c0), r0 = fmaf(s00, c0, -p0);
  const float m1 = __fmul_rn(s01, c1), r1 = fmaf(s01, c1, -m1);
  const float m2 = __fmul_rn(s02, c2), r2 = fmaf(s02, c2, -m2);
  float q1, q2;
  const float p1 = two_sum(p0, m1, q1);
  const float p2 = two_sum(p1, m2, q2);
  const float det = __fadd_rn(p2, __fadd_rn(__fadd_rn(r0, r1), __fadd_rn(__fadd_rn(q1, r2), q2)));
  if (!(det > 0.f)) return false;
  const float inv = 1.0f / det;
  a[0] = c0 * inv;
  a[1] = c1 * inv;
  a[2] = c2 * inv;
  return isfinite(a[0]);
}

}  // namespace fk
