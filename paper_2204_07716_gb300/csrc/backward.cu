// Hand-written backward of GCV (eq. 22) with respect to log h, y and x.
//
// With the Monte-Carlo trace of Sec. 2.1 (fixed probes w_p),
//   GCV = (RSS / N) / (1 - tr / N)^2,  RSS = sum_i (y_i - mhat_y(x_i))^2,
//   tr  = (N / Np) sum_p sum_i w_pi mhat_p(x_i) / (w_p^T w_p),
// and mhat_r(x_i) = e_1^T S(x_i)^-1 t_r(x_i) (eq. 3).  Every field value at a
// sample, Q_(i,f) = sum_j c_(f,j) w_f(x_j - x_i) with w_f(z) = z^g_f K_H(z), gets
// an adjoint Qbar_(i,f) = dGCV / dQ_(i,f):
//   t-fields of response r : g_(r,i) a_i             (a = S^-1 e_1)
//   s-field g              : -sum_(a+b=g) a_a bbar_b  (bbar = sum_r g_r S^-1 t_r)
// with g_y = -2 L_RSS (y_i - mhat_y), g_p = L_tr (N / Np) w_pi / (w_p^T w_p).
// Then
//   d/dlog sigma_j = sum_i Qbar_i . dQ_i/dlog sigma_j      (derivative fields at x_i)
//   d/dx_i (target) = sum_f Qbar_(i,f) grad_q Q_f(x_i)      (gradient fields at x_i)
//   d/dx_j (source) = sum_c c_(c,j) sum_(f in c) sum_i Qbar_(i,f) grad w_f(x_j - x_i)
//   d/dy_j          = 2 L_RSS (y_j - mhat_y(x_j)) + sum_(f in y) sum_i Qbar_(i,f) w_f(x_j - x_i)
// The last two are NUFFT convolutions of the adjoints spread as strengths.
// Field values at the samples come from the interpolation kernels' gather-only
// mode (same bin-window staging as the forward pass).
#include <cuda_runtime.h>

#include <algorithm>

#include "device_common.cuh"
#include "internal.h"

namespace fk {

namespace {

constexpr int kE1Threads = 256;

// Loss scalars for bandwidth b from the forward sums:
//   sc[0] = L_RSS = (1/N) / (1 - tr/N)^2
//   sc[1] = L_tr * N / Np,  L_tr = 2 (RSS/N) / (N (1 - tr/N)^3)
//   sc[2] = GCV
__global__ void loss_scalars_kernel(const double* __restrict__ sums, int b, int nacc, int n_probes,
                                    int64_t n, double* __restrict__ sc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double* sb = sums + int64_t(b) * nacc;
  double girard = 0.0;
  for (int p = 0; p < n_probes; ++p) girard += sb[1 + p] / sb[1 + n_probes + p];
  const double N = double(n);
  const double tr = N * girard / n_probes;
  const double rss = sb[0];
  const double den = 1.0 - tr / N;
  sc[0] = (1.0 / N) / (den * den);
  sc[1] = (2.0 * (rss / N) / (N * den * den * den)) * (N / n_probes);
  sc[2] = (rss / N) / (den * den);
}

// Per-sample adjoints.  V holds (1 + 2D) blocks of F2 fields: values, the D
// gradient fields and the D bandwidth-derivative fields.  Writes Qbar (as
// spreading strengths), the target-side x-gradient and the explicit y-term,
// and per-block partial sums of the bandwidth gradient.
template <typename T, int D>
__global__ void __launch_bounds__(kE1Threads)
adjoint_kernel(MonoTab mono, const BwDev* __restrict__ bwt, int b, int order, int64_t n, int F2,
               int n_probes, const T* __restrict__ V, const T* __restrict__ str,
               const double* __restrict__ sums, int nacc, const double* __restrict__ sc,
               T* __restrict__ qbar, T* __restrict__ dxt, T* __restrict__ dye,
               double* __restrict__ part) {
  __shared__ double red[kE1Threads / 32][3];
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool valid = s < n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const BwDev& B = bwt[b];
  const int ns = mono.n, nt = mono.nt, p = nt;
  double dth[3] = {0, 0, 0};
  if (valid) {
    const double* sb = sums + int64_t(b) * nacc;
    const double L_rss = sc[0], L_trn = sc[1];
    // scaled normal matrix and its inverse (FP64)
    double sv[kMaxMono];
#pragma unroll
    for (int k = 0; k < kMaxMono; ++k) sv[k] = k < ns ? double(V[int64_t(k) * n + s]) : 0.0;
    double Sinv[kMaxP][kMaxP];
    double tsc[kMaxP];
#pragma unroll
    for (int k = 0; k < kMaxP; ++k) tsc[k] = k < p ? 1.0 / tscale(mono, k, B.sigma) : 0.0;
    bool ok = true;
    if (order == 0) {
      ok = sv[0] > 0.0;
      Sinv[0][0] = ok ? 1.0 / sv[0] : 0.0;
    } else {
      // columns of the scaled inverse by elimination, then unscale
      for (int c = 0; c < p && ok; ++c) {
        double S[kMaxP][kMaxP], col[kMaxP];
        for (int i = 0; i < p; ++i)
          for (int j = 0; j < p; ++j) {
            const int e0 = mono.e[i][0] + mono.e[j][0], e1 = mono.e[i][1] + mono.e[j][1],
                      e2 = mono.e[i][2] + mono.e[j][2];
            S[i][j] = sv[mono_index(mono, ns, e0, e1, e2)] * tsc[i] * tsc[j];
          }
        // solve S col = e_c
        double rhs[kMaxP];
        for (int i = 0; i < p; ++i) rhs[i] = (i == c) ? 1.0 : 0.0;
        for (int cc = 0; cc < p && ok; ++cc) {
          int piv = cc;
          for (int i = cc + 1; i < p; ++i)
            if (fabs(S[i][cc]) > fabs(S[piv][cc])) piv = i;
          if (!(fabs(S[piv][cc]) > 0.0)) {
            ok = false;
            break;
          }
          if (piv != cc) {
            for (int j = 0; j < p; ++j) {
              const double t = S[cc][j];
              S[cc][j] = S[piv][j];
              S[piv][j] = t;
            }
            const double t = rhs[cc];
            rhs[cc] = rhs[piv];
            rhs[piv] = t;
          }
          for (int i = cc + 1; i < p; ++i) {
            const double fct = S[i][cc] / S[cc][cc];
            for (int j = cc; j < p; ++j) S[i][j] -= fct * S[cc][j];
            rhs[i] -= fct * rhs[cc];
          }
        }
        if (!ok) break;
        for (int i = p - 1; i >= 0; --i) {
          double v = rhs[i];
          for (int j = i + 1; j < p; ++j) v -= S[i][j] * col[j];
          col[i] = v / S[i][i];
        }
        for (int i = 0; i < p; ++i) Sinv[i][c] = col[i] * tsc[i] * tsc[c];
      }
    }
    double a[kMaxP] = {0, 0, 0, 0}, bbar[kMaxP] = {0, 0, 0, 0};
    if (ok)
      for (int i = 0; i < p; ++i) a[i] = Sinv[i][0];
    double dx_t[3] = {0, 0, 0};
    const int R = 1 + n_probes;
    const int nblk = 1 + 2 * D;
    for (int r = 0; r < R && ok; ++r) {
      double t[kMaxP];
      for (int k = 0; k < p; ++k) t[k] = double(V[int64_t(ns + r * nt + k) * n + s]);
      double mh = 0.0;
      for (int k = 0; k < p; ++k) mh += a[k] * t[k];
      const double c = double(str[int64_t(1 + r) * n + s]);
      double gr;
      if (r == 0) {
        gr = -2.0 * L_rss * (c - mh);
        dye[s] = T(2.0 * L_rss * (c - mh));
      } else {
        const int pp = r - 1;
        gr = L_trn * c / sb[1 + n_probes + pp];
      }
      for (int i = 0; i < p; ++i) {
        double beta = 0.0;
        for (int k = 0; k < p; ++k) beta += Sinv[i][k] * t[k];
        bbar[i] += gr * beta;
      }
      for (int k = 0; k < p; ++k) {
        const int f = ns + r * nt + k;
        const double q = gr * a[k];
        qbar[int64_t(f) * n + s] = T(q);
        for (int d = 0; d < D; ++d) dx_t[d] += q * double(V[(int64_t(1 + d) * F2 + f) * n + s]);
        for (int d = 0; d < D; ++d) dth[d] += q * double(V[(int64_t(1 + D + d) * F2 + f) * n + s]);
      }
    }
    // s-field adjoints: -sum_(a+b=g) a_a bbar_b over ordered pairs
    for (int gf = 0; gf < ns; ++gf) {
      double q = 0.0;
      if (ok)
        for (int i = 0; i < p; ++i)
          for (int j = 0; j < p; ++j)
            if (mono.e[i][0] + mono.e[j][0] == mono.e[gf][0] &&
                mono.e[i][1] + mono.e[j][1] == mono.e[gf][1] &&
                mono.e[i][2] + mono.e[j][2] == mono.e[gf][2])
              q -= a[i] * bbar[j];
      qbar[int64_t(gf) * n + s] = T(q);
      for (int d = 0; d < D; ++d) dx_t[d] += q * double(V[(int64_t(1 + d) * F2 + gf) * n + s]);
      for (int d = 0; d < D; ++d) dth[d] += q * double(V[(int64_t(1 + D + d) * F2 + gf) * n + s]);
    }
    if (!ok) {
      for (int f = 0; f < F2; ++f) qbar[int64_t(f) * n + s] = T(0);
      dye[s] = T(0);
    }
    for (int d = 0; d < D; ++d) dxt[int64_t(d) * n + s] = T(dx_t[d]);
    (void)nblk;
  }
  for (int d = 0; d < 3; ++d) {
    double v = dth[d];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][d] = v;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int wv = 0; wv < kE1Threads / 32; ++wv) t += red[wv][threadIdx.x];
    part[int64_t(blockIdx.x) * 3 + threadIdx.x] = t;
  }
}

// Index of the s-field of the monomial product z^(e_i + e_j) for the
// local-linear unknowns i, j (0 = intercept, k >= 1 = z_(k-1)) in the graded
// order of the s-fields (1, z_1..z_D, then z_u z_v, u <= v, lexicographic).
template <int D>
__host__ __device__ constexpr int sidx(int i, int j) {
  return i == 0 ? j
                : (j == 0 ? i
                          : 1 + D + (i <= j ? (i - 1) * D - (i - 1) * (i - 2) / 2 + (j - i)
                                            : (j - 1) * D - (j - 1) * (j - 2) / 2 + (i - j)));
}

// Inverse of the scaled normal matrix (p <= 3) in FP32: cofactors by Kahan's
// difference of products, the determinant by a compensated dot product
// (the same arithmetic as the at-sample solve).  Returns false if singular.
template <int P>
__device__ __forceinline__ bool sym_inverse_f32(const float (&m)[P][P], float (&inv)[P][P]) {
  if (P == 1) {
    inv[0][0] = 1.0f / m[0][0];
    return m[0][0] > 0.f;
  } else if (P == 2) {
    const float det = dop(m[0][0], m[1][1], m[0][1], m[0][1]);
    if (!(det > 0.f)) return false;
    const float r = 1.0f / det;
    inv[0][0] = m[1][1] * r;
    inv[1][1] = m[0][0] * r;
    inv[0][1] = inv[1][0] = -m[0][1] * r;
    return isfinite(inv[0][0]);
  } else {
    const float c00 = dop(m[1][1], m[2][2], m[1][2], m[1][2]);
    const float c01 = dop(m[1][2], m[0][2], m[0][1], m[2][2]);
    const float c02 = dop(m[0][1], m[1][2], m[1][1], m[0][2]);
    const float c11 = dop(m[0][0], m[2][2], m[0][2], m[0][2]);
    const float c12 = dop(m[0][1], m[0][2], m[0][0], m[1][2]);
    const float c22 = dop(m[0][0], m[1][1], m[0][1], m[0][1]);
    const float p0 = __fmul_rn(m[0][0], c00), r0 = fmaf(m[0][0], c00, -p0);
    const float m1 = __fmul_rn(m[0][1], c01), r1 = fmaf(m[0][1], c01, -m1);
    const float m2 = __fmul_rn(m[0][2], c02), r2 = fmaf(m[0][2], c02, -m2);
    float q1, q2;
    const float p1 = two_sum(p0, m1, q1);
    const float p2 = two_sum(p1, m2, q2);
    const float det = __fadd_rn(p2, __fadd_rn(__fadd_rn(r0, r1), __fadd_rn(__fadd_rn(q1, r2), q2)));
    if (!(det > 0.f)) return false;
    const float r = 1.0f / det;
    inv[0][0] = c00 * r;
    inv[1][1] = c11 * r;
    inv[2][2] = c22 * r;
    inv[0][1] = inv[1][0] = c01 * r;
    inv[0][2] = inv[2][0] = c02 * r;
    inv[1][2] = inv[2][1] = c12 * r;
    return isfinite(inv[0][0]);
  }
}

// FP32 form of adjoint_kernel for 1-D / 2-D systems known at compile time
// (NW: p = 1; local linear: p = D + 1).  Same quantities; FP32 per sample
// (the FP64 pipe is a small fraction of the FP32 rate on this part), FP64
// for the block sums of the bandwidth gradient.
template <int D, int ORD>
__global__ void __launch_bounds__(kE1Threads)
adjoint_f32_kernel(const BwDev* __restrict__ bwt, int b, int64_t n, int F2, int n_probes,
                   const float* __restrict__ V, const float* __restrict__ str,
                   const double* __restrict__ sums, int nacc, const double* __restrict__ sc,
                   float* __restrict__ qbar, float* __restrict__ dxt, float* __restrict__ dye,
                   double* __restrict__ part) {
  constexpr int P = ORD == 0 ? 1 : D + 1;
  constexpr int NS = ORD == 0 ? 1 : (D + 1) * (D + 2) / 2;
  __shared__ double red[kE1Threads / 32][3];
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool valid = s < n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const BwDev& B = bwt[b];
  float dth[3] = {0.f, 0.f, 0.f};
  if (valid) {
    const double* sb = sums + int64_t(b) * nacc;
    const float L_rss = float(sc[0]), L_trn = float(sc[1]);
    float dsc[P];
    dsc[0] = 1.f;
#pragma unroll
    for (int k = 1; k < P; ++k) dsc[k] = float(1.0 / B.sigma[k - 1]);
    float sv[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) sv[k] = V[int64_t(k) * n + s];
    float m[P][P], mi[P][P];
#pragma unroll
    for (int i = 0; i < P; ++i)
#pragma unroll
      for (int j = 0; j < P; ++j) m[i][j] = sv[sidx<D>(i, j)] * (dsc[i] * dsc[j]);
    const bool ok = sym_inverse_f32<P>(m, mi);
    float Sinv[P][P];
#pragma unroll
    for (int i = 0; i < P; ++i)
#pragma unroll
      for (int j = 0; j < P; ++j) Sinv[i][j] = ok ? mi[i][j] * (dsc[i] * dsc[j]) : 0.f;
    float a[P], bbar[P];
#pragma unroll
    for (int i = 0; i < P; ++i) {
      a[i] = Sinv[i][0];
      bbar[i] = 0.f;
    }
    float dx_t[3] = {0.f, 0.f, 0.f};
    const int R = 1 + n_probes;
#pragma unroll 2
    for (int r = 0; r < R; ++r) {
      float t[P];
#pragma unroll
      for (int k = 0; k < P; ++k) t[k] = V[int64_t(NS + r * P + k) * n + s];
      float mh = 0.f;
#pragma unroll
      for (int k = 0; k < P; ++k) mh += a[k] * t[k];
      const float c = str[int64_t(1 + r) * n + s];
      float gr;
      if (r == 0) {
        gr = -2.f * L_rss * (c - mh);
        dye[s] = ok ? 2.f * L_rss * (c - mh) : 0.f;
      } else {
        gr = L_trn * c / float(sb[1 + n_probes + (r - 1)]);
      }
      if (!ok) gr = 0.f;
#pragma unroll
      for (int i = 0; i < P; ++i) {
        float beta = 0.f;
#pragma unroll
        for (int k = 0; k < P; ++k) beta += Sinv[i][k] * t[k];
        bbar[i] += gr * beta;
      }
#pragma unroll
      for (int k = 0; k < P; ++k) {
        const int f = NS + r * P + k;
        const float q = gr * a[k];
        qbar[int64_t(f) * n + s] = q;
#pragma unroll
        for (int d = 0; d < D; ++d) {
          dx_t[d] += q * V[(int64_t(1 + d) * F2 + f) * n + s];
          dth[d] += q * V[(int64_t(1 + D + d) * F2 + f) * n + s];
        }
      }
    }
    // s-field adjoints: -sum_(a+b=g) a_a bbar_b over ordered pairs
    float qs[NS];
#pragma unroll
    for (int g = 0; g < NS; ++g) qs[g] = 0.f;
#pragma unroll
    for (int i = 0; i < P; ++i)
#pragma unroll
      for (int j = 0; j < P; ++j) qs[sidx<D>(i, j)] -= a[i] * bbar[j];
#pragma unroll
    for (int g = 0; g < NS; ++g) {
      qbar[int64_t(g) * n + s] = qs[g];
#pragma unroll
      for (int d = 0; d < D; ++d) {
        dx_t[d] += qs[g] * V[(int64_t(1 + d) * F2 + g) * n + s];
        dth[d] += qs[g] * V[(int64_t(1 + D + d) * F2 + g) * n + s];
      }
    }
#pragma unroll
    for (int d = 0; d < D; ++d) dxt[int64_t(d) * n + s] = dx_t[d];
  }
  for (int d = 0; d < 3; ++d) {
    double v = double(dth[d]);
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][d] = v;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int wv = 0; wv < kE1Threads / 32; ++wv) t += red[wv][threadIdx.x];
    part[int64_t(blockIdx.x) * 3 + threadIdx.x] = t;
  }
}

// Combine: dy_i = adjoint y-field + explicit term; dx_(i,d) = sum over
// strength classes c of c_(c,i) * adjoint field (c, d) + target-side term.
// Outputs in the original sample order.
template <typename T, int D>
__global__ void combine_kernel(int64_t n, int n_probes, const T* __restrict__ Vadj,
                               const T* __restrict__ str, const T* __restrict__ dxt,
                               const T* __restrict__ dye, const uint32_t* __restrict__ perm,
                               T* __restrict__ dy, T* __restrict__ dx) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const uint32_t i = perm[s];
  if (dy) dy[i] = Vadj[s] + dye[s];
  if (dx) {
    const int ncls = 2 + n_probes;
    for (int d = 0; d < D; ++d) {
      if constexpr (sizeof(T) == 4) {
        // compensated FP32 (exact products by fma, two-sum of the running
        // total): FP64 arithmetic runs on GB300's narrow FP64 pipe
        float hi = dxt[int64_t(d) * n + s], lo = 0.f;
        for (int c = 0; c < ncls; ++c) {
          const float cc = c == 0 ? 1.f : float(str[int64_t(c) * n + s]);
          const float v = float(Vadj[int64_t(1 + c * D + d) * n + s]);
          const float p = cc * v;
          const float pe = fmaf(cc, v, -p);
          const float t = hi + p;
          const float z = t - hi;
          lo += ((hi - (t - z)) + (p - z)) + pe;
          hi = t;
        }
        dx[int64_t(i) * D + d] = T(hi + lo);
      } else {
        double v = double(dxt[int64_t(d) * n + s]);
        for (int c = 0; c < ncls; ++c) {
          const double cc = c == 0 ? 1.0 : double(str[int64_t(c) * n + s]);
          v += cc * double(Vadj[int64_t(1 + c * D + d) * n + s]);
        }
        dx[int64_t(i) * D + d] = T(v);
      }
    }
  }
}

__global__ void reduce_theta(const double* __restrict__ part, int64_t nblk, int D,
                             double* __restrict__ out) {
  __shared__ double sh[256];
  const int d = blockIdx.x;
  double t = 0.0;
  for (int64_t k = threadIdx.x; k < nblk; k += blockDim.x) t += part[k * 3 + d];
  sh[threadIdx.x] = t;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[d] = sh[0];
}

}  // namespace

cudaError_t run_loss_scalars(fkreg_plan_s* P, int b, int n_probes, cudaStream_t st) {
  const int nacc = P->nrhs_real + 2 * n_probes + 1;
  const double* sums = wsp<double>(P, P->r_part) + P->nblk_interp * int64_t(P->nbw) * P->nacc;
  loss_scalars_kernel<<<1, 32, 0, st>>>(sums, b, nacc, n_probes, P->n, wsp<double>(P, P->r_bsc));
  P->launches += 1;
  return cudaGetLastError();
}

template <typename T>
static cudaError_t adjoint_t(fkreg_plan_s* P, int b, int n_probes, cudaStream_t st) {
  if (P->n == 0) return cudaSuccess;
  const int nacc = P->nrhs_real + 2 * n_probes + 1;
  const double* sums = wsp<double>(P, P->r_part) + P->nblk_interp * int64_t(P->nbw) * P->nacc;
  const int F2 = P->ns + (1 + n_probes) * P->nt;
  const unsigned blocks = unsigned((P->n + kE1Threads - 1) / kE1Threads);
  T* qbar = wsp<T>(P, P->r_str) + int64_t(P->smax) * P->n;
  T* dxt = wsp<T>(P, P->r_bdx);
  T* dye = dxt + int64_t(P->d) * P->n;
  if constexpr (sizeof(T) == 4) {
    if (P->d <= 2 || P->order == 0) {
#define FK_F(DD, OO)                                                                            \
  adjoint_f32_kernel<DD, OO><<<blocks, kE1Threads, 0, st>>>(                                    \
      wsp<BwDev>(P, P->r_bw), b, P->n, F2, n_probes, wsp<float>(P, P->r_bV),                   \
      wsp<float>(P, P->r_str), sums, nacc, wsp<double>(P, P->r_bsc), qbar, dxt, dye,           \
      wsp<double>(P, P->r_bpart))
      if (P->order == 0) {
        if (P->d == 1) FK_F(1, 0);
        else if (P->d == 2) FK_F(2, 0);
        else FK_F(3, 0);
      } else {
        if (P->d == 1) FK_F(1, 1);
        else FK_F(2, 1);
      }
#undef FK_F
      P->launches += 1;
      return cudaGetLastError();
    }
  }
#define FK_A(DD)                                                                              \
  adjoint_kernel<T, DD><<<blocks, kE1Threads, 0, st>>>(                                       \
      P->mono, wsp<BwDev>(P, P->r_bw), b, P->order, P->n, F2, n_probes, wsp<T>(P, P->r_bV),  \
      wsp<T>(P, P->r_str), sums, nacc, wsp<double>(P, P->r_bsc), qbar, dxt, dye,             \
      wsp<double>(P, P->r_bpart))
  if (P->d == 1)
    FK_A(1);
  else if (P->d == 2)
    FK_A(2);
  else
    FK_A(3);
#undef FK_A
  P->launches += 1;
  return cudaGetLastError();
}

cudaError_t run_adjoint(fkreg_plan_s* P, int b, int n_probes, cudaStream_t st) {
  return P->prec == FKREG_F32 ? adjoint_t<float>(P, b, n_probes, st)
                              : adjoint_t<double>(P, b, n_probes, st);
}

template <typename T>
static cudaError_t combine_t(fkreg_plan_s* P, int n_probes, void* dy, void* dx, double* dlogh,
                             cudaStream_t st) {
  if (P->n > 0) {
    const unsigned blocks = unsigned((P->n + 255) / 256);
    const T* dxt = wsp<T>(P, P->r_bdx);
    const T* dye = dxt + int64_t(P->d) * P->n;
#define FK_C(DD)                                                                                 \
  combine_kernel<T, DD><<<blocks, 256, 0, st>>>(P->n, n_probes, wsp<T>(P, P->r_bV),              \
                                                wsp<T>(P, P->r_str), dxt, dye, perm_ptr(P),      \
                                                static_cast<T*>(dy), static_cast<T*>(dx))
    if (P->d == 1)
      FK_C(1);
    else if (P->d == 2)
      FK_C(2);
    else
      FK_C(3);
#undef FK_C
    P->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (dlogh) {
    const int64_t nblk = (P->n + kE1Threads - 1) / kE1Threads;
    reduce_theta<<<P->d, 256, 0, st>>>(wsp<double>(P, P->r_bpart), nblk, P->d, dlogh);
    P->launches += 1;
  }
  return cudaGetLastError();
}

cudaError_t run_combine(fkreg_plan_s* P, int n_probes, void* dy, void* dx, double* dlogh,
                        cudaStream_t st) {
  return P->prec == FKREG_F32 ? combine_t<float>(P, n_probes, dy, dx, dlogh, st)
                              : combine_t<double>(P, n_probes, dy, dx, dlogh, st);
}

}  // namespace fk
