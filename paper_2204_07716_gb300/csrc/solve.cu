// Local-polynomial solves and the type-2 interpolation back to the samples.
//
// Grid stage: at every grid point the s- and t-fields give the normal
// equations S(g) beta = t(g) of eqs. 3 / 11 (S_ab = s_(a+b)).  They are
// assembled in FP64 in the scaled basis u = diag(sigma)^-1 (x_i - g) (which
// leaves the intercept unchanged), solved by Gaussian elimination with
// partial pivoting, and mhat = e_1^T S^-1 t.  Grid points whose density s_0
// is below mask_rho * max s_0 are masked (NaN, mask 0).
//
// Sample stage (type-2 NUFFT): every sorted sample gathers the fields of one
// bandwidth from that bandwidth's fine grid with the spreading kernel,
// solves the same system at q = x_i, and reduces:
//   rss_r      = sum_i (y_ri - mhat_r(x_i))^2           (numerator of eq. 22)
//   wSw_p      = sum_i w_pi (S w_p)_i,  ww_p = sum_i w_pi^2   (Sec. 2.1)
//   tr_exact   = K_H(0) sum_i [S(x_i)^-1]_11             (diagonal of S_h)
// Block partials are summed in a fixed order, so results are deterministic.
#include <cuda_runtime.h>

#include "internal.h"

namespace fk {

namespace {

constexpr int kInterpThreads = 256;
constexpr int kMaxAcc = 512;
constexpr int kMaxW = 24;

template <typename T>
__device__ __forceinline__ T phi(int kind, int w, T beta, T z) {
  if (kind == FKREG_SPREAD_ES) {
    const T t = T(2) * z / T(w);
    const T a = T(1) - t * t;
    return a > T(0) ? exp(beta * (sqrt(a) - T(1))) : T(0);
  }
  return (fabs(z) <= T(0.5) * T(w)) ? exp(-beta * z * z) : T(0);
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

// index of monomial (e_a + e_c) etc. in the s-field table
__device__ __forceinline__ int mono_index(const MonoTab& m, int nm, int e0, int e1, int e2) {
  for (int k = 0; k < nm; ++k)
    if (m.e[k][0] == e0 && m.e[k][1] == e1 && m.e[k][2] == e2) return k;
  return 0;
}

// Assemble the scaled normal matrix from s-fields and return a = S^-1 e_1.
// scale[f] = prod sigma^e (s-field f); t-field a is divided by tscale[a].
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

__device__ __forceinline__ double tscale(const MonoTab& mono, int a, const double* sigma) {
  double sc = 1.0;
  for (int j = 0; j < 3; ++j)
    for (int r = 0; r < mono.e[a][j]; ++r) sc *= sigma[j];
  return sc;
}

template <typename T>
__global__ void smax_kernel(GeoDev g, int64_t Mtot, const T* __restrict__ field, int fgrid,
                            int64_t lcells, T* __restrict__ smax, int bw_count) {
  const int64_t gid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (gid >= Mtot * bw_count) return;
  const int64_t m = gid % Mtot;
  const int bb = int(gid / Mtot);
  int64_t rem = m, lidx = 0, mi[3];
  for (int a = 2; a >= 0; --a) {
    mi[a] = rem % g.M[a];
    rem /= g.M[a];
  }
  for (int a = 0; a < 3; ++a) lidx = lidx * g.L[a] + mi[a];
  T v = field[(int64_t(bb) * fgrid) * lcells + lidx];
  if (!(v > T(0))) return;
  if (sizeof(T) == 4)
    atomicMax(reinterpret_cast<unsigned int*>(smax + bb), __float_as_uint(float(v)));
  else
    atomicMax(reinterpret_cast<unsigned long long*>(smax + bb),
              (unsigned long long)__double_as_longlong(double(v)));
}

struct GridOut {
  void* mhat;         // [n_bw][n_rhs][M] (complex if cplx)
  uint8_t* mask;      // [n_bw][M]
  void* moments;      // [n_bw][ns + n_rhs*nt*(1+cplx)][M]
  int cplx;           // real fields come in (re, im) pairs
  int n_rhs_out;      // responses in the output (pairs collapse when cplx)
};

template <typename T>
__global__ void grid_solve_kernel(GeoDev g, MonoTab mono, const BwDev* __restrict__ bwt,
                                  int bw_first, int bw_count, int order, int64_t Mtot,
                                  const T* __restrict__ field, int fgrid, int64_t lcells,
                                  int nrhs_fields, const T* __restrict__ smax, double rho,
                                  GridOut out) {
  const int64_t gid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (gid >= Mtot * bw_count) return;
  const int64_t m = gid % Mtot;
  const int bb = int(gid / Mtot);
  const int b = bw_first + bb;
  const BwDev& B = bwt[b];
  int64_t rem = m, lidx = 0, mi[3];
  for (int a = 2; a >= 0; --a) {
    mi[a] = rem % g.M[a];
    rem /= g.M[a];
  }
  for (int a = 0; a < 3; ++a) lidx = lidx * g.L[a] + mi[a];
  const T* f0 = field + int64_t(bb) * fgrid * lcells + lidx;
  const int ns = mono.n, nt = mono.nt;
  double s[kMaxMono];
  for (int k = 0; k < ns; ++k) s[k] = double(f0[int64_t(k) * lcells]);
  const int p = nt;
  double a[kMaxP] = {0, 0, 0, 0};
  bool ok = (s[0] > 0.0) && (s[0] >= rho * double(smax[bb]));
  if (ok) {
    if (order == 0)
      a[0] = 1.0 / s[0];
    else
      ok = lpr_weights(mono, p, s, B.sigma, a);
  }
  const T nan = T(__longlong_as_double(0x7ff8000000000000LL));
  const int mult = out.cplx ? 2 : 1;
  for (int q = 0; q < nrhs_fields; ++q) {
    double mh = 0.0;
    const T* tq = f0 + int64_t(ns + q * nt) * lcells;
    for (int k = 0; k < p; ++k) mh += a[k] * double(tq[int64_t(k) * lcells]) / tscale(mono, k, B.sigma);
    if (out.mhat) {
      const int r = q / mult, part = q % mult;
      T* o = static_cast<T*>(out.mhat);
      o[((int64_t(b) * out.n_rhs_out + r) * Mtot + m) * mult + part] = ok ? T(mh) : nan;
    }
  }
  if (out.mask) out.mask[int64_t(b) * Mtot + m] = ok ? 1 : 0;
  if (out.moments) {
    T* o = static_cast<T*>(out.moments);
    const int64_t slice = int64_t(ns + nrhs_fields * nt) * Mtot;
    T* ob = o + int64_t(b) * slice;
    for (int k = 0; k < ns; ++k) ob[int64_t(k) * Mtot + m] = f0[int64_t(k) * lcells];
    for (int q = 0; q < nrhs_fields; ++q) {
      const int r = q / mult, part = q % mult;
      for (int k = 0; k < nt; ++k)
        ob[int64_t(ns) * Mtot + ((int64_t(r) * nt + k) * Mtot + m) * mult + part] =
            f0[int64_t(ns + q * nt + k) * lcells];
    }
  }
}

template <typename T>
__device__ __forceinline__ T inv_h_b(const BwDev& B, int j) {
  return T(B.inv_h[j]);
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Interpolation of all fields of bandwidth b at the sorted samples, with the
// at-sample solve and the reductions.  Grid-stride over samples.
template <typename T, int D>
__global__ void __launch_bounds__(kInterpThreads)
interp_kernel(GeoDev g, MonoTab mono, const BwDev* __restrict__ bwt, int b, int order, int64_t n,
              const T* __restrict__ xs, const T* __restrict__ str, const uint32_t* __restrict__ perm,
              const T* __restrict__ fld, int n_rhs_real, int n_probes, int cplx, int n_rhs_out,
              T* __restrict__ mhat_at_x, int nacc, int nbw, double* __restrict__ part) {
  __shared__ double red[kInterpThreads / 32][kMaxAcc];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int a = lane; a < nacc; a += 32) red[warp][a] = 0.0;
  __syncwarp();
  const BwDev& B = bwt[b];
  int64_t nfb[3] = {B.nf[0], B.nf[1], B.nf[2]};
  const int64_t cells = nfb[0] * nfb[1] * nfb[2];
  const int w = g.w;
  const T beta = T(g.beta);
  const T halfw = T(0.5) * T(w);
  const int ns = mono.n, nt = mono.nt, p = nt;
  const int nq = n_rhs_real + n_probes;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  const int64_t start = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  // loop trip count is warp-uniform so that the shuffles below are safe
  const int64_t base_start = int64_t(blockIdx.x) * blockDim.x + (threadIdx.x & ~31);
  for (int64_t s0 = base_start, s = start; s0 < n; s0 += stride, s += stride) {
    const bool valid = s < n;
    T wt[D][kMaxW];
    int64_t i0[3] = {0, 0, 0};
    if (valid) {
      for (int j = 0; j < D; ++j) {
        const T u = xs[int64_t(j) * n + s] * inv_h_b<T>(B, j);
        const T f0 = ceil(u - halfw);
        i0[j] = int64_t(f0);
        for (int t = 0; t < w; ++t) wt[j][t] = phi<T>(g.skind, w, beta, (f0 + T(t)) - u);
      }
    }
    // gather fields [f_first, f_first + cnt) into v[]
    auto gather = [&](int f_first, int cnt, double* v) {
      T acc[kMaxMono];
      for (int c = 0; c < cnt; ++c) acc[c] = T(0);
      if (valid) {
        const T* G = fld + int64_t(f_first) * cells;
        if (D == 1) {
          for (int t0 = 0; t0 < w; ++t0) {
            int64_t m0 = (i0[0] + t0) % nfb[0];
            if (m0 < 0) m0 += nfb[0];
            for (int c = 0; c < cnt; ++c) acc[c] += G[int64_t(c) * cells + m0] * wt[0][t0];
          }
        } else if (D == 2) {
          for (int t0 = 0; t0 < w; ++t0) {
            int64_t m0 = (i0[0] + t0) % nfb[0];
            if (m0 < 0) m0 += nfb[0];
            T r[kMaxMono];
            for (int c = 0; c < cnt; ++c) r[c] = T(0);
            for (int t1 = 0; t1 < w; ++t1) {
              int64_t m1 = (i0[1] + t1) % nfb[1];
              if (m1 < 0) m1 += nfb[1];
              const int64_t idx = m0 * nfb[1] + m1;
              for (int c = 0; c < cnt; ++c) r[c] += G[int64_t(c) * cells + idx] * wt[D - 1][t1];
            }
            for (int c = 0; c < cnt; ++c) acc[c] += r[c] * wt[0][t0];
          }
        } else {
          for (int t0 = 0; t0 < w; ++t0) {
            int64_t m0 = (i0[0] + t0) % nfb[0];
            if (m0 < 0) m0 += nfb[0];
            for (int t1 = 0; t1 < w; ++t1) {
              int64_t m1 = (i0[1] + t1) % nfb[1];
              if (m1 < 0) m1 += nfb[1];
              const T w01 = wt[0][t0] * wt[1 % D][t1];
              T r[kMaxMono];
              for (int c = 0; c < cnt; ++c) r[c] = T(0);
              for (int t2 = 0; t2 < w; ++t2) {
                int64_t m2 = (i0[2] + t2) % nfb[2];
                if (m2 < 0) m2 += nfb[2];
                const int64_t idx = (m0 * nfb[1] + m1) * nfb[2] + m2;
                for (int c = 0; c < cnt; ++c) r[c] += G[int64_t(c) * cells + idx] * wt[D - 1][t2];
              }
              for (int c = 0; c < cnt; ++c) acc[c] += r[c] * w01;
            }
          }
        }
      }
      for (int c = 0; c < cnt; ++c) v[c] = double(acc[c]);
    };
    double sv[kMaxMono];
    gather(0, ns, sv);
    double a[kMaxP] = {0, 0, 0, 0};
    bool ok = valid;
    if (valid) {
      if (order == 0) {
        a[0] = 1.0 / sv[0];
        ok = sv[0] > 0.0;
      } else {
        ok = lpr_weights(mono, p, sv, B.sigma, a);
      }
      if (!ok) a[0] = a[1] = a[2] = a[3] = 0.0;
    }
    const uint32_t orig = valid ? perm[s] : 0u;
    // exact trace term
    {
      double tv = valid ? B.k0 * a[0] : 0.0;
      tv = warp_sum(tv);
      if (lane == 0) red[warp][nacc - 1] += tv;
    }
    for (int q = 0; q < nq; ++q) {
      double tv[kMaxP];
      gather(ns + q * nt, nt, tv);
      double mh = 0.0;
      for (int k = 0; k < p; ++k) mh += a[k] * tv[k] / tscale(mono, k, B.sigma);
      const double c = valid ? double(str[int64_t(1 + q) * n + s]) : 0.0;
      if (q < n_rhs_real) {
        const double r = valid ? (c - mh) : 0.0;
        double v = warp_sum(r * r);
        if (lane == 0) red[warp][q] += v;
        if (valid && mhat_at_x) {
          const int mult = cplx ? 2 : 1;
          const int rr = q / mult, pt = q % mult;
          mhat_at_x[((int64_t(b) * n_rhs_out + rr) * n + orig) * mult + pt] = T(mh);
        }
      } else {
        const int pp = q - n_rhs_real;
        double v1 = warp_sum(valid ? c * mh : 0.0);
        double v2 = warp_sum(valid ? c * c : 0.0);
        if (lane == 0) {
          red[warp][n_rhs_real + pp] += v1;
          red[warp][n_rhs_real + n_probes + pp] += v2;
        }
      }
    }
  }
  __syncthreads();
  for (int a = threadIdx.x; a < nacc; a += blockDim.x) {
    double t = 0.0;
    for (int wv = 0; wv < kInterpThreads / 32; ++wv) t += red[wv][a];
    part[(int64_t(blockIdx.x) * nbw + b) * nacc + a] = t;
  }
}

// sum block partials in a fixed order: sums[b][a]
__global__ void reduce_partials(const double* __restrict__ part, int64_t nblk, int nbw, int nacc,
                                double* __restrict__ sums) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= nbw * nacc) return;
  double t = 0.0;
  for (int64_t k = 0; k < nblk; ++k) t += part[k * nbw * nacc + gid];
  sums[gid] = t;
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
cudaError_t launch_grid_solve(fkreg_plan_s* P, int bw_first, int bw_count, int nrhs_fields,
                              const fkreg_outputs* out, void* sigma2, cudaStream_t st) {
  const GeoDev& g = P->geo;
  int64_t Mtot = 1, lcells = 1;
  for (int a = 0; a < 3; ++a) {
    Mtot *= g.M[a];
    lcells *= g.L[a];
  }
  const int fgrid = P->ns + nrhs_fields * P->nt;
  T* smax = wsp<T>(P, P->r_smax);
  cudaError_t e = cudaMemsetAsync(smax, 0, sizeof(T) * bw_count, st);
  if (e != cudaSuccess) return e;
  const T* field = wsp<T>(P, P->r_gfield);
  const unsigned blocks = unsigned((Mtot * bw_count + 255) / 256);
  smax_kernel<T><<<blocks, 256, 0, st>>>(g, Mtot, field, fgrid, lcells, smax, bw_count);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  GridOut go{};
  const double rho = P->o.mask_rho > 0 ? P->o.mask_rho : 1e-3;
  if (sigma2) {
    go.mhat = sigma2;
    go.cplx = 0;
    go.n_rhs_out = nrhs_fields;
  } else {
    go.mhat = out ? out->mhat_grid : nullptr;
    go.mask = out ? out->mask : nullptr;
    go.moments = out ? out->moments : nullptr;
    go.cplx = P->o.y_complex;
    go.n_rhs_out = P->nrhs;
  }
  grid_solve_kernel<T><<<blocks, 256, 0, st>>>(g, P->mono, wsp<BwDev>(P, P->r_bw), bw_first,
                                               bw_count, P->order, Mtot, field, fgrid, lcells,
                                               nrhs_fields, smax, rho, go);
  P->launches += 2;
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_interp(fkreg_plan_s* P, int b, int n_rhs_str, int n_probes, void* mhat_at_x,
                          cudaStream_t st) {
  const int n_rhs_real = n_rhs_str;
  const unsigned blocks = unsigned(std::min<int64_t>((P->n + kInterpThreads - 1) / kInterpThreads,
                                                     P->nblk_interp));
  const int nacc = n_rhs_real + 2 * n_probes + 1;
  if (nacc > kMaxAcc) return cudaErrorInvalidValue;
  if (blocks == 0) return cudaSuccess;
#define FK_IK(DD)                                                                                  \
  interp_kernel<T, DD><<<blocks, kInterpThreads, 0, st>>>(                                         \
      P->geo, P->mono, wsp<BwDev>(P, P->r_bw), b, P->order, P->n, wsp<T>(P, P->r_xs),              \
      wsp<T>(P, P->r_str), P->perm_in_vals1 ? wsp<uint32_t>(P, P->r_vals1)                         \
                                            : wsp<uint32_t>(P, P->r_vals0),                        \
      wsp<T>(P, P->r_t2field), n_rhs_real, n_probes, P->o.y_complex, P->nrhs,                      \
      static_cast<T*>(mhat_at_x), nacc, P->nbw, wsp<double>(P, P->r_part))
  if (P->d == 1)
    FK_IK(1);
  else if (P->d == 2)
    FK_IK(2);
  else
    FK_IK(3);
#undef FK_IK
  P->launches += 1;
  return cudaGetLastError();
}

}  // namespace

cudaError_t run_grid_solve(fkreg_plan_s* P, int bw_first, int bw_count, int nrhs_fields,
                           const void*, const fkreg_outputs* out, void* sigma2, cudaStream_t st) {
  return P->prec == FKREG_F32
             ? launch_grid_solve<float>(P, bw_first, bw_count, nrhs_fields, out, sigma2, st)
             : launch_grid_solve<double>(P, bw_first, bw_count, nrhs_fields, out, sigma2, st);
}

cudaError_t run_interp(fkreg_plan_s* P, int b, int n_rhs_str, int n_probes, const void*,
                       void* mhat_at_x, cudaStream_t st) {
  return P->prec == FKREG_F32 ? launch_interp<float>(P, b, n_rhs_str, n_probes, mhat_at_x, st)
                              : launch_interp<double>(P, b, n_rhs_str, n_probes, mhat_at_x, st);
}

// Sum the partials of the last interpolation passes and derive DF and GCV.
cudaError_t run_finalize(fkreg_plan_s* P, int n_probes, const fkreg_outputs* out, cudaStream_t st) {
  const int nacc = P->nrhs_real + 2 * n_probes + 1;
  double* sums = wsp<double>(P, P->r_part) + P->nblk_interp * int64_t(P->nbw) * P->nacc;
  const int64_t nblk = std::min<int64_t>((P->n + kInterpThreads - 1) / kInterpThreads, P->nblk_interp);
  const int tot = P->nbw * nacc;
  reduce_partials<<<(tot + 127) / 128, 128, 0, st>>>(wsp<double>(P, P->r_part), nblk, P->nbw, nacc,
                                                     sums);
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
