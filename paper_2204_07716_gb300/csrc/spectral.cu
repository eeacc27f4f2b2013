// Fourier-domain kernel multiply with deconvolution (Sec. 1.1 "convolution
// ... in the frequency domain", eq. 20 deconvolution).
//
// After the forward FFT of the fine grid, B_k ~ phihat(k) F_k with
// F_k = sum_i c_i exp(-2 pi i k (x_i - lo) / P).  A moment field
// T_g(q) = sum_i c_i K_H(x_i - q) (x_i - q)^g is the correlation of the point
// measure with w_g(z) = z^g K_H(z), so on the period P
//   T_g(lo + m delta) = sum_k A_g[k] exp(2 pi i k m / L),
//   A_g[k] = F_k W_g(k/P) / prod_j P_j,
//   W_g(xi) = integral w_g(z) exp(+2 pi i xi.z) dz:
//     g = 0        : G(xi) = exp(-2 pi^2 xi^T H xi)
//     g = e_a      : 2 pi i (H xi)_a G(xi)
//     g = e_a + e_c: (H_ac - 4 pi^2 (H xi)_a (H xi)_c) G(xi)
// (the transforms of the Gaussian and its first two moments).
// Grid stage: A is folded modulo L onto the half spectrum of a length-L
// real inverse DFT (exact aliasing when the kept modes exceed L).
// Type-2 stage: A / phihat_b is placed on the per-bandwidth fine grid
// (zero elsewhere) for the interpolation back to the samples.
#include <cuda_runtime.h>

#include "internal.h"

namespace fk {

namespace {

template <typename T>
struct Cx;
template <>
struct Cx<float> {
  using type = float2;
};
template <>
struct Cx<double> {
  using type = double2;
};

template <typename C, typename T>
__device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}

// F_q at signed mode kk from the R2C half spectrum of the type-1 fine grid.
template <typename T, typename C>
__device__ __forceinline__ C fetch_F(const GeoDev& g, const C* __restrict__ F, const int64_t kk[3],
                                     int D) {
  const int64_t last = kk[D - 1];
  const bool neg = last < 0;
  int64_t idx = 0;
  for (int a = 0; a < D; ++a) {
    int64_t k = neg ? -kk[a] : kk[a];
    int64_t n = (a == D - 1) ? (g.nf[a] / 2 + 1) : g.nf[a];
    if (a < D - 1) {
      k %= g.nf[a];
      if (k < 0) k += g.nf[a];
    }
    idx = idx * n + k;
  }
  C v = F[idx];
  if (neg) v.y = -v.y;
  return v;
}

// multiplier data for one mode and bandwidth
template <typename T>
struct ModeMul {
  T G;
  T hx[3];
};

template <typename T>
__device__ __forceinline__ ModeMul<T> mode_mul(const GeoDev& g, const BwDev& B, const int64_t kk[3],
                                               int D) {
  ModeMul<T> m;
  T xi[3] = {T(0), T(0), T(0)};
  for (int a = 0; a < D; ++a) xi[a] = T(kk[a]) / T(g.P[a]);
  T q = T(0);
  for (int a = 0; a < 3; ++a) {
    T s = T(0);
    for (int c = 0; c < D; ++c) s += T(B.H[a * 3 + c]) * xi[c];
    m.hx[a] = (a < D) ? s : T(0);
    q += xi[a] * m.hx[a];
  }
  const T twopi = T(6.283185307179586476925286766559);
  m.G = exp(-T(0.5) * twopi * twopi * q);
  return m;
}

// Transform of z^g K_H for |g| <= 4: W_g = (2 pi i)^-|g| d^g G / dxi^g, and
// the derivatives of a Gaussian sum over the ways to split the index list of
// g into pairs (each -4 pi^2 H_ab) and singletons (each u_a = -4 pi^2 (H xi)_a)
// (Isserlis' rule).  Returns c with W_g = c G (real, |g| even) or
// W_g = i c G (|g| odd, *imag = true).
template <typename T>
__device__ __forceinline__ T moment_factor(const MonoTab& mono, int f, const ModeMul<T>& m,
                                           const BwDev& B, bool* imag) {
  const T twopi = T(6.283185307179586476925286766559);
  const T fpi2 = twopi * twopi;  // 4 pi^2
  int id[4] = {0, 0, 0, 0}, k = 0;
  for (int j = 0; j < 3; ++j)
    for (int r = 0; r < mono.e[f][j]; ++r) id[k++] = j;
  T u[4], P[4][4];
  for (int x = 0; x < k; ++x) {
    u[x] = -fpi2 * m.hx[id[x]];
    for (int y = 0; y < k; ++y) P[x][y] = -fpi2 * T(B.H[id[x] * 3 + id[y]]);
  }
  T poly;
  if (k == 0) {
    poly = T(1);
  } else if (k == 1) {
    poly = u[0];
  } else if (k == 2) {
    poly = u[0] * u[1] + P[0][1];
  } else if (k == 3) {
    poly = u[0] * u[1] * u[2] + P[0][1] * u[2] + P[0][2] * u[1] + P[1][2] * u[0];
  } else {
    poly = u[0] * u[1] * u[2] * u[3] + P[0][1] * u[2] * u[3] + P[0][2] * u[1] * u[3] +
           P[0][3] * u[1] * u[2] + P[1][2] * u[0] * u[3] + P[1][3] * u[0] * u[2] +
           P[2][3] * u[0] * u[1] + P[0][1] * P[2][3] + P[0][2] * P[1][3] + P[0][3] * P[1][2];
  }
  // (2 pi i)^-k: k = 1: -i/(2 pi); 2: -1/(4 pi^2); 3: i/(8 pi^3); 4: 1/(16 pi^4)
  const T ip = T(1) / twopi;
  *imag = (k & 1) != 0;
  switch (k) {
    case 0: return poly;
    case 1: return -ip * poly;
    case 2: return -ip * ip * poly;
    case 3: return ip * ip * ip * poly;
    default: return ip * ip * ip * ip * poly;
  }
}

// accumulate base * W_g for the first nf monomials
template <typename T, typename C>
__device__ __forceinline__ void acc_fields(C* acc, C base, const ModeMul<T>& m, const BwDev& B,
                                           const MonoTab& mono, int nfields) {
  const T twopi = T(6.283185307179586476925286766559);
  for (int f = 0; f < nfields; ++f) {
    int deg = mono.e[f][0] + mono.e[f][1] + mono.e[f][2];
    if (deg == 0) {
      acc[f].x += base.x;
      acc[f].y += base.y;
    } else if (deg == 1) {
      int a = mono.e[f][0] ? 0 : (mono.e[f][1] ? 1 : 2);
      const T s = twopi * m.hx[a];  // multiply by i * s
      acc[f].x += -base.y * s;
      acc[f].y += base.x * s;
    } else if (deg == 2) {
      int a = -1, c = -1;
      for (int j = 0; j < 3; ++j)
        for (int r = 0; r < mono.e[f][j]; ++r) {
          if (a < 0)
            a = j;
          else
            c = j;
        }
      const T s = T(B.H[a * 3 + c]) - twopi * twopi * m.hx[a] * m.hx[c];
      acc[f].x += base.x * s;
      acc[f].y += base.y * s;
    } else {
      bool imag;
      const T s = moment_factor<T>(mono, f, m, B, &imag);
      if (imag) {
        acc[f].x += -base.y * s;
        acc[f].y += base.x * s;
      } else {
        acc[f].x += base.x * s;
        acc[f].y += base.y * s;
      }
    }
  }
}

// Grid stage: thread per (half-spectrum index j on the L grid, bandwidth, strength q).
template <typename T, int D>
__global__ void kmul_grid_kernel(GeoDev g, const BwDev* __restrict__ bwt,
                                 const double* __restrict__ tab, int64_t phi1_0, int64_t phi1_1,
                                 int64_t phi1_2, MonoTab mono, const typename Cx<T>::type* __restrict__ F,
                                 int64_t fine_half, int str_dens, int str_rhs, int nrhs_fields,
                                 int bw_first, int bw_count, int fgrid, int64_t lhalf,
                                 typename Cx<T>::type* __restrict__ out) {
  using C = typename Cx<T>::type;
  const int nq = (str_dens >= 0 ? 1 : 0) + nrhs_fields;
  const int64_t gid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t total = lhalf * bw_count * nq;
  if (gid >= total) return;
  const int64_t j = gid % lhalf;
  const int q = int((gid / lhalf) % nq);
  const int bb = int(gid / (lhalf * nq));
  const BwDev& B = bwt[bw_first + bb];
  const bool dens = (str_dens >= 0) && q == 0;
  const int strength = dens ? str_dens : str_rhs + (q - (str_dens >= 0 ? 1 : 0));
  const int nfld = dens ? mono.n : mono.nt;
  const int fbase = dens ? 0 : ((str_dens >= 0 ? mono.n : 0) + (q - (str_dens >= 0 ? 1 : 0)) * mono.nt);
  const C* Fq = F + int64_t(strength) * fine_half;
  // output multi-index
  int64_t jj[3] = {0, 0, 0};
  {
    int64_t rem = j;
    for (int a = D - 1; a >= 0; --a) {
      const int64_t n = (a == D - 1) ? (g.L[a] / 2 + 1) : g.L[a];
      jj[a] = rem % n;
      rem /= n;
    }
  }
  // alias ranges
  int64_t k0[3], cnt[3];
  for (int a = 0; a < D; ++a) {
    const int64_t hk = B.K[a] / 2 - 1;
    const int64_t lo = -hk;
    int64_t r = (jj[a] - lo) % g.L[a];
    if (r < 0) r += g.L[a];
    k0[a] = lo + r;
    cnt[a] = (k0[a] > hk) ? 0 : ((hk - k0[a]) / g.L[a] + 1);
  }
  C acc[kMaxMono];
  for (int f = 0; f < kMaxMono; ++f) acc[f] = C{T(0), T(0)};
  const int64_t phi1[3] = {phi1_0, phi1_1, phi1_2};
  T invP = T(1);
  for (int a = 0; a < D; ++a) invP /= T(g.P[a]);
  const int64_t c1 = (D > 1) ? cnt[1] : 1, c2 = (D > 2) ? cnt[2] : 1;
  for (int64_t i0 = 0; i0 < cnt[0]; ++i0)
    for (int64_t i1 = 0; i1 < c1; ++i1)
      for (int64_t i2 = 0; i2 < c2; ++i2) {
        int64_t kk[3] = {k0[0] + i0 * g.L[0], 0, 0};
        if (D > 1) kk[1] = k0[1] + i1 * g.L[1];
        if (D > 2) kk[2] = k0[2] + i2 * g.L[2];
        T dec = invP;
        for (int a = 0; a < D; ++a) dec *= T(tab[phi1[a] + (kk[a] < 0 ? -kk[a] : kk[a])]);
        const ModeMul<T> m = mode_mul<T>(g, B, kk, D);
        C base = fetch_F<T, C>(g, Fq, kk, D);
        const T s = dec * m.G;
        base.x *= s;
        base.y *= s;
        acc_fields<T, C>(acc, base, m, B, mono, nfld);
      }
  for (int f = 0; f < nfld; ++f) out[(int64_t(bb) * fgrid + fbase + f) * lhalf + j] = acc[f];
}

// base * W_f for monomial f (one field of acc_fields)
template <typename T, typename C>
__device__ __forceinline__ C mult_field(C base, const ModeMul<T>& m, const BwDev& B,
                                        const MonoTab& mono, int f) {
  const T twopi = T(6.283185307179586476925286766559);
  const int deg = mono.e[f][0] + mono.e[f][1] + mono.e[f][2];
  C r;
  if (deg == 0) {
    r = base;
  } else if (deg == 1) {
    const int a = mono.e[f][0] ? 0 : (mono.e[f][1] ? 1 : 2);
    const T sc = twopi * m.hx[a];  // multiply by i * sc
    r.x = -base.y * sc;
    r.y = base.x * sc;
  } else if (deg == 2) {
    int a = -1, c = -1;
    for (int j = 0; j < 3; ++j)
      for (int q = 0; q < mono.e[f][j]; ++q) {
        if (a < 0)
          a = j;
        else
          c = j;
      }
    const T sc = T(B.H[a * 3 + c]) - twopi * twopi * m.hx[a] * m.hx[c];
    r.x = base.x * sc;
    r.y = base.y * sc;
  } else {
    bool imag;
    const T sc = moment_factor<T>(mono, f, m, B, &imag);
    r.x = imag ? -base.y * sc : base.x * sc;
    r.y = imag ? base.x * sc : base.y * sc;
  }
  return r;
}

// Type-2 stage for one bandwidth: thread per fine half-spectrum index; the
// mode's multiplier and deconvolution are formed once and applied to every
// strength (density and responses / probes).  Modes outside the kept box
// are written as zeros.
template <typename T, int D>
__global__ void kmul_t2_kernel(GeoDev g, const BwDev* __restrict__ bwt, int b,
                               const double* __restrict__ tab, int64_t phi1_0, int64_t phi1_1,
                               int64_t phi1_2, MonoTab mono, const typename Cx<T>::type* __restrict__ F,
                               int64_t fine_half, int str_dens, int str_rhs, int n_rhs_str,
                               int64_t t2half, typename Cx<T>::type* __restrict__ out) {
  using C = typename Cx<T>::type;
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= t2half) return;
  const BwDev& B = bwt[b];
  const int nfields = mono.n + n_rhs_str * mono.nt;
  int64_t kk[3] = {0, 0, 0};
  bool inside = true;
  {
    int64_t rem = j;
    for (int a = D - 1; a >= 0; --a) {
      const int64_t n = (a == D - 1) ? (B.nf[a] / 2 + 1) : B.nf[a];
      const int64_t idx = rem % n;
      rem /= n;
      const int64_t k = (a == D - 1) ? idx : (idx < (B.nf[a] + 1) / 2 ? idx : idx - B.nf[a]);
      kk[a] = k;
      if ((k < 0 ? -k : k) > B.K[a] / 2 - 1) inside = false;
    }
  }
  if (!inside) {
    for (int f = 0; f < nfields; ++f) out[int64_t(f) * t2half + j] = C{T(0), T(0)};
    return;
  }
  const int64_t phi1[3] = {phi1_0, phi1_1, phi1_2};
  T dec = T(1);
  for (int a = 0; a < D; ++a) {
    const int64_t ak = kk[a] < 0 ? -kk[a] : kk[a];
    dec *= T(tab[phi1[a] + ak] * tab[B.phi2_off[a] + ak] / g.P[a]);
  }
  const ModeMul<T> m = mode_mul<T>(g, B, kk, D);
  const T sc = dec * m.G;
  // index of the mode in the type-1 half spectrum (conjugate for k_last < 0)
  const bool neg = kk[D - 1] < 0;
  int64_t fidx = 0;
  for (int a = 0; a < D; ++a) {
    int64_t k = neg ? -kk[a] : kk[a];
    const int64_t n = (a == D - 1) ? (g.nf[a] / 2 + 1) : g.nf[a];
    if (a < D - 1) {
      k %= g.nf[a];
      if (k < 0) k += g.nf[a];
    }
    fidx = fidx * n + k;
  }
  for (int q = 0; q <= n_rhs_str; ++q) {
    const int strength = q == 0 ? str_dens : str_rhs + q - 1;
    const int nfld = q == 0 ? mono.n : mono.nt;
    const int fbase = q == 0 ? 0 : mono.n + (q - 1) * mono.nt;
    C base = F[int64_t(strength) * fine_half + fidx];
    if (neg) base.y = -base.y;
    base.x *= sc;
    base.y *= sc;
    for (int f = 0; f < nfld; ++f)
      out[int64_t(fbase + f) * t2half + j] = mult_field<T, C>(base, m, B, mono, f);
  }
}

template <typename T>
cudaError_t launch_grid(fkreg_plan_s* P, int str_dens, int str_rhs, int nrhs_fields, int bw_first,
                        int bw_count, void* out, cudaStream_t st) {
  using C = typename Cx<T>::type;
  const GeoDev& g = P->geo;
  const int D = P->d;
  int64_t lhalf = 1, fhalf = 1;
  for (int a = 0; a < D; ++a) {
    lhalf *= (a == D - 1) ? (g.L[a] / 2 + 1) : g.L[a];
    fhalf *= (a == D - 1) ? (g.nf[a] / 2 + 1) : g.nf[a];
  }
  const int nq = (str_dens >= 0 ? 1 : 0) + nrhs_fields;
  const int64_t total = lhalf * bw_count * nq;
  const unsigned blocks = unsigned((total + 255) / 256);
  const int fgrid = (str_dens >= 0 ? P->ns : 0) + nrhs_fields * P->nt;
  auto* F = wsp<C>(P, P->r_spec);
  auto* bwt = wsp<BwDev>(P, P->r_bw);
  auto* tab = wsp<double>(P, P->r_tab);
  C* o = static_cast<C*>(out);
#define FK_KG(DD)                                                                                  \
  kmul_grid_kernel<T, DD><<<blocks, 256, 0, st>>>(g, bwt, tab, P->phi1_off[0], P->phi1_off[1],      \
                                                  P->phi1_off[2], P->mono, F, fhalf, str_dens,      \
                                                  str_rhs, nrhs_fields, bw_first, bw_count, fgrid, \
                                                  lhalf, o)
  if (D == 1)
    FK_KG(1);
  else if (D == 2)
    FK_KG(2);
  else
    FK_KG(3);
#undef FK_KG
  P->launches += 1;
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_t2(fkreg_plan_s* P, int b, int str_dens, int str_rhs, int n_rhs_str,
                      cudaStream_t st) {
  using C = typename Cx<T>::type;
  const GeoDev& g = P->geo;
  const int D = P->d;
  const BwDev& B = P->bw[b];
  int64_t t2half = 1, fhalf = 1;
  for (int a = 0; a < D; ++a) {
    t2half *= (a == D - 1) ? (B.nf[a] / 2 + 1) : B.nf[a];
    fhalf *= (a == D - 1) ? (g.nf[a] / 2 + 1) : g.nf[a];
  }
  const unsigned blocks = unsigned((t2half + 255) / 256);
  auto* F = wsp<C>(P, P->r_spec);
  auto* bwt = wsp<BwDev>(P, P->r_bw);
  auto* tab = wsp<double>(P, P->r_tab);
  C* o = wsp<C>(P, P->r_t2spec);
#define FK_KT(DD)                                                                               \
  kmul_t2_kernel<T, DD><<<blocks, 256, 0, st>>>(g, bwt, b, tab, P->phi1_off[0], P->phi1_off[1], \
                                                P->phi1_off[2], P->mono, F, fhalf, str_dens,    \
                                                str_rhs, n_rhs_str, t2half, o)
  if (D == 1)
    FK_KT(1);
  else if (D == 2)
    FK_KT(2);
  else
    FK_KT(3);
#undef FK_KT
  P->launches += 1;
  return cudaGetLastError();
}


// ---- multipliers for the backward pass ----------------------------------------
// Fourier multiplier of field f (monomial exponent e_f) at xi = k / P:
//  kind 0: conj(w^_f(xi))             forward field T_f(q) = sum_i c_i w_f(x_i - q)
//  kind 1: 2 pi i xi_d conj(w^_f)     its gradient in the evaluation point q_d
//  kind 2: d conj(w^_f) / d log sigma_j   (H = diag(sigma^2))
//  kind 3: w^_f(xi)                   adjoint field sum_m e_m w_f(q - x_m)
//  kind 4: 2 pi i xi_d w^_f(xi)       adjoint field of the kernel derivative
// with w^_0 = G, w^_(e_a) = -2 pi i (H xi)_a G, w^_(e_a+e_b) = (H_ab - 4 pi^2 (H xi)_a (H xi)_b) G.
template <typename T, typename C>
__device__ __forceinline__ C field_mult(const MonoTab& mono, int f, int kind, int axis, const T xi[3],
                                        const ModeMul<T>& m, const BwDev& B) {
  const T twopi = T(6.283185307179586476925286766559);
  const T fpi2 = twopi * twopi;
  const int deg = mono.e[f][0] + mono.e[f][1] + mono.e[f][2];
  int a = -1, b = -1;
  for (int j = 0; j < 3; ++j)
    for (int r = 0; r < mono.e[f][j]; ++r) {
      if (a < 0)
        a = j;
      else
        b = j;
    }
  C W{T(0), T(0)};
  if (kind == 2) {
    const int j = axis;
    const T s2 = T(B.H[j * 3 + j]);
    const T dG = -T(0.5) * fpi2 * T(2) * s2 * xi[j] * xi[j] * m.G;  // -4 pi^2 sigma_j^2 xi_j^2 G
    const T dxa = (a == j) ? T(2) * s2 * xi[j] : T(0);
    if (deg == 0) {
      W.x = dG;
    } else if (deg == 1) {
      W.y = twopi * (dxa * m.G + m.hx[a] * dG);
    } else {
      const T dxb = (b == j) ? T(2) * s2 * xi[j] : T(0);
      const T dH = (a == j && b == j) ? T(2) * s2 : T(0);
      W.x = (dH - fpi2 * (dxa * m.hx[b] + m.hx[a] * dxb)) * m.G +
            (T(B.H[a * 3 + b]) - fpi2 * m.hx[a] * m.hx[b]) * dG;
    }
    return W;
  }
  const bool adjoint = kind >= 3;
  if (deg == 0) {
    W.x = m.G;
  } else if (deg == 1) {
    W.y = (adjoint ? -twopi : twopi) * m.hx[a] * m.G;
  } else {
    W.x = (T(B.H[a * 3 + b]) - fpi2 * m.hx[a] * m.hx[b]) * m.G;
  }
  if (kind == 1 || kind == 4) {  // times 2 pi i xi_d
    const T s = twopi * xi[axis];
    const C r{-W.y * s, W.x * s};
    return r;
  }
  return W;
}

// Type-2 spectra of the forward fields under multiplier `kind` (0, 1, 2), for
// one bandwidth: thread per (fine half-spectrum index, strength q).
template <typename T, int D>
__global__ void kmul_t2_mode_kernel(GeoDev g, const BwDev* __restrict__ bwt, int b,
                                    const double* __restrict__ tab, int64_t phi1_0, int64_t phi1_1,
                                    int64_t phi1_2, MonoTab mono,
                                    const typename Cx<T>::type* __restrict__ F, int64_t fine_half,
                                    int str_dens, int str_rhs, int n_rhs_str, int kind, int axis,
                                    int64_t t2half, typename Cx<T>::type* __restrict__ out) {
  using C = typename Cx<T>::type;
  const int nq = 1 + n_rhs_str;
  const int64_t gid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (gid >= t2half * nq) return;
  const int64_t j = gid % t2half;
  const int q = int(gid / t2half);
  const BwDev& B = bwt[b];
  const bool dens = q == 0;
  const int strength = dens ? str_dens : str_rhs + q - 1;
  const int nfld = dens ? mono.n : mono.nt;
  const int fbase = dens ? 0 : mono.n + (q - 1) * mono.nt;
  int64_t kk[3] = {0, 0, 0};
  bool inside = true;
  {
    int64_t rem = j;
    for (int a = D - 1; a >= 0; --a) {
      const int64_t nn = (a == D - 1) ? (B.nf[a] / 2 + 1) : B.nf[a];
      int64_t idx = rem % nn;
      rem /= nn;
      int64_t k = (a == D - 1) ? idx : (idx < (B.nf[a] + 1) / 2 ? idx : idx - B.nf[a]);
      kk[a] = k;
      if ((k < 0 ? -k : k) > B.K[a] / 2 - 1) inside = false;
    }
  }
  C res[kMaxMono];
  for (int f = 0; f < kMaxMono; ++f) res[f] = C{T(0), T(0)};
  if (inside) {
    const int64_t phi1[3] = {phi1_0, phi1_1, phi1_2};
    T dec = T(1);
    T xi[3] = {T(0), T(0), T(0)};
    for (int a = 0; a < D; ++a) {
      const int64_t ak = kk[a] < 0 ? -kk[a] : kk[a];
      dec *= T(tab[phi1[a] + ak] * tab[B.phi2_off[a] + ak] / g.P[a]);
      xi[a] = T(kk[a]) / T(g.P[a]);
    }
    const ModeMul<T> m = mode_mul<T>(g, B, kk, D);
    C base = fetch_F<T, C>(g, F + int64_t(strength) * fine_half, kk, D);
    base.x *= dec;
    base.y *= dec;
    for (int f = 0; f < nfld; ++f) {
      const C W = field_mult<T, C>(mono, dens ? f : f, kind, axis, xi, m, B);
      res[f] = cmul<C, T>(W, base);
    }
  }
  for (int f = 0; f < nfld; ++f) out[int64_t(fbase + f) * t2half + j] = res[f];
}

// Adjoint fields on bandwidth b's type-2 grid from the spectra E_f of the
// adjoint strengths (strength index sb + f for field f):
//   output 0            : sum_{f in class y} w^_f(xi) E_f                (d/dy)
//   output 1 + c D + d  : sum_{f in class c} 2 pi i xi_d w^_f(xi) E_f     (d/dx, source side)
// classes: c = 0 the s-fields (density), c >= 1 the t-fields of response /
// probe c - 1.  Thread per (fine half-spectrum index, output).
template <typename T, int D>
__global__ void kmul_adj_kernel(GeoDev g, const BwDev* __restrict__ bwt, int b,
                                const double* __restrict__ tab, int64_t phi1_0, int64_t phi1_1,
                                int64_t phi1_2, MonoTab mono,
                                const typename Cx<T>::type* __restrict__ F, int64_t fine_half, int sb,
                                int n_classes, int64_t t2half, typename Cx<T>::type* __restrict__ out) {
  using C = typename Cx<T>::type;
  const int nout = 1 + n_classes * D;
  const int64_t gid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (gid >= t2half * nout) return;
  const int64_t j = gid % t2half;
  const int o = int(gid / t2half);
  const BwDev& B = bwt[b];
  int64_t kk[3] = {0, 0, 0};
  bool inside = true;
  {
    int64_t rem = j;
    for (int a = D - 1; a >= 0; --a) {
      const int64_t nn = (a == D - 1) ? (B.nf[a] / 2 + 1) : B.nf[a];
      int64_t idx = rem % nn;
      rem /= nn;
      int64_t k = (a == D - 1) ? idx : (idx < (B.nf[a] + 1) / 2 ? idx : idx - B.nf[a]);
      kk[a] = k;
      if ((k < 0 ? -k : k) > B.K[a] / 2 - 1) inside = false;
    }
  }
  C acc{T(0), T(0)};
  if (inside) {
    const int64_t phi1[3] = {phi1_0, phi1_1, phi1_2};
    T dec = T(1);
    T xi[3] = {T(0), T(0), T(0)};
    for (int a = 0; a < D; ++a) {
      const int64_t ak = kk[a] < 0 ? -kk[a] : kk[a];
      dec *= T(tab[phi1[a] + ak] * tab[B.phi2_off[a] + ak] / g.P[a]);
      xi[a] = T(kk[a]) / T(g.P[a]);
    }
    const ModeMul<T> m = mode_mul<T>(g, B, kk, D);
    int cls, kind, axis = 0;
    if (o == 0) {
      cls = 1;
      kind = 3;
    } else {
      cls = (o - 1) / D;
      axis = (o - 1) % D;
      kind = 4;
    }
    const int f0 = cls == 0 ? 0 : mono.n + (cls - 1) * mono.nt;
    const int nf = cls == 0 ? mono.n : mono.nt;
    for (int q = 0; q < nf; ++q) {
      const int f = f0 + q;
      const int mf = cls == 0 ? q : q;  // monomial index inside the class
      C e = fetch_F<T, C>(g, F + int64_t(sb + f) * fine_half, kk, D);
      const C W = field_mult<T, C>(mono, mf, kind, axis, xi, m, B);
      const C t = cmul<C, T>(W, e);
      acc.x += t.x;
      acc.y += t.y;
    }
    acc.x *= dec;
    acc.y *= dec;
  }
  out[int64_t(o) * t2half + j] = acc;
}

// ---- vector-Jacobian product of the grid estimate ---------------------------
// The grid fields are T_f(lo + m delta) = sum_|k|<K/2 A_f[k] exp(2 pi i k m / L)
// with A_f[k] = W_f(k/P) F_k / prod P (see the top of this file).  For adjoint
// grid values Qbar_f(m) (zero off the output points) the adjoint map gives
//   Fbar_k = (1 / prod P) conj(W_f(k/P)) Ebar_f[k],  Ebar_f[k] = sum_m Qbar_f(m) exp(-2 pi i k m / L),
// i.e. Ebar_f is the length-L forward DFT of Qbar_f, periodic in k with period
// L (the adjoint of the fold), and conj(W_f) = w^_f.  Evaluating
// sum_k Fbar_k exp(2 pi i k (x - lo) / P) at the samples (type 2) gives the
// adjoint function E_f(x) = sum_g Qbar_f(g) w_f(x - g) and, with the factor
// 2 pi i xi_d, its gradient.

// Ebar at signed mode kk from the R2C half spectrum of a real field on the
// length-L lattice (periodic in k, Hermitian).
template <typename T, typename C>
__device__ __forceinline__ C fetch_lattice(const GeoDev& g, const C* __restrict__ E,
                                           const int64_t kk[3], int D) {
  int64_t k[3] = {0, 0, 0};
  for (int a = 0; a < D; ++a) {
    k[a] = kk[a] % g.L[a];
    if (k[a] < 0) k[a] += g.L[a];
  }
  const bool cj = k[D - 1] > g.L[D - 1] / 2;
  if (cj)
    for (int a = 0; a < D; ++a) k[a] = (g.L[a] - k[a]) % g.L[a];
  int64_t idx = 0;
  for (int a = 0; a < D; ++a) idx = idx * ((a == D - 1) ? (g.L[a] / 2 + 1) : g.L[a]) + k[a];
  C v = E[idx];
  if (cj) v.y = -v.y;
  return v;
}

// Type-2 spectra on bandwidth b's fine grid of the adjoint functions:
//   output r (< nrhs)        : sum_{f in t-fields of response r} w^_f Ebar_f      (d/dy)
//   output nrhs + c D + d    : sum_{f in class c} 2 pi i xi_d w^_f Ebar_f           (d/dx)
// classes: c = 0 the s-fields (density), c = 1 + r the t-fields of response r.
// Thread per (fine half-spectrum index, output).
template <typename T, int D>
__global__ void kmul_adj_lattice_kernel(GeoDev g, const BwDev* __restrict__ bwt, int b,
                                        const double* __restrict__ tab, MonoTab mono,
                                        const typename Cx<T>::type* __restrict__ E, int64_t lhalf,
                                        int nrhs, int64_t t2half,
                                        typename Cx<T>::type* __restrict__ out) {
  using C = typename Cx<T>::type;
  const int nout = nrhs + (1 + nrhs) * D;
  const int64_t gid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (gid >= t2half * nout) return;
  const int64_t j = gid % t2half;
  const int o = int(gid / t2half);
  const BwDev& B = bwt[b];
  int64_t kk[3] = {0, 0, 0};
  bool inside = true;
  {
    int64_t rem = j;
    for (int a = D - 1; a >= 0; --a) {
      const int64_t nn = (a == D - 1) ? (B.nf[a] / 2 + 1) : B.nf[a];
      const int64_t idx = rem % nn;
      rem /= nn;
      const int64_t k = (a == D - 1) ? idx : (idx < (B.nf[a] + 1) / 2 ? idx : idx - B.nf[a]);
      kk[a] = k;
      if ((k < 0 ? -k : k) > B.K[a] / 2 - 1) inside = false;
    }
  }
  C acc{T(0), T(0)};
  if (inside) {
    T dec = T(1);
    T xi[3] = {T(0), T(0), T(0)};
    for (int a = 0; a < D; ++a) {
      const int64_t ak = kk[a] < 0 ? -kk[a] : kk[a];
      dec *= T(tab[B.phi2_off[a] + ak] / g.P[a]);
      xi[a] = T(kk[a]) / T(g.P[a]);
    }
    const ModeMul<T> m = mode_mul<T>(g, B, kk, D);
    int cls, kind, axis = 0;
    if (o < nrhs) {
      cls = 1 + o;
      kind = 3;
    } else {
      cls = (o - nrhs) / D;
      axis = (o - nrhs) % D;
      kind = 4;
    }
    const int f0 = cls == 0 ? 0 : mono.n + (cls - 1) * mono.nt;
    const int nf = cls == 0 ? mono.n : mono.nt;
    for (int q = 0; q < nf; ++q) {
      const C e = fetch_lattice<T, C>(g, E + int64_t(f0 + q) * lhalf, kk, D);
      const C W = field_mult<T, C>(mono, q, kind, axis, xi, m, B);
      const C t = cmul<C, T>(W, e);
      acc.x += t.x;
      acc.y += t.y;
    }
    acc.x *= dec;
    acc.y *= dec;
  }
  out[int64_t(o) * t2half + j] = acc;
}

// d L / d log sigma_j = sum_f sum_m Qbar_f(m) dT_f(m)/dlog sigma_j
//   = sum_|k|<K/2 Re[ dW_f(k/P)/dlog sigma_j (F_k / prod P) conj(Ebar_f[k]) ]
// (Parseval on the lattice; the terms of k and -k are conjugate, so the sum
// runs over k_last >= 0 with weight 2 for k_last > 0).  Thread per mode of
// that half box; per-block FP64 partial sums part[block][3].
template <typename T, int D>
__global__ void dlogh_lattice_kernel(GeoDev g, const BwDev* __restrict__ bwt, int b,
                                     const double* __restrict__ tab, int64_t phi1_0,
                                     int64_t phi1_1, int64_t phi1_2, MonoTab mono,
                                     const typename Cx<T>::type* __restrict__ F, int64_t fine_half,
                                     const typename Cx<T>::type* __restrict__ E, int64_t lhalf,
                                     int nrhs, int64_t nmodes, double* __restrict__ part) {
  using C = typename Cx<T>::type;
  __shared__ double red[8][3];
  const int64_t gid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const BwDev& B = bwt[b];
  double dth[3] = {0.0, 0.0, 0.0};
  if (gid < nmodes) {
    int64_t kk[3] = {0, 0, 0};
    int64_t rem = gid;
    for (int a = D - 1; a >= 0; --a) {
      const int64_t hk = B.K[a] / 2 - 1;
      const int64_t nn = (a == D - 1) ? (hk + 1) : (2 * hk + 1);
      const int64_t idx = rem % nn;
      rem /= nn;
      kk[a] = (a == D - 1) ? idx : idx - hk;
    }
    const int64_t phi1[3] = {phi1_0, phi1_1, phi1_2};
    double dec = 1.0;
    T xi[3] = {T(0), T(0), T(0)};
    for (int a = 0; a < D; ++a) {
      const int64_t ak = kk[a] < 0 ? -kk[a] : kk[a];
      dec *= tab[phi1[a] + ak] / g.P[a];
      xi[a] = T(kk[a]) / T(g.P[a]);
    }
    const double wgt = kk[D - 1] == 0 ? 1.0 : 2.0;
    const ModeMul<T> m = mode_mul<T>(g, B, kk, D);
    const int fgrid = mono.n + nrhs * mono.nt;
    for (int f = 0; f < fgrid; ++f) {
      const int strength = f < mono.n ? 0 : 1 + (f - mono.n) / mono.nt;
      const int mf = f < mono.n ? f : (f - mono.n) % mono.nt;
      const C Fk = fetch_F<T, C>(g, F + int64_t(strength) * fine_half, kk, D);
      const C e = fetch_lattice<T, C>(g, E + int64_t(f) * lhalf, kk, D);
      // (F_k / prod P) conj(Ebar)
      const double px = dec * (double(Fk.x) * double(e.x) + double(Fk.y) * double(e.y));
      const double py = dec * (double(Fk.y) * double(e.x) - double(Fk.x) * double(e.y));
      for (int j = 0; j < D; ++j) {
        const C W2 = field_mult<T, C>(mono, mf, 2, j, xi, m, B);
        dth[j] += wgt * (double(W2.x) * px - double(W2.y) * py);
      }
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = 0; d < 3; ++d) {
    double v = dth[d];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][d] = v;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int wv = 0; wv < int(blockDim.x >> 5); ++wv) t += red[wv][threadIdx.x];
    part[int64_t(blockIdx.x) * 3 + threadIdx.x] = t;
  }
}

__global__ void sum_partials3(const double* __restrict__ part, int64_t nblk, int D,
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

template <typename T>
cudaError_t launch_adj_lattice(fkreg_plan_s* P, int b, int nrhs, const void* E, cudaStream_t st) {
  using C = typename Cx<T>::type;
  const GeoDev& g = P->geo;
  const int D = P->d;
  const BwDev& B = P->bw[b];
  int64_t t2half = 1, lhalf = 1;
  for (int a = 0; a < D; ++a) {
    t2half *= (a == D - 1) ? (B.nf[a] / 2 + 1) : B.nf[a];
    lhalf *= (a == D - 1) ? (g.L[a] / 2 + 1) : g.L[a];
  }
  const int nout = nrhs + (1 + nrhs) * D;
  const unsigned blocks = unsigned((t2half * nout + 255) / 256);
  const C* Ein = static_cast<const C*>(E);
  C* o = wsp<C>(P, P->r_t2spec);
#define FK_KL(DD)                                                                               \
  kmul_adj_lattice_kernel<T, DD><<<blocks, 256, 0, st>>>(g, wsp<BwDev>(P, P->r_bw), b,          \
                                                         wsp<double>(P, P->r_tab), P->mono, Ein, \
                                                         lhalf, nrhs, t2half, o)
  if (D == 1)
    FK_KL(1);
  else if (D == 2)
    FK_KL(2);
  else
    FK_KL(3);
#undef FK_KL
  P->launches += 1;
  return cudaGetLastError();
}

int64_t dlogh_modes(const fkreg_plan_s* P, int b) {
  const BwDev& B = P->bw[b];
  int64_t nm = 1;
  for (int a = 0; a < P->d; ++a) {
    const int64_t hk = B.K[a] / 2 - 1;
    nm *= (a == P->d - 1) ? (hk + 1) : (2 * hk + 1);
  }
  return nm;
}

template <typename T>
cudaError_t launch_dlogh_lattice(fkreg_plan_s* P, int b, int nrhs, const void* E, double* part,
                                 double* dlogh, cudaStream_t st) {
  using C = typename Cx<T>::type;
  const GeoDev& g = P->geo;
  const int D = P->d;
  int64_t lhalf = 1, fhalf = 1;
  for (int a = 0; a < D; ++a) {
    lhalf *= (a == D - 1) ? (g.L[a] / 2 + 1) : g.L[a];
    fhalf *= (a == D - 1) ? (g.nf[a] / 2 + 1) : g.nf[a];
  }
  const int64_t nmodes = dlogh_modes(P, b);
  const int64_t nblk = (nmodes + 255) / 256;
  const C* Ein = static_cast<const C*>(E);
#define FK_DL(DD)                                                                                  \
  dlogh_lattice_kernel<T, DD><<<unsigned(nblk), 256, 0, st>>>(                                     \
      g, wsp<BwDev>(P, P->r_bw), b, wsp<double>(P, P->r_tab), P->phi1_off[0], P->phi1_off[1],      \
      P->phi1_off[2], P->mono, wsp<C>(P, P->r_spec), fhalf, Ein, lhalf, nrhs, nmodes, part)
  if (D == 1)
    FK_DL(1);
  else if (D == 2)
    FK_DL(2);
  else
    FK_DL(3);
#undef FK_DL
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  sum_partials3<<<D, 256, 0, st>>>(part, nblk, D, dlogh);
  P->launches += 2;
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_t2_mode(fkreg_plan_s* P, int b, int str_dens, int str_rhs, int n_rhs_str,
                           int kind, int axis, cudaStream_t st) {
  using C = typename Cx<T>::type;
  const GeoDev& g = P->geo;
  const int D = P->d;
  const BwDev& B = P->bw[b];
  int64_t t2half = 1, fhalf = 1;
  for (int a = 0; a < D; ++a) {
    t2half *= (a == D - 1) ? (B.nf[a] / 2 + 1) : B.nf[a];
    fhalf *= (a == D - 1) ? (g.nf[a] / 2 + 1) : g.nf[a];
  }
  const int64_t total = t2half * (1 + n_rhs_str);
  const unsigned blocks = unsigned((total + 255) / 256);
  auto* F = wsp<C>(P, P->r_spec);
  auto* bwt = wsp<BwDev>(P, P->r_bw);
  auto* tab = wsp<double>(P, P->r_tab);
  C* o = wsp<C>(P, P->r_t2spec);
#define FK_KM(DD)                                                                                    \
  kmul_t2_mode_kernel<T, DD><<<blocks, 256, 0, st>>>(g, bwt, b, tab, P->phi1_off[0], P->phi1_off[1], \
                                                     P->phi1_off[2], P->mono, F, fhalf, str_dens,    \
                                                     str_rhs, n_rhs_str, kind, axis, t2half, o)
  if (D == 1)
    FK_KM(1);
  else if (D == 2)
    FK_KM(2);
  else
    FK_KM(3);
#undef FK_KM
  P->launches += 1;
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adj(fkreg_plan_s* P, int b, int sb, int n_classes, cudaStream_t st) {
  using C = typename Cx<T>::type;
  const GeoDev& g = P->geo;
  const int D = P->d;
  const BwDev& B = P->bw[b];
  int64_t t2half = 1, fhalf = 1;
  for (int a = 0; a < D; ++a) {
    t2half *= (a == D - 1) ? (B.nf[a] / 2 + 1) : B.nf[a];
    fhalf *= (a == D - 1) ? (g.nf[a] / 2 + 1) : g.nf[a];
  }
  const int nout = 1 + n_classes * D;
  const int64_t total = t2half * nout;
  const unsigned blocks = unsigned((total + 255) / 256);
  auto* F = wsp<C>(P, P->r_spec);
  auto* bwt = wsp<BwDev>(P, P->r_bw);
  auto* tab = wsp<double>(P, P->r_tab);
  C* o = wsp<C>(P, P->r_t2spec);
#define FK_KA(DD)                                                                                 \
  kmul_adj_kernel<T, DD><<<blocks, 256, 0, st>>>(g, bwt, b, tab, P->phi1_off[0], P->phi1_off[1], \
                                                 P->phi1_off[2], P->mono, F, fhalf, sb, n_classes, \
                                                 t2half, o)
  if (D == 1)
    FK_KA(1);
  else if (D == 2)
    FK_KA(2);
  else
    FK_KA(3);
#undef FK_KA
  P->launches += 1;
  return cudaGetLastError();
}

}  // namespace

cudaError_t run_kmul_grid(fkreg_plan_s* P, int str_dens, int str_rhs, int nrhs_fields, int bw_first,
                          int bw_count, void* out_spec, cudaStream_t st) {
  return P->prec == FKREG_F32
             ? launch_grid<float>(P, str_dens, str_rhs, nrhs_fields, bw_first, bw_count, out_spec, st)
             : launch_grid<double>(P, str_dens, str_rhs, nrhs_fields, bw_first, bw_count, out_spec, st);
}

cudaError_t run_kmul_t2(fkreg_plan_s* P, int b, int str_dens, int str_rhs, int n_rhs_str,
                        cudaStream_t st) {
  return P->prec == FKREG_F32 ? launch_t2<float>(P, b, str_dens, str_rhs, n_rhs_str, st)
                              : launch_t2<double>(P, b, str_dens, str_rhs, n_rhs_str, st);
}

cudaError_t run_kmul_t2_mode(fkreg_plan_s* P, int b, int str_dens, int str_rhs, int n_rhs_str,
                             int kind, int axis, cudaStream_t st) {
  return P->prec == FKREG_F32
             ? launch_t2_mode<float>(P, b, str_dens, str_rhs, n_rhs_str, kind, axis, st)
             : launch_t2_mode<double>(P, b, str_dens, str_rhs, n_rhs_str, kind, axis, st);
}

cudaError_t run_kmul_adj(fkreg_plan_s* P, int b, int sb, int n_classes, cudaStream_t st) {
  return P->prec == FKREG_F32 ? launch_adj<float>(P, b, sb, n_classes, st)
                              : launch_adj<double>(P, b, sb, n_classes, st);
}

cudaError_t run_kmul_adj_lattice(fkreg_plan_s* P, int b, int nrhs, const void* E, cudaStream_t st) {
  return P->prec == FKREG_F32 ? launch_adj_lattice<float>(P, b, nrhs, E, st)
                              : launch_adj_lattice<double>(P, b, nrhs, E, st);
}

int64_t run_dlogh_lattice_blocks(const fkreg_plan_s* P, int b) {
  return (dlogh_modes(P, b) + 255) / 256;
}

cudaError_t run_dlogh_lattice(fkreg_plan_s* P, int b, int nrhs, const void* E, double* part,
                              double* dlogh, cudaStream_t st) {
  return P->prec == FKREG_F32 ? launch_dlogh_lattice<float>(P, b, nrhs, E, part, dlogh, st)
                              : launch_dlogh_lattice<double>(P, b, nrhs, E, part, dlogh, st);
}

}  // namespace fk

// ---- interleave the type-2 fields into cell records ----------------------------
// The inverse FFT of the type-2 spectra runs in place (cuFFT's padded real
// layout: field f, row r, column i at f * 2 t2half + r * 2 (n_last/2 + 1) + i),
// which is over twice as fast on large 3-D grids as writing strided records
// directly.  This kernel then gathers the fields of 32 cells at a time through
// shared memory into the record layout [cell][rec] that the interpolation
// reads (coalesced reads along cells, coalesced writes along records).
namespace fk {
namespace {

template <typename T>
__global__ void t2_interleave_kernel(const T* __restrict__ src, int64_t cells, int64_t nlast,
                                     int64_t row_pitch, int64_t fdist, int F, int rec,
                                     T* __restrict__ dst) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tile = reinterpret_cast<T*>(smem_raw);  // [F][33]
  const int64_t c0 = int64_t(blockIdx.x) * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int nty = blockDim.x >> 5;
  const int64_t c = c0 + tx;
  if (c < cells) {
    const int64_t off = (c / nlast) * row_pitch + c % nlast;
    for (int f = ty; f < F; f += nty) tile[f * 33 + tx] = src[int64_t(f) * fdist + off];
  }
  __syncthreads();
  const int ncell = int(min(int64_t(32), cells - c0));
  for (int idx = threadIdx.x; idx < ncell * F; idx += blockDim.x) {
    const int i = idx / F, f = idx - i * F;
    dst[(c0 + i) * rec + f] = tile[f * 33 + i];
  }
}

}  // namespace

cudaError_t run_t2_interleave(fkreg_plan_s* P, const int64_t* dims, int F, const void* src,
                              void* dst, cudaStream_t st) {
  const int D = P->d;
  int64_t cells = 1, rows = 1;
  for (int a = 0; a < D; ++a) cells *= dims[a];
  for (int a = 0; a < D - 1; ++a) rows *= dims[a];
  const int64_t nlast = dims[D - 1];
  const int64_t row_pitch = 2 * (nlast / 2 + 1);
  const int64_t fdist = rows * row_pitch;
  const int rec = t2_record_stride(F);
  if (cells == 0 || F == 0) return cudaSuccess;
  const unsigned blocks = unsigned((cells + 31) / 32);
  const size_t smem = size_t(F) * 33 * P->tsize;
  if (P->prec == FKREG_F32) {
    cudaError_t e = cudaFuncSetAttribute(t2_interleave_kernel<float>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    t2_interleave_kernel<float><<<blocks, 256, smem, st>>>(static_cast<const float*>(src), cells,
                                                           nlast, row_pitch, fdist, F, rec,
                                                           static_cast<float*>(dst));
  } else {
    cudaError_t e = cudaFuncSetAttribute(t2_interleave_kernel<double>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    t2_interleave_kernel<double><<<blocks, 256, smem, st>>>(static_cast<const double*>(src), cells,
                                                            nlast, row_pitch, fdist, F, rec,
                                                            static_cast<double*>(dst));
  }
  P->launches += 1;
  return cudaGetLastError();
}

}  // namespace fk
