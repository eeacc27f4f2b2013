// Host planner: validation, NUFFT geometry, spreading-kernel transforms.
//
// Geometry (per axis j, all bandwidths b of the plan):
//  * Grid spacing delta_j = (hi_j - lo_j) / (M_j - 1), endpoints included
//    (eq. 6; the garbled tau_j of Sec. 1.1 read as this).
//  * Kernel tail radius R_bj = r sigma_bj, r the smallest value with
//    exp(-r^2/2) max(1, r^2)^l <= tol/10 (the Gaussian moment kernel
//    z^g K_H(z) with |g| <= 2l is below tol of its natural size beyond R).
//  * Period P_j = L_j delta_j with L_j >= (M_j - 1) + max_b R_bj / delta_j, so
//    the periodic images of the samples never reach the grid box.  This is
//    the job the zero padding of eq. 18 does in the paper.
//  * Modes: the transform of K_H is exp(-2 pi^2 xi^T H xi); with its moment
//    factors it is below tol/10 of its size once 2 pi^2 xi^T H xi >= Q,
//    exp(-Q)(1 + 2Q)^l = tol/10.  Along axis j that bounds
//    |xi_j| <= sqrt(Q / (2 pi^2)) sqrt((H^-1)_jj), i.e. |k_j| <= xi_j P_j.
//  * Type-1 spreading onto an oversampled fine grid nf_j >= 2 K_j
//    (oversampling 2, as the M_r = 2L of Sec. 1.2 eq. 17).
//  * Spreading kernel: exponential of semicircle
//    phi(z) = exp(beta (sqrt(1 - (2z/w)^2) - 1)), |z| <= w/2, with
//    w = ceil(log10(1/tol)) + 1 and beta = 2.30 w (Barnett, Magland &
//    af Klinteberg, SIAM J. Sci. Comput. 41, 2019), or the truncated
//    Gaussian of eq. 17, phi(z) = exp(-(3 pi / (4 m)) z^2), |z| <= m,
//    m = ceil(log10(1/tol)) + 1 cells per side (Greengard & Lee 2004 with
//    oversampling 2), about twice as wide.
//  * Deconvolution (eq. 20): divide mode k by
//    phihat(k) = integral phi(z) cos(2 pi k z / nf) dz, evaluated by
//    Gauss-Legendre quadrature in FP64.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "internal.h"

namespace fk {

int nmono(int d, int deg) {
  long num = 1, den = 1;
  for (int k = 1; k <= deg; ++k) {
    num *= (d + k);
    den *= k;
  }
  return int(num / den);
}

void monomials(int d, int deg, int (*e)[kMaxD]) {
  int m = 0;
  for (int k = 0; k <= deg; ++k) {
    int idx[4] = {0, 0, 0, 0};
    for (;;) {
      for (int j = 0; j < kMaxD; ++j) e[m][j] = 0;
      for (int j = 0; j < k; ++j) e[m][idx[j]] += 1;
      ++m;
      int p = k - 1;
      while (p >= 0 && idx[p] == d - 1) --p;
      if (p < 0) break;
      idx[p] += 1;
      for (int j = p + 1; j < k; ++j) idx[j] = idx[p];
    }
  }
}

static bool is_fast(int64_t n) {
  for (int f : {2, 3, 5, 7})
    while (n % f == 0) n /= f;
  return n == 1;
}

int64_t next_fast(int64_t n) {
  if (n < 1) n = 1;
  while (!is_fast(n)) ++n;
  return n;
}

static int64_t next_fast_even(int64_t n) {
  if (n < 2) n = 2;
  if (n & 1) ++n;
  while (!is_fast(n)) n += 2;
  return n;
}

double spread_phi(int kind, int w, double beta, double z) {
  if (kind == FKREG_SPREAD_ES) {
    double t = 2.0 * z / w;
    if (std::fabs(t) > 1.0) return 0.0;
    return std::exp(beta * (std::sqrt(1.0 - t * t) - 1.0));
  }
  if (std::fabs(z) > 0.5 * w) return 0.0;
  return std::exp(-beta * z * z);
}

// Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_n.
static void gauss_legendre(int n, std::vector<double>* x, std::vector<double>* wt) {
  x->assign(n, 0.0);
  wt->assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double pp = 0;
    for (int it = 0; it < 100; ++it) {
      double p1 = 1.0, p2 = 0.0;
      for (int k = 1; k <= n; ++k) {
        double p3 = p2;
        p2 = p1;
        p1 = ((2.0 * k - 1.0) * z * p2 - (k - 1.0) * p3) / k;
      }
      pp = n * (z * p1 - p2) / (z * z - 1.0);
      double dz = p1 / pp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    (*x)[i] = -z;
    (*x)[n - 1 - i] = z;
    (*wt)[i] = (*wt)[n - 1 - i] = 2.0 / ((1.0 - z * z) * pp * pp);
  }
}

void spread_phihat(int kind, int w, double beta, int64_t nf, int64_t nk, double* out) {
  // phi is even: phihat(k) = 2 * integral_0^{w/2} phi(z) cos(2 pi k z / nf) dz.
  // The ES kernel has a square-root edge, so use many nodes.
  const int q = 8 * w + 64;
  std::vector<double> x, wt;
  gauss_legendre(q, &x, &wt);
  const double a = 0.5 * w;
  for (int64_t k = 0; k < nk; ++k) {
    double s = 0;
    for (int i = 0; i < q; ++i) {
      double z = 0.5 * a * (x[i] + 1.0);  // map [-1,1] -> [0, a]
      s += wt[i] * spread_phi(kind, w, beta, z) * std::cos(2.0 * M_PI * k * z / nf);
    }
    out[k] = 2.0 * 0.5 * a * s;
  }
}

static bool spd_inverse(int d, const double* H, double* Hinv, double* det) {
  // symmetric check
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) {
      double u = H[a * d + b], v = H[b * d + a];
      if (!std::isfinite(u)) return false;
      if (std::fabs(u - v) > 1e-12 * (std::fabs(u) + std::fabs(v)) + 1e-300) return false;
    }
  // Cholesky for positive definiteness
  double L[9] = {0};
  for (int i = 0; i < d; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = H[i * d + j];
      for (int k = 0; k < j; ++k) s -= L[i * 3 + k] * L[j * 3 + k];
      if (i == j) {
        if (!(s > 0)) return false;
        L[i * 3 + i] = std::sqrt(s);
      } else {
        L[i * 3 + j] = s / L[j * 3 + j];
      }
    }
  double dt = 1;
  for (int i = 0; i < d; ++i) dt *= L[i * 3 + i] * L[i * 3 + i];
  *det = dt;
  // inverse by solving H X = I with the Cholesky factor
  for (int c = 0; c < d; ++c) {
    double y[3], xv[3];
    for (int i = 0; i < d; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s -= L[i * 3 + k] * y[k];
      y[i] = s / L[i * 3 + i];
    }
    for (int i = d - 1; i >= 0; --i) {
      double s = y[i];
      for (int k = i + 1; k < d; ++k) s -= L[k * 3 + i] * xv[k];
      xv[i] = s / L[i * 3 + i];
    }
    for (int i = 0; i < d; ++i) Hinv[i * d + c] = xv[i];
  }
  return true;
}

static fkreg_status fail(std::string* err, fkreg_status st, const char* msg) {
  if (err) *err = msg;
  return st;
}

// Unit-mass constant c_d of the compact radial profile k on the unit ball in
// d dimensions (V_d = unit-ball volume): uniform 1/V_d, Epanechnikov
// (d+2)/(2 V_d), triangle (d+1)/V_d, biweight (d+2)(d+4)/(8 V_d), triweight
// (d+2)(d+4)(d+6)/(48 V_d).
static double compact_constant(int kernel, int d) {
  const double vd = d == 1 ? 2.0 : (d == 2 ? M_PI : 4.0 * M_PI / 3.0);
  switch (kernel) {
    case FKREG_KERNEL_UNIFORM: return 1.0 / vd;
    case FKREG_KERNEL_EPANECHNIKOV: return (d + 2) / (2.0 * vd);
    case FKREG_KERNEL_TRIANGLE: return (d + 1) / vd;
    case FKREG_KERNEL_BIWEIGHT: return (d + 2) * (d + 4) / (8.0 * vd);
    case FKREG_KERNEL_GAUSSIAN_DIRECT: return std::pow(2.0 * M_PI, -0.5 * d);
    default: return (d + 2) * (d + 4) * (d + 6) / (48.0 * vd);
  }
}

// Geometry of the direct-sum path (compact kernels): samples are binned on
// the output lattice itself (cell j = floor((x - lo) / delta)), bins of T
// cells with T about half the widest support half-width, so a point's
// support spans a few bins per axis.  No FFT grids.
static fkreg_status compute_geometry_direct(const fkreg_opts* o, fkreg_geometry* g,
                                            std::string* err, std::vector<BwDev>* bwv,
                                            std::vector<double>* tab, int64_t phi1_off[3],
                                            GeoDev* geo, const std::vector<double>& Hinv,
                                            const std::vector<double>& det) {
  const int d = o->dim, nbw = o->n_bw, order = o->order;
  std::memset(g, 0, sizeof(*g));
  g->dim = d;
  g->w = 2;
  g->beta = 0.0;
  std::vector<BwDev> bws(nbw);
  const double cd = compact_constant(o->kernel, d);
  // the support is the unit ball of the metric H^-1 / r2: r2 = 1 for the
  // compact kernels, R^2 for the Gaussian cut at Mahalanobis radius R
  const bool gcut = o->kernel == FKREG_KERNEL_GAUSSIAN_DIRECT;
  const double r2 = gcut ? 2.0 * std::log(10.0 / o->tol) : 1.0;
  for (int b = 0; b < nbw; ++b) {
    BwDev& B = bws[b];
    std::memset(&B, 0, sizeof(B));
    const double* Hb = o->H + size_t(b) * d * d;
    for (int a = 0; a < d; ++a)
      for (int c = 0; c < d; ++c) {
        B.H[a * 3 + c] = r2 * Hb[a * d + c];
        B.Hinv[a * 3 + c] = Hinv[size_t(b) * d * d + a * d + c] / r2;
      }
    B.kscale = cd / std::sqrt(det[b]);
    B.k0 = B.kscale;
    B.kr2 = gcut ? r2 : 0.0;
    for (int j = 0; j < 3; ++j) {
      B.sigma[j] = j < d ? std::sqrt(r2 * Hb[j * d + j]) : 1.0;
      B.K[j] = 1;
      B.nf[j] = j < d ? o->grid_n[j] : 1;
    }
  }
  for (int j = 0; j < 3; ++j) {
    if (j >= d) {
      g->ldft[j] = g->modes[j] = g->nf[j] = g->tile[j] = g->nbins[j] = 1;
      g->period[j] = g->delta[j] = g->inv_h[j] = 1;
      continue;
    }
    const int64_t M = o->grid_n[j];
    const double delta = (o->grid_hi[j] - o->grid_lo[j]) / double(M - 1);
    g->delta[j] = delta;
    g->ldft[j] = M;
    g->modes[j] = 1;
    g->nf[j] = M;
    g->period[j] = delta * double(M);
    g->inv_h[j] = double(M - 1) / (o->grid_hi[j] - o->grid_lo[j]);
    if (o->precision == FKREG_F32) g->inv_h[j] = double(float(g->inv_h[j]));
    double rmax = 0;
    for (int b = 0; b < nbw; ++b) rmax = std::max(rmax, bws[b].sigma[j] / delta);
    int64_t t = o->tile > 0 ? o->tile : std::max<int64_t>(1, std::min<int64_t>(64, int64_t(std::ceil(0.25 * rmax))));
    t = std::min<int64_t>(t, M);
    g->tile[j] = t;
    g->nbins[j] = (M + t - 1) / t;
    for (auto& B : bws) B.inv_h[j] = g->inv_h[j];
  }
  g->ns = nmono(d, 2 * order);
  g->nt = nmono(d, order);
  double nb = 1;
  for (int j = 0; j < d; ++j) nb *= double(g->nbins[j]);
  if (nb > 4.0e9) return fail(err, FKREG_ERR_UNSUPPORTED, "too many bins (raise tile)");
  if (tab) tab->clear();
  if (phi1_off)
    for (int j = 0; j < 3; ++j) phi1_off[j] = 0;
  if (bwv) *bwv = bws;
  if (geo) {
    std::memset(geo, 0, sizeof(*geo));
    geo->d = d;
    geo->w = g->w;
    geo->pad = (g->w + 1) / 2;
    geo->skind = o->spread_kernel;
    geo->beta = 0.0;
    geo->kern = o->kernel;
    for (int j = 0; j < 3; ++j) {
      geo->nf[j] = g->nf[j];
      geo->L[j] = g->ldft[j];
      geo->M[j] = (j < d) ? o->grid_n[j] : 1;
      geo->K[j] = 1;
      geo->P[j] = g->period[j];
      geo->lo[j] = (j < d) ? o->grid_lo[j] : 0;
      geo->hi[j] = (j < d) ? o->grid_hi[j] : 0;
      geo->inv_h[j] = g->inv_h[j];
      geo->inv_h_f[j] = float(g->inv_h[j]);
      geo->tile[j] = g->tile[j];
      geo->nbins[j] = g->nbins[j];
    }
    geo->kbits = key_local_bits(d, geo->tile, geo->nbins);
  }
  return FKREG_OK;
}

fkreg_status compute_geometry(const fkreg_opts* o, fkreg_geometry* g, std::string* err,
                              std::vector<BwDev>* bwv, std::vector<double>* tab,
                              int64_t phi1_off[3], GeoDev* geo) {
  if (!o || !g) return fail(err, FKREG_ERR_INVALID_ARG, "opts and output must be non-NULL");
  const int d = o->dim;
  if (d < 1 || d > 3) return fail(err, FKREG_ERR_INVALID_ARG, "dim must be 1, 2 or 3");
  if (o->order < 0 || o->order > 2) return fail(err, FKREG_ERR_INVALID_ARG, "order must be 0, 1 or 2");
  if (o->order == 2 && o->dim > 2)
    return fail(err, FKREG_ERR_UNSUPPORTED, "order 2 (local quadratic) is supported in 1-D and 2-D");
  if (o->kernel < FKREG_KERNEL_GAUSSIAN || o->kernel > FKREG_KERNEL_GAUSSIAN_DIRECT)
    return fail(err, FKREG_ERR_INVALID_ARG, "unknown regression kernel");
  if (o->kernel != FKREG_KERNEL_GAUSSIAN && (o->flags & FKREG_WANT_BACKWARD))
    return fail(err, FKREG_ERR_UNSUPPORTED, "the backward needs the Gaussian kernel");
  if (o->spread_kernel != FKREG_SPREAD_ES && o->spread_kernel != FKREG_SPREAD_GAUSS)
    return fail(err, FKREG_ERR_INVALID_ARG, "spread_kernel must be FKREG_SPREAD_ES or FKREG_SPREAD_GAUSS");
  if (o->precision != FKREG_F32 && o->precision != FKREG_F64)
    return fail(err, FKREG_ERR_INVALID_ARG, "precision must be FKREG_F32 or FKREG_F64");
  if (o->y_complex != 0 && o->y_complex != 1) return fail(err, FKREG_ERR_INVALID_ARG, "y_complex must be 0 or 1");
  if (o->n_bw < 1 || !o->H) return fail(err, FKREG_ERR_INVALID_ARG, "need n_bw >= 1 bandwidth matrices");
  if (o->n_rhs < 1) return fail(err, FKREG_ERR_INVALID_ARG, "n_rhs must be >= 1");
  if (o->max_probes < 0) return fail(err, FKREG_ERR_INVALID_ARG, "max_probes must be >= 0");
  if (!(o->tol >= 1e-15 && o->tol <= 1e-1)) return fail(err, FKREG_ERR_INVALID_ARG, "tol must lie in [1e-15, 1e-1]");
  if (!(o->mask_rho >= 0 && o->mask_rho < 1)) return fail(err, FKREG_ERR_INVALID_ARG, "mask_rho must lie in [0, 1)");
  if (o->tile < 0 || o->tile > 4096) return fail(err, FKREG_ERR_INVALID_ARG, "tile must lie in [0, 4096]");
  for (int j = 0; j < d; ++j) {
    if (o->grid_n[j] < 2 || o->grid_n[j] > (1 << 20))
      return fail(err, FKREG_ERR_INVALID_ARG, "grid_n must lie in [2, 2^20] on every axis");
    if (!(std::isfinite(o->grid_lo[j]) && std::isfinite(o->grid_hi[j]) && o->grid_hi[j] > o->grid_lo[j]))
      return fail(err, FKREG_ERR_INVALID_ARG, "grid_lo < grid_hi (finite) required on every axis");
  }
  const int order = o->order;
  const int nbw = o->n_bw;
  std::vector<double> Hinv(size_t(nbw) * d * d), det(nbw);
  for (int b = 0; b < nbw; ++b)
    if (!spd_inverse(d, o->H + size_t(b) * d * d, &Hinv[size_t(b) * d * d], &det[b]))
      return fail(err, FKREG_ERR_INVALID_ARG, "every bandwidth matrix H must be symmetric positive definite");

  if (o->kernel != FKREG_KERNEL_GAUSSIAN)
    return compute_geometry_direct(o, g, err, bwv, tab, phi1_off, geo, Hinv, det);

  std::memset(g, 0, sizeof(*g));
  g->dim = d;
  const double tol = o->tol;
  const int digits = int(std::ceil(std::log10(1.0 / tol) - 1e-9));
  int w;
  double beta;
  if (o->spread_kernel == FKREG_SPREAD_ES) {
    w = std::min(16, std::max(2, digits + 1));
    beta = 2.30 * w;
  } else {
    int m = std::min(12, std::max(2, digits + 1));
    w = 2 * m;
    beta = 3.0 * M_PI / (4.0 * m);
  }
  if (d * w > 64)
    return fail(err, FKREG_ERR_UNSUPPORTED, "spreading width too large for this dimension (dim * w <= 64)");
  g->w = w;
  g->beta = beta;

  // tail radius in standard deviations
  double r = 1.0;
  while (std::exp(-0.5 * r * r) * std::pow(std::max(1.0, r * r), order) > 0.1 * tol) r += 0.01;
  // spectral extent
  double Q = 1.0;
  while (std::exp(-Q) * std::pow(1.0 + 2.0 * Q, order) > 0.1 * tol) Q += 0.01;
  const double xi_fac = std::sqrt(Q / (2.0 * M_PI * M_PI));

  std::vector<BwDev> bws(nbw);
  int64_t K1[3] = {0, 0, 0};
  for (int j = 0; j < d; ++j) {
    const double lo = o->grid_lo[j], hi = o->grid_hi[j];
    const int64_t M = o->grid_n[j];
    const double delta = (hi - lo) / double(M - 1);
    double rmax = 0;
    for (int b = 0; b < nbw; ++b) rmax = std::max(rmax, r * std::sqrt(o->H[size_t(b) * d * d + j * d + j]));
    int64_t L = (M - 1) + int64_t(std::ceil(rmax / delta)) + 1;
    L = next_fast(std::max<int64_t>(L, M));
    g->delta[j] = delta;
    g->ldft[j] = L;
    g->period[j] = double(L) * delta;
  }
  for (int b = 0; b < nbw; ++b) {
    BwDev& B = bws[b];
    std::memset(&B, 0, sizeof(B));
    const double* Hb = o->H + size_t(b) * d * d;
    for (int a = 0; a < d; ++a)
      for (int c = 0; c < d; ++c) B.H[a * 3 + c] = Hb[a * d + c];
    B.k0 = 1.0 / std::sqrt(std::pow(2.0 * M_PI, d) * det[b]);
    for (int j = 0; j < d; ++j) {
      B.sigma[j] = std::sqrt(Hb[j * d + j]);
      const double xi = xi_fac * std::sqrt(Hinv[size_t(b) * d * d + j * d + j]);
      int64_t half = int64_t(std::ceil(xi * g->period[j])) + 1;
      int64_t K = std::max<int64_t>(4, 2 * half);
      B.K[j] = K;
      B.nf[j] = next_fast_even(std::max<int64_t>(2 * K, 2 * w + 2));
      B.inv_h[j] = double(B.nf[j]) / g->period[j];
      K1[j] = std::max(K1[j], K);
    }
    for (int j = d; j < 3; ++j) {
      B.K[j] = 1;
      B.nf[j] = 1;
      B.sigma[j] = 1;
    }
  }
  for (int j = 0; j < d; ++j) {
    g->modes[j] = K1[j];
    g->nf[j] = next_fast_even(std::max<int64_t>(2 * K1[j], 2 * w + 2));
    g->inv_h[j] = double(g->nf[j]) / g->period[j];
    if (o->precision == FKREG_F32) g->inv_h[j] = double(float(g->inv_h[j]));
    int64_t t = o->tile;
    if (t == 0) {
      // largest tile whose padded copy fits 96 KB of shared memory per strength
      const int64_t tsz = (o->precision == FKREG_F32) ? 4 : 8;
      const int64_t pad2 = 2 * ((w + 1) / 2);
      const int64_t cand[] = {2048, 64, 32, 16, 12, 8, 6, 4, 2};
      t = 2;
      for (int64_t c : cand) {
        // 2-D tiles of 16 keep the interpolation window of a bin cache-sized
        if ((d == 2 && c > 16) || (d == 3 && c > 16)) continue;
        int64_t cells = 1;
        for (int a = 0; a < d; ++a) cells *= (c + pad2);
        if (cells * tsz <= 96 * 1024) {
          t = c;
          break;
        }
      }
    }
    t = std::min<int64_t>(t, g->nf[j]);
    g->tile[j] = t;
    g->nbins[j] = (g->nf[j] + t - 1) / t;
  }
  for (int j = d; j < 3; ++j) {
    g->ldft[j] = 1;
    g->modes[j] = 1;
    g->nf[j] = 1;
    g->tile[j] = 1;
    g->nbins[j] = 1;
    g->period[j] = 1;
    g->delta[j] = 1;
    g->inv_h[j] = 1;
  }
  g->ns = nmono(d, 2 * order);
  g->nt = nmono(d, order);

  // bins must fit 32-bit keys and the fine grids 64-bit cell counts
  double nb = 1;
  for (int j = 0; j < d; ++j) nb *= double(g->nbins[j]);
  if (nb > 4.0e9) return fail(err, FKREG_ERR_UNSUPPORTED, "too many spreading bins (raise tile)");
  // cell indices of the fine grids are 32-bit inside the kernels
  {
    double c1 = 1;
    for (int j = 0; j < d; ++j) c1 *= double(g->nf[j]);
    double c2 = 0;
    for (int b = 0; b < nbw; ++b) {
      double cb = 1;
      for (int j = 0; j < d; ++j) cb *= double(bws[b].nf[j]);
      c2 = std::max(c2, cb);
    }
    if (c1 >= 2.0e9 || c2 >= 2.0e9)
      return fail(err, FKREG_ERR_UNSUPPORTED, "fine grid too large (more than 2^31 cells)");
  }

  // 1/phihat tables: type-1 per axis, then per bandwidth per axis (k >= 0 half)
  if (tab) {
    tab->clear();
    for (int j = 0; j < d; ++j) {
      phi1_off[j] = int64_t(tab->size());
      int64_t nk = g->modes[j] / 2;
      std::vector<double> ph(nk);
      spread_phihat(o->spread_kernel, w, beta, g->nf[j], nk, ph.data());
      for (int64_t k = 0; k < nk; ++k) tab->push_back(1.0 / ph[k]);
    }
    for (int b = 0; b < nbw; ++b)
      for (int j = 0; j < d; ++j) {
        bws[b].phi2_off[j] = int64_t(tab->size());
        int64_t nk = bws[b].K[j] / 2;
        std::vector<double> ph(nk);
        spread_phihat(o->spread_kernel, w, beta, bws[b].nf[j], nk, ph.data());
        for (int64_t k = 0; k < nk; ++k) tab->push_back(1.0 / ph[k]);
      }
  }
  if (bwv) *bwv = bws;
  if (geo) {
    std::memset(geo, 0, sizeof(*geo));
    geo->d = d;
    geo->w = w;
    geo->pad = (w + 1) / 2;
    geo->skind = o->spread_kernel;
    geo->beta = beta;
    for (int j = 0; j < 3; ++j) {
      geo->nf[j] = g->nf[j];
      geo->L[j] = g->ldft[j];
      geo->M[j] = (j < d) ? o->grid_n[j] : 1;
      geo->K[j] = g->modes[j];
      geo->P[j] = g->period[j];
      geo->lo[j] = (j < d) ? o->grid_lo[j] : 0;
      geo->hi[j] = (j < d) ? o->grid_hi[j] : 0;
      geo->inv_h[j] = g->inv_h[j];
      geo->inv_h_f[j] = float(g->inv_h[j]);
      geo->tile[j] = g->tile[j];
      geo->nbins[j] = g->nbins[j];
    }
    geo->kbits = key_local_bits(d, geo->tile, geo->nbins);
    geo->kern = FKREG_KERNEL_GAUSSIAN;
  }
  return FKREG_OK;
}

}  // namespace fk
