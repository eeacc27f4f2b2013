/*
 * FP64 direct-sum oracle for the binned kernel smoother of
 * "FKreg: A MATLAB toolbox for fast Multivariate Kernel Regression".
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA path and must never be used as a fallback for it.
 *
 * What it computes is the plain definition, written out with O(N) work per
 * query point and no approximation of any kind:
 *
 *   K_H(z)    = (2 pi)^(-d/2) |H|^(-1/2) exp(-z^T H^-1 z / 2)      (Sec. 1, eq. 2:
 *               the scaled kernel |h|^(-1/2) K(h^(-1/2) u) with Gaussian K)
 *   s_g(q)    = sum_i K_H(x_i - q) (x_i - q)^g         |g| <= 2l   (eq. 9)
 *   t_a(q)    = sum_i K_H(x_i - q) (x_i - q)^a y_i     |a| <= l    (eq. 9)
 *   mhat(q)   = e_1^T S(q)^-1 t(q),  S_ab = s_(a+b)               (eqs. 3, 11)
 *
 * The sign of the moment is (x_i - q), as in the design matrix of eq. 4; eq. 9
 * prints the opposite sign, which only flips odd moments and leaves mhat
 * unchanged.  Monomials z^g are enumerated by total degree, and inside one
 * degree as non-decreasing index tuples (1), (2), ..., (1,1), (1,2), ...
 * (the order of itertools.combinations_with_replacement).
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC -ffp-contract=off oracle.c -lm
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXD 3
#define OR_MAXMONO 35 /* degree <= 4 in 3-D */

/* Number of monomials of total degree <= deg in d variables: C(d+deg, deg). */
int or_nmono(int d, int deg) {
  long num = 1, den = 1;
  for (int k = 1; k <= deg; ++k) {
    num *= (d + k);
    den *= k;
  }
  return (int)(num / den);
}

/* Exponent table exps[m*d + j] of the m-th monomial. Returns the count. */
int or_monomials(int d, int deg, int* exps) {
  int m = 0;
  int idx[8];
  for (int k = 0; k <= deg; ++k) {
    /* all non-decreasing tuples idx[0..k-1] over {0..d-1} */
    for (int j = 0; j < k; ++j) idx[j] = 0;
    for (;;) {
      for (int j = 0; j < d; ++j) exps[m * d + j] = 0;
      for (int j = 0; j < k; ++j) exps[m * d + idx[j]] += 1;
      ++m;
      /* advance */
      int p = k - 1;
      while (p >= 0 && idx[p] == d - 1) --p;
      if (p < 0) break;
      idx[p] += 1;
      for (int j = p + 1; j < k; ++j) idx[j] = idx[p];
    }
  }
  return m;
}

/* Inverse and determinant of an SPD d x d matrix (d <= 3) by cofactors. */
static int inv_det(int d, const double* H, double* Hinv, double* det) {
  if (d == 1) {
    *det = H[0];
    if (!(H[0] > 0)) return -1;
    Hinv[0] = 1.0 / H[0];
    return 0;
  }
  if (d == 2) {
    double a = H[0], b = H[1], c = H[2], e = H[3];
    double D = a * e - b * c;
    *det = D;
    if (!(D > 0) || !(a > 0)) return -1;
    Hinv[0] = e / D;
    Hinv[1] = -b / D;
    Hinv[2] = -c / D;
    Hinv[3] = a / D;
    return 0;
  }
  /* d == 3 */
  double c00 = H[4] * H[8] - H[5] * H[7];
  double c01 = -(H[3] * H[8] - H[5] * H[6]);
  double c02 = H[3] * H[7] - H[4] * H[6];
  double D = H[0] * c00 + H[1] * c01 + H[2] * c02;
  *det = D;
  if (!(D > 0) || !(H[0] > 0)) return -1;
  double c10 = -(H[1] * H[8] - H[2] * H[7]);
  double c11 = H[0] * H[8] - H[2] * H[6];
  double c12 = -(H[0] * H[7] - H[1] * H[6]);
  double c20 = H[1] * H[5] - H[2] * H[4];
  double c21 = -(H[0] * H[5] - H[2] * H[3]);
  double c22 = H[0] * H[4] - H[1] * H[3];
  /* inverse = adjugate / det, adjugate = cofactor^T */
  Hinv[0] = c00 / D; Hinv[1] = c10 / D; Hinv[2] = c20 / D;
  Hinv[3] = c01 / D; Hinv[4] = c11 / D; Hinv[5] = c21 / D;
  Hinv[6] = c02 / D; Hinv[7] = c12 / D; Hinv[8] = c22 / D;
  return 0;
}

/* Gaussian density K_H at z (Sec. 1, scaled kernel with Gaussian K). */
double or_kernel(int d, const double* H, const double* z) {
  double Hinv[9], det;
  if (inv_det(d, H, Hinv, &det)) return NAN;
  double q = 0;
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) q += z[a] * Hinv[a * d + b] * z[b];
  return exp(-0.5 * q) / sqrt(pow(2.0 * M_PI, d) * det);
}

static void set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
}

/*
 * Moment sums (eq. 9) at nq query points for nstr strength vectors.
 *   x    [n][d]        sample locations
 *   c    [nstr][n]     strengths (1 for s-fields, y for t-fields)
 *   H    [d][d]        bandwidth matrix
 *   q    [nq][d]       query points (grid points or samples)
 *   out  [nq][nstr][nmono(d,deg)]
 * Returns 0, or -1 if H is not SPD.
 */
int or_moment_sums(int d, int64_t n, const double* x, int nstr, const double* c,
                   const double* H, int deg, int64_t nq, const double* q,
                   double* out, int nthreads) {
  double Hinv[9], det;
  if (d < 1 || d > OR_MAXD) return -2;
  if (inv_det(d, H, Hinv, &det)) return -1;
  const double norm = 1.0 / sqrt(pow(2.0 * M_PI, d) * det);
  const int nm = or_nmono(d, deg);
  int exps[OR_MAXMONO * OR_MAXD];
  or_monomials(d, deg, exps);
  set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t k = 0; k < nq; ++k) {
    double acc[16 * OR_MAXMONO];
    double* accp = acc;
    double* heap = NULL;
    if (nstr * nm > 16 * OR_MAXMONO) {
      heap = (double*)malloc(sizeof(double) * (size_t)nstr * nm);
      accp = heap;
    }
    memset(accp, 0, sizeof(double) * (size_t)nstr * nm);
    const double* qk = q + k * d;
    for (int64_t i = 0; i < n; ++i) {
      double z[OR_MAXD];
      for (int a = 0; a < d; ++a) z[a] = x[i * d + a] - qk[a];
      double e = 0;
      for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) e += z[a] * Hinv[a * d + b] * z[b];
      const double kv = norm * exp(-0.5 * e);
      for (int m = 0; m < nm; ++m) {
        double mono = kv;
        for (int a = 0; a < d; ++a)
          for (int p = 0; p < exps[m * d + a]; ++p) mono *= z[a];
        for (int s = 0; s < nstr; ++s) accp[s * nm + m] += mono * c[(int64_t)s * n + i];
      }
    }
    memcpy(out + k * (int64_t)nstr * nm, accp, sizeof(double) * (size_t)nstr * nm);
    free(heap);
  }
  return 0;
}

/*
 * The moment sums of or_moment_sums with the far pairs left out (the cutoff
 * mode for large N): a term with Mahalanobis radius z^T H^-1 z > r2max is
 * skipped.  With r2max = 2 ln(1e18) every skipped kernel value is below
 * 1e-18 K_H(0), beneath the FP64 rounding of any sum that holds a term near
 * its centre, so the result equals the full sum of eq. 9 to rounding.
 *
 * Neighbours are found through a uniform cell list over the samples (a
 * counting sort by cell, built here on every call).  The ellipse
 * z^T H^-1 z <= r2max lies in the box |z_j| <= sqrt(r2max H_jj); cells are at
 * least that wide per axis, so every neighbour of a query lies in the 3^d
 * cells around the query's own cell.  Inside a cell the samples keep their
 * input order.  Same arguments and output layout as or_moment_sums.
 * Returns 0, -1 if H is not SPD, -2 for a bad d or r2max, -3 if out of memory.
 */
int or_moment_sums_cutoff(int d, int64_t n, const double* x, int nstr, const double* c,
                          const double* H, int deg, int64_t nq, const double* q,
                          double r2max, double* out, int nthreads) {
  double Hinv[9], det;
  if (d < 1 || d > OR_MAXD || !(r2max > 0)) return -2;
  if (inv_det(d, H, Hinv, &det)) return -1;
  const double norm = 1.0 / sqrt(pow(2.0 * M_PI, d) * det);
  const int nm = or_nmono(d, deg);
  int exps[OR_MAXMONO * OR_MAXD];
  or_monomials(d, deg, exps);
  /* cell list: cell edge >= the half-width of the ellipse's bounding box */
  double lo[OR_MAXD] = {0, 0, 0}, cs[OR_MAXD] = {1, 1, 1};
  int64_t nc[OR_MAXD] = {1, 1, 1};
  for (int a = 0; a < d; ++a) {
    double mn = INFINITY, mx = -INFINITY;
    for (int64_t i = 0; i < n; ++i) {
      mn = fmin(mn, x[i * d + a]);
      mx = fmax(mx, x[i * d + a]);
    }
    if (n == 0) mn = mx = 0.0;
    lo[a] = mn;
    cs[a] = sqrt(r2max * H[a * d + a]) * (1.0 + 1e-9);
    nc[a] = (int64_t)floor((mx - mn) / cs[a]) + 1;
  }
  const int64_t cap = n > 0 ? 2 * n + 64 : 64;
  for (;;) {
    int64_t tot = 1;
    for (int a = 0; a < d; ++a) tot *= nc[a];
    if (tot <= cap) break;
    for (int a = 0; a < d; ++a) {
      cs[a] *= 2.0;
      nc[a] = nc[a] / 2 + 1;
    }
  }
  int64_t ncell = 1;
  for (int a = 0; a < d; ++a) ncell *= nc[a];
  int64_t* start = (int64_t*)calloc((size_t)ncell + 1, sizeof(int64_t));
  int64_t* cell_of = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!start || !cell_of || !order) {
    free(start);
    free(cell_of);
    free(order);
    return -3;
  }
  for (int64_t i = 0; i < n; ++i) {
    int64_t k = 0;
    for (int a = 0; a < d; ++a) {
      int64_t kj = (int64_t)floor((x[i * d + a] - lo[a]) / cs[a]);
      if (kj < 0) kj = 0;
      if (kj > nc[a] - 1) kj = nc[a] - 1;
      k = k * nc[a] + kj;
    }
    cell_of[i] = k;
    start[k + 1] += 1;
  }
  for (int64_t k = 0; k < ncell; ++k) start[k + 1] += start[k];
  {
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncell);
    if (!fill) {
      free(start);
      free(cell_of);
      free(order);
      return -3;
    }
    memcpy(fill, start, sizeof(int64_t) * (size_t)ncell);
    for (int64_t i = 0; i < n; ++i) order[fill[cell_of[i]]++] = i;
    free(fill);
  }
  set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t k = 0; k < nq; ++k) {
    double acc[16 * OR_MAXMONO];
    double* accp = acc;
    double* heap = NULL;
    if (nstr * nm > 16 * OR_MAXMONO) {
      heap = (double*)malloc(sizeof(double) * (size_t)nstr * nm);
      accp = heap;
    }
    memset(accp, 0, sizeof(double) * (size_t)nstr * nm);
    const double* qk = q + k * d;
    /* the 3^d cells around the query's cell, clipped to the list */
    int64_t klo[OR_MAXD] = {0, 0, 0}, khi[OR_MAXD] = {0, 0, 0};
    int empty = (n == 0);
    for (int a = 0; a < d; ++a) {
      const double f = floor((qk[a] - lo[a]) / cs[a]);
      const double fl = f - 1.0 < 0.0 ? 0.0 : f - 1.0;
      const double fh = f + 1.0 > (double)(nc[a] - 1) ? (double)(nc[a] - 1) : f + 1.0;
      if (fl > fh) empty = 1;
      klo[a] = (int64_t)fl;
      khi[a] = (int64_t)fh;
    }
    int64_t kk[OR_MAXD] = {klo[0], klo[1], klo[2]};
    while (!empty) {
      int64_t cell = 0;
      for (int a = 0; a < d; ++a) cell = cell * nc[a] + kk[a];
      for (int64_t p = start[cell]; p < start[cell + 1]; ++p) {
        const int64_t i = order[p];
        double z[OR_MAXD];
        for (int a = 0; a < d; ++a) z[a] = x[i * d + a] - qk[a];
        double e = 0;
        for (int a = 0; a < d; ++a)
          for (int b = 0; b < d; ++b) e += z[a] * Hinv[a * d + b] * z[b];
        if (e > r2max) continue;
        const double kv = norm * exp(-0.5 * e);
        for (int m = 0; m < nm; ++m) {
          double mono = kv;
          for (int a = 0; a < d; ++a)
            for (int pp = 0; pp < exps[m * d + a]; ++pp) mono *= z[a];
          for (int s = 0; s < nstr; ++s) accp[s * nm + m] += mono * c[(int64_t)s * n + i];
        }
      }
      /* next cell of the neighbourhood (last axis fastest) */
      int a = d - 1;
      while (a >= 0 && kk[a] == khi[a]) {
        kk[a] = klo[a];
        --a;
      }
      if (a < 0) break;
      kk[a] += 1;
    }
    memcpy(out + k * (int64_t)nstr * nm, accp, sizeof(double) * (size_t)nstr * nm);
    free(heap);
  }
  free(start);
  free(cell_of);
  free(order);
  return 0;
}

/* Position of the monomial with exponent vector e inside the table. */
static int mono_index(int d, int nm, const int* exps, const int* e) {
  for (int m = 0; m < nm; ++m) {
    int ok = 1;
    for (int a = 0; a < d; ++a) ok &= (exps[m * d + a] == e[a]);
    if (ok) return m;
  }
  return -1;
}

/*
 * Solve S a = r for a p x p system by Gaussian elimination with partial
 * pivoting (FP64).  Returns 0, or -1 if a pivot is exactly zero.
 */
static int gauss_solve(int p, double* S, double* r) {
  for (int col = 0; col < p; ++col) {
    int piv = col;
    for (int row = col + 1; row < p; ++row)
      if (fabs(S[row * p + col]) > fabs(S[piv * p + col])) piv = row;
    if (S[piv * p + col] == 0.0) return -1;
    if (piv != col) {
      for (int j = 0; j < p; ++j) {
        double t = S[col * p + j];
        S[col * p + j] = S[piv * p + j];
        S[piv * p + j] = t;
      }
      double t = r[col];
      r[col] = r[piv];
      r[piv] = t;
    }
    for (int row = col + 1; row < p; ++row) {
      double f = S[row * p + col] / S[col * p + col];
      for (int j = col; j < p; ++j) S[row * p + j] -= f * S[col * p + j];
      r[row] -= f * r[col];
    }
  }
  for (int row = p - 1; row >= 0; --row) {
    double v = r[row];
    for (int j = row + 1; j < p; ++j) v -= S[row * p + j] * r[j];
    r[row] = v / S[row * p + row];
  }
  return 0;
}

/*
 * Local-polynomial estimate from moment sums (eqs. 3, 11):
 *   s   [nq][nmono(d,2l)]         s-fields at each query point
 *   t   [nq][nrhs][nmono(d,l)]    t-fields
 *   mhat[nq][nrhs]                e_1^T S^-1 t (NaN where S is singular)
 *   sinv11[nq] (optional)          [S^-1]_11, so S_ii = K_H(0) [S^-1]_11 at a sample
 */
int or_lpr_solve(int d, int order, int64_t nq, const double* s, int nrhs,
                 const double* t, double* mhat, double* sinv11) {
  const int p = or_nmono(d, order);
  const int ns = or_nmono(d, 2 * order);
  int exps[OR_MAXMONO * OR_MAXD];
  or_monomials(d, 2 * order, exps);
  int sidx[16 * 16];
  for (int a = 0; a < p; ++a)
    for (int b = 0; b < p; ++b) {
      int e[OR_MAXD];
      for (int j = 0; j < d; ++j) e[j] = exps[a * d + j] + exps[b * d + j];
      sidx[a * p + b] = mono_index(d, ns, exps, e);
    }
  for (int64_t k = 0; k < nq; ++k) {
    double S[16 * 16], Sc[16 * 16], r[16];
    for (int a = 0; a < p * p; ++a) S[a] = s[k * ns + sidx[a]];
    for (int q = 0; q < nrhs; ++q) {
      memcpy(Sc, S, sizeof(double) * p * p);
      for (int a = 0; a < p; ++a) r[a] = t[(k * nrhs + q) * p + a];
      mhat[k * nrhs + q] = gauss_solve(p, Sc, r) ? NAN : r[0];
    }
    if (sinv11) {
      memcpy(Sc, S, sizeof(double) * p * p);
      for (int a = 0; a < p; ++a) r[a] = (a == 0);
      sinv11[k] = gauss_solve(p, Sc, r) ? NAN : r[0];
    }
  }
  return 0;
}

/*
 * SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): one 64-bit output per counter value.
 */
static uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/*
 * Counter-based Gaussian probes for the Monte-Carlo DF estimate (Sec. 2.1,
 * step i; the paper leaves the generator open).  Word k >= 1 of the SplitMix64
 * stream seeded with `seed` is splitmix64(seed + (k - 1) gamma), gamma the
 * generator's increment.  Probes come in Box-Muller pairs (Box & Muller,
 * 1958): for pair j = p / 2 and ORIGINAL sample index i, with
 * c = (j << 40) | i, the two words
 *   a = word 2c + 1,  b = word 2c + 2
 * give u1 = ((a >> 11) + 1) 2^-53 in (0, 1], u2 = (b >> 11) 2^-53 in [0, 1),
 * r = sqrt(-2 ln u1), and
 *   probe 2j = r cos(2 pi u2),  probe 2j + 1 = r sin(2 pi u2).
 * out[p][i] for p < np, i < n (an odd np uses the cosine of its last pair).
 */
#define OR_GAMMA 0x9E3779B97F4A7C15ULL

static void or_probe_words(uint64_t seed, int p, int64_t i, uint64_t* a, uint64_t* b) {
  const uint64_t c = ((uint64_t)(p >> 1) << 40) | (uint64_t)i;
  *a = splitmix64(seed + (2 * c) * OR_GAMMA);
  *b = splitmix64(seed + (2 * c + 1) * OR_GAMMA);
}

void or_probes(uint64_t seed, int np, int64_t n, double* out) {
  for (int p = 0; p < np; ++p)
    for (int64_t i = 0; i < n; ++i) {
      uint64_t a, b;
      or_probe_words(seed, p, i, &a, &b);
      const double u1 = ((double)(a >> 11) + 1.0) * 0x1.0p-53;
      const double u2 = (double)(b >> 11) * 0x1.0p-53;
      const double r = sqrt(-2.0 * log(u1)), t = 2.0 * M_PI * u2;
      out[(int64_t)p * n + i] = (p & 1) ? r * sin(t) : r * cos(t);
    }
}

/*
 * The same probes evaluated in single precision (the generator an FP32 plan
 * draws on the device): the same words, 24-bit uniforms
 * u1 = ((a >> 40) + 1) 2^-24, u2 = (b >> 40) 2^-24, Box-Muller in float.
 */
void or_probes_f32(uint64_t seed, int np, int64_t n, float* out) {
  for (int p = 0; p < np; ++p)
    for (int64_t i = 0; i < n; ++i) {
      uint64_t a, b;
      or_probe_words(seed, p, i, &a, &b);
      const float u1 = (float)((uint32_t)(a >> 40) + 1u) * 0x1.0p-24f;
      const float u2 = (float)(uint32_t)(b >> 40) * 0x1.0p-24f;
      const float r = sqrtf(-2.0f * logf(u1)), t = 2.0f * (float)M_PI * u2;
      out[(int64_t)p * n + i] = (p & 1) ? r * sinf(t) : r * cosf(t);
    }
}

uint64_t or_splitmix64(uint64_t z) { return splitmix64(z); }
