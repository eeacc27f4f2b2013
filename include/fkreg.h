/*
 * fkreg.h - C ABI of the GB300 NUFFT kernel smoother.
 *
 * The library computes, for N scattered samples x_i in R^d (d = 1..3) with
 * responses y_i, the local-polynomial kernel regression of
 * "FKreg: A MATLAB toolbox for fast Multivariate Kernel Regression":
 *
 *   s_g(q) = sum_i K_H(x_i - q) (x_i - q)^g        |g| <= 2l   (Sec. 1.1, eq. 9)
 *   t_a(q) = sum_i K_H(x_i - q) (x_i - q)^a y_i    |a| <= l    (eq. 9)
 *   mhat(q) = e_1^T S(q)^-1 t(q),   S_ab = s_(a+b)             (eqs. 3, 11)
 *
 * with the Gaussian kernel K_H(z) = (2 pi)^(-d/2) |H|^(-1/2) exp(-z^T H^-1 z / 2)
 * (the scaled kernel of Sec. 1), at the points q of a uniform grid (eq. 6) and
 * at the samples themselves.  The sums are evaluated to a requested tolerance
 * by type-1 NUFFT spreading (Sec. 1.2, eqs. 16-20), a Fourier-domain multiply
 * by the transform of the moment kernels z^g K_H(z), and inverse FFTs
 * (eq. 21); values at the samples use the type-2 (uniform to non-uniform)
 * NUFFT that Sec. 1.1 mentions.  On top of the sums the library gives the
 * fast Monte-Carlo trace of the smoother matrix (Sec. 2.1), GCV (eq. 22) and
 * the conditional-variance pass (eq. 23).
 *
 * Conventions shared by every call:
 *  - Every pointer named *_dev is DEVICE memory owned by the caller.  The
 *    library never allocates device memory: all scratch lives in the
 *    workspace the caller hands to fkreg_set_workspace.  Host pointers are
 *    read during the call only.
 *  - Every call that takes a `stream` (a cudaStream_t passed as void*; NULL =
 *    legacy default stream) is asynchronous on that stream.  Results are valid
 *    after the stream is synchronised.
 *  - No call aborts, traps or prints.  Argument errors return immediately with
 *    a status and a message in fkreg_last_error().  Errors detected on the
 *    device (a sample outside the grid box or not finite) set an error word
 *    that fkreg_sync_status() reports as FKREG_ERR_DEVICE.
 *  - Arrays are C-contiguous.  Samples are [n][d] (row-major, "AoS").  Grid
 *    arrays are [..., M_1, ..., M_d] with the last axis fastest.  Complex
 *    values are interleaved (re, im).  The floating type of every float
 *    array is the plan's precision: float for FKREG_F32, double for FKREG_F64.
 *  - Monomials z^g are ordered by total degree and, inside one degree, as
 *    non-decreasing index tuples: 1, z1, .., zd, z1 z1, z1 z2, .., zd zd.
 *    ns = C(d + 2l, 2l) s-fields and nt = C(d + l, l) t-fields per response.
 */
#ifndef FKREG_H
#define FKREG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fkreg_plan_s* fkreg_plan;

typedef enum {
  FKREG_OK = 0,
  FKREG_ERR_INVALID_ARG = 1,  /* bad sizes, non-SPD H, NULL where required   */
  FKREG_ERR_UNSUPPORTED = 2,  /* a valid request this build does not handle  */
  FKREG_ERR_WORKSPACE = 3,    /* workspace missing, too small or misaligned  */
  FKREG_ERR_CUDA = 4,         /* a CUDA runtime call failed                  */
  FKREG_ERR_CUFFT = 5,        /* a cuFFT call failed                         */
  FKREG_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up          */
  FKREG_ERR_DEVICE = 7,       /* device flagged a bad sample (NaN, outside)  */
  FKREG_ERR_STATE = 8         /* call order violated (e.g. smooth before set_points) */
} fkreg_status;

enum { FKREG_F32 = 0, FKREG_F64 = 1 };
enum { FKREG_SPREAD_ES = 0, FKREG_SPREAD_GAUSS = 1 };
enum {
  FKREG_KERNEL_GAUSSIAN = 0,
  /* compact radial kernels on the unit ball of u = H^(-1/2) z (Table 1; Sec. 1) */
  FKREG_KERNEL_UNIFORM = 1,       /* k = 1                                     */
  FKREG_KERNEL_EPANECHNIKOV = 2,  /* k = 1 - |u|^2                             */
  FKREG_KERNEL_TRIANGLE = 3,      /* k = 1 - |u|                               */
  FKREG_KERNEL_BIWEIGHT = 4,      /* k = (1 - |u|^2)^2                         */
  FKREG_KERNEL_TRIWEIGHT = 5,     /* k = (1 - |u|^2)^3                         */
  FKREG_KERNEL_GAUSSIAN_DIRECT = 6 /* the Gaussian by direct sums (see below)   */
};

/* fkreg_opts.flags */
enum {
  FKREG_GCV_EXACT_TRACE = 1,  /* GCV uses the exact trace K_H(0) sum_i [S(x_i)^-1]_11
                                 instead of Girard's Monte-Carlo estimate */
  FKREG_WANT_BACKWARD = 2     /* reserve workspace and FFT plans for fkreg_backward */
};

/*
 * Problem description (the arguments of cv_fkreg in Sec. 4 and Table 1).
 *   dim            d, 1..3
 *   order          l: 0 = Nadaraya-Watson (eq. 7), 1 = local linear (eq. 3),
 *                  2 = local quadratic (d <= 2; 3-D and its backward are
 *                  refused with UNSUPPORTED)
 *   kernel         FKREG_KERNEL_GAUSSIAN: the NUFFT path (the transform of the
 *                  Gaussian moment kernels decays fast enough for tol to
 *                  control the truncation).  The compact kernels
 *                  (FKREG_KERNEL_UNIFORM ... TRIWEIGHT, normalised to unit
 *                  mass in d dimensions, K_H(z) = |H|^(-1/2) K(H^(-1/2) z))
 *                  use exact direct sums over the binned samples inside each
 *                  point's support instead (tol and spread_kernel unused);
 *                  fkreg_backward and FKREG_WANT_BACKWARD are refused for
 *                  them, and so is a plan whose s-fields plus the t-fields
 *                  of (n_rhs + max_probes) strengths exceed 64 (UNSUPPORTED).
 *                  FKREG_KERNEL_GAUSSIAN_DIRECT is the Gaussian kernel of
 *                  FKREG_KERNEL_GAUSSIAN evaluated by the same direct sums,
 *                  over the samples within Mahalanobis distance R of each
 *                  point, R^2 = 2 ln(10 / tol): every dropped term is below
 *                  tol / 10 of K_H(0).  It needs no Fourier grid, so it
 *                  serves bandwidths so narrow that few samples fall within
 *                  R (fkreg_sweep chooses it per group by its cost model);
 *                  the limits of the compact kernels apply.
 *   spread_kernel  NUFFT spreading kernel: exponential of semicircle (default)
 *                  or the Gaussian of Sec. 1.2 eq. 17 (about twice as wide)
 *   precision      FKREG_F32 (spreading, FFT, interpolation in float, FP64
 *                  per-point solves and reductions) or FKREG_F64 (all double)
 *   y_complex      0: real responses; 1: complex responses (interleaved)
 *   grid_n/lo/hi   the grid of eq. 6 per axis: grid_n[j] >= 2 points from
 *                  grid_lo[j] to grid_hi[j], endpoints included.  Samples
 *                  must lie inside [lo, hi] (callers clip beforehand).
 *   n_bw, H        host array [n_bw][d][d] of SPD bandwidth matrices (a
 *                  per-axis standard deviation sigma_j means H = diag(sigma^2))
 *   n_rhs          responses that share the geometry (stacked right-hand sides)
 *   max_probes     largest number of Monte-Carlo probes a later fkreg_df uses
 *   tol            NUFFT tolerance (e.g. 1e-6 for F32, 1e-12 for F64)
 *   mask_rho       grid points with s_0(g) < mask_rho * max_g s_0 are masked
 *                  (NaN estimate, mask byte 0); 0 selects the default 1e-3
 *   tile           spreading tile edge in fine-grid cells per axis (0 = auto:
 *                  for the compact kernels a quarter of the widest support
 *                  half-width, in grid cells)
 *   flags          FKREG_GCV_EXACT_TRACE, FKREG_WANT_BACKWARD
 */
typedef struct {
  int dim;
  int order;
  int kernel;
  int spread_kernel;
  int precision;
  int y_complex;
  int64_t grid_n[3];
  double grid_lo[3];
  double grid_hi[3];
  int n_bw;
  const double* H;
  int n_rhs;
  int max_probes;
  double tol;
  double mask_rho;
  int tile;
  int flags;
} fkreg_opts;

/*
 * Geometry the planner derives (host only; for inspection and tests).
 *   delta[j]   grid spacing (hi - lo) / (M_j - 1)            (eq. 6)
 *   period[j]  P_j = L_j delta_j >= (hi - lo) + kernel tail: the period of the
 *              Fourier series, chosen so no wrap-around reaches the box
 *              (the role of the zero padding of eq. 18)
 *   ldft[j]    L_j, length of the inverse DFT onto the grid lattice (eq. 21)
 *   modes[j]   K_j, even; Fourier modes |k_j| <= K_j/2 - 1 are kept
 *   nf[j]      fine (oversampled) grid of the type-1 spreading, >= 2 K_j
 *   w, beta    spreading width in fine cells and ES shape parameter
 *   tile[j]    spreading tile edge; nbins[j] = ceil(nf / tile)
 *   inv_h[j]   the factor nf_j / P_j that maps x - lo to fine-grid units,
 *              rounded to the plan precision (the bin rule uses it)
 */
typedef struct {
  int dim;
  double delta[3];
  double period[3];
  int64_t ldft[3];
  int64_t modes[3];
  int64_t nf[3];
  int w;
  double beta;
  int64_t tile[3];
  int64_t nbins[3];
  double inv_h[3];
  int ns;          /* s-fields */
  int nt;          /* t-fields per response */
} fkreg_geometry;

/*
 * Output buffers of fkreg_smooth / fkreg_df (device; any may be NULL).
 *   mhat_grid  [n_bw][n_rhs][M]   estimate of eq. 11 on the grid (complex if y_complex)
 *   mask       [n_bw][M] uint8    1 where s_0(g) >= mask_rho * max s_0
 *   moments    [n_bw][ns + n_rhs*nt][M]  s-fields then t-fields of eq. 9 on the
 *              grid (t-fields complex if y_complex)
 *   mhat_at_x  [n_bw][n_rhs][n]   (S_h y)_i at the samples, ORIGINAL order
 *   rss        [n_bw][n_rhs] double  ||y - S_h y||^2 (numerator of eq. 22)
 *   trace      [n_bw][3] double   Girard estimate N mean_p(w^T S w / w^T w)
 *              (Sec. 2.1), Hutchinson mean_p w^T S w, and the exact trace
 *              K_H(0) sum_i [S(x_i)^-1]_11 (fkreg_df only)
 *   gcv        [n_bw][n_rhs] double  eq. 22 (fkreg_df only)
 */
typedef struct {
  void* mhat_grid;
  uint8_t* mask;
  void* moments;
  void* mhat_at_x;
  double* rss;
  double* trace;
  double* gcv;
} fkreg_outputs;

/* Host-only: validate opts and compute the geometry. No CUDA call is made. */
fkreg_status fkreg_geometry_query(const fkreg_opts* opts, fkreg_geometry* out);

/*
 * Host-only: the Fourier transform of the spreading kernel,
 * phihat[k] = integral over |z| <= w/2 of phi(z) cos(2 pi k z / nf) dz for
 * k = 0..nk-1 (Gauss-Legendre quadrature in FP64).  The deconvolution of
 * eq. 20 divides by it.  kind: FKREG_SPREAD_ES or FKREG_SPREAD_GAUSS.
 */
fkreg_status fkreg_spread_kernel_ft(int kind, int w, double beta, int64_t nf,
                                    int64_t nk, double* phihat);

/*
 * Device: the spreading kernel phi(z) of Sec. 1.2 (eq. 17 for
 * FKREG_SPREAD_GAUSS, the exponential of semicircle for FKREG_SPREAD_ES) at
 * n offsets z_dev[i] (fine cells), evaluated by the same device function the
 * spreading and interpolation kernels call, in `precision` (FKREG_F32: float
 * z and out, FKREG_F64: double).  out_dev[i] = phi(z_dev[i]), 0 outside
 * |z| <= w/2.  One launch on `stream`; no synchronisation.  Returns
 * FKREG_ERR_INVALID_ARG for a bad kind, precision, w outside [2, 32], n < 0
 * or a NULL pointer with n > 0, FKREG_ERR_CUDA if the launch fails.
 */
fkreg_status fkreg_spread_kernel_values(int kind, int w, double beta, int precision, int64_t n,
                                        const void* z_dev, void* out_dev, void* stream);

/*
 * Create a plan for up to max_n samples.  Computes the geometry and the
 * spreading-kernel tables on the host and creates the cuFFT plans (needs a
 * current CUDA device).  The plan owns host tables, cuFFT handles, and one
 * non-blocking CUDA stream with two events on the current device: a
 * fkreg_smooth / fkreg_df call on at least 65,536 samples that wants both
 * grid and at-sample outputs runs its grid branch on that stream, forked from the caller's stream and
 * joined back into it before the call returns (so every call stays ordered
 * on the caller's stream, and a stream capture records the two branches).
 * It allocates no device memory.
 */
fkreg_status fkreg_plan_create(const fkreg_opts* opts, int64_t max_n, fkreg_plan* out);

/* Bytes of device workspace the plan needs (256-byte aligned start). */
fkreg_status fkreg_workspace_bytes(fkreg_plan plan, size_t* bytes);

/* Hand the plan its workspace and upload the small tables (async on stream). */
fkreg_status fkreg_set_workspace(fkreg_plan plan, void* ws_dev, size_t bytes, void* stream);

/*
 * Bin and sort the samples x_dev [n][d] (plan precision), n <= max_n.
 * With u_j = fl(fl(x_j - lo_j) * inv_h_j) (round-to-nearest IEEE operations,
 * no fused multiply-add) each sample gets
 *   the bin of its fine-grid cell c_j = min(floor(u_j), nf_j - 1):
 *     b_j = c_j / tile_j, bin = row-major index of b over nbins;
 *   the centre cell of its spreading window, relative to the bin,
 *     e_j = clamp(ceil(fl(u_j - w/2)) + floor(w/2) - b_j tile_j, 0, tile_j),
 *     local = serpentine index of e over (tile_j + 1) values per axis:
 *     local_0 = e_0, local_j = local_(j-1) (tile_j + 1) + e'_j with
 *     e'_j = tile_j - e_j if local_(j-1) is odd, else e_j;
 * and the key (bin << kbits) | local, kbits = bits of prod_j (tile_j + 1)
 * (kbits = 0, i.e. bin-only keys, if the key would exceed 32 bits).  A stable
 * counting sort orders the samples by key, then by original index: the
 * permutation is unique and bit-exact, bins are contiguous, and samples that
 * share a window are adjacent.  All later calls share this geometry until
 * the next fkreg_set_points.
 */
fkreg_status fkreg_set_points(fkreg_plan plan, int64_t n, const void* x_dev, void* stream);

/*
 * Copy the sort result: perm_dev[s] = original index of the s-th sorted
 * sample (uint32, n entries) and bin_start_dev (uint32, nbins+1 entries,
 * exclusive prefix sum of the bin counts).  Either pointer may be NULL.
 */
fkreg_status fkreg_get_sort(fkreg_plan plan, uint32_t* perm_dev, uint32_t* bin_start_dev,
                            int64_t* nbins, void* stream);

/*
 * Smooth the responses y_dev [n_rhs][n] (complex interleaved if y_complex)
 * for every bandwidth of the plan: grid estimates and/or values at the
 * samples, per the non-NULL members of `out` (trace and gcv are ignored).
 */
fkreg_status fkreg_smooth(fkreg_plan plan, const void* y_dev, const fkreg_outputs* out,
                          void* stream);

/*
 * Smooth y together with n_probes Gaussian probe vectors w_p (Sec. 2.1) and
 * return the DF estimates and GCV (eq. 22) for every bandwidth, plus any of
 * the smoothing outputs.  probes_dev [n_probes][n] (plan precision, ORIGINAL
 * sample order) or NULL: then the probes are drawn on the device in
 * Box-Muller pairs from the SplitMix64 stream seeded with `seed` (word k >= 1
 * is splitmix64(seed + (k - 1) gamma), gamma = 0x9E3779B97F4A7C15): pair
 * j = p / 2 of original sample i takes the words a = 2c + 1 and b = 2c + 2,
 * c = (j << 40) | i, and gives probes 2j and 2j + 1 as r cos(2 pi u2) and
 * r sin(2 pi u2), r = sqrt(-2 ln u1), in the plan precision:
 * FKREG_F64: u1 = ((a >> 11) + 1) 2^-53, u2 = (b >> 11) 2^-53;
 * FKREG_F32: u1 = ((a >> 40) + 1) 2^-24, u2 = (b >> 40) 2^-24.
 * n_probes <= max_probes.
 */
fkreg_status fkreg_df(fkreg_plan plan, const void* y_dev, int n_probes, uint64_t seed,
                      const void* probes_dev, const fkreg_outputs* out, void* stream);

/*
 * Conditional-variance pass (Sec. 3, eq. 23): smooth r_i = |y_i - mhat(x_i)|^2
 * with the plan's order and bandwidths, reusing the s-field spectrum of the
 * last fkreg_smooth / fkreg_df on these points.  mhat_at_x_dev is that call's
 * mhat_at_x output [n_bw][n_rhs][n] (original order); bandwidth b's residuals
 * are smoothed with bandwidth b.  sigma2_grid_dev [n_bw][n_rhs][M] (real).
 */
fkreg_status fkreg_variance(fkreg_plan plan, const void* y_dev, const void* mhat_at_x_dev,
                            void* sigma2_grid_dev, void* stream);

/*
 * Log-variance estimator of Sec. 3 (eqs. 24-26), for real responses:
 *   l_i      = log(r_i + 1/N),  r_i = (y_i - mhat(x_i))^2         (eq. 25)
 *   v(q)     = the plan's local-polynomial smooth of l at q        (eq. 25)
 *   kappa    = [ (1/N) sum_i r_i exp(-v(x_i)) ]^-1
 *   sigma2(q)= exp(v(q)) / kappa > 0                               (eq. 26)
 * with bandwidth b's residuals smoothed with bandwidth b and the s-field
 * spectrum of the last fkreg_smooth / fkreg_df on these points reused.
 *   y_dev           [n_rhs][n] responses (plan precision, original order)
 *   mhat_at_x_dev   [n_bw][n_rhs][n] that call's mhat_at_x output
 *   v_grid_dev      out [n_bw][n_rhs][M]: v on the grid (NaN where masked)
 *   v_at_x_dev      out [n_bw][n_rhs][n]: v at the samples (original order)
 *   kappa_dev       out [n_bw][n_rhs] FP64
 *   sigma2_grid_dev out [n_bw][n_rhs][M] or NULL
 * All pointers but sigma2_grid_dev are required; n >= 1.  Complex
 * responses return FKREG_ERR_UNSUPPORTED.  The call overwrites the plan's
 * internal strength, field and partial-sum buffers (not the caller's
 * outputs of earlier calls).
 */
fkreg_status fkreg_log_variance(fkreg_plan plan, const void* y_dev, const void* mhat_at_x_dev,
                                void* v_grid_dev, void* v_at_x_dev, double* kappa_dev,
                                void* sigma2_grid_dev, void* stream);

/*
 * Pointwise 100(1 - alpha) % interval of eq. 28: lower/upper =
 * mhat -/+ z_(1 - alpha/2) sqrt(var), z the standard normal quantile, for
 * count elements (any layout; typically a grid estimate and the variance
 * estimate of fkreg_variance or fkreg_log_variance, or a scalar variance
 * broadcast by the caller).  A negative or NaN variance gives NaN bounds.
 * precision FKREG_F32 / FKREG_F64 is the element type of all four arrays.
 * 0 < alpha < 1, else FKREG_ERR_INVALID_ARG.  No plan is needed.
 */
fkreg_status fkreg_interval(int precision, int64_t count, const void* mhat_dev,
                            const void* var_dev, double alpha, void* lower_dev, void* upper_dev,
                            void* stream);

/*
 * Values of grid estimates at new points (the grid-to-point interpolation
 * the paper applies to its grid estimates, Sec. 1.1).
 *   precision        FKREG_F32 / FKREG_F64: element type of grid, xq and out
 *   dim, grid_n/lo/hi the lattice of eq. 6 (host arrays of dim entries)
 *   grid_dev         [count][M_1..M_dim] device, last axis fastest (e.g. the
 *                    mhat_grid output: count = n_bw * n_rhs)
 *   xq_dev           [nq][dim] device query points
 *   method           0: multilinear, extended linearly from the boundary
 *                    cell outside the box; 1: cubic convolution (Keys 1981,
 *                    a = -1/2) with Keys' boundary rows, NaN outside the box
 *   out_dev          [count][nq] device
 * Needs grid_n[j] >= 2 (linear) or >= 4 (cubic).  NaN grid values (masked
 * points) propagate to the queries that use them.  No plan is needed.
 */
fkreg_status fkreg_predict(int precision, int dim, const int64_t* grid_n, const double* grid_lo,
                           const double* grid_hi, int count, const void* grid_dev, int64_t nq,
                           const void* xq_dev, int method, void* out_dev, void* stream);

/*
 * Gradient of GCV (eq. 22) for bandwidth b, with the Monte-Carlo trace of
 * Sec. 2.1 over n_probes fixed probes (given, or drawn as in fkreg_df from
 * seed), with respect to the log bandwidths, the responses and the samples.
 * Runs the forward fkreg_df itself, then the hand-written backward: the
 * adjoints of the moment fields at the samples (FP64 per-sample solves),
 * derivative fields for d/dlog sigma_j and the evaluation-point gradient, and
 * one adjoint spreading pass (the adjoint of type-2 interpolation is type-1
 * spreading) for the source-side d/dx and for d/dy.
 * Requires a plan created with FKREG_WANT_BACKWARD, n_rhs = 1, real y,
 * diagonal H (H = diag(sigma^2), the derivative is in log sigma_j) and the
 * Monte-Carlo trace (no FKREG_GCV_EXACT_TRACE); otherwise
 * FKREG_ERR_UNSUPPORTED.
 *   y_dev       [n] responses;  probes_dev [n_probes][n] or NULL (seeded)
 *   gcv_dev     double, the GCV value of bandwidth b (may be NULL)
 *   dlogh_dev   [dim] double, dGCV / dlog sigma_j (may be NULL)
 *   dy_dev      [n] dGCV / dy_i, original order (may be NULL)
 *   dx_dev      [n][dim] dGCV / dx_i, original order (may be NULL)
 */
fkreg_status fkreg_backward(fkreg_plan plan, const void* y_dev, int n_probes, uint64_t seed,
                            const void* probes_dev, int b, double* gcv_dev, double* dlogh_dev,
                            void* dy_dev, void* dx_dev, void* stream);

/*
 * Vector-Jacobian product of the grid estimate (eqs. 3, 9, 11) of bandwidth b:
 * for L = sum_r sum_g Gbar_r(g) mhat_r(g) over the unmasked grid points, the
 * gradients of L with respect to the log bandwidths, the responses and the
 * samples.  Runs the forward grid path itself (spreading, FFT, kernel
 * multiply, inverse FFT, the FP64 per-grid-point solves and the mask), then
 * the hand-written backward: the adjoint of each grid point's solve
 * (dmhat = a^T dt - a^T dS S^-1 t with a = S^-1 e_1) as adjoint fields on the
 * grid lattice, their forward DFT (the adjoint of the inverse DFT onto the
 * grid), the kernel multipliers and a type-2 evaluation at the samples (the
 * adjoint of type-1 spreading) for dy and the x-gradient, and a spectral
 * inner product with the derivative of the kernel transform for d/dlog sigma.
 * Requires a plan created with FKREG_WANT_BACKWARD, the Gaussian kernel, real
 * responses, order 0 or 1 and a diagonal H for bandwidth b (the derivative is
 * in log sigma_j, H = diag(sigma^2)); otherwise FKREG_ERR_UNSUPPORTED.
 *   y_dev         [n_rhs][n] responses (plan precision, original order)
 *   grad_mhat_dev [n_rhs][M] dL/dmhat on the grid of bandwidth b (plan
 *                 precision); values at masked points and non-finite values
 *                 are ignored
 *   dlogh_dev     [dim] double, dL/dlog sigma_j (may be NULL)
 *   dy_dev        [n_rhs][n] dL/dy, original order (may be NULL)
 *   dx_dev        [n][dim] dL/dx, original order (may be NULL)
 * The call overwrites the plan's internal buffers (a later fkreg_variance
 * needs a new fkreg_smooth / fkreg_df first).
 */
fkreg_status fkreg_backward_grid(fkreg_plan plan, const void* y_dev, const void* grad_mhat_dev,
                                 int b, double* dlogh_dev, void* dy_dev, void* dx_dev,
                                 void* stream);

/*
 * Stage timers (profiling).  With timing enabled every stage of a call is
 * bracketed by CUDA events recorded on the call's stream; fkreg_stage_times
 * waits for those events, returns the accumulated milliseconds and launch
 * counts per stage since the previous query (arrays of FKREG_N_STAGES, either
 * may be NULL) and resets them.  kernel_launches (may be NULL) receives the
 * number of this library's own kernel launches since the previous query
 * (cuFFT's kernels are not counted).  Timing adds two event records per stage.
 */
enum {
  FKREG_STAGE_SORT = 0,       /* bin keys, radix sort, bin offsets, sorted coordinates */
  FKREG_STAGE_STRENGTHS = 1,  /* responses / probes / residuals in sorted order */
  FKREG_STAGE_SPREAD = 2,     /* type-1 spreading */
  FKREG_STAGE_FFT_FWD = 3,    /* cuFFT forward of the fine grids */
  FKREG_STAGE_KMUL_GRID = 4,  /* kernel multiply + fold for the grid lattice */
  FKREG_STAGE_FFT_GRID = 5,   /* cuFFT inverse onto the lattice */
  FKREG_STAGE_GRID_SOLVE = 6, /* FP64 per-grid-point solves */
  FKREG_STAGE_KMUL_T2 = 7,    /* kernel multiply + deconvolution for type-2 */
  FKREG_STAGE_FFT_T2 = 8,     /* cuFFT inverse onto the type-2 fine grids */
  FKREG_STAGE_INTERP = 9,     /* interpolation at the samples + solves + reductions */
  FKREG_STAGE_FINALIZE = 10,  /* DF / GCV */
  FKREG_STAGE_BACKWARD = 11,  /* derivative fields, adjoints, adjoint spreading */
  FKREG_N_STAGES = 12
};
fkreg_status fkreg_set_timing(fkreg_plan plan, int enable);
fkreg_status fkreg_stage_times(fkreg_plan plan, double* ms, int64_t* launches,
                               int64_t* kernel_launches);

/*
 * Allocation-free stable bin sort.  The paper has no counterpart: this is an
 * entry point for callers that cannot allocate device memory while they run
 * (a host program whose memory pool owns every device byte, a plug-in that
 * is handed buffers but no allocator, a loop that forbids allocation after
 * start-up).  It computes the same permutation and bin offsets as
 * fkreg_set_points + fkreg_get_sort, but keeps its scratch in a device array
 * that the library owns (about 4.3 MB, held on every GPU that loads the
 * library until the process exits) instead of a workspace.
 *   geom           geometry from fkreg_geometry_query (dim, nf, w, tile,
 *                  nbins, inv_h are used; 2 <= w <= 32)
 *   grid_lo/hi     host [dim], the grid box of the plan options
 *   precision      FKREG_F32 or FKREG_F64: the type of x_dev
 *   n              samples, 0 <= n <= 262144 (2^18); at most 65536 bins
 *   x_dev          [n][dim] samples (device)
 *   perm_dev       [n] uint32 out: original index of the s-th sorted sample
 *   bin_start_dev  [nbins + 1] uint32 out: exclusive prefix sum of bin counts
 *   bad_dev        optional int32 out: 1 if a sample lay outside the box or
 *                  was not finite (it is then sorted into the first bin along
 *                  that axis), else 0
 * Larger n or more bins return FKREG_ERR_INVALID_ARG before anything runs.
 * The call allocates nothing.  Outside a stream capture every call looks up
 * the array's device address (cudaGetSymbolAddress) with the current device,
 * so a device reset that reloads the library's module is followed; inside a
 * capture the address found by an earlier call on that device is used, so
 * make the first call on a device before any stream capture.  Every call on a device
 * shares the one array and the array keeps the previous call's contents
 * (the call clears what must start at zero), so calls whose work overlaps on
 * the GPU (other streams, other host threads) race: serialise them.
 */
fkreg_status fkreg_bin_sort_static(const fkreg_geometry* geom, const double* grid_lo,
                                   const double* grid_hi, int precision, int64_t n,
                                   const void* x_dev, uint32_t* perm_dev, uint32_t* bin_start_dev,
                                   int32_t* bad_dev, void* stream);

/*
 * Uneven batches of independent problems in one captured CUDA graph (the
 * many-responses / many-datasets use of Sec. 4 and the EEG spectra of
 * Sec. 4.4).  Each problem has its own options (dimension, grid, bandwidth,
 * tile) and plan; all plans share one caller-owned workspace.
 *   fkreg_batch_create          opts[n_problems], max_n[n_problems]; host only
 *                               besides the cuFFT plans of each problem
 *   fkreg_batch_workspace_bytes total bytes (256-byte aligned start)
 *   fkreg_batch_set_workspace   hands each plan its slice (synchronises stream)
 *   fkreg_batch_capture         records, per problem p on one of up to 16
 *                               forked branches: fkreg_set_points(n[p], x[p]),
 *                               fkreg_smooth(y[p], &outs[p]) and, when
 *                               sigma2[p] is not NULL, fkreg_variance(y[p],
 *                               outs[p].mhat_at_x, sigma2[p]); then a global
 *                               timer stamp.  Inputs and outputs must keep
 *                               their addresses for later launches.  The
 *                               capture stream must not be capturing already.
 *   fkreg_batch_launch          replays the graph on `stream`
 *   fkreg_batch_latencies       ms[p] = completion time of problem p relative
 *                               to the start of the last launch (synchronises)
 *   fkreg_batch_plan            the plan of problem p (for inspection)
 */
typedef struct fkreg_batch_s* fkreg_batch;
fkreg_status fkreg_batch_create(int n_problems, const fkreg_opts* opts, const int64_t* max_n,
                                fkreg_batch* out);
fkreg_status fkreg_batch_workspace_bytes(fkreg_batch batch, size_t* bytes);
fkreg_status fkreg_batch_set_workspace(fkreg_batch batch, void* ws_dev, size_t bytes, void* stream);
fkreg_status fkreg_batch_capture(fkreg_batch batch, const int64_t* n, const void* const* x_dev,
                                 const void* const* y_dev, const fkreg_outputs* outs,
                                 void* const* sigma2_dev, void* stream);
fkreg_status fkreg_batch_launch(fkreg_batch batch, void* stream);
fkreg_status fkreg_batch_latencies(fkreg_batch batch, double* ms, void* stream);
fkreg_plan fkreg_batch_plan(fkreg_batch batch, int p);
const char* fkreg_batch_last_error(fkreg_batch batch);
void fkreg_batch_destroy(fkreg_batch batch);

/*
 * Failure-path knob (the paper has no counterpart): the kernels that stage
 * field windows in shared memory wait for each window's bulk copies with a
 * bounded number of polls, then record FKREG_ERR_TIMEOUT in the error word
 * that fkreg_sync_status reports, wait (with the full budget) for any copy
 * still in flight and return.  polls >= 0 sets that number for this plan's
 * later calls (0 gives up at the first wait, which tests the failure path);
 * polls < 0 restores the default (2^22 polls).  Results of a call that timed
 * out are not valid; the plan stays usable.
 */
fkreg_status fkreg_set_wait_limit(fkreg_plan plan, int64_t polls);

/* Synchronise the stream and report device-detected errors (then clear them). */
fkreg_status fkreg_sync_status(fkreg_plan plan, void* stream);

/*
 * The checked build.  libfkreg_checked.so is built from the same sources with
 * FKREG_CHECKED defined: the main kernels (sort scatter, spreading tile and
 * flush, interpolation window and field reads, grid solve, direct-sum bin
 * ranges) range-check their index arithmetic before each access; a failed
 * check skips the access and records the site and index in the plan's error
 * word, which fkreg_sync_status reports as FKREG_ERR_DEVICE ("bounds check
 * failed ..., site S, index I").  No check traps.
 * fkreg_checked_build: 1 in the checked library, 0 otherwise.
 * fkreg_check_selftest: launches one checked access at an index outside its
 * logical bound (both inside the plan's error-word region, so the access
 * cannot leave the workspace whether or not it is checked); in the checked
 * library the next fkreg_sync_status reports site 15, index 20.  Needs the
 * workspace; FKREG_ERR_CUDA if the launch fails.
 */
int fkreg_checked_build(void);
fkreg_status fkreg_check_selftest(fkreg_plan plan, void* stream);

/* Message of the last failing call on this plan ("" if none). */
const char* fkreg_last_error(fkreg_plan plan);

/* Message of the last failing plan-less call (geometry query, create). */
const char* fkreg_global_error(void);

void fkreg_plan_destroy(fkreg_plan plan);

#ifdef __cplusplus
}
#endif

#endif /* FKREG_H */
