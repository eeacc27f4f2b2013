// Internal declarations shared by the planner, the kernels and the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>

#include <cstdint>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/fkreg.h"

namespace fk {

constexpr int kMaxD = 3;
constexpr int kMaxMono = 35;     // monomials of degree <= 4 in 3-D (s-fields of local quadratic)
constexpr int kMaxP = 10;        // unknowns of the local-quadratic system in 3-D
constexpr int kSubMax = 1024;    // samples per spreading sub-problem
constexpr int kRadixBits = 8;
constexpr int kSortTileKeys = 4096;  // keys per radix-sort tile (one block)
constexpr uint32_t kDefaultWaitLimit = 1u << 22;  // polls of a staged-window wait

// Geometry of the whole plan, passed to kernels by value.
struct GeoDev {
  int d;
  int w;            // spreading width (fine cells)
  int pad;          // ceil(w/2): tile halo on each side
  int skind;        // FKREG_SPREAD_ES / FKREG_SPREAD_GAUSS
  double beta;      // ES shape, or Gaussian exponent factor
  int64_t nf[3];    // type-1 fine grid
  int64_t L[3];     // inverse-DFT length onto the grid lattice
  int64_t M[3];     // output grid points
  int64_t K[3];     // type-1 modes (kept: |k| <= K/2 - 1)
  double P[3];      // period
  double lo[3];
  double hi[3];
  double inv_h[3];  // nf / P (double; the T-rounded copy is inv_h_t)
  float inv_h_f[3];
  int64_t tile[3];
  int64_t nbins[3];
  int kbits;        // within-bin bits of the sort key (see key_local_bits)
  int kern;         // regression kernel: FKREG_KERNEL_GAUSSIAN (NUFFT) or a compact one (direct)
  uint32_t wait_limit;  // polls of a staged-window wait before it gives up (fkreg_set_wait_limit)
  int* errw;            // the plan's error word (errw[0] bits kErr*; errw[1..3] the first
                        // failed bounds check of a checked build: site, index low, high)
};

// Bits of the plan's device error word.
constexpr int kErrOutside = 1;  // a sample outside the grid box or not finite
constexpr int kErrTimeout = 2;  // a bounded device-side wait gave up
constexpr int kErrBounds = 4;   // a bounds check of the checked build failed (access skipped)

// Sort keys are (bin << kbits) | local, local = serpentine index of the
// centre cell of the sample's spreading window relative to its bin's first
// cell, tile_j + 1 values per axis.  kbits = 0 (bin-only keys) if the key would not
// fit 32 bits.
inline int key_local_bits(int d, const int64_t* tile, const int64_t* nbins) {
  int64_t cells = 1, bins = 1;
  for (int j = 0; j < d; ++j) {
    cells *= tile[j] + 1;
    bins *= nbins[j];
  }
  int lb = 0, bb = 0;
  while ((int64_t(1) << lb) < cells) ++lb;
  while ((int64_t(1) << bb) < bins) ++bb;
  return bb + lb <= 32 ? lb : 0;
}

// One bandwidth, stored in the workspace (device reads it).
struct BwDev {
  double H[9];
  double sigma[3];     // sqrt(H_jj)
  double k0;           // K_H(0)
  int64_t K[3];        // modes this bandwidth needs
  int64_t nf[3];       // type-2 fine grid for this bandwidth
  double inv_h[3];     // nf_b / P
  int64_t phi2_off[3]; // offset (doubles) of 1/phihat tables (k >= 0) for type-2
  double Hinv[9];      // H^-1 (compact kernels)
  double kscale;       // c_d / sqrt(det H): K_H(z) = kscale k(|H^(-1/2) z|^2) (compact kernels)
  double kr2;          // R^2 of the truncated Gaussian (FKREG_KERNEL_GAUSSIAN_DIRECT), else 0
};

// Monomial exponents (degree <= 2) for device code.
struct MonoTab {
  int n;               // monomials of degree <= 2l  (s-fields)
  int nt;              // monomials of degree <= l   (t-fields)
  int e[kMaxMono][kMaxD];
};

struct Region {
  size_t off = 0, bytes = 0;
};

}  // namespace fk

struct fkreg_plan_s {
  fkreg_opts o{};
  std::vector<double> H;        // [nbw][d][d]
  fkreg_geometry g{};
  fk::GeoDev geo{};
  fk::MonoTab mono{};
  int64_t max_n = 0;
  int d = 0, order = 0, prec = 0, ns = 0, nt = 0, p = 0;
  int nbw = 0, nrhs = 0, nrhs_real = 0, max_probes = 0;
  int smax = 0;                 // strengths of the largest pass
  int f2max = 0;                // type-2 fields of the largest pass
  int fgrid = 0;                // grid fields (ns + nrhs_real * nt)
  size_t tsize = 4;             // sizeof(T)
  std::vector<fk::BwDev> bw;    // host copy of the bandwidth table
  std::vector<double> tab;      // 1/phihat tables (type-1 per axis, then type-2)
  int64_t phi1_off[3] = {0, 0, 0};
  int64_t nbins_total = 0;
  int64_t nsub_max = 0;
  int64_t nblk_interp = 0;      // blocks of the interpolation kernel (partials)
  int sm_count = 0;             // streaming multiprocessors of the plan's device
  int nacc = 0;                 // accumulators per (block, bandwidth)

  // workspace regions
  fk::Region r_err, r_bw, r_tab, r_xs, r_keys0, r_vals0, r_keys1, r_vals1, r_counts,
      r_binstart, r_nsub, r_substart, r_subbin, r_subfirst, r_hist, r_hist2, r_dtot, r_scan, r_str,
      r_fine, r_spec, r_gspec, r_gfield, r_t2spec, r_t2field, r_part, r_smax, r_fftwork,
      r_fftwork_g,
      r_bV, r_bdx, r_bsc, r_bpart, r_gmask, r_gadj, r_gpart, r_gavec;
  bool backward = false;        // workspace reserved for fkreg_backward
  bool direct = false;          // compact kernel: direct sums instead of the NUFFT
  int f2bwd = 0;                // fields of the backward passes (one response + probes)
  size_t ws_bytes = 0;
  size_t fft_work_reserved = 0;
  size_t fft_work_reserved_g = 0;  // inverse grid transforms (their own area: they overlap)
  char* ws = nullptr;
  size_t ws_given = 0;

  // cuFFT plan cache: (kind, n0, n1, n2, batch) -> handle
  std::map<std::tuple<int, int64_t, int64_t, int64_t, int>, cufftHandle> ffts;

  // state
  int64_t n = 0;
  bool points_set = false;
  bool dens_valid = false;
  bool avec_valid = false;      // r_gavec holds the grid weights of the last smooth/df
  int perm_in_vals1 = 0;        // which ping-pong buffer holds the permutation
  std::string err;
  int device = -1;

  // profiling: own kernel launches, per-stage events
  int64_t launches = 0;
  bool timing = false;
  struct Pending {
    int stage;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> ev_pool;
  // second stream for the grid branch of a df/smooth call, which runs beside
  // the type-2 branch (both only read the forward spectrum)
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  double stage_ms[FKREG_N_STAGES] = {0};
  int64_t stage_calls[FKREG_N_STAGES] = {0};
};

namespace fk {

// planner.cpp
fkreg_status compute_geometry(const fkreg_opts* o, fkreg_geometry* g, std::string* err,
                              std::vector<BwDev>* bw, std::vector<double>* tab,
                              int64_t phi1_off[3], GeoDev* geo);
double spread_phi(int kind, int w, double beta, double z);
void spread_phihat(int kind, int w, double beta, int64_t nf, int64_t nk, double* out);
int nmono(int d, int deg);
void monomials(int d, int deg, int (*e)[kMaxD]);
int64_t next_fast(int64_t n);

// sort.cu
cudaError_t run_sort(fkreg_plan_s* P, int64_t n, const void* x, cudaStream_t s);

// spread.cu
cudaError_t run_spread(fkreg_plan_s* P, int s0, int ns_count, cudaStream_t s);
cudaError_t run_gather_strengths(fkreg_plan_s* P, const void* y, int first_str, int n_probes,
                                 uint64_t seed, const void* probes, int with_density,
                                 cudaStream_t s);
cudaError_t run_residual_strengths(fkreg_plan_s* P, const void* y, const void* mhat_at_x,
                                   int b, int first_str, cudaStream_t s);
cudaError_t run_logres_strengths(fkreg_plan_s* P, const void* y, const void* mhat_at_x, int b,
                                 int first_str, cudaStream_t s);

// spectral.cu
cudaError_t run_kmul_grid(fkreg_plan_s* P, int str_dens, int str_rhs, int nrhs_fields,
                          int bw_first, int bw_count, void* out_spec, cudaStream_t s);
cudaError_t run_kmul_t2(fkreg_plan_s* P, int b, int str_dens, int str_rhs, int n_rhs_str,
                        cudaStream_t s);
cudaError_t run_kmul_t2_mode(fkreg_plan_s* P, int b, int str_dens, int str_rhs, int n_rhs_str,
                             int kind, int axis, cudaStream_t s);
cudaError_t run_kmul_adj(fkreg_plan_s* P, int b, int sb, int n_classes, cudaStream_t s);
// grid-estimate backward: type-2 spectra of the adjoint functions of the
// lattice adjoint fields (their R2C spectra E [fgrid][L half]), and
// d L / d log sigma as a spectral inner product (part: FP64 partial sums of
// run_dlogh_lattice_blocks blocks x 3)
cudaError_t run_kmul_adj_lattice(fkreg_plan_s* P, int b, int nrhs, const void* E, cudaStream_t s);
int64_t run_dlogh_lattice_blocks(const fkreg_plan_s* P, int b);
cudaError_t run_dlogh_lattice(fkreg_plan_s* P, int b, int nrhs, const void* E, double* part,
                              double* dlogh, cudaStream_t s);
// backward_grid.cu: adjoint of the per-grid-point solves -> lattice adjoint
// fields qbar [fgrid][L cells] (zero where masked); and the combination of
// the gathered adjoint functions into dy [nrhs][n] and dx [n][d] (original order)
cudaError_t run_grid_adjoint(fkreg_plan_s* P, int b, int nrhs, const uint8_t* mask,
                             const void* gbar, void* qbar, cudaStream_t s);
cudaError_t run_combine_grid(fkreg_plan_s* P, int nrhs, const void* V, void* dy, void* dx,
                             cudaStream_t s);

// backward.cu
cudaError_t run_gather_fields(fkreg_plan_s* P, int b, int F, void* V, cudaStream_t s);
// Persistent interpolation kernel (FP32, width 7, 1-D / 2-D, F2 <= 64):
// launched only when it applies (*launched); vout != NULL selects the
// gather-only form (F2 fields into vout[f][n]).
cudaError_t run_interp_direct(fkreg_plan_s* P, int b, int n_rhs_real, int n_probes,
                              void* mhat_at_x, cudaStream_t st, int nacc, int F2, void* vout,
                              bool* launched);
// Lane-per-sample kernel over the global field grid (FP32, width 7, 3-D
// Nadaraya-Watson or gather-only, F2 <= 64), launched only when it applies.
cudaError_t run_interp_global_lane(fkreg_plan_s* P, int b, int n_rhs_real, int n_probes,
                                   void* mhat_at_x, cudaStream_t st, int nacc, int F2,
                                   void* vout, bool* launched);
cudaError_t run_loss_scalars(fkreg_plan_s* P, int b, int n_probes, cudaStream_t s);
cudaError_t run_adjoint(fkreg_plan_s* P, int b, int n_probes, cudaStream_t s);
cudaError_t run_combine(fkreg_plan_s* P, int n_probes, void* dy, void* dx, double* dlogh,
                        cudaStream_t s);

// solve.cu
// avec (may be null): [bw][p][M] the solved weights a_k / tscale_k of each
// grid point (NaN where masked), kept for a variance pass on the same points
cudaError_t run_grid_solve(fkreg_plan_s* P, int bw_first, int bw_count, int nrhs_fields,
                           double* avec, const fkreg_outputs* out, void* sigma2, cudaStream_t s);
// sigma2[b][r][M] = sum_k avec[b][k] t_(r,k) from the grid t-fields alone
// (r_gfield holds nrhs_fields x p t-fields; no s-fields, no solve)
cudaError_t run_grid_apply(fkreg_plan_s* P, int b, int nrhs_fields, void* sigma2, cudaStream_t s);
cudaError_t run_interp(fkreg_plan_s* P, int b, int n_rhs_str, int n_probes, const void* y,
                       void* mhat_at_x, cudaStream_t s);
// direct path (compact kernels): grid fields of strengths [str_first, str_first + nstr)
// plus the s-fields, bandwidths [bw_first, bw_first + bw_count), into r_gfield
cudaError_t run_direct_grid(fkreg_plan_s* P, int str_first, int nstr, int bw_first,
                            int bw_count, cudaStream_t s);
cudaError_t run_direct_interp(fkreg_plan_s* P, int b, int n_rhs_str, int n_probes,
                              void* mhat_at_x, cudaStream_t s);
cudaError_t run_finalize(fkreg_plan_s* P, int n_probes, const fkreg_outputs* out,
                         cudaStream_t s);
// kappa (eq. 26 normaliser) of bandwidth b for every response, and
// sigma2(g) = exp(v(g)) / kappa when sigma2 != NULL.
cudaError_t run_kappa_sigma2(fkreg_plan_s* P, int b, const void* y, const void* mhat_at_x,
                             const void* v_at_x, const void* v_grid, double* kappa, void* sigma2,
                             cudaStream_t s);

const uint32_t* perm_ptr(fkreg_plan_s* P);
int t2_record_stride(int F2);
// Interleave F in-place C2R outputs (padded real rows) at src into cell records
// [cell][t2_record_stride(F)] at dst.
cudaError_t run_t2_interleave(fkreg_plan_s* P, const int64_t* dims, int F, const void* src,
                              void* dst, cudaStream_t st);

// fft helpers (api.cu)
fkreg_status fft_get(fkreg_plan_s* P, int kind, const int64_t* dims, int batch, cufftHandle* h);

template <typename T>
T* wsp(fkreg_plan_s* P, const Region& r) {
  return reinterpret_cast<T*>(P->ws + r.off);
}

}  // namespace fk
