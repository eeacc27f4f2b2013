// C ABI: plan lifetime, workspace layout and the stage launcher.
//
// One fkreg_smooth / fkreg_df call runs, on the caller's stream:
//   strengths (density 1, responses, probes) in sorted order
//   -> type-1 spreading -> forward FFT (cuFFT)
//   -> grid stage: kernel multiply + fold -> inverse FFT -> FP64 grid solve
//   -> sample stage, per bandwidth: kernel multiply / deconvolve onto that
//      bandwidth's fine grid -> inverse FFT -> interpolation + at-sample
//      solve + reductions
//   -> DF / GCV finalisation.
// No host synchronisation happens inside a call.
#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "internal.h"

using fk::Region;

namespace {

std::string g_last_error;
std::mutex g_mu;

fkreg_status set_global_error(fkreg_status st, const std::string& msg) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_last_error = msg;
  return st;
}

fkreg_status plan_err(fkreg_plan_s* P, fkreg_status st, const std::string& msg) {
  if (P) P->err = msg;
  return st;
}

fkreg_status cuda_err(fkreg_plan_s* P, cudaError_t e, const char* where) {
  return plan_err(P, FKREG_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Records a (start, stop) event pair around one stage when timing is on.
struct StageScope {
  fkreg_plan_s* P;
  int stage;
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
  StageScope(fkreg_plan_s* P_, int st, cudaStream_t s_) : P(P_), stage(st), s(s_) {
    if (!P->timing) return;
    a = take();
    b = take();
    if (a) cudaEventRecord(a, s);
  }
  ~StageScope() {
    if (!P->timing || !a || !b) return;
    cudaEventRecord(b, s);
    P->pending.push_back({stage, a, b});
  }
  cudaEvent_t take() {
    if (!P->ev_pool.empty()) {
      cudaEvent_t e = P->ev_pool.back();
      P->ev_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  }
};

// Joins a forked branch back into the caller's stream when it leaves scope
// (also on early error returns, so no work of the branch is left unordered).
struct Join {
  fkreg_plan_s* P = nullptr;
  cudaStream_t branch = nullptr, caller = nullptr;
  bool joined = false;
  bool ok = true;
  bool done() {
    if (P && !joined) {
      joined = true;
      ok = cudaEventRecord(P->ev_join, branch) == cudaSuccess &&
           cudaStreamWaitEvent(caller, P->ev_join, 0) == cudaSuccess;
    }
    return ok;
  }
  Join() = default;
  Join(fkreg_plan_s* p, cudaStream_t b, cudaStream_t c) : P(p), branch(b), caller(c) {}
  Join& operator=(Join&& o) noexcept {
    P = o.P;
    branch = o.branch;
    caller = o.caller;
    joined = o.joined;
    ok = o.ok;
    o.P = nullptr;
    return *this;
  }
  Join(const Join&) = delete;
  ~Join() { done(); }
};

constexpr size_t kAlign = 256;

struct Layout {
  size_t cur = 0;
  void take(Region& r, size_t bytes) {
    cur = (cur + kAlign - 1) / kAlign * kAlign;
    r.off = cur;
    r.bytes = bytes;
    cur += std::max<size_t>(bytes, 1);
  }
};

int64_t half_cells(const int64_t* n, int d) {
  int64_t h = 1;
  for (int a = 0; a < d; ++a) h *= (a == d - 1) ? (n[a] / 2 + 1) : n[a];
  return h;
}

int64_t full_cells(const int64_t* n, int d) {
  int64_t h = 1;
  for (int a = 0; a < d; ++a) h *= n[a];
  return h;
}

}  // namespace

namespace fk {

// kind 0: forward R2C, kind 1: inverse C2R, kind 2: inverse C2R in place whose
// outputs exec_fft then interleaves into cell records, kind 3: forward R2C
// (the lattice adjoint fields of the grid-estimate backward)
fkreg_status fft_get(fkreg_plan_s* P, int kind, const int64_t* dims, int batch, cufftHandle* h) {
  auto key = std::make_tuple(kind, dims[0], P->d > 1 ? dims[1] : 1, P->d > 2 ? dims[2] : 1, batch);
  auto it = P->ffts.find(key);
  if (it != P->ffts.end()) {
    *h = it->second;
    return FKREG_OK;
  }
  cufftHandle hd;
  if (cufftCreate(&hd) != CUFFT_SUCCESS) return plan_err(P, FKREG_ERR_CUFFT, "cufftCreate failed");
  cufftSetAutoAllocation(hd, 0);
  long long n[3] = {dims[0], dims[1], dims[2]};
  cufftType type;
  const bool fwd = kind == 0 || kind == 3;
  if (P->prec == FKREG_F32)
    type = fwd ? CUFFT_R2C : CUFFT_C2R;
  else
    type = fwd ? CUFFT_D2Z : CUFFT_Z2D;
  size_t work = 0;
  cufftResult r;
  if (kind == 2) {
    // in-place inverse transform (padded real rows of 2 (n_last/2 + 1));
    // run_t2_interleave then builds the cell records
    long long inembed[3] = {n[0], n[1], n[2]};
    inembed[P->d - 1] = n[P->d - 1] / 2 + 1;
    long long onembed[3] = {n[0], n[1], n[2]};
    onembed[P->d - 1] = 2 * (n[P->d - 1] / 2 + 1);
    long long idist = 1;
    for (int a = 0; a < P->d; ++a) idist *= inembed[a];
    r = cufftMakePlanMany64(hd, P->d, n, inembed, 1, idist, onembed, 1, 2 * idist, type, batch,
                            &work);
  } else {
    r = cufftMakePlanMany64(hd, P->d, n, nullptr, 1, 0, nullptr, 1, 0, type, batch, &work);
  }
  if (r != CUFFT_SUCCESS) {
    cufftDestroy(hd);
    return plan_err(P, FKREG_ERR_CUFFT, "cufftMakePlanMany64 failed (" + std::to_string(int(r)) + ")");
  }
  // the inverse grid transforms run beside the others: their own work area
  const fk::Region& wr = kind == 1 ? P->r_fftwork_g : P->r_fftwork;
  if (P->ws && work > wr.bytes) {
    cufftDestroy(hd);
    return plan_err(P, FKREG_ERR_WORKSPACE, "cuFFT work area larger than the reserved region");
  }
  if (P->ws) cufftSetWorkArea(hd, P->ws + wr.off);
  if (kind == 1)
    P->fft_work_reserved_g = std::max(P->fft_work_reserved_g, work);
  else
    P->fft_work_reserved = std::max(P->fft_work_reserved, work);
  P->ffts[key] = hd;
  *h = hd;
  return FKREG_OK;
}

}  // namespace fk

extern "C" {

fkreg_status fkreg_geometry_query(const fkreg_opts* opts, fkreg_geometry* out) {
  std::string err;
  fkreg_status st = fk::compute_geometry(opts, out, &err, nullptr, nullptr, nullptr, nullptr);
  if (st != FKREG_OK) set_global_error(st, err);
  return st;
}

fkreg_status fkreg_spread_kernel_ft(int kind, int w, double beta, int64_t nf, int64_t nk,
                                    double* phihat) {
  if (!phihat || w < 2 || w > 32 || nf < 2 || nk < 0 || !(beta > 0))
    return set_global_error(FKREG_ERR_INVALID_ARG, "fkreg_spread_kernel_ft: bad arguments");
  if (kind != FKREG_SPREAD_ES && kind != FKREG_SPREAD_GAUSS)
    return set_global_error(FKREG_ERR_INVALID_ARG, "fkreg_spread_kernel_ft: bad kind");
  fk::spread_phihat(kind, w, beta, nf, nk, phihat);
  return FKREG_OK;
}

const char* fkreg_global_error(void) { return g_last_error.c_str(); }

fkreg_status fkreg_plan_create(const fkreg_opts* opts, int64_t max_n, fkreg_plan* out) {
  if (!out) return set_global_error(FKREG_ERR_INVALID_ARG, "out must be non-NULL");
  *out = nullptr;
  if (max_n < 0 || max_n > (int64_t(1) << 31))
    return set_global_error(FKREG_ERR_INVALID_ARG, "max_n must lie in [0, 2^31]");
  auto* P = new fkreg_plan_s();
  std::string err;
  fkreg_status st = fk::compute_geometry(opts, &P->g, &err, &P->bw, &P->tab, P->phi1_off, &P->geo);
  if (st != FKREG_OK) {
    delete P;
    return set_global_error(st, err);
  }
  P->o = *opts;
  P->geo.wait_limit = fk::kDefaultWaitLimit;
  const int d = opts->dim;
  P->H.assign(opts->H, opts->H + size_t(opts->n_bw) * d * d);
  P->o.H = P->H.data();
  P->max_n = max_n;
  P->d = d;
  P->order = opts->order;
  P->prec = opts->precision;
  P->tsize = P->prec == FKREG_F32 ? 4 : 8;
  P->ns = P->g.ns;
  P->nt = P->g.nt;
  P->p = P->nt;
  P->nbw = opts->n_bw;
  P->nrhs = opts->n_rhs;
  P->nrhs_real = opts->n_rhs * (opts->y_complex ? 2 : 1);
  P->max_probes = opts->max_probes;
  P->mono.n = P->ns;
  P->mono.nt = P->nt;
  fk::monomials(d, 2 * P->order, P->mono.e);
  P->smax = 1 + P->nrhs_real + P->max_probes;
  P->f2max = P->ns + (P->nrhs_real + P->max_probes) * P->nt;
  P->fgrid = P->ns + P->nrhs_real * P->nt;
  P->nacc = P->nrhs_real + 2 * P->max_probes + 1;
  P->backward = (opts->flags & FKREG_WANT_BACKWARD) != 0;
  P->direct = opts->kernel != FKREG_KERNEL_GAUSSIAN;
  P->f2bwd = P->ns + (1 + P->max_probes) * P->nt;
  const int nout_bwd = 1 + (2 + P->max_probes) * opts->dim;
  // grid-estimate backward: adjoint values per response, gradients per class
  const int nout_grid = P->nrhs_real + (1 + P->nrhs_real) * opts->dim;
  const int strengths_total = P->smax + (P->backward ? P->f2bwd : 0);
  const int t2_fields =
      std::max(P->f2max, P->backward ? std::max(std::max(P->f2bwd, nout_bwd), nout_grid) : 0);
  if (P->nacc > 512) {
    delete P;
    return set_global_error(FKREG_ERR_UNSUPPORTED, "n_rhs (real parts) + 2 max_probes must be <= 511");
  }
  if (P->direct && P->f2max > 64) {
    delete P;
    return set_global_error(FKREG_ERR_UNSUPPORTED,
                            "compact kernels: s-fields + (responses + probes) t-fields must be <= 64");
  }
  if (P->nt * (P->nrhs_real + P->max_probes) + P->ns > 4096) {
    delete P;
    return set_global_error(FKREG_ERR_UNSUPPORTED, "too many fields");
  }
  int64_t nb = 1;
  for (int a = 0; a < d; ++a) nb *= P->g.nbins[a];
  P->nbins_total = nb;
  P->nsub_max = nb + (max_n + fk::kSubMax - 1) / fk::kSubMax;
  // device and its SM count (persistent grids are sized from it)
  if (cudaGetDevice(&P->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&P->sm_count, cudaDevAttrMultiProcessorCount, P->device) !=
          cudaSuccess ||
      P->sm_count < 1) {
    delete P;
    return set_global_error(FKREG_ERR_CUDA, "no CUDA device");
  }
  P->nblk_interp = int64_t(P->sm_count) * 8;
  // tile + halo must fit shared memory for one strength
  {
    size_t cells = 1;
    for (int a = 0; a < d; ++a) cells *= size_t(P->g.tile[a] + 2 * ((P->g.w + 1) / 2));
    if (cells * P->tsize > 200 * 1024) {
      delete P;
      return set_global_error(FKREG_ERR_UNSUPPORTED, "spreading tile too large for shared memory");
    }
  }
  // workspace layout
  const size_t T = P->tsize;
  const int64_t nf_cells = full_cells(P->g.nf, d), nf_half = half_cells(P->g.nf, d);
  const int64_t l_cells = full_cells(P->g.ldft, d), l_half = half_cells(P->g.ldft, d);
  int64_t t2_cells = 1, t2_half = 1;
  for (const auto& B : P->bw) {
    t2_cells = std::max(t2_cells, full_cells(B.nf, d));
    t2_half = std::max(t2_half, half_cells(B.nf, d));
  }
  const int64_t ntiles = (max_n + fk::kSortTileKeys - 1) / fk::kSortTileKeys;
  const int64_t scan_len = std::max<int64_t>(1024 * ntiles, nb + 1);  // up to 10-bit digits
  Layout L;
  L.take(P->r_err, 256);
  L.take(P->r_bw, sizeof(fk::BwDev) * P->nbw);
  L.take(P->r_tab, sizeof(double) * std::max<size_t>(1, P->tab.size()));
  L.take(P->r_xs, T * d * std::max<int64_t>(1, max_n));
  for (Region* r : {&P->r_keys0, &P->r_vals0, &P->r_keys1, &P->r_vals1})
    L.take(*r, 4 * std::max<int64_t>(1, max_n));
  L.take(P->r_counts, 4 * nb);
  L.take(P->r_binstart, 4 * (nb + 1));
  L.take(P->r_nsub, 4 * nb);
  L.take(P->r_substart, 4 * (nb + 1));
  L.take(P->r_subbin, 4 * P->nsub_max);
  L.take(P->r_subfirst, 4 * P->nsub_max);
  L.take(P->r_hist, 4 * (1024 * ntiles + 1));
  L.take(P->r_hist2, 4 * (1024 * ntiles + 1));
  L.take(P->r_dtot, 4 * 2048);
  L.take(P->r_scan, 4 * (scan_len / 1024 + 2));
  L.take(P->r_str, T * strengths_total * std::max<int64_t>(1, max_n));
  // the direct path (compact kernels) needs only the grid fields
  const int64_t fft_scale = P->direct ? 0 : 1;
  L.take(P->r_fine, std::max<int64_t>(256, fft_scale * T * strengths_total * nf_cells));
  L.take(P->r_spec, std::max<int64_t>(256, fft_scale * 2 * T * strengths_total * nf_half));
  L.take(P->r_gspec, std::max<int64_t>(256, fft_scale * 2 * T * int64_t(P->nbw) * P->fgrid * l_half));
  L.take(P->r_gfield, T * size_t(P->nbw) * P->fgrid * l_cells);
  {
    int64_t mt = 1;
    for (int a = 0; a < d; ++a) mt *= opts->grid_n[a];
    L.take(P->r_gavec, sizeof(double) * size_t(P->nbw) * P->p * mt);
  }
  L.take(P->r_t2spec, std::max<int64_t>(256, fft_scale * 2 * T * int64_t(t2_fields) * t2_half));
  L.take(P->r_t2field,
         std::max<int64_t>(256, fft_scale * T * int64_t(fk::t2_record_stride(t2_fields)) * t2_cells));
  L.take(P->r_part, sizeof(double) * size_t(P->nblk_interp + 1) * P->nbw * P->nacc);
  L.take(P->r_smax, 8 * size_t(P->nbw));
  if (P->backward) {
    const int64_t nn = std::max<int64_t>(1, max_n);
    int64_t mtot = 1;
    for (int a = 0; a < d; ++a) mtot *= opts->grid_n[a];
    int64_t gblk = 1;
    for (int b = 0; b < P->nbw; ++b) gblk = std::max(gblk, fk::run_dlogh_lattice_blocks(P, b));
    L.take(P->r_gmask, size_t(P->nbw) * mtot);
    L.take(P->r_gadj, T * size_t(P->ns + P->nrhs_real * P->nt) * l_cells);
    L.take(P->r_gpart, 8 * 3 * size_t(gblk));
    L.take(P->r_bV, T * size_t(1 + 2 * d) * std::max(std::max(P->f2bwd, nout_bwd), nout_grid) * nn);
    L.take(P->r_bdx, T * size_t(d + 1) * nn);
    L.take(P->r_bsc, 8 * 16);
    L.take(P->r_bpart, 8 * 3 * size_t((nn + 255) / 256 + 1));
  }
  // cuFFT plans for the standard passes (work sizes decide the reserved area)
  if (!P->direct) {
    int64_t dims[3];
    cufftHandle h;
    std::vector<int> fwd_batches = {1 + P->nrhs_real, P->nrhs};
    if (P->max_probes > 0) fwd_batches.push_back(P->smax);
    for (int bt : fwd_batches) {
      for (int a = 0; a < 3; ++a) dims[a] = P->g.nf[a];
      if ((st = fk::fft_get(P, 0, dims, bt, &h)) != FKREG_OK) {
        std::string m = P->err;
        fkreg_plan_destroy(P);
        return set_global_error(st, m);
      }
    }
    for (int a = 0; a < 3; ++a) dims[a] = P->g.ldft[a];
    for (int bt : {P->nbw * P->fgrid, P->ns + P->nrhs * P->nt}) {
      if ((st = fk::fft_get(P, 1, dims, bt, &h)) != FKREG_OK) {
        std::string m = P->err;
        fkreg_plan_destroy(P);
        return set_global_error(st, m);
      }
    }
    if (P->backward) {
      for (int a = 0; a < 3; ++a) dims[a] = P->g.nf[a];
      if ((st = fk::fft_get(P, 0, dims, P->f2bwd, &h)) != FKREG_OK) {
        std::string m = P->err;
        fkreg_plan_destroy(P);
        return set_global_error(st, m);
      }
      // the lattice adjoint fields of the grid-estimate backward
      for (int a = 0; a < 3; ++a) dims[a] = P->g.ldft[a];
      if ((st = fk::fft_get(P, 3, dims, P->ns + P->nrhs_real * P->nt, &h)) != FKREG_OK) {
        std::string m = P->err;
        fkreg_plan_destroy(P);
        return set_global_error(st, m);
      }
    }
    for (const auto& B : P->bw) {
      for (int a = 0; a < 3; ++a) dims[a] = B.nf[a];
      std::vector<int> bts = {P->ns + P->nrhs_real * P->nt};
      if (P->max_probes > 0) bts.push_back(P->f2max);
      if (P->backward) {
        bts.push_back(P->f2bwd);
        bts.push_back(nout_bwd);
        bts.push_back(nout_grid);
      }
      for (int bt : bts)
        if ((st = fk::fft_get(P, 2, dims, bt, &h)) != FKREG_OK) {
          std::string m = P->err;
          fkreg_plan_destroy(P);
          return set_global_error(st, m);
        }
    }
  }
  L.take(P->r_fftwork, std::max<size_t>(P->fft_work_reserved, 256));
  L.take(P->r_fftwork_g, std::max<size_t>(P->fft_work_reserved_g, 256));
  if (cudaStreamCreateWithFlags(&P->aux, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    fkreg_plan_destroy(P);
    return set_global_error(FKREG_ERR_CUDA, "stream or event creation failed");
  }
  P->ws_bytes = L.cur + kAlign;
  *out = P;
  return FKREG_OK;
}

fkreg_status fkreg_workspace_bytes(fkreg_plan P, size_t* bytes) {
  if (!P || !bytes) return FKREG_ERR_INVALID_ARG;
  *bytes = P->ws_bytes;
  return FKREG_OK;
}

fkreg_status fkreg_set_workspace(fkreg_plan P, void* ws, size_t bytes, void* stream) {
  if (!P) return FKREG_ERR_INVALID_ARG;
  if (!ws) return plan_err(P, FKREG_ERR_WORKSPACE, "workspace pointer is NULL");
  if (reinterpret_cast<uintptr_t>(ws) % kAlign)
    return plan_err(P, FKREG_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  if (bytes < P->ws_bytes)
    return plan_err(P, FKREG_ERR_WORKSPACE,
                    "workspace too small: need " + std::to_string(P->ws_bytes) + " bytes");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  P->ws = static_cast<char*>(ws);
  P->ws_given = bytes;
  P->geo.errw = reinterpret_cast<int*>(P->ws + P->r_err.off);
  for (auto& kv : P->ffts) {
    const fk::Region& wr = std::get<0>(kv.first) == 1 ? P->r_fftwork_g : P->r_fftwork;
    if (cufftSetWorkArea(kv.second, P->ws + wr.off) != CUFFT_SUCCESS)
      return plan_err(P, FKREG_ERR_CUFFT, "cufftSetWorkArea failed");
  }
  cudaError_t e;
  if ((e = cudaMemsetAsync(P->ws + P->r_err.off, 0, 256, s)) != cudaSuccess) return cuda_err(P, e, "memset");
  if ((e = cudaMemcpyAsync(P->ws + P->r_bw.off, P->bw.data(), sizeof(fk::BwDev) * P->nbw,
                           cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cuda_err(P, e, "upload bandwidth table");
  if (!P->tab.empty() &&
      (e = cudaMemcpyAsync(P->ws + P->r_tab.off, P->tab.data(), sizeof(double) * P->tab.size(),
                           cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cuda_err(P, e, "upload tables");
  // the host tables must outlive the copies: wait for them
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_err(P, e, "sync");
  P->points_set = false;
  P->dens_valid = false;
  P->avec_valid = false;
  return FKREG_OK;
}

fkreg_status fkreg_set_points(fkreg_plan P, int64_t n, const void* x, void* stream) {
  if (!P) return FKREG_ERR_INVALID_ARG;
  if (!P->ws) return plan_err(P, FKREG_ERR_STATE, "fkreg_set_workspace must come first");
  if (n < 0 || n > P->max_n) return plan_err(P, FKREG_ERR_INVALID_ARG, "n must lie in [0, max_n]");
  if (n > 0 && !x) return plan_err(P, FKREG_ERR_INVALID_ARG, "x is NULL");
  P->n = n;
  P->points_set = false;
  P->dens_valid = false;
  P->avec_valid = false;
  cudaError_t e;
  {
    StageScope sc(P, FKREG_STAGE_SORT, static_cast<cudaStream_t>(stream));
    e = fk::run_sort(P, n, x, static_cast<cudaStream_t>(stream));
  }
  if (e != cudaSuccess) return cuda_err(P, e, "bin sort");
  P->points_set = true;
  return FKREG_OK;
}

fkreg_status fkreg_get_sort(fkreg_plan P, uint32_t* perm, uint32_t* bin_start, int64_t* nbins,
                            void* stream) {
  if (!P) return FKREG_ERR_INVALID_ARG;
  if (nbins) *nbins = P->nbins_total;
  if (!P->points_set) return plan_err(P, FKREG_ERR_STATE, "fkreg_set_points must come first");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (perm && P->n > 0 &&
      (e = cudaMemcpyAsync(perm, fk::perm_ptr(P), 4 * P->n, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
    return cuda_err(P, e, "copy perm");
  if (bin_start &&
      (e = cudaMemcpyAsync(bin_start, P->ws + P->r_binstart.off, 4 * (P->nbins_total + 1),
                           cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
    return cuda_err(P, e, "copy bin_start");
  return FKREG_OK;
}

}  // extern "C"

namespace {

fkreg_status exec_fft(fkreg_plan_s* P, int kind, const int64_t* dims, int batch, void* in, void* out,
                      cudaStream_t s) {
  cufftHandle h;
  fkreg_status st = fk::fft_get(P, kind, dims, batch, &h);
  if (st != FKREG_OK) return st;
  if (cufftSetStream(h, s) != CUFFT_SUCCESS) return plan_err(P, FKREG_ERR_CUFFT, "cufftSetStream failed");
  cufftResult r;
  void* dst = kind == 2 ? in : out;  // kind 2 runs in place, then interleaves into out
  const bool fwd = kind == 0 || kind == 3;
  if (P->prec == FKREG_F32) {
    r = fwd ? cufftExecR2C(h, static_cast<cufftReal*>(in), static_cast<cufftComplex*>(dst))
            : cufftExecC2R(h, static_cast<cufftComplex*>(in), static_cast<cufftReal*>(dst));
  } else {
    r = fwd ? cufftExecD2Z(h, static_cast<cufftDoubleReal*>(in), static_cast<cufftDoubleComplex*>(dst))
            : cufftExecZ2D(h, static_cast<cufftDoubleComplex*>(in), static_cast<cufftDoubleReal*>(dst));
  }
  if (r != CUFFT_SUCCESS) return plan_err(P, FKREG_ERR_CUFFT, "cuFFT exec failed (" + std::to_string(int(r)) + ")");
  if (kind == 2) {
    const cudaError_t e = fk::run_t2_interleave(P, dims, batch, in, out, s);
    if (e != cudaSuccess) return cuda_err(P, e, "interleave type-2 fields");
  }
  return FKREG_OK;
}

#define FK_CHECK(call, what)                         \
  do {                                               \
    cudaError_t _e = (call);                         \
    if (_e != cudaSuccess) return cuda_err(P, _e, what); \
  } while (0)
#define FK_STATUS(call)                 \
  do {                                  \
    fkreg_status _s = (call);           \
    if (_s != FKREG_OK) return _s;      \
  } while (0)

fkreg_status pipeline(fkreg_plan_s* P, const void* y, int n_probes, uint64_t seed, const void* probes,
                      const fkreg_outputs* out, bool want_df, cudaStream_t s) {
  if (!P->ws) return plan_err(P, FKREG_ERR_STATE, "fkreg_set_workspace must come first");
  if (!P->points_set) return plan_err(P, FKREG_ERR_STATE, "fkreg_set_points must come first");
  if (P->n > 0 && !y) return plan_err(P, FKREG_ERR_INVALID_ARG, "y is NULL");
  if (n_probes < 0 || n_probes > P->max_probes)
    return plan_err(P, FKREG_ERR_INVALID_ARG, "n_probes must lie in [0, max_probes]");
  const int d = P->d;
  const int S = 1 + P->nrhs_real + n_probes;
  const size_t T = P->tsize;
  const int64_t nf_cells = full_cells(P->g.nf, d);
  (void)nf_cells;
  P->dens_valid = false;
  P->avec_valid = false;
#define FK_STAGE(id) StageScope _sc##id(P, id, s)
  {
    FK_STAGE(FKREG_STAGE_STRENGTHS);
    FK_CHECK(fk::run_gather_strengths(P, y, 0, n_probes, seed, probes, 1, s), "strengths");
  }
  if (P->direct) {
    // compact kernels: direct sums for the grid and at the samples
    if (out && (out->mhat_grid || out->mask || out->moments)) {
      {
        FK_STAGE(FKREG_STAGE_KMUL_GRID);
        FK_CHECK(fk::run_direct_grid(P, 1, P->nrhs_real, 0, P->nbw, s), "direct grid sums");
      }
      {
        FK_STAGE(FKREG_STAGE_GRID_SOLVE);
        FK_CHECK(fk::run_grid_solve(P, 0, P->nbw, P->nrhs_real, nullptr, out, nullptr, s), "grid solve");
      }
    }
    if (want_df || n_probes > 0 || (out && (out->mhat_at_x || out->rss))) {
      for (int b = 0; b < P->nbw; ++b) {
        FK_STAGE(FKREG_STAGE_INTERP);
        FK_CHECK(fk::run_interp(P, b, P->nrhs_real, n_probes, y, out ? out->mhat_at_x : nullptr, s),
                 "direct sums at the samples");
      }
      FK_STAGE(FKREG_STAGE_FINALIZE);
      FK_CHECK(fk::run_finalize(P, n_probes, out, s), "finalize");
    }
    (void)T;
    P->dens_valid = true;
    return FKREG_OK;
  }
  {
    FK_STAGE(FKREG_STAGE_SPREAD);
    FK_CHECK(fk::run_spread(P, 0, S, s), "spread");
  }
  {
    FK_STAGE(FKREG_STAGE_FFT_FWD);
    FK_STATUS(exec_fft(P, 0, P->g.nf, S, P->ws + P->r_fine.off, P->ws + P->r_spec.off, s));
  }
  const bool grid = out && (out->mhat_grid || out->mask || out->moments);
  const bool at = want_df || n_probes > 0 || (out && (out->mhat_at_x || out->rss));
  // The grid branch (kernel multiply, inverse transform, grid solve) and the
  // type-2 branch both only read the forward spectrum: with both wanted, the
  // grid branch runs on the plan's second stream, forked from and joined
  // back into the caller's stream (a captured graph gets the same fork).
  // Small problems, whose kernels take microseconds, stay on one stream:
  // there the fork's own cost is larger than the overlap.
  constexpr int64_t kForkMinSamples = int64_t(1) << 16;
  Join join;
  bool grid_weights = false;  // the grid solve kept its weights for a variance pass
  if (grid) {
    cudaStream_t sg = s;
    if (at && P->aux && P->n >= kForkMinSamples) {
      cudaError_t e = cudaEventRecord(P->ev_fork, s);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(P->aux, P->ev_fork, 0);
      if (e != cudaSuccess) return cuda_err(P, e, "fork the grid branch");
      sg = P->aux;
      join = Join{P, sg, s};
    }
    {
      const cudaStream_t s = sg;  // the branch's own stream for its stages
      {
        FK_STAGE(FKREG_STAGE_KMUL_GRID);
        FK_CHECK(fk::run_kmul_grid(P, 0, 1, P->nrhs_real, 0, P->nbw, P->ws + P->r_gspec.off, s),
                 "kmul grid");
      }
      {
        FK_STAGE(FKREG_STAGE_FFT_GRID);
        FK_STATUS(exec_fft(P, 1, P->g.ldft, P->nbw * P->fgrid, P->ws + P->r_gspec.off,
                           P->ws + P->r_gfield.off, s));
      }
      {
        FK_STAGE(FKREG_STAGE_GRID_SOLVE);
        FK_CHECK(fk::run_grid_solve(P, 0, P->nbw, P->nrhs_real, fk::wsp<double>(P, P->r_gavec), out,
                                     nullptr, s),
                 "grid solve");
        grid_weights = true;
      }
    }
  }
  if (at) {
    const int n_rhs_str = P->nrhs_real + n_probes;
    const int f2 = P->ns + n_rhs_str * P->nt;
    for (int b = 0; b < P->nbw; ++b) {
      {
        FK_STAGE(FKREG_STAGE_KMUL_T2);
        FK_CHECK(fk::run_kmul_t2(P, b, 0, 1, n_rhs_str, s), "kmul type-2");
      }
      {
        FK_STAGE(FKREG_STAGE_FFT_T2);
        FK_STATUS(exec_fft(P, 2, P->bw[b].nf, f2, P->ws + P->r_t2spec.off, P->ws + P->r_t2field.off, s));
      }
      {
        FK_STAGE(FKREG_STAGE_INTERP);
        FK_CHECK(fk::run_interp(P, b, P->nrhs_real, n_probes, y, out ? out->mhat_at_x : nullptr, s),
                 "interpolation");
      }
    }
    FK_STAGE(FKREG_STAGE_FINALIZE);
    FK_CHECK(fk::run_finalize(P, n_probes, out, s), "finalize");
  }
  if (join.P && !join.done()) return cuda_err(P, cudaErrorUnknown, "join the grid branch");
  (void)T;
  P->dens_valid = true;
  P->avec_valid = grid_weights;
  return FKREG_OK;
}

}  // namespace

extern "C" {

fkreg_status fkreg_smooth(fkreg_plan P, const void* y, const fkreg_outputs* out, void* stream) {
  if (!P) return FKREG_ERR_INVALID_ARG;
  return pipeline(P, y, 0, 0, nullptr, out, false, static_cast<cudaStream_t>(stream));
}

fkreg_status fkreg_df(fkreg_plan P, const void* y, int n_probes, uint64_t seed, const void* probes,
                      const fkreg_outputs* out, void* stream) {
  if (!P) return FKREG_ERR_INVALID_ARG;
  if (n_probes < 1) return plan_err(P, FKREG_ERR_INVALID_ARG, "fkreg_df needs n_probes >= 1");
  return pipeline(P, y, n_probes, seed, probes, out, true, static_cast<cudaStream_t>(stream));
}

fkreg_status fkreg_backward(fkreg_plan P, const void* y, int n_probes, uint64_t seed,
                            const void* probes, int b, double* gcv, double* dlogh, void* dy,
                            void* dx, void* stream) {
  if (!P) return FKREG_ERR_INVALID_ARG;
  if (!P->backward)
    return plan_err(P, FKREG_ERR_UNSUPPORTED, "fkreg_backward needs a plan created with FKREG_WANT_BACKWARD");
  if (P->nrhs != 1 || P->o.y_complex)
    return plan_err(P, FKREG_ERR_UNSUPPORTED, "fkreg_backward supports one real response");
  if (P->o.flags & FKREG_GCV_EXACT_TRACE)
    return plan_err(P, FKREG_ERR_UNSUPPORTED, "fkreg_backward differentiates the Monte-Carlo trace");
  if (P->order > 1)
    return plan_err(P, FKREG_ERR_UNSUPPORTED, "fkreg_backward supports orders 0 and 1");
  if (n_probes < 1 || n_probes > P->max_probes)
    return plan_err(P, FKREG_ERR_INVALID_ARG, "n_probes must lie in [1, max_probes]");
  if (b < 0 || b >= P->nbw) return plan_err(P, FKREG_ERR_INVALID_ARG, "bandwidth index out of range");
  {
    const double* Hb = P->H.data() + size_t(b) * P->d * P->d;
    for (int i = 0; i < P->d; ++i)
      for (int j = 0; j < P->d; ++j)
        if (i != j && Hb[i * P->d + j] != 0.0)
          return plan_err(P, FKREG_ERR_UNSUPPORTED, "fkreg_backward needs a diagonal bandwidth matrix");
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  fkreg_outputs out{};
  FK_STATUS(pipeline(P, y, n_probes, seed, probes, &out, true, s));
  if (P->n == 0) return FKREG_OK;
  const int d = P->d;
  const int R = 1 + n_probes;
  const int F2 = P->ns + R * P->nt;
  const int nout = 1 + (1 + R) * d;
  const int64_t n = P->n;
  const size_t T = P->tsize;
  const int64_t nf_cells = full_cells(P->g.nf, d), nf_half = half_cells(P->g.nf, d);
  FK_STAGE(FKREG_STAGE_BACKWARD);
  FK_CHECK(fk::run_loss_scalars(P, b, n_probes, s), "loss scalars");
  // values, evaluation-point gradients, bandwidth derivatives of the fields
  for (int mode = 0; mode < 1 + 2 * d; ++mode) {
    const int kind = mode == 0 ? 0 : (mode <= d ? 1 : 2);
    const int axis = mode == 0 ? 0 : (mode <= d ? mode - 1 : mode - 1 - d);
    FK_CHECK(fk::run_kmul_t2_mode(P, b, 0, 1, R, kind, axis, s), "derivative spectra");
    FK_STATUS(exec_fft(P, 2, P->bw[b].nf, F2, P->ws + P->r_t2spec.off, P->ws + P->r_t2field.off, s));
    FK_CHECK(fk::run_gather_fields(P, b, F2, P->ws + P->r_bV.off + T * size_t(mode) * F2 * n, s),
             "gather fields");
  }
  FK_CHECK(fk::run_adjoint(P, b, n_probes, s), "adjoints");
  // adjoint spreading of Qbar (strengths smax .. smax + F2)
  FK_CHECK(fk::run_spread(P, P->smax, F2, s), "adjoint spread");
  FK_STATUS(exec_fft(P, 0, P->g.nf, F2, P->ws + P->r_fine.off + T * P->smax * nf_cells,
                     P->ws + P->r_spec.off + 2 * T * P->smax * nf_half, s));
  FK_CHECK(fk::run_kmul_adj(P, b, P->smax, 1 + R, s), "adjoint spectra");
  FK_STATUS(exec_fft(P, 2, P->bw[b].nf, nout, P->ws + P->r_t2spec.off, P->ws + P->r_t2field.off, s));
  FK_CHECK(fk::run_gather_fields(P, b, nout, P->ws + P->r_bV.off, s), "gather adjoint fields");
  FK_CHECK(fk::run_combine(P, n_probes, dy, dx, dlogh, s), "combine");
  if (gcv) {
    cudaError_t e = cudaMemcpyAsync(gcv, P->ws + P->r_bsc.off + 2 * sizeof(double), sizeof(double),
                                    cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_err(P, e, "copy gcv");
  }
  return FKREG_OK;
}

fkreg_status fkreg_backward_grid(fkreg_plan P, const void* y, const void* grad_mhat, int b,
                                 double* dlogh, void* dy, void* dx, void* stream) {
  if (!P) return FKREG_ERR_INVALID_ARG;
  if (!P->backward)
    return plan_err(P, FKREG_ERR_UNSUPPORTED,
                    "fkreg_backward_grid needs a plan created with FKREG_WANT_BACKWARD");
  if (P->direct) return plan_err(P, FKREG_ERR_UNSUPPORTED, "fkreg_backward_grid needs the Gaussian kernel");
  if (P->o.y_complex)
    return plan_err(P, FKREG_ERR_UNSUPPORTED, "fkreg_backward_grid takes real responses");
  if (P->order > 1)
    return plan_err(P, FKREG_ERR_UNSUPPORTED, "fkreg_backward_grid supports orders 0 and 1");
  if (!P->ws) return plan_err(P, FKREG_ERR_STATE, "fkreg_set_workspace must come first");
  if (!P->points_set) return plan_err(P, FKREG_ERR_STATE, "fkreg_set_points must come first");
  if (b < 0 || b >= P->nbw) return plan_err(P, FKREG_ERR_INVALID_ARG, "bandwidth index out of range");
  if (!grad_mhat || (P->n > 0 && !y))
    return plan_err(P, FKREG_ERR_INVALID_ARG, "y and grad_mhat are required");
  {
    const double* Hb = P->H.data() + size_t(b) * P->d * P->d;
    for (int i = 0; i < P->d; ++i)
      for (int j = 0; j < P->d; ++j)
        if (i != j && Hb[i * P->d + j] != 0.0)
          return plan_err(P, FKREG_ERR_UNSUPPORTED,
                          "fkreg_backward_grid needs a diagonal bandwidth matrix");
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int d = P->d;
  const int R = P->nrhs;
  const int fgrid = P->ns + R * P->nt;
  const int nout = R + (1 + R) * d;
  P->dens_valid = false;
  P->avec_valid = false;
  // forward grid fields of bandwidth b: strengths, spreading, forward FFT,
  // kernel multiply, inverse FFT onto the lattice, and the mask of the solve
  {
    FK_STAGE(FKREG_STAGE_STRENGTHS);
    FK_CHECK(fk::run_gather_strengths(P, y, 0, 0, 0, nullptr, 1, s), "strengths");
  }
  {
    FK_STAGE(FKREG_STAGE_SPREAD);
    FK_CHECK(fk::run_spread(P, 0, 1 + R, s), "spread");
  }
  {
    FK_STAGE(FKREG_STAGE_FFT_FWD);
    FK_STATUS(exec_fft(P, 0, P->g.nf, 1 + R, P->ws + P->r_fine.off, P->ws + P->r_spec.off, s));
  }
  {
    FK_STAGE(FKREG_STAGE_KMUL_GRID);
    FK_CHECK(fk::run_kmul_grid(P, 0, 1, R, b, 1, P->ws + P->r_gspec.off, s), "kmul grid");
  }
  {
    FK_STAGE(FKREG_STAGE_FFT_GRID);
    FK_STATUS(exec_fft(P, 1, P->g.ldft, fgrid, P->ws + P->r_gspec.off, P->ws + P->r_gfield.off, s));
  }
  uint8_t* mask = reinterpret_cast<uint8_t*>(P->ws + P->r_gmask.off);
  {
    FK_STAGE(FKREG_STAGE_GRID_SOLVE);
    fkreg_outputs mo{};
    mo.mask = mask;  // the solve writes bandwidth b's mask at mask + b M
    FK_CHECK(fk::run_grid_solve(P, b, 1, R, nullptr, &mo, nullptr, s), "grid solve");
  }
  int64_t mtot = 1;
  for (int a = 0; a < d; ++a) mtot *= P->o.grid_n[a];
  FK_STAGE(FKREG_STAGE_BACKWARD);
  // adjoints of the per-grid-point solves as lattice fields, and their spectra
  void* qbar = P->ws + P->r_gadj.off;
  FK_CHECK(fk::run_grid_adjoint(P, b, R, mask + size_t(b) * mtot, grad_mhat, qbar, s),
           "grid adjoints");
  FK_STATUS(exec_fft(P, 3, P->g.ldft, fgrid, qbar, P->ws + P->r_gspec.off, s));
  if (dlogh)
    FK_CHECK(fk::run_dlogh_lattice(P, b, R, P->ws + P->r_gspec.off,
                                   reinterpret_cast<double*>(P->ws + P->r_gpart.off), dlogh, s),
             "bandwidth gradient");
  if ((dy || dx) && P->n > 0) {
    FK_CHECK(fk::run_kmul_adj_lattice(P, b, R, P->ws + P->r_gspec.off, s), "adjoint spectra");
    FK_STATUS(exec_fft(P, 2, P->bw[b].nf, nout, P->ws + P->r_t2spec.off, P->ws + P->r_t2field.off, s));
    FK_CHECK(fk::run_gather_fields(P, b, nout, P->ws + P->r_bV.off, s), "gather adjoint functions");
    FK_CHECK(fk::run_combine_grid(P, R, P->ws + P->r_bV.off, dy, dx, s), "combine");
  }
  return FKREG_OK;
}

fkreg_status fkreg_variance(fkreg_plan P, const void* y, const void* mhat_at_x, void* sigma2,
                            void* stream) {
  if (!P) return FKREG_ERR_INVALID_ARG;
  if (!P->dens_valid)
    return plan_err(P, FKREG_ERR_STATE, "fkreg_variance must follow fkreg_smooth/fkreg_df on the same points");
  if (P->n > 0 && (!y || !mhat_at_x)) return plan_err(P, FKREG_ERR_INVALID_ARG, "y and mhat_at_x are required");
  if (!sigma2) return plan_err(P, FKREG_ERR_INVALID_ARG, "sigma2_grid is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int d = P->d;
  const int64_t nf_cells = full_cells(P->g.nf, d), nf_half = half_cells(P->g.nf, d);
  const int R = P->nrhs;
  for (int b = 0; b < P->nbw; ++b) {
    {
      FK_STAGE(FKREG_STAGE_STRENGTHS);
      FK_CHECK(fk::run_residual_strengths(P, y, mhat_at_x, b, 1, s), "residuals");
    }
    if (P->direct) {
      {
        FK_STAGE(FKREG_STAGE_KMUL_GRID);
        FK_CHECK(fk::run_direct_grid(P, 1, R, b, 1, s), "direct grid sums");
      }
      FK_STAGE(FKREG_STAGE_GRID_SOLVE);
      FK_CHECK(fk::run_grid_solve(P, b, 1, R, nullptr, nullptr, sigma2, s), "grid solve");
      continue;
    }
    {
      FK_STAGE(FKREG_STAGE_SPREAD);
      FK_CHECK(fk::run_spread(P, 1, R, s), "spread");
    }
    {
      FK_STAGE(FKREG_STAGE_FFT_FWD);
      FK_STATUS(exec_fft(P, 0, P->g.nf, R, P->ws + P->r_fine.off + P->tsize * nf_cells,
                         P->ws + P->r_spec.off + 2 * P->tsize * nf_half, s));
    }
    // with the grid weights of the smoothing pass (same points, same
    // s-fields, so the same systems and mask) only the residuals' t-fields
    // are needed on the grid: sigma^2(g) = sum_k a_k(g) t_k(g)
    const bool reuse = P->avec_valid;
    {
      FK_STAGE(FKREG_STAGE_KMUL_GRID);
      FK_CHECK(fk::run_kmul_grid(P, reuse ? -1 : 0, 1, R, b, 1, P->ws + P->r_gspec.off, s),
               "kmul grid");
    }
    {
      FK_STAGE(FKREG_STAGE_FFT_GRID);
      FK_STATUS(exec_fft(P, 1, P->g.ldft, (reuse ? 0 : P->ns) + R * P->nt,
                         P->ws + P->r_gspec.off, P->ws + P->r_gfield.off, s));
    }
    {
      FK_STAGE(FKREG_STAGE_GRID_SOLVE);
      if (reuse)
        FK_CHECK(fk::run_grid_apply(P, b, R, sigma2, s), "grid weights");
      else
        FK_CHECK(fk::run_grid_solve(P, b, 1, R, nullptr, nullptr, sigma2, s), "grid solve");
    }
  }
  return FKREG_OK;
}

fkreg_status fkreg_log_variance(fkreg_plan P, const void* y, const void* mhat_at_x, void* v_grid,
                                void* v_at_x, double* kappa, void* sigma2, void* stream) {
  if (!P) return FKREG_ERR_INVALID_ARG;
  if (!P->dens_valid)
    return plan_err(P, FKREG_ERR_STATE, "fkreg_log_variance must follow fkreg_smooth/fkreg_df on the same points");
  if (P->o.y_complex)
    return plan_err(P, FKREG_ERR_UNSUPPORTED, "fkreg_log_variance takes real responses");
  if (P->n < 1) return plan_err(P, FKREG_ERR_INVALID_ARG, "fkreg_log_variance needs at least one sample");
  if (!y || !mhat_at_x || !v_grid || !v_at_x || !kappa)
    return plan_err(P, FKREG_ERR_INVALID_ARG, "y, mhat_at_x, v_grid, v_at_x and kappa are required");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int d = P->d;
  const int64_t nf_cells = full_cells(P->g.nf, d), nf_half = half_cells(P->g.nf, d);
  const int R = P->nrhs;
  const int f2 = P->ns + R * P->nt;
  for (int b = 0; b < P->nbw; ++b) {
    {
      FK_STAGE(FKREG_STAGE_STRENGTHS);
      FK_CHECK(fk::run_logres_strengths(P, y, mhat_at_x, b, 1, s), "log residuals");
    }
    if (P->direct) {
      {
        FK_STAGE(FKREG_STAGE_KMUL_GRID);
        FK_CHECK(fk::run_direct_grid(P, 1, R, b, 1, s), "direct grid sums");
      }
      {
        FK_STAGE(FKREG_STAGE_GRID_SOLVE);
        FK_CHECK(fk::run_grid_solve(P, b, 1, R, nullptr, nullptr, v_grid, s), "grid solve");
      }
      {
        FK_STAGE(FKREG_STAGE_INTERP);
        FK_CHECK(fk::run_interp(P, b, R, 0, y, v_at_x, s), "direct sums at the samples");
      }
      FK_STAGE(FKREG_STAGE_FINALIZE);
      FK_CHECK(fk::run_kappa_sigma2(P, b, y, mhat_at_x, v_at_x, v_grid, kappa, sigma2, s), "kappa");
      continue;
    }
    {
      FK_STAGE(FKREG_STAGE_SPREAD);
      FK_CHECK(fk::run_spread(P, 1, R, s), "spread");
    }
    {
      FK_STAGE(FKREG_STAGE_FFT_FWD);
      FK_STATUS(exec_fft(P, 0, P->g.nf, R, P->ws + P->r_fine.off + P->tsize * nf_cells,
                         P->ws + P->r_spec.off + 2 * P->tsize * nf_half, s));
    }
    {
      FK_STAGE(FKREG_STAGE_KMUL_GRID);
      FK_CHECK(fk::run_kmul_grid(P, P->avec_valid ? -1 : 0, 1, R, b, 1, P->ws + P->r_gspec.off, s),
               "kmul grid");
    }
    {
      FK_STAGE(FKREG_STAGE_FFT_GRID);
      FK_STATUS(exec_fft(P, 1, P->g.ldft, (P->avec_valid ? 0 : P->ns) + R * P->nt, P->ws + P->r_gspec.off,
                         P->ws + P->r_gfield.off, s));
    }
    {
      FK_STAGE(FKREG_STAGE_GRID_SOLVE);
      // the grid weights of the smoothing pass, as in fkreg_variance
      if (P->avec_valid)
        FK_CHECK(fk::run_grid_apply(P, b, R, v_grid, s), "grid weights");
      else
        FK_CHECK(fk::run_grid_solve(P, b, 1, R, nullptr, nullptr, v_grid, s), "grid solve");
    }
    // v at the samples: type-2 of the same fields
    {
      FK_STAGE(FKREG_STAGE_KMUL_T2);
      FK_CHECK(fk::run_kmul_t2(P, b, 0, 1, R, s), "kmul type-2");
    }
    {
      FK_STAGE(FKREG_STAGE_FFT_T2);
      FK_STATUS(exec_fft(P, 2, P->bw[b].nf, f2, P->ws + P->r_t2spec.off, P->ws + P->r_t2field.off, s));
    }
    {
      FK_STAGE(FKREG_STAGE_INTERP);
      FK_CHECK(fk::run_interp(P, b, R, 0, y, v_at_x, s), "interpolation");
    }
    {
      FK_STAGE(FKREG_STAGE_FINALIZE);
      FK_CHECK(fk::run_kappa_sigma2(P, b, y, mhat_at_x, v_at_x, v_grid, kappa, sigma2, s), "kappa");
    }
  }
  return FKREG_OK;
}

fkreg_status fkreg_set_wait_limit(fkreg_plan P, int64_t polls) {
  if (!P) return FKREG_ERR_INVALID_ARG;
  if (polls > int64_t(UINT32_MAX)) return plan_err(P, FKREG_ERR_INVALID_ARG, "polls must be < 2^32");
  P->geo.wait_limit = polls < 0 ? fk::kDefaultWaitLimit : uint32_t(polls);
  return FKREG_OK;
}

fkreg_status fkreg_set_timing(fkreg_plan P, int enable) {
  if (!P) return FKREG_ERR_INVALID_ARG;
  P->timing = enable != 0;
  return FKREG_OK;
}

fkreg_status fkreg_stage_times(fkreg_plan P, double* ms, int64_t* launches, int64_t* kernel_launches) {
  if (!P) return FKREG_ERR_INVALID_ARG;
  for (auto& pe : P->pending) {
    float t = 0.f;
    cudaError_t e = cudaEventSynchronize(pe.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, pe.a, pe.b);
    if (e != cudaSuccess) return cuda_err(P, e, "stage timer");
    P->stage_ms[pe.stage] += t;
    P->stage_calls[pe.stage] += 1;
    P->ev_pool.push_back(pe.a);
    P->ev_pool.push_back(pe.b);
  }
  P->pending.clear();
  for (int i = 0; i < FKREG_N_STAGES; ++i) {
    if (ms) ms[i] = P->stage_ms[i];
    if (launches) launches[i] = P->stage_calls[i];
    P->stage_ms[i] = 0;
    P->stage_calls[i] = 0;
  }
  if (kernel_launches) *kernel_launches = P->launches;
  P->launches = 0;
  return FKREG_OK;
}

fkreg_status fkreg_sync_status(fkreg_plan P, void* stream) {
  if (!P) return FKREG_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_err(P, e, "stream");
  if (!P->ws) return FKREG_OK;
  int word[4] = {0, 0, 0, 0};
  if ((e = cudaMemcpy(word, P->ws + P->r_err.off, sizeof(word), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_err(P, e, "read error word");
  if (word[0]) {
    cudaMemset(P->ws + P->r_err.off, 0, sizeof(word));
    if (word[0] & fk::kErrBounds) {
      const int64_t idx = int64_t(uint64_t(uint32_t(word[2])) | (uint64_t(uint32_t(word[3])) << 32));
      return plan_err(P, FKREG_ERR_DEVICE,
                      "bounds check failed (checked build): site " + std::to_string(word[1]) +
                          ", index " + std::to_string(idx));
    }
    if (word[0] & fk::kErrTimeout) return plan_err(P, FKREG_ERR_TIMEOUT, "a bounded device-side wait gave up");
    return plan_err(P, FKREG_ERR_DEVICE, "a sample lies outside the grid box or is not finite");
  }
  return FKREG_OK;
}

const char* fkreg_last_error(fkreg_plan P) { return P ? P->err.c_str() : ""; }

void fkreg_plan_destroy(fkreg_plan P) {
  if (!P) return;
  for (auto& kv : P->ffts) cufftDestroy(kv.second);
  for (auto& pe : P->pending) {
    cudaEventDestroy(pe.a);
    cudaEventDestroy(pe.b);
  }
  for (auto e : P->ev_pool) cudaEventDestroy(e);
  if (P->ev_fork) cudaEventDestroy(P->ev_fork);
  if (P->ev_join) cudaEventDestroy(P->ev_join);
  if (P->aux) cudaStreamDestroy(P->aux);
  delete P;
}

}  // extern "C"
