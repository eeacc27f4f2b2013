// Bandwidth sweeps with one Fourier period per group of bandwidths: the
// contiguous split of the bandwidth list that minimises a cost model of the
// step, one plan per group, the groups run one after another on the
// caller's stream.  The groups' plans are ordinary plans; this file only
// chooses the split and routes the calls and the output slices.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "fkreg_sweep.h"
#include "internal.h"

struct fkreg_sweep_s {
  fkreg_opts o{};
  std::vector<double> H;
  std::vector<fkreg_plan> plans;
  std::vector<int> first;     // first bandwidth of each group, then n_bw
  std::vector<int> kern;      // regression kernel of each group's plan
  std::vector<size_t> ws_off; // workspace offset of each group
  size_t ws_bytes = 0;
  int64_t M = 1;              // grid points
  int64_t n = 0;              // samples of the last set_points
  size_t tsize = 4;
  int ns = 0, nt = 0;
  std::string err;
};

namespace {

// Seconds per unit of the modelled step on GB300, from the 3-D sweep's
// measured stage times: spreading per (sample, window cell, strength), the
// type-1 transform (with its memset) per (fine cell, strength), per bandwidth
// the type-2 transform and record interleave per (fine cell, field) and the
// gather per (sample, window cell, field); a fixed cost per group for its
// sort and launches.
constexpr double kSpreadUnit = 1.3e-12;
constexpr double kType1Unit = 1.7e-11;
constexpr double kType2Unit = 1.6e-11;
constexpr double kGatherUnit = 3.3e-13;
constexpr double kGroupFixed = 3e-4;
// The direct sums (FKREG_KERNEL_GAUSSIAN_DIRECT) per (sample pair, field),
// from the at-sample pass of the compact-kernel path.
constexpr double kPairUnit = 2.4e-13;

int64_t cells(const int64_t* nf, int d) {
  int64_t c = 1;
  for (int j = 0; j < d; ++j) c *= nf[j];
  return c;
}

// Modelled seconds of one group [b0, b1) of the sweep with the NUFFT path;
// < 0 if the group's geometry is refused.
double nufft_cost(const fkreg_opts& o, int64_t max_n, int b0, int b1) {
  fkreg_opts g = o;
  const int d = o.dim;
  g.n_bw = b1 - b0;
  g.H = o.H + size_t(b0) * d * d;
  fkreg_geometry geo{};
  std::vector<fk::BwDev> bw;
  std::string err;
  if (fk::compute_geometry(&g, &geo, &err, &bw, nullptr, nullptr, nullptr) != FKREG_OK) return -1.0;
  const int nrhs_real = o.n_rhs * (o.y_complex ? 2 : 1);
  const double S = 1 + nrhs_real + o.max_probes;
  const double F = geo.ns + double(nrhs_real + o.max_probes) * geo.nt;
  double wd = 1.0;
  for (int j = 0; j < d; ++j) wd *= geo.w;
  double c = kGroupFixed + S * (kSpreadUnit * double(max_n) * wd +
                                kType1Unit * double(cells(geo.nf, d)));
  for (const auto& B : bw)
    c += F * (kType2Unit * double(cells(B.nf, d)) + kGatherUnit * double(max_n) * wd);
  return c;
}

// The same with direct sums over the samples within Mahalanobis radius R
// (FKREG_KERNEL_GAUSSIAN_DIRECT): per bandwidth, (samples + grid points) x
// the samples inside a support x the fields, the samples taken as spread
// evenly over the box; < 0 where that path is refused.
double direct_cost(const fkreg_opts& o, int64_t max_n, int b0, int b1) {
  fkreg_opts g = o;
  const int d = o.dim;
  g.kernel = FKREG_KERNEL_GAUSSIAN_DIRECT;
  g.n_bw = b1 - b0;
  g.H = o.H + size_t(b0) * d * d;
  g.flags &= ~FKREG_WANT_BACKWARD;
  fkreg_geometry geo{};
  std::vector<fk::BwDev> bw;
  std::string err;
  if (o.flags & FKREG_WANT_BACKWARD) return -1.0;
  if (fk::compute_geometry(&g, &geo, &err, &bw, nullptr, nullptr, nullptr) != FKREG_OK) return -1.0;
  const int nrhs_real = o.n_rhs * (o.y_complex ? 2 : 1);
  const double F2 = geo.ns + double(nrhs_real + o.max_probes) * geo.nt;
  const double Fg = geo.ns + double(nrhs_real) * geo.nt;
  if (F2 > 64) return -1.0;
  double vol = 1.0, M = 1.0;
  for (int j = 0; j < d; ++j) {
    vol *= o.grid_hi[j] - o.grid_lo[j];
    M *= double(o.grid_n[j]);
  }
  const double vd = d == 1 ? 2.0 : (d == 2 ? M_PI : 4.0 * M_PI / 3.0);
  double c = kGroupFixed;
  for (const auto& B : bw) {
    double ext = vd;  // volume of the support ellipsoid {z' H^-1 z <= R^2}
    for (int j = 0; j < d; ++j) ext *= B.sigma[j];
    // (a correlated H has a smaller ellipsoid than its axis extents give)
    const double nbr = std::min(double(max_n), double(max_n) * ext / vol);
    c += kPairUnit * nbr * (double(max_n) * F2 + M * Fg);
  }
  return c;
}

// The cheaper path for the group: its modelled seconds and its kernel.
double group_cost(const fkreg_opts& o, int64_t max_n, int b0, int b1, int* kernel) {
  const double cn = nufft_cost(o, max_n, b0, b1);
  const double cd = direct_cost(o, max_n, b0, b1);
  if (cd >= 0 && (cn < 0 || cd < cn)) {
    *kernel = FKREG_KERNEL_GAUSSIAN_DIRECT;
    return cd;
  }
  *kernel = FKREG_KERNEL_GAUSSIAN;
  return cn;
}

fkreg_status sweep_err(fkreg_sweep S, fkreg_status st, const std::string& m) {
  S->err = m;
  return st;
}

fkreg_status child_err(fkreg_sweep S, size_t gidx, fkreg_status st) {
  if (st != FKREG_OK)
    S->err = "group " + std::to_string(gidx) + ": " + fkreg_last_error(S->plans[gidx]);
  return st;
}

char* byte_off(void* p, size_t off) { return p ? static_cast<char*>(p) + off : nullptr; }

// The slice of `out` that holds bandwidths [b0, ...).
fkreg_outputs slice(const fkreg_sweep S, const fkreg_outputs* out, int b0) {
  fkreg_outputs r{};
  if (!out) return r;
  const bool cplx = S->o.y_complex != 0;
  const size_t esz = S->tsize * (cplx ? 2 : 1);
  const size_t R = size_t(S->o.n_rhs);
  const size_t per_mom = size_t(S->ns) + R * S->nt * (cplx ? 2 : 1);
  r.mhat_grid = byte_off(out->mhat_grid, size_t(b0) * R * S->M * esz);
  r.mask = out->mask ? out->mask + size_t(b0) * S->M : nullptr;
  r.moments = byte_off(out->moments, size_t(b0) * per_mom * S->M * S->tsize);
  r.mhat_at_x = byte_off(out->mhat_at_x, size_t(b0) * R * size_t(S->n) * esz);
  r.rss = out->rss ? out->rss + size_t(b0) * R : nullptr;
  r.trace = out->trace ? out->trace + size_t(b0) * 3 : nullptr;
  r.gcv = out->gcv ? out->gcv + size_t(b0) * R : nullptr;
  return r;
}

}  // namespace

extern "C" {

fkreg_status fkreg_sweep_split(const fkreg_opts* opts, int64_t max_n, int max_groups,
                               int* n_groups, int* first_bw, int* group_kernel,
                               double* modelled_s) {
  if (!opts || !opts->H || !n_groups || opts->n_bw < 1 || max_groups < 1 || max_n < 0 ||
      opts->dim < 1 || opts->dim > 3)
    return FKREG_ERR_INVALID_ARG;
  if (opts->kernel != FKREG_KERNEL_GAUSSIAN) max_groups = 1;
  const int nbw = opts->n_bw;
  // best[k][b] = least modelled cost of bandwidths [0, b) in k groups
  const int K = std::min(max_groups, nbw);
  std::vector<std::vector<double>> cost(nbw + 1, std::vector<double>(nbw + 1, -2.0));
  std::vector<std::vector<int>> kern(nbw + 1, std::vector<int>(nbw + 1, opts->kernel));
  const bool gauss = opts->kernel == FKREG_KERNEL_GAUSSIAN;
  auto gc = [&](int a, int b) {
    if (cost[a][b] == -2.0)
      cost[a][b] = gauss ? group_cost(*opts, max_n, a, b, &kern[a][b])
                         : (max_groups == 1 ? 0.0 : -1.0);
    return cost[a][b];
  };
  const double inf = 1e300;
  std::vector<std::vector<double>> best(K + 1, std::vector<double>(nbw + 1, inf));
  std::vector<std::vector<int>> from(K + 1, std::vector<int>(nbw + 1, -1));
  best[0][0] = 0.0;
  for (int k = 1; k <= K; ++k)
    for (int b = 1; b <= nbw; ++b)
      for (int a = k - 1; a < b; ++a) {
        if (best[k - 1][a] >= inf) continue;
        const double c = gc(a, b);
        if (c < 0) continue;
        if (best[k - 1][a] + c < best[k][b]) {
          best[k][b] = best[k - 1][a] + c;
          from[k][b] = a;
        }
      }
  int kbest = 0;
  for (int k = 1; k <= K; ++k)
    if (best[k][nbw] < inf && (kbest == 0 || best[k][nbw] < best[kbest][nbw])) kbest = k;
  std::vector<int> cuts{nbw};
  if (kbest > 0) {
    for (int k = kbest, b = nbw; k > 0; --k) {
      b = from[k][b];
      cuts.push_back(b);
    }
  } else {
    cuts.push_back(0);  // one group: plan creation reports why the geometry is refused
  }
  std::reverse(cuts.begin(), cuts.end());
  *n_groups = int(cuts.size()) - 1;
  if (first_bw) std::copy(cuts.begin(), cuts.end(), first_bw);
  if (group_kernel)
    for (int gi = 0; gi + 1 < int(cuts.size()); ++gi)
      group_kernel[gi] = kbest > 0 ? kern[cuts[gi]][cuts[gi + 1]] : opts->kernel;
  if (modelled_s) *modelled_s = kbest > 0 ? best[kbest][nbw] : -1.0;
  return FKREG_OK;
}

fkreg_status fkreg_sweep_create(const fkreg_opts* opts, int64_t max_n, int max_groups,
                                fkreg_sweep* out) {
  if (!out) return FKREG_ERR_INVALID_ARG;
  *out = nullptr;
  int ng0 = 0;
  std::vector<int> first(opts && opts->n_bw > 0 ? opts->n_bw + 1 : 1);
  std::vector<int> gk(first.size(), FKREG_KERNEL_GAUSSIAN);
  fkreg_status st0 =
      fkreg_sweep_split(opts, max_n, max_groups, &ng0, first.data(), gk.data(), nullptr);
  if (st0 != FKREG_OK) return st0;
  auto* S = new fkreg_sweep_s();
  S->o = *opts;
  const int d = opts->dim, nbw = opts->n_bw;
  S->H.assign(opts->H, opts->H + size_t(nbw) * d * d);
  S->o.H = S->H.data();
  for (int j = 0; j < d; ++j) S->M *= opts->grid_n[j];
  S->tsize = opts->precision == FKREG_F32 ? 4 : 8;
  S->first.assign(first.begin(), first.begin() + ng0 + 1);
  S->kern.assign(gk.begin(), gk.begin() + ng0);
  const int ng = int(S->first.size()) - 1;
  for (int gi = 0; gi < ng; ++gi) {
    fkreg_opts g = S->o;
    g.n_bw = S->first[gi + 1] - S->first[gi];
    g.H = S->H.data() + size_t(S->first[gi]) * d * d;
    g.kernel = S->kern[gi];
    fkreg_plan p = nullptr;
    const fkreg_status st = fkreg_plan_create(&g, max_n, &p);
    if (st != FKREG_OK) {
      for (auto q : S->plans) fkreg_plan_destroy(q);
      delete S;
      return st;
    }
    S->plans.push_back(p);
    size_t b = 0;
    fkreg_workspace_bytes(p, &b);
    S->ws_off.push_back(S->ws_bytes);
    S->ws_bytes += (b + 255) / 256 * 256;
  }
  fkreg_geometry g0{};
  fkreg_geometry_query(opts, &g0);
  S->ns = g0.ns;
  S->nt = g0.nt;
  *out = S;
  return FKREG_OK;
}

fkreg_status fkreg_sweep_groups(fkreg_sweep S, int* n_groups, int* first_bw,
                                int* group_kernel, fkreg_geometry* geoms) {
  if (!S || !n_groups) return FKREG_ERR_INVALID_ARG;
  const int ng = int(S->plans.size());
  *n_groups = ng;
  if (first_bw)
    for (int gi = 0; gi <= ng; ++gi) first_bw[gi] = S->first[gi];
  if (group_kernel)
    for (int gi = 0; gi < ng; ++gi) group_kernel[gi] = S->kern[gi];
  if (geoms)
    for (int gi = 0; gi < ng; ++gi) {
      fkreg_opts g = S->o;
      g.n_bw = S->first[gi + 1] - S->first[gi];
      g.H = S->H.data() + size_t(S->first[gi]) * S->o.dim * S->o.dim;
      g.kernel = S->kern[gi];
      const fkreg_status st = fkreg_geometry_query(&g, &geoms[gi]);
      if (st != FKREG_OK) return sweep_err(S, st, fkreg_global_error());
    }
  return FKREG_OK;
}

fkreg_status fkreg_sweep_workspace_bytes(fkreg_sweep S, size_t* bytes) {
  if (!S || !bytes) return FKREG_ERR_INVALID_ARG;
  *bytes = S->ws_bytes;
  return FKREG_OK;
}

fkreg_status fkreg_sweep_set_workspace(fkreg_sweep S, void* ws, size_t bytes, void* stream) {
  if (!S || !ws) return FKREG_ERR_INVALID_ARG;
  if (bytes < S->ws_bytes) return sweep_err(S, FKREG_ERR_INVALID_ARG, "workspace too small");
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0)
    return sweep_err(S, FKREG_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  for (size_t gi = 0; gi < S->plans.size(); ++gi) {
    const size_t nb = (gi + 1 < S->plans.size() ? S->ws_off[gi + 1] : S->ws_bytes) - S->ws_off[gi];
    const fkreg_status st =
        fkreg_set_workspace(S->plans[gi], static_cast<char*>(ws) + S->ws_off[gi], nb, stream);
    if (st != FKREG_OK) return child_err(S, gi, st);
  }
  return FKREG_OK;
}

fkreg_status fkreg_sweep_set_points(fkreg_sweep S, int64_t n, const void* x_dev, void* stream) {
  if (!S) return FKREG_ERR_INVALID_ARG;
  for (size_t gi = 0; gi < S->plans.size(); ++gi) {
    const fkreg_status st = fkreg_set_points(S->plans[gi], n, x_dev, stream);
    if (st != FKREG_OK) return child_err(S, gi, st);
  }
  S->n = n;
  return FKREG_OK;
}

fkreg_status fkreg_sweep_smooth(fkreg_sweep S, const void* y_dev, const fkreg_outputs* out,
                                void* stream) {
  if (!S) return FKREG_ERR_INVALID_ARG;
  for (size_t gi = 0; gi < S->plans.size(); ++gi) {
    const fkreg_outputs o = slice(S, out, S->first[gi]);
    const fkreg_status st = fkreg_smooth(S->plans[gi], y_dev, out ? &o : nullptr, stream);
    if (st != FKREG_OK) return child_err(S, gi, st);
  }
  return FKREG_OK;
}

fkreg_status fkreg_sweep_df(fkreg_sweep S, const void* y_dev, int n_probes, uint64_t seed,
                            const void* probes_dev, const fkreg_outputs* out, void* stream) {
  if (!S) return FKREG_ERR_INVALID_ARG;
  for (size_t gi = 0; gi < S->plans.size(); ++gi) {
    const fkreg_outputs o = slice(S, out, S->first[gi]);
    const fkreg_status st =
        fkreg_df(S->plans[gi], y_dev, n_probes, seed, probes_dev, out ? &o : nullptr, stream);
    if (st != FKREG_OK) return child_err(S, gi, st);
  }
  return FKREG_OK;
}

fkreg_status fkreg_sweep_variance(fkreg_sweep S, const void* y_dev, const void* mhat_at_x_dev,
                                  void* sigma2_grid_dev, void* stream) {
  if (!S) return FKREG_ERR_INVALID_ARG;
  const size_t esz = S->tsize * (S->o.y_complex ? 2 : 1);
  const size_t R = size_t(S->o.n_rhs);
  for (size_t gi = 0; gi < S->plans.size(); ++gi) {
    const size_t b0 = size_t(S->first[gi]);
    const void* mh = mhat_at_x_dev ? static_cast<const char*>(mhat_at_x_dev) +
                                         b0 * R * size_t(S->n) * esz
                                   : nullptr;
    void* s2 = byte_off(sigma2_grid_dev, b0 * R * size_t(S->M) * S->tsize);
    const fkreg_status st = fkreg_variance(S->plans[gi], y_dev, mh, s2, stream);
    if (st != FKREG_OK) return child_err(S, gi, st);
  }
  return FKREG_OK;
}

fkreg_status fkreg_sweep_log_variance(fkreg_sweep S, const void* y_dev, const void* mhat_at_x_dev,
                                      void* v_grid_dev, void* v_at_x_dev, double* kappa_dev,
                                      void* sigma2_grid_dev, void* stream) {
  if (!S) return FKREG_ERR_INVALID_ARG;
  const size_t R = size_t(S->o.n_rhs), T = S->tsize;
  for (size_t gi = 0; gi < S->plans.size(); ++gi) {
    const size_t b0 = size_t(S->first[gi]);
    const void* mh = mhat_at_x_dev
                         ? static_cast<const char*>(mhat_at_x_dev) + b0 * R * size_t(S->n) * T
                         : nullptr;
    const fkreg_status st = fkreg_log_variance(
        S->plans[gi], y_dev, mh, byte_off(v_grid_dev, b0 * R * size_t(S->M) * T),
        byte_off(v_at_x_dev, b0 * R * size_t(S->n) * T), kappa_dev ? kappa_dev + b0 * R : nullptr,
        byte_off(sigma2_grid_dev, b0 * R * size_t(S->M) * T), stream);
    if (st != FKREG_OK) return child_err(S, gi, st);
  }
  return FKREG_OK;
}

fkreg_status fkreg_sweep_backward(fkreg_sweep S, const void* y_dev, int n_probes, uint64_t seed,
                                  const void* probes_dev, int b, double* gcv_dev,
                                  double* dlogh_dev, void* dy_dev, void* dx_dev, void* stream) {
  if (!S) return FKREG_ERR_INVALID_ARG;
  if (b < 0 || b >= S->o.n_bw) return sweep_err(S, FKREG_ERR_INVALID_ARG, "b outside [0, n_bw)");
  size_t gi = 0;
  while (gi + 1 < S->plans.size() && b >= S->first[gi + 1]) ++gi;
  const fkreg_status st = fkreg_backward(S->plans[gi], y_dev, n_probes, seed, probes_dev,
                                         b - S->first[gi], gcv_dev, dlogh_dev, dy_dev, dx_dev,
                                         stream);
  return child_err(S, gi, st);
}

fkreg_status fkreg_sweep_sync_status(fkreg_sweep S, void* stream) {
  if (!S) return FKREG_ERR_INVALID_ARG;
  fkreg_status first = FKREG_OK;
  for (size_t gi = 0; gi < S->plans.size(); ++gi) {
    const fkreg_status st = fkreg_sync_status(S->plans[gi], stream);
    if (st != FKREG_OK && first == FKREG_OK) first = child_err(S, gi, st);
  }
  return first;
}

fkreg_status fkreg_sweep_set_timing(fkreg_sweep S, int enable) {
  if (!S) return FKREG_ERR_INVALID_ARG;
  for (auto p : S->plans) fkreg_set_timing(p, enable);
  return FKREG_OK;
}

fkreg_status fkreg_sweep_stage_times(fkreg_sweep S, double* ms, int64_t* launches,
                                     int64_t* kernel_launches) {
  if (!S) return FKREG_ERR_INVALID_ARG;
  double tms[FKREG_N_STAGES] = {};
  int64_t tl[FKREG_N_STAGES] = {};
  int64_t tk = 0;
  for (size_t gi = 0; gi < S->plans.size(); ++gi) {
    double m[FKREG_N_STAGES];
    int64_t l[FKREG_N_STAGES], k = 0;
    const fkreg_status st = fkreg_stage_times(S->plans[gi], m, l, &k);
    if (st != FKREG_OK) return child_err(S, gi, st);
    for (int i = 0; i < FKREG_N_STAGES; ++i) {
      tms[i] += m[i];
      tl[i] += l[i];
    }
    tk += k;
  }
  for (int i = 0; i < FKREG_N_STAGES; ++i) {
    if (ms) ms[i] = tms[i];
    if (launches) launches[i] = tl[i];
  }
  if (kernel_launches) *kernel_launches = tk;
  return FKREG_OK;
}

const char* fkreg_sweep_last_error(fkreg_sweep S) { return S ? S->err.c_str() : ""; }

void fkreg_sweep_destroy(fkreg_sweep S) {
  if (!S) return;
  for (auto p : S->plans) fkreg_plan_destroy(p);
  delete S;
}

}  // extern "C"
