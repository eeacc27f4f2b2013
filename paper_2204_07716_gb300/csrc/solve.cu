// Local-polynomial solves on the grid lattice.
//
// At every grid point the s- and t-fields give the normal equations
// S(g) beta = t(g) of eqs. 3 / 11 (S_ab = s_(a+b)).  They are assembled in
// FP64 in the scaled basis u = diag(sigma)^-1 (x_i - g), which leaves the
// intercept unchanged, solved in closed form (p <= 3) or by Gaussian
// elimination with partial pivoting (p = 4), and mhat = e_1^T S^-1 t.  Grid points whose density s_0 is below
// mask_rho * max s_0 are masked (NaN estimate, mask 0).
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "internal.h"

namespace fk {

namespace {

template <typename T>
__global__ void smax_kernel(GeoDev g, int64_t Mtot, const T* __restrict__ field, int fgrid,
                            int64_t lcells, T* __restrict__ smax, int bw_count) {
  // every lane stays to the end (warp shuffles below); out-of-range lanes add 0
  const int64_t gid0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool in_range = gid0 < Mtot * bw_count;
  const int64_t gid = in_range ? gid0 : Mtot * bw_count - 1;
  const int64_t m = gid % Mtot;
  const int bb = int(gid / Mtot);
  int64_t rem = m, lidx = 0, mi[3];
  for (int a = 2; a >= 0; --a) {
    mi[a] = rem % g.M[a];
    rem /= g.M[a];
  }
  for (int a = 0; a < 3; ++a) lidx = lidx * g.L[a] + mi[a];
  T v = in_range ? field[(int64_t(bb) * fgrid) * lcells + lidx] : T(0);
  if (!(v > T(0))) v = T(0);
  // block maximum first, then one atomic per block (all threads of a block
  // share the bandwidth unless a block straddles two of them: then per warp)
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_down_sync(0xffffffffu, v, o));
  const int bb0 = __shfl_sync(0xffffffffu, bb, 0);
  const bool uniform = __all_sync(0xffffffffu, bb == bb0);
  if ((threadIdx.x & 31) == 0 && v > T(0)) {
    if (!uniform) {
      // rare: the warp spans two bandwidths; fall back to per-thread atomics below
    } else if (sizeof(T) == 4) {
      atomicMax(reinterpret_cast<unsigned int*>(smax + bb), __float_as_uint(float(v)));
    } else {
      atomicMax(reinterpret_cast<unsigned long long*>(smax + bb),
                (unsigned long long)__double_as_longlong(double(v)));
    }
  }
  if (!uniform && in_range) {
    T vv = field[(int64_t(bb) * fgrid) * lcells + lidx];
    if (vv > T(0)) {
      if (sizeof(T) == 4)
        atomicMax(reinterpret_cast<unsigned int*>(smax + bb), __float_as_uint(float(vv)));
      else
        atomicMax(reinterpret_cast<unsigned long long*>(smax + bb),
                  (unsigned long long)__double_as_longlong(double(vv)));
    }
  }
}

struct GridOut {
  void* mhat;         // [n_bw][n_rhs][M] (complex if cplx)
  uint8_t* mask;      // [n_bw][M]
  void* moments;      // [n_bw][ns + n_rhs*nt*(1+cplx)][M]
  int cplx;           // real fields come in (re, im) pairs
  int n_rhs_out;      // responses in the output (pairs collapse when cplx)
  double* avec;       // [n_bw][p][M] a_k / tscale_k (NaN where masked), or null
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
  if (!in_range(g.errw, kSiteSolveField, lidx, lcells)) return;
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
    {
      const double isg[3] = {1.0 / B.sigma[0], 1.0 / B.sigma[1], 1.0 / B.sigma[2]};
      ok = lpr_weights_fast(mono, p, s, B.sigma, isg, a);
    }
  }
  const T nan = T(__longlong_as_double(0x7ff8000000000000LL));
  if (out.avec)
    for (int k = 0; k < p; ++k)
      out.avec[(int64_t(b) * p + k) * Mtot + m] =
          ok ? a[k] / tscale(mono, k, B.sigma) : __longlong_as_double(0x7ff8000000000000LL);
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

// sigma2[b][r][m] = sum_k avec[b][k][m] t_(r,k)(g_m): the estimate of the
// variance pass from the grid weights a smoothing pass kept (NaN where that
// pass masked the point); field holds the R x p t-fields only.
template <typename T>
__global__ void grid_apply_kernel(GeoDev g, int64_t Mtot, int p, int nrhs_fields,
                                  const double* __restrict__ avec, const T* __restrict__ field,
                                  int64_t lcells, T* __restrict__ sigma2) {
  const int64_t m = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (m >= Mtot) return;
  int64_t rem = m, lidx = 0, mi[3];
  for (int a = 2; a >= 0; --a) {
    mi[a] = rem % g.M[a];
    rem /= g.M[a];
  }
  for (int a = 0; a < 3; ++a) lidx = lidx * g.L[a] + mi[a];
  if (!in_range(g.errw, kSiteSolveField, lidx, lcells)) return;
  double w[kMaxP];
  for (int k = 0; k < p; ++k) w[k] = avec[int64_t(k) * Mtot + m];
  for (int r = 0; r < nrhs_fields; ++r) {
    double v = 0.0;
    for (int k = 0; k < p; ++k) v += w[k] * double(field[(int64_t(r) * p + k) * lcells + lidx]);
    sigma2[int64_t(r) * Mtot + m] = T(v);  // NaN weights give NaN
  }
}

template <typename T>
cudaError_t launch_grid_apply(fkreg_plan_s* P, int b, int nrhs_fields, void* sigma2,
                              cudaStream_t st) {
  const GeoDev& g = P->geo;
  int64_t Mtot = 1, lcells = 1;
  for (int a = 0; a < 3; ++a) {
    Mtot *= g.M[a];
    lcells *= g.L[a];
  }
  const unsigned blocks = unsigned((Mtot + 255) / 256);
  grid_apply_kernel<T><<<blocks, 256, 0, st>>>(
      g, Mtot, P->p, nrhs_fields, wsp<double>(P, P->r_gavec) + int64_t(b) * P->p * Mtot,
      wsp<T>(P, P->r_gfield), lcells, static_cast<T*>(sigma2) + int64_t(b) * nrhs_fields * Mtot);
  P->launches += 1;
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_grid_solve(fkreg_plan_s* P, int bw_first, int bw_count, int nrhs_fields,
                              double* avec, const fkreg_outputs* out, void* sigma2,
                              cudaStream_t st) {
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
  go.avec = avec;
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

}  // namespace

cudaError_t run_grid_solve(fkreg_plan_s* P, int bw_first, int bw_count, int nrhs_fields,
                           double* avec, const fkreg_outputs* out, void* sigma2, cudaStream_t st) {
  return P->prec == FKREG_F32
             ? launch_grid_solve<float>(P, bw_first, bw_count, nrhs_fields, avec, out, sigma2, st)
             : launch_grid_solve<double>(P, bw_first, bw_count, nrhs_fields, avec, out, sigma2, st);
}

cudaError_t run_grid_apply(fkreg_plan_s* P, int b, int nrhs_fields, void* sigma2, cudaStream_t st) {
  return P->prec == FKREG_F32 ? launch_grid_apply<float>(P, b, nrhs_fields, sigma2, st)
                              : launch_grid_apply<double>(P, b, nrhs_fields, sigma2, st);
}

}  // namespace fk

// ---- log-variance estimator (Sec. 3, eqs. 24-26) ------------------------------
// kappa_r = [ (1/N) sum_i r_i exp(-v_r(x_i)) ]^-1 with r_i = (y_ri - mhat_r(x_i))^2,
// then sigma2_r(g) = exp(v_r(g)) / kappa_r on the grid.  Block partial sums in
// FP64, summed in a fixed order (deterministic).
namespace fk {
namespace {

template <typename T>
__global__ void kappa_partial_kernel(int64_t n, int n_rhs, int b, const T* __restrict__ y,
                                     const T* __restrict__ mh, const T* __restrict__ v,
                                     double* __restrict__ part) {
  __shared__ double red[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r = 0; r < n_rhs; ++r) {
    double t = 0.0;
    const T* yr = y + int64_t(r) * n;
    const T* mr = mh + (int64_t(b) * n_rhs + r) * n;
    const T* vr = v + (int64_t(b) * n_rhs + r) * n;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
      const T d = yr[i] - mr[i];
      t += double(d * d * exp(-vr[i]));
    }
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) red[warp] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < int(blockDim.x >> 5); ++w) s += red[w];
      part[int64_t(blockIdx.x) * n_rhs + r] = s;
    }
    __syncthreads();
  }
}

__global__ void kappa_finish_kernel(const double* __restrict__ part, int nblk, int n_rhs, int b,
                                    int64_t n, double* __restrict__ kappa) {
  __shared__ double sh[256];
  const int r = blockIdx.x;
  double t = 0.0;
  for (int k = threadIdx.x; k < nblk; k += blockDim.x) t += part[int64_t(k) * n_rhs + r];
  sh[threadIdx.x] = t;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) kappa[int64_t(b) * n_rhs + r] = double(n) / sh[0];
}

template <typename T>
__global__ void sigma2_from_v_kernel(int64_t Mtot, int n_rhs, int b, const T* __restrict__ v,
                                     const double* __restrict__ kappa, T* __restrict__ sigma2) {
  const int64_t gid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (gid >= Mtot * n_rhs) return;
  const int r = int(gid / Mtot);
  const int64_t o = int64_t(b) * n_rhs * Mtot + gid;
  sigma2[o] = T(double(exp(v[o])) / kappa[int64_t(b) * n_rhs + r]);
}

}  // namespace

cudaError_t run_kappa_sigma2(fkreg_plan_s* P, int b, const void* y, const void* mhat_at_x,
                             const void* v_at_x, const void* v_grid, double* kappa, void* sigma2,
                             cudaStream_t st) {
  const int R = P->nrhs;
  const int nblk = 512;
  double* part = wsp<double>(P, P->r_part);
  int64_t Mtot = 1;
  for (int a = 0; a < 3; ++a) Mtot *= P->geo.M[a];
  const unsigned gb = unsigned((Mtot * R + 255) / 256);
  if (P->prec == FKREG_F32) {
    kappa_partial_kernel<float><<<nblk, 256, 0, st>>>(P->n, R, b, static_cast<const float*>(y),
                                                      static_cast<const float*>(mhat_at_x),
                                                      static_cast<const float*>(v_at_x), part);
  } else {
    kappa_partial_kernel<double><<<nblk, 256, 0, st>>>(P->n, R, b, static_cast<const double*>(y),
                                                       static_cast<const double*>(mhat_at_x),
                                                       static_cast<const double*>(v_at_x), part);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  kappa_finish_kernel<<<R, 256, 0, st>>>(part, nblk, R, b, P->n, kappa);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (sigma2) {
    if (P->prec == FKREG_F32)
      sigma2_from_v_kernel<float><<<gb, 256, 0, st>>>(Mtot, R, b, static_cast<const float*>(v_grid),
                                                      kappa, static_cast<float*>(sigma2));
    else
      sigma2_from_v_kernel<double><<<gb, 256, 0, st>>>(Mtot, R, b, static_cast<const double*>(v_grid),
                                                       kappa, static_cast<double*>(sigma2));
  }
  P->launches += sigma2 ? 3 : 2;
  return cudaGetLastError();
}

}  // namespace fk

// ---- pointwise interval (Sec. 4.2, eq. 28) -------------------------------------
namespace fk {
namespace {

template <typename T>
__global__ void interval_kernel(int64_t count, const T* __restrict__ mhat, const T* __restrict__ var,
                                double alpha, T* __restrict__ lower, T* __restrict__ upper) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const T z = T(normcdfinv(1.0 - 0.5 * alpha));  // z_(1 - alpha/2)
  const T v = var[i];
  const T sd = v >= T(0) ? sqrt(v) : T(__longlong_as_double(0x7ff8000000000000LL));
  lower[i] = mhat[i] - z * sd;
  upper[i] = mhat[i] + z * sd;
}

}  // namespace
}  // namespace fk

extern "C" fkreg_status fkreg_interval(int precision, int64_t count, const void* mhat_dev,
                                       const void* var_dev, double alpha, void* lower_dev,
                                       void* upper_dev, void* stream) {
  using namespace fk;
  if (precision != FKREG_F32 && precision != FKREG_F64) return FKREG_ERR_INVALID_ARG;
  if (count < 0 || !(alpha > 0.0 && alpha < 1.0)) return FKREG_ERR_INVALID_ARG;
  if (count == 0) return FKREG_OK;
  if (!mhat_dev || !var_dev || !lower_dev || !upper_dev) return FKREG_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const unsigned blocks = unsigned((count + 255) / 256);
  if (precision == FKREG_F32)
    interval_kernel<float><<<blocks, 256, 0, s>>>(count, static_cast<const float*>(mhat_dev),
                                                  static_cast<const float*>(var_dev), alpha,
                                                  static_cast<float*>(lower_dev),
                                                  static_cast<float*>(upper_dev));
  else
    interval_kernel<double><<<blocks, 256, 0, s>>>(count, static_cast<const double*>(mhat_dev),
                                                   static_cast<const double*>(var_dev), alpha,
                                                   static_cast<double*>(lower_dev),
                                                   static_cast<double*>(upper_dev));
  return cudaGetLastError() == cudaSuccess ? FKREG_OK : FKREG_ERR_CUDA;
}
