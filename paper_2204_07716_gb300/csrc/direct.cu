// Direct-sum path for the compact regression kernels (Table 1: uniform,
// Epanechnikov, triangle, biweight, triweight).  Their Fourier transforms
// decay only algebraically, so the NUFFT's truncation cannot be controlled by
// a tolerance; instead the moment sums of eq. 9 are summed exactly over the
// samples inside each point's support (an ellipsoid |H^(-1/2) z| <= 1), found
// through the bins of the sort.  This file computes the grid fields; the
// grid solve (solve.cu) and the at-sample pass (interp.cu) follow as for the
// Gaussian path.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "internal.h"

namespace fk {

namespace {

constexpr int kDirectMaxFields = 64;

// thread per (grid point m, bandwidth bw_first + bb): fields [bb][fgrid][Mtot]
template <typename T>
__global__ void direct_grid_kernel(GeoDev g, MonoTab mono, const BwDev* __restrict__ bwt,
                                   int bw_first, int bw_count, int64_t Mtot, int64_t n,
                                   const T* __restrict__ xs, const T* __restrict__ str,
                                   int str_first, int nstr, const uint32_t* __restrict__ bin_start,
                                   int fgrid, T* __restrict__ field) {
  const int64_t gid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (gid >= Mtot * bw_count) return;
  const int64_t m = gid % Mtot;
  const int bb = int(gid / Mtot);
  const BwDev& B = bwt[bw_first + bb];
  double q[3] = {0.0, 0.0, 0.0};
  int64_t rem = m;
  for (int a = g.d - 1; a >= 0; --a) {
    const int64_t idx = rem % g.M[a];
    rem /= g.M[a];
    q[a] = double(idx) * (g.hi[a] - g.lo[a]) / double(g.M[a] - 1);
  }
  double acc[kDirectMaxFields];
  direct_sums<T>(g, mono, B, n, xs, str, str_first, nstr, bin_start, q, acc);
  for (int f = 0; f < fgrid; ++f) field[(int64_t(bb) * fgrid + f) * Mtot + m] = T(acc[f]);
}

}  // namespace

cudaError_t run_direct_grid(fkreg_plan_s* P, int str_first, int nstr, int bw_first,
                            int bw_count, cudaStream_t st) {
  int64_t Mtot = 1;
  for (int a = 0; a < 3; ++a) Mtot *= P->geo.M[a];
  const int fgrid = P->ns + nstr * P->nt;
  if (fgrid > kDirectMaxFields) return cudaErrorInvalidValue;
  const unsigned blocks = unsigned((Mtot * bw_count + 127) / 128);
  if (P->prec == FKREG_F32)
    direct_grid_kernel<float><<<blocks, 128, 0, st>>>(
        P->geo, P->mono, wsp<BwDev>(P, P->r_bw), bw_first, bw_count, Mtot, P->n,
        wsp<float>(P, P->r_xs), wsp<float>(P, P->r_str), str_first, nstr,
        wsp<uint32_t>(P, P->r_binstart), fgrid, wsp<float>(P, P->r_gfield));
  else
    direct_grid_kernel<double><<<blocks, 128, 0, st>>>(
        P->geo, P->mono, wsp<BwDev>(P, P->r_bw), bw_first, bw_count, Mtot, P->n,
        wsp<double>(P, P->r_xs), wsp<double>(P, P->r_str), str_first, nstr,
        wsp<uint32_t>(P, P->r_binstart), fgrid, wsp<double>(P, P->r_gfield));
  P->launches += 1;
  return cudaGetLastError();
}

}  // namespace fk
