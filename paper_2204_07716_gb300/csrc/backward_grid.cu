// Vector-Jacobian product of the grid estimate mhat(g) = e_1^T S(g)^-1 t(g)
// (eqs. 3, 9, 11) for caller-supplied adjoints Gbar_r(g) = dL/dmhat_r(g):
//
//   per grid point (FP64): a = S^-1 e_1, beta_r = S^-1 t_r,
//     tbar_(r,k) = Gbar_r a_k                           (dL/dt_(r,k)(g))
//     sbar_g     = -sum_(i+j = g) a_i sum_r Gbar_r beta_(r,j)   (dL/ds_g(g))
//   written as real adjoint fields Qbar on the length-L lattice of the grid
//   (zero off the output points and at masked points, whose estimate is NaN);
//   their forward DFT and the kernel multipliers give the adjoint functions
//   E_f(x) = sum_g Qbar_f(g) w_f(x - g) at the samples (spectral.cu), so
//     dL/dy_(r,j) = sum_(f in t-fields of r) E_f(x_j)
//     dL/dx_j     = sum_f c_(class f, j) grad E_f(x_j)   (c = 1 for the s-fields)
//   and dL/dlog sigma is a spectral inner product (spectral.cu).
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "internal.h"

namespace fk {

namespace {

template <typename T>
__global__ void grid_adjoint_kernel(GeoDev g, MonoTab mono, const BwDev* __restrict__ bwt, int b,
                                    int order, int64_t Mtot, const T* __restrict__ field,
                                    int64_t lcells, int nrhs, const uint8_t* __restrict__ mask,
                                    const T* __restrict__ gbar, T* __restrict__ qbar) {
  const int64_t m = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (m >= Mtot || !mask[m]) return;
  int64_t rem = m, lidx = 0, mi[3];
  for (int a = 2; a >= 0; --a) {
    mi[a] = rem % g.M[a];
    rem /= g.M[a];
  }
  for (int a = 0; a < 3; ++a) lidx = lidx * g.L[a] + mi[a];
  const BwDev& B = bwt[b];
  const int ns = mono.n, nt = mono.nt, p = nt;
  double sv[kMaxMono];
  for (int k = 0; k < kMaxMono; ++k) sv[k] = k < ns ? double(field[int64_t(k) * lcells + lidx]) : 0.0;
  // unscaled inverse of S from the scaled system (elimination, FP64)
  double tsc[kMaxP];
  for (int k = 0; k < kMaxP; ++k) tsc[k] = k < p ? 1.0 / tscale(mono, k, B.sigma) : 0.0;
  double Sinv[kMaxP][kMaxP];
  bool ok = true;
  if (order == 0) {
    ok = sv[0] > 0.0;
    Sinv[0][0] = ok ? 1.0 / sv[0] : 0.0;
  } else {
    for (int c = 0; c < p && ok; ++c) {
      double S[kMaxP][kMaxP], rhs[kMaxP], col[kMaxP];
      for (int i = 0; i < p; ++i) {
        rhs[i] = (i == c) ? 1.0 : 0.0;
        for (int j = 0; j < p; ++j) {
          const int e0 = mono.e[i][0] + mono.e[j][0], e1 = mono.e[i][1] + mono.e[j][1],
                    e2 = mono.e[i][2] + mono.e[j][2];
          S[i][j] = sv[mono_index(mono, ns, e0, e1, e2)] * tsc[i] * tsc[j];
        }
      }
      for (int cc = 0; cc < p && ok; ++cc) {
        int piv = cc;
        for (int i = cc + 1; i < p; ++i)
          if (fabs(S[i][cc]) > fabs(S[piv][cc])) piv = i;
        if (!(fabs(S[piv][cc]) > 0.0)) {
          ok = false;
          break;
        }
        if (piv != cc) {
          for (int j = 0; j < p; ++j) {
            const double t = S[cc][j];
            S[cc][j] = S[piv][j];
            S[piv][j] = t;
          }
          const double t = rhs[cc];
          rhs[cc] = rhs[piv];
          rhs[piv] = t;
        }
        for (int i = cc + 1; i < p; ++i) {
          const double fct = S[i][cc] / S[cc][cc];
          for (int j = cc; j < p; ++j) S[i][j] -= fct * S[cc][j];
          rhs[i] -= fct * rhs[cc];
        }
      }
      if (!ok) break;
      for (int i = p - 1; i >= 0; --i) {
        double v = rhs[i];
        for (int j = i + 1; j < p; ++j) v -= S[i][j] * col[j];
        col[i] = v / S[i][i];
      }
      for (int i = 0; i < p; ++i) Sinv[i][c] = col[i] * tsc[i] * tsc[c];
    }
  }
  if (!ok) return;
  double a[kMaxP], bbar[kMaxP];
  for (int i = 0; i < p; ++i) {
    a[i] = Sinv[i][0];
    bbar[i] = 0.0;
  }
  for (int r = 0; r < nrhs; ++r) {
    double gr = double(gbar[int64_t(r) * Mtot + m]);
    if (!isfinite(gr)) gr = 0.0;
    double t[kMaxP];
    for (int k = 0; k < p; ++k) t[k] = double(field[int64_t(ns + r * nt + k) * lcells + lidx]);
    for (int i = 0; i < p; ++i) {
      double beta = 0.0;
      for (int k = 0; k < p; ++k) beta += Sinv[i][k] * t[k];
      bbar[i] += gr * beta;
    }
    for (int k = 0; k < p; ++k) qbar[int64_t(ns + r * nt + k) * lcells + lidx] = T(gr * a[k]);
  }
  for (int gf = 0; gf < ns; ++gf) {
    double q = 0.0;
    for (int i = 0; i < p; ++i)
      for (int j = 0; j < p; ++j)
        if (mono.e[i][0] + mono.e[j][0] == mono.e[gf][0] &&
            mono.e[i][1] + mono.e[j][1] == mono.e[gf][1] &&
            mono.e[i][2] + mono.e[j][2] == mono.e[gf][2])
          q -= a[i] * bbar[j];
    qbar[int64_t(gf) * lcells + lidx] = T(q);
  }
}

// V [nrhs + (1 + nrhs) D][n] (sorted order): the adjoint functions' values
// for each response, then their gradients per class (density, responses).
template <typename T, int D>
__global__ void combine_grid_kernel(int64_t n, int nrhs, const T* __restrict__ V,
                                    const T* __restrict__ str, const uint32_t* __restrict__ perm,
                                    T* __restrict__ dy, T* __restrict__ dx) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const uint32_t i = perm[s];
  if (dy)
    for (int r = 0; r < nrhs; ++r) dy[int64_t(r) * n + i] = V[int64_t(r) * n + s];
  if (dx)
    for (int d = 0; d < D; ++d) {
      if constexpr (sizeof(T) == 4) {
        // compensated FP32 (exact products by fma, two-sum of the total)
        float hi = V[int64_t(nrhs + d) * n + s], lo = 0.f;
        for (int r = 0; r < nrhs; ++r) {
          const float c = str[int64_t(1 + r) * n + s];
          const float v = V[int64_t(nrhs + (1 + r) * D + d) * n + s];
          const float p = c * v, pe = fmaf(c, v, -p);
          const float t = hi + p, z = t - hi;
          lo += ((hi - (t - z)) + (p - z)) + pe;
          hi = t;
        }
        dx[int64_t(i) * D + d] = T(hi + lo);
      } else {
        double v = double(V[int64_t(nrhs + d) * n + s]);
        for (int r = 0; r < nrhs; ++r)
          v += double(str[int64_t(1 + r) * n + s]) * double(V[int64_t(nrhs + (1 + r) * D + d) * n + s]);
        dx[int64_t(i) * D + d] = T(v);
      }
    }
}

template <typename T>
cudaError_t grid_adjoint_t(fkreg_plan_s* P, int b, int nrhs, const uint8_t* mask, const void* gbar,
                           void* qbar, cudaStream_t st) {
  const GeoDev& g = P->geo;
  int64_t Mtot = 1, lcells = 1;
  for (int a = 0; a < 3; ++a) {
    Mtot *= g.M[a];
    lcells *= g.L[a];
  }
  const int fgrid = P->ns + nrhs * P->nt;
  cudaError_t e = cudaMemsetAsync(qbar, 0, sizeof(T) * size_t(fgrid) * lcells, st);
  if (e != cudaSuccess) return e;
  const unsigned blocks = unsigned((Mtot + 127) / 128);
  grid_adjoint_kernel<T><<<blocks, 128, 0, st>>>(g, P->mono, wsp<BwDev>(P, P->r_bw), b, P->order,
                                                Mtot, wsp<T>(P, P->r_gfield), lcells, nrhs, mask,
                                                static_cast<const T*>(gbar), static_cast<T*>(qbar));
  P->launches += 1;
  return cudaGetLastError();
}

template <typename T>
cudaError_t combine_grid_t(fkreg_plan_s* P, int nrhs, const void* V, void* dy, void* dx,
                           cudaStream_t st) {
  if (P->n == 0) return cudaSuccess;
  const unsigned blocks = unsigned((P->n + 255) / 256);
#define FK_CG(DD)                                                                                \
  combine_grid_kernel<T, DD><<<blocks, 256, 0, st>>>(P->n, nrhs, static_cast<const T*>(V),       \
                                                     wsp<T>(P, P->r_str), perm_ptr(P),           \
                                                     static_cast<T*>(dy), static_cast<T*>(dx))
  if (P->d == 1)
    FK_CG(1);
  else if (P->d == 2)
    FK_CG(2);
  else
    FK_CG(3);
#undef FK_CG
  P->launches += 1;
  return cudaGetLastError();
}

}  // namespace

cudaError_t run_grid_adjoint(fkreg_plan_s* P, int b, int nrhs, const uint8_t* mask,
                             const void* gbar, void* qbar, cudaStream_t st) {
  return P->prec == FKREG_F32 ? grid_adjoint_t<float>(P, b, nrhs, mask, gbar, qbar, st)
                              : grid_adjoint_t<double>(P, b, nrhs, mask, gbar, qbar, st);
}

cudaError_t run_combine_grid(fkreg_plan_s* P, int nrhs, const void* V, void* dy, void* dx,
                             cudaStream_t st) {
  return P->prec == FKREG_F32 ? combine_grid_t<float>(P, nrhs, V, dy, dx, st)
                              : combine_grid_t<double>(P, nrhs, V, dy, dx, st);
}

}  // namespace fk
