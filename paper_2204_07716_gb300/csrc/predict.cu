// Values of a grid estimate at new points: the griddedInterpolant step that
// the paper uses to carry grid estimates to arbitrary locations (Sec. 1.1;
// "linear interpolation and extrapolation" in its Sec. 4 timings).
//   linear: multilinear on the lattice of eq. 6, extended linearly from the
//           boundary cell outside the box;
//   cubic:  separable cubic convolution (Keys 1981, a = -1/2) with Keys'
//           boundary rows f[-1] = 3 f[0] - 3 f[1] + f[2] (and the mirror at
//           the top), which keeps it exact for quadratics up to the edges;
//           NaN outside the box.
// One thread per query point; every grid vector (responses, bandwidths) is
// evaluated with the same weights.
#include <cuda_runtime.h>

#include <cmath>

#include "internal.h"

namespace fk {

namespace {

struct PredGeo {
  int64_t M[3];
  double lo[3];
  double inv_delta[3];
  int64_t Mtot;
};

template <typename T, int D, int METHOD>
__global__ void predict_kernel(int64_t nq, const T* __restrict__ xq, int count,
                               const T* __restrict__ grid, PredGeo pg, T* __restrict__ out) {
  constexpr int NW = METHOD == 0 ? 2 : 4;  // window per axis
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  int64_t base[3] = {0, 0, 0};
  T ew[3][NW];
  bool outside = false;
  for (int j = 0; j < D; ++j) {
    const int64_t M = pg.M[j];
    const double u = (double(xq[q * D + j]) - pg.lo[j]) * pg.inv_delta[j];
    int64_t i = int64_t(floor(u));
    i = i < 0 ? 0 : (i > M - 2 ? M - 2 : i);
    const double t = u - double(i);
    for (int k = 0; k < NW; ++k) ew[j][k] = T(0);
    if (METHOD == 0) {
      base[j] = i;
      ew[j][0] = T(1.0 - t);
      ew[j][1] = T(t);
    } else {
      if (u < 0.0 || u > double(M - 1)) outside = true;
      const double tc = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
      const double a = -0.5;
      double w[4];
      for (int k = 0; k < 4; ++k) {
        const double s = fabs(tc + 1.0 - double(k));  // distance to tap i - 1 + k
        w[k] = s <= 1.0 ? ((a + 2.0) * s - (a + 3.0)) * s * s + 1.0
                        : (s < 2.0 ? ((a * s - 5.0 * a) * s + 8.0 * a) * s - 4.0 * a : 0.0);
      }
      const int64_t b0 = i - 1 < 0 ? 0 : (i - 1 > M - 4 ? M - 4 : i - 1);
      base[j] = b0;
      for (int k = 0; k < 4; ++k) {
        const int64_t ii = i - 1 + k;
        if (ii == -1) {
          ew[j][0 - b0] += T(3.0 * w[k]);
          ew[j][1 - b0] += T(-3.0 * w[k]);
          ew[j][2 - b0] += T(w[k]);
        } else if (ii == M) {
          ew[j][M - 1 - b0] += T(3.0 * w[k]);
          ew[j][M - 2 - b0] += T(-3.0 * w[k]);
          ew[j][M - 3 - b0] += T(w[k]);
        } else {
          ew[j][ii - b0] += T(w[k]);
        }
      }
    }
  }
  const T nan = T(__longlong_as_double(0x7ff8000000000000LL));
  for (int c = 0; c < count; ++c) {
    const T* gc = grid + int64_t(c) * pg.Mtot;
    T v = T(0);
    for (int k0 = 0; k0 < NW; ++k0) {
      const int64_t r0 = base[0] + k0;
      if (D == 1) {
        v += ew[0][k0] * gc[r0];
        continue;
      }
      for (int k1 = 0; k1 < NW; ++k1) {
        const int64_t r1 = r0 * pg.M[1] + base[1] + k1;
        const T w01 = ew[0][k0] * ew[1][k1];
        if (D == 2) {
          v += w01 * gc[r1];
          continue;
        }
        for (int k2 = 0; k2 < NW; ++k2) v += w01 * ew[2][k2] * gc[r1 * pg.M[2] + base[2] + k2];
      }
    }
    out[int64_t(c) * nq + q] = outside ? nan : v;
  }
}

template <typename T, int D>
void launch_predict(int method, int64_t nq, const void* xq, int count, const void* grid,
                    const PredGeo& pg, void* out, cudaStream_t s) {
  const unsigned blocks = unsigned((nq + 255) / 256);
  if (method == 0)
    predict_kernel<T, D, 0><<<blocks, 256, 0, s>>>(nq, static_cast<const T*>(xq), count,
                                                   static_cast<const T*>(grid), pg,
                                                   static_cast<T*>(out));
  else
    predict_kernel<T, D, 1><<<blocks, 256, 0, s>>>(nq, static_cast<const T*>(xq), count,
                                                   static_cast<const T*>(grid), pg,
                                                   static_cast<T*>(out));
}

}  // namespace

}  // namespace fk

extern "C" fkreg_status fkreg_predict(int precision, int dim, const int64_t* grid_n,
                                      const double* grid_lo, const double* grid_hi, int count,
                                      const void* grid_dev, int64_t nq, const void* xq_dev,
                                      int method, void* out_dev, void* stream) {
  using namespace fk;
  if (precision != FKREG_F32 && precision != FKREG_F64) return FKREG_ERR_INVALID_ARG;
  if (dim < 1 || dim > 3 || !grid_n || !grid_lo || !grid_hi) return FKREG_ERR_INVALID_ARG;
  if (method != 0 && method != 1) return FKREG_ERR_INVALID_ARG;
  if (count < 0 || nq < 0) return FKREG_ERR_INVALID_ARG;
  PredGeo pg{};
  pg.Mtot = 1;
  for (int j = 0; j < 3; ++j) {
    pg.M[j] = 1;
    pg.lo[j] = 0.0;
    pg.inv_delta[j] = 0.0;
  }
  for (int j = 0; j < dim; ++j) {
    if (grid_n[j] < (method == 0 ? 2 : 4) || !(grid_hi[j] > grid_lo[j])) return FKREG_ERR_INVALID_ARG;
    pg.M[j] = grid_n[j];
    pg.lo[j] = grid_lo[j];
    pg.inv_delta[j] = double(grid_n[j] - 1) / (grid_hi[j] - grid_lo[j]);
    pg.Mtot *= grid_n[j];
  }
  if (nq == 0 || count == 0) return FKREG_OK;
  if (!grid_dev || !xq_dev || !out_dev) return FKREG_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == FKREG_F32) {
    if (dim == 1) launch_predict<float, 1>(method, nq, xq_dev, count, grid_dev, pg, out_dev, s);
    else if (dim == 2) launch_predict<float, 2>(method, nq, xq_dev, count, grid_dev, pg, out_dev, s);
    else launch_predict<float, 3>(method, nq, xq_dev, count, grid_dev, pg, out_dev, s);
  } else {
    if (dim == 1) launch_predict<double, 1>(method, nq, xq_dev, count, grid_dev, pg, out_dev, s);
    else if (dim == 2) launch_predict<double, 2>(method, nq, xq_dev, count, grid_dev, pg, out_dev, s);
    else launch_predict<double, 3>(method, nq, xq_dev, count, grid_dev, pg, out_dev, s);
  }
  return cudaGetLastError() == cudaSuccess ? FKREG_OK : FKREG_ERR_CUDA;
}
