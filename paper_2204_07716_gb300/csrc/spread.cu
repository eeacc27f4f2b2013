// Type-1 spreading (the gridding of Sec. 1.2, eqs. 16-17) and strength setup.
//
// fine_s[m] = sum_i c_{s,i} prod_j phi(m_j - u_ij),  u_ij = (x_ij - lo_j) nf_j / P_j,
// periodic in m_j (mod nf_j).  One CTA owns one sub-problem: up to kSubMax
// sorted samples of one bin, accumulated into a shared-memory copy of the
// bin's tile plus a halo of ceil(w/2) cells per side; the CTA then adds the
// tile to the fine grid in global memory with one atomic per non-zero cell.
// Two kernels fill the tile.  1-D and 2-D plans of a compile-time width use
// spread_run_kernel: the lanes of a warp cover the window cells and sum runs
// of consecutive samples that share a window (the sort puts them together)
// in registers before one shared-memory atomic per cell and strength.  3-D
// and runtime widths use spread_kernel: each thread adds one sample's w^d
// window at a time.  Strengths go in chunks that fit the shared-memory
// budget.
#include <cuda_runtime.h>

#include <algorithm>

#include "device_common.cuh"
#include "internal.h"

namespace fk {

namespace {

constexpr int kSpreadThreads = 256;
constexpr int kMaxChunk = 8;
constexpr int kMaxWRun = 24;
constexpr int kMaxChunk2 = 16;  // strengths per launch of the run kernel

// Shared-memory accumulator of the tile.  FP32 plans accumulate in 32-bit
// fixed point (native integer shared-memory atomics); the scale of each
// strength is 2^30 / sum_i |c_i| over the sub-problem, so no cell can
// overflow (every spreading weight is <= 1) and one rounding step is
// sum_i |c_i| / 2^31.  FP64 plans accumulate doubles directly.
template <typename T>
struct TileAcc {
  using type = T;
  static __device__ __forceinline__ void add(T* p, T v) { atomicAdd(p, v); }
};
template <>
struct TileAcc<float> {
  using type = int;
  static __device__ __forceinline__ void add(int* p, float v) { atomicAdd(p, __float2int_rn(v)); }
};

template <typename T, int D, int W, int CN>
__global__ void __launch_bounds__(kSpreadThreads)
spread_kernel(GeoDev g, int64_t n, const T* __restrict__ xs, const T* __restrict__ str, int s0,
              int scount, int chunk, const uint32_t* __restrict__ sub_bin,
              const uint32_t* __restrict__ sub_first, const uint32_t* __restrict__ bin_start,
              const uint32_t* __restrict__ sub_total, T* __restrict__ fine) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using A = typename TileAcc<T>::type;
  A* sm = reinterpret_cast<A*>(smem_raw);
  __shared__ T s_scale[kMaxChunk], s_inv[kMaxChunk];
  __shared__ T s_red[kSpreadThreads / 32][kMaxChunk];
  const uint32_t k = blockIdx.x;
  if (k >= *sub_total) return;
  const uint32_t b = sub_bin[k];
  const uint32_t first = sub_first[k];
  const uint32_t last = min(first + uint32_t(kSubMax), bin_start[b + 1]);
  int64_t bj[3] = {0, 0, 0};
  {
    int64_t rem = b;
    for (int j = D - 1; j >= 0; --j) {
      bj[j] = rem % g.nbins[j];
      rem /= g.nbins[j];
    }
  }
  int64_t o[3] = {0, 0, 0};
  int W3[3] = {1, 1, 1};
  for (int j = 0; j < D; ++j) {
    o[j] = bj[j] * g.tile[j] - g.pad;
    W3[j] = int(g.tile[j]) + 2 * g.pad;
  }
  const int cells = W3[0] * W3[1] * W3[2];
  const int w = W > 0 ? W : g.w;
  const T beta = T(g.beta);
  const T halfw = T(0.5) * T(w);
  const int64_t fine_cells = g.nf[0] * g.nf[1] * g.nf[2];
  constexpr int WR = W > 0 ? W : kMaxWRun;

  // one launch handles CN strengths [s0, s0 + CN) (scount and chunk are CN)
  for (int c0 = 0; c0 < 1; ++c0) {
    constexpr int cn = CN;
    for (int idx = threadIdx.x; idx < cn * cells; idx += blockDim.x) sm[idx] = A(0);
    if (sizeof(A) == 4) {
      // fixed-point scale per strength: 2^30 / sum |c| over this sub-problem
      T part[CN];
#pragma unroll
      for (int c = 0; c < CN; ++c) part[c] = T(0);
      for (uint32_t p = first + threadIdx.x; p < last; p += blockDim.x)
#pragma unroll
        for (int c = 0; c < CN; ++c) part[c] += fabs(str[int64_t(s0 + c0 + c) * n + p]);
#pragma unroll
      for (int c = 0; c < CN; ++c) {
        const T v = warp_sum_t<T>(part[c]);
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5][c] = v;
      }
      __syncthreads();
      if (threadIdx.x < CN) {
        T tot = T(0);
        for (int wv = 0; wv < kSpreadThreads / 32; ++wv) tot += s_red[wv][threadIdx.x];
        const T sc = tot > T(0) ? T(1073741824.0) / tot : T(0);
        s_scale[threadIdx.x] = sc;
        s_inv[threadIdx.x] = tot > T(0) ? tot / T(1073741824.0) : T(0);
      }
    } else if (threadIdx.x < CN) {
      s_scale[threadIdx.x] = T(1);
      s_inv[threadIdx.x] = T(1);
    }
    __syncthreads();
    for (uint32_t p = first + threadIdx.x; p < last; p += blockDim.x) {
      T wt[D][WR];
      int l[3] = {0, 0, 0};
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const T u = mul_rn(xs[int64_t(j) * n + p], inv_h_of<T>(g, j));
        const T f0 = ceil(u - halfw);
        l[j] = int(int64_t(f0) - o[j]);
        const T off = f0 - u;
        if constexpr (W > 0) {
#pragma unroll
          for (int t = 0; t < W; ++t) wt[j][t] = phi<T>(g.skind, w, beta, off + T(t));
        } else {
          for (int t = 0; t < w; ++t) wt[j][t] = phi<T>(g.skind, w, beta, off + T(t));
        }
      }
      if constexpr (kChecked) {  // the whole window inside the tile
        bool okw = true;
        for (int j = 0; j < D; ++j) okw = okw && in_range(g.errw, kSiteSpreadTile, l[j], W3[j] - w + 1);
        if (!okw) continue;
      }
      T cv[CN];
#pragma unroll
      for (int c = 0; c < CN; ++c) cv[c] = str[int64_t(s0 + c0 + c) * n + p] * s_scale[c];
      if constexpr (W > 0) {
        if (D == 1) {
#pragma unroll
          for (int t0 = 0; t0 < W; ++t0) {
            const int idx = l[0] + t0;
#pragma unroll
            for (int c = 0; c < CN; ++c) TileAcc<T>::add(&sm[c * cells + idx], cv[c] * wt[0][t0]);
          }
        } else if (D == 2) {
#pragma unroll
          for (int t0 = 0; t0 < W; ++t0) {
            const int row = (l[0] + t0) * W3[1] + l[1];
            const T w0 = wt[0][t0];
#pragma unroll
            for (int t1 = 0; t1 < W; ++t1) {
              const T v = w0 * wt[D - 1][t1];
#pragma unroll
              for (int c = 0; c < CN; ++c) TileAcc<T>::add(&sm[c * cells + row + t1], cv[c] * v);
            }
          }
        } else {
#pragma unroll 1
          for (int t0 = 0; t0 < W; ++t0)
#pragma unroll
            for (int t1 = 0; t1 < W; ++t1) {
              const int row = ((l[0] + t0) * W3[1] + (l[1] + t1)) * W3[2] + l[2];
              const T v01 = wt[0][t0] * wt[1 % D][t1];
#pragma unroll
              for (int t2 = 0; t2 < W; ++t2) {
                const T v = v01 * wt[D - 1][t2];
#pragma unroll
                for (int c = 0; c < CN; ++c) TileAcc<T>::add(&sm[c * cells + row + t2], cv[c] * v);
              }
            }
        }
      } else {
        // runtime width: plain loops over the window
        int ncw = 1;
        for (int j = 0; j < D; ++j) ncw *= w;
#pragma unroll 1
        for (int cidx = 0; cidx < ncw; ++cidx) {
          int rem = cidx, lidx = 0, mult = 1;
          T v = T(1);
          for (int j = D - 1; j >= 0; --j) {
            const int t = rem % w;
            rem /= w;
            v *= wt[j][t];
            lidx += (l[j] + t) * mult;
            mult *= W3[j];
          }
#pragma unroll 1
          for (int c = 0; c < cn; ++c) TileAcc<T>::add(&sm[c * cells + lidx], cv[c] * v);
        }
      }
    }
    __syncthreads();
    // flush the tile (periodic wrap) into the fine grid
    for (int idx = threadIdx.x; idx < cells; idx += blockDim.x) {
      int rem = idx;
      int lj[3];
      for (int j = 2; j >= 0; --j) {
        lj[j] = rem % W3[j];
        rem /= W3[j];
      }
      int64_t gidx = 0;
      for (int j = 0; j < 3; ++j) {
        int64_t m = 0;
        if (j < D) m = wrap_idx(o[j] + lj[j], g.nf[j]);
        gidx = gidx * g.nf[j] + m;
      }
      if (!in_range(g.errw, kSiteSpreadFlush, gidx, fine_cells)) continue;
      for (int c = 0; c < cn; ++c) {
        const A a = sm[c * cells + idx];
        if (a != A(0)) atomicAdd(&fine[int64_t(s0 + c0 + c) * fine_cells + gidx], T(a) * s_inv[c]);
      }
    }
    __syncthreads();
  }
}

// Run-aggregated spreading (1-D and 2-D, fixed width).  Same sub-problem,
// tile and flush as spread_kernel, but warps take groups of 32 consecutive
// sorted samples: each lane stages one sample of the group (window origin in
// the tile, the 1-D kernel values, the scaled strengths) in shared memory,
// then the warp walks the group's samples in order with its lanes over the
// window cells.  A lane keeps the running sums of its cells for the current
// window in registers and adds them to the tile only when the window changes;
// the sort puts samples that share a window next to each other, so the
// shared-memory atomics drop from one per sample, cell and strength to one
// per run of samples, cell and strength.
template <typename T, int D, int W, int CN>
__global__ void __launch_bounds__(kSpreadThreads)
spread_run_kernel(GeoDev g, int64_t n, const T* __restrict__ xs, const T* __restrict__ str,
                  int s0, const uint32_t* __restrict__ sub_bin,
                  const uint32_t* __restrict__ sub_first, const uint32_t* __restrict__ bin_start,
                  const uint32_t* __restrict__ sub_total, T* __restrict__ fine) {
  static_assert(D <= 2 && W > 0, "run spreading serves 1-D and 2-D with a fixed width");
  constexpr int NC = D == 1 ? W : W * W;      // window cells
  constexpr int CS = (NC + 31) / 32;          // cell slots per lane
  constexpr int PS = D * W + 1;               // staged kernel values per sample (odd stride)
  constexpr int NWARP = kSpreadThreads / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using A = typename TileAcc<T>::type;
  __shared__ T s_scale[kMaxChunk2], s_inv[kMaxChunk2];
  __shared__ T s_red[NWARP][kMaxChunk2];
  A* sm = reinterpret_cast<A*>(smem_raw);
  const uint32_t k = blockIdx.x;
  if (k >= *sub_total) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t b = sub_bin[k];
  const uint32_t first = sub_first[k];
  const uint32_t last = min(first + uint32_t(kSubMax), bin_start[b + 1]);
  int64_t bj[2] = {0, 0};
  {
    int64_t rem = b;
    for (int j = D - 1; j >= 0; --j) {
      bj[j] = rem % g.nbins[j];
      rem /= g.nbins[j];
    }
  }
  int64_t o[2] = {0, 0};
  int W3[2] = {1, 1};
  for (int j = 0; j < D; ++j) {
    o[j] = bj[j] * g.tile[j] - g.pad;
    W3[j] = int(g.tile[j]) + 2 * g.pad;
  }
  const int cells = W3[0] * W3[1];
  // per-warp staging rows after the tile: strengths [32][CN], kernel values
  // [32][PS], window origins [32]
  const size_t tile_bytes = (size_t(CN) * cells * sizeof(A) + 15) / 16 * 16;
  T* str_rows = reinterpret_cast<T*>(smem_raw + tile_bytes) + warp * 32 * CN;
  T* phi_rows = reinterpret_cast<T*>(smem_raw + tile_bytes) + NWARP * 32 * CN + warp * 32 * PS;
  int* org_row = reinterpret_cast<int*>(reinterpret_cast<T*>(smem_raw + tile_bytes) +
                                        NWARP * 32 * (CN + PS)) + warp * 32;
  const T beta = T(g.beta);
  const T halfw = T(0.5) * T(W);
  const int64_t fine_cells = g.nf[0] * g.nf[1] * g.nf[2];
  for (int idx = threadIdx.x; idx < CN * cells; idx += blockDim.x) sm[idx] = A(0);
  if (sizeof(A) == 4) {
    // fixed-point scale per strength: 2^30 / sum |c| over this sub-problem
    T part[CN];
#pragma unroll
    for (int c = 0; c < CN; ++c) part[c] = T(0);
    for (uint32_t p = first + threadIdx.x; p < last; p += blockDim.x)
#pragma unroll
      for (int c = 0; c < CN; ++c) part[c] += fabs(str[int64_t(s0 + c) * n + p]);
#pragma unroll
    for (int c = 0; c < CN; ++c) {
      const T v = warp_sum_t<T>(part[c]);
      if (lane == 0) s_red[warp][c] = v;
    }
    __syncthreads();
    if (threadIdx.x < CN) {
      T tot = T(0);
      for (int wv = 0; wv < NWARP; ++wv) tot += s_red[wv][threadIdx.x];
      s_scale[threadIdx.x] = tot > T(0) ? T(1073741824.0) / tot : T(0);
      s_inv[threadIdx.x] = tot > T(0) ? tot / T(1073741824.0) : T(0);
    }
  } else if (threadIdx.x < CN) {
    s_scale[threadIdx.x] = T(1);
    s_inv[threadIdx.x] = T(1);
  }
  __syncthreads();
  // this lane's window cells: tile offset relative to the window origin
  int rel[CS];
  bool act[CS];
#pragma unroll
  for (int a = 0; a < CS; ++a) {
    const int ci = lane + 32 * a;
    act[a] = ci < NC;
    const int t0 = D == 2 ? ci / W : ci, t1 = D == 2 ? ci % W : 0;
    rel[a] = D == 2 ? t0 * W3[1] + t1 : t0;
  }
  const int ngr = int((last - first + 31) / 32);
  for (int gi = warp; gi < ngr; gi += NWARP) {
    const int64_t g0 = int64_t(first) + int64_t(gi) * 32;
    const int cnt = int(min(int64_t(32), int64_t(last) - g0));
    if (lane < cnt) {
      const int64_t p = g0 + lane;
      int org = 0;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const T u = mul_rn(xs[int64_t(j) * n + p], inv_h_of<T>(g, j));
        const T f0 = ceil(u - halfw);
        const int l = int(int64_t(f0) - o[j]);
        org = j == 0 ? l : org * W3[1] + l;
        const T off = f0 - u;
#pragma unroll
        for (int t = 0; t < W; ++t) phi_rows[lane * PS + j * W + t] = phi<T>(g.skind, W, beta, off + T(t));
      }
      org_row[lane] = org;
#pragma unroll
      for (int c = 0; c < CN; ++c) str_rows[lane * CN + c] = str[int64_t(s0 + c) * n + p] * s_scale[c];
    }
    __syncwarp();
    T acc[CS][CN];
#pragma unroll
    for (int a = 0; a < CS; ++a)
#pragma unroll
      for (int c = 0; c < CN; ++c) acc[a][c] = T(0);
    int cur = org_row[0];
    // two samples per iteration in flight (measured: 5 % off the spreading)
#pragma unroll 2
    for (int j = 0; j < cnt; ++j) {
      const int org = org_row[j];
      if (org != cur) {
#pragma unroll
        for (int a = 0; a < CS; ++a)
          if (act[a] && in_range(g.errw, kSiteSpreadTile, cur + rel[a], cells))
#pragma unroll
            for (int c = 0; c < CN; ++c) {
              TileAcc<T>::add(&sm[c * cells + cur + rel[a]], acc[a][c]);
              acc[a][c] = T(0);
            }
        cur = org;
      }
      const T* ph = phi_rows + j * PS;
      T cv[CN];
#pragma unroll
      for (int c = 0; c < CN; ++c) cv[c] = str_rows[j * CN + c];
#pragma unroll
      for (int a = 0; a < CS; ++a) {
        const int ci = lane + 32 * a;
        const int t0 = D == 2 ? ci / W : ci, t1 = D == 2 ? ci % W : 0;
        T wa = T(0);
        if (act[a]) wa = D == 2 ? ph[t0] * ph[W + t1] : ph[t0];
        if constexpr (sizeof(T) == 4 && CN % 2 == 0) {
          // two strengths per packed FP32 FMA
          const float2 w2 = make_float2(wa, wa);
#pragma unroll
          for (int c = 0; c < CN; c += 2) {
            const float2 r = __ffma2_rn(w2, make_float2(cv[c], cv[c + 1]),
                                        make_float2(acc[a][c], acc[a][c + 1]));
            acc[a][c] = r.x;
            acc[a][c + 1] = r.y;
          }
        } else {
#pragma unroll
          for (int c = 0; c < CN; ++c) acc[a][c] += wa * cv[c];
        }
      }
    }
#pragma unroll
    for (int a = 0; a < CS; ++a)
      if (act[a] && in_range(g.errw, kSiteSpreadTile, cur + rel[a], cells))
#pragma unroll
        for (int c = 0; c < CN; ++c) TileAcc<T>::add(&sm[c * cells + cur + rel[a]], acc[a][c]);
    __syncwarp();  // staging rows are rewritten by the next group
  }
  __syncthreads();
  // flush the tile (periodic wrap) into the fine grid
  for (int idx = threadIdx.x; idx < cells; idx += blockDim.x) {
    const int l0 = D == 2 ? idx / W3[1] : idx, l1 = D == 2 ? idx % W3[1] : 0;
    int64_t gidx = wrap_idx(o[0] + l0, g.nf[0]);
    if (D == 2) gidx = gidx * g.nf[1] + wrap_idx(o[1] + l1, g.nf[1]);
    if (!in_range(g.errw, kSiteSpreadFlush, gidx, fine_cells)) continue;
    for (int c = 0; c < CN; ++c) {
      const A av = sm[c * cells + idx];
      if (av != A(0)) atomicAdd(&fine[int64_t(s0 + c) * fine_cells + gidx], T(av) * s_inv[c]);
    }
  }
}

template <typename T, int D, int W, int CN>
cudaError_t launch_spread_cn(fkreg_plan_s* P, int s0, cudaStream_t st) {
  const GeoDev& g = P->geo;
  int cells = 1;
  for (int j = 0; j < D; ++j) cells *= int(g.tile[j]) + 2 * g.pad;
  const size_t smem = size_t(cells) * sizeof(typename TileAcc<T>::type) * CN;
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(spread_kernel<T, D, W, CN>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  const unsigned grid = unsigned(P->nsub_max);
  const uint32_t* sub_total = wsp<uint32_t>(P, P->r_substart) + P->nbins_total;
  spread_kernel<T, D, W, CN><<<grid, kSpreadThreads, smem, st>>>(
      g, P->n, wsp<T>(P, P->r_xs), wsp<T>(P, P->r_str), s0, CN, CN,
      wsp<uint32_t>(P, P->r_subbin), wsp<uint32_t>(P, P->r_subfirst),
      wsp<uint32_t>(P, P->r_binstart), sub_total, wsp<T>(P, P->r_fine));
  P->launches += 1;
  return cudaGetLastError();
}

// Shared memory of one run-kernel block: the tile for CN strengths plus the
// per-warp staging rows.
template <typename T, int D, int W, int CN>
size_t spread_run_smem(const GeoDev& g) {
  using A = typename TileAcc<T>::type;
  int cells = 1;
  for (int j = 0; j < D; ++j) cells *= int(g.tile[j]) + 2 * g.pad;
  const size_t tile_bytes = (size_t(CN) * cells * sizeof(A) + 15) / 16 * 16;
  return tile_bytes + size_t(kSpreadThreads) * (CN + D * W + 1) * sizeof(T) +
         size_t(kSpreadThreads) * sizeof(int);
}

template <typename T, int D, int W, int CN>
cudaError_t launch_spread_run(fkreg_plan_s* P, int s0, cudaStream_t st) {
  const GeoDev& g = P->geo;
  const size_t smem = spread_run_smem<T, D, W, CN>(g);
  if (smem > 220 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(spread_run_kernel<T, D, W, CN>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  const unsigned grid = unsigned(P->nsub_max);
  const uint32_t* sub_total = wsp<uint32_t>(P, P->r_substart) + P->nbins_total;
  spread_run_kernel<T, D, W, CN><<<grid, kSpreadThreads, smem, st>>>(
      g, P->n, wsp<T>(P, P->r_xs), wsp<T>(P, P->r_str), s0, wsp<uint32_t>(P, P->r_subbin),
      wsp<uint32_t>(P, P->r_subfirst), wsp<uint32_t>(P, P->r_binstart), sub_total,
      wsp<T>(P, P->r_fine));
  P->launches += 1;
  return cudaGetLastError();
}

// All strengths through the run kernel in launches of the largest chunk
// sizes that fit shared memory (FP32: 16, 12, 8, 4, 2, 1; FP64: 4, 2, 1).
template <typename T, int D, int W>
cudaError_t launch_spread_runs(fkreg_plan_s* P, int s0, int scount, cudaStream_t st) {
  int done = 0;
  while (done < scount) {
    const int rem = scount - done;
    cudaError_t e = cudaErrorInvalidConfiguration;
    int used = 0;
    if constexpr (sizeof(T) == 4) {
      if (rem >= 16 && spread_run_smem<T, D, W, 16>(P->geo) <= 220 * 1024) {
        e = launch_spread_run<T, D, W, 16>(P, s0 + done, st);
        used = 16;
      } else if (rem >= 12 && spread_run_smem<T, D, W, 12>(P->geo) <= 220 * 1024) {
        e = launch_spread_run<T, D, W, 12>(P, s0 + done, st);
        used = 12;
      } else if (rem >= 8 && spread_run_smem<T, D, W, 8>(P->geo) <= 220 * 1024) {
        e = launch_spread_run<T, D, W, 8>(P, s0 + done, st);
        used = 8;
      }
    }
    if (!used) {
      if (rem >= 4 && spread_run_smem<T, D, W, 4>(P->geo) <= 220 * 1024) {
        e = launch_spread_run<T, D, W, 4>(P, s0 + done, st);
        used = 4;
      } else if (rem >= 2 && spread_run_smem<T, D, W, 2>(P->geo) <= 220 * 1024) {
        e = launch_spread_run<T, D, W, 2>(P, s0 + done, st);
        used = 2;
      } else {
        e = launch_spread_run<T, D, W, 1>(P, s0 + done, st);
        used = 1;
      }
    }
    if (e != cudaSuccess) return e;
    done += used;
  }
  return cudaSuccess;
}

// Strengths go in launches of 8, 4, 2 or 1 (compile-time chunk sizes, as
// many as the shared-memory budget allows per launch); 1-D / 2-D plans of a
// compile-time width use the run kernel instead (launch_spread_runs).
template <typename T, int D, int W>
cudaError_t launch_spread_w(fkreg_plan_s* P, int s0, int scount, cudaStream_t st) {
  const GeoDev& g = P->geo;
  if constexpr (W > 0 && D <= 2) {
    if (spread_run_smem<T, D, W, 1>(g) <= 220 * 1024) return launch_spread_runs<T, D, W>(P, s0, scount, st);
  }
  int cells = 1;
  for (int j = 0; j < D; ++j) cells *= int(g.tile[j]) + 2 * g.pad;
  const size_t per = size_t(cells) * sizeof(typename TileAcc<T>::type);
  const int cap = int(std::max<size_t>(1, std::min<size_t>((100 * 1024) / per, kMaxChunk)));
  int done = 0;
  while (done < scount) {
    const int rem = std::min(scount - done, cap);
    cudaError_t e;
    int used;
    if (rem >= 8) {
      e = launch_spread_cn<T, D, W, 8>(P, s0 + done, st);
      used = 8;
    } else if (rem >= 4) {
      e = launch_spread_cn<T, D, W, 4>(P, s0 + done, st);
      used = 4;
    } else if (rem >= 2) {
      e = launch_spread_cn<T, D, W, 2>(P, s0 + done, st);
      used = 2;
    } else {
      e = launch_spread_cn<T, D, W, 1>(P, s0 + done, st);
      used = 1;
    }
    if (e != cudaSuccess) return e;
    done += used;
  }
  return cudaSuccess;
}

template <typename T, int D>
cudaError_t launch_spread(fkreg_plan_s* P, int s0, int scount, cudaStream_t st) {
  const int w = P->geo.w;
  if (w == 7) return launch_spread_w<T, D, 7>(P, s0, scount, st);
  if constexpr (sizeof(T) == 8 && D < 3) {
    if (w == 10) return launch_spread_w<T, D, 10>(P, s0, scount, st);
    if (w == 13) return launch_spread_w<T, D, 13>(P, s0, scount, st);
  }
  if (w > kMaxWRun) return cudaErrorInvalidValue;
  return launch_spread_w<T, D, 0>(P, s0, scount, st);
}

template <typename T>
cudaError_t launch_spread_d(fkreg_plan_s* P, int s0, int scount, cudaStream_t st) {
  switch (P->d) {
    case 1: return launch_spread<T, 1>(P, s0, scount, st);
    case 2: return launch_spread<T, 2>(P, s0, scount, st);
    default: return launch_spread<T, 3>(P, s0, scount, st);
  }
}

// ---- strengths in sorted order --------------------------------------------
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Gaussian probes in Box-Muller pairs from counter-based SplitMix64 words:
// word k >= 1 of the stream seeded with `seed` is splitmix64(seed + (k-1) gamma);
// pair j of ORIGINAL sample i takes words 2c+1 and 2c+2, c = (j << 40) | i, as
// the uniforms u1 in (0, 1] and u2 in [0, 1) (53-bit in FP64, the words' top
// 24 bits in FP32) and gives r cos(2 pi u2), r sin(2 pi u2), r = sqrt(-2 ln u1),
// evaluated in the plan precision.
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ULL;

__device__ __forceinline__ void probe_words(uint64_t seed, int j, uint32_t i, uint64_t& a,
                                            uint64_t& b) {
  const uint64_t c = (uint64_t(j) << 40) | uint64_t(i);
  const uint64_t base = seed + (2 * c) * kGamma;
  a = splitmix64(base);
  b = splitmix64(base + kGamma);
}

template <typename T>
__device__ __forceinline__ void probe_pair(uint64_t seed, int j, uint32_t i, T& z0, T& z1);
template <>
__device__ __forceinline__ void probe_pair<double>(uint64_t seed, int j, uint32_t i, double& z0,
                                                   double& z1) {
  uint64_t a, b;
  probe_words(seed, j, i, a, b);
  const double u1 = (double(a >> 11) + 1.0) * 0x1.0p-53;
  const double u2 = double(b >> 11) * 0x1.0p-53;
  const double r = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  z0 = r * cs;
  z1 = r * sn;
}
template <>
__device__ __forceinline__ void probe_pair<float>(uint64_t seed, int j, uint32_t i, float& z0,
                                                  float& z1) {
  uint64_t a, b;
  probe_words(seed, j, i, a, b);
  const float u1 = float(uint32_t(a >> 40) + 1u) * 0x1.0p-24f;
  const float u2 = float(uint32_t(b >> 40)) * 0x1.0p-24f;
  const float r = sqrtf(-2.0f * logf(u1));
  float sn, cs;
  sincospif(2.0f * u2, &sn, &cs);
  z0 = r * cs;
  z1 = r * sn;
}

template <typename T>
__global__ void kernel_values_kernel(int kind, int w, T beta, int64_t n, const T* __restrict__ z,
                                     T* __restrict__ out) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) out[i] = phi<T>(kind, w, beta, z[i]);
}

template <typename T>
__global__ void gather_strengths_kernel(int64_t n, const uint32_t* __restrict__ perm,
                                        const T* __restrict__ y, int n_rhs, int y_complex,
                                        int with_density, int n_probes, uint64_t seed,
                                        const T* __restrict__ probes, T* __restrict__ str,
                                        int first) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const uint32_t i = perm[s];
  int k = first;
  if (with_density) str[int64_t(k++) * n + s] = T(1);
  for (int r = 0; r < n_rhs; ++r) {
    if (y_complex) {
      str[int64_t(k++) * n + s] = y[(int64_t(r) * n + i) * 2 + 0];
      str[int64_t(k++) * n + s] = y[(int64_t(r) * n + i) * 2 + 1];
    } else {
      str[int64_t(k++) * n + s] = y[int64_t(r) * n + i];
    }
  }
  if (probes) {
    for (int p = 0; p < n_probes; ++p) str[int64_t(k++) * n + s] = probes[int64_t(p) * n + i];
  } else {
    for (int p = 0; p < n_probes; p += 2) {
      T z0, z1;
      probe_pair<T>(seed, p >> 1, i, z0, z1);
      str[int64_t(k++) * n + s] = z0;
      if (p + 1 < n_probes) str[int64_t(k++) * n + s] = z1;
    }
  }
}

// r_i = |y_i - mhat_b(x_i)|^2 for every response (eq. 23), sorted order.
template <typename T>
__global__ void residual_strengths_kernel(int64_t n, const uint32_t* __restrict__ perm,
                                          const T* __restrict__ y, const T* __restrict__ mh,
                                          int n_rhs, int y_complex, int b, T* __restrict__ str,
                                          int first) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const uint32_t i = perm[s];
  for (int r = 0; r < n_rhs; ++r) {
    T v;
    if (y_complex) {
      const int64_t yi = (int64_t(r) * n + i) * 2;
      const int64_t mi = ((int64_t(b) * n_rhs + r) * n + i) * 2;
      const T dr = y[yi] - mh[mi], di = y[yi + 1] - mh[mi + 1];
      v = dr * dr + di * di;
    } else {
      const T dr = y[int64_t(r) * n + i] - mh[(int64_t(b) * n_rhs + r) * n + i];
      v = dr * dr;
    }
    str[int64_t(first + r) * n + s] = v;
  }
}

// l_i = log(|y_i - mhat_b(x_i)|^2 + 1/N) for every real response (eq. 25),
// sorted order.
template <typename T>
__global__ void logres_strengths_kernel(int64_t n, const uint32_t* __restrict__ perm,
                                        const T* __restrict__ y, const T* __restrict__ mh,
                                        int n_rhs, int b, T* __restrict__ str, int first) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const uint32_t i = perm[s];
  const T inv_n = T(1) / T(n);
  for (int r = 0; r < n_rhs; ++r) {
    const T dr = y[int64_t(r) * n + i] - mh[(int64_t(b) * n_rhs + r) * n + i];
    str[int64_t(first + r) * n + s] = log(dr * dr + inv_n);
  }
}

}  // namespace

const uint32_t* perm_ptr(fkreg_plan_s* P) {
  return P->perm_in_vals1 ? wsp<uint32_t>(P, P->r_vals1) : wsp<uint32_t>(P, P->r_vals0);
}

cudaError_t run_spread(fkreg_plan_s* P, int s0, int scount, cudaStream_t st) {
  const int64_t fine_cells = P->geo.nf[0] * P->geo.nf[1] * P->geo.nf[2];
  cudaError_t e = cudaMemsetAsync(P->ws + P->r_fine.off + size_t(s0) * fine_cells * P->tsize, 0,
                                  size_t(scount) * fine_cells * P->tsize, st);
  if (e != cudaSuccess || P->n == 0 || scount == 0) return e;
  return P->prec == FKREG_F32 ? launch_spread_d<float>(P, s0, scount, st)
                              : launch_spread_d<double>(P, s0, scount, st);
}

cudaError_t run_gather_strengths(fkreg_plan_s* P, const void* y, int first_str, int n_probes,
                                 uint64_t seed, const void* probes, int with_density,
                                 cudaStream_t st) {
  if (P->n == 0) return cudaSuccess;
  const unsigned blocks = unsigned((P->n + 255) / 256);
  const uint32_t* perm = perm_ptr(P);
  if (P->prec == FKREG_F32)
    gather_strengths_kernel<float><<<blocks, 256, 0, st>>>(
        P->n, perm, static_cast<const float*>(y), P->nrhs, P->o.y_complex, with_density, n_probes,
        seed, static_cast<const float*>(probes), wsp<float>(P, P->r_str), first_str);
  else
    gather_strengths_kernel<double><<<blocks, 256, 0, st>>>(
        P->n, perm, static_cast<const double*>(y), P->nrhs, P->o.y_complex, with_density, n_probes,
        seed, static_cast<const double*>(probes), wsp<double>(P, P->r_str), first_str);
  P->launches += 1;
  return cudaGetLastError();
}

cudaError_t run_residual_strengths(fkreg_plan_s* P, const void* y, const void* mhat_at_x, int b,
                                   int first_str, cudaStream_t st) {
  if (P->n == 0) return cudaSuccess;
  const unsigned blocks = unsigned((P->n + 255) / 256);
  const uint32_t* perm = perm_ptr(P);
  if (P->prec == FKREG_F32)
    residual_strengths_kernel<float><<<blocks, 256, 0, st>>>(
        P->n, perm, static_cast<const float*>(y), static_cast<const float*>(mhat_at_x), P->nrhs,
        P->o.y_complex, b, wsp<float>(P, P->r_str), first_str);
  else
    residual_strengths_kernel<double><<<blocks, 256, 0, st>>>(
        P->n, perm, static_cast<const double*>(y), static_cast<const double*>(mhat_at_x), P->nrhs,
        P->o.y_complex, b, wsp<double>(P, P->r_str), first_str);
  P->launches += 1;
  return cudaGetLastError();
}

}  // namespace fk

namespace fk {

cudaError_t run_logres_strengths(fkreg_plan_s* P, const void* y, const void* mhat_at_x, int b,
                                 int first_str, cudaStream_t st) {
  if (P->n == 0) return cudaSuccess;
  const unsigned blocks = unsigned((P->n + 255) / 256);
  const uint32_t* perm = perm_ptr(P);
  if (P->prec == FKREG_F32)
    logres_strengths_kernel<float><<<blocks, 256, 0, st>>>(
        P->n, perm, static_cast<const float*>(y), static_cast<const float*>(mhat_at_x), P->nrhs,
        b, wsp<float>(P, P->r_str), first_str);
  else
    logres_strengths_kernel<double><<<blocks, 256, 0, st>>>(
        P->n, perm, static_cast<const double*>(y), static_cast<const double*>(mhat_at_x), P->nrhs,
        b, wsp<double>(P, P->r_str), first_str);
  P->launches += 1;
  return cudaGetLastError();
}

}  // namespace fk

extern "C" fkreg_status fkreg_spread_kernel_values(int kind, int w, double beta, int precision,
                                                   int64_t n, const void* z_dev, void* out_dev,
                                                   void* stream) {
  using namespace fk;
  if (kind != FKREG_SPREAD_ES && kind != FKREG_SPREAD_GAUSS) return FKREG_ERR_INVALID_ARG;
  if (precision != FKREG_F32 && precision != FKREG_F64) return FKREG_ERR_INVALID_ARG;
  if (w < 2 || w > 32 || n < 0 || (n > 0 && (!z_dev || !out_dev))) return FKREG_ERR_INVALID_ARG;
  if (n == 0) return FKREG_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const unsigned blocks = unsigned((n + 255) / 256);
  if (precision == FKREG_F32)
    kernel_values_kernel<float><<<blocks, 256, 0, s>>>(kind, w, float(beta), n,
                                                       static_cast<const float*>(z_dev),
                                                       static_cast<float*>(out_dev));
  else
    kernel_values_kernel<double><<<blocks, 256, 0, s>>>(kind, w, beta, n,
                                                        static_cast<const double*>(z_dev),
                                                        static_cast<double*>(out_dev));
  return cudaGetLastError() == cudaSuccess ? FKREG_OK : FKREG_ERR_CUDA;
}
