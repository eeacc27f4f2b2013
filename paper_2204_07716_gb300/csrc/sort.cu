// Bin assignment and stable counting sort of the samples.
//
// Every sample gets the spreading bin that holds its fine-grid cell:
//   u_j   = fl(fl(x_j - lo_j) * inv_h_j)      (round-to-nearest, no FMA)
//   c_j   = min(floor(u_j), nf_j - 1)
//   bin   = row-major index of (c_j / tile_j)
// and, inside the bin, the centre cell of its spreading window
//   o_j   = ceil(fl(u_j - w/2)),   e_j = o_j + floor(w/2)   (c_j or c_j + 1)
//   local = serpentine index of c_j = clamp(e_j - b_j tile_j, 0, tile_j) over
//           (tile_j + 1) values per axis: local = local (tile_j + 1) + c_j, with
//           c_j replaced by tile_j - c_j when the local of the axes before is
//           odd
// The key (bin << kbits) | local orders the samples by bin and, inside a bin,
// by the window they touch, so consecutive sorted samples share windows.
// The samples are ordered by key with a least-significant-digit radix sort
// (8-bit digits).  Each pass is a stable counting sort: per-tile digit
// histograms, one exclusive scan over (digit, tile), and a scatter that ranks
// equal digits inside a tile in index order with warp match masks.  The
// resulting permutation is therefore unique: key first, original index second.
// The paper bins the samples onto the grid too (Sec. 1.1, O(N) gridding); the
// counting sort is this implementation's own device-side organisation of it.
#include <cuda_runtime.h>

#include <mutex>

#include "checked.cuh"
#include "internal.h"

namespace fk {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortTile = kSortTileKeys;               // keys per tile
constexpr int kSortRounds = kSortTile / kSortThreads;  // keys per thread per tile
constexpr int kScanThreads = 256;
constexpr int kScanChunk = 1024;                     // elements per scan block

__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

template <typename T>
__device__ __forceinline__ T inv_h_of(const GeoDev& g, int j);
template <>
__device__ __forceinline__ float inv_h_of<float>(const GeoDev& g, int j) { return g.inv_h_f[j]; }
template <>
__device__ __forceinline__ double inv_h_of<double>(const GeoDev& g, int j) { return g.inv_h[j]; }

template <typename T>
__global__ void bin_keys_kernel(GeoDev g, int64_t n, const T* __restrict__ x,
                                uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                uint32_t* __restrict__ counts, int* __restrict__ errw) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t bin = 0, local = 0;
  bool bad = false;
  const T halfw = T(0.5) * T(g.w);
  for (int j = 0; j < g.d; ++j) {
    T xv = x[i * g.d + j];
    const T lo = T(g.lo[j]), hi = T(g.hi[j]);
    if (!(xv >= lo && xv <= hi)) {
      bad = true;
      xv = lo;
    }
    const T u = mul_rn(sub_rn(xv, lo), inv_h_of<T>(g, j));
    int64_t c = int64_t(floor(u));
    if (c < 0) c = 0;
    if (c > g.nf[j] - 1) c = g.nf[j] - 1;
    const int64_t b = c / g.tile[j];
    int64_t e = int64_t(ceil(sub_rn(u, halfw))) + g.w / 2 - b * g.tile[j];
    e = e < 0 ? 0 : (e > g.tile[j] ? g.tile[j] : e);
    bin = bin * uint32_t(g.nbins[j]) + uint32_t(b);
    // serpentine order: an axis runs backwards when the index of the axes
    // before it is odd, so consecutive keys are neighbouring windows
    local = local * uint32_t(g.tile[j] + 1) +
            uint32_t((local & 1u) ? g.tile[j] - e : e);
  }
  if (bad) atomicOr(errw, 1);
  keys[i] = g.kbits ? (bin << g.kbits) | local : bin;
  vals[i] = uint32_t(i);
  if (counts) atomicAdd(&counts[bin], 1u);
}

// The key of sample i (see the header of this file); `bad` is set when the
// sample lies outside the box (it is then keyed as if at the lower corner).
template <typename T>
__device__ __forceinline__ uint32_t sample_key(const GeoDev& g, const T* __restrict__ x, int64_t i,
                                               bool& bad, uint32_t& bin) {
  const T halfw = T(0.5) * T(g.w);
  uint32_t local = 0;
  bin = 0;
  for (int j = 0; j < g.d; ++j) {
    T xv = x[i * g.d + j];
    const T lo = T(g.lo[j]), hi = T(g.hi[j]);
    if (!(xv >= lo && xv <= hi)) {
      bad = true;
      xv = lo;
    }
    const T u = mul_rn(sub_rn(xv, lo), inv_h_of<T>(g, j));
    // 32-bit integer arithmetic: cells, tiles and bins are below 2^31
    const int nfj = int(g.nf[j]), tj = int(g.tile[j]);
    int c = int(floor(u));
    if (c < 0) c = 0;
    if (c > nfj - 1) c = nfj - 1;
    const int b = c / tj;
    int e = int(ceil(sub_rn(u, halfw))) + g.w / 2 - b * tj;
    e = e < 0 ? 0 : (e > tj ? tj : e);
    bin = bin * uint32_t(g.nbins[j]) + uint32_t(b);
    local = local * uint32_t(tj + 1) + uint32_t((local & 1u) ? tj - e : e);
  }
  return g.kbits ? (bin << g.kbits) | local : bin;
}

// ---- fused sort (plans with at most kFusedMaxBins bins) --------------------
// Five launches for two passes: keys with the bin counts and the first
// pass's tile histograms; per pass one scan of the tile histograms and one
// scatter.  A scatter that is not the last counts the next pass's digits of
// the keys it writes, by destination tile (global atomics) and in total
// (shared, then one atomic per digit and block); the last scatter writes the
// permutation and the sorted, shifted coordinates, not the keys.  The first
// scan's extra block turns the bin counts into bin starts and spreading
// sub-problems.
constexpr int64_t kFusedMaxBins = 8192;
constexpr int kKeysThreads = 512;
constexpr int kDigitScanWarps = 8;

template <typename T, int B>
__global__ void __launch_bounds__(kKeysThreads)
keys_tiles_kernel(GeoDev g, int64_t n, int64_t nbins, int64_t ntiles, const T* __restrict__ x,
                  uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                  uint32_t* __restrict__ counts, uint32_t* __restrict__ hist,
                  uint32_t* __restrict__ dtot, int* __restrict__ errw) {
  constexpr uint32_t R = 1u << B;
  extern __shared__ uint32_t ksm[];
  uint32_t* hb = ksm;          // [nbins] bin counts of this block
  uint32_t* hd = ksm + nbins;  // [R] digit counts of the current tile
  for (int64_t b = threadIdx.x; b < nbins; b += blockDim.x) hb[b] = 0;
  bool bad = false;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    for (uint32_t d = threadIdx.x; d < R; d += blockDim.x) hd[d] = 0;
    __syncthreads();
    const int64_t base = t * kSortTile;
    for (int k = threadIdx.x; k < kSortTile; k += blockDim.x) {
      const int64_t i = base + k;
      if (i >= n) break;
      uint32_t bin;
      const uint32_t key = sample_key<T>(g, x, i, bad, bin);
      keys[i] = key;
      vals[i] = uint32_t(i);
      atomicAdd(&hb[bin], 1u);
      atomicAdd(&hd[key & (R - 1u)], 1u);
    }
    __syncthreads();
    for (uint32_t d = threadIdx.x; d < R; d += blockDim.x) {
      const uint32_t c = hd[d];
      hist[int64_t(d) * ntiles + t] = c;
      if (c) atomicAdd(&dtot[d], c);
    }
    __syncthreads();
  }
  if (bad) atomicOr(errw, 1);
  __syncthreads();
  for (int64_t b = threadIdx.x; b < nbins; b += blockDim.x)
    if (hb[b]) atomicAdd(&counts[b], hb[b]);
}

// Bin starts and spreading sub-problems (at most kSubMax samples each) from
// the bin counts, by one block of kDigitScanWarps warps: each thread owns a
// contiguous chunk of bins, the block scans the chunk totals of samples and
// sub-problems, and each thread writes its bins' starts and sub-problems.
struct BinsArgs {
  const uint32_t* counts;
  int64_t nbins;
  uint32_t* bin_start;  // [nbins + 1]
  uint32_t* sub_start;  // [nbins + 1]
  uint32_t* sub_bin;
  uint32_t* sub_first;
};

__device__ void bins_block(const BinsArgs& a) {
  constexpr int NT = kDigitScanWarps * 32;
  __shared__ uint32_t wc[kDigitScanWarps], ws[kDigitScanWarps];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t chunk = (a.nbins + NT - 1) / NT;
  const int64_t b0 = min(a.nbins, int64_t(tid) * chunk), b1 = min(a.nbins, b0 + chunk);
  uint32_t tc = 0, ts = 0;
  for (int64_t b = b0; b < b1; ++b) {
    const uint32_t c = a.counts[b];
    tc += c;
    ts += (c + kSubMax - 1) / kSubMax;
  }
  uint32_t ic = tc, is = ts;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t vc = __shfl_up_sync(0xffffffffu, ic, o);
    const uint32_t vs = __shfl_up_sync(0xffffffffu, is, o);
    if (lane >= o) {
      ic += vc;
      is += vs;
    }
  }
  if (lane == 31) {
    wc[warp] = ic;
    ws[warp] = is;
  }
  __syncthreads();
  uint32_t rc = ic - tc, rs = is - ts, totc = 0, tots = 0;
  for (int w = 0; w < kDigitScanWarps; ++w) {
    if (w < warp) {
      rc += wc[w];
      rs += ws[w];
    }
    totc += wc[w];
    tots += ws[w];
  }
  for (int64_t b = b0; b < b1; ++b) {
    const uint32_t c = a.counts[b], ns = (c + kSubMax - 1) / kSubMax;
    a.bin_start[b] = rc;
    a.sub_start[b] = rs;
    for (uint32_t k = 0; k < ns; ++k) {
      a.sub_bin[rs + k] = uint32_t(b);
      a.sub_first[rs + k] = rc + k * kSubMax;
    }
    rc += c;
    rs += ns;
  }
  if (tid == 0) {
    a.bin_start[a.nbins] = totc;
    a.sub_start[a.nbins] = tots;
  }
}

// hist[d][t] (tile counts of digit d) -> first output position of digit d's
// keys from tile t: the digits' exclusive prefix of the totals dtot plus the
// exclusive prefix over the tiles before t.  One warp per digit; grid
// R / kDigitScanWarps blocks (+1 when bins.counts is set: that block runs
// bins_block).  With hist_next set, the same warps zero the next pass's
// tile histograms and totals, which the scatter of this pass fills.
template <int B>
__global__ void __launch_bounds__(kDigitScanWarps * 32)
digit_scan_kernel(uint32_t* __restrict__ hist, int64_t ntiles, const uint32_t* __restrict__ dtot,
                  uint32_t* __restrict__ hist_next, uint32_t* __restrict__ dtot_next,
                  BinsArgs bins) {
  constexpr int R = 1 << B;
  constexpr int NT = kDigitScanWarps * 32;
  constexpr int DPT = R / NT;
  static_assert(DPT * NT == R, "digits per thread");
  if (bins.counts && blockIdx.x == gridDim.x - 1) {
    bins_block(bins);
    return;
  }
  __shared__ uint32_t base[R];
  __shared__ uint32_t wsum[kDigitScanWarps];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t v[DPT], own = 0;
#pragma unroll
  for (int u = 0; u < DPT; ++u) {
    v[u] = dtot[tid * DPT + u];
    own += v[u];
  }
  uint32_t inc = own;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  uint32_t run = inc - own;
  for (int w = 0; w < warp; ++w) run += wsum[w];
#pragma unroll
  for (int u = 0; u < DPT; ++u) {
    base[tid * DPT + u] = run;
    run += v[u];
  }
  __syncthreads();
  const int d = blockIdx.x * kDigitScanWarps + warp;
  uint32_t carry = base[d];
  uint32_t* row = hist + int64_t(d) * ntiles;
  constexpr int V = 8;  // consecutive tiles per lane and segment
  for (int64_t t0 = 0; t0 < ntiles; t0 += 32 * V) {
    uint32_t c[V], tot = 0;
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const int64_t t = t0 + int64_t(lane) * V + k;
      c[k] = t < ntiles ? row[t] : 0u;
      tot += c[k];
    }
    uint32_t incl = tot;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    uint32_t r = carry + incl - tot;
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const int64_t t = t0 + int64_t(lane) * V + k;
      if (t < ntiles) row[t] = r;
      r += c[k];
    }
    carry += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (hist_next) {
    for (int64_t t = lane; t < ntiles; t += 32) hist_next[int64_t(d) * ntiles + t] = 0;
    if (lane == 0) dtot_next[d] = 0;
  }
}

// ---- exclusive scan of uint32 (three kernels, any length) ----------------
__global__ void scan_block_sums(const uint32_t* __restrict__ in, int64_t n,
                                uint32_t* __restrict__ sums) {
  __shared__ uint32_t red[kScanThreads / 32];
  const int64_t base = int64_t(blockIdx.x) * kScanChunk;
  uint32_t s = 0;
  for (int k = threadIdx.x; k < kScanChunk; k += kScanThreads) {
    int64_t i = base + k;
    if (i < n) s += in[i];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) t += red[w];
    sums[blockIdx.x] = t;
  }
}

// Exclusive scan of `sums` in place by one block, chunk after chunk.
__global__ void scan_sums_single(uint32_t* __restrict__ sums, int64_t nb, uint32_t* total) {
  __shared__ uint32_t buf[1024];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nb; base += 1024) {
    const int64_t i = base + threadIdx.x;
    uint32_t v = (i < nb) ? sums[i] : 0u;
    buf[threadIdx.x] = v;
    __syncthreads();
    // Hillis-Steele inclusive scan
    for (int o = 1; o < 1024; o <<= 1) {
      uint32_t t = (threadIdx.x >= o) ? buf[threadIdx.x - o] : 0u;
      __syncthreads();
      buf[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < nb) sums[i] = carry + buf[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += buf[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

// out[i] = offset(block) + exclusive prefix inside the block; in may alias out.
__global__ void scan_apply(const uint32_t* in, int64_t n, const uint32_t* __restrict__ sums,
                           uint32_t* out) {
  __shared__ uint32_t wsum[kScanThreads / 32];
  const int64_t base = int64_t(blockIdx.x) * kScanChunk;
  constexpr int per = kScanChunk / kScanThreads;  // 4 consecutive elements per thread
  uint32_t v[per];
  uint32_t run = 0;
  for (int k = 0; k < per; ++k) {
    int64_t i = base + threadIdx.x * per + k;
    v[k] = (i < n) ? in[i] : 0u;
    run += v[k];
  }
  // warp inclusive scan of per-thread totals
  uint32_t inc = run;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  uint32_t woff = 0;
  for (int w = 0; w < warp; ++w) woff += wsum[w];
  uint32_t off = sums[blockIdx.x] + woff + inc - run;
  for (int k = 0; k < per; ++k) {
    int64_t i = base + threadIdx.x * per + k;
    if (i < n) out[i] = off;
    off += v[k];
  }
}

// ---- radix sort passes ---------------------------------------------------
// A tile of kSortTile keys is split into one contiguous chunk per warp.  Both
// kernels group equal digits of a 32-key round with match_digit, so one
// lane per group updates a counter: the upsweep adds to the tile histogram
// (shared atomics, warps run concurrently); the downsweep first counts per
// warp, turns the counts into per-warp offsets (warps in chunk order after
// the tile's scanned global base), then re-walks its keys from registers and
// writes each key at offset + rank among the equal digits of lower lanes.
// Order is preserved within a round, across rounds, across warps and across
// tiles, so every pass is stable.
// Lanes of the warp holding the same (B + 1)-bit value (a digit, or 2^B
// for "no key"): one ballot per bit, AND of the agreeing masks.
template <int B>
__device__ __forceinline__ uint32_t match_digit(uint32_t dig) {
  uint32_t m = 0xffffffffu;
#pragma unroll
  for (int b = 0; b <= B; ++b) {
    const uint32_t bit = (dig >> b) & 1u;
    const uint32_t bal = __ballot_sync(0xffffffffu, bit);
    m &= bit ? bal : ~bal;
  }
  return m;
}

// B-bit digits (R = 2^B buckets); hist[digit][tile]
template <int B>
__global__ void __launch_bounds__(kSortThreads)
radix_upsweep(const uint32_t* __restrict__ keys, int64_t n, int shift, int64_t ntiles,
              uint32_t* __restrict__ hist) {
  constexpr uint32_t R = 1u << B;
  __shared__ uint32_t h[R];
  for (uint32_t d = threadIdx.x; d < R; d += kSortThreads) h[d] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t base = int64_t(blockIdx.x) * kSortTile;
  uint32_t dg[kSortRounds];  // every load of the tile in flight before the first use
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t i = base + int64_t(r) * kSortThreads + threadIdx.x;
    dg[r] = i < n ? (keys[i] >> shift) & (R - 1u) : R;
  }
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const uint32_t dig = dg[r];
    const uint32_t peers = match_digit<B>(dig);
    if (dig < R && (__ffs(peers) - 1) == lane) atomicAdd(&h[dig], uint32_t(__popc(peers)));
  }
  __syncthreads();
  for (uint32_t d = threadIdx.x; d < R; d += kSortThreads)
    hist[int64_t(d) * ntiles + blockIdx.x] = h[d];
}

// What a scatter writes besides the plain keys and values (the fused sort):
// kDownPlain  keys and values;
// kDownCount  keys and values, and the next pass's digit counts per
//             destination tile (hist_next[digit][tile]) and in total;
// kDownLast   values (the permutation) and the sorted coordinates
//             xs[j][pos] = x_ij - lo_j (a sample outside the box as at lo).
constexpr int kDownPlain = 0, kDownCount = 1, kDownLast = 2;
struct DownExtra {
  uint32_t* hist_next;
  uint32_t* dtot_next;
  GeoDev g;
  const void* x;
  void* xs;
};

// dynamic shared memory of radix_downsweep<B, ...>
template <int B>
constexpr size_t radix_down_smem() {
  return sizeof(uint32_t) * ((kSortThreads / 32 + 3) * (size_t(1) << B) + kSortThreads / 32 +
                             2 * size_t(kSortTile));
}

template <int B, int MODE = kDownPlain, typename T = float>
__global__ void __launch_bounds__(kSortThreads, 2)
radix_downsweep(const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                int64_t n, int shift, int64_t ntiles, const uint32_t* __restrict__ hist_scanned,
                uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out, DownExtra ex) {
  constexpr int NW = kSortThreads / 32;
  constexpr int RW = kSortTile / NW / 32;  // rounds of 32 keys per warp
  constexpr uint32_t R = 1u << B;
  constexpr int DPT = int(R) / kSortThreads;  // digits per thread
  static_assert(RW * NW * 32 == kSortTile && DPT >= 1 && DPT * kSortThreads == int(R),
                "tile and digit layout");
  extern __shared__ __align__(16) uint32_t dsm[];
  uint32_t* wh = dsm;                  // [NW][R] per-warp counts, then offsets in the digit's run
  uint32_t* dstart = wh + NW * R;      // [R] first tile position of each digit
  uint32_t* gbase = dstart + R;        // [R] first output position of each digit
  uint32_t* wsum = gbase + R;          // [NW]
  uint32_t* skey = wsum + NW;          // [kSortTile]
  uint32_t* sval = skey + kSortTile;   // [kSortTile]
  uint32_t* hn = sval + kSortTile;     // [R] next pass's digit totals (kDownCount)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (uint32_t d = tid; d < NW * R; d += kSortThreads) wh[d] = 0;
  if (MODE == kDownCount)
    for (uint32_t d = tid; d < R; d += kSortThreads) hn[d] = 0;
  __syncthreads();
  const int64_t tbase = int64_t(blockIdx.x) * kSortTile;
  const int64_t wbase = tbase + int64_t(warp) * (RW * 32);
  const uint32_t lt_mask = (1u << lane) - 1u;
  uint32_t key[RW], val[RW];
#pragma unroll
  for (int r = 0; r < RW; ++r) {  // every load of the chunk in flight first
    const int64_t i = wbase + r * 32 + lane;
    key[r] = i < n ? keys_in[i] : 0u;
    val[r] = i < n ? vals_in[i] : 0u;
  }
#pragma unroll
  for (int r = 0; r < RW; ++r) {
    const int64_t i = wbase + r * 32 + lane;
    const uint32_t dig = i < n ? (key[r] >> shift) & (R - 1u) : R;
    const uint32_t peers = match_digit<B>(dig);
    if (dig < R && (peers & lt_mask) == 0) wh[warp * R + dig] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // thread tid owns digits [tid DPT, (tid + 1) DPT): per-warp offsets inside
  // each digit's run, the digits' totals, then an exclusive scan of the
  // totals over all R digits
  uint32_t tot[DPT], own = 0;
#pragma unroll
  for (int u = 0; u < DPT; ++u) {
    const uint32_t d = uint32_t(tid * DPT + u);
    uint32_t t = 0;
    for (int w = 0; w < NW; ++w) {
      const uint32_t c = wh[w * R + d];
      wh[w * R + d] = t;
      t += c;
    }
    tot[u] = t;
    own += t;
    gbase[d] = hist_scanned[int64_t(d) * ntiles + blockIdx.x];
  }
  uint32_t inc = own;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  uint32_t run = inc - own;
  for (int w = 0; w < warp; ++w) run += wsum[w];
#pragma unroll
  for (int u = 0; u < DPT; ++u) {
    dstart[tid * DPT + u] = run;
    run += tot[u];
  }
  __syncthreads();
  // tile-local scatter into shared memory (sorted by digit, stable)
#pragma unroll
  for (int r = 0; r < RW; ++r) {
    const int64_t i = wbase + r * 32 + lane;
    const uint32_t dig = i < n ? (key[r] >> shift) & (R - 1u) : R;
    const uint32_t peers = match_digit<B>(dig);
    uint32_t off = 0;
    if (dig < R) {
      off = wh[warp * R + dig];
      const uint32_t lp = dstart[dig] + off + __popc(peers & lt_mask);
      skey[lp] = key[r];
      sval[lp] = val[r];
    }
    __syncwarp();  // every lane has read its group's offset
    if (dig < R && (peers & lt_mask) == 0) wh[warp * R + dig] = off + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // write out in tile order: consecutive threads write consecutive positions
  // of one digit's run
  const int cnt = int(n - tbase < kSortTile ? n - tbase : kSortTile);
  for (int t = tid; t < cnt; t += kSortThreads) {
    const uint32_t k = skey[t];
    const uint32_t dig = (k >> shift) & (R - 1u);
    const uint32_t pos = gbase[dig] + uint32_t(t) - dstart[dig];
    if (!in_range(ex.g.errw, kSiteSortScatter, pos, n)) continue;
    const uint32_t v = sval[t];
    vals_out[pos] = v;
    if (MODE != kDownLast) keys_out[pos] = k;
    if (MODE == kDownCount) {
      const uint32_t dn = (k >> (shift + B)) & (R - 1u);
      const int64_t hx = int64_t(dn) * ntiles + pos / uint32_t(kSortTile);
      if (in_range(ex.g.errw, kSiteSortHist, hx, int64_t(R) * ntiles)) atomicAdd(&ex.hist_next[hx], 1u);
      atomicAdd(&hn[dn], 1u);
    }
    if (MODE == kDownLast && in_range(ex.g.errw, kSiteSortCoords, v, n)) {
      const T* x = static_cast<const T*>(ex.x);
      T* xs = static_cast<T*>(ex.xs);
      for (int j = 0; j < ex.g.d; ++j) {
        T xv = x[int64_t(v) * ex.g.d + j];
        const T lo = T(ex.g.lo[j]), hi = T(ex.g.hi[j]);
        if (!(xv >= lo && xv <= hi)) xv = lo;
        xs[int64_t(j) * n + pos] = sub_rn(xv, lo);
      }
    }
  }
  if (MODE == kDownCount) {
    __syncthreads();
    for (uint32_t d = tid; d < R; d += kSortThreads)
      if (hn[d]) atomicAdd(&ex.dtot_next[d], hn[d]);
  }
}


template <typename T>
__global__ void gather_coords_kernel(GeoDev g, int64_t n, const T* __restrict__ x,
                                     const uint32_t* __restrict__ perm, T* __restrict__ xs) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const uint32_t i = perm[s];
  for (int j = 0; j < g.d; ++j) {
    T xv = x[int64_t(i) * g.d + j];
    const T lo = T(g.lo[j]), hi = T(g.hi[j]);
    if (!(xv >= lo && xv <= hi)) xv = lo;
    xs[int64_t(j) * n + s] = sub_rn(xv, lo);
  }
}

__global__ void nsub_kernel(const uint32_t* __restrict__ counts, int64_t nbins,
                            uint32_t* __restrict__ nsub) {
  const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (b >= nbins) return;
  nsub[b] = (counts[b] + kSubMax - 1) / kSubMax;
}

__global__ void fill_sub_kernel(const uint32_t* __restrict__ bin_start, int64_t nbins,
                                const uint32_t* __restrict__ sub_start,
                                uint32_t* __restrict__ sub_bin, uint32_t* __restrict__ sub_first) {
  const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (b >= nbins) return;
  const uint32_t s0 = sub_start[b], s1 = sub_start[b + 1];
  for (uint32_t k = s0; k < s1; ++k) {
    sub_bin[k] = uint32_t(b);
    sub_first[k] = bin_start[b] + (k - s0) * kSubMax;
  }
}

// Exclusive scan by one block of 1024 threads (short arrays such as the bin
// counts, at most 4 elements per thread): each thread sums a contiguous chunk, the
// block scans the chunk sums, and each thread writes its chunk's prefixes.
// in may alias out.
__global__ void __launch_bounds__(1024) scan_one_block(const uint32_t* in, int64_t n,
                                                       uint32_t* out) {
  __shared__ uint32_t wsum[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t chunk = (n + 1023) / 1024;
  const int64_t b0 = min(n, int64_t(tid) * chunk), b1 = min(n, b0 + chunk);
  uint32_t t = 0;
  for (int64_t i = b0; i < b1; ++i) t += in[i];
  uint32_t inc = t;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = wsum[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += v;
    }
    wsum[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  uint32_t run = (warp > 0 ? wsum[warp - 1] : 0u) + inc - t;
  for (int64_t i = b0; i < b1; ++i) {
    const uint32_t v = in[i];
    out[i] = run;
    run += v;
  }
  if (tid == 1023) out[n] = wsum[31];
}

// exclusive scan of in[0..n) into out[0..n], out[n] = total
cudaError_t exclusive_scan(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* scratch,
                           cudaStream_t s, int64_t* launches) {
  if (n <= 0) return cudaMemsetAsync(out, 0, sizeof(uint32_t), s);
  if (n <= 4096) {
    *launches += 1;
    scan_one_block<<<1, 1024, 0, s>>>(in, n, out);
    return cudaGetLastError();
  }
  *launches += 3;
  const int64_t nb = (n + kScanChunk - 1) / kScanChunk;
  scan_block_sums<<<unsigned(nb), kScanThreads, 0, s>>>(in, n, scratch);
  scan_sums_single<<<1, 1024, 0, s>>>(scratch, nb, out + n);
  scan_apply<<<unsigned(nb), kScanThreads, 0, s>>>(in, n, scratch, out);
  return cudaGetLastError();
}

// One LSD pass with B-bit digits: tile histograms, their scan, the scatter.
template <int B>
cudaError_t radix_pass(const uint32_t* kin, const uint32_t* vin, int64_t n, int shift,
                       int64_t ntiles, uint32_t* hist, uint32_t* scratch, uint32_t* kout,
                       uint32_t* vout, cudaStream_t s, int64_t* launches) {
  radix_upsweep<B><<<unsigned(ntiles), kSortThreads, 0, s>>>(kin, n, shift, ntiles, hist);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = exclusive_scan(hist, hist, (int64_t(1) << B) * ntiles, scratch, s, launches)) !=
      cudaSuccess)
    return e;
  constexpr size_t sm = radix_down_smem<B>();
  if ((e = cudaFuncSetAttribute(radix_downsweep<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(sm))) != cudaSuccess)
    return e;
  radix_downsweep<B><<<unsigned(ntiles), kSortThreads, sm, s>>>(kin, vin, n, shift, ntiles, hist,
                                                                kout, vout, DownExtra{});
  if (launches) *launches += 2;
  return cudaGetLastError();
}

}  // namespace

namespace {

// The fused sort: keys_tiles, then per pass digit_scan and a scatter.
template <int B, typename T>
cudaError_t run_sort_fused(fkreg_plan_s* P, int64_t n, const T* x, int passes, int64_t ntiles,
                           cudaStream_t s) {
  const GeoDev& g = P->geo;
  const int64_t nbins = P->nbins_total;
  uint32_t* keys[2] = {wsp<uint32_t>(P, P->r_keys0), wsp<uint32_t>(P, P->r_keys1)};
  uint32_t* vals[2] = {wsp<uint32_t>(P, P->r_vals0), wsp<uint32_t>(P, P->r_vals1)};
  uint32_t* hist[2] = {wsp<uint32_t>(P, P->r_hist), wsp<uint32_t>(P, P->r_hist2)};
  uint32_t* dtot[2] = {wsp<uint32_t>(P, P->r_dtot), wsp<uint32_t>(P, P->r_dtot) + 1024};
  uint32_t* counts = wsp<uint32_t>(P, P->r_counts);
  // the bin counts and the first pass's digit totals start at zero
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(uint32_t) * nbins, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(dtot[0], 0, sizeof(uint32_t) << B, s);
  if (e != cudaSuccess) return e;
  const unsigned kb = unsigned(std::min<int64_t>(ntiles, int64_t(P->sm_count) * 2));
  const size_t ks = sizeof(uint32_t) * (size_t(nbins) + (size_t(1) << B));
  keys_tiles_kernel<T, B><<<kb, kKeysThreads, ks, s>>>(g, n, nbins, ntiles, x, keys[0], vals[0],
                                                       counts, hist[0], dtot[0],
                                                       wsp<int>(P, P->r_err));
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  P->launches += 1;
  constexpr size_t sm = radix_down_smem<B>();
  const BinsArgs bins{counts,
                      nbins,
                      wsp<uint32_t>(P, P->r_binstart),
                      wsp<uint32_t>(P, P->r_substart),
                      wsp<uint32_t>(P, P->r_subbin),
                      wsp<uint32_t>(P, P->r_subfirst)};
  const unsigned sb = unsigned((1 << B) / kDigitScanWarps);
  int cur = 0;
  for (int p = 0; p < passes; ++p) {
    const bool last = p == passes - 1;
    const int nx = (p + 1) & 1;
    digit_scan_kernel<B><<<sb + (p == 0 ? 1u : 0u), kDigitScanWarps * 32, 0, s>>>(
        hist[p & 1], ntiles, dtot[p & 1], last ? nullptr : hist[nx], last ? nullptr : dtot[nx],
        p == 0 ? bins : BinsArgs{});
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    DownExtra ex{last ? nullptr : hist[nx], last ? nullptr : dtot[nx], g, x,
                 wsp<T>(P, P->r_xs)};
    if (last) {
      if ((e = cudaFuncSetAttribute(radix_downsweep<B, kDownLast, T>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm))) !=
          cudaSuccess)
        return e;
      radix_downsweep<B, kDownLast, T><<<unsigned(ntiles), kSortThreads, sm, s>>>(
          keys[cur], vals[cur], n, p * B, ntiles, hist[p & 1], keys[cur ^ 1], vals[cur ^ 1], ex);
    } else {
      if ((e = cudaFuncSetAttribute(radix_downsweep<B, kDownCount, T>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm))) !=
          cudaSuccess)
        return e;
      radix_downsweep<B, kDownCount, T><<<unsigned(ntiles), kSortThreads, sm, s>>>(
          keys[cur], vals[cur], n, p * B, ntiles, hist[p & 1], keys[cur ^ 1], vals[cur ^ 1], ex);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    P->launches += 2;
    cur ^= 1;
  }
  P->perm_in_vals1 = cur;
  return cudaSuccess;
}

}  // namespace

cudaError_t run_sort(fkreg_plan_s* P, int64_t n, const void* x, cudaStream_t s) {
  const GeoDev& g = P->geo;
  const int64_t nbins = P->nbins_total;
  // radix passes over the significant bits of the key
  int bits = g.kbits;
  while ((int64_t(1) << (bits - g.kbits)) < nbins) ++bits;
  // keys of 17..20 bits over at least 16 tiles: two passes of 10-bit digits;
  // otherwise 8-bit digits (small sorts are bound by the per-pass fixed
  // costs, which grow with the digit range)
  const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
  const int dbits = (bits > 16 && bits <= 20 && ntiles >= 16) ? 10 : kRadixBits;
  const int passes = (bits + dbits - 1) / dbits;
  if (n > 0 && passes >= 1 && nbins <= kFusedMaxBins) {
    const bool f32 = P->prec == FKREG_F32;
    if (dbits == 10)
      return f32 ? run_sort_fused<10>(P, n, static_cast<const float*>(x), passes, ntiles, s)
                 : run_sort_fused<10>(P, n, static_cast<const double*>(x), passes, ntiles, s);
    return f32 ? run_sort_fused<8>(P, n, static_cast<const float*>(x), passes, ntiles, s)
               : run_sort_fused<8>(P, n, static_cast<const double*>(x), passes, ntiles, s);
  }
  uint32_t* keys0 = wsp<uint32_t>(P, P->r_keys0);
  uint32_t* vals0 = wsp<uint32_t>(P, P->r_vals0);
  uint32_t* keys1 = wsp<uint32_t>(P, P->r_keys1);
  uint32_t* vals1 = wsp<uint32_t>(P, P->r_vals1);
  uint32_t* counts = wsp<uint32_t>(P, P->r_counts);
  uint32_t* bstart = wsp<uint32_t>(P, P->r_binstart);
  uint32_t* scratch = wsp<uint32_t>(P, P->r_scan);
  int* errw = wsp<int>(P, P->r_err);
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(uint32_t) * nbins, s);
  if (e != cudaSuccess) return e;
  if (n > 0) {
    const unsigned blocks = unsigned((n + 255) / 256);
    if (P->prec == FKREG_F32)
      bin_keys_kernel<float><<<blocks, 256, 0, s>>>(g, n, static_cast<const float*>(x), keys0, vals0,
                                                    counts, errw);
    else
      bin_keys_kernel<double><<<blocks, 256, 0, s>>>(g, n, static_cast<const double*>(x), keys0,
                                                     vals0, counts, errw);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    P->launches += 1;
  }
  uint32_t* hist = wsp<uint32_t>(P, P->r_hist);
  uint32_t *kin = keys0, *vin = vals0, *kout = keys1, *vout = vals1;
  int in_is_1 = 0;
  for (int p = 0; p < passes && n > 0; ++p) {
    const int shift = p * dbits;
    e = dbits == 10 ? radix_pass<10>(kin, vin, n, shift, ntiles, hist, scratch, kout, vout, s,
                                     &P->launches)
                    : radix_pass<8>(kin, vin, n, shift, ntiles, hist, scratch, kout, vout, s,
                                    &P->launches);
    if (e != cudaSuccess) return e;
    std::swap(kin, kout);
    std::swap(vin, vout);
    in_is_1 ^= 1;
  }
  P->perm_in_vals1 = in_is_1;
  if ((e = exclusive_scan(counts, bstart, nbins, scratch, s, &P->launches)) != cudaSuccess) return e;
  if (n > 0) {
    const unsigned blocks = unsigned((n + 255) / 256);
    if (P->prec == FKREG_F32)
      gather_coords_kernel<float><<<blocks, 256, 0, s>>>(g, n, static_cast<const float*>(x), vin,
                                                         wsp<float>(P, P->r_xs));
    else
      gather_coords_kernel<double><<<blocks, 256, 0, s>>>(g, n, static_cast<const double*>(x), vin,
                                                          wsp<double>(P, P->r_xs));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    P->launches += 1;
  }
  // spreading sub-problems: at most kSubMax samples each
  uint32_t* nsub = wsp<uint32_t>(P, P->r_nsub);
  uint32_t* sstart = wsp<uint32_t>(P, P->r_substart);
  const unsigned bb = unsigned((nbins + 255) / 256);
  nsub_kernel<<<bb, 256, 0, s>>>(counts, nbins, nsub);
  P->launches += 2;
  if ((e = exclusive_scan(nsub, sstart, nbins, scratch, s, &P->launches)) != cudaSuccess) return e;
  fill_sub_kernel<<<bb, 256, 0, s>>>(bstart, nbins, sstart, wsp<uint32_t>(P, P->r_subbin),
                                     wsp<uint32_t>(P, P->r_subfirst));
  return cudaGetLastError();
}

// ---- bin sort with library-owned static scratch ----------------------------
// Some callers cannot allocate device memory once they are running: a host
// program whose memory pool owns every device byte, a plug-in that is given
// buffers but no allocator, or a latency-critical loop that forbids
// allocation after start-up.  For them the stable bin sort has a variant
// whose scratch lives in this file-scope device array instead of a caller
// workspace.  Every GPU that loads the library holds the array until exit.
namespace {

constexpr int64_t kStaticMaxN = int64_t(1) << 18;      // samples per call
constexpr int64_t kStaticMaxBins = int64_t(1) << 16;   // spreading bins
constexpr int64_t kStaticTiles = (kStaticMaxN + kSortTile - 1) / kSortTile;
constexpr int64_t kStaticScanLen =
    (256 * kStaticTiles > kStaticMaxBins + 1) ? 256 * kStaticTiles : kStaticMaxBins + 1;
// word offsets inside the array (each region starts on a 256-byte boundary)
constexpr int64_t kOffKeys0 = 0;
constexpr int64_t kOffVals0 = kOffKeys0 + kStaticMaxN;
constexpr int64_t kOffKeys1 = kOffVals0 + kStaticMaxN;
constexpr int64_t kOffVals1 = kOffKeys1 + kStaticMaxN;
constexpr int64_t kOffCounts = kOffVals1 + kStaticMaxN;
constexpr int64_t kOffHist = kOffCounts + kStaticMaxBins;
constexpr int64_t kOffScan = kOffHist + ((256 * kStaticTiles + 1 + 63) / 64) * 64;
constexpr int64_t kOffErr = kOffScan + ((kStaticScanLen / 1024 + 2 + 63) / 64) * 64;
constexpr int64_t kStaticWords = kOffErr + 64;

static __device__ __align__(256) uint32_t g_sort_scratch[kStaticWords];

std::mutex g_static_mu;
constexpr int kMaxDevices = 64;
uint32_t* g_static_base[kMaxDevices] = {nullptr};

}  // namespace

}  // namespace fk

extern "C" fkreg_status fkreg_bin_sort_static(const fkreg_geometry* geom, const double* grid_lo,
                                              const double* grid_hi, int precision, int64_t n,
                                              const void* x_dev, uint32_t* perm_dev,
                                              uint32_t* bin_start_dev, int32_t* bad_dev,
                                              void* stream) {
  using namespace fk;
  if (!geom || !grid_lo || !grid_hi) return FKREG_ERR_INVALID_ARG;
  const int d = geom->dim;
  if (d < 1 || d > 3) return FKREG_ERR_INVALID_ARG;
  if (precision != FKREG_F32 && precision != FKREG_F64) return FKREG_ERR_INVALID_ARG;
  if (n < 0 || n > kStaticMaxN) return FKREG_ERR_INVALID_ARG;
  if (geom->w < 2 || geom->w > 32) return FKREG_ERR_INVALID_ARG;
  if ((n > 0 && !x_dev) || !perm_dev || !bin_start_dev) return FKREG_ERR_INVALID_ARG;
  int64_t nbins = 1;
  for (int j = 0; j < d; ++j) {
    if (geom->nf[j] < 1 || geom->tile[j] < 1 || geom->nbins[j] < 1 ||
        geom->nbins[j] != (geom->nf[j] + geom->tile[j] - 1) / geom->tile[j] ||
        !(geom->inv_h[j] > 0) || !(grid_hi[j] > grid_lo[j]))
      return FKREG_ERR_INVALID_ARG;
    nbins *= geom->nbins[j];
  }
  if (nbins > kStaticMaxBins) return FKREG_ERR_INVALID_ARG;
  // the device address of the array (host code cannot use the symbol itself,
  // which names a host-side shadow): looked up on every call outside a stream
  // capture, so a device reset that reloads the module is followed; during a
  // capture the address from an earlier call on this device is used
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FKREG_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  const bool capturing =
      cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone;
  uint32_t* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!capturing || !g_static_base[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess || !p) return FKREG_ERR_CUDA;
      g_static_base[dev] = static_cast<uint32_t*>(p);
    }
    base = g_static_base[dev];
  }
  GeoDev g{};
  g.d = d;
  for (int j = 0; j < 3; ++j) {
    g.nf[j] = j < d ? geom->nf[j] : 1;
    g.tile[j] = j < d ? geom->tile[j] : 1;
    g.nbins[j] = j < d ? geom->nbins[j] : 1;
    g.lo[j] = j < d ? grid_lo[j] : 0.0;
    g.hi[j] = j < d ? grid_hi[j] : 0.0;
    g.inv_h[j] = j < d ? geom->inv_h[j] : 1.0;
    g.inv_h_f[j] = float(g.inv_h[j]);
  }
  g.w = geom->w;
  g.kbits = key_local_bits(d, g.tile, g.nbins);
  uint32_t* keys0 = base + kOffKeys0;
  uint32_t* vals0 = base + kOffVals0;
  uint32_t* keys1 = base + kOffKeys1;
  uint32_t* vals1 = base + kOffVals1;
  uint32_t* counts = base + kOffCounts;
  uint32_t* hist = base + kOffHist;
  uint32_t* scan = base + kOffScan;
  int* errw = reinterpret_cast<int*>(base + kOffErr);
  int64_t launches = 0;
  // the array keeps the previous call's contents: zero what must start at zero
  if (cudaMemsetAsync(counts, 0, sizeof(uint32_t) * nbins, s) != cudaSuccess) return FKREG_ERR_CUDA;
  if (cudaMemsetAsync(errw, 0, sizeof(int), s) != cudaSuccess) return FKREG_ERR_CUDA;
  if (n > 0) {
    const unsigned blocks = unsigned((n + 255) / 256);
    if (precision == FKREG_F32)
      bin_keys_kernel<float><<<blocks, 256, 0, s>>>(g, n, static_cast<const float*>(x_dev), keys0,
                                                    vals0, counts, errw);
    else
      bin_keys_kernel<double><<<blocks, 256, 0, s>>>(g, n, static_cast<const double*>(x_dev), keys0,
                                                     vals0, counts, errw);
    if (cudaGetLastError() != cudaSuccess) return FKREG_ERR_CUDA;
  }
  int bits = g.kbits;
  while ((int64_t(1) << (bits - g.kbits)) < nbins) ++bits;
  const int passes = (bits + kRadixBits - 1) / kRadixBits;
  const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
  uint32_t *kin = keys0, *vin = vals0, *kout = keys1, *vout = vals1;
  for (int p = 0; p < passes && n > 0; ++p) {
    const int shift = p * kRadixBits;
    if (radix_pass<8>(kin, vin, n, shift, ntiles, hist, scan, kout, vout, s, &launches) !=
        cudaSuccess)
      return FKREG_ERR_CUDA;
    std::swap(kin, kout);
    std::swap(vin, vout);
  }
  if (exclusive_scan(counts, bin_start_dev, nbins, scan, s, &launches) != cudaSuccess) return FKREG_ERR_CUDA;
  if (n > 0 && cudaMemcpyAsync(perm_dev, vin, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s) !=
                   cudaSuccess)
    return FKREG_ERR_CUDA;
  if (bad_dev && cudaMemcpyAsync(bad_dev, errw, sizeof(int32_t), cudaMemcpyDeviceToDevice, s) !=
                     cudaSuccess)
    return FKREG_ERR_CUDA;
  return FKREG_OK;
}

