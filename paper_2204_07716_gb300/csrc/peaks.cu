// Microbenchmarks of the SM-side rates that bound the spreading and
// interpolation kernels (fkreg_measure_peaks): FP32 FMA throughput (scalar
// and packed), warp-level TF32 tensor products, shared-memory load delivery
// for 4/8/16-byte lanes and for a warp-wide broadcast, and shared / global
// atomic rates.  Each test runs
// a fixed amount of work on every SM in one wave, timed with CUDA events on
// the caller's stream after an untimed warm-up launch.  The SM clock is read
// from clock64() inside the FP32 test; no device setting is touched.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/fkreg_peaks.h"

namespace {

constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;
constexpr int kUnroll = 8;
constexpr int kSmemBytes = 16384;

__global__ void __launch_bounds__(kThreads) fma_kernel(int iters, float seed,
                                                       float* __restrict__ sink,
                                                       long long* __restrict__ cycles) {
  float a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = seed + 1e-3f * float(threadIdx.x & 7) + float(k);
  const float m = 0.99999988f, c = 1e-7f;
  const long long t0 = clock64();
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], m, c);
  }
  const long long t1 = clock64();
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == -1.0f) sink[blockIdx.x] = s;  // never true: keeps every chain live
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

__global__ void __launch_bounds__(kThreads) fma2_kernel(int iters, float seed,
                                                        float* __restrict__ sink) {
  float2 a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    a[k].x = seed + 1e-3f * float(threadIdx.x & 7) + float(k);
    a[k].y = a[k].x + 0.5f;
  }
  const float2 m = make_float2(0.99999988f, 0.99999988f), c = make_float2(1e-7f, 1e-7f);
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = __ffma2_rn(a[k], m, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k].x + a[k].y;
  if (s == -1.0f) sink[blockIdx.x] = s;
}

// Warp-level TF32 tensor products (mma.sync m16n8k8, FP32 accumulate): eight
// independent accumulator tiles per warp, operands held in registers.
__global__ void __launch_bounds__(kThreads) mma_tf32_kernel(int iters, float* __restrict__ sink) {
  uint32_t a[4], b[2];
#pragma unroll
  for (int k = 0; k < 4; ++k) a[k] = __float_as_uint(1.0f + 1e-3f * float(threadIdx.x + k));
  b[0] = __float_as_uint(0.5f);
  b[1] = __float_as_uint(0.25f + 1e-3f * float(threadIdx.x & 7));
  float d[8][4];
#pragma unroll
  for (int t = 0; t < 8; ++t)
#pragma unroll
    for (int k = 0; k < 4; ++k) d[t][k] = 0.f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int t = 0; t < 8; ++t)
      asm volatile(
          "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, "
          "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
          : "+f"(d[t][0]), "+f"(d[t][1]), "+f"(d[t][2]), "+f"(d[t][3])
          : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  }
  float s = 0.f;
#pragma unroll
  for (int t = 0; t < 8; ++t) s += d[t][0] + d[t][1] + d[t][2] + d[t][3];
  if (s == -1.0f) sink[blockIdx.x] = s;
}

__device__ __forceinline__ void xor_into(unsigned& a, unsigned v) { a ^= v; }
__device__ __forceinline__ void xor_into(uint2& a, uint2 v) {
  a.x ^= v.x;
  a.y ^= v.y;
}
__device__ __forceinline__ void xor_into(uint4& a, uint4 v) {
  a.x ^= v.x;
  a.y ^= v.y;
  a.z ^= v.z;
  a.w ^= v.w;
}
__device__ __forceinline__ unsigned fold(unsigned a) { return a; }
__device__ __forceinline__ unsigned fold(uint2 a) { return a.x ^ a.y; }
__device__ __forceinline__ unsigned fold(uint4 a) { return a.x ^ a.y ^ a.z ^ a.w; }

// Shared loads of sizeof(V) bytes per lane: consecutive lanes read
// consecutive elements (no bank conflicts), or with bcast every lane of a
// warp reads the same element.  Indices wrap inside the 16 KB buffer.
template <typename V>
__global__ void __launch_bounds__(kThreads) smem_load_kernel(int iters, int bcast,
                                                             unsigned* __restrict__ sink) {
  __shared__ __align__(16) unsigned buf[kSmemBytes / 4];
  for (int i = threadIdx.x; i < kSmemBytes / 4; i += blockDim.x) buf[i] = unsigned(i) * 2654435761u;
  __syncthreads();
  const V* b = reinterpret_cast<const V*>(buf);
  constexpr int nv = kSmemBytes / int(sizeof(V));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  V acc{};
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int k = i * kUnroll + u + warp;
      const int idx = bcast ? (k & (nv - 1)) : ((lane + 32 * k) & (nv - 1));
      xor_into(acc, b[idx]);
    }
  }
  if (fold(acc) == 0x9E3779B9u) sink[blockIdx.x] = fold(acc);
}

__global__ void __launch_bounds__(kThreads) smem_atomic_kernel(int iters,
                                                               unsigned* __restrict__ sink) {
  __shared__ unsigned buf[1024];
  for (int i = threadIdx.x; i < 1024; i += blockDim.x) buf[i] = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int k = (i * kUnroll + u + warp) & 31;
      atomicAdd(&buf[lane + 32 * k], 1u);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && buf[0] == 0x9E3779B9u) sink[blockIdx.x] = buf[0];
}

// FP32 atomicAdd to global memory: lanes of a warp hit consecutive words of
// a 4 MB span (it stays in L2), warps and iterations walk through it.
__global__ void __launch_bounds__(kThreads) gmem_atomic_kernel(int iters, float* __restrict__ dst,
                                                               int nwords) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nthr = gridDim.x * blockDim.x;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const long long k = (long long)tid + (long long)nthr * (i * kUnroll + u);
      atomicAdd(&dst[int(k % nwords)], 1.0f);
    }
  }
}

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaStream_t s;
  explicit Timer(cudaStream_t st) : s(st) {}
  bool init() {
    return cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess;
  }
  ~Timer() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
  // milliseconds of one launch made by f (after an untimed warm-up launch)
  template <typename F>
  bool time(F f, float* ms) {
    f();
    if (cudaGetLastError() != cudaSuccess) return false;
    if (cudaEventRecord(a, s) != cudaSuccess) return false;
    f();
    if (cudaGetLastError() != cudaSuccess) return false;
    if (cudaEventRecord(b, s) != cudaSuccess) return false;
    if (cudaEventSynchronize(b) != cudaSuccess) return false;
    return cudaEventElapsedTime(ms, a, b) == cudaSuccess;
  }
};

}  // namespace

extern "C" fkreg_status fkreg_measure_peaks(fkreg_peaks* out, void* scratch_dev,
                                            size_t scratch_bytes, void* stream) {
  if (!out || !scratch_dev || scratch_bytes < FKREG_PEAKS_SCRATCH_BYTES)
    return FKREG_ERR_INVALID_ARG;
  *out = fkreg_peaks{};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return FKREG_ERR_CUDA;
  out->sm_count = sms;
  const int blocks = sms * kBlocksPerSm;
  const double threads = double(blocks) * kThreads;
  // scratch: [0, 64 KB) sinks and cycle counters, the rest the atomic span
  char* base = static_cast<char*>(scratch_dev);
  float* sinkf = reinterpret_cast<float*>(base);
  unsigned* sinku = reinterpret_cast<unsigned*>(base + 16384);
  long long* cycles = reinterpret_cast<long long*>(base + 32768);
  float* span = reinterpret_cast<float*>(base + 65536);
  const int nwords = int((scratch_bytes - 65536) / sizeof(float));
  if (blocks * int(sizeof(long long)) > 32768) return FKREG_ERR_INVALID_ARG;
  Timer t(s);
  if (!t.init()) return FKREG_ERR_CUDA;
  float ms = 0.f;
  // FP32 FMA, scalar; the SM clock from the blocks' cycle counts
  const int it_fma = 1 << 16;
  if (!t.time([&] { fma_kernel<<<blocks, kThreads, 0, s>>>(it_fma, 1.0f, sinkf, cycles); }, &ms))
    return FKREG_ERR_CUDA;
  out->fp32_tflops = 2.0 * 8.0 * it_fma * threads / (ms * 1e-3) / 1e12;
  {
    long long cyc[4096];
    const int nb = std::min(blocks, 4096);
    if (cudaMemcpyAsync(cyc, cycles, sizeof(long long) * nb, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return FKREG_ERR_CUDA;
    double mx = 0.0;
    for (int i = 0; i < nb; ++i) mx = std::max(mx, double(cyc[i]));
    out->sm_mhz = mx / (ms * 1e-3) / 1e6;
  }
  if (!t.time([&] { fma2_kernel<<<blocks, kThreads, 0, s>>>(it_fma, 1.0f, sinkf); }, &ms))
    return FKREG_ERR_CUDA;
  out->fp32x2_tflops = 4.0 * 8.0 * it_fma * threads / (ms * 1e-3) / 1e12;
  // TF32 tensor products through mma.sync (2 x 16 x 8 x 8 flop per warp-instruction)
  const int it_mma = 1 << 12;
  if (!t.time([&] { mma_tf32_kernel<<<blocks, kThreads, 0, s>>>(it_mma, sinkf); }, &ms))
    return FKREG_ERR_CUDA;
  out->tf32_mma_tflops = 2.0 * 16 * 8 * 8 * 8.0 * it_mma * (threads / 32.0) / (ms * 1e-3) / 1e12;
  // shared-memory loads
  const int it_ld = 1 << 13;
  const double loads = double(it_ld) * kUnroll * threads;
  if (!t.time([&] { smem_load_kernel<unsigned><<<blocks, kThreads, 0, s>>>(it_ld, 0, sinku); }, &ms))
    return FKREG_ERR_CUDA;
  out->smem_load_gbs[0] = loads * 4.0 / (ms * 1e-3) / 1e9;
  if (!t.time([&] { smem_load_kernel<uint2><<<blocks, kThreads, 0, s>>>(it_ld, 0, sinku); }, &ms))
    return FKREG_ERR_CUDA;
  out->smem_load_gbs[1] = loads * 8.0 / (ms * 1e-3) / 1e9;
  if (!t.time([&] { smem_load_kernel<uint4><<<blocks, kThreads, 0, s>>>(it_ld, 0, sinku); }, &ms))
    return FKREG_ERR_CUDA;
  out->smem_load_gbs[2] = loads * 16.0 / (ms * 1e-3) / 1e9;
  if (!t.time([&] { smem_load_kernel<uint4><<<blocks, kThreads, 0, s>>>(it_ld, 1, sinku); }, &ms))
    return FKREG_ERR_CUDA;
  out->smem_bcast16_gbs = loads * 16.0 / (ms * 1e-3) / 1e9;
  // atomics
  const int it_sa = 1 << 12;
  if (!t.time([&] { smem_atomic_kernel<<<blocks, kThreads, 0, s>>>(it_sa, sinku); }, &ms))
    return FKREG_ERR_CUDA;
  out->smem_atomic_gops = double(it_sa) * kUnroll * threads / (ms * 1e-3) / 1e9;
  const int it_ga = 1 << 8;
  if (!t.time([&] { gmem_atomic_kernel<<<blocks, kThreads, 0, s>>>(it_ga, span, nwords); }, &ms))
    return FKREG_ERR_CUDA;
  out->gmem_atomic_gops = double(it_ga) * kUnroll * threads / (ms * 1e-3) / 1e9;
  return FKREG_OK;
}
