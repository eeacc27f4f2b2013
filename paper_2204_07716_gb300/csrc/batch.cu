// Uneven batches of independent problems in one captured CUDA graph.
//
// Each problem has its own plan (own geometry, cuFFT plans and workspace
// slice of one caller-owned buffer).  fkreg_batch_capture records, for every
// problem, bin sort -> smooth (grid estimate + values at the samples) ->
// conditional-variance pass, on branches forked from the capture stream (up
// to kBranches concurrent branches), stamps the global timer when each
// problem's last kernel is done, joins the branches and instantiates the
// graph.  fkreg_batch_launch replays it; fkreg_batch_latencies reads the
// per-problem completion times relative to the graph's start stamp.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "internal.h"

namespace {

constexpr int kBranches = 16;
constexpr size_t kAlignB = 256;

__global__ void stamp_kernel(unsigned long long* out) {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  *out = t;
}

}  // namespace

struct fkreg_batch_s {
  std::vector<fkreg_plan> plans;
  std::vector<size_t> offs;     // workspace offset of each plan
  size_t stamp_off = 0;         // (problems + 1) 64-bit timer stamps
  size_t ws_bytes = 0;
  char* ws = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  cudaStream_t cap = nullptr;   // capture origin (the legacy stream cannot be captured)
  std::string err;
};

namespace {

fkreg_status batch_err(fkreg_batch_s* B, fkreg_status st, const std::string& m) {
  if (B) B->err = m;
  return st;
}

void release_graph(fkreg_batch_s* B) {
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  B->exec = nullptr;
  B->graph = nullptr;
}

}  // namespace

extern "C" {

fkreg_status fkreg_batch_create(int n_problems, const fkreg_opts* opts, const int64_t* max_n,
                                fkreg_batch* out) {
  if (!out || n_problems < 1 || !opts || !max_n) return FKREG_ERR_INVALID_ARG;
  *out = nullptr;
  auto* B = new fkreg_batch_s();
  size_t cur = 0;
  for (int p = 0; p < n_problems; ++p) {
    fkreg_plan P = nullptr;
    fkreg_status st = fkreg_plan_create(&opts[p], max_n[p], &P);
    if (st != FKREG_OK) {
      for (auto q : B->plans) fkreg_plan_destroy(q);
      delete B;
      return st;
    }
    size_t bytes = 0;
    fkreg_workspace_bytes(P, &bytes);
    cur = (cur + kAlignB - 1) / kAlignB * kAlignB;
    B->offs.push_back(cur);
    cur += bytes;
    B->plans.push_back(P);
  }
  cur = (cur + kAlignB - 1) / kAlignB * kAlignB;
  B->stamp_off = cur;
  cur += sizeof(unsigned long long) * (n_problems + 1);
  B->ws_bytes = cur + kAlignB;
  *out = B;
  return FKREG_OK;
}

fkreg_status fkreg_batch_workspace_bytes(fkreg_batch B, size_t* bytes) {
  if (!B || !bytes) return FKREG_ERR_INVALID_ARG;
  *bytes = B->ws_bytes;
  return FKREG_OK;
}

fkreg_plan fkreg_batch_plan(fkreg_batch B, int p) {
  if (!B || p < 0 || p >= int(B->plans.size())) return nullptr;
  return B->plans[p];
}

fkreg_status fkreg_batch_set_workspace(fkreg_batch B, void* ws, size_t bytes, void* stream) {
  if (!B || !ws) return FKREG_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(ws) % kAlignB)
    return batch_err(B, FKREG_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  if (bytes < B->ws_bytes) return batch_err(B, FKREG_ERR_WORKSPACE, "batch workspace too small");
  B->ws = static_cast<char*>(ws);
  for (size_t p = 0; p < B->plans.size(); ++p) {
    size_t need = 0;
    fkreg_workspace_bytes(B->plans[p], &need);
    fkreg_status st = fkreg_set_workspace(B->plans[p], B->ws + B->offs[p], need, stream);
    if (st != FKREG_OK)
      return batch_err(B, st, "problem " + std::to_string(p) + ": " + fkreg_last_error(B->plans[p]));
  }
  release_graph(B);
  return FKREG_OK;
}

fkreg_status fkreg_batch_capture(fkreg_batch B, const int64_t* n, const void* const* x,
                                 const void* const* y, const fkreg_outputs* outs,
                                 void* const* sigma2, void* stream) {
  if (!B || !n || !x || !y || !outs) return FKREG_ERR_INVALID_ARG;
  if (!B->ws) return batch_err(B, FKREG_ERR_STATE, "fkreg_batch_set_workspace must come first");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int np = int(B->plans.size());
  for (int p = 0; p < np; ++p)
    if (sigma2 && sigma2[p] && !outs[p].mhat_at_x)
      return batch_err(B, FKREG_ERR_INVALID_ARG, "the variance pass needs mhat_at_x");
  release_graph(B);
  if (B->streams.empty()) {
    for (int i = 0; i < kBranches; ++i) {
      cudaStream_t t;
      if (cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking) != cudaSuccess)
        return batch_err(B, FKREG_ERR_CUDA, "stream create");
      B->streams.push_back(t);
    }
    for (int i = 0; i < kBranches + 1; ++i) {
      cudaEvent_t e;
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
        return batch_err(B, FKREG_ERR_CUDA, "event create");
      B->events.push_back(e);
    }
  }
  if (!B->cap && cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking) != cudaSuccess)
    return batch_err(B, FKREG_ERR_CUDA, "stream create");
  // nothing is executed while capturing; finish the caller's pending work first
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return batch_err(B, FKREG_ERR_CUDA, std::string("sync: ") + cudaGetErrorString(e));
  s = B->cap;
  auto* stamps = reinterpret_cast<unsigned long long*>(B->ws + B->stamp_off);
  e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return batch_err(B, FKREG_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
  fkreg_status st = FKREG_OK;
  std::string msg;
  stamp_kernel<<<1, 1, 0, s>>>(stamps + np);
  cudaEventRecord(B->events[kBranches], s);
  const int nb = std::min(kBranches, np);
  for (int i = 0; i < nb; ++i) cudaStreamWaitEvent(B->streams[i], B->events[kBranches], 0);
  for (int p = 0; p < np && st == FKREG_OK; ++p) {
    cudaStream_t t = B->streams[p % nb];
    fkreg_plan P = B->plans[p];
    st = fkreg_set_points(P, n[p], x[p], t);
    if (st == FKREG_OK) st = fkreg_smooth(P, y[p], &outs[p], t);
    if (st == FKREG_OK && sigma2 && sigma2[p])
      st = fkreg_variance(P, y[p], outs[p].mhat_at_x, sigma2[p], t);
    if (st != FKREG_OK) msg = "problem " + std::to_string(p) + ": " + fkreg_last_error(P);
    stamp_kernel<<<1, 1, 0, t>>>(stamps + p);
  }
  for (int i = 0; i < nb; ++i) {
    cudaEventRecord(B->events[i], B->streams[i]);
    cudaStreamWaitEvent(s, B->events[i], 0);
  }
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(s, &g);
  if (st != FKREG_OK) {
    if (g) cudaGraphDestroy(g);
    return batch_err(B, st, msg);
  }
  if (e != cudaSuccess) return batch_err(B, FKREG_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(e));
  B->graph = g;
  e = cudaGraphInstantiate(&B->exec, g, 0);
  if (e != cudaSuccess) {
    release_graph(B);
    return batch_err(B, FKREG_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
  }
  return FKREG_OK;
}

fkreg_status fkreg_batch_launch(fkreg_batch B, void* stream) {
  if (!B) return FKREG_ERR_INVALID_ARG;
  if (!B->exec) return batch_err(B, FKREG_ERR_STATE, "fkreg_batch_capture must come first");
  cudaError_t e = cudaGraphLaunch(B->exec, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return batch_err(B, FKREG_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  return FKREG_OK;
}

fkreg_status fkreg_batch_latencies(fkreg_batch B, double* ms, void* stream) {
  if (!B || !ms) return FKREG_ERR_INVALID_ARG;
  const int np = int(B->plans.size());
  std::vector<unsigned long long> h(np + 1);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(h.data(), B->ws + B->stamp_off, sizeof(unsigned long long) * (np + 1),
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return batch_err(B, FKREG_ERR_CUDA, std::string("latencies: ") + cudaGetErrorString(e));
  for (int p = 0; p < np; ++p) ms[p] = double(h[p] - h[np]) * 1e-6;
  return FKREG_OK;
}

const char* fkreg_batch_last_error(fkreg_batch B) { return B ? B->err.c_str() : ""; }

void fkreg_batch_destroy(fkreg_batch B) {
  if (!B) return;
  release_graph(B);
  for (auto t : B->streams) cudaStreamDestroy(t);
  if (B->cap) cudaStreamDestroy(B->cap);
  for (auto ev : B->events) cudaEventDestroy(ev);
  for (auto P : B->plans) fkreg_plan_destroy(P);
  delete B;
}

}  // extern "C"
