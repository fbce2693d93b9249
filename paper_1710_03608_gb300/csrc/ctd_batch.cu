// Batched CTD-S: n independent tensors (Algorithm 1 on each) decomposed
// concurrently.  Each tensor's pipeline has data-dependent sizes (s', s~,
// nnz(R), nnz(C)) that the host must read back before it can size the next
// buffers; run one tensor at a time and the GPU idles during every such
// read-back.  Here `workers` host threads each drive a library-owned CUDA
// stream and take tensors from a shared queue, largest first, so one
// tensor's read-backs overlap the kernels of the others.  The worker
// streams are ordered after the caller's stream on entry and the caller's
// stream after them on exit (events), so the call composes with stream
// order like a single launch.
#include <algorithm>
#include <atomic>
#include <numeric>
#include <thread>
#include <vector>

#include "ctd_internal.cuh"

using namespace ctd;

extern "C" ctd_status ctd_static_batched(int n, const ctd_coo3* X, int alpha, const int64_t* s,
                                         const uint64_t* seeds, double eps, int precision,
                                         unsigned flags, int workers, void* stream,
                                         ctd_factors** out) {
  if (n < 0 || (n > 0 && (!X || !s || !seeds || !out))) return fail(CTD_EINVAL, "NULL argument");
  if (n == 0) return CTD_OK;
  if (workers <= 0) workers = 8;
  workers = std::min(workers, std::min(n, 64));
  int dev = 0;
  CTD_CUDA(cudaGetDevice(&dev));
  cudaStream_t caller = static_cast<cudaStream_t>(stream);
  // fork: worker streams wait for the caller's stream
  cudaEvent_t fork = nullptr;
  std::vector<cudaStream_t> st(workers, nullptr);
  std::vector<cudaEvent_t> join(workers, nullptr);
  // on a failed set-up step, release what was created before it
  auto release = [&] {
    for (int w = 0; w < workers; ++w) {
      if (join[w]) cudaEventDestroy(join[w]);
      if (st[w]) cudaStreamDestroy(st[w]);
    }
    if (fork) cudaEventDestroy(fork);
  };
  cudaError_t ce = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaEventRecord(fork, caller);
  for (int w = 0; w < workers && ce == cudaSuccess; ++w) {
    ce = cudaStreamCreateWithFlags(&st[w], cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&join[w], cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(st[w], fork, 0);
  }
  if (ce != cudaSuccess) {
    release();
    for (int t = 0; t < n; ++t) out[t] = nullptr;
    return fail(CTD_ECUDA, std::string("ctd_static_batched set-up: ") + cudaGetErrorString(ce));
  }
  // largest tensors first: the queue's tail is short work
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return X[a].nnz > X[b].nnz; });
  std::vector<ctd_status> rc(n, CTD_OK);
  std::vector<std::string> msg(n);
  std::atomic<int> next{0};
  auto work = [&](int w) {
    cudaSetDevice(dev);
    for (int q = next.fetch_add(1); q < n; q = next.fetch_add(1)) {
      const int t = order[q];
      ctd_factors* F = nullptr;
      rc[t] = ctd_static(&X[t], alpha, s[t], eps, seeds[t], precision, flags, st[w], &F);
      if (rc[t] == CTD_OK) {
        out[t] = F;
      } else {
        out[t] = nullptr;
        msg[t] = ctd_last_error();
      }
    }
    cudaEventRecord(join[w], st[w]);
  };
  std::vector<std::thread> pool;
  // a thread that cannot be started leaves its share of the queue to the
  // others (no exception crosses the C ABI)
  for (int w = 1; w < workers; ++w) {
    try {
      pool.emplace_back(work, w);
    } catch (...) {
      cudaEventRecord(join[w], st[w]);
    }
  }
  work(0);
  for (auto& th : pool) th.join();
  // join: the caller's stream waits for every worker stream
  for (int w = 0; w < workers; ++w) cudaStreamWaitEvent(caller, join[w], 0);
  for (int w = 0; w < workers; ++w) {
    cudaEventDestroy(join[w]);
    // the factors keep using their worker stream for getters: hand them the
    // caller's stream instead, which is now ordered after the worker's work
  }
  cudaEventDestroy(fork);
  for (int t = 0; t < n; ++t)
    if (out[t]) {
      cudaStreamSynchronize(out[t]->stream);
      out[t]->stream = caller;
      out[t]->mem.st = caller;
    }
  for (int w = 0; w < workers; ++w) cudaStreamDestroy(st[w]);
  for (int t = 0; t < n; ++t)
    if (rc[t] != CTD_OK) {
      for (int u = 0; u < n; ++u)
        if (out[u]) {
          ctd_free(out[u]);
          out[u] = nullptr;
        }
      return fail(rc[t], "tensor " + std::to_string(t) + ": " + msg[t]);
    }
  return CTD_OK;
}
