// Serving loop for CTD-D (Algorithm 2) with continuous batching.
//
// A server owns one CTD-D state per stream (kept on the device for the
// server's life).  Requests -- one new slice for one stream -- are queued
// per stream and run in submission order within a stream.  `workers` host
// threads, each with its own CUDA stream, take the oldest waiting request
// whose stream is idle, as soon as a worker frees up: steps of different
// streams overlap on the device, and a request that arrives while others
// run is admitted without waiting for a batch boundary.  Admission also
// checks device memory: a step starts only if the memory available to the
// library, less the estimates of the steps already running, covers its own
// estimate (at least one step always runs, so the queue cannot stall).
// Available: a fraction of the device's free memory with the library's own
// pool; with an allocator hook (ctd_set_allocator), whose cache keeps what
// the library frees out of the device's free count, a budget fixed at
// creation (that fraction of free memory plus what the library then held)
// less the bytes the library holds now.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "ctd_internal.cuh"

using namespace ctd;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int stream = 0;
  ctd_coo3 X{};
  Clock::time_point t_submit, t_start, t_done;
  size_t estimate = 0;
  ctd_status rc = CTD_OK;
  bool done = false;
  std::string msg;
};

}  // namespace

struct ctd_server {
  int n_streams = 0;
  int64_t d = 0;
  double eps = 0.0;
  double mem_fraction = 0.9;
  size_t budget = 0;   // with an allocator hook: bytes the library may hold
  int dev = 0;
  std::vector<ctd_factors*> states;
  // per stream, the state's kept count and column count after its last
  // finished step: submit sizes its estimate from these (under the lock)
  // rather than reading a state that a worker may be updating
  std::vector<int64_t> kept_seen, cols_seen;
  std::vector<std::deque<int64_t>> queue;   // tickets per stream
  std::vector<char> busy;
  std::vector<Request> req;                  // by ticket
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  size_t running_bytes = 0;
  int running = 0;
  std::vector<std::thread> pool;
  std::vector<cudaStream_t> cstream;
};

namespace {

size_t step_estimate(int64_t s_kept, int64_t n_cols, const ctd_coo3& X, int64_t d) {
  const double dt = (double)s_kept + (double)d;
  // COO staging + CSC + CDF (~64 B/nnz), candidates' Gram/Schur/W (FP64),
  // U/L growth, the new-column block (bounded by nnz * d~ / 8 B on average)
  return (size_t)(64.0 * X.nnz + 8.0 * (double)n_cols * 6.0 + 24.0 * dt * d +
                  16.0 * dt * dt * 0.25 + 12.0 * (double)X.nnz * 16.0);
}

void worker(ctd_server* S, int w) {
  cudaSetDevice(S->dev);
  while (true) {
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    int64_t ticket = -1;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      while (true) {
        if (S->stop) return;
        // oldest waiting request on an idle stream that fits in memory
        int64_t best = -1;
        for (int s = 0; s < S->n_streams; ++s) {
          if (S->busy[s] || S->queue[s].empty()) continue;
          const int64_t t = S->queue[s].front();
          if (best < 0 || t < best) best = t;
        }
        if (best >= 0) {
          Request& r = S->req[best];
          size_t avail = (size_t)((double)free_b * S->mem_fraction);
          if (allocator_hooked()) {
            const size_t held = live_bytes();
            avail = S->budget > held ? S->budget - held : 0;
          }
          const bool fits = S->running == 0 || S->running_bytes + r.estimate <= avail;
          if (fits) {
            ticket = best;
            S->busy[r.stream] = 1;
            S->queue[r.stream].pop_front();
            S->running_bytes += r.estimate;
            S->running += 1;
            break;
          }
        }
        S->cv.wait_for(lk, std::chrono::milliseconds(2));
        lk.unlock();
        cudaMemGetInfo(&free_b, &total_b);
        lk.lock();
      }
    }
    Request& r = S->req[ticket];
    r.t_start = Clock::now();
    r.rc = ctd_dynamic_step(S->states[r.stream], &r.X, S->d, S->eps, S->cstream[w]);
    if (r.rc != CTD_OK) r.msg = ctd_last_error();
    r.t_done = Clock::now();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      r.done = true;
      S->kept_seen[r.stream] = S->states[r.stream]->s_kept;
      S->cols_seen[r.stream] = S->states[r.stream]->n_cols;
      S->busy[r.stream] = 0;
      S->running_bytes -= r.estimate;
      S->running -= 1;
    }
    S->cv.notify_all();
  }
}

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

extern "C" ctd_status ctd_server_create(int n_streams, const int64_t dims2[2], int alpha,
                                        int precision, uint64_t seed, int64_t d, double eps,
                                        int workers, double mem_fraction, ctd_server** out) {
  if (!out || !dims2) return fail(CTD_EINVAL, "NULL argument");
  if (n_streams < 1 || n_streams > 65536) return fail(CTD_EINVAL, "n_streams out of range");
  if (d < 1 || d > 8192) return fail(CTD_EINVAL, "d must be in [1, 8192]");
  if (!(eps >= 0.0 && eps < 1.0)) return fail(CTD_EINVAL, "eps must be in [0, 1)");
  if (workers <= 0) workers = 8;
  if (!(mem_fraction > 0.0 && mem_fraction <= 1.0)) mem_fraction = 0.9;
  ctd_server* S = new (std::nothrow) ctd_server();
  if (!S) return fail(CTD_ENOMEM, "host allocation failed");
  S->n_streams = n_streams;
  S->d = d;
  S->eps = eps;
  S->mem_fraction = mem_fraction;
  cudaGetDevice(&S->dev);
  {
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    S->budget = (size_t)(mem_fraction * (double)(free_b + live_bytes()));
  }
  S->states.assign(n_streams, nullptr);
  S->queue.resize(n_streams);
  S->busy.assign(n_streams, 0);
  S->req.reserve(1 << 16);
  for (int k = 0; k < n_streams; ++k) {
    ctd_status rc = ctd_dynamic_create(dims2, alpha, precision, seed, (uint64_t)k, 0, &S->states[k]);
    if (rc != CTD_OK) {
      ctd_server_free(S);
      return rc;
    }
  }
  S->kept_seen.assign(n_streams, 0);
  S->cols_seen.assign(n_streams, 0);
  for (int k = 0; k < n_streams; ++k) {
    S->kept_seen[k] = S->states[k]->s_kept;
    S->cols_seen[k] = S->states[k]->n_cols;
  }
  S->cstream.assign(workers, nullptr);
  for (int w = 0; w < workers; ++w)
    if (cudaStreamCreateWithFlags(&S->cstream[w], cudaStreamNonBlocking) != cudaSuccess) {
      ctd_server_free(S);
      return fail(CTD_ECUDA, "stream creation failed");
    }
  for (int w = 0; w < workers; ++w) {
    try {
      S->pool.emplace_back(worker, S, w);
    } catch (...) {  // no exception crosses the C ABI; run with the threads started
      if (S->pool.empty()) {
        ctd_server_free(S);
        return fail(CTD_ENOMEM, "could not start a worker thread");
      }
      break;
    }
  }
  *out = S;
  return CTD_OK;
}

extern "C" ctd_status ctd_server_submit(ctd_server* S, int stream_id, const ctd_coo3* dX,
                                        int64_t* ticket) {
  if (!S || !dX || !ticket) return fail(CTD_EINVAL, "NULL argument");
  if (stream_id < 0 || stream_id >= S->n_streams) return fail(CTD_EINVAL, "stream out of range");
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->req.size() == S->req.capacity())
    return fail(CTD_ENOTSUP, "too many requests for one server (65536)");
  Request r;
  r.stream = stream_id;
  r.X = *dX;
  r.t_submit = Clock::now();
  r.estimate = step_estimate(S->kept_seen[stream_id], S->cols_seen[stream_id], *dX, S->d);
  S->req.push_back(r);
  const int64_t t = (int64_t)S->req.size() - 1;
  S->queue[stream_id].push_back(t);
  *ticket = t;
  S->cv.notify_one();
  return CTD_OK;
}

extern "C" ctd_status ctd_server_wait(ctd_server* S, int64_t ticket) {
  if (!S) return fail(CTD_EINVAL, "NULL argument");
  std::unique_lock<std::mutex> lk(S->mu);
  if (ticket >= (int64_t)S->req.size()) return fail(CTD_EINVAL, "unknown ticket");
  auto done = [&] {
    if (ticket >= 0) return S->req[ticket].done;
    for (const auto& r : S->req)
      if (!r.done) return false;
    return true;
  };
  while (!done()) S->cv.wait_for(lk, std::chrono::milliseconds(5));
  if (ticket >= 0 && S->req[ticket].rc != CTD_OK)
    return fail(S->req[ticket].rc, S->req[ticket].msg);
  if (ticket < 0)
    for (const auto& r : S->req)
      if (r.rc != CTD_OK) return fail(r.rc, r.msg);
  return CTD_OK;
}

extern "C" ctd_status ctd_server_result(ctd_server* S, int64_t ticket, int* status, double ms[3]) {
  if (!S || !ms) return fail(CTD_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  if (ticket < 0 || ticket >= (int64_t)S->req.size()) return fail(CTD_EINVAL, "unknown ticket");
  const Request& r = S->req[ticket];
  if (!r.done) return fail(CTD_EINVAL, "request still running");
  if (status) *status = r.rc;
  ms[0] = ms_between(r.t_submit, r.t_start);
  ms[1] = ms_between(r.t_start, r.t_done);
  ms[2] = ms_between(r.t_submit, r.t_done);
  return CTD_OK;
}

extern "C" ctd_status ctd_server_state(ctd_server* S, int stream_id, ctd_factors** state) {
  if (!S || !state) return fail(CTD_EINVAL, "NULL argument");
  if (stream_id < 0 || stream_id >= S->n_streams) return fail(CTD_EINVAL, "stream out of range");
  *state = S->states[stream_id];
  return CTD_OK;
}

extern "C" void ctd_server_free(ctd_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  for (auto& th : S->pool) th.join();
  for (auto* F : S->states)
    if (F) ctd_free(F);
  for (auto st : S->cstream)
    if (st) cudaStreamDestroy(st);
  delete S;
}
