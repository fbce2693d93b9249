// C ABI: allocation, errors, CTD-S (Algorithm 1) orchestration and getters.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <numeric>
#include <set>
#include <unordered_map>

#include "ctd_internal.cuh"

namespace ctd {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

ctd_status fail(ctd_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

ctd_status status_from_device(unsigned w) {
  if (w & DEV_BAD_INDEX) return fail(CTD_EINVAL, "a COO index lies outside its mode's extent");
  if (w & DEV_OVERFLOW) return fail(CTD_EOVERFLOW, "||X||_F^2 does not fit in 63 bits");
  if (w & DEV_CAPACITY) return fail(CTD_EINVAL, "a size exceeded its buffer bound");
  if (w & DEV_TIMEOUT) return fail(CTD_ETIMEOUT, "a bounded device wait gave up");
  return CTD_OK;
}

// ---------------------------------------------------------------------------
// diagnostics: launch counter and phase timers
// ---------------------------------------------------------------------------
static std::atomic<long long> g_launches{0};
static std::mutex g_prof_mu;
static std::atomic<bool> g_prof{false};  // read by every phase scope, on any thread
struct PhaseRec {
  std::string name;
  cudaEvent_t a, b;
};
static std::vector<PhaseRec> g_recs;

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

PhaseScope::PhaseScope(const char* n, cudaStream_t s) : name(n), st(s) {
  if (!g_prof) return;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    a = b = nullptr;
    return;
  }
  cudaEventRecord(a, st);
}

PhaseScope::~PhaseScope() {
  if (!a) return;
  cudaEventRecord(b, st);
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_recs.push_back(PhaseRec{name, a, b});
}

static void init_pool_once() {
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;  // keep freed blocks cached in the pool
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  });
}

ctd_status allow_max_smem(const void* fn) {
  static std::mutex mu;
  static std::set<std::pair<int, const void*>> done;
  int dev = 0;
  CTD_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if (done.count({dev, fn})) return CTD_OK;
  int optin = 0;
  CTD_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa{};
  CTD_CUDA(cudaFuncGetAttributes(&fa, fn));  // static shared memory counts against the limit
  CTD_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes));
  done.insert({dev, fn});
  return CTD_OK;
}

// Fault injection for tests (ctd_fault_inject_alloc): after this many more
// successful device allocations every allocation fails with CTD_ENOMEM;
// -1 disables.
static std::atomic<long long> g_alloc_fail_after{-1};

// The allocator hook (ctd_set_allocator) and the library's live device
// bytes.  Every live allocation is recorded with its size and the release
// function of the hook that made it (none: the library's pool), so a block
// goes back to whoever made it even if the hook changes in between, and
// live_bytes() counts what the library holds.
namespace {
struct AllocHook {
  ctd_alloc_fn alloc = nullptr;
  ctd_release_fn release = nullptr;
};
struct LiveBlock {
  size_t bytes;
  ctd_release_fn release;
};
std::mutex g_hook_mu;
AllocHook g_hook;
std::unordered_map<void*, LiveBlock> g_live;
size_t g_live_bytes = 0;
}  // namespace

size_t live_bytes() {
  std::lock_guard<std::mutex> lk(g_hook_mu);
  return g_live_bytes;
}

bool allocator_hooked() {
  std::lock_guard<std::mutex> lk(g_hook_mu);
  return g_hook.alloc != nullptr;
}

ctd_status dalloc(void** p, size_t bytes, cudaStream_t st) {
  const long long fa = g_alloc_fail_after.load();
  if (fa >= 0) {
    if (fa == 0) {
      *p = nullptr;
      return fail(CTD_ENOMEM, "device allocation refused (fault injection)");
    }
    g_alloc_fail_after.fetch_sub(1);
  }
  const size_t nb = bytes ? bytes : 1;
  AllocHook h;
  {
    std::lock_guard<std::mutex> lk(g_hook_mu);
    h = g_hook;
  }
  if (h.alloc) {
    *p = h.alloc(nb, st);
    if (!*p)
      return fail(CTD_ENOMEM, std::string("device allocation of ") + std::to_string(bytes) +
                                  " bytes refused by the allocator hook");
  } else {
    init_pool_once();
    cudaError_t e = cudaMallocAsync(p, nb, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      return fail(CTD_ENOMEM, std::string("device allocation of ") + std::to_string(bytes) +
                                  " bytes failed: " + cudaGetErrorString(e));
    }
  }
  std::lock_guard<std::mutex> lk(g_hook_mu);
  g_live[*p] = LiveBlock{nb, h.alloc ? h.release : nullptr};
  g_live_bytes += nb;
  return CTD_OK;
}

void dfree(void* p, cudaStream_t st) {
  if (!p) return;
  ctd_release_fn rel = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_hook_mu);
    auto it = g_live.find(p);
    if (it != g_live.end()) {
      rel = it->second.release;
      g_live_bytes -= it->second.bytes;
      g_live.erase(it);
    }
  }
  if (rel)
    rel(p, st);
  else
    cudaFreeAsync(p, st);
}

ctd_status d2h_bytes(void* host, const void* dev, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return CTD_OK;
  CTD_CUDA(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, st));
  return CTD_OK;
}

ctd_status sync(cudaStream_t st) {
  CTD_CUDA(cudaStreamSynchronize(st));
  return CTD_OK;
}

namespace {
struct TuneSpec {
  const char* key;
  int64_t def, lo, hi;
};
constexpr TuneSpec kTune[TUNE_N] = {{"qform_hot_kb", 200, 0, 200},
                                    {"cfill_dense_kb", 220, 64, 220},
                                    {"copy_blocks_per_sm", 8, 1, 32}};
std::atomic<int64_t> g_tune[TUNE_N] = {{200}, {220}, {8}};
int tune_index(const char* key) {
  if (!key) return -1;
  for (int k = 0; k < TUNE_N; ++k)
    if (std::strcmp(kTune[k].key, key) == 0) return k;
  return -1;
}
}  // namespace

int64_t tuning(TuneKey k) { return g_tune[k].load(std::memory_order_relaxed); }

namespace {
thread_local SideStream t_side;
}

SideStream::~SideStream() {
  // at thread exit; errors (a runtime already shut down) are of no use here
  if (ev_fork) cudaEventDestroy(ev_fork);
  if (ev_join) cudaEventDestroy(ev_join);
  if (st) cudaStreamDestroy(st);
}

ctd_status SideStream::fork(cudaStream_t main) {
  CTD_CUDA(cudaEventRecord(ev_fork, main));
  CTD_CUDA(cudaStreamWaitEvent(st, ev_fork, 0));
  return CTD_OK;
}

ctd_status SideStream::join(cudaStream_t main) {
  CTD_CUDA(cudaEventRecord(ev_join, st));
  CTD_CUDA(cudaStreamWaitEvent(main, ev_join, 0));
  return CTD_OK;
}

ctd_status side_stream(SideStream** out) {
  int dev = 0;
  CTD_CUDA(cudaGetDevice(&dev));
  SideStream& s = t_side;
  if (s.dev != dev) {
    if (s.ev_fork) cudaEventDestroy(s.ev_fork);
    if (s.ev_join) cudaEventDestroy(s.ev_join);
    if (s.st) cudaStreamDestroy(s.st);
    s = SideStream();
    CTD_CUDA(cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking));
    CTD_CUDA(cudaEventCreateWithFlags(&s.ev_fork, cudaEventDisableTiming));
    CTD_CUDA(cudaEventCreateWithFlags(&s.ev_join, cudaEventDisableTiming));
    s.dev = dev;
  }
  *out = &s;
  return CTD_OK;
}

// ---------------------------------------------------------------------------
// batched small read-backs through pinned staging
// ---------------------------------------------------------------------------
namespace {
constexpr size_t RB_CHUNK = 1 << 20;
struct PinnedPool {
  std::vector<char*> free_chunks;
  ~PinnedPool() {
    for (char* c : free_chunks) cudaFreeHost(c);
  }
};
thread_local PinnedPool t_pinned;
}  // namespace

Readback::Readback(cudaStream_t s) : st(s) {
  if (!t_pinned.free_chunks.empty()) {
    chunk = t_pinned.free_chunks.back();
    t_pinned.free_chunks.pop_back();
  } else if (cudaMallocHost(reinterpret_cast<void**>(&chunk), RB_CHUNK) != cudaSuccess) {
    cudaGetLastError();
    chunk = nullptr;  // direct copies only
  }
}

Readback::~Readback() {
  // copies still in flight into the chunk must land before it is reused
  if (!items.empty()) cudaStreamSynchronize(st);
  if (chunk) t_pinned.free_chunks.push_back(chunk);
  if (ev) cudaEventDestroy(ev);
}

ctd_status Readback::mark() {
  if (!ev) CTD_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  CTD_CUDA(cudaEventRecord(ev, st));
  return CTD_OK;
}

ctd_status Readback::wait_mark() {
  if (!ev) return wait();
  CTD_CUDA(cudaEventSynchronize(ev));
  for (const Item& it : items) std::memcpy(it.host, chunk + it.off, it.bytes);
  items.clear();
  used = 0;
  return CTD_OK;
}

ctd_status Readback::add_bytes(void* host, const void* dev, size_t bytes) {
  if (bytes == 0) return CTD_OK;
  const size_t need = (bytes + 15) & ~size_t(15);
  if (!chunk || bytes > RB_CHUNK) return d2h_bytes(host, dev, bytes, st);  // synchronous copy
  if (used + need > RB_CHUNK) CTD_TRY(wait());
  CTD_CUDA(cudaMemcpyAsync(chunk + used, dev, bytes, cudaMemcpyDeviceToHost, st));
  items.push_back({host, used, bytes});
  used += need;
  return CTD_OK;
}

ctd_status Readback::wait() {
  CTD_CUDA(cudaStreamSynchronize(st));
  for (const Item& it : items) std::memcpy(it.host, chunk + it.off, it.bytes);
  items.clear();
  used = 0;
  return CTD_OK;
}

// Validate a COO descriptor; produce device views (copying host inputs in).
ctd_status stage_coo(const ctd_coo3* X, int alpha, Arena& scratch, cudaStream_t st, CooDev* out) {
  if (!X) return fail(CTD_EINVAL, "tensor descriptor is NULL");
  if (alpha < 1 || alpha > 3) return fail(CTD_EINVAL, "alpha must be 1, 2 or 3");
  for (int d = 0; d < 3; ++d)
    if (X->dims[d] < 1 || X->dims[d] > INT32_MAX)
      return fail(CTD_EINVAL, "each dimension must be in [1, 2^31)");
  if (X->nnz < 0 || X->nnz > INT32_MAX) return fail(CTD_EINVAL, "nnz must be in [0, 2^31)");
  if (X->nnz > 0 && (!X->i || !X->j || !X->k || !X->val))
    return fail(CTD_EINVAL, "index or value pointer is NULL");
  if (X->memory != CTD_MEM_DEVICE && X->memory != CTD_MEM_HOST)
    return fail(CTD_EINVAL, "unknown memory kind");
  int64_t n_rows, n_cols;
  mode_extents(X->dims, alpha, &n_rows, &n_cols);
  if (n_cols > INT32_MAX) return fail(CTD_EINVAL, "N_alpha must be < 2^31");
  CooDev c;
  c.nnz = X->nnz;
  c.alpha = alpha;
  for (int d = 0; d < 3; ++d) c.dims[d] = X->dims[d];
  if (X->memory == CTD_MEM_HOST && X->nnz > 0) {
    // each array starts on a 16-byte boundary (the streaming kernels read
    // four entries per load when all four do)
    const int64_t ld = (X->nnz + 3) & ~(int64_t)3;
    int32_t* buf;
    CTD_TRY(scratch.get(&buf, 4 * (size_t)ld));
    const int32_t* src[4] = {X->i, X->j, X->k, X->val};
    for (int a = 0; a < 4; ++a)
      CTD_CUDA(cudaMemcpyAsync(buf + a * ld, src[a], X->nnz * sizeof(int32_t),
                               cudaMemcpyHostToDevice, st));
    c.i = buf;
    c.j = buf + ld;
    c.k = buf + 2 * ld;
    c.v = buf + 3 * ld;
  } else {
    c.i = X->i;
    c.j = X->j;
    c.k = X->k;
    c.v = X->val;
  }
  *out = c;
  return CTD_OK;
}

// Algorithm 1's matricization and squared norms (and the layout later steps
// read): count entries per column, scan the counts into column offsets (the
// scan also leaves each column's u32 cursor in the count array), scatter the
// entries, then the squared column norms as a segmented sum over each
// column's contiguous entries, fused with the first pass of their prefix
// sum (the CDF).
ctd_status matricize(const CooDev& X, Arena& A, cudaStream_t st, Matricized* M, bool sort_cols,
                     Arena* dist, int wshift) {
  mode_extents(X.dims, X.alpha, &M->n_rows, &M->n_cols);
  M->nnz = X.nnz;
  Arena& D = dist ? *dist : A;
  uint32_t* rowcnt;
  CTD_TRY(A.get(&rowcnt, M->n_rows));
  M->rowcnt = rowcnt;
  CTD_TRY(D.get(&M->norm2, M->n_cols));
  CTD_TRY(D.get(&M->cdf, M->n_cols));
  CTD_TRY(A.get(&M->colptr, M->n_cols + 1));
  CTD_TRY(A.get(&M->csc_row, X.nnz));
  CTD_TRY(A.get(&M->csc_val, X.nnz));
  CTD_TRY(A.get(&M->minval, 2));
  CTD_TRY(A.get(&M->status, 1));
  CTD_TRY(A.get(&M->tmp, scan_tmp_elems(std::max(M->n_cols, M->n_rows) + 1)));
  CTD_CUDA(cudaMemsetAsync(rowcnt, 0, M->n_rows * 4, st));
  CTD_CUDA(cudaMemsetAsync(M->status, 0, 4, st));
  CTD_CUDA(cudaMemsetAsync(M->minval, 0xff, 8, st));  // codes of "no value yet"
  bool bucketed = false;
  CTD_TRY(matricize_bucketed(X, A, st, M, &bucketed, wshift));
  if (!bucketed) {
    uint32_t* colcnt;
    CTD_TRY(A.get(&colcnt, M->n_cols));
    CTD_CUDA(cudaMemsetAsync(colcnt, 0, M->n_cols * 4, st));
    launch_count(X, colcnt, rowcnt, M->status, st);
    // column offsets; colcnt becomes each column's cursor (its first position)
    launch_scan_u32(colcnt, M->colptr, M->n_cols, false, M->tmp, M->status, st, colcnt);
    launch_coo_scatter(X, colcnt, M->csc_row, M->csc_val, st);
  }
  if (sort_cols) {
    // one entry order per column, whatever order the scatter's atomics took;
    // the CDF array is not written yet and serves as the sort's scratch when
    // it is long enough (the squared norms are exact in any order)
    uint64_t* keys = M->cdf;
    if (M->n_cols < X.nnz) CTD_TRY(A.get(&keys, X.nnz));
    CTD_TRY(launch_sort_cols(M->colptr, M->n_cols, X.nnz, M->csc_row, M->csc_val, keys, A, st));
  }
  if (bucketed)
    launch_scan_finish(M->norm2, M->cdf, M->n_cols, M->tmp, M->status, st);
  else
    launch_sqnorms_cdf(M->colptr, M->csc_val, M->n_cols, M->norm2, M->cdf, M->minval, M->tmp,
                       M->status, st, wshift);
  CTD_CUDA(cudaGetLastError());
  return CTD_OK;
}

}  // namespace ctd

using namespace ctd;

// kpos[idx[p]] = p: the place of each kept candidate among the kept ones
__global__ void k_kept_positions(const int* __restrict__ idx, int kept, int* __restrict__ kpos) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < kept; p += gridDim.x * blockDim.x)
    kpos[idx[p]] = p;
}

// *out = max |val[e]| over the first *count entries (out zeroed beforehand)
__global__ void k_abs_max(const int32_t* __restrict__ val, const uint64_t* __restrict__ count,
                          int* __restrict__ out) {
  const int64_t n = (int64_t)*count;
  int m = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int v = val[e];
    m = max(m, v == INT32_MIN ? INT32_MAX : abs(v));
  }
  for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// ---------------------------------------------------------------------------
// CTD-S
// ---------------------------------------------------------------------------
extern "C" ctd_status ctd_static(const ctd_coo3* Xd, int alpha, int64_t s, double eps,
                                 uint64_t seed, int precision, unsigned flags, void* stream,
                                 ctd_factors** out) {
  if (!out) return fail(CTD_EINVAL, "out is NULL");
  if (s < 1 || s > 8192) return fail(CTD_EINVAL, "s must be in [1, 8192]");
  if (!(eps >= 0.0 && eps < 1.0)) return fail(CTD_EINVAL, "eps must be in [0, 1)");
  if (precision != CTD_FP64 && precision != CTD_FP32_BULK)
    return fail(CTD_EINVAL, "unknown precision");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  PhaseScope ph_call("call", st);  // the whole call; the named phases below sit inside it
  Arena scratch;
  scratch.st = st;
  CooDev X;
  {
    PhaseScope ph("stage", st);
    CTD_TRY(stage_coo(Xd, alpha, scratch, st, &X));
  }
  return static_impl(X, s, eps, seed, precision, flags, st, scratch, 0, out);
}

namespace ctd {
// Algorithm 1 on a staged tensor (device COO, mode and dims in X); real:
// the values' payloads hold FP32 values.
ctd_status static_impl(const CooDev& X, int64_t s, double eps, uint64_t seed, int precision,
                       unsigned flags, cudaStream_t st, Arena& scratch, int real,
                       ctd_factors** out) {
  const int alpha = X.alpha;
  int wshift = WSHIFT_INT;
  if (real) CTD_TRY(real_weight_shift(X.v, X.nnz, &wshift, scratch, st));

  ctd_factors* F = new ctd_factors();
  F->real = real != 0;
  F->mem.st = st;
  F->kind = 0;
  F->alpha = alpha;
  F->precision = precision;
  F->stream = st;
  F->seed = seed;
  for (int d = 0; d < 3; ++d) F->dims[d] = X.dims[d];
  F->nnz_X = X.nnz;
  F->s = s;
  // the error's stream (set once it has work queued)
  SideStream* side = nullptr;
  auto bail = [&](ctd_status rc) {
    cudaStreamSynchronize(st);
    if (side) cudaStreamSynchronize(side->st);
    delete F;
    return rc;
  };
#define STEP(expr)                     \
  do {                                 \
    ctd_status _r = (expr);            \
    if (_r != CTD_OK) return bail(_r); \
  } while (0)
#define STEPC(call)                                                                   \
  do {                                                                                \
    cudaError_t _e = (call);                                                          \
    if (_e != cudaSuccess)                                                            \
      return bail(fail(CTD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(_e))); \
  } while (0)

  // matricization and squared norms
  Matricized M;
  {
    PhaseScope ph("matricize", st);
    STEP(matricize(X, scratch, st, &M, (flags & CTD_DETERMINISTIC) != 0,
                   (flags & CTD_KEEP_DIST) ? &F->mem : nullptr, wshift));
  }
  if (flags & CTD_KEEP_DIST) {
    F->norm2 = M.norm2;
    F->cdf = M.cdf;
  }
  F->n_rows = M.n_rows;
  F->n_cols = M.n_cols;
  // draws, then their unique set
  STEP(F->mem.get(&F->I, s));
  STEP(F->mem.get(&F->Iu, s));
  int* d_count;
  STEP(scratch.get(&d_count, 4));
  {
    PhaseScope ph("sample_unique", st);
    launch_sample(M.cdf, M.n_cols, s, seed, 0, 0, F->I, st);
    launch_sort_unique(F->I, s, F->Iu, d_count, st);
  }
  // candidate column sizes from the device count (entries past it are zero),
  // so one read-back gives T, s' and nnz(R') together
  std::unique_ptr<PhaseScope> ph_cand(new PhaseScope("candidates", st));
  uint64_t *rc_ptr, *rc_sizes;
  STEP(scratch.get(&rc_sizes, s + 1));
  STEP(scratch.get(&rc_ptr, s + 1));
  launch_column_sizes(M.colptr, F->Iu, d_count, (int)s, rc_sizes, st);
  launch_scan_u64(rc_sizes, rc_ptr, s, false, M.tmp, M.status, st);
  STEPC(cudaGetLastError());
  unsigned status = 0;
  unsigned minkey[2] = {0, 0};
  int s_unique = 0;
  uint64_t T = 0, nnz_cand = 0;
  {
    Readback rb(st);
    STEP(rb.add(&status, M.status, 1));
    STEP(rb.add(minkey, M.minval, 2));
    STEP(rb.add(&s_unique, d_count, 1));
    STEP(rb.add(&nnz_cand, rc_ptr + s, 1));
    if (M.n_cols > 0) STEP(rb.add(&T, M.cdf + (M.n_cols - 1), 1));
    STEP(rb.wait());
  }
  STEP(status_from_device(status));
  F->T = T;
  // integer counts: the smallest value (all positive: the C fill copies R's
  // rows for one-nonzero columns) and whether they fit int8 (four products
  // per instruction); neither applies to real values
  const int minval = real ? 0 : decode_min(minkey[0]);
  const bool x_int8 = !real && minval >= -128 && decode_max(minkey[1]) <= 127;
  F->min_val = minval;
  F->s_unique = s_unique;
  if (T == 0) F->s = 0;  // nothing to draw from
  const int su = s_unique;

  int32_t *rc_row, *rc_val, *rcr_col, *rcr_val;
  uint64_t* rcr_ptr;
  STEP(scratch.get(&rc_row, nnz_cand));
  STEP(scratch.get(&rc_val, nnz_cand));
  STEP(scratch.get(&rcr_col, nnz_cand));
  STEP(scratch.get(&rcr_val, nnz_cand));
  STEP(scratch.get(&rcr_ptr, M.n_rows + 1));
  launch_gather_columns(M.colptr, M.csc_row, M.csc_val, F->Iu, d_count, su, rc_ptr, rc_row,
                        rc_val, st);
  // rows of each gathered column in ascending order, so every floating-point
  // sum over a candidate's entries is reproducible
  launch_sort_segments(rc_ptr, su, rc_row, rc_val, rcr_col, rcr_val, M.n_rows, st);
  STEP(build_csr_from_csc(rc_ptr, rc_row, rc_val, su, nnz_cand, M.n_rows, 0, rcr_ptr, rcr_col,
                          rcr_val, scratch, st));

  ph_cand.reset();
  // independence test: Gram matrix, in-order Cholesky with skip (+ explicit re-test)
  double *G, *xn2;
  STEP(scratch.get(&G, (size_t)su * su));
  STEP(scratch.get(&xn2, su));
  CsrDev Rc{rcr_ptr, rcr_col, rcr_val, su};
  {
    PhaseScope ph("gram", st);
    if (real)
      STEP(real_gram(rc_ptr, rc_row, rc_val, d_count, su, M.n_rows, G, scratch, st));
    else
      STEP(launch_spmm_dense(M.csc(), F->Iu, d_count, su, Rc, G, su, st, &scratch));
    launch_thresholds(G, su, su, 1.0, xn2, st);
  }
  FilterIn fi;
  fi.du = su;
  fi.S = G;
  fi.xnorm2 = xn2;
  fi.eps = eps;
  fi.cptr = rc_ptr;
  fi.crow = rc_row;
  fi.cval = rc_val;
  fi.c_rowptr = rcr_ptr;
  fi.c_col = rcr_col;
  fi.c_val = rcr_val;
  fi.n_rows = M.n_rows;
  fi.real = real;
  FilterOut fo;
  STEP(run_filter(fi, fo, scratch, st));
  const int kept = fo.kept;
  int* idx = fo.idx;
  F->s_kept = kept;

  // U = (R^T R)^{-1} = L^{-T} L^{-1}: an output only, so it is formed on
  // the second stream (below) beside R's build and C's fill
  double* Z = fo.Li;
  STEP(F->mem.get(&F->U, (size_t)kept * kept));
  if (kept > 0) {
    SideStream* ss = nullptr;
    STEP(side_stream(&ss));
    STEP(ss->fork(st));
    side = ss;
    PhaseScope ph("u_inverse", side->st);
    u_from_linv(Z, kept, kept, F->U, kept, side->st);
  }

  // R: kept columns of R', CSC and row-major
  std::unique_ptr<PhaseScope> ph_r(new PhaseScope("r_build", st));
  STEP(F->mem.get(&F->kept_pos, kept));
  STEP(F->mem.get(&F->fibers, kept));
  STEPC(cudaMemcpyAsync(F->kept_pos, idx, kept * sizeof(int), cudaMemcpyDeviceToDevice, st));
  launch_gather_i64(F->Iu, idx, fo.count, kept, F->fibers, st);
  uint64_t* r_sizes;
  STEP(scratch.get(&r_sizes, kept + 1));
  STEP(F->mem.get(&F->Rcolptr, kept + 1));
  launch_column_sizes(M.colptr, F->fibers, fo.count, kept, r_sizes, st);
  launch_scan_u64(r_sizes, F->Rcolptr, kept, false, M.tmp, M.status, st);
  // nnz(R) <= nnz(R'): size R by that bound and read nnz(R) at the next read-back
  const uint64_t nnzR_cap = std::max<uint64_t>(nnz_cand, 1);
  STEP(F->mem.get(&F->Rrow, nnzR_cap));
  STEP(F->mem.get(&F->Rval, nnzR_cap));
  STEP(F->mem.get(&F->Rrowptr, M.n_rows + 1));
  STEP(F->mem.get(&F->Rcol, nnzR_cap));
  STEP(F->mem.get(&F->Rcval, nnzR_cap));
  launch_gather_columns(M.colptr, M.csc_row, M.csc_val, F->fibers, fo.count, kept, F->Rcolptr,
                        F->Rrow, F->Rval, st);
  // R by row: the rows of R' (sorted by candidate) restricted to the kept
  // candidates, each renumbered to its place among them
  int* kpos;
  STEP(scratch.get(&kpos, std::max(su, 1)));
  STEPC(cudaMemsetAsync(kpos, 0xff, (size_t)std::max(su, 1) * sizeof(int), st));  // -1
  if (kept > 0)
    CTD_LAUNCH(k_kept_positions, (grid_for(kept, 256, 64)), (256), 0, st, idx, kept, kpos);
  STEP(csr_keep_columns(rcr_ptr, rcr_col, rcr_val, M.n_rows, kpos, F->Rrowptr, F->Rcol,
                        F->Rcval, scratch, st));
  CsrDev R{F->Rrowptr, F->Rcol, F->Rcval, kept};
  ph_r.reset();

  // Eq. (error): e = (T - ||Q^T X||_F^2) / T with Q = R L^{-T}.  It needs
  // neither C nor C's capacity, so it runs on the second stream beside the
  // read-back of that capacity and C's fill; the main stream joins that
  // stream before the final read-back.
  double* d_pu = nullptr;
  Arena side_scratch;
  if (!(flags & CTD_SKIP_ERROR) && kept > 0) {
    STEP(scratch.get(&d_pu, 1));
    STEP(side->fork(st));  // after R
    side_scratch.st = side->st;
    PhaseScope ph("error_qform", side->st);
    if (real)
      STEP(real_error_qform(M.csc(), M.n_cols, M.n_rows, F->Rcolptr, F->Rrow, F->Rval, kept, Z,
                            kept, d_pu, side_scratch, side->st));
    else
      STEP(launch_error_qform(M.csc(), M.n_cols, M.n_rows, M.nnz, R, Z, kept, M.rowcnt,
                              precision == CTD_FP32_BULK, d_pu, side_scratch, side->st));
  }

  // C = R^T X_(alpha)
  Readback rbc(st);
  uint64_t cap = 0, nnzR = 0;
  int rmax = -1;
  int* d_rmax = nullptr;
  // the C fill's column lists come out of the C bounds' pass when the fill
  // takes its dense-row path (integer values, exact int32 partial sums,
  // at most 1024 kept fibers)
  CfillLists lists;
  const bool fused_lists = !real && T < (1ull << 31) && kept <= 1024;
  if (!(flags & CTD_SKIP_C)) {
    uint32_t* ub;
    STEP(scratch.get(&ub, M.n_cols));
    STEP(F->mem.get(&F->Coff, M.n_cols + 1));
    STEP(F->mem.get(&F->Ccnt, M.n_cols));
    if (fused_lists) {
      const int64_t list_cap = std::max<int64_t>(1, std::min<int64_t>(M.n_cols, M.nnz));
      STEP(scratch.get(&lists.single, list_cap));
      STEP(scratch.get(&lists.heavy, list_cap));
      STEP(scratch.get(&lists.multi, list_cap));
      STEP(scratch.get(&lists.counts, 3));
    }
    {
      PhaseScope ph("c_bounds", st);
      if (fused_lists)
        STEP(launch_c_bounds_lists(M.csc(), M.n_cols, R, ub, minval > 0, F->Ccnt, lists, st));
      else
        launch_c_bounds(M.csc(), M.n_cols, R, ub, st);
      launch_scan_u32(ub, F->Coff, M.n_cols, false, M.tmp, M.status, st);
    }
    // largest |R| (the C fill stores its longest rows as int16 when they fit)
    STEP(scratch.get(&d_rmax, 1));
    STEPC(cudaMemsetAsync(d_rmax, 0, sizeof(int), st));
    if (!real)
      CTD_LAUNCH(k_abs_max, (grid_for((int64_t)nnzR_cap, 256, (int64_t)num_sms() * 4)), (256), 0,
                 st, F->Rval, F->Rcolptr + kept, d_rmax);
    STEP(rbc.add(&cap, F->Coff + M.n_cols, 1));
    STEP(rbc.add(&nnzR, F->Rcolptr + kept, 1));
    STEP(rbc.add(&rmax, (const int*)d_rmax, 1));
    STEP(rbc.mark());
  }
  double* d_sq = nullptr;  // real values: ||X||_F^2 in FP64
  if (real) {
    STEP(scratch.get(&d_sq, 1));
    STEP(real_sqnorm(M.csc_val, M.nnz, d_sq, scratch, st));
  }
  if (!(flags & CTD_SKIP_C)) {
    STEP(rbc.wait_mark());
    F->nnz_R = (int64_t)nnzR;
    R.nnz = F->nnz_R;
    R.max_abs = rmax;
    F->C_cap = cap;
    STEP(F->mem.get(&F->Crow, cap));
    const size_t vsz = precision == CTD_FP32_BULK ? 4 : 8;
    void* cv = nullptr;
    STEP(dalloc(&cv, (cap ? cap : 1) * vsz, st));
    F->mem.ptrs.push_back(cv);
    F->Cval = cv;
    PhaseScope ph("c_fill", st);
    if (real)
      STEP(real_c_fill(M.csc(), M.n_cols, R, F->Coff, F->Ccnt, F->Crow, F->Cval,
                       precision == CTD_FP32_BULK, st));
    else
      STEP(launch_c_fill(M.csc(), M.n_cols, M.n_rows, M.nnz, R, F->Coff, F->Ccnt, F->Crow,
                         F->Cval, precision == CTD_FP32_BULK, minval > 0, x_int8, T, st,
                         fused_lists ? &lists : nullptr));
  }
  uint64_t* d_nnzc;
  STEP(scratch.get(&d_nnzc, 1));
  if (F->Ccnt) launch_sum_u32(F->Ccnt, M.n_cols, d_nnzc, st, C_COUNT);
  uint64_t nnzC = 0, nnzR_final = 0;
  double pu = 0.0;
  if (side) STEP(side->join(st));
  {
    Readback rb(st);
    STEP(rb.add(&nnzR_final, F->Rcolptr + kept, 1));
    if (F->Ccnt) STEP(rb.add(&nnzC, d_nnzc, 1));
    if (d_pu) STEP(rb.add(&pu, d_pu, 1));
    if (d_sq) STEP(rb.add(&F->sqnorm_real, d_sq, 1));
    STEP(rb.add(&status, M.status, 1));
    STEPC(cudaGetLastError());
    STEP(rb.wait());
  }
  STEP(status_from_device(status));
  F->nnz_C = (int64_t)nnzC;
  F->nnz_R = (int64_t)nnzR_final;
  if (!(flags & CTD_SKIP_ERROR)) {
    F->have_err = true;
    const double tot = real ? F->sqnorm_real : (double)T;
    F->err = tot > 0.0 ? std::max(0.0, (tot - pu) / tot) : 0.0;
  }
  *out = F;
#undef STEP
#undef STEPC
  return CTD_OK;
}
}  // namespace ctd

// ---------------------------------------------------------------------------
// getters
// ---------------------------------------------------------------------------
extern "C" ctd_status ctd_error(const ctd_factors* F, double* rel_err) {
  if (!F || !rel_err) return fail(CTD_EINVAL, "NULL argument");
  if (!F->have_err) return fail(CTD_EINVAL, "the error was not computed (CTD_SKIP_ERROR)");
  *rel_err = F->err;
  return CTD_OK;
}

extern "C" ctd_status ctd_get_sizes(const ctd_factors* F, ctd_sizes* o) {
  if (!F || !o) return fail(CTD_EINVAL, "NULL argument");
  CTD_TRY(sync(F->stream));
  if (F->kind == 1) return dyn_sizes(F, o);
  o->n_rows = F->n_rows;
  o->n_cols = F->n_cols;
  o->s_draws = F->s;
  o->s_unique = F->s_unique;
  o->s_kept = F->s_kept;
  o->nnz_R = F->nnz_R;
  o->nnz_C = F->nnz_C;
  o->t_steps = 0;
  o->nnz_X = F->nnz_X;
  o->sqnorm_X = F->real ? F->sqnorm_real : (double)F->T;
  return CTD_OK;
}

extern "C" ctd_status ctd_get_samples(const ctd_factors* F, int64_t* I, int64_t* Iu) {
  if (!F) return fail(CTD_EINVAL, "NULL argument");
  if (F->kind == 1) return dyn_samples(F, I, Iu);
  if (I) CTD_TRY(d2h(I, F->I, (size_t)F->s, F->stream));
  if (Iu) CTD_TRY(d2h(Iu, F->Iu, (size_t)F->s_unique, F->stream));
  return sync(F->stream);
}

extern "C" ctd_status ctd_get_column_dist(const ctd_factors* F, uint64_t* norm2, uint64_t* cdf) {
  if (!F) return fail(CTD_EINVAL, "NULL argument");
  if (F->kind != 0) return fail(CTD_EINVAL, "the column distribution is kept for CTD-S only");
  if (!F->cdf) return fail(CTD_EINVAL, "factors were made without CTD_KEEP_DIST");
  if (norm2) CTD_TRY(d2h(norm2, F->norm2, (size_t)F->n_cols, F->stream));
  if (cdf) CTD_TRY(d2h(cdf, F->cdf, (size_t)F->n_cols, F->stream));
  return sync(F->stream);
}

extern "C" ctd_status ctd_get_fibers(const ctd_factors* F, int64_t* fiber, int64_t* step) {
  if (!F) return fail(CTD_EINVAL, "NULL argument");
  if (F->kind == 1) return dyn_fibers(F, fiber, step);
  if (fiber) CTD_TRY(d2h(fiber, F->fibers, (size_t)F->s_kept, F->stream));
  CTD_TRY(sync(F->stream));
  if (step)
    for (int64_t c = 0; c < F->s_kept; ++c) step[c] = 0;
  return CTD_OK;
}

// Copy a device CSC (s~ columns) to host and sort rows within columns.
static ctd_status csc_to_host_sorted(const uint64_t* dptr, const int32_t* drow, const int32_t* dval,
                                     int64_t ncols, int64_t nnz, cudaStream_t st,
                                     int64_t* colptr, int32_t* row, int32_t* val) {
  std::vector<uint64_t> p(ncols + 1);
  std::vector<int32_t> r(nnz), v(nnz);
  CTD_TRY(d2h(p.data(), dptr, ncols + 1, st));
  CTD_TRY(d2h(r.data(), drow, nnz, st));
  CTD_TRY(d2h(v.data(), dval, nnz, st));
  CTD_TRY(sync(st));
  std::vector<int64_t> ord;
  for (int64_t c = 0; c < ncols; ++c) {
    const int64_t a = (int64_t)p[c], b = (int64_t)p[c + 1];
    ord.resize(b - a);
    std::iota(ord.begin(), ord.end(), a);
    std::sort(ord.begin(), ord.end(), [&](int64_t x, int64_t y) { return r[x] < r[y]; });
    for (int64_t q = a; q < b; ++q) {
      row[q] = r[ord[q - a]];
      val[q] = v[ord[q - a]];
    }
    colptr[c] = a;
  }
  colptr[ncols] = (int64_t)p[ncols];
  return CTD_OK;
}

extern "C" ctd_status ctd_get_R(const ctd_factors* F, int64_t* colptr, int32_t* row,
                                int32_t* val) {
  if (!F || !colptr || (F->nnz_R && (!row || !val))) return fail(CTD_EINVAL, "NULL argument");
  return guarded([&] {
    if (F->kind == 1) return dyn_R(F, colptr, row, val);
    return csc_to_host_sorted(F->Rcolptr, F->Rrow, F->Rval, F->s_kept, F->nnz_R, F->stream,
                              colptr, row, val);
  });
}

extern "C" ctd_status ctd_get_R_f64(const ctd_factors* F, int64_t* colptr, int32_t* row,
                                    double* val) {
  if (!F || !colptr || (F->nnz_R && (!row || !val))) return fail(CTD_EINVAL, "NULL argument");
  return guarded([&]() -> ctd_status {
    std::vector<int32_t> bits((size_t)std::max<int64_t>(F->nnz_R, 1));
    CTD_TRY(ctd_get_R(F, colptr, row, bits.data()));
    for (int64_t q = 0; q < F->nnz_R; ++q) {
      if (F->real) {
        float x;
        std::memcpy(&x, &bits[q], sizeof(float));
        val[q] = x;
      } else {
        val[q] = bits[q];
      }
    }
    return CTD_OK;
  });
}

extern "C" ctd_status ctd_get_U(const ctd_factors* F, double* U) {
  if (!F || (!U && F->s_kept)) return fail(CTD_EINVAL, "NULL argument");
  if (F->kind == 1) return dyn_U(F, U);
  CTD_TRY(d2h(U, F->U, (size_t)F->s_kept * F->s_kept, F->stream));
  return sync(F->stream);
}

namespace ctd {
template <typename V>
__global__ void k_c_columns(const unsigned long long* __restrict__ coff,
                            const unsigned* __restrict__ ccnt, const uint16_t* __restrict__ crow,
                            const V* __restrict__ cval, const int64_t* __restrict__ cols,
                            int64_t ncols, int64_t height, double* __restrict__ out) {
  for (int64_t c = blockIdx.x; c < ncols; c += gridDim.x) {
    const int64_t f = cols[c];
    const unsigned long long o = coff[f];
    const unsigned n = ccnt[f];
    if (n & C_DENSE) {
      for (int64_t m = threadIdx.x; m < height; m += blockDim.x)
        out[c * height + m] = (double)cval[o + m];
    } else {
      for (unsigned q = threadIdx.x; q < n; q += blockDim.x)
        out[c * height + crow[o + q]] = (double)cval[o + q];
    }
  }
}
}  // namespace ctd

extern "C" ctd_status ctd_get_C_columns(const ctd_factors* F, int64_t ncols, const int64_t* cols,
                                        double* out) {
  if (!F || ncols < 0 || (ncols && (!cols || !out))) return fail(CTD_EINVAL, "NULL argument");
  if (F->kind == 1) return guarded([&] { return dyn_C_columns(F, ncols, cols, out); });
  if (!F->Coff) return fail(CTD_EINVAL, "C was not materialized (CTD_SKIP_C)");
  for (int64_t c = 0; c < ncols; ++c)
    if (cols[c] < 0 || cols[c] >= F->n_cols) return fail(CTD_EINVAL, "column out of range");
  const int64_t h = F->s_kept;
  if (ncols == 0 || h == 0) {
    std::fill(out, out + ncols * h, 0.0);
    return CTD_OK;
  }
  cudaStream_t st = F->stream;
  Arena a;
  a.st = st;
  int64_t* dcols;
  double* dout;
  CTD_TRY(a.get(&dcols, ncols));
  CTD_TRY(a.get(&dout, (size_t)ncols * h));
  CTD_CUDA(cudaMemcpyAsync(dcols, cols, ncols * 8, cudaMemcpyHostToDevice, st));
  CTD_CUDA(cudaMemsetAsync(dout, 0, (size_t)ncols * h * 8, st));
  const unsigned g = grid_for(ncols, 1, 4096);
  if (F->precision == CTD_FP32_BULK)
    CTD_LAUNCH(k_c_columns<float>, (g), (128), 0, st, reinterpret_cast<const unsigned long long*>(F->Coff),
                                          F->Ccnt, F->Crow, static_cast<const float*>(F->Cval),
                                          dcols, ncols, h, dout);
  else
    CTD_LAUNCH(k_c_columns<double>, (g), (128), 0, st, reinterpret_cast<const unsigned long long*>(F->Coff),
                                           F->Ccnt, F->Crow, static_cast<const double*>(F->Cval),
                                           dcols, ncols, h, dout);
  CTD_CUDA(cudaGetLastError());
  CTD_TRY(d2h(out, dout, (size_t)ncols * h, st));
  return sync(st);
}

static ctd_status get_C_host(const ctd_factors* F, int64_t* colptr, int32_t* row, double* val);

extern "C" ctd_status ctd_get_C(const ctd_factors* F, int64_t* colptr, int32_t* row, double* val) {
  if (!F || !colptr) return fail(CTD_EINVAL, "NULL argument");
  if (F->kind != 0) return fail(CTD_ENOTSUP, "CTD-D keeps C implicit; use ctd_get_C_columns");
  if (!F->Coff) return fail(CTD_EINVAL, "C was not materialized (CTD_SKIP_C)");
  return guarded([&] { return get_C_host(F, colptr, row, val); });
}

// C's stored layout (offsets with capacity, counts, rows, values) to a packed host CSC.
static ctd_status get_C_host(const ctd_factors* F, int64_t* colptr, int32_t* row, double* val) {
  cudaStream_t st = F->stream;
  const int64_t n = F->n_cols;
  std::vector<uint64_t> off(n + 1);
  std::vector<uint32_t> cnt(n);
  std::vector<uint16_t> r(F->C_cap);
  CTD_TRY(d2h(off.data(), F->Coff, n + 1, st));
  CTD_TRY(d2h(cnt.data(), F->Ccnt, n, st));
  CTD_TRY(d2h(r.data(), F->Crow, F->C_cap, st));
  std::vector<double> v(F->C_cap);
  if (F->precision == CTD_FP32_BULK) {
    std::vector<float> vf(F->C_cap);
    CTD_TRY(d2h(vf.data(), static_cast<const float*>(F->Cval), F->C_cap, st));
    CTD_TRY(sync(st));
    for (size_t q = 0; q < vf.size(); ++q) v[q] = vf[q];
  } else {
    CTD_TRY(d2h(v.data(), static_cast<const double*>(F->Cval), F->C_cap, st));
    CTD_TRY(sync(st));
  }
  int64_t pos = 0;
  const int64_t h = F->s_kept;
  for (int64_t f = 0; f < n; ++f) {
    colptr[f] = pos;
    if (cnt[f] & C_DENSE) {
      for (int64_t m = 0; m < h; ++m)
        if (v[off[f] + m] != 0.0) {
          if (row) row[pos] = (int32_t)m;
          if (val) val[pos] = v[off[f] + m];
          ++pos;
        }
      continue;
    }
    for (uint32_t q = 0; q < cnt[f]; ++q) {
      if (row) row[pos] = r[off[f] + q];
      if (val) val[pos] = v[off[f] + q];
      ++pos;
    }
  }
  colptr[n] = pos;
  return CTD_OK;
}

extern "C" void ctd_free(ctd_factors* F) {
  if (!F) return;
  cudaStreamSynchronize(F->stream);
  delete F;
}

extern "C" ctd_status ctd_set_allocator(ctd_alloc_fn alloc, ctd_release_fn release) {
  if ((alloc == nullptr) != (release == nullptr))
    return fail(CTD_EINVAL, "give both functions, or neither (the library's own pool)");
  std::lock_guard<std::mutex> lk(g_hook_mu);
  g_hook.alloc = alloc;
  g_hook.release = release;
  return CTD_OK;
}

extern "C" ctd_status ctd_allocated_bytes(size_t* bytes) {
  if (!bytes) return fail(CTD_EINVAL, "NULL argument");
  *bytes = live_bytes();
  return CTD_OK;
}

extern "C" ctd_status ctd_set_tuning(const char* key, int64_t value) {
  const int k = tune_index(key);
  if (k < 0) return fail(CTD_EINVAL, std::string("unknown tuning key: ") + (key ? key : "NULL"));
  if (value == -1) value = kTune[k].def;
  if (value < kTune[k].lo || value > kTune[k].hi)
    return fail(CTD_EINVAL, std::string("tuning value out of range for ") + key);
  g_tune[k].store(value);
  return CTD_OK;
}

extern "C" ctd_status ctd_get_tuning(const char* key, int64_t* value) {
  const int k = tune_index(key);
  if (k < 0 || !value) return fail(CTD_EINVAL, "unknown tuning key or NULL");
  *value = g_tune[k].load();
  return CTD_OK;
}

extern "C" ctd_status ctd_profile(int enable) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (auto& r : g_recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g_recs.clear();
  g_launches.store(0);
  g_prof = enable != 0;
  return CTD_OK;
}

extern "C" ctd_status ctd_profile_report(char* buf, size_t len) {
  if (!buf || len == 0) return fail(CTD_EINVAL, "NULL buffer");
  std::lock_guard<std::mutex> lk(g_prof_mu);
  std::vector<std::string> names;
  std::vector<double> ms;
  std::vector<long long> calls;
  for (auto& r : g_recs) {
    CTD_CUDA(cudaEventSynchronize(r.b));
    float t = 0.f;
    CTD_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
    size_t q = 0;
    while (q < names.size() && names[q] != r.name) ++q;
    if (q == names.size()) {
      names.push_back(r.name);
      ms.push_back(0.0);
      calls.push_back(0);
    }
    ms[q] += t;
    calls[q] += 1;
  }
  std::string js = "{\"launches\": " + std::to_string(g_launches.load()) + ", \"phases\": {";
  for (size_t q = 0; q < names.size(); ++q) {
    char item[256];
    snprintf(item, sizeof(item), "%s\"%s\": {\"ms\": %.6f, \"calls\": %lld}", q ? ", " : "",
             names[q].c_str(), ms[q], calls[q]);
    js += item;
  }
  js += "}}";
  snprintf(buf, len, "%s", js.c_str());
  return CTD_OK;
}

extern "C" const char* ctd_last_error(void) { return ctd::g_last_error.c_str(); }

extern "C" const char* ctd_version(void) { return "ctd-gb300 0.1 (sm_103a)"; }

extern "C" ctd_status ctd_fault_inject_alloc(int64_t fail_after) {
  ctd::g_alloc_fail_after.store(fail_after < 0 ? -1 : (long long)fail_after);
  return CTD_OK;
}
