// An entry point that allocates no device memory: the column distribution,
// the draws and their unique set of ctd_static (the first steps of Algorithm 1),
// with its scratch in file-scope device arrays.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// allocator's arena or a memory-capped context where an extra allocation
// fails or is forbidden, and real-time paths that must not touch the
// driver's allocator at all.  They pass only inputs and outputs; the
// intermediate CDF and the prefix-sum tile totals live in the arrays below,
// which every GPU that loads the library keeps until the process exits.
#include <mutex>

#include "ctd_internal.cuh"

namespace ctd {
namespace {

constexpr int64_t NA_MAX_COLS = CTD_NOALLOC_MAX_COLS;

// Column sums of squares, then (in place) their inclusive prefix sums.
static __device__ __align__(256) unsigned long long g_na_cdf[NA_MAX_COLS];
// Scratch of the prefix sum: scan_tmp_elems(n) = 9 * ceil(n / 4096) + 4
// entries (a tile sum and eight warp sums per 4096-entry tile); checked on
// the host before every call.
constexpr int64_t NA_TILES_ELEMS = 9 * ((NA_MAX_COLS + 4095) / 4096) + 8;
static __device__ __align__(256) unsigned long long g_na_tiles[NA_TILES_ELEMS];
// Status word (bad index, overflow) and the unique count.
static __device__ __align__(256) unsigned g_na_status[2];

struct Addr {
  unsigned long long* cdf = nullptr;
  unsigned long long* tiles = nullptr;
  unsigned* status = nullptr;
  bool ready = false;
};
constexpr int MAX_DEVICES = 64;
Addr g_addr[MAX_DEVICES];
std::mutex g_addr_mu;

// Device addresses of the arrays for the current device.  In host code the
// arrays' names are host-side stand-ins, so their device addresses come
// from cudaGetSymbolAddress, once per device, with that device current.
ctd_status device_addresses(Addr* out) {
  int dev = 0;
  CTD_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= MAX_DEVICES) return fail(CTD_ENOTSUP, "device index out of range");
  std::lock_guard<std::mutex> lk(g_addr_mu);
  Addr& a = g_addr[dev];
  if (!a.ready) {
    CTD_CUDA(cudaGetSymbolAddress(reinterpret_cast<void**>(&a.cdf), g_na_cdf));
    CTD_CUDA(cudaGetSymbolAddress(reinterpret_cast<void**>(&a.tiles), g_na_tiles));
    CTD_CUDA(cudaGetSymbolAddress(reinterpret_cast<void**>(&a.status), g_na_status));
    a.ready = true;
  }
  *out = a;
  return CTD_OK;
}

// Squared column norms by one atomic add per entry (no column-major layout
// exists here).  The add returns the column's previous sum: a sum that
// wraps past 2^64 shows as a result below its previous value and sets
// DEV_OVERFLOW (a sum in [2^63, 2^64) is flagged by the prefix sum).
__global__ void k_na_sqnorms(const int32_t* __restrict__ ii, const int32_t* __restrict__ jj,
                             const int32_t* __restrict__ kk, const int32_t* __restrict__ vv,
                             int64_t nnz, ModeMap mm, unsigned long long* __restrict__ sq,
                             unsigned* status) {
  bool bad = false, wrapped = false;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    int32_t row;
    int64_t col;
    if (!mm.map(ii[e], jj[e], kk[e], &row, &col)) {
      bad = true;
      continue;
    }
    const long long v = vv[e];
    const unsigned long long v2 = (unsigned long long)(v * v);
    const unsigned long long old = atomicAdd(sq + col, v2);
    if (old + v2 < old) wrapped = true;
  }
  if (bad) atomicOr(status, DEV_BAD_INDEX);
  if (wrapped) atomicOr(status, DEV_OVERFLOW);
}

}  // namespace
}  // namespace ctd

using namespace ctd;

extern "C" ctd_status ctd_sample_noalloc(const ctd_coo3* X, int alpha, int64_t s, uint64_t seed,
                                         int64_t* draws, int64_t* unique, int* n_unique,
                                         void* stream) {
  if (!X || !draws || !unique || !n_unique) return fail(CTD_EINVAL, "NULL argument");
  if (X->memory != CTD_MEM_DEVICE)
    return fail(CTD_EINVAL, "ctd_sample_noalloc takes device memory only");
  if (alpha < 1 || alpha > 3) return fail(CTD_EINVAL, "alpha must be 1, 2 or 3");
  if (s < 1 || s > 8192) return fail(CTD_EINVAL, "s must be in [1, 8192]");
  for (int d = 0; d < 3; ++d)
    if (X->dims[d] < 1 || X->dims[d] > INT32_MAX)
      return fail(CTD_EINVAL, "each dimension must be in [1, 2^31)");
  if (X->nnz < 0 || X->nnz > INT32_MAX) return fail(CTD_EINVAL, "nnz must be in [0, 2^31)");
  if (X->nnz > 0 && (!X->i || !X->j || !X->k || !X->val))
    return fail(CTD_EINVAL, "index or value pointer is NULL");
  int64_t n_rows, n_cols;
  mode_extents(X->dims, alpha, &n_rows, &n_cols);
  if (n_cols > NA_MAX_COLS)
    return fail(CTD_EINVAL, "N_alpha exceeds CTD_NOALLOC_MAX_COLS (" +
                                std::to_string(NA_MAX_COLS) + ")");
  if (scan_tmp_elems(n_cols) > (size_t)NA_TILES_ELEMS)
    return fail(CTD_EINVAL, "prefix-sum scratch too small for N_alpha");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Addr a;
  CTD_TRY(device_addresses(&a));
  // the arrays keep the previous call's contents: clear what accumulates
  CTD_CUDA(cudaMemsetAsync(a.cdf, 0, (size_t)n_cols * sizeof(unsigned long long), st));
  CTD_CUDA(cudaMemsetAsync(a.status, 0, 2 * sizeof(unsigned), st));
  if (X->nnz > 0)
    CTD_LAUNCH(k_na_sqnorms, (grid_for(X->nnz, 256, (int64_t)num_sms() * 8)), (256), 0, st,
               X->i, X->j, X->k, X->val, X->nnz, make_mode_map(X->dims, alpha), a.cdf, a.status);
  uint64_t* cdf = reinterpret_cast<uint64_t*>(a.cdf);
  launch_scan_u64(cdf, cdf, n_cols, true, reinterpret_cast<uint64_t*>(a.tiles), a.status, st);
  launch_sample(cdf, n_cols, s, seed, 0, 0, draws, st);
  launch_sort_unique(draws, s, unique, reinterpret_cast<int*>(a.status + 1), st);
  unsigned h[2] = {0, 0};
  CTD_CUDA(cudaMemcpyAsync(h, a.status, sizeof(h), cudaMemcpyDeviceToHost, st));
  CTD_CUDA(cudaGetLastError());
  CTD_CUDA(cudaStreamSynchronize(st));
  CTD_TRY(status_from_device(h[0]));
  *n_unique = (int)h[1];
  return CTD_OK;
}
