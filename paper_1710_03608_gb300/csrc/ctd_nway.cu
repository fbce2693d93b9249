// CTD-S on an N-way tensor (Section 2.1: the mode-alpha matricization of a
// tensor of any order).  Every nonzero is mapped on the device to its row
// (the mode-alpha index) and its little-endian column over the other modes;
// the matricized tensor is then the 3-way tensor I_alpha x N_alpha x 1 with
// alpha = 1, which ctd_static decomposes.  The mapping is the only N-way
// specific step: Algorithm 1 never looks at more than the matricization.
#include "ctd_internal.cuh"

namespace ctd {
namespace {

struct NwayMap {
  int order, alpha;
  int64_t dims[CTD_MAX_ORDER];
  int64_t stride[CTD_MAX_ORDER];   // column stride of each mode (0 for mode alpha)
  const int32_t* idx[CTD_MAX_ORDER];
};

// row[e], col[e] (int32: N_alpha < 2^31 is checked on the host), k[e] = 0,
// v[e] = val[e]; an index outside its mode sets DEV_BAD_INDEX and maps the
// entry to row 0, column 0 with value 0 (the caller then fails the call).
__global__ void k_nway_map(NwayMap m, const int32_t* __restrict__ val, int64_t nnz,
                           int32_t* __restrict__ row, int32_t* __restrict__ col,
                           int32_t* __restrict__ kk, int32_t* __restrict__ v,
                           unsigned* status) {
  bool bad = false;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t c = 0;
    int32_t r = 0;
    bool ok = true;
    for (int n = 0; n < m.order; ++n) {
      const int32_t x = __ldg(m.idx[n] + e);
      if (x < 0 || x >= m.dims[n]) ok = false;
      if (n == m.alpha - 1)
        r = x;
      else
        c += (int64_t)x * m.stride[n];
    }
    if (!ok) bad = true;
    row[e] = ok ? r : 0;
    col[e] = ok ? (int32_t)c : 0;
    kk[e] = 0;
    v[e] = ok ? __ldg(val + e) : 0;
  }
  if (bad) atomicOr(status, DEV_BAD_INDEX);
}

}  // namespace
}  // namespace ctd

using namespace ctd;

extern "C" ctd_status ctd_static_nway(const ctd_coon* X, int alpha, int64_t s, double eps,
                                      uint64_t seed, int precision, unsigned flags,
                                      void* stream, ctd_factors** out) {
  if (!X || !out) return fail(CTD_EINVAL, "NULL argument");
  *out = nullptr;
  const int N = X->order;
  if (N < 1 || N > CTD_MAX_ORDER) return fail(CTD_EINVAL, "order must be in 1 .. CTD_MAX_ORDER");
  if (alpha < 1 || alpha > N) return fail(CTD_EINVAL, "alpha must be in 1 .. order");
  if (X->nnz < 0 || X->nnz > INT32_MAX) return fail(CTD_EINVAL, "nnz must be in [0, 2^31)");
  if (X->memory != CTD_MEM_DEVICE && X->memory != CTD_MEM_HOST)
    return fail(CTD_EINVAL, "unknown memory kind");
  if (X->val_type != CTD_VAL_INT32 && X->val_type != CTD_VAL_FP32)
    return fail(CTD_EINVAL, "unknown value type");
  if (s < 1 || s > 8192) return fail(CTD_EINVAL, "s must be in [1, 8192]");
  if (!(eps >= 0.0 && eps < 1.0)) return fail(CTD_EINVAL, "eps must be in [0, 1)");
  if (precision != CTD_FP64 && precision != CTD_FP32_BULK)
    return fail(CTD_EINVAL, "unknown precision");
  NwayMap m{};
  m.order = N;
  m.alpha = alpha;
  int64_t n_cols = 1;
  for (int n = 0; n < N; ++n) {
    if (X->dims[n] < 1 || X->dims[n] > INT32_MAX)
      return fail(CTD_EINVAL, "each dimension must be in [1, 2^31)");
    if (X->nnz > 0 && !X->idx[n]) return fail(CTD_EINVAL, "index pointer is NULL");
    m.dims[n] = X->dims[n];
    if (n == alpha - 1) continue;
    m.stride[n] = n_cols;
    n_cols *= X->dims[n];
    if (n_cols > INT32_MAX) return fail(CTD_EINVAL, "N_alpha must be < 2^31");
  }
  if (X->nnz > 0 && !X->val) return fail(CTD_EINVAL, "value pointer is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Arena scratch;
  scratch.st = st;
  const int64_t nnz = X->nnz;
  // the mapped tensor: row, column, a zero third index and the values, each
  // array starting on a 16-byte boundary
  const int64_t ld = (nnz + 3) & ~(int64_t)3;
  int32_t* buf;
  unsigned* status;
  CTD_TRY(scratch.get(&buf, 4 * (size_t)std::max<int64_t>(ld, 1)));
  CTD_TRY(scratch.get(&status, 1));
  CTD_CUDA(cudaMemsetAsync(status, 0, sizeof(unsigned), st));
  // values move as 32-bit payloads (int32 counts or FP32 bits)
  const int32_t* src_val = static_cast<const int32_t*>(X->val);
  if (X->memory == CTD_MEM_HOST && nnz > 0) {
    // the index arrays and values copied in, then mapped on the device
    int32_t* in;
    CTD_TRY(scratch.get(&in, (size_t)(N + 1) * ld));
    for (int n = 0; n < N; ++n) {
      CTD_CUDA(cudaMemcpyAsync(in + n * ld, X->idx[n], nnz * sizeof(int32_t),
                               cudaMemcpyHostToDevice, st));
      m.idx[n] = in + n * ld;
    }
    CTD_CUDA(cudaMemcpyAsync(in + N * ld, X->val, nnz * sizeof(int32_t), cudaMemcpyHostToDevice,
                             st));
    src_val = in + N * ld;
  } else {
    for (int n = 0; n < N; ++n) m.idx[n] = X->idx[n];
  }
  if (nnz > 0)
    CTD_LAUNCH(k_nway_map, (grid_for(nnz, 256, (int64_t)num_sms() * 8)), (256), 0, st, m,
               src_val, nnz, buf, buf + ld, buf + 2 * ld, buf + 3 * ld, status);
  unsigned h_status = 0;
  CTD_TRY(d2h(&h_status, status, 1, st));
  CTD_CUDA(cudaGetLastError());
  CTD_TRY(sync(st));
  if (h_status & DEV_BAD_INDEX) return fail(CTD_EINVAL, "an index is outside its mode");
  CooDev x3;
  x3.dims[0] = X->dims[alpha - 1];
  x3.dims[1] = n_cols;
  x3.dims[2] = 1;
  x3.alpha = 1;
  x3.nnz = nnz;
  x3.i = buf;
  x3.j = buf + ld;
  x3.k = buf + 2 * ld;
  x3.v = buf + 3 * ld;
  PhaseScope ph_call("call", st);
  return static_impl(x3, s, eps, seed, precision, flags, st, scratch,
                     X->val_type == CTD_VAL_FP32, out);
}
