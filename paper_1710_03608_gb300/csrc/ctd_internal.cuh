// Internal declarations shared by the CTD CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <exception>
#include <new>
#include <string>
#include <vector>

#include "ctd.h"

namespace ctd {

// ---------------------------------------------------------------------------
// status / errors
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
ctd_status fail(ctd_status st, const std::string& msg);

// Runs fn() and turns a host allocation failure inside it into CTD_ENOMEM:
// no exception may cross the C ABI (getters size host buffers by the data).
template <typename Fn>
ctd_status guarded(Fn&& fn) {
  try {
    return fn();
  } catch (const std::bad_alloc&) {
    return fail(CTD_ENOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(CTD_EINVAL, std::string("unexpected host error: ") + e.what());
  }
}

#define CTD_CUDA(call)                                                        \
  do {                                                                        \
    cudaError_t _e = (call);                                                  \
    if (_e != cudaSuccess) {                                                  \
      return ::ctd::fail(_e == cudaErrorMemoryAllocation ? CTD_ENOMEM         \
                                                         : CTD_ECUDA,         \
                         std::string(#call) + ": " + cudaGetErrorString(_e)); \
    }                                                                         \
  } while (0)

#define CTD_TRY(expr)                     \
  do {                                    \
    ctd_status _s = (expr);               \
    if (_s != CTD_OK) return _s;          \
  } while (0)

// Every kernel launch goes through CTD_LAUNCH so the library can report how
// many kernels it started (a diagnostic, see ctd_profile_report).
void note_launch();
#define CTD_LAUNCH(kern, grid, block, smem, st, ...) \
  do {                                               \
    ::ctd::note_launch();                            \
    kern<<<grid, block, smem, st>>>(__VA_ARGS__);    \
  } while (0)

// Device-time phase timer: records a CUDA event pair on `st` around a scope
// when profiling is on (ctd_profile(1)); no-op otherwise.
struct PhaseScope {
  PhaseScope(const char* name, cudaStream_t st);
  ~PhaseScope();
  const char* name;
  cudaStream_t st;
  cudaEvent_t a = nullptr, b = nullptr;
};

// Bits of the device status word every pipeline carries.
enum : unsigned {
  DEV_BAD_INDEX = 1u,   // a COO index outside its mode's extent
  DEV_OVERFLOW = 2u,    // an exact sum left its integer range
  DEV_CAPACITY = 4u,    // a size exceeded a buffer bound
  DEV_TIMEOUT = 8u      // a bounded wait gave up
};
ctd_status status_from_device(unsigned word);

// ---------------------------------------------------------------------------
// stream-ordered device memory
// ---------------------------------------------------------------------------
ctd_status dalloc(void** p, size_t bytes, cudaStream_t st);
void dfree(void* p, cudaStream_t st);
// Device bytes the library holds now, and whether an allocator hook is set.
size_t live_bytes();
bool allocator_hooked();

template <typename T>
ctd_status dalloc_n(T** p, size_t n, cudaStream_t st) {
  return dalloc(reinterpret_cast<void**>(p), n * sizeof(T), st);
}

// A list of device allocations freed together.
struct Arena {
  std::vector<void*> ptrs;
  cudaStream_t st = nullptr;
  template <typename T>
  ctd_status get(T** p, size_t n) {
    void* q = nullptr;
    CTD_TRY(dalloc(&q, (n ? n : 1) * sizeof(T), st));
    ptrs.push_back(q);
    *p = static_cast<T*>(q);
    return CTD_OK;
  }
  void release() {
    for (void* q : ptrs) dfree(q, st);
    ptrs.clear();
  }
  ~Arena() { release(); }
};

// Let `fn` use up to the device's opt-in shared memory per block.  Set once
// per kernel and device, under a lock: each call site used to set the limit
// to its own need, so concurrent host threads could lower it under another's
// launch.  A higher limit does not change launches that ask for less.
ctd_status allow_max_smem(const void* fn);

// Launch-shape knobs (ctd_set_tuning): shared memory for the Q-form's
// staged rows and for the C fill's dense rows (bytes), blocks per SM of the
// one-nonzero copy.
enum TuneKey { TUNE_QFORM_HOT, TUNE_CFILL_DENSE, TUNE_COPY_BLOCKS, TUNE_N };
int64_t tuning(TuneKey k);

inline int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 148;
  }
  return n;
}

inline unsigned grid_for(int64_t work, int per_block, int64_t cap) {
  int64_t g = (work + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return static_cast<unsigned>(g);
}

// ---------------------------------------------------------------------------
// kernel launchers (one translation unit each)
// ---------------------------------------------------------------------------

// ctd_stream.cu ------------------------------------------------------------
struct CooDev {
  const int32_t* i;
  const int32_t* j;
  const int32_t* k;
  const int32_t* v;
  int64_t nnz;
  int64_t dims[3];
  int alpha;  // 1..3
};

// Mode-alpha row extent and column count.
void mode_extents(const int64_t dims[3], int alpha, int64_t* n_rows, int64_t* n_cols);

// Row (mode-alpha index) and column of X_(alpha) for one nonzero: the
// little-endian order of the other two modes (alpha = 1: f = j + J k;
// alpha = 2: f = i + I k; alpha = 3: f = i + I j).  false for an index
// outside its mode's extent.  Every kernel that maps COO entries to
// columns goes through this one definition.
struct ModeMap {
  int alpha;
  int64_t I, J, K;
  __device__ __forceinline__ bool map(int32_t a, int32_t b, int32_t c, int32_t* row,
                                      int64_t* col) const {
    if (a < 0 || b < 0 || c < 0 || a >= I || b >= J || c >= K) return false;
    if (alpha == 1) {
      *row = a;
      *col = (int64_t)b + J * (int64_t)c;
    } else if (alpha == 2) {
      *row = b;
      *col = (int64_t)a + I * (int64_t)c;
    } else {
      *row = c;
      *col = (int64_t)a + I * (int64_t)b;
    }
    return true;
  }
};
inline ModeMap make_mode_map(const int64_t dims[3], int alpha) {
  ModeMap m;
  m.alpha = alpha;
  m.I = dims[0];
  m.J = dims[1];
  m.K = dims[2];
  return m;
}

// The sampling weight of one value of X (Eq. 1's summand).  Integer counts
// (wshift == WSHIFT_INT): the exact square.  Real values (the 32-bit payload
// holds an FP32 value): the square on a fixed-point grid, floor(v^2 *
// 2^wshift), with 2^-wshift = 2^(E - 32) where 2^E bounds the largest
// square; v^2 is exact in FP64 and the scaling is a power of
// two, so the weight is exact and the same on every device.
constexpr int WSHIFT_INT = -0x7fffffff - 1;
__device__ __forceinline__ unsigned long long sample_weight(int32_t bits, int wshift) {
  if (wshift == WSHIFT_INT) return (unsigned long long)((long long)bits * (long long)bits);
  const double f = (double)__int_as_float(bits);
  return (unsigned long long)floor(ldexp(f * f, wshift));
}

// A value of X (or R) as FP64: an integer count, or (real) the FP32 value
// its 32-bit payload holds.
__device__ __forceinline__ double value_f64(int32_t bits, int real) {
  return real ? (double)__int_as_float(bits) : (double)bits;
}

// K1a: entries per column (colcnt) and per row (rowcnt) of X_(alpha);
// both zeroed beforehand.  Out-of-range indices set DEV_BAD_INDEX.
void launch_count(const CooDev& X, uint32_t* colcnt, uint32_t* rowcnt, unsigned* status,
                  cudaStream_t st);
// K1b: squared column norms from the column-major layout: norm2[f] = the
// sum of val[p]^2 over p in [colptr[f], colptr[f+1]) (saturating u64),
// followed by their inclusive prefix sum cdf (the column distribution).
// Also reduces the smallest value into minkey[0] as the order-preserving
// code (unsigned)v ^ 2^31, and the largest into minkey[1] as the complement
// of its code (both initialized to all ones; decode_min / decode_max).
// A total at or past 2^63 sets DEV_OVERFLOW.
void launch_sqnorms_cdf(const uint64_t* colptr, const int32_t* val, int64_t n_cols,
                        uint64_t* norm2, uint64_t* cdf, unsigned* minkey, uint64_t* tmp,
                        unsigned* status, cudaStream_t st, int wshift = WSHIFT_INT);

// K2: prefix sums.  out[n] (inclusive) or out[n+1] (exclusive, out[0]=0).
// `tmp` needs scan_tmp_elems(n) entries.  Sums are saturating u64 adds; a
// total at or past 2^63 sets DEV_OVERFLOW in *status.  in == out is
// allowed for the inclusive u64 scan (each element is read before it is
// written, by the same thread).  cur32 (optional, u32 scan only) receives
// the exclusive prefix of every element as u32 and may alias `in`.  Up to
// 16,384 elements take one launch (one block), longer inputs three
// (reduce, scan of the tile sums, apply).
size_t scan_tmp_elems(int64_t n);
// Tiling of the scans: a tile of SCAN_TILE elements is one block of
// SCAN_WARPS warps, each warp a segment of SCAN_PER_WARP elements.
constexpr int SCAN_WARPS = 8;
constexpr int SCAN_PER_WARP = 512;                       // 16 per lane
constexpr int SCAN_TILE = SCAN_WARPS * SCAN_PER_WARP;    // 4096
void launch_scan_u64(const uint64_t* in, uint64_t* out, int64_t n, bool inclusive,
                     uint64_t* tmp, unsigned* status, cudaStream_t st);
void launch_scan_u32(const uint32_t* in, uint64_t* out, int64_t n, bool inclusive,
                     uint64_t* tmp, unsigned* status, cudaStream_t st,
                     uint32_t* cur32 = nullptr);
// Tile scan and apply of an inclusive u64 scan whose tile and warp sums were
// written by another kernel into tmp (same layout and tiling as the scans
// above: 4096-element tiles of eight 512-element warp segments).
void launch_scan_finish(const uint64_t* in, uint64_t* out, int64_t n, uint64_t* tmp,
                        unsigned* status, cudaStream_t st);

// K5a: counting-sort scatter of the COO into the column-major layout (CSC:
// row, val).  cur[f] starts as column f's first position (u32: nnz < 2^31)
// and is consumed.
void launch_coo_scatter(const CooDev& X, uint32_t* cur, int32_t* csc_row, int32_t* csc_val,
                        cudaStream_t st);

// Copy u64 -> u64 (cursor initialization) for n elements.
// Sort every column's entries of a compressed layout by (row, value), in
// place; `keys` holds at least nnz u64 (scratch for columns longer than one
// block's shared memory).
ctd_status launch_sort_cols(const uint64_t* colptr, int64_t n_cols, int64_t nnz, int32_t* row,
                            int32_t* val, uint64_t* keys, Arena& A, cudaStream_t st);
void launch_copy_u64(const uint64_t* in, uint64_t* out, int64_t n, cudaStream_t st);
// out[0] = sum of n u32 values (as u64), each masked with `mask` first.
void launch_sum_u32(const uint32_t* in, int64_t n, uint64_t* out, cudaStream_t st,
                    uint32_t mask = 0xffffffffu);
// out[c] = in[idx[c]] for c < *count.
void launch_gather_i64(const int64_t* in, const int* idx, const int* count, int nmax,
                       int64_t* out, cudaStream_t st);

// K5b: gather columns `fibers[0..nf)` of a CSC matrix into a compact CSC
// (colptr_out[nf+1] must already hold the exclusive sizes).
void launch_column_sizes(const uint64_t* colptr, const int64_t* fibers, const int* nf_dev,
                         int nf_max, uint64_t* sizes, cudaStream_t st);
void launch_gather_columns(const uint64_t* colptr, const int32_t* row, const int32_t* val,
                           const int64_t* fibers, const int* nf_dev, int nf_max,
                           const uint64_t* colptr_out, int32_t* row_out, int32_t* val_out,
                           cudaStream_t st);

// Build a row-major copy (rowptr over n_rows, col, val) of a small CSC with
// ncols columns whose column c gets index col_base + c; rows are sorted by
// column.  nnz is an upper bound on the entries (sizes the temporaries).
// The rows of a factor by row (rowptr, col, val; rows sorted by column)
// restricted to the columns c with kpos[c] >= 0, renumbered to kpos[c]
// (increasing on those columns): the output rows stay sorted.  rowptr_out:
// n_rows + 1 entries; col_out / val_out: room for the kept entries.
ctd_status csr_keep_columns(const uint64_t* rowptr, const int32_t* col, const int32_t* val,
                            int64_t n_rows, const int* kpos, uint64_t* rowptr_out,
                            int32_t* col_out, int32_t* val_out, Arena& scratch,
                            cudaStream_t st);
ctd_status build_csr_from_csc(const uint64_t* colptr, const int32_t* row, const int32_t* val,
                              int64_t ncols, int64_t nnz, int64_t n_rows, int col_base,
                              uint64_t* rowptr_out, int32_t* col_out, int32_t* val_out,
                              Arena& scratch, cudaStream_t st);

// ctd_sample.cu ------------------------------------------------------------
// K3: s draws.  total = cdf[n-1] (read on device).
void launch_sample(const uint64_t* cdf, int64_t n, int64_t s, uint64_t seed,
                   uint64_t step, uint64_t stream_id, int64_t* out, cudaStream_t st);
// K4: ascending unique of s values (s <= 8192); writes out[0..s') and *count.
void launch_sort_unique(const int64_t* in, int64_t s, int64_t* out, int* count,
                        cudaStream_t st);

// ctd_spmm.cu --------------------------------------------------------------
struct CscDev {        // X_(alpha) by column
  const uint64_t* colptr;
  const int32_t* row;
  const int32_t* val;
};
struct CsrDev {        // a factor by row: row i holds (col, val) pairs
  const uint64_t* rowptr;
  const int32_t* col;
  const int32_t* val;
  int width;           // number of columns
  int64_t nnz = -1;    // number of entries (-1: not known on the host)
  int max_abs = -1;    // largest |value| (-1: not known on the host)
};

// Dense products: out(:, c) = R^T x_{fibers[c]} for c < nf (column-major,
// leading dimension ld), exact integer sums stored as double.  With a
// scratch arena (and R at most 6,144 wide) each column's entries are spread
// over several blocks through an int64 accumulator; without, a block per
// column.
ctd_status launch_spmm_dense(const CscDev& X, const int64_t* fibers, const int* nf_dev,
                             int nf_max, const CsrDev& R, double* out, int64_t ld,
                             cudaStream_t st, Arena* scratch = nullptr);

// Sparse product C = R^T X_(alpha) over all n_cols columns.
// bounds: ub[f] = min(width, sum of R row lengths over column f) rounded up
// to a multiple of 4 (the column's capacity; columns start 4-aligned).
// Column f's storage at offset coff[f]: ccnt[f] & C_COUNT nonzeros; if
// ccnt[f] & C_DENSE the column is stored densely (cval[coff[f] + m] for
// rows m < width, zeros included; crow unused), else as ascending 16-bit
// rows crow[coff[f] + q] with values cval[coff[f] + q].
constexpr uint32_t C_DENSE = 0x80000000u;
constexpr uint32_t C_COUNT = 0x7fffffffu;
void launch_c_bounds(const CscDev& X, int64_t n_cols, const CsrDev& R, uint32_t* ub,
                     cudaStream_t st);
// fill: column f's entries go to [coff[f], coff[f] + ccnt[f]) with rows
// ascending (16-bit row indices).  Values stored as float (fp32 != 0) or
// double.  R's rows must be sorted by column.  positive: every value of X
// and R is > 0 (enables the one-nonzero copy path).  x_int8: every value of
// X is in [-128, 127] (four products per instruction on int8 rows of R).
// The C fill's column lists (built with the C bounds by
// launch_c_bounds_lists): one-nonzero columns, columns with at least 128
// nonzeros, the other multi-nonzero columns, and their three counts.
struct CfillLists {
  int64_t* single = nullptr;
  int64_t* heavy = nullptr;
  int64_t* multi = nullptr;
  unsigned* counts = nullptr;
};
ctd_status launch_c_fill(const CscDev& X, int64_t n_cols, int64_t n_rows, int64_t nnz,
                         const CsrDev& R, const uint64_t* coff, uint32_t* ccnt, uint16_t* crow,
                         void* cval, int fp32, int positive, int x_int8, uint64_t sqnorm_X,
                         cudaStream_t st, const CfillLists* lists = nullptr);
// The same with the longest rows of R dense in shared memory and register
// accumulators (ctd_cfill.cu); requires sqnorm_X < 2^31 and width <= 1024.
ctd_status c_fill_dense_rows(const CscDev& X, int64_t n_cols, int64_t n_rows, int64_t nnz,
                             const CsrDev& R, const uint64_t* coff, uint32_t* ccnt,
                             uint16_t* crow, void* cval, int fp32, int positive, int x_int8,
                             cudaStream_t st, const CfillLists* lists = nullptr);
// The C bounds (as launch_c_bounds) and, in the same pass over the columns,
// the C fill's column lists (list_cap entries each; counts zeroed here) and
// ccnt = 0 for the columns C leaves empty.  positive: every value of X and R
// is > 0 (one-nonzero columns are then copies).
ctd_status launch_c_bounds_lists(const CscDev& X, int64_t n_cols, const CsrDev& R, uint32_t* ub,
                                 int positive, uint32_t* ccnt, const CfillLists& L,
                                 cudaStream_t st);
// list[0..count) = columns with >= minc nonzeros and a nonzero C bound
void launch_list_columns(const uint64_t* colptr, const uint64_t* coff, int64_t n_cols,
                         uint64_t minc, int64_t* list, unsigned* count, cudaStream_t st);
// Sort each row of a row-major factor by column (col/val copied to *_out).
// Sort every segment of (ptr, idx, val) by idx in place (tmp_* hold as many
// entries as idx; used for segments longer than 2048).  The indices lie in
// [0, index_range); a range of at most 65,536 lets long segments be ranked
// through a bitmap of their indices.
void launch_sort_segments(const uint64_t* ptr, int64_t nseg, int32_t* idx, int32_t* val,
                          int32_t* tmp_idx, int32_t* tmp_val, int64_t index_range,
                          cudaStream_t st);
// Sort each row of (rowptr, col, val) by column into the out arrays; the
// columns lie in [col_base, col_base + ncols) (ncols <= 8192 enables the
// bitmap ranking of long rows; 0 or larger: comparisons only).
void launch_sort_rows(const uint64_t* rowptr, int64_t n_rows, const int32_t* col_in,
                      const int32_t* val_in, int32_t* col_out, int32_t* val_out, int col_base,
                      int64_t ncols, cudaStream_t st);

// Relative-error numerator ||Q^T X_(alpha)||_F^2 with Q = R Z^T, Z = L^{-1}
// (kept x kept, column-major, ld ldz).  The rows of X with the most
// nonzeros (rowcnt, on the device) have their Q rows staged in shared memory.
ctd_status launch_error_qform(const CscDev& X, int64_t n_cols, int64_t n_rows, int64_t X_nnz,
                              const CsrDev& R, const double* Z, int64_t ldz,
                              const uint32_t* rowcnt, int fp32, double* out, Arena& scratch,
                              cudaStream_t st);

// ||Q^T X_(alpha)||_F^2 for FP64 Q by rows (row i at Q + i * ld, ld a
// multiple of 512, zero past `width`), with row norms qn.
ctd_status launch_qform_rows(const CscDev& X, int64_t n_cols, int64_t nnz, const double* Q,
                             int64_t ld, int64_t width, const double* qn, int64_t n_rows,
                             double* out, Arena& scratch, cudaStream_t st);
// Columns with at least minc nonzeros: list + count (any order).
void launch_list_columns_nnz(const uint64_t* colptr, int64_t n_cols, uint64_t minc, int64_t* list,
                             unsigned* count, cudaStream_t st);
// For the listed columns f (at most max_heavy, count on the device): y_f =
// sum over the column's entries of v Q(i, :) (Q by rows, row i at Qt + i*ld,
// d entries), split over blocks and added in a fixed order; stores y_f in
// W(:, f) (ld d) when W is given and ||y_f||^2 in norms[h] when given.
ctd_status launch_heavy_columns(const int64_t* list, const unsigned* nlist, int64_t max_heavy,
                                const uint64_t* cptr, const int32_t* crow, const int32_t* cval,
                                const double* Qt, int64_t ld, int64_t d, double* W,
                                double* norms, Arena& scratch, cudaStream_t st);

// *out = the sum of in[0 .. n) in a fixed order (the same on every run).
ctd_status sum_f64(const double* in, int64_t n, double* out, Arena& scratch, cudaStream_t st);

// ctd_real.cu: the stages of Algorithm 1 that differ for real (FP32) values.
ctd_status real_weight_shift(const int32_t* v, int64_t nnz, int* wshift, Arena& scratch,
                             cudaStream_t st);
ctd_status real_sqnorm(const int32_t* v, int64_t nnz, double* out, Arena& scratch,
                       cudaStream_t st);
ctd_status real_gram(const uint64_t* cptr, const int32_t* crow, const int32_t* cval,
                     const int* nc_dev, int su, int64_t n_rows, double* G, Arena& scratch,
                     cudaStream_t st);
ctd_status real_c_fill(const CscDev& X, int64_t n_cols, const CsrDev& R, const uint64_t* coff,
                       uint32_t* ccnt, uint16_t* crow, void* cval, int fp32, cudaStream_t st);
ctd_status real_error_qform(const CscDev& X, int64_t n_cols, int64_t n_rows,
                            const uint64_t* Rcolptr, const int32_t* Rrow, const int32_t* Rval,
                            int kept, const double* Z, int64_t ldz, double* out, Arena& scratch,
                            cudaStream_t st);
// Algorithm 1 on a staged tensor; real: the values' payloads are FP32.
ctd_status static_impl(const CooDev& X, int64_t s, double eps, uint64_t seed, int precision,
                       unsigned flags, cudaStream_t st, Arena& scratch, int real,
                       ctd_factors** out);

// ctd_dense.cu -------------------------------------------------------------
// C = alpha op(A) op(B) + beta C, column-major FP64.
void dgemm(bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha, const double* A,
           int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
           cudaStream_t st);
// In-order Cholesky with skip on the n x n SPD-or-singular matrix A
// (column-major, lower triangle used).  Column k is kept iff its Schur
// diagonal exceeds thr[k].  Kept columns hold L, skipped ones are zeroed.
// keep[k] in {0,1}.
// force (optional): -1 decide by pivot, 0 skip, 1 keep.  fpiv (optional):
// for a forced keep with fpiv[k] > 0, the pivot used in place of the Schur
// diagonal (the explicit residual's squared norm).  piv (optional)
// receives each column's pivot before its decision; a forced keep without a
// positive pivot sets DEV_CAPACITY in status[0]; a grid barrier that gives
// up sets DEV_TIMEOUT.  status must hold 4 words (status[1..2] are the grid
// barrier's counter and generation, status[3] counts the parts of each next
// diagonal block's update).
ctd_status launch_chol_skip(double* A, int64_t n, int64_t lda, const double* thr, int* keep,
                            cudaStream_t st, const int* force, double* piv, unsigned* status,
                            const double* fpiv = nullptr);
// B <- L^{-T} B for lower-triangular L, by backward substitution.
void tri_solve_lower_T(const double* L, int64_t ldl, int64_t n, double* B, int64_t ldb,
                       int64_t nrhs, cudaStream_t st);
// idx[0..count) = positions k with keep[k] != 0 (ascending); *count on device.
void launch_compact_flags(const int* keep, int n, int* idx, int* count, cudaStream_t st);
// B (nk x nk) = A[idx, idx] for the lower triangle (upper zeroed).
void launch_gather_lower(const double* A, int64_t lda, const int* idx, const int* count_dev,
                         int nk_max, double* B, int64_t ldb, cudaStream_t st);
// Z = L^{-1} for lower-triangular L (n x n), in place into Z (Z != L).
ctd_status tri_inverse(const double* L, int64_t ldl, int64_t n, double* Z, int64_t ldz,
                       cudaStream_t st);
// U = Z^T Z (symmetric, full) for lower-triangular Z.
void u_from_linv(const double* Z, int64_t n, int64_t ldz, double* U, int64_t ldu,
                 cudaStream_t st);
// Zero a column-major m x n matrix.
void launch_zero_f64(double* A, int64_t m, int64_t n, int64_t lda, cudaStream_t st);
// Copy lower triangle into upper (symmetrize).
void launch_symmetrize(double* A, int64_t n, int64_t lda, cudaStream_t st);
// thr[k] = eps^2 * diag[k] for the n diagonal entries of D (stride ldd+1).
void launch_thresholds(const double* D, int64_t n, int64_t ldd, double eps2, double* thr,
                       cudaStream_t st);

// ctd_api.cu (host helpers shared by the entry points) -------------------
// Several small device-to-host reads behind one stream synchronization:
// each add() enqueues an asynchronous copy into a pinned staging chunk (a
// per-thread pool, so concurrent calls on other threads do not collide);
// wait() synchronizes the stream once and copies the values out.  Reads too
// large for a chunk fall back to a direct copy.
struct Readback {
  explicit Readback(cudaStream_t s);
  ~Readback();
  template <typename T>
  ctd_status add(T* host, const T* dev, size_t n) {
    return add_bytes(host, dev, n * sizeof(T));
  }
  ctd_status add_bytes(void* host, const void* dev, size_t bytes);
  ctd_status wait();
  // mark() records an event after the copies queued so far; wait_mark()
  // waits for that event only (work queued after mark() keeps running) and
  // delivers those copies
  ctd_status mark();
  ctd_status wait_mark();
  cudaStream_t st;
  cudaEvent_t ev = nullptr;
  char* chunk = nullptr;
  size_t used = 0;
  struct Item { void* host; size_t off, bytes; };
  std::vector<Item> items;
};

ctd_status d2h_bytes(void* host, const void* dev, size_t bytes, cudaStream_t st);
template <typename T>
inline ctd_status d2h(T* host, const T* dev, size_t n, cudaStream_t st) {
  return d2h_bytes(host, dev, n * sizeof(T), st);
}
ctd_status sync(cudaStream_t st);

// A second stream of the calling host thread (non-blocking, on the current
// device, kept for the thread's lifetime) for work that can run beside the
// main chain, with a fork and a join event.  fork(st) orders the side stream
// after everything queued on st so far; join(st) orders st after everything
// queued on the side stream so far.
struct SideStream {
  cudaStream_t st = nullptr;
  ctd_status fork(cudaStream_t main);
  ctd_status join(cudaStream_t main);
  int dev = -1;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  ~SideStream();
};
ctd_status side_stream(SideStream** out);
ctd_status stage_coo(const ctd_coo3* X, int alpha, Arena& scratch, cudaStream_t st, CooDev* out);

// X_(alpha) by column plus its column distribution.
struct Matricized {
  int64_t n_rows = 0, n_cols = 0, nnz = 0;
  uint64_t* norm2 = nullptr;    // [n_cols] squared column norms
  uint64_t* cdf = nullptr;      // [n_cols] inclusive prefix of squared norms
  uint64_t* colptr = nullptr;   // [n_cols+1]
  int32_t* csc_row = nullptr;
  int32_t* csc_val = nullptr;
  unsigned* minval = nullptr;   // [2] codes of the smallest and largest value (see
                                // launch_sqnorms_cdf)
  unsigned* status = nullptr;
  uint64_t* tmp = nullptr;
  uint32_t* rowcnt = nullptr;   // [n_rows] nonzeros per row
  CscDev csc() const { return CscDev{colptr, csc_row, csc_val}; }
};
// ctd_matricize.cu: the same layout, norms and scan tile sums by a bucketed
// counting sort (coalesced writes), for shapes with many columns.  *used is
// false (and nothing the plain passes need was written) when the shape does
// not suit it; then the caller runs the plain passes.  M's arrays are
// allocated, rowcnt/status zeroed and minval initialized by the caller; on
// success norm2 holds the squared norms and tmp the scan's tile and warp
// sums (finish with launch_scan_finish).
ctd_status matricize_bucketed(const CooDev& X, Arena& A, cudaStream_t st, Matricized* M,
                              bool* used, int wshift = WSHIFT_INT);
// The smallest value from its order-preserving code (INT32_MAX when X has
// no entries).
inline int decode_min(unsigned key) { return (int)(key ^ 0x80000000u); }
// The largest value from its code (INT32_MIN when X has no entries).
inline int decode_max(unsigned key) { return (int)(~key ^ 0x80000000u); }
// Algorithm 1's first steps: the column-major layout of X_(alpha), the
// squared column norms and their CDF.  sort_cols: put each column's entries
// in (row, value) order (CTD_DETERMINISTIC).  dist (optional): the arena
// that receives norm2 and cdf (so a caller can keep them); A otherwise.
// wshift: WSHIFT_INT for integer counts, else the real values' weight grid
// (sample_weight).
ctd_status matricize(const CooDev& X, Arena& A, cudaStream_t st, Matricized* M,
                     bool sort_cols = false, Arena* dist = nullptr, int wshift = WSHIFT_INT);

// ctd_filter.cu: the independence filter over a block of du candidates.
// S (du x du, ld du) holds the candidates' Schur complement against R^(t)
// (X_c^T X_c when R^(t) is empty) and is overwritten by the skip-Cholesky
// storage; xnorm2 = ||x_k||^2.  cptr/crow/cval: the candidates as CSC.
// For CTD-D: dt = columns of R^(t), Lt (ld ldl) its Cholesky factor,
// W = Lt^{-1} R^(t)^T X_c (dt x du), and R^(t) as CSC (rptr, rrow, rval).
struct FilterIn {
  int du = 0;
  double* S = nullptr;
  const double* xnorm2 = nullptr;
  double eps = 0.0;
  const uint64_t* cptr = nullptr;
  const int32_t* crow = nullptr;
  const int32_t* cval = nullptr;
  // CTD-D: the candidates are tested against range(R^(t)) through its
  // orthonormal basis Q (n_rows x dt; Q(i, j) at Qt[j + i * ldq]) and
  // W = Q^T X_c (dt x du)
  int64_t dt = 0;
  const double* Qt = nullptr;
  int64_t ldq = 0;
  const double* W = nullptr;
  // the candidates by row (rows sorted by column), for the explicit residuals
  const uint64_t* c_rowptr = nullptr;
  const int32_t* c_col = nullptr;
  const int32_t* c_val = nullptr;
  int64_t n_rows = 0;
  int real = 0;  // the values' payloads hold FP32 values (else integer counts)
};
// keep[du], idx[kept] (device), count (device, = kept), Lk = factor of the
// kept block (kept x kept, lower), Li = Lk^{-1}.
struct FilterOut {
  int* keep = nullptr;
  int* idx = nullptr;
  int* count = nullptr;
  int kept = 0;
  double* Lk = nullptr;
  double* Li = nullptr;
  std::vector<double>* ratios = nullptr;
  // host copies of the final decisions: keep flag, pivot (the squared
  // residual the factorization used) and ||x||^2 per candidate
  std::vector<int> keep_h;
  std::vector<double> piv_h, xn_h;
};
ctd_status run_filter(const FilterIn& in, FilterOut& out, Arena& scratch, cudaStream_t st);

}  // namespace ctd

// The library-owned factors.
struct ctd_factors {
  int kind = 0;          // 0 = CTD-S, 1 = CTD-D
  int alpha = 1;
  int precision = 0;
  cudaStream_t stream = nullptr;
  int64_t dims[3] = {0, 0, 0};
  int64_t n_rows = 0, n_cols = 0;
  uint64_t seed = 0, stream_id = 0;
  // sizes
  int64_t s = 0, s_unique = 0, s_kept = 0, nnz_R = 0, nnz_C = 0, nnz_X = 0;
  uint64_t T = 0;
  bool real = false;             // the values (of X and R) are FP32, not integer counts
  double sqnorm_real = 0.0;      // real values: ||X||_F^2 in FP64
  int min_val = 0;               // CTD-S: the smallest value of X (positive values allow the
                                 // C fill's row copies)
  double err = 0.0;
  bool have_err = false;
  // device arrays (owned)
  ctd::Arena mem;
  int64_t* I = nullptr;          // [s]
  int64_t* Iu = nullptr;         // [s']
  int64_t* fibers = nullptr;     // [s~]
  int* kept_pos = nullptr;       // [s~] positions in I'
  uint64_t* Rcolptr = nullptr;   // [s~+1]
  int32_t* Rrow = nullptr;
  int32_t* Rval = nullptr;
  uint64_t* Rrowptr = nullptr;   // [n_rows+1]
  int32_t* Rcol = nullptr;
  int32_t* Rcval = nullptr;
  double* U = nullptr;           // s~ x s~ column-major (symmetric)
  bool U_valid = false;          // CTD-D: U is formed from L on request and cached
  double* L = nullptr;           // CTD-D: Cholesky factor of R^T R (lower, ld as U)
  double* Qt = nullptr;          // CTD-D: Q^T, Q an orthonormal basis of range(R); row i of Q
                                 // at Qt + i * ld (ld as U), zero past the kept count
  double* qn = nullptr;          // CTD-D: ||Q(i, :)||^2 per row
  uint64_t* Coff = nullptr;      // [n_cols+1]
  uint32_t* Ccnt = nullptr;      // [n_cols]
  uint16_t* Crow = nullptr;
  void* Cval = nullptr;          // float or double
  uint64_t C_cap = 0;
  uint64_t* norm2 = nullptr;     // CTD-S with CTD_KEEP_DIST: [n_cols] squared column norms
  uint64_t* cdf = nullptr;       // and their inclusive prefix sums
  // CTD-D extras live in ctd_dynamic.cu
  struct Dyn;
  Dyn* dyn = nullptr;
  ~ctd_factors();
};

namespace ctd {
// CTD-D views used by the common getters (ctd_dynamic.cu)
ctd_status dyn_sizes(const ctd_factors* F, ctd_sizes* o);
ctd_status dyn_samples(const ctd_factors* F, int64_t* I, int64_t* Iu);
ctd_status dyn_fibers(const ctd_factors* F, int64_t* fiber, int64_t* step);
ctd_status dyn_U(const ctd_factors* F, double* U);
ctd_status dyn_C_columns(const ctd_factors* F, int64_t ncols, const int64_t* cols, double* out);
ctd_status dyn_R(const ctd_factors* F, int64_t* colptr, int32_t* row, int32_t* val);
// CTD_EINVAL if a failed step left this CTD-D state part-way changed; CTD_OK otherwise
ctd_status dyn_check_complete(const ctd_factors* F);
}  // namespace ctd
