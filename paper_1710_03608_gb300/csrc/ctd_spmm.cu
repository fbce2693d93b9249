// Sparse products with the factor R:
//   * dense columns  out(:, c) = R^T x_f      (the Gram matrices of the
//     independence filter, Algorithm 1 lines 6-15 / Algorithm 2 lines 6-16),
//   * the sparse core C_(alpha) = R^T X_(alpha) (Algorithm 1 line 16, Eq. 3),
//   * the Gram form of the error numerator R^T (X_(alpha) X_(alpha)^T) R,
//     which with U gives ||P_R X||_F^2 = <U, C C^T> (Eq. error, Lemma 3.2).
//
// Every product is an exact integer sum (int32 x int32 -> int64 terms).
// Column f of X is expanded into (row entry of R) work items which a warp
// spreads over its lanes; partial sums go to a dense int64 accumulator in
// shared memory and a bitmap marks the touched rows of R^T x_f, so results
// come out in ascending row order without a sort.
#include "ctd_internal.cuh"

namespace ctd {

constexpr int WARP_MODE_MAX_WIDTH = 1024;  // accumulator per warp
constexpr int CTA_MODE_MAX_WIDTH = 24576;  // accumulator per block
constexpr int SPMM_THREADS = 256;

// Expand 32 column entries (one per lane) into their R-row work items and
// apply fn(m, product) to every item.  Lanes without an entry pass rlen=0.
template <typename Fn>
__device__ __forceinline__ void expand_chunk(unsigned long long rstart, int rlen, int v,
                                             const int32_t* __restrict__ rcol,
                                             const int32_t* __restrict__ rval, Fn fn) {
  const int lane = threadIdx.x & 31;
  int incl = rlen;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  const int excl = incl - rlen;
  for (int base = 0; base < total; base += 32) {
    const int t = base + lane;
    // owner = smallest lane with incl > t
    int lo = 0, hi = 31;
#pragma unroll
    for (int it = 0; it < 5; ++it) {
      const int mid = (lo + hi) >> 1;
      const int im = __shfl_sync(0xffffffffu, incl, mid);
      if (im > t)
        hi = mid;
      else
        lo = mid + 1;
    }
    const int owner = lo;
    const unsigned long long os = __shfl_sync(0xffffffffu, rstart, owner);
    const int oe = __shfl_sync(0xffffffffu, excl, owner);
    const int ov = __shfl_sync(0xffffffffu, v, owner);
    if (t < total) {
      const unsigned long long q = os + (unsigned long long)(t - oe);
      const int m = __ldg(rcol + q);
      const long long prod = (long long)ov * (long long)__ldg(rval + q);
      fn(m, prod);
    }
  }
}

// Accumulate R^T x_f for column f into acc/bitmap; warps of the group
// [gwarp0, gwarp0 + gwarps) take interleaved 32-entry chunks.
__device__ __forceinline__ void accumulate_column(const CscDev& X, const CsrDev& R, int64_t f,
                                                  unsigned long long* acc, unsigned* bitmap,
                                                  int gwarp, int gwarps) {
  const unsigned long long a = X.colptr[f], b = X.colptr[f + 1];
  const int lane = threadIdx.x & 31;
  for (unsigned long long p0 = a + (unsigned long long)gwarp * 32; p0 < b;
       p0 += (unsigned long long)gwarps * 32) {
    const unsigned long long p = p0 + lane;
    unsigned long long rs = 0;
    int rl = 0, v = 0;
    if (p < b) {
      const int i = __ldg(X.row + p);
      v = __ldg(X.val + p);
      rs = __ldg(reinterpret_cast<const unsigned long long*>(R.rowptr) + i);
      rl = (int)(__ldg(reinterpret_cast<const unsigned long long*>(R.rowptr) + i + 1) - rs);
    }
    expand_chunk(rs, rl, v, R.col, R.val, [&](int m, long long prod) {
      atomicAdd(acc + m, (unsigned long long)prod);
      if (bitmap) atomicOr(bitmap + (m >> 5), 1u << (m & 31));
    });
  }
}

// ---------------------------------------------------------------------------
// dense output (one block per column)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(SPMM_THREADS)
    k_spmm_dense(CscDev X, const int64_t* __restrict__ fibers, const int* nf_dev, int nf_max,
                 CsrDev R, double* __restrict__ out, int64_t ld) {
  extern __shared__ unsigned long long acc[];
  const int nf = min(*nf_dev, nf_max);
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int m = threadIdx.x; m < R.width; m += blockDim.x) acc[m] = 0;
  __syncthreads();
  for (int c = blockIdx.x; c < nf; c += gridDim.x) {
    accumulate_column(X, R, fibers[c], acc, nullptr, warp, nw);
    __syncthreads();
    for (int m = threadIdx.x; m < R.width; m += blockDim.x) {
      out[(int64_t)c * ld + m] = (double)(long long)acc[m];
      acc[m] = 0;
    }
    __syncthreads();
  }
}

ctd_status launch_spmm_dense(const CscDev& X, const int64_t* fibers, const int* nf_dev,
                             int nf_max, const CsrDev& R, double* out, int64_t ld,
                             cudaStream_t st) {
  if (nf_max <= 0 || R.width <= 0) return CTD_OK;
  if (R.width > CTA_MODE_MAX_WIDTH)
    return fail(CTD_EINVAL, "factor wider than the supported maximum (24576 columns)");
  const size_t smem = (size_t)R.width * sizeof(unsigned long long);
  if (smem > 48 * 1024)
    CTD_CUDA(cudaFuncSetAttribute(k_spmm_dense, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
  unsigned g = (unsigned)std::min<int64_t>(nf_max, (int64_t)num_sms() * 4);
  CTD_LAUNCH(k_spmm_dense, (g), (SPMM_THREADS), smem, st, X, fibers, nf_dev, nf_max, R, out, ld);
  CTD_CUDA(cudaGetLastError());
  return CTD_OK;
}

// ---------------------------------------------------------------------------
// C bounds: ub[f] = min(width, sum over column f of R row lengths)
// ---------------------------------------------------------------------------
__global__ void k_c_bounds(CscDev X, int64_t n_cols, CsrDev R, unsigned* __restrict__ ub) {
  const unsigned long long* rp = reinterpret_cast<const unsigned long long*>(R.rowptr);
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < n_cols;
       f += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long a = X.colptr[f], b = X.colptr[f + 1];
    unsigned long long s = 0;
    for (unsigned long long p = a; p < b && s < (unsigned long long)R.width; ++p) {
      const int i = __ldg(X.row + p);
      s += __ldg(rp + i + 1) - __ldg(rp + i);
    }
    ub[f] = (unsigned)min(s, (unsigned long long)R.width);
  }
}

void launch_c_bounds(const CscDev& X, int64_t n_cols, const CsrDev& R, uint32_t* ub,
                     cudaStream_t st) {
  if (n_cols <= 0) return;
  CTD_LAUNCH(k_c_bounds, (grid_for(n_cols, 256, (int64_t)num_sms() * 16)), (256), 0, st, X, n_cols, R, ub);
}

// ---------------------------------------------------------------------------
// C fill
// ---------------------------------------------------------------------------
template <typename V>
__device__ __forceinline__ V convert_exact(long long x) {
  return (V)x;
}

// Emit the touched entries of acc (ascending m) for one column, zeroing
// them.  Group = `gthreads` threads starting at thread `gtid0` (a warp or the
// whole block).  wpre: scratch with nwords+1 ints for this group.
template <typename V>
__device__ void emit_column(unsigned long long* acc, unsigned* bitmap, int width, int* wpre,
                            int gtid, int gthreads, bool may_cancel, unsigned long long off,
                            int32_t* __restrict__ crow, V* __restrict__ cval, int* total_out,
                            bool block_group) {
  const int nwords = (width + 31) >> 5;
  // drop exact zeros (only possible with signed inputs)
  if (may_cancel) {
    for (int w = gtid; w < nwords; w += gthreads) {
      unsigned bits = bitmap[w], keep = bits;
      while (bits) {
        const int bpos = __ffs(bits) - 1;
        bits &= bits - 1;
        if (acc[w * 32 + bpos] == 0ull) keep &= ~(1u << bpos);
      }
      bitmap[w] = keep;
    }
    if (block_group) __syncthreads(); else __syncwarp();
  }
  // word prefix counts (sequential over chunks of gthreads words)
  int carry = 0;
  for (int w0 = 0; w0 < nwords; w0 += gthreads) {
    const int w = w0 + gtid;
    const int c = w < nwords ? __popc(bitmap[w]) : 0;
    // inclusive scan over the group
    int incl = c;
    const int lane = gtid & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (block_group) {
      __shared__ int wtot[32];
      const int warp = gtid >> 5;
      if (lane == 31) wtot[warp] = incl;
      __syncthreads();
      int before = 0;
      for (int q = 0; q < warp; ++q) before += wtot[q];
      int all = 0;
      for (int q = 0; q < (gthreads >> 5); ++q) all += wtot[q];
      if (w < nwords) wpre[w] = carry + before + incl - c;
      __syncthreads();
      carry += all;
    } else {
      if (w < nwords) wpre[w] = carry + incl - c;
      carry += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
  if (gtid == 0) wpre[nwords] = carry;
  if (block_group) __syncthreads(); else __syncwarp();
  const int total = carry;
  for (int k = gtid; k < total; k += gthreads) {
    // word containing the k-th set bit: largest w with wpre[w] <= k
    int lo = 0, hi = nwords - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (wpre[mid] <= k)
        lo = mid;
      else
        hi = mid - 1;
    }
    const unsigned bits = bitmap[lo];
    const int bpos = __fns(bits, 0, k - wpre[lo] + 1);
    const int m = lo * 32 + bpos;
    const long long x = (long long)acc[m];
    crow[off + k] = m;
    cval[off + k] = convert_exact<V>(x);
  }
  if (block_group) __syncthreads(); else __syncwarp();
  // zero what was touched (including dropped exact zeros)
  for (int w = gtid; w < nwords; w += gthreads) bitmap[w] = 0;
  for (int m = gtid; m < width; m += gthreads) acc[m] = 0;
  if (block_group) __syncthreads(); else __syncwarp();
  if (total_out && gtid == 0) *total_out = total;
}

// Warp mode: each warp owns an accumulator and takes columns from a global
// counter in chunks.
template <typename V>
__global__ void __launch_bounds__(SPMM_THREADS)
    k_c_fill_warp(CscDev X, int64_t n_cols, CsrDev R, const unsigned long long* __restrict__ coff,
                  unsigned* __restrict__ ccnt, int32_t* __restrict__ crow, V* __restrict__ cval,
                  int may_cancel, unsigned long long* work) {
  extern __shared__ unsigned long long smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int width = R.width, nwords = (width + 31) >> 5;
  unsigned long long* acc = smem + (size_t)warp * width;
  unsigned* bitmaps = reinterpret_cast<unsigned*>(smem + (size_t)nw * width);
  unsigned* bitmap = bitmaps + warp * nwords;
  int* wpres = reinterpret_cast<int*>(bitmaps + nw * nwords);
  int* wpre = wpres + warp * (nwords + 1);
  for (int m = lane; m < width; m += 32) acc[m] = 0;
  for (int w = lane; w < nwords; w += 32) bitmap[w] = 0;
  __syncwarp();
  constexpr int CHUNK = 64;
  while (true) {
    unsigned long long f0 = 0;
    if (lane == 0) f0 = atomicAdd(work, (unsigned long long)CHUNK);
    f0 = __shfl_sync(0xffffffffu, f0, 0);
    if (f0 >= (unsigned long long)n_cols) break;
    const int64_t f1 = min((int64_t)f0 + CHUNK, n_cols);
    for (int64_t f = (int64_t)f0; f < f1; ++f) {
      const unsigned long long o = coff[f];
      if (coff[f + 1] == o) {
        if (lane == 0) ccnt[f] = 0;
        continue;
      }
      accumulate_column(X, R, f, acc, bitmap, 0, 1);
      __syncwarp();
      int total = 0;
      emit_column<V>(acc, bitmap, width, wpre, lane, 32, may_cancel != 0, o, crow, cval, &total,
                     false);
      if (lane == 0) ccnt[f] = (unsigned)total;
    }
  }
}

// Block mode: the whole block works on one column at a time.
template <typename V>
__global__ void __launch_bounds__(SPMM_THREADS)
    k_c_fill_block(CscDev X, int64_t n_cols, CsrDev R, const unsigned long long* __restrict__ coff,
                   unsigned* __restrict__ ccnt, int32_t* __restrict__ crow, V* __restrict__ cval,
                   int may_cancel, unsigned long long* work) {
  extern __shared__ unsigned long long smem[];
  const int width = R.width, nwords = (width + 31) >> 5;
  unsigned long long* acc = smem;
  unsigned* bitmap = reinterpret_cast<unsigned*>(smem + width);
  int* wpre = reinterpret_cast<int*>(bitmap + nwords);
  __shared__ unsigned long long fcur;
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int m = threadIdx.x; m < width; m += blockDim.x) acc[m] = 0;
  for (int w = threadIdx.x; w < nwords; w += blockDim.x) bitmap[w] = 0;
  __syncthreads();
  while (true) {
    if (threadIdx.x == 0) fcur = atomicAdd(work, 1ull);
    __syncthreads();
    const unsigned long long f = fcur;
    __syncthreads();
    if (f >= (unsigned long long)n_cols) break;
    const unsigned long long o = coff[f];
    if (coff[f + 1] == o) {
      if (threadIdx.x == 0) ccnt[f] = 0;
      continue;
    }
    accumulate_column(X, R, (int64_t)f, acc, bitmap, warp, nw);
    __syncthreads();
    int total = 0;
    emit_column<V>(acc, bitmap, width, wpre, threadIdx.x, blockDim.x, may_cancel != 0, o, crow,
                   cval, &total, true);
    if (threadIdx.x == 0) ccnt[f] = (unsigned)total;
  }
}

template <typename V>
static ctd_status c_fill_impl(const CscDev& X, int64_t n_cols, const CsrDev& R,
                              const uint64_t* coff, uint32_t* ccnt, int32_t* crow, V* cval,
                              int may_cancel, unsigned long long* work, cudaStream_t st) {
  const int width = R.width, nwords = (width + 31) >> 5;
  if (width <= WARP_MODE_MAX_WIDTH) {
    const int nw = SPMM_THREADS / 32;
    const size_t smem = (size_t)nw * width * 8 + (size_t)nw * nwords * 4 +
                        (size_t)nw * (nwords + 1) * 4;
    if (smem > 48 * 1024)
      CTD_CUDA(cudaFuncSetAttribute(k_c_fill_warp<V>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    CTD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_c_fill_warp<V>,
                                                           SPMM_THREADS, smem));
    if (per_sm < 1) per_sm = 1;
    CTD_LAUNCH(k_c_fill_warp<V>, (num_sms() * per_sm), (SPMM_THREADS), smem, st, 
        X, n_cols, R, reinterpret_cast<const unsigned long long*>(coff), ccnt, crow, cval,
        may_cancel, work);
  } else {
    if (width > CTA_MODE_MAX_WIDTH)
      return fail(CTD_EINVAL, "factor wider than the supported maximum (24576 columns)");
    const size_t smem = (size_t)width * 8 + (size_t)nwords * 4 + (size_t)(nwords + 1) * 4;
    if (smem > 48 * 1024)
      CTD_CUDA(cudaFuncSetAttribute(k_c_fill_block<V>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    CTD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_c_fill_block<V>,
                                                           SPMM_THREADS, smem));
    if (per_sm < 1) per_sm = 1;
    CTD_LAUNCH(k_c_fill_block<V>, (num_sms() * per_sm), (SPMM_THREADS), smem, st, 
        X, n_cols, R, reinterpret_cast<const unsigned long long*>(coff), ccnt, crow, cval,
        may_cancel, work);
  }
  CTD_CUDA(cudaGetLastError());
  return CTD_OK;
}

ctd_status launch_c_fill(const CscDev& X, int64_t n_cols, const CsrDev& R, const uint64_t* coff,
                         uint32_t* ccnt, int32_t* crow, void* cval, int fp32, int may_cancel,
                         cudaStream_t st) {
  if (n_cols <= 0) return CTD_OK;
  unsigned long long* work;
  CTD_TRY(dalloc_n(&work, 1, st));
  CTD_CUDA(cudaMemsetAsync(work, 0, sizeof(unsigned long long), st));
  ctd_status rc;
  if (R.width <= 0) {
    CTD_CUDA(cudaMemsetAsync(ccnt, 0, n_cols * sizeof(uint32_t), st));
    rc = CTD_OK;
  } else if (fp32) {
    rc = c_fill_impl<float>(X, n_cols, R, coff, ccnt, crow, static_cast<float*>(cval), may_cancel,
                            work, st);
  } else {
    rc = c_fill_impl<double>(X, n_cols, R, coff, ccnt, crow, static_cast<double*>(cval),
                             may_cancel, work, st);
  }
  dfree(work, st);
  return rc;
}

// ---------------------------------------------------------------------------
// Gram form of the error numerator: CCt = R^T H R with H = X_(alpha) X_(alpha)^T.
// Work item = (row i of R's support, chunk of X's row i).  For the chunk,
// h = sum over its entries (f, x_if) of x_if * x_f  (dense over rows, in
// shared memory), w = R^T h, and CCt(m, :) += R(i, m) * w for m in row i of R.
// By linearity the chunks of one row add up to r_i (H R)(i, :).
// ---------------------------------------------------------------------------
constexpr int HF_CHUNK = 2048;
constexpr int HF_MAX_ROWS = 16384;  // int64 h in shared memory
constexpr int HF_MAX_WIDTH = 8192;

__global__ void k_hform_items(const unsigned long long* __restrict__ xrowptr,
                              const unsigned long long* __restrict__ rrowptr, int64_t n_rows,
                              unsigned* __restrict__ items) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_rows;
       i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long xl = xrowptr[i + 1] - xrowptr[i];
    const unsigned long long rl = rrowptr[i + 1] - rrowptr[i];
    items[i] = (rl > 0 && xl > 0) ? (unsigned)((xl + HF_CHUNK - 1) / HF_CHUNK) : 0u;
  }
}

__global__ void __launch_bounds__(SPMM_THREADS)
    k_hform(CsrX Xr, CscDev Xc, int64_t n_rows, CsrDev R,
            const unsigned long long* __restrict__ item_off, long long* __restrict__ CCt,
            unsigned long long* work) {
  extern __shared__ unsigned long long sm[];
  unsigned long long* h = sm;                 // [n_rows]
  unsigned long long* w = sm + n_rows;        // [width]
  __shared__ unsigned long long cur;
  const int width = R.width;
  const unsigned long long n_items = item_off[n_rows];
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5, lane = threadIdx.x & 31;
  const unsigned long long* rp = reinterpret_cast<const unsigned long long*>(R.rowptr);
  for (int64_t q = threadIdx.x; q < n_rows; q += blockDim.x) h[q] = 0;
  for (int m = threadIdx.x; m < width; m += blockDim.x) w[m] = 0;
  __syncthreads();
  while (true) {
    if (threadIdx.x == 0) cur = atomicAdd(work, 1ull);
    __syncthreads();
    const unsigned long long it = cur;
    __syncthreads();
    if (it >= n_items) break;
    // row i: largest i with item_off[i] <= it
    int64_t lo = 0, hi = n_rows - 1;
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) >> 1;
      if (item_off[mid] <= it)
        lo = mid;
      else
        hi = mid - 1;
    }
    const int64_t i = lo;
    const unsigned long long c = it - item_off[i];
    const unsigned long long xa = (unsigned long long)Xr.rowptr[i] + c * HF_CHUNK;
    const unsigned long long xb = min((unsigned long long)Xr.rowptr[i + 1], xa + (unsigned long long)HF_CHUNK);
    // h = sum_{(f, x) in chunk} x * X(:, f)
    for (unsigned long long e = xa + warp; e < xb; e += nw) {
      const int f = __ldg(Xr.col + e);
      const long long xv = __ldg(Xr.val + e);
      const unsigned long long a = Xc.colptr[f], b = Xc.colptr[f + 1];
      for (unsigned long long p = a + lane; p < b; p += 32)
        atomicAdd(h + __ldg(Xc.row + p), (unsigned long long)(xv * (long long)__ldg(Xc.val + p)));
    }
    __syncthreads();
    // w = R^T h (rows q with h[q] != 0), zero h on the way
    for (int64_t q = threadIdx.x; q < n_rows; q += blockDim.x) {
      const long long hq = (long long)h[q];
      if (hq != 0) {
        h[q] = 0;
        for (unsigned long long r = rp[q]; r < rp[q + 1]; ++r)
          atomicAdd(w + __ldg(R.col + r), (unsigned long long)(hq * (long long)__ldg(R.val + r)));
      }
    }
    __syncthreads();
    // CCt(m, :) += R(i, m) * w
    for (unsigned long long r = rp[i]; r < rp[i + 1]; ++r) {
      const int m = __ldg(R.col + r);
      const long long rv = __ldg(R.val + r);
      for (int m2 = threadIdx.x; m2 < width; m2 += blockDim.x) {
        const long long wv = (long long)w[m2];
        if (wv != 0) atomicAdd(reinterpret_cast<unsigned long long*>(CCt + (int64_t)m2 * width + m),
                               (unsigned long long)(rv * wv));
      }
    }
    __syncthreads();
    for (int m = threadIdx.x; m < width; m += blockDim.x) w[m] = 0;
    __syncthreads();
  }
}

ctd_status launch_gram_hform(const CsrX& Xr, const CscDev& Xc, int64_t n_rows, const CsrDev& R,
                             long long* CCt, Arena& scratch, cudaStream_t st) {
  if (R.width <= 0 || n_rows <= 0) return CTD_OK;
  if (n_rows > HF_MAX_ROWS || R.width > HF_MAX_WIDTH)
    return fail(CTD_ENOTSUP, "error form limited to I_alpha <= 16384 and s~ <= 8192");
  unsigned* items;
  uint64_t* item_off;
  uint64_t* tmp;
  unsigned* status;
  unsigned long long* work;
  CTD_TRY(scratch.get(&items, n_rows));
  CTD_TRY(scratch.get(&item_off, n_rows + 1));
  CTD_TRY(scratch.get(&tmp, scan_tmp_elems(n_rows)));
  CTD_TRY(scratch.get(&status, 1));
  CTD_TRY(scratch.get(&work, 1));
  CTD_CUDA(cudaMemsetAsync(status, 0, 4, st));
  CTD_CUDA(cudaMemsetAsync(work, 0, 8, st));
  CTD_LAUNCH(k_hform_items, (grid_for(n_rows, 256, 1024)), (256), 0, st, 
      reinterpret_cast<const unsigned long long*>(Xr.rowptr),
      reinterpret_cast<const unsigned long long*>(R.rowptr), n_rows, items);
  launch_scan_u32(items, item_off, n_rows, false, tmp, status, st);
  const size_t smem = (size_t)(n_rows + R.width) * 8;
  if (smem > 48 * 1024)
    CTD_CUDA(cudaFuncSetAttribute(k_hform, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  CTD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hform, SPMM_THREADS, smem));
  if (per_sm < 1) per_sm = 1;
  CTD_LAUNCH(k_hform, (num_sms() * per_sm), (SPMM_THREADS), smem, st, 
      Xr, Xc, n_rows, R, reinterpret_cast<const unsigned long long*>(item_off), CCt, work);
  CTD_CUDA(cudaGetLastError());
  return CTD_OK;
}

// <U, CCt> in FP64 (deterministic two-level reduction)
__global__ void k_frob_dot(const double* __restrict__ U, const long long* __restrict__ CCt,
                           int64_t nn, double* out) {
  __shared__ double part[32];
  double acc = 0.0;
  for (int64_t e = threadIdx.x; e < nn; e += blockDim.x) acc += U[e] * (double)CCt[e];
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    *out = t;
  }
}

void launch_frob_dot(const double* U, const long long* CCt, int64_t n, double* out,
                     cudaStream_t st) {
  CTD_LAUNCH(k_frob_dot, (1), (1024), 0, st, U, CCt, n * n, out);
}

}  // namespace ctd
