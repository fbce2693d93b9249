// CTD-S on real-valued tensors (Algorithm 1 with X's values in FP32).
//
// The integer path (ctd_api.cu) keeps every stage before U exact in
// integer arithmetic.  With real values only the draws stay exact: the
// sampling weight of a value is its square on a fixed-point grid
// (sample_weight), so the column distribution, the CDF and the draws
// are integers again, exact and the same on every device.  Everything after
// the draws is FP64 on the FP32 inputs (their products are exact in FP64;
// only the order of additions differs from a plain FP64 evaluation):
//   * the Gram matrix of the candidates, as DᵀD with D the candidates as a
//     dense FP64 matrix (the FP64 GEMM), then the same filter as the integer
//     path (the explicit-residual re-test reads the values as FP32);
//   * C = Rᵀ X_(alpha): a warp per column of X accumulates the rows of R its
//     entries select in a shared FP64 accumulator, then emits the nonzeros
//     in ascending row order (sparse form only);
//   * the error through Q = R L^-T (a dense FP64 GEMM), ||Qᵀ x_f||^2 per
//     column by a warp in FP64, summed in a fixed order.
// The stages shared with the integer path move values as 32-bit payloads.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "ctd_internal.cuh"

namespace ctd {
namespace {

// The largest |v| (FP32 bits with the sign cleared: for finite values their
// order is the order of the magnitudes) and whether any value is not
// finite.
__global__ void k_absmax_f32(const int32_t* __restrict__ v, int64_t n, unsigned* out,
                             unsigned* status) {
  unsigned m = 0;
  bool bad = false;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const unsigned a = (unsigned)v[e] & 0x7fffffffu;
    if (a >= 0x7f800000u) bad = true;  // inf or NaN
    else m = max(m, a);
  }
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
  if (bad) atomicOr(status, DEV_BAD_INDEX);
}

// Dense FP64 copy of ncols compressed columns (colptr, row, payloads),
// column-major with leading dimension ld (zeroed beforehand); a block per
// column.
__global__ void k_densify_cols(const unsigned long long* __restrict__ colptr,
                               const int32_t* __restrict__ row, const int32_t* __restrict__ val,
                               const int* __restrict__ ncols_dev, int ncols_max, int64_t ld,
                               double* __restrict__ out) {
  const int nc = min(*ncols_dev, ncols_max);
  for (int c = blockIdx.x; c < nc; c += gridDim.x)
    for (unsigned long long p = colptr[c] + threadIdx.x; p < colptr[c + 1]; p += blockDim.x)
      out[(int64_t)c * ld + row[p]] = (double)__int_as_float(val[p]);
}

// Dense FP64 copy of R by rows: Rd[i * w + c] = R(i, c) (zeroed beforehand).
__global__ void k_dense_rows(const unsigned long long* __restrict__ colptr,
                             const int32_t* __restrict__ row, const int32_t* __restrict__ val,
                             int w, double* __restrict__ Rd) {
  for (int c = blockIdx.x; c < w; c += gridDim.x)
    for (unsigned long long p = colptr[c] + threadIdx.x; p < colptr[c + 1]; p += blockDim.x)
      Rd[(int64_t)row[p] * w + c] = (double)__int_as_float(val[p]);
}

// C = Rᵀ X_(alpha) for real values: a warp per column of X, its entries in
// their stored order, each selecting row i of R (by-row layout, columns
// ascending) scaled by the entry's value, added into the warp's FP64
// accumulator (a row's entries hit distinct accumulator words, so the
// lanes never collide); then the nonzeros are emitted in ascending row
// order from ballots and the accumulator is cleared.
template <typename V>
__global__ void __launch_bounds__(256)
    k_cfill_real(CscDev X, int64_t n_cols, CsrDev R, const unsigned long long* __restrict__ coff,
                 unsigned* __restrict__ ccnt, uint16_t* __restrict__ crow, V* __restrict__ cval) {
  extern __shared__ double accs[];
  const int W = R.width;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* acc = accs + (size_t)warp * W;
  for (int m = lane; m < W; m += 32) acc[m] = 0.0;
  __syncwarp();
  const unsigned long long* rp = reinterpret_cast<const unsigned long long*>(R.rowptr);
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t f = gw; f < n_cols; f += nw) {
    const unsigned long long o = coff[f];
    if (coff[f + 1] == o) {  // no row of R meets this column
      if (lane == 0) ccnt[f] = 0;
      continue;
    }
    for (unsigned long long p = X.colptr[f]; p < X.colptr[f + 1]; ++p) {
      const int i = X.row[p];
      const double v = value_f64(X.val[p], 1);
      for (unsigned long long q = rp[i] + lane; q < rp[i + 1]; q += 32)
        acc[R.col[q]] += v * value_f64(R.val[q], 1);
      __syncwarp();
    }
    unsigned pos = 0;
    for (int m0 = 0; m0 < W; m0 += 32) {
      const int m = m0 + lane;
      const double x = m < W ? acc[m] : 0.0;
      if (m < W) acc[m] = 0.0;
      const unsigned nzb = __ballot_sync(0xffffffffu, x != 0.0);
      if (x != 0.0) {
        const unsigned k = pos + __popc(nzb & ((1u << lane) - 1));
        crow[o + k] = (uint16_t)m;
        cval[o + k] = (V)x;
      }
      pos += __popc(nzb);
    }
    __syncwarp();
    if (lane == 0) ccnt[f] = pos;
  }
}

// ||Qᵀ x_f||^2 per column f of X (Q dense by rows, n_rows x w): a warp per
// column, lane l owning y[m] for m = l, l + 32, ...; the column's entries in
// their stored order, FP64 throughout.
__global__ void __launch_bounds__(256)
    k_qform_real(CscDev X, int64_t n_cols, const double* __restrict__ Q, int w,
                 double* __restrict__ colsum) {
  extern __shared__ double ys[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* y = ys + (size_t)warp * w;
  for (int m = lane; m < w; m += 32) y[m] = 0.0;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t f = gw; f < n_cols; f += nw) {
    const unsigned long long a = X.colptr[f], b = X.colptr[f + 1];
    for (unsigned long long p = a; p < b; ++p) {
      const double v = value_f64(X.val[p], 1);
      const double* q = Q + (int64_t)X.row[p] * w;
      for (int m = lane; m < w; m += 32) y[m] = fma(v, q[m], y[m]);
    }
    double s = 0.0;
    for (int m = lane; m < w; m += 32) {
      s = fma(y[m], y[m], s);
      y[m] = 0.0;
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) colsum[f] = s;
  }
}

// Per block, the sum of squares of the FP32 values in its range, in a
// fixed order (thread-strided, then the warps in order).
__global__ void k_sq_ranges(const int32_t* __restrict__ v, int64_t n, int64_t per,
                            double* __restrict__ out) {
  __shared__ double part[32];
  const int64_t a = (int64_t)blockIdx.x * per, b = min(n, a + per);
  double acc = 0.0;
  for (int64_t e = a + threadIdx.x; e < b; e += blockDim.x) {
    const double x = (double)__int_as_float(v[e]);
    acc = fma(x, x, acc);
  }
  for (int w = 16; w; w >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, w);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    out[blockIdx.x] = t;
  }
}

}  // namespace

// ||X||_F^2 of real values in FP64, summed in a fixed order, into *out.
ctd_status real_sqnorm(const int32_t* v, int64_t nnz, double* out, Arena& scratch,
                       cudaStream_t st) {
  if (nnz <= 0) {
    CTD_CUDA(cudaMemsetAsync(out, 0, sizeof(double), st));
    return CTD_OK;
  }
  const int64_t nb = std::min<int64_t>((int64_t)num_sms() * 4, (nnz + 255) / 256);
  const int64_t per = (nnz + nb - 1) / nb;
  double* part;
  CTD_TRY(scratch.get(&part, nb));
  CTD_LAUNCH(k_sq_ranges, ((unsigned)nb), (256), 0, st, v, nnz, per, part);
  return sum_f64(part, nb, out, scratch, st);
}

// The sampling grid of real values: 2^-wshift = 2^(E - 32)
// with 2^E the smallest power of two above the largest square (wshift = 0
// when every value is zero); CTD_EINVAL for a value that is not finite.
ctd_status real_weight_shift(const int32_t* v, int64_t nnz, int* wshift, Arena& scratch,
                             cudaStream_t st) {
  unsigned *d, h[2] = {0, 0};
  CTD_TRY(scratch.get(&d, 2));
  CTD_CUDA(cudaMemsetAsync(d, 0, 2 * sizeof(unsigned), st));
  if (nnz > 0)
    CTD_LAUNCH(k_absmax_f32, (grid_for(nnz, 256, (int64_t)num_sms() * 8)), (256), 0, st, v, nnz,
               d, d + 1);
  CTD_TRY(d2h(h, d, 2, st));
  CTD_CUDA(cudaGetLastError());
  CTD_TRY(sync(st));
  if (h[1]) return fail(CTD_EINVAL, "a value is not finite");
  float m;
  std::memcpy(&m, &h[0], sizeof(float));
  const double M = (double)m * (double)m;
  int E = 0;
  if (M > 0.0) std::frexp(M, &E);  // M = f 2^E, f in [1/2, 1): M < 2^E
  *wshift = M > 0.0 ? 32 - E : 0;
  return CTD_OK;
}

// The candidates' Gram matrix, real values: G = DᵀD with D (n_rows x su,
// column-major) the candidate columns as dense FP64.
ctd_status real_gram(const uint64_t* cptr, const int32_t* crow, const int32_t* cval,
                     const int* nc_dev, int su, int64_t n_rows, double* G, Arena& scratch,
                     cudaStream_t st) {
  if (su <= 0) return CTD_OK;
  if ((double)n_rows * su > (double)(1ll << 31))
    return fail(CTD_ENOTSUP, "real values: the candidates' dense copy exceeds 2^31 entries");
  double* D;
  CTD_TRY(scratch.get(&D, (size_t)n_rows * su));
  CTD_CUDA(cudaMemsetAsync(D, 0, (size_t)n_rows * su * sizeof(double), st));
  CTD_LAUNCH(k_densify_cols, (grid_for(su, 1, (int64_t)num_sms() * 8)), (256), 0, st,
             reinterpret_cast<const unsigned long long*>(cptr), crow, cval, nc_dev, su, n_rows,
             D);
  dgemm(true, false, su, su, n_rows, 1.0, D, n_rows, D, n_rows, 0.0, G, su, st);
  return CTD_OK;
}

// C = Rᵀ X_(alpha) for real values (sparse columns, ascending rows).
ctd_status real_c_fill(const CscDev& X, int64_t n_cols, const CsrDev& R, const uint64_t* coff,
                       uint32_t* ccnt, uint16_t* crow, void* cval, int fp32, cudaStream_t st) {
  if (n_cols <= 0) return CTD_OK;
  if (R.width <= 0) {
    CTD_CUDA(cudaMemsetAsync(ccnt, 0, n_cols * sizeof(uint32_t), st));
    return CTD_OK;
  }
  int warps = (int)std::min<int64_t>(8, (200 * 1024) / ((int64_t)R.width * 8));
  if (warps < 1) return fail(CTD_ENOTSUP, "real values: too many kept fibers for the C fill");
  const size_t smem = (size_t)warps * R.width * sizeof(double);
  const auto* co = reinterpret_cast<const unsigned long long*>(coff);
  const unsigned g = grid_for(n_cols, warps, (int64_t)num_sms() * 8);
  if (fp32) {
    CTD_TRY(allow_max_smem((const void*)k_cfill_real<float>));
    CTD_LAUNCH(k_cfill_real<float>, (g), (warps * 32), smem, st, X, n_cols, R, co, ccnt, crow,
               static_cast<float*>(cval));
  } else {
    CTD_TRY(allow_max_smem((const void*)k_cfill_real<double>));
    CTD_LAUNCH(k_cfill_real<double>, (g), (warps * 32), smem, st, X, n_cols, R, co, ccnt, crow,
               static_cast<double*>(cval));
  }
  CTD_CUDA(cudaGetLastError());
  return CTD_OK;
}

// ||Qᵀ X_(alpha)||_F^2 for real values, Q = R Zᵀ with Z = L^-1 (kept x kept,
// column-major, ld ldz): R dense by rows, Qᵀ = Z Rdᵀ by the FP64 GEMM, the
// per-column norms by k_qform_real, summed in a fixed order into *out.
ctd_status real_error_qform(const CscDev& X, int64_t n_cols, int64_t n_rows,
                            const uint64_t* Rcolptr, const int32_t* Rrow, const int32_t* Rval,
                            int kept, const double* Z, int64_t ldz, double* out, Arena& scratch,
                            cudaStream_t st) {
  if (kept <= 0 || n_cols <= 0) {
    CTD_CUDA(cudaMemsetAsync(out, 0, sizeof(double), st));
    return CTD_OK;
  }
  if ((double)n_rows * kept > (double)(1ll << 31))
    return fail(CTD_ENOTSUP, "real values: the dense copy of R exceeds 2^31 entries");
  double *Rd, *Q, *colsum;
  CTD_TRY(scratch.get(&Rd, (size_t)n_rows * kept));
  CTD_TRY(scratch.get(&Q, (size_t)n_rows * kept));
  CTD_TRY(scratch.get(&colsum, (size_t)n_cols));
  CTD_CUDA(cudaMemsetAsync(Rd, 0, (size_t)n_rows * kept * sizeof(double), st));
  CTD_LAUNCH(k_dense_rows, (grid_for(kept, 1, (int64_t)num_sms() * 8)), (256), 0, st,
             reinterpret_cast<const unsigned long long*>(Rcolptr), Rrow, Rval, kept, Rd);
  // Q by rows (n_rows x kept) is Qᵀ column-major: Qᵀ = Z Rdᵀ
  dgemm(false, false, kept, n_rows, kept, 1.0, Z, ldz, Rd, kept, 0.0, Q, kept, st);
  int warps = (int)std::min<int64_t>(8, (200 * 1024) / ((int64_t)kept * 8));
  if (warps < 1) return fail(CTD_ENOTSUP, "real values: too many kept fibers for the error");
  const size_t smem = (size_t)warps * kept * sizeof(double);
  CTD_TRY(allow_max_smem((const void*)k_qform_real));
  CTD_LAUNCH(k_qform_real, (grid_for(n_cols, warps, (int64_t)num_sms() * 8)), (warps * 32), smem,
             st, X, n_cols, Q, kept, colsum);
  CTD_TRY(sum_f64(colsum, n_cols, out, scratch, st));
  CTD_CUDA(cudaGetLastError());
  return CTD_OK;
}

}  // namespace ctd
