// Section 5 (CTD at work): the online DDoS detector on R's fibers.  With
// alpha = 1 (source mode) every fiber of R is the traffic one destination
// received (in one time step); fibers are grouped by destination, the first
// fiber of a destination in R's column order represents it, and a
// destination is a candidate when its representative's 2-norm is above the
// average norm of all representatives.
//
// The paper gives the average no precision; here it does not depend on a
// summation order: every norm is a double >= 1 (the square root of a
// nonzero integer), hence an integer multiple of 2^-52, so the norms are
// added exactly as 128-bit fixed point numbers and the sum is rounded to
// double once.  Any parallel evaluation then gives the same bits as the
// exactly rounded sum.
#include "ctd_internal.cuh"

namespace ctd {
namespace {

constexpr int DD_THREADS = 512;
constexpr int DD_NONE = 0x7f7f7f7f;  // the byte-filled "no column yet" marker

typedef unsigned __int128 u128;

// Pass 1 (one warp per column of R): the destination key, the exact sum of
// squares, and the first column of each destination (the smallest column
// index, i.e. the first in R's column order).
__global__ void k_ddos_columns(const uint64_t* __restrict__ colptr, const int32_t* __restrict__ val,
                               const int64_t* __restrict__ fib, int64_t ncols, int64_t nkeys,
                               int32_t* __restrict__ key, unsigned long long* __restrict__ sq,
                               int* __restrict__ first, unsigned* status) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = gw; c < ncols; c += nw) {
    const int64_t a = (int64_t)colptr[c], b = (int64_t)colptr[c + 1];
    unsigned long long s = 0;
    for (int64_t q = a + lane; q < b; q += 32) {
      const long long v = val[q];
      s += (unsigned long long)(v * v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) {
      const int64_t k = fib[c] % nkeys;
      if (fib[c] < 0) {
        atomicOr(status, DEV_BAD_INDEX);
        key[c] = -1;
      } else {
        key[c] = (int32_t)k;
        atomicMin(first + k, (int)c);
      }
      sq[c] = s;
    }
  }
}

__device__ __forceinline__ double norm_of(unsigned long long s) {
  return __dsqrt_rn(__ull2double_rn(s));
}

// x >= 1 (or 0) as an integer count of 2^-52: integer part times 2^52 plus
// the fraction's 52 bits, both exact.
__device__ __forceinline__ u128 to_fixed(double x) {
  const unsigned long long ip = (unsigned long long)x;  // x < 2^32: exact truncation
  const double fr = x - (double)ip;                     // exact
  const unsigned long long fb = (unsigned long long)(fr * 4503599627370496.0);  // * 2^52, exact
  return ((u128)ip << 52) + fb;
}

// Round V * 2^-52 to the nearest double, ties to even.
__device__ double fixed_to_double(u128 v) {
  if (v == 0) return 0.0;
  const unsigned long long hi = (unsigned long long)(v >> 64), lo = (unsigned long long)v;
  const int n = hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)lo);
  if (n <= 53) return ldexp((double)lo, -52);
  const int sh = n - 53;
  unsigned long long m = (unsigned long long)(v >> sh);
  const u128 rem = v & (((u128)1 << sh) - 1);
  const u128 half = (u128)1 << (sh - 1);
  if (rem > half || (rem == half && (m & 1ull))) ++m;  // m <= 2^53: still exact
  return ldexp((double)m, sh - 52);
}

__device__ __forceinline__ void add128(unsigned long long& hi, unsigned long long& lo,
                                       unsigned long long ohi, unsigned long long olo) {
  const unsigned long long l = lo + olo;
  hi += ohi + (l < lo ? 1ull : 0ull);
  lo = l;
}

// Pass 2 (one block): the exact sum of the representatives' norms and their
// count, the average, then the candidates in ascending destination order.
__global__ void __launch_bounds__(DD_THREADS)
    k_ddos_select(const int32_t* __restrict__ key, const unsigned long long* __restrict__ sq,
                  const int* __restrict__ first, int64_t ncols, int64_t nkeys, int64_t cap,
                  int64_t* __restrict__ out, int64_t* __restrict__ out_n, double* __restrict__ out_mean) {
  __shared__ unsigned long long s_hi[32], s_lo[32], s_cnt[32];
  __shared__ double s_mean;
  __shared__ int s_wsum[32];
  __shared__ long long s_base;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  u128 acc = 0;
  unsigned long long cnt = 0;
  for (int64_t c = tid; c < ncols; c += DD_THREADS) {
    const int k = key[c];
    if (k >= 0 && first[k] == (int)c) {
      acc += to_fixed(norm_of(sq[c]));
      ++cnt;
    }
  }
  unsigned long long hi = (unsigned long long)(acc >> 64), lo = (unsigned long long)acc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ohi = __shfl_down_sync(0xffffffffu, hi, o);
    const unsigned long long olo = __shfl_down_sync(0xffffffffu, lo, o);
    cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    add128(hi, lo, ohi, olo);
  }
  if (lane == 0) {
    s_hi[w] = hi;
    s_lo[w] = lo;
    s_cnt[w] = cnt;
  }
  __syncthreads();
  if (tid == 0) {
    unsigned long long H = 0, Lo = 0, N = 0;
    for (int q = 0; q < DD_THREADS / 32; ++q) {
      add128(H, Lo, s_hi[q], s_lo[q]);
      N += s_cnt[q];
    }
    const double total = fixed_to_double(((u128)H << 64) | Lo);
    s_mean = N ? total / (double)N : 0.0;
    s_base = 0;
    *out_mean = s_mean;
  }
  __syncthreads();
  const double mean = s_mean;
  for (int64_t k0 = 0; k0 < nkeys; k0 += DD_THREADS) {
    const int64_t k = k0 + tid;
    bool flag = false;
    if (k < nkeys) {
      const int c = first[k];
      flag = c != DD_NONE && norm_of(sq[c]) > mean;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, flag);
    if (lane == 0) s_wsum[w] = __popc(bal);
    __syncthreads();
    int before = 0, all = 0;
    for (int q = 0; q < DD_THREADS / 32; ++q) {
      const int v = s_wsum[q];
      before += q < w ? v : 0;
      all += v;
    }
    const long long pos = s_base + before + __popc(bal & ((1u << lane) - 1u));
    if (flag && pos < cap) out[pos] = k;
    __syncthreads();
    if (tid == 0) s_base += all;
    __syncthreads();
  }
  if (tid == 0) *out_n = s_base;
}

}  // namespace
}  // namespace ctd

using namespace ctd;

extern "C" ctd_status ctd_ddos_candidates(const ctd_factors* F, int64_t cap, int64_t* dst,
                                          int64_t* n_found, double* mean_norm) {
  if (!F || !n_found || cap < 0 || (cap > 0 && !dst)) return fail(CTD_EINVAL, "NULL argument or cap < 0");
  if (F->alpha != 1) return fail(CTD_EINVAL, "the detector reads destinations from alpha = 1 fibers");
  if (F->real) return fail(CTD_ENOTSUP, "the detector takes integer counts");
  CTD_TRY(dyn_check_complete(F));
  cudaStream_t st = F->stream;
  const int64_t ncols = F->s_kept, nkeys = F->dims[1];
  *n_found = 0;
  if (mean_norm) *mean_norm = 0.0;
  if (ncols == 0) return sync(st);
  if (ncols >= (int64_t)DD_NONE) return fail(CTD_EINVAL, "too many columns in R");
  PhaseScope ph("ddos", st);
  Arena a;
  a.st = st;
  int32_t* key;
  unsigned long long* sq;
  int* first;
  int64_t *out, *outn;
  double* mean;
  unsigned* status;
  CTD_TRY(a.get(&key, ncols));
  CTD_TRY(a.get(&sq, ncols));
  CTD_TRY(a.get(&first, nkeys));
  CTD_TRY(a.get(&out, std::max<int64_t>(cap, 1)));
  CTD_TRY(a.get(&outn, 1));
  CTD_TRY(a.get(&mean, 1));
  CTD_TRY(a.get(&status, 1));
  CTD_CUDA(cudaMemsetAsync(first, 0x7f, (size_t)nkeys * sizeof(int), st));
  CTD_CUDA(cudaMemsetAsync(status, 0, sizeof(unsigned), st));
  CTD_LAUNCH(k_ddos_columns, (grid_for(ncols * 32, 256, (int64_t)num_sms() * 8)), (256), 0, st,
             F->Rcolptr, F->Rval, F->fibers, ncols, nkeys, key, sq, first, status);
  CTD_LAUNCH(k_ddos_select, (1), (DD_THREADS), 0, st, key, sq, first, ncols, nkeys, cap, out, outn,
             mean);
  unsigned h_status = 0;
  int64_t h_n = 0;
  double h_mean = 0.0;
  CTD_TRY(d2h(&h_status, status, 1, st));
  CTD_TRY(d2h(&h_n, outn, 1, st));
  CTD_TRY(d2h(&h_mean, mean, 1, st));
  CTD_TRY(sync(st));
  if (h_status) return fail(status_from_device(h_status), "bad fiber id in R");
  const int64_t m = std::min(h_n, cap);
  if (m > 0) {
    CTD_TRY(d2h(dst, out, (size_t)m, st));
    CTD_TRY(sync(st));
  }
  *n_found = h_n;
  if (mean_norm) *mean_norm = h_mean;
  return CTD_OK;
}
