// Norm-proportional sampling with replacement (the draws of
// Algorithms 1 and 2) and the unique step.
//
// Draw k of step t in counter space `stream_id` uses Philox4x64-10
// (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2,
// 3", SC'11) with key (seed, 0) and counter (k, t, stream_id, 0).  Its first
// output word u gives the integer target floor(u * T / 2^64) in [0, T),
// T = ||X||_F^2; the drawn column is the smallest f with cdf[f] > target,
// so column f is drawn with probability norm2[f] / T (up to T / 2^64).
#include "ctd_internal.cuh"

namespace ctd {

// Round multipliers and Weyl key increments of Philox4x64 (Salmon et al.).
__device__ __constant__ unsigned long long kPhiloxMul[2] = {0xD2E7470EE14C6C93ull,
                                                            0xCA5A826395121157ull};
__device__ __constant__ unsigned long long kPhiloxWeyl[2] = {0x9E3779B97F4A7C15ull,
                                                             0xBB67AE8584CAA73Bull};

__device__ __forceinline__ void philox4x64_10(unsigned long long x[4], unsigned long long k0,
                                              unsigned long long k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += kPhiloxWeyl[0];
      k1 += kPhiloxWeyl[1];
    }
    const unsigned long long lo0 = kPhiloxMul[0] * x[0];
    const unsigned long long hi0 = __umul64hi(kPhiloxMul[0], x[0]);
    const unsigned long long lo1 = kPhiloxMul[1] * x[2];
    const unsigned long long hi1 = __umul64hi(kPhiloxMul[1], x[2]);
    const unsigned long long y0 = hi1 ^ x[1] ^ k0;
    const unsigned long long y2 = hi0 ^ x[3] ^ k1;
    x[0] = y0;
    x[1] = lo1;
    x[2] = y2;
    x[3] = lo0;
  }
}

// Smallest f in [0, n) with cdf[f] > target (cdf nondecreasing, cdf[n-1] > target).
__device__ __forceinline__ int64_t upper_bound_u64(const unsigned long long* cdf, int64_t n,
                                                   unsigned long long target) {
  int64_t lo = 0, hi = n - 1;
  while (lo < hi) {
    const int64_t mid = lo + ((hi - lo) >> 1);
    if (__ldg(cdf + mid) > target)
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
}

__global__ void k_sample(const unsigned long long* __restrict__ cdf, int64_t n, int64_t s,
                         unsigned long long seed, unsigned long long step,
                         unsigned long long stream_id, int64_t* __restrict__ out) {
  const unsigned long long T = n > 0 ? cdf[n - 1] : 0ull;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < s;
       k += (int64_t)gridDim.x * blockDim.x) {
    if (T == 0) {
      out[k] = -1;  // nothing to draw from (all-zero input)
      continue;
    }
    unsigned long long x[4] = {(unsigned long long)k, step, stream_id, 0ull};
    philox4x64_10(x, seed, 0ull);
    const unsigned long long target = __umul64hi(x[0], T);
    out[k] = upper_bound_u64(cdf, n, target);
  }
}

void launch_sample(const uint64_t* cdf, int64_t n, int64_t s, uint64_t seed, uint64_t step,
                   uint64_t stream_id, int64_t* out, cudaStream_t st) {
  if (s <= 0) return;
  CTD_LAUNCH(k_sample, (grid_for(s, 128, 1024)), (128), 0, st, 
      reinterpret_cast<const unsigned long long*>(cdf), n, s, seed, step, stream_id, out);
}

// ---------------------------------------------------------------------------
// K4: sort-unique of s <= 8192 draws in one block (bitonic sort in shared
// memory, then a flag scan).  Negative entries (no draw) are dropped.
// ---------------------------------------------------------------------------
constexpr int SU_THREADS = 1024;

__global__ void __launch_bounds__(SU_THREADS) k_sort_unique(const int64_t* __restrict__ in,
                                                            int64_t s, int64_t* __restrict__ out,
                                                            int* count) {
  extern __shared__ unsigned long long keys[];  // [npow2]
  __shared__ int wsum[SU_THREADS / 32];
  int npow2 = 1;
  while (npow2 < s) npow2 <<= 1;
  for (int e = threadIdx.x; e < npow2; e += blockDim.x) {
    long long v = e < s ? in[e] : -1;
    keys[e] = v < 0 ? ~0ull : (unsigned long long)v;
  }
  __syncthreads();
  for (int size = 2; size <= npow2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int e = threadIdx.x; e < npow2; e += blockDim.x) {
        const int partner = e ^ stride;
        if (partner > e) {
          const bool up = (e & size) == 0;
          const unsigned long long a = keys[e], b = keys[partner];
          if ((a > b) == up) {
            keys[e] = b;
            keys[partner] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  // keep first of each run; drop the ~0 padding
  int base = 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int chunk = 0; chunk < npow2; chunk += blockDim.x) {
    const int e = chunk + threadIdx.x;
    int flag = 0;
    if (e < npow2) {
      const unsigned long long v = keys[e];
      flag = (v != ~0ull) && (e == 0 || keys[e - 1] != v);
    }
    const unsigned ball = __ballot_sync(0xffffffffu, flag);
    const int wpre = __popc(ball & ((1u << lane) - 1));
    if (lane == 0) wsum[warp] = __popc(ball);
    __syncthreads();
    int before = base;
    int total = 0;
    for (int w = 0; w < SU_THREADS / 32; ++w) {
      if (w < warp) before += wsum[w];
      total += wsum[w];
    }
    if (flag) out[before + wpre] = (int64_t)keys[e];
    __syncthreads();
    base += total;
  }
  if (threadIdx.x == 0) *count = base;
}

void launch_sort_unique(const int64_t* in, int64_t s, int64_t* out, int* count, cudaStream_t st) {
  int npow2 = 1;
  while (npow2 < s) npow2 <<= 1;
  const size_t smem = (size_t)npow2 * sizeof(unsigned long long);
  if (smem > 48 * 1024)
    allow_max_smem((const void*)k_sort_unique);
  CTD_LAUNCH(k_sort_unique, (1), (SU_THREADS), smem, st, in, s, out, count);
}

}  // namespace ctd
