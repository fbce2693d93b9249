// Warp-level expansion of sparse column entries into R-row work items,
// shared by the sparse-product kernels.
#pragma once
#include <cstdint>

namespace ctd {

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

}  // namespace ctd
