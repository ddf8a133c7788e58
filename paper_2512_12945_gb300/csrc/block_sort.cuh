// CTA-level primitives for a 256-thread block: exclusive scan and a stable
// LSD radix sort of 32-bit words in shared memory (8-bit digits; each warp
// owns a contiguous chunk; ranks from __match_any_sync so equal digits keep
// their order).
#pragma once
#include "common.cuh"

namespace slim {

constexpr int kCtaThreads = 256;
constexpr int kCtaWarps = kCtaThreads / 32;

// Exclusive scan of one value per thread; *total gets the sum. warp_tot is
// kCtaWarps words of shared memory. Contains __syncthreads().
__device__ __forceinline__ uint32_t cta_exclusive_scan(uint32_t v, uint32_t* warp_tot,
                                                       uint32_t* total) {
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
    if ((int)lane >= off) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  uint32_t before = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < kCtaWarps; ++w) {
    uint32_t t = warp_tot[w];
    before += (w < (int)warp) ? t : 0u;
    tot += t;
  }
  __syncthreads();
  *total = tot;
  return before + x - v;
}

// Stable sort of a[0..n) by bits [lo, lo + nbits) of each word, using b as
// the ping-pong buffer and hist (256 * kCtaWarps words) as scratch. Returns
// the buffer holding the result. n <= 8192 * kCtaWarps.
__device__ __forceinline__ uint32_t* cta_radix_sort(uint32_t* a, uint32_t* b, int n, int lo,
                                                    int nbits, uint32_t* hist,
                                                    uint32_t* warp_tot) {
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  const int chunk = (n + kCtaWarps - 1) / kCtaWarps;
  const int beg = min(n, (int)warp * chunk), end = min(n, beg + chunk);
  for (int shift = lo; shift < lo + nbits; shift += 8) {
    const int bits = min(8, lo + nbits - shift);
    const uint32_t mask = (1u << bits) - 1u;
    for (int i = threadIdx.x; i < 256 * kCtaWarps; i += kCtaThreads) hist[i] = 0;
    __syncthreads();
    // per-warp digit counts, layout [digit][warp]
    for (int base = beg; base < end; base += 32) {
      const int i = base + lane;
      const bool act = i < end;
      const uint32_t dig = act ? (a[i] >> shift) & mask : 0xFFFFFFFFu;
      const unsigned peers = __match_any_sync(0xFFFFFFFFu, dig);
      if (act && (int)lane == __ffs(peers) - 1) hist[dig * kCtaWarps + warp] += __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    // exclusive scan over the 256 * kCtaWarps counters in (digit, warp) order
    {
      uint32_t loc[kCtaWarps];
      uint32_t s = 0;
#pragma unroll
      for (int k = 0; k < kCtaWarps; ++k) {
        loc[k] = s;
        s += hist[threadIdx.x * kCtaWarps + k];
      }
      uint32_t tot;
      const uint32_t off = cta_exclusive_scan(s, warp_tot, &tot);
#pragma unroll
      for (int k = 0; k < kCtaWarps; ++k) hist[threadIdx.x * kCtaWarps + k] = off + loc[k];
    }
    __syncthreads();
    // scatter: rank among equal digits = earlier lanes this round + running count
    for (int base = beg; base < end; base += 32) {
      const int i = base + lane;
      const bool act = i < end;
      const uint32_t w = act ? a[i] : 0u;
      const uint32_t dig = act ? (w >> shift) & mask : 0xFFFFFFFFu;
      const unsigned peers = __match_any_sync(0xFFFFFFFFu, dig);
      if (act) {
        const uint32_t pos = hist[dig * kCtaWarps + warp] + __popc(peers & ((1u << lane) - 1u));
        b[pos] = w;
      }
      __syncwarp();
      if (act && (int)lane == __ffs(peers) - 1) hist[dig * kCtaWarps + warp] += __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    uint32_t* t = a;
    a = b;
    b = t;
  }
  return a;
}

}  // namespace slim
