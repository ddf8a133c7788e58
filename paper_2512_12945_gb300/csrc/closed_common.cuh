// Device helpers shared by the closed-set integration kernels (shared-memory
// hash tiles and direct per-pair reductions).
#pragma once
#include "common.cuh"
#include "internal.h"

namespace slim {

// Bucket of a block key in the tile's block table (a cheap 32-bit mix: the
// table holds a few dozen keys per tile).
__device__ __forceinline__ uint32_t tile_hash(uint64_t kb) {
  uint32_t h = ((uint32_t)kb * 0x9E3779B1u) ^ ((uint32_t)(kb >> 32) * 0x85EBCA77u);
  return h ^ (h >> 15);
}

// Index of the largest of K probabilities (ties to the lowest index). The
// loads of a group of 16 are issued together before any comparison.
__device__ __forceinline__ uint32_t argmax_row(const float* __restrict__ row, int K) {
  float bv = -INFINITY;
  uint32_t best = 0;
  if ((K & 3) == 0 && (reinterpret_cast<uintptr_t>(row) & 15) == 0) {
    const float4* r4 = reinterpret_cast<const float4*>(row);
    const int K4 = K >> 2;
    for (int c = 0; c < K4; c += 4) {
      float4 v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        v[q] = (c + q < K4) ? __ldcs(r4 + c + q)  // read once: evict first from the caches
                            : make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float e[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int k = 4 * (c + q) + u;
          if (k < K && (k == 0 || e[u] > bv)) {
            bv = e[u];
            best = (uint32_t)k;
          }
        }
      }
    }
  } else {
    for (int c = 0; c < K; c += 8) {
      float v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = (c + q < K) ? __ldg(row + c + q) : -INFINITY;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int k = c + q;
        if (k < K && (k == 0 || v[q] > bv)) {
          bv = v[q];
          best = (uint32_t)k;
        }
      }
    }
  }
  return best;
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ int job_of(const HashBatch& b, uint32_t t) {
  int jb = 0;
  while (jb + 1 < b.n_jobs && t >= b.job[jb + 1].tile_begin) ++jb;
  return jb;
}

}  // namespace slim
