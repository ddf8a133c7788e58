// Warp-cooperative open-addressing hash of 8^3 blocks (replaces the paper's
// OpenVDB tree, Sec. III-A): 32-entry buckets, one warp loads a whole bucket
// (256 B, one coalesced transaction) and resolves it with a ballot. Buckets
// are probed linearly for at most max_probe buckets; running out sets the
// map's sticky status instead of looping.
#pragma once
#include "common.cuh"

namespace slim {

__device__ __forceinline__ uint32_t bucket_of(const MapView& mv, uint64_t key) {
  return (uint32_t)(mix64(key) & (uint64_t)mv.bucket_mask);
}

// Slot of `key`, or kNoSlot when absent. All 32 lanes must call it with the
// same key. Read-only: valid once every insert of the key has completed
// (i.e. in a later kernel than the inserts).
__device__ __forceinline__ uint32_t warp_find(const MapView& mv, uint64_t key) {
  const unsigned lane = lane_id();
  uint32_t b = bucket_of(mv, key);
  for (int pr = 0; pr < mv.max_probe; ++pr) {
    const size_t idx = (size_t)b * kBucket + lane;
    const uint64_t cur = mv.hkeys[idx];
    const unsigned f = __ballot_sync(0xFFFFFFFFu, cur == key);
    if (f) {
      const int l = __ffs(f) - 1;
      uint32_t s = 0;
      if ((int)lane == l) s = mv.hvals[idx];
      return __shfl_sync(0xFFFFFFFFu, s, l);
    }
    if (__ballot_sync(0xFFFFFFFFu, cur == kEmptyKey)) return kNoSlot;
    b = (b + 1) & mv.bucket_mask;
  }
  return kNoSlot;
}

// Insert `key` if absent. The warp that wins the key takes a new block slot
// and runs init(slot) cooperatively (all 32 lanes) before publishing the slot
// value. Returns true when this warp created the block. All 32 lanes must
// call it with the same key.
template <class Init>
__device__ __forceinline__ bool warp_insert(const MapView& mv, uint64_t key, Init&& init) {
  const unsigned lane = lane_id();
  uint32_t b = bucket_of(mv, key);
  for (int pr = 0; pr < mv.max_probe; ++pr) {
    const size_t base = (size_t)b * kBucket;
    const uint64_t cur = *(volatile uint64_t*)&mv.hkeys[base + lane];
    if (__ballot_sync(0xFFFFFFFFu, cur == key)) return false;
    unsigned empty = __ballot_sync(0xFFFFFFFFu, cur == kEmptyKey);
    while (empty) {
      const int l = __ffs(empty) - 1;
      int won = 0;
      if ((int)lane == l) {
        const unsigned long long prev = atomicCAS(
            (unsigned long long*)&mv.hkeys[base + l], (unsigned long long)kEmptyKey,
            (unsigned long long)key);
        won = prev == kEmptyKey ? 1 : (prev == key ? 2 : 0);
      }
      won = __shfl_sync(0xFFFFFFFFu, won, l);
      if (won == 2) return false;
      if (won == 1) {
        uint32_t slot = 0;
        if (lane == 0) slot = atomicAdd(&mv.ctr[kCtrBlocks], 1u);
        slot = __shfl_sync(0xFFFFFFFFu, slot, 0);
        if (slot >= mv.block_cap) {
          if (lane == 0) raise_status(mv.ctr, kDevCapacity, 1);
          return false;  // key stays without a slot; later scans skip it
        }
        if (lane == 0) mv.blk_key[slot] = key;
        init(slot);
        __syncwarp();
        __threadfence();
        if (lane == 0) *(volatile uint32_t*)&mv.hvals[base + l] = slot;
        return true;
      }
      empty &= ~(1u << l);
    }
    b = (b + 1) & mv.bucket_mask;
  }
  if (lane == 0) raise_status(mv.ctr, kDevCapacity, 2);
  return false;
}

}  // namespace slim
