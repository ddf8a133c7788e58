// Open-addressing hash of 8^3 blocks (replaces the paper's OpenVDB tree,
// Sec. III-A): 64-bit block keys, linear probing over single entries from the
// key's hash position, at most max_probe entries (running out raises the
// map's sticky status instead of looping). Warps first drop duplicate keys
// with __match_any_sync; the remaining keys are probed by their lanes in
// parallel, so a warp whose 32 points fall in 32 different blocks (one LiDAR
// azimuth column) pays one probe latency, not 32 serialized ones.
#pragma once
#include "common.cuh"

namespace slim {

__device__ __forceinline__ uint32_t entry_of(const MapView& mv, uint64_t key) {
  return (uint32_t)(mix64(key) & (uint64_t)mv.entry_mask);
}

// Slot of `key`, or kNoSlot when absent. Read-only: valid once every insert
// of the key has completed (in a later kernel than the inserts).
__device__ __forceinline__ uint32_t hash_find(const MapView& mv, uint64_t key) {
  uint32_t h = entry_of(mv, key);
  for (int pr = 0; pr < mv.max_probe; ++pr) {
    const uint64_t cur = mv.hkeys[h];
    if (cur == key) return mv.hvals[h];
    if (cur == kEmptyKey) return kNoSlot;
    h = (h + 1) & mv.entry_mask;
  }
  return kNoSlot;
}

// Insert `key` if absent. Returns the entry index when this thread created
// it (the caller then assigns the slot), -1 when it was present or the probe
// limit ran out (status raised).
__device__ __forceinline__ int64_t hash_insert(const MapView& mv, uint64_t key) {
  uint32_t h = entry_of(mv, key);
  for (int pr = 0; pr < mv.max_probe; ++pr) {
    const uint64_t cur = *(volatile uint64_t*)&mv.hkeys[h];
    if (cur == key) return -1;
    if (cur == kEmptyKey) {
      const unsigned long long prev =
          atomicCAS((unsigned long long*)&mv.hkeys[h], (unsigned long long)kEmptyKey,
                    (unsigned long long)key);
      if (prev == kEmptyKey) return (int64_t)h;
      if (prev == key) return -1;
    }
    h = (h + 1) & mv.entry_mask;
  }
  raise_status(mv.ctr, kDevCapacity, 2);
  return -1;
}

}  // namespace slim
