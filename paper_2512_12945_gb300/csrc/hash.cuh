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
    const uint32_t v = mv.hvals[h];  // loaded with the key: one round trip
    if (cur == key) return v;
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

// Insert-or-find `key` in the map's hash; returns its slot, or kFailSlot
// after raising a fault (capacity, timeout) on the map's sticky status. A
// created block's slot comes from the allocation counter and is published
// with a relaxed store: the block pools are kept in their initial state
// beyond the counter, so a reader needs nothing else from the creator.
__device__ __forceinline__ uint32_t map_block_slot(const MapView& mv, uint64_t key) {
  uint32_t h = entry_of(mv, key);
  for (int pr = 0; pr < mv.max_probe; ++pr) {
    const uint64_t cur = *(volatile uint64_t*)&mv.hkeys[h];
    // the slot is loaded together with the key, so that finding a published
    // block costs one round trip; read before the key, it can only be older
    // (kNoSlot, then re-read below while unpublished)
    const uint32_t vpre = ld_relaxed(&mv.hvals[h]);
    bool mine = false, found = cur == key;
    if (!found && cur == kEmptyKey) {
      const unsigned long long prev = atomicCAS((unsigned long long*)&mv.hkeys[h],
                                                (unsigned long long)kEmptyKey,
                                                (unsigned long long)key);
      mine = prev == kEmptyKey;
      found = prev == key;
    }
    if (mine) {
      const uint32_t slot = atomicAdd(&mv.ctr[kCtrBlocks], 1u);
      uint32_t v = kFailSlot;
      if (slot >= mv.block_cap) {
        raise_status(mv.ctr, kDevCapacity, 1);
      } else {
        mv.blk_key[slot] = key;
        v = slot;
      }
      st_relaxed(&mv.hvals[h], v);
      return v;
    }
    if (found) {
      uint32_t v = vpre;
      if (v == kNoSlot) {
        const uint64_t t0 = global_ns();
        while ((v = ld_relaxed(&mv.hvals[h])) == kNoSlot) {
          if (global_ns() - t0 > kCrossCtaWaitNs) {
            raise_status(mv.ctr, kDevTimeout, 5);
            return kFailSlot;
          }
          __nanosleep(100);
        }
      }
      return v < mv.block_cap ? v : kFailSlot;
    }
    h = (h + 1) & mv.entry_mask;
  }
  raise_status(mv.ctr, kDevCapacity, 2);
  return kFailSlot;
}

}  // namespace slim
