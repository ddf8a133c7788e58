// Closed-set scan integration (Sec. III-A TSDF + Sec. III-C Dirichlet counts).
//
// One kernel per scan, k_fuse_closed, one 256-point tile per CTA:
//   1. band DDA per point; every kept (voxel, point) pair goes to shared
//      memory as (tile block, local voxel, d), pair k of point t at k * 256 + t
//      (bank-conflict free); the tile's distinct blocks go to a shared table;
//   2. each distinct block is inserted into (or found in) the map's hash by
//      its own thread; blocks this CTA creates are zeroed by the whole CTA and
//      then published, and only then does the CTA wait (time-bounded) for
//      blocks other CTAs are still publishing — every CTA publishes before it
//      waits, so no wait can be part of a cycle;
//   3. the pairs are sorted by voxel key (stable CTA radix sort) and reduced
//      per voxel run with warp shuffles; one red.add per voxel (and per
//      present class) goes to HBM instead of one atomic per pair.
//
// Voxel records (AoS, rs floats, 16-byte aligned; layouts in common.cuh)
// keep sums: S = W * D instead of D. With w~ = 1 the paper's running average
// D_t = (W_{t-1} D_{t-1} + d_t) / W_t is the same as S_t = S_{t-1} + d_t,
// W_t = W_{t-1} + 1 and D = S / W at read-out; keeping S makes every update
// of a scan an addition, so partial sums from different tiles merge exactly
// in any order (Theorem 1 for the counts). One-hot records split S and W by
// class, so one vector reduction carries a (voxel, class) partial.
#include "block_sort.cuh"
#include "common.cuh"
#include "geometry.cuh"
#include "hash.cuh"
#include "internal.h"

namespace slim {

constexpr int kTileCap = 6144;        // (voxel, point) pairs per tile
constexpr int kTblSize = 2048;        // tile block table (open addressing)
constexpr int kMaxTileBlocks = 1024;  // distinct blocks per tile
constexpr int kMaxBandBlocks = 8;     // distinct blocks per point band

// ------------------------------------------------------------------ K2
// Insert a block key into the tile's shared table; returns its entry.
__device__ __forceinline__ uint32_t tbl_insert(uint64_t* tb, uint64_t kb) {
  uint32_t h = (uint32_t)mix64(kb) & (kTblSize - 1);
  for (int it = 0; it < kTblSize; ++it) {
    const uint64_t cur = *(volatile uint64_t*)&tb[h];
    if (cur == kb) return h;
    if (cur == kEmptyKey) {
      const unsigned long long prev = atomicCAS((unsigned long long*)&tb[h],
                                                (unsigned long long)kEmptyKey,
                                                (unsigned long long)kb);
      if (prev == kEmptyKey || prev == kb) return h;
    }
    h = (h + 1) & (kTblSize - 1);
  }
  return 0xFFFFFFFFu;
}

size_t closed_smem_bytes(int mode, int K, int tile_points) {
  size_t b = kTblSize * 8 + kMaxTileBlocks * 4 + kTblSize * 2 + 3 * kTileCap * 4 +
             256 * kCtaWarps * 4 + 16 * 4 + 256;
  if (mode == 1) b += (size_t)tile_points * K * 4;
  return b;
}

template <int MODE>  // 0: one-hot counts, 1: soft counts
__global__ void __launch_bounds__(256, 2)
    k_fuse_closed(MapView mv, ScanGeom g, const float* __restrict__ pts,
                  const float* __restrict__ sem, int64_t n, int K, int tile_points) {
  extern __shared__ __align__(16) unsigned char sm[];
  uint64_t* tb_key = reinterpret_cast<uint64_t*>(sm);
  uint32_t* tb_slot = reinterpret_cast<uint32_t*>(tb_key + kTblSize);
  uint16_t* tb_dense = reinterpret_cast<uint16_t*>(tb_slot + kMaxTileBlocks);
  uint32_t* sA = reinterpret_cast<uint32_t*>(tb_dense + kTblSize);
  uint32_t* sB = sA + kTileCap;
  float* pd = reinterpret_cast<float*>(sB + kTileCap);
  uint32_t* hist = reinterpret_cast<uint32_t*>(pd + kTileCap);
  uint32_t* wtot = hist + 256 * kCtaWarps;
  uint32_t* misc = wtot + 8;
  uint8_t* cls = reinterpret_cast<uint8_t*>(misc + 8);
  float* probs = reinterpret_cast<float*>(cls + 256);

  const int tid = threadIdx.x;
  const unsigned lane = lane_id(), warp = tid >> 5;
  if (tid == 0) {
    misc[0] = *(volatile uint32_t*)&mv.ctr[kCtrStatus];
    misc[2] = 0;
  }
  for (int e = tid; e < kTblSize; e += kCtaThreads) tb_key[e] = kEmptyKey;
  __syncthreads();
  if (misc[0]) return;

  // 1. band DDA: pair k of this thread's point at raw index k * tile + tid
  const int64_t j = (int64_t)blockIdx.x * tile_points + tid;
  const int tp_shift = 31 - __clz(tile_points);  // tile_points is a power of two
  int np = 0;
  uint8_t mycls = 0;
  if (tid < tile_points && j < n) {
    Ray ry;
    if (ray_setup_at(g, pts, j, ry)) {
      const float* srow = sem + (size_t)j * K;
      if (MODE == 0) {
        int best = 0;
        float bv = srow[0];
        for (int k = 1; k < K; ++k) {
          const float v = srow[k];
          if (v > bv) {
            bv = v;
            best = k;
          }
        }
        mycls = (uint8_t)best;
      } else {
        for (int k = 0; k < K; ++k) probs[tid * K + k] = srow[k];
      }
      uint64_t last = kEmptyKey;
      uint32_t last_tb = 0;
      ray_for_each(g, ry, [&](int32_t i0, int32_t i1, int32_t i2, float d) {
        const uint64_t kb = pack_block(i0 >> 3, i1 >> 3, i2 >> 3);
        if (kb != last) {
          last = kb;
          last_tb = tbl_insert(tb_key, kb);
          if (last_tb == 0xFFFFFFFFu) misc[2] = 1;
        }
        if (last_tb != 0xFFFFFFFFu) {
          const int raw = (np << tp_shift) + tid;
          sB[raw] = (last_tb << 9) | (uint32_t)local_index(i0, i1, i2);
          pd[raw] = d;
          ++np;
        }
      });
    }
  }
  cls[tid] = mycls;
  __syncthreads();

  // 2. dense ids for the tile's blocks (8 table entries per thread)
  uint64_t* dkey = reinterpret_cast<uint64_t*>(sA);      // dense id -> key
  uint32_t* dent = reinterpret_cast<uint32_t*>(sA) + 2 * kMaxTileBlocks;  // hash entry
  uint32_t* dnew = dent + kMaxTileBlocks;                // ids of blocks created here
  {
    uint32_t occ = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) occ += tb_key[tid * 8 + k] != kEmptyKey;
    uint32_t nb;
    uint32_t off = cta_exclusive_scan(occ, wtot, &nb);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int e = tid * 8 + k;
      const uint64_t key = tb_key[e];
      if (key != kEmptyKey) {
        tb_dense[e] = (uint16_t)off;
        if (off < kMaxTileBlocks) dkey[off] = key;
        ++off;
      }
    }
    if (tid == 0) {
      misc[1] = nb;
      misc[3] = 0;
    }
  }
  uint32_t npairs;
  const uint32_t poff = cta_exclusive_scan((uint32_t)np, wtot, &npairs);
  __syncthreads();
  const uint32_t nb = misc[1];
  if (nb > kMaxTileBlocks || misc[2]) {
    if (tid == 0) raise_status(mv.ctr, kDevInternal, 4);
    return;
  }

  // 3. insert-or-find every distinct block (one thread each)
  for (uint32_t dd = tid; dd < nb; dd += kCtaThreads) {
    const uint64_t key = dkey[dd];
    uint32_t h = entry_of(mv, key);
    int state = -1;  // 0 found, 1 created here
    for (int pr = 0; pr < mv.max_probe; ++pr) {
      const uint64_t cur = *(volatile uint64_t*)&mv.hkeys[h];
      if (cur == key) {
        state = 0;
        break;
      }
      if (cur == kEmptyKey) {
        const unsigned long long prev =
            atomicCAS((unsigned long long*)&mv.hkeys[h], (unsigned long long)kEmptyKey,
                      (unsigned long long)key);
        if (prev == kEmptyKey) {
          state = 1;
          break;
        }
        if (prev == key) {
          state = 0;
          break;
        }
      }
      h = (h + 1) & mv.entry_mask;
    }
    dent[dd] = h;
    if (state < 0) {
      raise_status(mv.ctr, kDevCapacity, 2);
      tb_slot[dd] = kFailSlot;
    } else if (state == 1) {
      const uint32_t slot = atomicAdd(&mv.ctr[kCtrBlocks], 1u);
      if (slot >= mv.block_cap) {
        raise_status(mv.ctr, kDevCapacity, 1);
        *(volatile uint32_t*)&mv.hvals[h] = kFailSlot;
        tb_slot[dd] = kFailSlot;
      } else {
        mv.blk_key[slot] = key;
        tb_slot[dd] = slot;
        dnew[atomicAdd(&misc[3], 1u)] = dd;
      }
    } else {
      tb_slot[dd] = kNoSlot;  // resolved below
    }
  }
  __syncthreads();
  // zero the blocks created by this CTA, then publish their slots
  const uint32_t nnew = misc[3];
  for (uint32_t i = 0; i < nnew; ++i) {
    float4* p = reinterpret_cast<float4*>(mv.rec + (size_t)tb_slot[dnew[i]] * kBlockVoxels * mv.rs);
    const int n4 = kBlockVoxels * mv.rs / 4;
    for (int k = tid; k < n4; k += kCtaThreads) p[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __threadfence();
  __syncthreads();
  for (uint32_t i = tid; i < nnew; i += kCtaThreads) {
    const uint32_t dd = dnew[i];
    *(volatile uint32_t*)&mv.hvals[dent[dd]] = tb_slot[dd];
  }
  // wait for blocks other CTAs created and have not yet published
  for (uint32_t dd = tid; dd < nb; dd += kCtaThreads) {
    if (tb_slot[dd] != kNoSlot) continue;
    volatile uint32_t* hv = &mv.hvals[dent[dd]];
    uint32_t v = *hv;
    if (v == kNoSlot) {
      const uint64_t t0 = global_ns();
      while ((v = *hv) == kNoSlot) {
        if (global_ns() - t0 > kCrossCtaWaitNs) {
          raise_status(mv.ctr, kDevTimeout, 5);
          v = kFailSlot;
          break;
        }
        __nanosleep(100);
      }
    }
    tb_slot[dd] = v;
  }
  __threadfence();
  __syncthreads();

  // 4. sort keys: ((dense block << 9 | local) << 13) | raw pair index
  for (int k = 0; k < np; ++k) {
    const uint32_t raw = (uint32_t)((k << tp_shift) + tid);
    const uint32_t w = sB[raw];
    const uint32_t key2 = ((uint32_t)tb_dense[w >> 9] << 9) | (w & 511u);
    sA[poff + k] = (key2 << 13) | raw;
  }
  __syncthreads();
  const int tbits = nb <= 1 ? 0 : 32 - __clz((int)nb - 1);
  const uint32_t* sorted = cta_radix_sort(sA, sB, (int)npairs, 13, 9 + tbits, hist, wtot);

  // 5. warp segmented reduction over 32-pair windows of the sorted pairs;
  //    the first lane of each run flushes its sums. hist is free again and
  //    gives each warp 32 floats of scratch.
  float* ws = reinterpret_cast<float*>(hist) + warp * 32;
  for (int wb = (int)warp * 32; wb < (int)npairs; wb += kCtaThreads) {
    const int i = wb + (int)lane;
    const bool act = i < (int)npairs;
    const uint32_t c = act ? sorted[i] : 0u;
    const uint32_t key2 = act ? (c >> 13) : 0xFFFFFFFFu;
    const uint32_t raw = c & 0x1FFFu;
    const int pt = act ? (int)(raw & (uint32_t)(tile_points - 1)) : 0;
    const uint32_t slot = act ? tb_slot[key2 >> 9] : kNoSlot;
    float* r = (slot < kFailSlot) ? mv.rec + ((size_t)slot * kBlockVoxels + (key2 & 511u)) * mv.rs
                                  : nullptr;
    if (r) mark_touched(mv.blk_mask + slot, sub_bit(key2 & 511u), mv.blk_mask[slot]);
    if (MODE == 0) {
      // (voxel, class) groups: sum d per group leader through warp scratch
      const uint32_t cl = cls[pt];
      const uint32_t kc = act ? ((key2 << 7) | cl) : 0xFFFFFFFFu;
      const unsigned pc = __match_any_sync(0xFFFFFFFFu, kc);
      const int ldr = __ffs(pc) - 1;
      ws[lane] = 0.f;
      __syncwarp();
      if (act) atomicAdd(&ws[ldr], pd[raw]);
      __syncwarp();
      if (r && (int)lane == ldr) red_add_v2(r + 2 * cl, ws[lane], (float)__popc(pc));
      __syncwarp();
    } else {
      // soft counts: exact 64-bit fixed-point sums of the run's d and
      // probabilities (segmented over the window), one integer reduction
      // per field from the run's first lane
      const unsigned peers = __match_any_sync(0xFFFFFFFFu, key2);
      const int first = __ffs(peers) - 1, lastl = 31 - __clz(peers);
      unsigned long long* q = reinterpret_cast<unsigned long long*>(r);
      unsigned long long dsum = act ? fx32(pd[raw]) : 0ull;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long a1 = __shfl_down_sync(0xFFFFFFFFu, dsum, off);
        if ((int)lane + off <= lastl) dsum += a1;
      }
      if (r && (int)lane == first) {
        red_add_u64(q, dsum);
        red_add_u64(q + 1, (unsigned long long)__popc(peers) << 32);
      }
      for (int k = 0; k < K; ++k) {
        unsigned long long pv = act ? fx32(probs[pt * K + k]) : 0ull;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const unsigned long long a1 = __shfl_down_sync(0xFFFFFFFFu, pv, off);
          if ((int)lane + off <= lastl) pv += a1;
        }
        if (r && (int)lane == first) red_add_u64(q + 2 + k, pv);
      }
    }
  }
}

// ------------------------------------------------------------------ launch
cudaError_t closed_setup_attributes(int mode, int K, int tile_points) {
  const size_t sm = closed_smem_bytes(mode, K, tile_points);
  cudaError_t e = hash_setup_attributes();
  if (e != cudaSuccess) return e;
  if (mode == 0)
    return cudaFuncSetAttribute(k_fuse_closed<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sm);
  return cudaFuncSetAttribute(k_fuse_closed<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sm);
}

int closed_tile_points(int cap, int band_blocks) {
  int tp = 256;  // a power of two: the pair layout shifts by log2(tp)
  while (tp > 32 && (tp * cap > kTileCap || tp * band_blocks > kMaxTileBlocks)) tp >>= 1;
  return tp;
}

int max_band_blocks() { return kMaxBandBlocks; }

cudaError_t launch_fuse_closed(const MapView& mv, const ScanGeom& g, const float* pts,
                               const float* sem, int64_t n, int mode, int K, int tile_points,
                               cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)((n + tile_points - 1) / tile_points);
  const size_t sm = closed_smem_bytes(mode, K, tile_points);
  if (mode == 0)
    k_fuse_closed<0><<<grid, kCtaThreads, sm, st>>>(mv, g, pts, sem, n, K, tile_points);
  else
    k_fuse_closed<1><<<grid, kCtaThreads, sm, st>>>(mv, g, pts, sem, n, K, tile_points);
  return cudaGetLastError();
}

}  // namespace slim
