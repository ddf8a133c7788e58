// Closed-set one-hot integration with shared-memory hash aggregation
// (Sec. III-A TSDF + Sec. III-C / Theorem 1 Dirichlet counts), one tile of
// TP points per CTA (TP = 64, 128 or 256 threads), persistent over a batch
// of scans:
//   1. every thread loads its point and class probabilities first (the
//      probability row as independent float4 loads, argmax afterwards), then
//      marches the band; each kept pair is added at once into a tile-local
//      table keyed by (tile block entry, local voxel, class): an entry is a
//      32-bit key word and a 32-bit count side by side, plus a 32-bit sum of
//      the pair's SDF in fixed point (units of tau / 2^20); a pair costs one
//      shared load and two 32-bit shared atomic adds (plus a compare-and-swap
//      when it claims the entry); no pair list is staged, nothing is sorted;
//   2. each distinct block of the tile (compacted first) is inserted into
//      (or found in) the map's hash by its own thread; a block this thread
//      creates is published at once (its records are already zero: the pool
//      is kept zero outside the sub-blocks written since the last reset, see
//      k_zero_touched_blocks);
//      only then does the thread wait (time-bounded) for blocks other CTAs
//      are still publishing, so no wait can be part of a cycle;
//   3. flush: one vector red.add (S_k += sum d, c_k += count) per table
//      entry into the voxel's class-split record (see common.cuh).
// A pair whose table probe runs out is re-generated after the slots are
// known and sent to HBM on its own, in FP32.
// Fixed point: a kept pair has d in [-tau, tau]; q = rint(d * 2^20 / tau)
// is stored offset by 2^20 (so it is never negative), the rounding error is
// at most tau * 2^-21 (+ one FP32 rounding of the scale) per pair, and the
// tile sum (at most TP pairs per entry) is exact in the 30-bit field.
#include "block_sort.cuh"
#include "closed_common.cuh"
#include "common.cuh"
#include "geometry.cuh"
#include "hash.cuh"
#include "internal.h"

namespace slim {

constexpr uint32_t kVcEmpty = 0xFFFFFFFFu;  // key: tile block entry << 15 | local << 6 | class
constexpr uint32_t kQOne = 1u << 20;        // fixed-point unit of the SDF sum is tau / 2^20

template <int TP>
struct HashTile {
  static constexpr int kTbl = 4 * TP;    // block table entries (>= distinct blocks of a tile)
  static constexpr int kVc = 8 * TP;     // (voxel, class) accumulators
  static constexpr int kVcBits = kVc == 2048 ? 11 : (kVc == 1024 ? 10 : 9);
  // tb_key u64 + tb_slot u32 + block list u16 per block entry; per
  // accumulator a (key, count) u32 pair and a u32 sum; counters
  static constexpr size_t kSmem = (size_t)kTbl * 14 + (size_t)kVc * 12 + 16 * 4;
};

// Insert-or-find a block key; the thread that inserts it appends the entry
// to the tile's block list. Returns the entry, or 0xFFFFFFFF when full.
template <int TP>
__device__ __forceinline__ uint32_t htbl_insert(uint64_t* tb, uint64_t kb, uint16_t* blist,
                                                uint32_t* nblk) {
  constexpr int N = HashTile<TP>::kTbl;
  uint32_t h = tile_hash(kb) & (N - 1);
  for (int it = 0; it < N; ++it) {
    const uint64_t cur = *(volatile uint64_t*)&tb[h];
    if (cur == kb) return h;
    if (cur == kEmptyKey) {
      const unsigned long long prev = atomicCAS((unsigned long long*)&tb[h],
                                                (unsigned long long)kEmptyKey,
                                                (unsigned long long)kb);
      if (prev == kEmptyKey) {
        blist[atomicAdd(nblk, 1u)] = (uint16_t)h;
        return h;
      }
      if (prev == kb) return h;
    }
    h = (h + 1) & (N - 1);
  }
  return 0xFFFFFFFFu;
}

template <int TP>
__device__ __forceinline__ uint32_t htbl_find(const uint64_t* tb, uint64_t kb) {
  constexpr int N = HashTile<TP>::kTbl;
  uint32_t h = tile_hash(kb) & (N - 1);
  for (int it = 0; it < N; ++it) {
    const uint64_t cur = tb[h];
    if (cur == kb) return h;
    if (cur == kEmptyKey) return 0xFFFFFFFFu;
    h = (h + 1) & (N - 1);
  }
  return 0xFFFFFFFFu;
}

// Add one pair (key, q) to the (voxel, class) table: vkc[2e] is the entry's
// key (claimed by compare-and-swap), vkc[2e + 1] its count, vsum[e] its
// fixed-point SDF sum (q = rint(d 2^20 / tau) + 2^20, at most TP pairs per
// entry: below 2^30). Returns false when the probe runs out.
template <int TP>
__device__ __forceinline__ bool vc_add(uint32_t* vkc, uint32_t* vsum, uint32_t key, uint32_t q) {
  constexpr int N = HashTile<TP>::kVc;
  uint32_t h = (key * 2654435761u) >> (32 - HashTile<TP>::kVcBits);
  for (int it = 0; it < 64; ++it) {
    uint32_t cur = *(volatile uint32_t*)&vkc[2 * h];
    if (cur == kVcEmpty) {
      cur = atomicCAS(&vkc[2 * h], kVcEmpty, key);
      if (cur == kVcEmpty) cur = key;
    }
    if (cur == key) {
      atomicAdd(&vkc[2 * h + 1], 1u);
      atomicAdd(&vsum[h], q);
      return true;
    }
    h = (h + 1) & (N - 1);
  }
  return false;
}

// Ask L2 for this thread's point and probability row of tile t (the tile the
// CTA takes next), so that its loads at the start of that tile hit L2.
__device__ __forceinline__ void prefetch_tile(const HashBatch& b, uint32_t t) {
  const HashJob& J = b.job[job_of(b, t)];
  const int64_t j = (int64_t)(t - J.tile_begin) * J.tile_points + threadIdx.x;
  if ((int)threadIdx.x >= J.tile_points || j >= J.n) return;
  prefetch_l2(J.pts + 3 * j);
  const float* row = J.sem + (size_t)j * J.K;
  prefetch_l2(row);
  prefetch_l2(row + J.K - 1);
}

// One tile: points [tile * tile_points, (tile + 1) * tile_points) of a scan.
template <int TP>
__device__ __forceinline__ void fuse_hash_tile(const MapView& mv, const ScanGeom& g,
                                               const float* __restrict__ pts,
                                               const float* __restrict__ sem, int64_t n, int K,
                                               int tile_points, int64_t tile, unsigned char* sm,
                                               const HashBatch& b, const uint32_t* s_next) {
  using H = HashTile<TP>;
  uint64_t* tb_key = reinterpret_cast<uint64_t*>(sm);
  uint32_t* vkc = reinterpret_cast<uint32_t*>(tb_key + H::kTbl);  // (key, count) per entry
  uint32_t* vsum = vkc + 2 * H::kVc;
  uint32_t* tb_slot = vsum + H::kVc;
  uint16_t* blist = reinterpret_cast<uint16_t*>(tb_slot + H::kTbl);
  uint32_t* misc = reinterpret_cast<uint32_t*>(blist + H::kTbl);

  const int tid = threadIdx.x;
  // loads first: the point and its class probabilities
  const int64_t j = tile * tile_points + tid;
  const bool mine = tid < tile_points && j < n;
  float p0 = 0.f, p1 = 0.f, p2 = 0.f;
  uint32_t cls = 0;
  if (mine) {
    p0 = __ldg(pts + 3 * j);
    p1 = __ldg(pts + 3 * j + 1);
    p2 = __ldg(pts + 3 * j + 2);
    cls = argmax_row(sem + (size_t)j * K, K);
  }
  if (tid == 0) {
    misc[0] = *(volatile uint32_t*)&mv.ctr[kCtrStatus];
    misc[2] = 0;  // block table overflow
    misc[3] = 0;  // distinct blocks
  }
  for (int e = tid; e < H::kTbl / 2; e += TP)
    reinterpret_cast<ulonglong2*>(tb_key)[e] = make_ulonglong2(kEmptyKey, kEmptyKey);
  for (int e = tid; e < H::kVc / 2; e += TP)
    reinterpret_cast<uint4*>(vkc)[e] = make_uint4(kVcEmpty, 0u, kVcEmpty, 0u);
  for (int e = tid; e < H::kVc / 4; e += TP)
    reinterpret_cast<uint4*>(vsum)[e] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  if (misc[0]) return;
  if (s_next && *s_next < b.total_tiles) prefetch_tile(b, *s_next);

  // 1. band DDA, aggregating every pair into the (voxel, class) table
  const float qscale = __fdiv_rn(1048576.0f, g.tau);
  int ovf = -1;  // index of the first pair the table could not take
  Ray ry;
  const bool valid = mine && ray_setup(g, p0, p1, p2, ry);
  if (valid) {
    Ray r2 = ry;
    uint32_t last_tb = 0;
    int k = 0;
    ray_for_each_blk(g, r2, [&](int32_t i0, int32_t i1, int32_t i2, float d, bool new_block) {
      if (new_block) {
        last_tb = htbl_insert<TP>(tb_key, pack_block(i0 >> 3, i1 >> 3, i2 >> 3), blist, &misc[3]);
        if (last_tb == 0xFFFFFFFFu) misc[2] = 1;
      }
      const int idx = k++;
      if (last_tb == 0xFFFFFFFFu || ovf >= 0) return;
      const uint32_t key = (last_tb << 15) | ((uint32_t)local_index(i0, i1, i2) << 6) | cls;
      int qi = __float2int_rn(__fmul_rn(d, qscale));
      qi = max(-(int)kQOne, min((int)kQOne, qi));
      if (!vc_add<TP>(vkc, vsum, key, (uint32_t)(qi + (int)kQOne))) ovf = idx;
    });
  }
  __syncthreads();
  if (misc[2]) {
    if (tid == 0) raise_status(mv.ctr, kDevInternal, 4);
    return;
  }
  const int nblk = (int)misc[3];

  // 2. insert-or-find each distinct block (compacted items tid + TP q); a
  // created block is published at once, then blocks other CTAs created are
  // resolved (acquire: the slot read orders this CTA's reductions after it)
  constexpr int Q = H::kTbl / TP;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int i = tid + q * TP;
    if (i >= nblk) break;
    const int e = blist[i];
    const uint64_t key = tb_key[e];
    uint32_t h = entry_of(mv, key);
    int state = -1;
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
    uint32_t v = kFailSlot;
    if (state < 0) {
      raise_status(mv.ctr, kDevCapacity, 2);
    } else if (state == 1) {
      const uint32_t slot = atomicAdd(&mv.ctr[kCtrBlocks], 1u);
      if (slot >= mv.block_cap) {
        raise_status(mv.ctr, kDevCapacity, 1);
      } else {
        mv.blk_key[slot] = key;
        v = slot;
      }
      st_release(&mv.hvals[h], v);
    } else {
      uint32_t* hv = &mv.hvals[h];
      v = ld_acquire(hv);
      if (v == kNoSlot) {
        const uint64_t t0 = global_ns();
        while ((v = ld_acquire(hv)) == kNoSlot) {
          if (global_ns() - t0 > kCrossCtaWaitNs) {
            raise_status(mv.ctr, kDevTimeout, 5);
            v = kFailSlot;
            break;
          }
          __nanosleep(100);
        }
      }
      if (v != kFailSlot && v >= mv.block_cap) {  // consistency check, never expected
        raise_status(mv.ctr, kDevInternal, 9);
        v = kFailSlot;
      }
    }
    tb_slot[e] = v;
  }
  __syncthreads();

  // 3. flush: one vector red.add (S_k, c_k) per entry
  const float qunit = __fmul_rn(g.tau, 1.0f / 1048576.0f);  // exact: a power-of-two scale
  for (int e = tid; e < H::kVc; e += TP) {
    const uint2 kc = reinterpret_cast<const uint2*>(vkc)[e];
    const uint32_t key = kc.x;  // entry < kTbl, class < K by construction
    if (key == kVcEmpty) continue;
    const uint32_t slot = tb_slot[key >> 15];
    if (slot >= mv.block_cap) continue;  // kFailSlot: a fault was raised for the block
    const uint32_t cnt = kc.y;
    const int32_t qs = (int32_t)vsum[e] - (int32_t)(cnt * kQOne);
    const uint32_t loc = (key >> 6) & 511u;
    float* r = mv.rec + ((size_t)slot * kBlockVoxels + loc) * mv.rs;
    red_add_v2(r + 2 * (key & 63u), __fmul_rn((float)qs, qunit), (float)cnt);
    mark_touched(mv.blk_mask + slot, sub_bit(loc), mv.blk_mask[slot]);
  }

  // 4. pairs the table could not take go to HBM one by one
  if (valid && ovf >= 0) {
    uint64_t last = kEmptyKey;
    uint32_t slot = kFailSlot;
    int k = 0;
    ray_for_each(g, ry, [&](int32_t i0, int32_t i1, int32_t i2, float d) {
      const uint64_t kb = pack_block(i0 >> 3, i1 >> 3, i2 >> 3);
      if (kb != last) {
        last = kb;
        const uint32_t te = htbl_find<TP>(tb_key, kb);
        slot = te == 0xFFFFFFFFu ? kFailSlot : tb_slot[te];
      }
      if (k++ < ovf || slot >= kFailSlot) return;
      if (slot >= mv.block_cap) {
        raise_status(mv.ctr, kDevInternal, 8);
        return;
      }
      const int loc = local_index(i0, i1, i2);
      float* r = mv.rec + ((size_t)slot * kBlockVoxels + loc) * mv.rs;
      red_add_v2(r + 2 * cls, d, 1.f);
      mark_touched(mv.blk_mask + slot, sub_bit(loc), mv.blk_mask[slot]);
    });
  }
}

// Persistent form: a grid sized to the resident capacity takes tiles from a
// shared counter until every tile of every job (a scan of some map) is done
// (while tiles remain for another round, each CTA holds one reserved tile
// ahead, whose inputs it prefetches); the last CTA to finish resets the
// counter for the next launch. Tiles of
// different jobs (scans of the same or of different maps) run concurrently:
// the per-scan updates are additions (Theorem 1), so their order is free.
template <int TP>
__global__ void __launch_bounds__(TP, 1024 / TP) k_fuse_hash_persistent(const __grid_constant__ HashBatch b) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ uint32_t s_t;
  if (threadIdx.x == 0) s_t = atomicAdd(&b.work[0], 1u);
  __syncthreads();
  uint32_t t = s_t;
  __syncthreads();
  while (t < b.total_tiles) {
    // while at least another full round of tiles remains, reserve the next
    // tile now (the tile prefetches its inputs into L2); near the end take
    // it only when this one is done, so that no CTA holds work others wait for
    const bool ahead = t + gridDim.x < b.total_tiles;
    if (ahead && threadIdx.x == 0) s_t = atomicAdd(&b.work[0], 1u);
    const HashJob& J = b.job[job_of(b, t)];
    fuse_hash_tile<TP>(J.mv, J.g, J.pts, J.sem, J.n, J.K, J.tile_points, (int64_t)(t - J.tile_begin),
                       sm, b, ahead ? &s_t : nullptr);
    __syncthreads();
    if (!ahead) {
      if (threadIdx.x == 0) s_t = atomicAdd(&b.work[0], 1u);
      __syncthreads();
    }
    t = s_t;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&b.work[1], 1u) == gridDim.x - 1) {
      b.work[0] = 0;
      b.work[1] = 0;
    }
  }
}

static int g_resident[3] = {0, 0, 0};  // CTAs per SM of the 64 / 128 / 256 variants
static int g_sms = 0;

template <int TP>
static cudaError_t setup_one(int idx) {
  cudaError_t e = cudaFuncSetAttribute(k_fuse_hash_persistent<TP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)HashTile<TP>::kSmem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_resident[idx], k_fuse_hash_persistent<TP>,
                                                       TP, HashTile<TP>::kSmem);
}

cudaError_t hash_setup_attributes() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = setup_one<64>(0);
  if (e == cudaSuccess) e = setup_one<128>(1);
  if (e == cudaSuccess) e = setup_one<256>(2);
  return e;
}

// Keeps a record pool zero outside the sub-blocks integrations write: for
// each block [0, min(*nblocks, capacity)), zeroes the records of every 2 x 2
// x 2 sub-block its touched mask names (four runs of two consecutive
// records: z pairs at the four (x, y) of the sub-block) and clears the mask,
// so that a reset map hands out zeroed blocks. One warp per block. rs is
// even for every record layout, so each run starts and ends on a 16-byte
// boundary.
__global__ void __launch_bounds__(256) k_zero_touched_blocks(float4* rec, uint64_t* mask,
                                                             const uint32_t* nblocks,
                                                             uint32_t block_cap, int rs) {
  const uint32_t nb = min(*(volatile const uint32_t*)nblocks, block_cap);
  const unsigned lane = lane_id();
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int run4 = rs / 2;  // float4 per run of two records
  for (int64_t blk = gw; blk < (int64_t)nb; blk += nw) {
    uint64_t m = mask[blk];
    float4* base = rec + (size_t)blk * kBlockVoxels * (size_t)rs / 4;
    while (m) {
      const int sb = __ffsll((long long)m) - 1;
      m &= m - 1;
      const int x0 = 2 * (sb >> 4), y0 = 2 * ((sb >> 2) & 3), z0 = 2 * (sb & 3);
      // 4 runs x run4 float4, spread over the lanes
      for (int k = (int)lane; k < 4 * run4; k += 32) {
        const int run = k / run4, off = k - run * run4;
        const int loc = ((x0 + (run >> 1)) * 8 + (y0 + (run & 1))) * 8 + z0;
        base[(size_t)loc * rs / 4 + off] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    if (lane == 0) mask[blk] = 0ull;
  }
}

cudaError_t launch_zero_touched_blocks(float* rec, uint64_t* mask, const uint32_t* nblocks,
                                       uint32_t block_cap, int rs, cudaStream_t st) {
  if (!rec) return cudaSuccess;
  const int sms = g_sms > 0 ? g_sms : 152;
  k_zero_touched_blocks<<<(unsigned)(sms * 8), 256, 0, st>>>(reinterpret_cast<float4*>(rec),
                                                             mask, nblocks, block_cap, rs);
  return cudaGetLastError();
}

// Largest number of points a TP-thread tile may hold: its distinct blocks
// (at most points x band_blocks) must fit the block table.
int hash_tile_points(int TP, int band_blocks) {
  int tp = TP;
  while (tp > 16 && tp * band_blocks > HashTile<256>::kTbl / 256 * TP) tp >>= 1;
  return tp;
}

int hash_max_tile(int band_blocks) { return hash_tile_points(256, band_blocks); }

// Fill the tile ranges of b's jobs and launch the persistent kernel.
// `tile` selects the variant (64, 128 or 256 threads); ctas_per_sm = 0 uses
// the resident maximum.
cudaError_t launch_hash_batch(HashBatch& b, int tile, int ctas_per_sm, cudaStream_t st) {
  const int TP = tile <= 64 ? 64 : (tile <= 128 ? 128 : 256);
  const int idx = TP == 64 ? 0 : (TP == 128 ? 1 : 2);
  uint32_t total = 0;
  for (int j = 0; j < b.n_jobs; ++j) {
    b.job[j].tile_points = hash_tile_points(TP, b.job[j].band_blocks);
    b.job[j].tile_begin = total;
    total += (uint32_t)((b.job[j].n + b.job[j].tile_points - 1) / b.job[j].tile_points);
  }
  b.total_tiles = total;
  if (total == 0) return cudaSuccess;
  const int per_sm = ctas_per_sm > 0 ? std::min(ctas_per_sm, g_resident[idx]) : g_resident[idx];
  const uint32_t grid = std::min<uint32_t>(total, (uint32_t)std::max(1, per_sm * g_sms));
  if (TP == 64)
    k_fuse_hash_persistent<64><<<grid, 64, HashTile<64>::kSmem, st>>>(b);
  else if (TP == 128)
    k_fuse_hash_persistent<128><<<grid, 128, HashTile<128>::kSmem, st>>>(b);
  else
    k_fuse_hash_persistent<256><<<grid, 256, HashTile<256>::kSmem, st>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_fuse_hash(const MapView& mv, const ScanGeom& g, const float* pts,
                             const float* sem, int64_t n, int K, int tile, int band_blocks,
                             cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  HashBatch b;
  b.n_jobs = 1;
  b.job[0].mv = mv;
  b.job[0].g = g;
  b.job[0].pts = pts;
  b.job[0].sem = sem;
  b.job[0].n = n;
  b.job[0].K = K;
  b.job[0].band_blocks = band_blocks;
  b.job[0].latest = 0;
  b.job[0].soft = 0;
  b.work = mv.ctr + kCtrWork;
  return launch_hash_batch(b, tile, 0, st);
}

}  // namespace slim
