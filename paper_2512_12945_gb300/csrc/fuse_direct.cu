// Closed-set one-hot integration by direct per-pair reductions (Sec. III-A
// TSDF + Sec. III-C / Theorem 1 Dirichlet counts): one thread per point
// walks its band; every kept (voxel, point) pair is one vector
// red.global.add.v2.f32 (S_k += d, c_k += 1) into the voxel's class-split
// record. Theorem 1 makes the order of these additions free, so nothing is
// grouped on chip: a scan's records (a few tens of MB) stay in the 129 MB L2,
// where the reductions resolve, and the kernel keeps no shared tables, no
// barriers between its phases and a high occupancy.
//
// Blocks: when a ray enters an 8^3 block, the thread looks the block up in
// the map's hash (the hash table stays in L2), inserting it if it is new
// (slot from the allocation counter, published with a relaxed store) or
// waiting (time-bounded) for another thread's publication. A new block's
// records are already zero (the pool is zero outside the sub-blocks written
// since the last reset, see k_zero_touched_blocks) and readers use a slot
// only as the address of their reductions, so a publication orders nothing
// else and needs no release / acquire pair; the block's key in blk_key is
// read only by later kernels. A publication needs nothing but its own
// thread's earlier steps, so no wait can be part of a cycle. (A per-CTA
// shared-memory cache of block slots in front of the hash was measured
// slower: 1.81 vs 1.66 ms per 100 scans.) Each ray marks the 2 x 2 x 2
// sub-blocks it writes in the block's touched mask (read when it enters the
// block; reduced into only when a bit is missing) for the reset.
//
// One kernel serves a single scan and a batch of scans of many maps (the
// HashBatch job table): each CTA takes 256 points of one job.
//
// Latest-label maps (the non-Bayesian ablation) keep {S, W, stamp}: a pair
// adds (d, 1) to (S, W) and raises the 64-bit stamp scan << 40 | point << 8
// | label with atomicMax, so the label of the last observation in scan, then
// point order survives whatever order the reductions run in.
#include "closed_common.cuh"
#include "geometry.cuh"
#include "hash.cuh"
#include "internal.h"

namespace slim {

constexpr int kDirectThreads = 256;

// MODE: 0 one-hot, 1 soft counts, 2 latest label; WT: observations carry
// the weight w~ of the linear decay behind the surface instead of 1 (every
// job of a launch has the launch's mode and weighting, so the per-pair loop
// carries no branch on either).
template <int MODE, bool WT>
__global__ void __launch_bounds__(kDirectThreads) k_fuse_direct(const __grid_constant__ HashBatch b) {
  const uint32_t t = blockIdx.x;
  const HashJob& J = b.job[job_of(b, t)];
  const MapView& mv = J.mv;
  if (*(volatile uint32_t*)&mv.ctr[kCtrStatus]) return;
  const int64_t j = (int64_t)(t - J.tile_begin) * kDirectThreads + threadIdx.x;
  if (j >= J.n) return;
  Ray ry;
  if (!ray_setup_at(J.g, J.pts, j, ry)) return;
  const uint32_t cls = MODE == 1 ? 0u : argmax_row(J.sem + (size_t)j * J.K, J.K);
  uint32_t slot = kFailSlot;
  uint64_t bits = 0;  // sub-blocks this ray wrote in the current block
  uint64_t seen = 0;  // the block's touched mask, read when the ray entered it
  ray_for_each_blk(J.g, ry, [&](int32_t i0, int32_t i1, int32_t i2, float d, bool new_block) {
    if (new_block) {
      if (bits) mark_touched(mv.blk_mask + slot, bits, seen);
      bits = 0;
      slot = map_block_slot(mv, pack_block(i0 >> 3, i1 >> 3, i2 >> 3));
      if (slot < mv.block_cap) seen = mv.blk_mask[slot];
    }
    if (slot >= mv.block_cap) return;
    // the observation adds (w~ d, w~); an observation of weight 0 changes
    // nothing
    const float wt = WT ? obs_weight(J.g, d) : 1.f;
    if (WT && wt == 0.f) return;
    const float wd = WT ? __fmul_rn(wt, d) : d;
    const int loc = local_index(i0, i1, i2);
    bits |= sub_bit(loc);
    float* r = mv.rec + ((size_t)slot * kBlockVoxels + loc) * mv.rs;
    if (MODE == 0) {
      red_add_v2(r + 2 * cls, wd, wt);
    } else if (MODE == 1) {
      // soft counts: (S, W) += (w~ d, w~) and c += w~ p as exact 64-bit
      // fixed-point sums (one integer reduction per field)
      unsigned long long* q = reinterpret_cast<unsigned long long*>(r);
      red_add_u64(q, fx32(wd));
      red_add_u64(q + 1, WT ? fx32(wt) : (1ull << 32));
      const float* p = J.sem + (size_t)j * J.K;
      for (int k = 0; k < J.K; ++k) {
        const float a = WT ? __fmul_rn(wt, __ldg(p + k)) : __ldg(p + k);
        red_add_u64(q + 2 + k, fx32(a));
      }
    } else {
      const unsigned long long stamp = ((unsigned long long)J.g.scan_no << 40) |
                                       ((unsigned long long)(uint32_t)j << 8) | cls;
      red_add_v2(r, wd, wt);
      atomicMax(reinterpret_cast<unsigned long long*>(r + 2), stamp);
    }
  });
  if (bits) mark_touched(mv.blk_mask + slot, bits, seen);
}

// All jobs of b share one variant: mode (0 one-hot, 1 soft, 2 latest) + 3
// when the observations are weighted (linear decay).
cudaError_t launch_direct_batch(HashBatch& b, int mode, cudaStream_t st) {
  uint32_t total = 0;
  for (int j = 0; j < b.n_jobs; ++j) {
    b.job[j].tile_points = kDirectThreads;
    b.job[j].tile_begin = total;
    total += (uint32_t)((b.job[j].n + kDirectThreads - 1) / kDirectThreads);
  }
  b.total_tiles = total;
  if (total == 0) return cudaSuccess;
  switch (mode) {
    case 1: k_fuse_direct<1, false><<<total, kDirectThreads, 0, st>>>(b); break;
    case 2: k_fuse_direct<2, false><<<total, kDirectThreads, 0, st>>>(b); break;
    case 3: k_fuse_direct<0, true><<<total, kDirectThreads, 0, st>>>(b); break;
    case 4: k_fuse_direct<1, true><<<total, kDirectThreads, 0, st>>>(b); break;
    case 5: k_fuse_direct<2, true><<<total, kDirectThreads, 0, st>>>(b); break;
    default: k_fuse_direct<0, false><<<total, kDirectThreads, 0, st>>>(b); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_fuse_direct(const MapView& mv, const ScanGeom& g, const float* pts,
                               const float* sem, int64_t n, int K, int latest, int soft,
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
  b.job[0].band_blocks = 0;
  b.job[0].latest = latest;
  b.job[0].soft = soft;
  b.work = mv.ctr + kCtrWork;
  return launch_direct_batch(b, (soft ? 1 : (latest ? 2 : 0)) + (g.weighting ? 3 : 0), st);
}

}  // namespace slim
