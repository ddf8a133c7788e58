// Host-side interface between the C ABI (api.cu) and the kernel files.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/slim_gb300.h"
#include "common.cuh"

namespace slim {

// integrate_closed.cu
cudaError_t launch_fuse_closed(const MapView& mv, const ScanGeom& g, const float* pts,
                               const float* sem, int64_t n, int mode, int K, int tile_points,
                               cudaStream_t st);
cudaError_t closed_setup_attributes(int mode, int K, int tile_points);
// fuse_hash.cu: one-hot hash aggregation; tile = points per CTA (64, 128 or 256)
struct HashJob {
  MapView mv;
  ScanGeom g;
  const float* pts;
  const float* sem;
  int64_t n;
  int32_t K;
  int32_t band_blocks;
  int32_t latest;       // latest-label mode (direct reductions only)
  int32_t soft;         // soft counts (direct reductions)
  int32_t tile_points;  // set by launch_hash_batch
  uint32_t tile_begin;  // set by launch_hash_batch
};
constexpr int kMaxHashJobs = 64;  // 312 B each: ~20 KB of kernel parameters
struct HashBatch {
  HashJob job[kMaxHashJobs];
  int32_t n_jobs;
  uint32_t total_tiles;
  uint32_t* work;  // two zeroed device words (next tile, finished CTAs)
};
cudaError_t launch_hash_batch(HashBatch& b, int tile, int ctas_per_sm, cudaStream_t st);
cudaError_t hash_setup_attributes();
// Direct per-pair reductions, one scan / the jobs of b in one grid.
cudaError_t launch_fuse_direct(const MapView& mv, const ScanGeom& g, const float* pts,
                               const float* sem, int64_t n, int K, int latest, int soft,
                               cudaStream_t st);
cudaError_t launch_direct_batch(HashBatch& b, int mode, cudaStream_t st);
// Zero the records of the touched sub-blocks of blocks [0, *nblocks) of a
// closed-set record pool and clear their masks.
cudaError_t launch_zero_touched_blocks(float* rec, uint64_t* mask, const uint32_t* nblocks,
                                       uint32_t block_cap, int rs, cudaStream_t st);
cudaError_t launch_fuse_hash(const MapView& mv, const ScanGeom& g, const float* pts,
                             const float* sem, int64_t n, int K, int tile, int band_blocks,
                             cudaStream_t st);
int hash_max_tile(int band_blocks);
int closed_tile_points(int cap, int band_blocks);
int max_band_blocks();

// open.cu: open-set integration by tiles of pixels aggregated on chip.
// Per-row accumulators of one integration call of a map (exact integer
// sums, zero between calls):
//   rows[row * stride]: {sum d (int64, unit tau 2^-22), n (u32), pad,
//                        S1 of the L elements (int64, unit B 2^-32),
//                        S2 of the L elements (int64, unit B^2 2^-31)}
// with B the map's embed_bound.
struct OpenAcc {
  float* rows;      // [row_cap * stride], zero between calls
  uint32_t* listed; // [row_cap] 1 while the row is in list (cleared by the update)
  uint32_t* list;   // [row_cap] rows touched by the current call
  uint32_t* count;  // entries in list
  int32_t stride;   // floats per accumulator row: 4 + 4 L
};
struct OpenJob {  // 64-byte aligned by its tensor map
  CUtensorMap sem_map;  // the scan's embeddings as an L x n FP32 tensor
  MapView mv;
  ScanGeom g;
  OpenAcc acc;
  const float* pts;
  const float* sem;
  int64_t n;
  int32_t L;
  int32_t width;        // organized frames: pixels per image row; 0: unorganized
  int32_t tw_log2;      // organized frames: log2 of the tile width (3, 4, 5)
  float fx1, fx2;       // fixed-point scales of S1 and S2: 2^32 / B, 2^31 / B^2
  uint32_t tiles_x;     // set by launch_open_tiles
  uint32_t tile_begin;  // set by launch_open_tiles
};
constexpr int kMaxOpenJobs = 48;  // 512 B each: ~24 KB of kernel parameters
struct OpenBatch {
  OpenJob job[kMaxOpenJobs];
  int32_t n_jobs;
  uint32_t total_tiles;
};
struct OpenApplyJob {
  MapView mv;
  OpenAcc acc;
  int32_t L;
  float dunit;  // metres per unit of the accumulated sum of d: tau 2^-22
  float u1, u2; // units of the accumulated S1 and S2: B 2^-32, B^2 2^-31
};
struct OpenApplyBatch {
  OpenApplyJob job[kMaxOpenJobs];
  int32_t n_jobs;
};
bool open_encode_sem(CUtensorMap* map, const float* sem, int64_t n, int L, int row_pts);
cudaError_t launch_open_tiles(OpenBatch& b, int bf16, cudaStream_t st);
cudaError_t launch_open_apply(const OpenApplyBatch& a, int bf16, cudaStream_t st);
// Set the voxel-row tables of the blocks allocated so far back to -1.
cudaError_t launch_reset_vox_rows(const MapView& mv, cudaStream_t st);

// device_sort.cu: stable LSD radix sort of (key, value) pairs in global memory
// over key bits [0, bits). keys/vals are sorted in place using the tmp
// buffers; temp_bytes tells how much scratch `tmp` needs.
size_t radix_sort_temp_bytes(int64_t n);
cudaError_t radix_sort_u64(uint64_t* keys, uint32_t* vals, uint64_t* keys_tmp,
                           uint32_t* vals_tmp, void* tmp, int64_t n, int bits,
                           cudaStream_t st);
cudaError_t radix_sort_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp,
                           uint32_t* vals_tmp, void* tmp, int64_t n, int bits,
                           cudaStream_t st);
// As radix_sort_u32 with the item count read on the device from *n_dev
// (at most n_max items; the launch is sized for n_max). The sorted pairs are
// left in whichever of (keys, vals) / (keys_tmp, vals_tmp) the last pass
// wrote; *keys_out / *vals_out name it (no copy back).
cudaError_t radix_sort_u32_devn(uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp,
                                uint32_t* vals_tmp, void* tmp, int64_t n_max,
                                const uint32_t* n_dev, int bits, cudaStream_t st,
                                uint32_t** keys_out, uint32_t** vals_out);
// Exclusive scan of n uint32 counts into out (n + 1 entries, out[n] = total).
cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, void* tmp,
                               cudaStream_t st);

// extract.cu
struct ExtractArgs {
  int32_t* ijk;
  float* D;
  float* W;
  float* sem;
  float* beta;
  int32_t* index;
  float* unc;        // uncertainty read-out (closed n x (K+1), open n x l) or null
  int32_t flags;
  int32_t mode;
  int32_t K;
  int32_t L;
  int32_t bf16;
  float alpha0;
};
// Count voxels per sorted block (counts[b]) for b < nb (order = slots[b]).
cudaError_t launch_extract_count(const MapView& mv, const uint32_t* slots, int64_t nb,
                                 bool open, uint32_t* counts, cudaStream_t st);
cudaError_t launch_extract_write(const MapView& mv, const uint32_t* slots,
                                 const uint64_t* keys, int64_t nb, const uint32_t* offsets,
                                 const ExtractArgs& a, cudaStream_t st);
cudaError_t launch_gather_keys(const MapView& mv, int64_t nb, uint64_t* keys, uint32_t* slots,
                               cudaStream_t st);

}  // namespace slim
