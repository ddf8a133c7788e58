// Reverse mode of scan integration for a map integrated from empty (zero
// priors: the final state is the batch posterior of all observations,
// Theorems 1-2). For one scan, per point j and each of its (voxel v, point j)
// observations, recomputed by the same band DDA as the forward pass:
//   D_v = (sum d) / W_v         ->  dL/dd_vj = dL/dD_v / W_v  (0 if d clamped)
//   d = (x - c_v) . u, u = (x - o) / r
//                               ->  dd/dx = u + (I - u u^T)(x - c_v) / r
//   x = R p + t                 ->  dL/dp = R^T dL/dx
//   closed soft: c_v = sum p_j  ->  dL/dp_j += dL/dc_v
//   open: m_v = sum z / W_v, beta_v = 1/2 sum (z - m_v)^2
//                               ->  dL/dz_j += dL/dm_v / W_v
//                                              + dL/dbeta_v * (z_j - m_v)
// Open set: one warp per point, every lane walks the same DDA and lanes
// split the embedding dimension; closed set: one thread per point. The
// result is a gather (the adjoint of the forward scatter), so no atomics.
#include <cuda_bf16.h>

#include <algorithm>

#include "geometry.cuh"
#include "hash.cuh"
#include "map.h"

namespace slim {

template <int OPEN, int BF16>
__global__ void __launch_bounds__(256) k_backward(MapView mv, ScanGeom g,
                                                  const float* __restrict__ pts,
                                                  const float* __restrict__ sem, int64_t n,
                                                  int width, const float* __restrict__ gD,
                                                  const float* __restrict__ gS,
                                                  const float* __restrict__ gB, float* gsem,
                                                  float* gxyz, int sem_grad) {
  const unsigned lane = lane_id();
  const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j >= n) return;
  float acc[32];  // this lane's share of dL/dsem_j: elements lane + 32 k
  const int per = (width + 31) / 32;
#pragma unroll
  for (int k = 0; k < 32; ++k) acc[k] = 0.f;
  float gx0 = 0.f, gx1 = 0.f, gx2 = 0.f;
  Ray ry;
  const bool valid = ray_setup(g, pts[3 * j], pts[3 * j + 1], pts[3 * j + 2], ry);
  if (valid) {
    const float* zrow = sem + (size_t)j * width;
    uint64_t last = kEmptyKey;
    uint32_t slot = kNoSlot;
    ray_for_each(g, ry, [&](int32_t i0, int32_t i1, int32_t i2, float d) {
      const uint64_t kb = pack_block(i0 >> 3, i1 >> 3, i2 >> 3);
      if (kb != last) {
        last = kb;
        slot = hash_find(mv, kb);
      }
      if (slot == kNoSlot) return;
      const size_t vox = (size_t)slot * kBlockVoxels + local_index(i0, i1, i2);
      float Wv;
      size_t gi;
      if (OPEN) {
        const int32_t row = mv.vox_row[vox];
        if (row < 0) return;
        Wv = mv.tsdf[row].y;
        gi = (size_t)row;
      } else {
        Wv = rec_weight(mv.rec + vox * mv.rs, mv.K, mv.layout);
        gi = vox;
      }
      const float invW = 1.0f / Wv;
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        if (k >= per || !sem_grad) break;
        const int e = (int)lane + 32 * k;
        if (e >= width) break;
        const size_t o = gi * (size_t)width + e;
        if (OPEN) {
          float gm = gS[o] * invW;
          if (gB) {
            const float mval = BF16 ? __bfloat162float(static_cast<const __nv_bfloat16*>(mv.mrow)[o])
                                    : static_cast<const float*>(mv.mrow)[o];
            gm += gB[o] * (zrow[e] - mval);
          }
          acc[k] += gm;
        } else {
          acc[k] += gS[o];
        }
      }
      if (!(d < g.tau)) return;  // clamped at tau: no dependence on x
      const float gd = gD[gi] * invW;
      const float c0 = ((float)i0 + 0.5f) * g.v, c1 = ((float)i1 + 0.5f) * g.v,
                  c2 = ((float)i2 + 0.5f) * g.v;
      const float e0 = ry.x0 - c0, e1 = ry.x1 - c1, e2 = ry.x2 - c2;
      const float eu = e0 * ry.u0 + e1 * ry.u1 + e2 * ry.u2;
      const float ir = 1.0f / ry.r;
      gx0 += gd * (ry.u0 + (e0 - ry.u0 * eu) * ir);
      gx1 += gd * (ry.u1 + (e1 - ry.u1 * eu) * ir);
      gx2 += gd * (ry.u2 + (e2 - ry.u2 * eu) * ir);
    });
  }
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    if (k >= per) break;
    const int e = (int)lane + 32 * k;
    if (e < width) gsem[(size_t)j * width + e] = acc[k];
  }
  if (lane == 0) {
    // dL/dp = R^T dL/dx
    gxyz[3 * j + 0] = g.R[0] * gx0 + g.R[3] * gx1 + g.R[6] * gx2;
    gxyz[3 * j + 1] = g.R[1] * gx0 + g.R[4] * gx1 + g.R[7] * gx2;
    gxyz[3 * j + 2] = g.R[2] * gx0 + g.R[5] * gx1 + g.R[8] * gx2;
  }
}

// The geometric term of one pair: gx += gd dd/dx with
// dd/dx = u + (I - u u^T)(x - c) / r, c the centre of voxel (i0, i1, i2).
// Every operation is rounded on its own (no contraction), so the recomputing
// and the stored-pair kernels give the same bits.
__device__ __forceinline__ void add_sdf_grad(const Ray& ry, int32_t i0, int32_t i1, int32_t i2,
                                             float v, float gd, float& gx0, float& gx1,
                                             float& gx2) {
  const float e0 = __fsub_rn(ry.x0, __fmul_rn(__fadd_rn((float)i0, 0.5f), v));
  const float e1 = __fsub_rn(ry.x1, __fmul_rn(__fadd_rn((float)i1, 0.5f), v));
  const float e2 = __fsub_rn(ry.x2, __fmul_rn(__fadd_rn((float)i2, 0.5f), v));
  const float eu = __fadd_rn(__fadd_rn(__fmul_rn(e0, ry.u0), __fmul_rn(e1, ry.u1)),
                             __fmul_rn(e2, ry.u2));
  const float ir = __fdiv_rn(1.0f, ry.r);
  gx0 = __fadd_rn(gx0, __fmul_rn(gd, __fadd_rn(ry.u0, __fmul_rn(__fsub_rn(e0, __fmul_rn(ry.u0, eu)), ir))));
  gx1 = __fadd_rn(gx1, __fmul_rn(gd, __fadd_rn(ry.u1, __fmul_rn(__fsub_rn(e1, __fmul_rn(ry.u1, eu)), ir))));
  gx2 = __fadd_rn(gx2, __fmul_rn(gd, __fadd_rn(ry.u2, __fmul_rn(__fsub_rn(e2, __fmul_rn(ry.u2, eu)), ir))));
}

// dL/dp = R^T dL/dx, each operation rounded on its own.
__device__ __forceinline__ void store_point_grad(const ScanGeom& g, float gx0, float gx1,
                                                 float gx2, float* out) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
    out[a] = __fadd_rn(__fadd_rn(__fmul_rn(g.R[a], gx0), __fmul_rn(g.R[3 + a], gx1)),
                       __fmul_rn(g.R[6 + a], gx2));
}

// Closed set: one thread per point (the class gradient of a pair is a
// K-vector, so a warp per point would repeat the DDA 32 times). The thread
// accumulates its output row dL/dsem_j in registers (KMAX >= K, unrolled, so
// the row never leaves the register file) in pair order, reading each pair's
// K incoming class gradients as float4 where the row allows, and writes the
// row once.
template <int KMAX>
__global__ void __launch_bounds__(256) k_backward_closed(MapView mv, ScanGeom g,
                                                         const float* __restrict__ pts, int64_t n,
                                                         int K, const float* __restrict__ gD,
                                                         const float* __restrict__ gS,
                                                         float* gsem, float* gxyz, int sem_grad) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  float acc[KMAX];
#pragma unroll
  for (int k = 0; k < KMAX; ++k) acc[k] = 0.f;
  const bool vec = (K & 3) == 0;
  float gx0 = 0.f, gx1 = 0.f, gx2 = 0.f;
  Ray ry;
  if (ray_setup(g, pts[3 * j], pts[3 * j + 1], pts[3 * j + 2], ry)) {
    uint64_t last = kEmptyKey;
    uint32_t slot = kNoSlot;
    ray_for_each(g, ry, [&](int32_t i0, int32_t i1, int32_t i2, float d) {
      const uint64_t kb = pack_block(i0 >> 3, i1 >> 3, i2 >> 3);
      if (kb != last) {
        last = kb;
        slot = hash_find(mv, kb);
      }
      if (slot >= mv.block_cap) return;
      const size_t vox = (size_t)slot * kBlockVoxels + local_index(i0, i1, i2);
      const float Wv = rec_weight(mv.rec + vox * mv.rs, mv.K, mv.layout);
      const float invW = __fdiv_rn(1.0f, Wv);
      if (sem_grad) {
        const float* row = gS + vox * (size_t)K;
        if (vec) {
#pragma unroll
          for (int k = 0; k < KMAX; k += 4) {
            if (k < K) {
              const float4 v = __ldg(reinterpret_cast<const float4*>(row + k));
              acc[k] += v.x;
              acc[k + 1] += v.y;
              acc[k + 2] += v.z;
              acc[k + 3] += v.w;
            }
          }
        } else {
#pragma unroll
          for (int k = 0; k < KMAX; ++k)
            if (k < K) acc[k] += __ldg(row + k);
        }
      }
      if (!(d < g.tau)) return;  // clamped at tau: no dependence on x
      add_sdf_grad(ry, i0, i1, i2, g.v, __fmul_rn(gD[vox], invW), gx0, gx1, gx2);
    });
  }
  float* out = gsem + (size_t)j * K;
#pragma unroll
  for (int k = 0; k < KMAX; ++k)
    if (k < K) out[k] = acc[k];
  store_point_grad(g, gx0, gx1, gx2, gxyz + 3 * j);
}

// Stored pair list (closed set): the (voxel, point) observations of one scan
// of a complete map, in point order and ray order within a point (CSR by
// point), each pair the voxel's record index slot * 512 + local. WRITE = 0
// counts each point's pairs, WRITE = 1 writes them at offsets[j].
template <int WRITE>
__global__ void __launch_bounds__(256) k_pairs_walk(MapView mv, ScanGeom g,
                                                    const float* __restrict__ pts, int64_t n,
                                                    uint32_t* counts,
                                                    const uint32_t* __restrict__ offsets,
                                                    uint32_t* vox) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  uint32_t k = 0;
  Ray ry;
  if (ray_setup(g, pts[3 * j], pts[3 * j + 1], pts[3 * j + 2], ry)) {
    uint32_t* out = WRITE ? vox + offsets[j] : nullptr;
    uint64_t last = kEmptyKey;
    uint32_t slot = kNoSlot;
    ray_for_each(g, ry, [&](int32_t i0, int32_t i1, int32_t i2, float) {
      const uint64_t kb = pack_block(i0 >> 3, i1 >> 3, i2 >> 3);
      if (kb != last) {
        last = kb;
        slot = hash_find(mv, kb);
      }
      if (slot >= mv.block_cap) return;
      if (WRITE) out[k] = slot * (uint32_t)kBlockVoxels + (uint32_t)local_index(i0, i1, i2);
      ++k;
    });
  }
  if (!WRITE) counts[j] = k;
}

// The reverse mode of k_backward_closed over a stored pair list: the same
// per-pair terms in the same order (so the same result bit for bit), with
// each pair's voxel read from the list instead of found by the band walk
// and the hash. The ray (x, u, r) is set up again per point and each pair's
// SDF recomputed from its voxel's coordinates in the forward's FP32 order.
template <int KMAX>
__global__ void __launch_bounds__(256) k_backward_pairs(MapView mv, ScanGeom g,
                                                        const float* __restrict__ pts, int64_t n,
                                                        const uint32_t* __restrict__ offsets,
                                                        const uint32_t* __restrict__ vox, int K,
                                                        const float* __restrict__ gD,
                                                        const float* __restrict__ gS,
                                                        float* gsem, float* gxyz, int sem_grad) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  float acc[KMAX];
#pragma unroll
  for (int k = 0; k < KMAX; ++k) acc[k] = 0.f;
  const bool vec = (K & 3) == 0;
  float gx0 = 0.f, gx1 = 0.f, gx2 = 0.f;
  Ray ry;
  if (ray_setup(g, pts[3 * j], pts[3 * j + 1], pts[3 * j + 2], ry)) {
    const uint32_t p1 = offsets[j + 1];
    for (uint32_t p = offsets[j]; p < p1; ++p) {
      const uint32_t v = vox[p];
      const uint32_t slot = v / (uint32_t)kBlockVoxels, loc = v % (uint32_t)kBlockVoxels;
      int32_t b0, b1, b2;
      unpack_block(mv.blk_key[slot], b0, b1, b2);
      ry.i0 = b0 * 8 + (int32_t)(loc >> 6);
      ry.i1 = b1 * 8 + (int32_t)((loc >> 3) & 7u);
      ry.i2 = b2 * 8 + (int32_t)(loc & 7u);
      const size_t vx = (size_t)v;
      const float Wv = rec_weight(mv.rec + vx * mv.rs, mv.K, mv.layout);
      const float invW = __fdiv_rn(1.0f, Wv);
      if (sem_grad) {
        const float* row = gS + vx * (size_t)K;
        if (vec) {
#pragma unroll
          for (int k = 0; k < KMAX; k += 4) {
            if (k < K) {
              const float4 q = __ldg(reinterpret_cast<const float4*>(row + k));
              acc[k] += q.x;
              acc[k + 1] += q.y;
              acc[k + 2] += q.z;
              acc[k + 3] += q.w;
            }
          }
        } else {
#pragma unroll
          for (int k = 0; k < KMAX; ++k)
            if (k < K) acc[k] += __ldg(row + k);
        }
      }
      if (!(ray_sdf(ry, g.v) < g.tau)) continue;  // clamped at tau: no dependence on x
      add_sdf_grad(ry, ry.i0, ry.i1, ry.i2, g.v, __fmul_rn(gD[vx], invW), gx0, gx1, gx2);
    }
  }
  float* out = gsem + (size_t)j * K;
#pragma unroll
  for (int k = 0; k < KMAX; ++k)
    if (k < K) out[k] = acc[k];
  store_point_grad(g, gx0, gx1, gx2, gxyz + 3 * j);
}

slim_status run_backward(slim_map* m, const ScanGeom& g, const float* pts, const float* sem,
                         int64_t n, const float* gD, const float* gS, const float* gB,
                         float* gsem, float* gxyz, cudaStream_t st) {
  if (n <= 0) return SLIM_OK;
  const int width = m->mode == SLIM_OPEN ? m->L : m->K;
  const unsigned grid = (unsigned)((n * 32 + 255) / 256);
  const int tok = prof_begin(m, SLIM_KERNEL_BACKWARD, st);
  const int sg = m->mode == SLIM_CLOSED_ONEHOT ? 0 : 1;  // argmax has no gradient
  if (m->mode == SLIM_OPEN) {
    if (m->bf16)
      k_backward<1, 1><<<grid, 256, 0, st>>>(m->mv, g, pts, sem, n, width, gD, gS, gB, gsem, gxyz,
                                             sg);
    else
      k_backward<1, 0><<<grid, 256, 0, st>>>(m->mv, g, pts, sem, n, width, gD, gS, gB, gsem, gxyz,
                                             sg);
  } else {
    const unsigned cg = (unsigned)((n + 255) / 256);
    if (width <= 16)
      k_backward_closed<16><<<cg, 256, 0, st>>>(m->mv, g, pts, n, width, gD, gS, gsem, gxyz, sg);
    else if (width <= 32)
      k_backward_closed<32><<<cg, 256, 0, st>>>(m->mv, g, pts, n, width, gD, gS, gsem, gxyz, sg);
    else
      k_backward_closed<64><<<cg, 256, 0, st>>>(m->mv, g, pts, n, width, gD, gS, gsem, gxyz, sg);
  }
  prof_end(m, tok, st);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(SLIM_ERR_CUDA, cudaGetErrorString(e));
  return SLIM_OK;
}

// Pairs of one scan into offsets (n + 1 entries) and vox (cap entries): a
// counting walk, an exclusive scan, then (cap large enough) a writing walk.
// *n_pairs receives the total; the call synchronises the stream.
slim_status run_record_pairs(slim_map* m, const ScanGeom& g, const float* pts, int64_t n,
                             uint32_t* offsets, uint32_t* vox, int64_t cap, int64_t* n_pairs,
                             cudaStream_t st) {
  const int64_t np = std::max<int64_t>(m->p.max_points, 1);
  if (!m->pr_counts) {  // first use: the count buffer and the scan's partials
    slim_status s;
    if ((s = m->alloc(&m->pr_counts, (size_t)np)) != SLIM_OK) return s;
    if ((s = m->alloc(&m->pr_tmp, (size_t)((np + 4095) / 4096 + 64))) != SLIM_OK) return s;
  }
  cudaError_t e = cudaSuccess;
  if (n > 0) {
    const unsigned grid = (unsigned)((n + 255) / 256);
    k_pairs_walk<0><<<grid, 256, 0, st>>>(m->mv, g, pts, n, m->pr_counts, nullptr, nullptr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = exclusive_scan_u32(m->pr_counts, offsets, n, m->pr_tmp, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(m->pinned + kNumCounters, offsets + n, sizeof(uint32_t),
                        cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(SLIM_ERR_CUDA, cudaGetErrorString(e));
  const int64_t total = (int64_t)m->pinned[kNumCounters];
  *n_pairs = total;
  if (cap == 0) return SLIM_OK;
  if (cap < total) return fail(SLIM_ERR_CAPACITY, "cap smaller than the scan's pair count");
  if (n > 0 && total > 0) {
    const unsigned grid = (unsigned)((n + 255) / 256);
    k_pairs_walk<1><<<grid, 256, 0, st>>>(m->mv, g, pts, n, nullptr, offsets, vox);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(SLIM_ERR_CUDA, cudaGetErrorString(e));
  }
  return SLIM_OK;
}

slim_status run_backward_pairs(slim_map* m, const ScanGeom& g, const float* pts, int64_t n,
                               const uint32_t* offsets, const uint32_t* vox, const float* gD,
                               const float* gS, float* gsem, float* gxyz, cudaStream_t st) {
  if (n <= 0) return SLIM_OK;
  const int K = m->K;
  const int sg = m->mode == SLIM_CLOSED_ONEHOT ? 0 : 1;  // argmax has no gradient
  const unsigned cg = (unsigned)((n + 255) / 256);
  const int tok = prof_begin(m, SLIM_KERNEL_BACKWARD, st);
  if (K <= 16)
    k_backward_pairs<16><<<cg, 256, 0, st>>>(m->mv, g, pts, n, offsets, vox, K, gD, gS, gsem,
                                             gxyz, sg);
  else if (K <= 32)
    k_backward_pairs<32><<<cg, 256, 0, st>>>(m->mv, g, pts, n, offsets, vox, K, gD, gS, gsem,
                                             gxyz, sg);
  else
    k_backward_pairs<64><<<cg, 256, 0, st>>>(m->mv, g, pts, n, offsets, vox, K, gD, gS, gsem,
                                             gxyz, sg);
  prof_end(m, tok, st);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(SLIM_ERR_CUDA, cudaGetErrorString(e));
  return SLIM_OK;
}

}  // namespace slim
