// Map export (read-out): every allocated voxel (W > 0) in block-key order,
// then local order, with D = S / W, W and the semantic state; the closed-set
// posterior predictive of Eq. (dir_to_cat), (alpha0 + c_i) / (K alpha0 + sum c),
// is formed here on request, and so is the uncertainty read-out: the
// variance of each class probability under the Dirichlet posterior and the
// entropy of its predictive (closed set), or the variance of the Student-t
// predictive of Eq. (student_t) with lambda = 2 nu = W (open set).
#include <cuda_bf16.h>

#include "block_sort.cuh"
#include "internal.h"

namespace slim {

__global__ void k_gather_keys(const uint64_t* __restrict__ blk_key, int64_t nb, uint64_t* keys,
                              uint32_t* slots) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < nb) {
    keys[s] = blk_key[s];
    slots[s] = (uint32_t)s;
  }
}

__device__ __forceinline__ bool voxel_present(const MapView& mv, bool open, uint32_t slot,
                                              int l, int32_t* row) {
  if (open) {
    const int32_t r = mv.vox_row[(size_t)slot * kBlockVoxels + l];
    *row = r;
    return r >= 0 && mv.tsdf[r].y > 0.f;
  }
  *row = -1;
  return rec_weight(mv.rec + ((size_t)slot * kBlockVoxels + l) * mv.rs, mv.K, mv.layout) > 0.f;
}

__global__ void __launch_bounds__(256) k_extract_count(MapView mv, const uint32_t* __restrict__ slots,
                                                       int64_t nb, int open, uint32_t* counts) {
  __shared__ uint32_t wt[kCtaWarps];
  const uint32_t slot = slots[blockIdx.x];
  int32_t row;
  uint32_t c = voxel_present(mv, open, slot, 2 * threadIdx.x, &row) +
               voxel_present(mv, open, slot, 2 * threadIdx.x + 1, &row);
  uint32_t tot;
  cta_exclusive_scan(c, wt, &tot);
  if (threadIdx.x == 0) counts[blockIdx.x] = tot;
}

__device__ __forceinline__ float load_elem(const void* p, size_t i, int bf16) {
  if (bf16) return __bfloat162float(static_cast<const __nv_bfloat16*>(p)[i]);
  return static_cast<const float*>(p)[i];
}

__global__ void __launch_bounds__(256) k_extract_write(MapView mv, const uint32_t* __restrict__ slots,
                                                       const uint64_t* __restrict__ keys,
                                                       const uint32_t* __restrict__ offsets,
                                                       ExtractArgs a) {
  __shared__ uint32_t wt[kCtaWarps];
  const uint32_t slot = slots[blockIdx.x];
  int32_t bx, by, bz;
  unpack_block(keys[blockIdx.x], bx, by, bz);
  const bool open = a.mode == 2;
  int32_t row[2];
  bool pr[2];
  uint32_t c = 0;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    pr[h] = voxel_present(mv, open, slot, 2 * threadIdx.x + h, &row[h]);
    c += pr[h];
  }
  uint32_t tot;
  uint32_t pos = offsets[blockIdx.x] + cta_exclusive_scan(c, wt, &tot);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    if (!pr[h]) continue;
    const int l = 2 * threadIdx.x + h;
    const size_t o = pos++;
    if (a.ijk) {
      a.ijk[3 * o + 0] = bx * 8 + (l >> 6);
      a.ijk[3 * o + 1] = by * 8 + ((l >> 3) & 7);
      a.ijk[3 * o + 2] = bz * 8 + (l & 7);
    }
    if (!open && a.mode == SLIM_CLOSED_LATEST) {
      // {S, W, stamp}: the label is the stamp's low byte
      const float* r = mv.rec + ((size_t)slot * kBlockVoxels + l) * mv.rs;
      if (a.D) a.D[o] = r[0] / r[1];
      if (a.W) a.W[o] = r[1];
      if (a.index) a.index[o] = (int32_t)(slot * kBlockVoxels + l);
      if (a.sem) {
        const uint32_t lab = (uint32_t)(*reinterpret_cast<const unsigned long long*>(r + 2) & 0xFF);
        for (int k = 0; k < a.K; ++k) a.sem[o * a.K + k] = k == (int)lab ? 1.f : 0.f;
      }
    } else if (!open) {
      const float* r = mv.rec + ((size_t)slot * kBlockVoxels + l) * mv.rs;
      // one-hot records hold (S_k, c_k) pairs, soft records fixed-point
      // (S, W, c_k)
      const int lay = mv.layout;
      const float W = rec_weight(r, a.K, lay);
      if (a.D) a.D[o] = rec_sdf(r, a.K, lay);
      if (a.W) a.W[o] = W;
      if (a.index) a.index[o] = (int32_t)(slot * kBlockVoxels + l);
      if (a.unc) {
        // Dir(alpha~), alpha~_i = alpha0 + c_i, A = sum alpha~:
        // Var theta_i = alpha~_i (A - alpha~_i) / (A^2 (A + 1)); entropy of p = alpha~ / A
        const float A = (float)a.K * a.alpha0 + rec_count_sum(r, a.K, lay);
        const float den = A * A * (A + 1.f);
        float H = 0.f;
        for (int k = 0; k < a.K; ++k) {
          const float al = a.alpha0 + rec_count(r, k, lay);
          a.unc[o * (a.K + 1) + k] = al * (A - al) / den;
          const float p = al / A;
          if (p > 0.f) H -= p * logf(p);
        }
        a.unc[o * (a.K + 1) + a.K] = H;
      }
      if (a.sem) {
        if (a.flags & SLIM_EXTRACT_POSTERIOR) {
          const float den = (float)a.K * a.alpha0 + rec_count_sum(r, a.K, lay);
          for (int k = 0; k < a.K; ++k)
            a.sem[o * a.K + k] = (a.alpha0 + rec_count(r, k, lay)) / den;
        } else {
          for (int k = 0; k < a.K; ++k) a.sem[o * a.K + k] = rec_count(r, k, lay);
        }
      }
    } else {
      const int32_t rw = row[h];
      const float2 sw = mv.tsdf[rw];
      if (a.D) a.D[o] = sw.x / sw.y;
      if (a.W) a.W[o] = sw.y;
      if (a.index) a.index[o] = rw;
      if (a.sem)
        for (int k = 0; k < a.L; ++k)
          a.sem[o * a.L + k] = load_elem(mv.mrow, (size_t)rw * a.L + k, a.bf16);
      if (a.beta)
        for (int k = 0; k < a.L; ++k)
          a.beta[o * a.L + k] = load_elem(mv.brow, (size_t)rw * a.L + k, a.bf16);
      if (a.unc) {
        // Student-t with 2 nu = W degrees of freedom: variance
        // 2 beta (W + 1) / (W (W - 2)) for W > 2, else infinite
        const float Wv = sw.y;
        const float f = Wv > 2.f ? 2.f * (Wv + 1.f) / (Wv * (Wv - 2.f)) : INFINITY;
        for (int k = 0; k < a.L; ++k)
          a.unc[o * a.L + k] =
              Wv > 2.f ? f * load_elem(mv.brow, (size_t)rw * a.L + k, a.bf16) : INFINITY;
      }
    }
  }
}

cudaError_t launch_gather_keys(const MapView& mv, int64_t nb, uint64_t* keys, uint32_t* slots,
                               cudaStream_t st) {
  if (nb <= 0) return cudaSuccess;
  k_gather_keys<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(mv.blk_key, nb, keys, slots);
  return cudaGetLastError();
}

cudaError_t launch_extract_count(const MapView& mv, const uint32_t* slots, int64_t nb,
                                 bool open, uint32_t* counts, cudaStream_t st) {
  if (nb <= 0) return cudaSuccess;
  k_extract_count<<<(unsigned)nb, kCtaThreads, 0, st>>>(mv, slots, nb, open ? 1 : 0, counts);
  return cudaGetLastError();
}

cudaError_t launch_extract_write(const MapView& mv, const uint32_t* slots,
                                 const uint64_t* keys, int64_t nb, const uint32_t* offsets,
                                 const ExtractArgs& a, cudaStream_t st) {
  if (nb <= 0) return cudaSuccess;
  k_extract_write<<<(unsigned)nb, kCtaThreads, 0, st>>>(mv, slots, keys, offsets, a);
  return cudaGetLastError();
}

}  // namespace slim
