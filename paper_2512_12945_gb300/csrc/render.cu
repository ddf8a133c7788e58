// Ray-cast render of the map from a pinhole camera (Sec. III-E: the map is
// rendered from a camera viewpoint rather than meshed; the paper renders the
// VDB grid with NanoVDB). One thread per pixel (row-major): the camera ray
// enters voxels for t in [near, far] by the same FP32 Amanatides & Woo
// traversal as integration (explicitly rounded ops in a fixed order, ties to
// the lowest axis); the block of the current voxel is looked up in the
// map's hash only when the ray enters a new block. A voxel is observed when
// its weight is positive; its ray parameter is the projection of its centre
// t_c = (c - o) . u. The surface is the first pair of consecutive entered
// voxels, both observed, with D_prev > 0 >= D: depth = t_prev +
// (t_c - t_prev) D_prev / (D_prev - D). At that voxel the kernel writes its
// indices, the closed-set label (largest count, ties to the lowest class)
// and, for the open set and a query q, the cosine m . q / (|m| |q|).
#include <cuda_bf16.h>

#include "closed_common.cuh"
#include "geometry.cuh"
#include "hash.cuh"
#include "map.h"

namespace slim {

struct RenderArgs {
  MapView mv;
  const int32_t* bounds;  // min bx, by, bz, max bx, by, bz of the allocated blocks
  float R[9];  // world_from_camera rotation (FP32)
  float o[3];  // camera centre
  float fx, fy, cx, cy;
  int32_t width, height;
  float t0, t1, v;
  int32_t cap;  // 3 ceil((far - near) / v) + 3
  int32_t open, latest, K, L, bf16;
  const float* q;  // open set: l-vector or null
  float* depth;
  int32_t* ijk;
  int32_t* label;
  float* sim;
};

__device__ __forceinline__ float render_elem(const void* p, size_t i, int bf16) {
  if (bf16) return __bfloat162float(static_cast<const __nv_bfloat16*>(p)[i]);
  return static_cast<const float*>(p)[i];
}

__global__ void __launch_bounds__(256) k_render(const __grid_constant__ RenderArgs a) {
  __shared__ float s_qinv;
  if (threadIdx.x < 32) {  // 1 / |q| of the query (open set)
    float s = 0.f;
    if (a.q)
      for (int c = threadIdx.x; c < a.L; c += 32) s += a.q[c] * a.q[c];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, off);
    if (threadIdx.x == 0) s_qinv = s > 0.f ? rsqrtf(s) : 0.f;
  }
  __syncthreads();
  const int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= (int64_t)a.width * a.height) return;
  const int32_t px = (int32_t)(pix % a.width), py = (int32_t)(pix / a.width);
  const MapView& mv = a.mv;
  // camera ray, FP32 in a fixed order
  const float dx = __fdiv_rn(__fsub_rn(__fadd_rn((float)px, 0.5f), a.cx), a.fx);
  const float dy = __fdiv_rn(__fsub_rn(__fadd_rn((float)py, 0.5f), a.cy), a.fy);
  const float n2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), 1.0f);
  const float nn = __fsqrt_rn(n2);
  const float d[3] = {__fdiv_rn(dx, nn), __fdiv_rn(dy, nn), __fdiv_rn(1.0f, nn)};
  float u[3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
    u[k] = __fadd_rn(__fadd_rn(__fmul_rn(a.R[k * 3 + 0], d[0]), __fmul_rn(a.R[k * 3 + 1], d[1])),
                     __fmul_rn(a.R[k * 3 + 2], d[2]));
  // traversal state, initialised as in integration with t in [t0, t1]
  Ray ry;
  ry.u0 = u[0];
  ry.u1 = u[1];
  ry.u2 = u[2];
  ry.t1 = a.t1;
  {
    int32_t ii[3], st[3];
    float tm[3], td[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float s = __fadd_rn(a.o[k], __fmul_rn(a.t0, u[k]));
      ii[k] = (int32_t)floorf(__fdiv_rn(s, a.v));
      st[k] = u[k] > 0.0f ? 1 : (u[k] < 0.0f ? -1 : 0);
      if (u[k] != 0.0f) {
        td[k] = __fdiv_rn(a.v, fabsf(u[k]));
        const float bnd = __fmul_rn((float)(ii[k] + (st[k] > 0 ? 1 : 0)), a.v);
        tm[k] = __fadd_rn(a.t0, __fdiv_rn(__fsub_rn(bnd, s), u[k]));
      } else {
        td[k] = __int_as_float(0x7f800000);
        tm[k] = __int_as_float(0x7f800000);
      }
    }
    ry.i0 = ii[0]; ry.i1 = ii[1]; ry.i2 = ii[2];
    ry.s0 = st[0]; ry.s1 = st[1]; ry.s2 = st[2];
    ry.m0 = tm[0]; ry.m1 = tm[1]; ry.m2 = tm[2];
    ry.e0 = td[0]; ry.e1 = td[1]; ry.e2 = td[2];
  }
  // the allocated blocks' bounding box: once the ray is beyond it on an
  // axis it does not travel back along, no later voxel can be observed
  const int32_t lo0 = a.bounds[0], lo1 = a.bounds[1], lo2 = a.bounds[2];
  const int32_t hi0 = a.bounds[3], hi1 = a.bounds[4], hi2 = a.bounds[5];
  bool fresh = true, have_prev = false;
  uint32_t slot = kNoSlot;
  float Dp = 0.f, tp = 0.f;
  for (int k = 0; k < a.cap; ++k) {
    if (fresh) {
      const int32_t b0 = ry.i0 >> 3, b1 = ry.i1 >> 3, b2 = ry.i2 >> 3;
      if ((b0 > hi0 && ry.s0 >= 0) || (b0 < lo0 && ry.s0 <= 0) || (b1 > hi1 && ry.s1 >= 0) ||
          (b1 < lo1 && ry.s1 <= 0) || (b2 > hi2 && ry.s2 >= 0) || (b2 < lo2 && ry.s2 <= 0))
        break;
      slot = hash_find(mv, pack_block(b0, b1, b2));
      fresh = false;
    }
    float W = 0.f, D = 0.f;
    int32_t row = -1;
    if (slot < mv.block_cap) {
      const size_t vox = (size_t)slot * kBlockVoxels + local_index(ry.i0, ry.i1, ry.i2);
      if (a.open) {
        row = mv.vox_row[vox];
        if (row >= 0) {
          const float2 sw = mv.tsdf[row];
          W = sw.y;
          D = W > 0.f ? sw.x / sw.y : 0.f;
        }
      } else {
        const float* r = mv.rec + vox * mv.rs;
        W = rec_weight(r, mv.K, mv.layout);
        D = rec_sdf(r, mv.K, mv.layout);
      }
    }
    if (W > 0.f) {
      const float c0 = __fmul_rn(__fadd_rn((float)ry.i0, 0.5f), a.v);
      const float c1 = __fmul_rn(__fadd_rn((float)ry.i1, 0.5f), a.v);
      const float c2 = __fmul_rn(__fadd_rn((float)ry.i2, 0.5f), a.v);
      const float tc = __fadd_rn(__fadd_rn(__fmul_rn(__fsub_rn(c0, a.o[0]), u[0]),
                                           __fmul_rn(__fsub_rn(c1, a.o[1]), u[1])),
                                 __fmul_rn(__fsub_rn(c2, a.o[2]), u[2]));
      if (have_prev && Dp > 0.f && D <= 0.f) {
        a.depth[pix] = tp + (tc - tp) * Dp / (Dp - D);
        if (a.ijk) {
          a.ijk[3 * pix + 0] = ry.i0;
          a.ijk[3 * pix + 1] = ry.i1;
          a.ijk[3 * pix + 2] = ry.i2;
        }
        int32_t lab = -1;
        if (a.latest) {
          const size_t vox = (size_t)slot * kBlockVoxels + local_index(ry.i0, ry.i1, ry.i2);
          const float* r = mv.rec + vox * mv.rs;
          lab = (int32_t)(*reinterpret_cast<const unsigned long long*>(r + 2) & 0xFF);
        } else if (!a.open) {
          const size_t vox = (size_t)slot * kBlockVoxels + local_index(ry.i0, ry.i1, ry.i2);
          const float* r = mv.rec + vox * mv.rs;
          lab = 0;
          if (mv.layout == kRecSoftFx) {  // exact integer counts
            const long long* q = rec_fx(r) + 2;
            long long bv = q[0];
            for (int c = 1; c < mv.K; ++c)
              if (q[c] > bv) {
                bv = q[c];
                lab = c;
              }
          } else {
            float bv = r[1];
            for (int c = 1; c < mv.K; ++c)
              if (r[2 * c + 1] > bv) {
                bv = r[2 * c + 1];
                lab = c;
              }
          }
        }
        if (a.label) a.label[pix] = lab;
        if (a.sim) {
          float s = 0.f;
          if (a.open && a.q) {
            float dot = 0.f;
            for (int c = 0; c < a.L; ++c)
              dot += render_elem(mv.mrow, (size_t)row * a.L + c, a.bf16) * a.q[c];
            const float m2 = mv.mnorm2[row];
            s = m2 > 0.f ? dot * rsqrtf(m2) * s_qinv : 0.f;
          }
          a.sim[pix] = s;
        }
        return;
      }
      have_prev = true;
      Dp = D;
      tp = tc;
    } else {
      have_prev = false;
    }
    bool crossed;
    if (!ray_step_blk(ry, crossed)) break;
    fresh = crossed;
  }
  a.depth[pix] = __int_as_float(0x7f800000);
  if (a.ijk) a.ijk[3 * pix + 0] = a.ijk[3 * pix + 1] = a.ijk[3 * pix + 2] = INT32_MIN;
  if (a.label) a.label[pix] = -1;
  if (a.sim) a.sim[pix] = 0.f;
}

// Bounding box of the allocated blocks (slots below the allocation counter).
__global__ void __launch_bounds__(256) k_block_bounds(const uint64_t* __restrict__ blk_key,
                                                      const uint32_t* ctr, uint32_t block_cap,
                                                      int32_t* bounds) {
  const uint32_t nb = min(*(volatile const uint32_t*)&ctr[kCtrBlocks], block_cap);
  int32_t lo[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, hi[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < nb; s += gridDim.x * blockDim.x) {
    int32_t b[3];
    unpack_block(blk_key[s], b[0], b[1], b[2]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      lo[k] = min(lo[k], b[k]);
      hi[k] = max(hi[k], b[k]);
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      lo[k] = min(lo[k], __shfl_xor_sync(0xFFFFFFFFu, lo[k], off));
      hi[k] = max(hi[k], __shfl_xor_sync(0xFFFFFFFFu, hi[k], off));
    }
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      atomicMin(&bounds[k], lo[k]);
      atomicMax(&bounds[3 + k], hi[k]);
    }
  }
}

__global__ void k_bounds_init(int32_t* bounds) {
  if (threadIdx.x < 3) bounds[threadIdx.x] = INT32_MAX;
  else if (threadIdx.x < 6) bounds[threadIdx.x] = INT32_MIN;
}

slim_status run_render(slim_map* m, const double world_from_camera[16], float fx, float fy,
                       float cx, float cy, int32_t width, int32_t height, float near_t,
                       float far_t, const float* q, float* depth, int32_t* ijk, int32_t* label,
                       float* sim, cudaStream_t st) {
  RenderArgs a;
  a.mv = m->mv;
  a.bounds = m->render_bounds;
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) a.R[r * 3 + c] = (float)world_from_camera[r * 4 + c];
    a.o[r] = (float)world_from_camera[r * 4 + 3];
  }
  a.fx = fx;
  a.fy = fy;
  a.cx = cx;
  a.cy = cy;
  a.width = width;
  a.height = height;
  a.t0 = near_t;
  a.t1 = far_t;
  a.v = m->p.voxel_size;
  a.cap = 3 * (int32_t)std::ceil(((double)far_t - (double)near_t) / (double)a.v) + 3;
  a.open = m->mode == SLIM_OPEN ? 1 : 0;
  a.latest = m->mode == SLIM_CLOSED_LATEST ? 1 : 0;
  a.K = m->K;
  a.L = m->L;
  a.bf16 = m->bf16 ? 1 : 0;
  a.q = a.open ? q : nullptr;
  a.depth = depth;
  a.ijk = ijk;
  a.label = label;
  a.sim = sim;
  const int64_t n = (int64_t)width * height;
  const int tok = prof_begin(m, SLIM_KERNEL_RENDER, st);
  k_bounds_init<<<1, 32, 0, st>>>(m->render_bounds);
  k_block_bounds<<<152 * 2, 256, 0, st>>>(m->mv.blk_key, m->mv.ctr, m->mv.block_cap,
                                         m->render_bounds);
  k_render<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a);
  prof_end(m, tok, st);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(SLIM_ERR_CUDA, cudaGetErrorString(e));
  return SLIM_OK;
}

}  // namespace slim
