// Open-set scan integration (Sec. III-D): per voxel and per embedding element
// the Normal-Inverse-Gamma update of Theorem 2 with lambda = W and nu = W / 2
// (the implementation simplification of Sec. III-D), applied once per scan
// to the scan's set of n observations of the voxel, in the form the theorem
// states (Eqs. norm_update_1 and norm_update_4):
//   zbar = batch mean,  M2 = sum (z - zbar)^2,  W' = W + n,
//   m'    = (W m + n zbar) / W'            = m + (zbar - m) n / W'
//   beta' = beta + M2 / 2 + (W n / W') (zbar - m)^2 / 2.
// zbar and M2 are accumulated about the batch's first observation s
// (S1 = sum (z - s), S2 = sum (z - s)^2, zbar = s + S1 / n,
// M2 = S2 - S1^2 / n), which keeps the sums small and free of cancellation.
//
// Pipeline per scan (besides the shared block-allocation pass):
//   k_open_pairs  band DDA per point; the point's distinct blocks are looked
//                 up warp-cooperatively; every (voxel, point) pair is written
//                 as key = slot << 9 | local, with its d and point index.
//   radix sort    device-wide, by voxel key (count of pairs read on device).
//   k_open_heads  segment starts (first pair of each voxel run).
//   k_open_apply  one warp per voxel run: exclusive owner of the voxel, so
//                 the state is read once, updated in FP32 registers and
//                 written once (f32 or bf16 storage), no atomics on records.
#include <cuda_bf16.h>

#include "block_sort.cuh"
#include "geometry.cuh"
#include "hash.cuh"
#include "map.h"

namespace slim {

constexpr int kOpenBandBlocks = 8;
// device counters of the open-set scratch
enum { kOpPairs = 0, kOpSegs = 1, kOpCounters = 4 };

__global__ void __launch_bounds__(256) k_open_pairs(MapView mv, ScanGeom g,
                                                    const float* __restrict__ pts, int64_t n,
                                                    uint32_t* keys, uint32_t* vals, float* pair_d,
                                                    uint32_t* pair_pt, uint32_t* ctr,
                                                    uint32_t pair_cap) {
  __shared__ uint64_t kbuf[256][kOpenBandBlocks];
  __shared__ uint32_t sbuf[256][kOpenBandBlocks];
  __shared__ uint32_t s_status;
  if (threadIdx.x == 0) s_status = *(volatile uint32_t*)&mv.ctr[kCtrStatus];
  __syncthreads();
  if (s_status) return;
  const unsigned lane = lane_id();
  const int64_t j = (int64_t)blockIdx.x * 256 + threadIdx.x;
  int cnt = 0, np = 0;
  Ray ry;
  const bool valid = j < n && ray_setup(g, pts[3 * j], pts[3 * j + 1], pts[3 * j + 2], ry);
  if (valid) {
    Ray r2 = ry;
    uint64_t last = kEmptyKey;
    ray_for_each(g, r2, [&](int32_t i0, int32_t i1, int32_t i2, float) {
      const uint64_t kb = pack_block(i0 >> 3, i1 >> 3, i2 >> 3);
      if (kb != last) {
        if (cnt < kOpenBandBlocks) kbuf[threadIdx.x][cnt] = kb;
        ++cnt;
        last = kb;
      }
      ++np;
    });
  }
  if (cnt > kOpenBandBlocks) {
    raise_status(mv.ctr, kDevInternal, 10);
    cnt = kOpenBandBlocks;
    np = 0;
  }
  // lookups of the distinct blocks: duplicates dropped per warp, leaders
  // probe in parallel and share the slot with their peers
  const int maxc = __reduce_max_sync(0xFFFFFFFFu, cnt);
  for (int r = 0; r < maxc; ++r) {
    const bool has = r < cnt;
    const uint64_t key = has ? kbuf[threadIdx.x][r] : kEmptyKey;
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, (unsigned long long)key);
    const int ldr = __ffs(peers) - 1;
    uint32_t slot = kNoSlot;
    if (has && (int)lane == ldr) slot = hash_find(mv, key);
    slot = __shfl_sync(0xFFFFFFFFu, slot, ldr);
    if (has) sbuf[threadIdx.x][r] = slot;
  }
  // positions: one atomic per warp
  uint32_t x = (uint32_t)np;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
    if ((int)lane >= off) x += y;
  }
  uint32_t base = 0;
  if (lane == 31) base = atomicAdd(&ctr[kOpPairs], x);
  base = __shfl_sync(0xFFFFFFFFu, base, 31) + x - (uint32_t)np;
  if (valid && np > 0) {
    if (base + (uint32_t)np > pair_cap) {
      raise_status(mv.ctr, kDevCapacity, 11);
      return;
    }
    uint64_t last = kEmptyKey;
    int r = -1;
    uint32_t k = 0;
    ray_for_each(g, ry, [&](int32_t i0, int32_t i1, int32_t i2, float d) {
      const uint64_t kb = pack_block(i0 >> 3, i1 >> 3, i2 >> 3);
      if (kb != last) {
        last = kb;
        ++r;
      }
      const uint32_t slot = sbuf[threadIdx.x][r];
      const uint32_t pos = base + k++;
      keys[pos] = slot == kNoSlot ? 0xFFFFFFFFu : ((slot << 9) | (uint32_t)local_index(i0, i1, i2));
      vals[pos] = pos;
      pair_d[pos] = d;
      pair_pt[pos] = (uint32_t)j;
    });
  }
}

// First pair of every run of equal keys -> seg_start (order irrelevant).
__global__ void __launch_bounds__(256) k_open_heads(const uint32_t* __restrict__ keys,
                                                    uint32_t* ctr, uint32_t* seg_start,
                                                    int64_t n_max) {
  const int64_t n = min(n_max, (int64_t)ctr[kOpPairs]);
  const unsigned lane = lane_id();
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = b + threadIdx.x;
    bool head = false;
    if (i < n) {
      const uint32_t k = keys[i];
      head = k != 0xFFFFFFFFu && (i == 0 || keys[i - 1] != k);
    }
    const unsigned hm = __ballot_sync(0xFFFFFFFFu, head);
    uint32_t base = 0;
    if (lane == 0 && hm) base = atomicAdd(&ctr[kOpSegs], (uint32_t)__popc(hm));
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if (head) seg_start[base + __popc(hm & ((1u << lane) - 1u))] = (uint32_t)i;
  }
}

// s += y with the rounding error carried in c (Kahan); explicit _rn ops
// keep the compiler from contracting or reassociating them.
__device__ __forceinline__ void kahan_add(float& s, float& c, float y) {
  const float yc = __fsub_rn(y, c);
  const float t = __fadd_rn(s, yc);
  c = __fsub_rn(__fsub_rn(t, s), yc);
  s = t;
}

template <int BF16>
__device__ __forceinline__ float4 load4(const void* base, size_t idx) {
  if (BF16) {
    const uint2 u = *reinterpret_cast<const uint2*>(static_cast<const __nv_bfloat16*>(base) + idx);
    const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162*>(&u.x);
    const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&u.y);
    const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
  }
  return *reinterpret_cast<const float4*>(static_cast<const float*>(base) + idx);
}

template <int BF16>
__device__ __forceinline__ void store4(void* base, size_t idx, float4 v) {
  if (BF16) {
    const __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y);
    const __nv_bfloat162 b = __floats2bfloat162_rn(v.z, v.w);
    uint2 u;
    u.x = *reinterpret_cast<const uint32_t*>(&a);
    u.y = *reinterpret_cast<const uint32_t*>(&b);
    *reinterpret_cast<uint2*>(static_cast<__nv_bfloat16*>(base) + idx) = u;
  } else {
    *reinterpret_cast<float4*>(static_cast<float*>(base) + idx) = v;
  }
}

// One warp per voxel run. Lane q holds elements [4q, 4q + 4) of each
// 128-element chunk of the embedding.
template <int BF16>
__global__ void __launch_bounds__(256) k_open_apply(MapView mv, const uint32_t* __restrict__ keys,
                                                    const uint32_t* __restrict__ vals,
                                                    const float* __restrict__ pair_d,
                                                    const uint32_t* __restrict__ pair_pt,
                                                    const uint32_t* __restrict__ seg_start,
                                                    const uint32_t* __restrict__ ctr,
                                                    const float* __restrict__ sem, int L,
                                                    int64_t n_max) {
  if (*(volatile uint32_t*)&mv.ctr[kCtrStatus]) return;
  const unsigned lane = lane_id();
  const int64_t n = min(n_max, (int64_t)ctr[kOpPairs]);
  const uint32_t nseg = ctr[kOpSegs];
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < nseg; s += warps) {
    const int64_t start = seg_start[s];
    const uint32_t key = keys[start];
    // run end: first differing key
    int64_t end = n;
    for (int64_t b = start + 1; b < n; b += 32) {
      const int64_t i = b + lane;
      const bool diff = i < n && keys[i] != key;
      const unsigned dm = __ballot_sync(0xFFFFFFFFu, diff);
      if (dm) {
        end = b + __ffs(dm) - 1;
        break;
      }
      if (b + 32 >= n) break;
    }
    const uint32_t slot = key >> 9, local = key & 511u;
    int32_t row = 0;
    int fresh = 0;
    if (lane == 0) {
      int32_t* vr = mv.vox_row + (size_t)slot * kBlockVoxels + local;
      row = *vr;
      if (row < 0) {
        const uint32_t r = atomicAdd(&mv.ctr[kCtrRows], 1u);
        if (r >= mv.row_cap) {
          raise_status(mv.ctr, kDevCapacity, 12);
          row = -1;
        } else {
          row = (int32_t)r;
          *vr = row;
          fresh = 1;
        }
      }
    }
    row = __shfl_sync(0xFFFFFFFFu, row, 0);
    fresh = __shfl_sync(0xFFFFFFFFu, fresh, 0);
    if (row < 0) continue;
    const float cnt = (float)(end - start);
    // sum of d over the run
    float sd = 0.f;
    for (int64_t i = start + lane; i < end; i += 32) sd += pair_d[vals[i]];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) sd += __shfl_xor_sync(0xFFFFFFFFu, sd, off);
    const float2 sw = fresh ? make_float2(0.f, 0.f) : mv.tsdf[row];
    const float Wn = sw.y + cnt;
    const float invn = 1.0f / cnt;
    const float fm = cnt / Wn;              // n / W'
    const float fb = sw.y * cnt / Wn;       // W n / W'
    const size_t rbase = (size_t)row * L;
    const float* zfirst = sem + (size_t)pair_pt[vals[start]] * L;
    float nrm = 0.f;
    for (int c0 = 0; c0 < L; c0 += 128) {
      const int e = c0 + 4 * (int)lane;
      if (e >= L) continue;
      const float4 sh = *reinterpret_cast<const float4*>(zfirst + e);
      // compensated (Kahan) sums: a voxel may collect thousands of
      // observations in one depth frame
      float s1a[4] = {0.f, 0.f, 0.f, 0.f}, s1c[4] = {0.f, 0.f, 0.f, 0.f};
      float s2a[4] = {0.f, 0.f, 0.f, 0.f}, s2c[4] = {0.f, 0.f, 0.f, 0.f};
      const float shv[4] = {sh.x, sh.y, sh.z, sh.w};
      for (int64_t i = start; i < end; ++i) {
        const uint32_t pt = pair_pt[vals[i]];
        const float4 z = *reinterpret_cast<const float4*>(sem + (size_t)pt * L + e);
        const float zv[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float y = __fsub_rn(zv[q], shv[q]);
          kahan_add(s1a[q], s1c[q], y);
          kahan_add(s2a[q], s2c[q], __fmul_rn(y, y));
        }
      }
      const float4 s1 = make_float4(s1a[0], s1a[1], s1a[2], s1a[3]);
      const float4 s2 = make_float4(s2a[0], s2a[1], s2a[2], s2a[3]);
      float4 m = fresh ? make_float4(0.f, 0.f, 0.f, 0.f) : load4<BF16>(mv.mrow, rbase + e);
      float4 b = fresh ? make_float4(0.f, 0.f, 0.f, 0.f) : load4<BF16>(mv.brow, rbase + e);
      const float zb0 = sh.x + s1.x * invn, zb1 = sh.y + s1.y * invn;
      const float zb2 = sh.z + s1.z * invn, zb3 = sh.w + s1.w * invn;
      const float d0 = zb0 - m.x, d1 = zb1 - m.y, d2 = zb2 - m.z, d3 = zb3 - m.w;
      b.x += 0.5f * ((s2.x - s1.x * s1.x * invn) + fb * d0 * d0);
      b.y += 0.5f * ((s2.y - s1.y * s1.y * invn) + fb * d1 * d1);
      b.z += 0.5f * ((s2.z - s1.z * s1.z * invn) + fb * d2 * d2);
      b.w += 0.5f * ((s2.w - s1.w * s1.w * invn) + fb * d3 * d3);
      m.x += d0 * fm; m.y += d1 * fm; m.z += d2 * fm; m.w += d3 * fm;
      store4<BF16>(mv.mrow, rbase + e, m);
      store4<BF16>(mv.brow, rbase + e, b);
      if (BF16) m = load4<BF16>(mv.mrow, rbase + e);  // norm of the stored values
      nrm += m.x * m.x + m.y * m.y + m.z * m.z + m.w * m.w;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) nrm += __shfl_xor_sync(0xFFFFFFFFu, nrm, off);
    if (lane == 0) {
      mv.tsdf[row] = make_float2(sw.x + sd, Wn);
      mv.mnorm2[row] = nrm;
    }
  }
}

slim_status open_alloc_scratch(slim_map* m, OpenScratch& o, int64_t max_points) {
  const int64_t cap = std::max<int64_t>(1, max_points) * m->cap;
  if (cap > (int64_t)0xFFFFFFF0ll) return fail(SLIM_ERR_ARG, "max_points * band cap too large");
  o.pair_cap = cap;
  slim_status s;
  if ((s = m->alloc(&o.keys, (size_t)cap)) != SLIM_OK) return s;
  if ((s = m->alloc(&o.vals, (size_t)cap)) != SLIM_OK) return s;
  if ((s = m->alloc(&o.keys_tmp, (size_t)cap)) != SLIM_OK) return s;
  if ((s = m->alloc(&o.vals_tmp, (size_t)cap)) != SLIM_OK) return s;
  if ((s = m->alloc(&o.pair_d, (size_t)cap)) != SLIM_OK) return s;
  if ((s = m->alloc(&o.pair_pt, (size_t)cap)) != SLIM_OK) return s;
  if ((s = m->alloc(&o.seg_start, (size_t)cap)) != SLIM_OK) return s;
  if ((s = m->alloc(&o.ctr, (size_t)kOpCounters)) != SLIM_OK) return s;
  unsigned char* tmp = nullptr;
  if ((s = m->alloc(&tmp, radix_sort_temp_bytes(cap))) != SLIM_OK) return s;
  o.tmp = tmp;
  return SLIM_OK;
}

cudaError_t open_setup_attributes(slim_map*) { return cudaSuccess; }

static int ceil_log2(uint64_t x) {
  int b = 0;
  while ((1ull << b) < x) ++b;
  return b;
}

slim_status open_integrate(slim_map* m, const MapView& mv, OpenScratch& o, const ScanGeom& g,
                           const float* pts, const float* sem, int64_t n, int L, int bf16,
                           cudaStream_t st) {
  if (n <= 0) return SLIM_OK;
  cudaError_t e = cudaMemsetAsync(o.ctr, 0, kOpCounters * sizeof(uint32_t), st);
  if (e != cudaSuccess) return fail(SLIM_ERR_CUDA, cudaGetErrorString(e));
  const unsigned grid = (unsigned)((n + 255) / 256);
  int tok = prof_begin(m, SLIM_KERNEL_OPEN_PAIRS, st);
  k_open_pairs<<<grid, 256, 0, st>>>(mv, g, pts, n, o.keys, o.vals, o.pair_d, o.pair_pt, o.ctr,
                                     (uint32_t)o.pair_cap);
  const int64_t n_max = std::min<int64_t>(o.pair_cap, n * (int64_t)g.cap);
  const int bits = 9 + ceil_log2((uint64_t)mv.block_cap);
  e = radix_sort_u32_devn(o.keys, o.vals, o.keys_tmp, o.vals_tmp, o.tmp, n_max, o.ctr + kOpPairs,
                          bits, st);
  if (e != cudaSuccess) return fail(SLIM_ERR_CUDA, cudaGetErrorString(e));
  const unsigned hgrid = (unsigned)std::min<int64_t>((n_max + 255) / 256, 152 * 16);
  k_open_heads<<<hgrid, 256, 0, st>>>(o.keys, o.ctr, o.seg_start, n_max);
  prof_end(m, tok, st);
  tok = prof_begin(m, SLIM_KERNEL_OPEN_APPLY, st);
  const unsigned agrid = 152 * 8;
  if (bf16)
    k_open_apply<1><<<agrid, 256, 0, st>>>(mv, o.keys, o.vals, o.pair_d, o.pair_pt, o.seg_start,
                                           o.ctr, sem, L, n_max);
  else
    k_open_apply<0><<<agrid, 256, 0, st>>>(mv, o.keys, o.vals, o.pair_d, o.pair_pt, o.seg_start,
                                           o.ctr, sem, L, n_max);
  prof_end(m, tok, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(SLIM_ERR_CUDA, cudaGetErrorString(e));
  return SLIM_OK;
}

}  // namespace slim
