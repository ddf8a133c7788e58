// Open-set scan integration (Sec. III-D): per voxel and per embedding element
// the Normal-Inverse-Gamma update of Theorem 2 with lambda = W and nu = W / 2
// (the implementation simplification of Sec. III-D), applied once per scan
// to the scan's set of n observations of the voxel, in the form the theorem
// states (Eqs. norm_update_1 and norm_update_4):
//   zbar = batch mean,  M2 = sum (z - zbar)^2,  W' = W + n,
//   m'    = (W m + n zbar) / W'            = m + (zbar - m) n / W'
//   beta' = beta + M2 / 2 + (W n / W') (zbar - m)^2 / 2.
// zbar and M2 of a run of observations are accumulated about its first
// observation s (S1 = sum (z - s), S2 = sum (z - s)^2, zbar = s + S1 / n,
// M2 = S2 - S1^2 / n), which keeps the sums small and free of cancellation;
// runs longer than one piece are merged from per-piece statistics.
//
// Pipeline per scan (besides the shared block-allocation pass):
//   k_open_pairs  band DDA per point; the point's distinct blocks are looked
//                 up warp-cooperatively; every (voxel, point) pair is written
//                 as key = slot << 9 | local, with its d and point index.
//   radix sort    device-wide, by voxel key (count of pairs read on device).
//   k_open_frag   one warp per piece of 64 sorted pairs: whole runs are
//                 applied at once (the warp owns the voxel: state read once,
//                 updated in FP32 registers, written once, f32 or bf16
//                 storage, no atomics on records); runs cut by a piece
//                 boundary leave per-piece statistics.
//   k_open_merge  one warp per cut run: merge its pieces and apply.
#include <cuda_bf16.h>

#include "block_sort.cuh"
#include "geometry.cuh"
#include "hash.cuh"
#include "map.h"

namespace slim {

constexpr int kOpenBandBlocks = 8;
// device counters of the open-set scratch
enum { kOpPairs = 0, kOpCounters = 4 };

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
  const bool valid = j < n && ray_setup_at(g, pts, j, ry);
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

// ---------------------------------------------------------------- apply
// Sorted pairs are cut into pieces of kPiece consecutive pairs, one warp per
// piece. A piece holds fragments (maximal runs of one voxel key). A fragment
// that is a whole run is applied at once by its warp (exclusive owner of the
// voxel for this scan). A fragment cut by a piece boundary leaves its
// statistics (n, sum d, per element mean and M2) in a side slot of its
// piece: side 0 for the fragment that began in an earlier piece, side 1 for
// the fragment that goes on into the next one. k_open_merge then takes, for
// every run that starts in a piece p and leaves it, the side-1 slot of p and
// the side-0 slots of the following pieces up to the run's end, merges them
// with the pairwise update of Chan, Golub and LeVeque (count, mean, M2;
// compensated sums) and applies the run. No warp walks more than kPiece
// observations, however many pixels a voxel collects in one frame.
constexpr int kPiece = 64;
enum { kFragValid = 1, kFragHead = 2, kFragEnd = 4 };

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, off);
  return x;
}

// Point index of piece position k (lane k & 31 of pt0 / pt1).
__device__ __forceinline__ uint32_t piece_pt(uint32_t pt0, uint32_t pt1, int k) {
  return __shfl_sync(0xFFFFFFFFu, k < 32 ? pt0 : pt1, k & 31);
}

__device__ __forceinline__ float4 sem4(const float* __restrict__ sem, uint32_t pt, int L, int e,
                                       bool on) {
  return on ? *reinterpret_cast<const float4*>(sem + (size_t)pt * L + e)
            : make_float4(0.f, 0.f, 0.f, 0.f);
}

// Batch mean and M2 of one fragment [fb, fe) for G groups of 4 elements
// (e[g] = the lane's first element of group g), accumulated about the
// fragment's first observation s (S1 = sum (z - s), S2 = sum (z - s)^2,
// mean = s + S1 / n, M2 = S2 - S1^2 / n): one walk over the observations,
// G independent 16-byte loads per observation, two observations per step.
template <int G>
__device__ __forceinline__ void frag_stats_g(const float* __restrict__ sem, int L, uint32_t pt0,
                                             uint32_t pt1, int fb, int fe, const int (&e)[G],
                                             const bool (&on)[G], float (&mean)[G][4],
                                             float (&m2)[G][4]) {
  float sh[G][4], s1[G][4], s2[G][4];
  {
    const uint32_t pf = piece_pt(pt0, pt1, fb);
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const float4 v = sem4(sem, pf, L, e[g], on[g]);
      sh[g][0] = v.x; sh[g][1] = v.y; sh[g][2] = v.z; sh[g][3] = v.w;
#pragma unroll
      for (int q = 0; q < 4; ++q) s1[g][q] = s2[g][q] = 0.f;
    }
  }
  int k = fb + 1;
  for (; k + 1 < fe; k += 2) {
    const uint32_t pa = piece_pt(pt0, pt1, k), pb = piece_pt(pt0, pt1, k + 1);
    float4 za[G], zb[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      za[g] = sem4(sem, pa, L, e[g], on[g]);
      zb[g] = sem4(sem, pb, L, e[g], on[g]);
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const float va[4] = {za[g].x, za[g].y, za[g].z, za[g].w};
      const float vb[4] = {zb[g].x, zb[g].y, zb[g].z, zb[g].w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float ya = __fsub_rn(va[q], sh[g][q]);
        const float yb = __fsub_rn(vb[q], sh[g][q]);
        s1[g][q] = __fadd_rn(s1[g][q], __fadd_rn(ya, yb));
        s2[g][q] = __fadd_rn(s2[g][q], __fadd_rn(__fmul_rn(ya, ya), __fmul_rn(yb, yb)));
      }
    }
  }
  if (k < fe) {
    const uint32_t pa = piece_pt(pt0, pt1, k);
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const float4 z = sem4(sem, pa, L, e[g], on[g]);
      const float va[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float ya = __fsub_rn(va[q], sh[g][q]);
        s1[g][q] = __fadd_rn(s1[g][q], ya);
        s2[g][q] = __fadd_rn(s2[g][q], __fmul_rn(ya, ya));
      }
    }
  }
  const float invn = __fdiv_rn(1.0f, (float)(fe - fb));
#pragma unroll
  for (int g = 0; g < G; ++g)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      mean[g][q] = __fadd_rn(sh[g][q], __fmul_rn(s1[g][q], invn));
      m2[g][q] = fmaxf(__fsub_rn(s2[g][q], __fmul_rn(__fmul_rn(s1[g][q], s1[g][q]), invn)), 0.f);
    }
}

// Voxel row of key (slot << 9 | local), allocated on its first observation
// by lane 0 (the calling warp owns the voxel for this scan); -1 on a
// capacity fault.
__device__ __forceinline__ int32_t voxel_row(const MapView& mv, uint32_t key, int* fresh) {
  int32_t row = 0;
  int fr = 0;
  if (lane_id() == 0) {
    int32_t* vr = mv.vox_row + (size_t)(key >> 9) * kBlockVoxels + (key & 511u);
    row = *vr;
    if (row < 0) {
      const uint32_t r = atomicAdd(&mv.ctr[kCtrRows], 1u);
      if (r >= mv.row_cap) {
        raise_status(mv.ctr, kDevCapacity, 12);
        row = -1;
      } else {
        row = (int32_t)r;
        *vr = row;
        fr = 1;
      }
    }
  }
  *fresh = __shfl_sync(0xFFFFFFFFu, fr, 0);
  return __shfl_sync(0xFFFFFFFFu, row, 0);
}

// Theorem 2 update of elements [e, e + 4) of a row with the batch
// statistics: m' = m + (zbar - m) n / W', beta' = beta + M2 / 2 +
// (W n / W') (zbar - m)^2 / 2 (fm = n / W', fb = W n / W'). Returns the
// partial |m'|^2 of the stored values.
template <int BF16>
__device__ __forceinline__ float nig_apply4(const MapView& mv, size_t rbase, int e, int fresh,
                                            float fm, float fb, const float mean[4],
                                            const float m2[4]) {
  float4 m = fresh ? make_float4(0.f, 0.f, 0.f, 0.f) : load4<BF16>(mv.mrow, rbase + e);
  float4 b = fresh ? make_float4(0.f, 0.f, 0.f, 0.f) : load4<BF16>(mv.brow, rbase + e);
  float mv4[4] = {m.x, m.y, m.z, m.w}, bv4[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float d = mean[q] - mv4[q];
    bv4[q] += 0.5f * (m2[q] + fb * d * d);
    mv4[q] += d * fm;
  }
  m = make_float4(mv4[0], mv4[1], mv4[2], mv4[3]);
  b = make_float4(bv4[0], bv4[1], bv4[2], bv4[3]);
  store4<BF16>(mv.mrow, rbase + e, m);
  store4<BF16>(mv.brow, rbase + e, b);
  if (BF16) m = load4<BF16>(mv.mrow, rbase + e);  // norm of the stored values
  return m.x * m.x + m.y * m.y + m.z * m.z + m.w * m.w;
}

template <int BF16>
__global__ void __launch_bounds__(256) k_open_frag(MapView mv, const uint32_t* __restrict__ keys,
                                                   const uint32_t* __restrict__ vals,
                                                   const float* __restrict__ pair_d,
                                                   const uint32_t* __restrict__ pair_pt,
                                                   const uint32_t* __restrict__ ctr,
                                                   const float* __restrict__ sem, int L,
                                                   int64_t n_max, float2* part, uint4* meta) {
  if (*(volatile uint32_t*)&mv.ctr[kCtrStatus]) return;
  const unsigned lane = lane_id();
  const int64_t n = min(n_max, (int64_t)ctr[kOpPairs]);
  const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t base = p * kPiece;
  if (base >= n) return;
  const int m = (int)(n - base < kPiece ? n - base : (int64_t)kPiece);
  constexpr uint32_t kInv = 0xFFFFFFFFu;
  const int64_t i0 = base + lane, i1 = base + 32 + lane;
  const uint32_t key0 = (int)lane < m ? keys[i0] : kInv;
  const uint32_t key1 = 32 + (int)lane < m ? keys[i1] : kInv;
  uint32_t pt0 = 0, pt1 = 0;
  float d0 = 0.f, d1 = 0.f;
  if (key0 != kInv) {
    const uint32_t v = vals[i0];
    pt0 = pair_pt[v];
    d0 = pair_d[v];
  }
  if (key1 != kInv) {
    const uint32_t v = vals[i1];
    pt1 = pair_pt[v];
    d1 = pair_d[v];
  }
  const uint32_t prev_key = base > 0 ? keys[base - 1] : kInv;
  const uint32_t next_key = base + kPiece < n ? keys[base + kPiece] : kInv;
  // fragment starts as a 64-bit mask over the piece positions
  const uint32_t up0 = __shfl_up_sync(0xFFFFFFFFu, key0, 1);
  const uint32_t up1 = __shfl_up_sync(0xFFFFFFFFu, key1, 1);
  const uint32_t last0 = __shfl_sync(0xFFFFFFFFu, key0, 31);
  const bool st0 = lane == 0 || key0 != up0;
  const bool st1 = lane == 0 ? key1 != last0 : key1 != up1;
  const uint64_t smask = (uint64_t)__ballot_sync(0xFFFFFFFFu, st0) |
                         ((uint64_t)__ballot_sync(0xFFFFFFFFu, st1) << 32);
  if (lane == 0) meta[2 * p + 1] = make_uint4(0u, 0u, 0u, 0u);
  int fb = 0;
  while (fb < m) {
    const uint64_t rest = fb < 63 ? (smask >> (fb + 1)) << (fb + 1) : 0ull;
    const int fe = rest ? min(m, __ffsll((long long)rest) - 1) : m;
    const uint32_t key = __shfl_sync(0xFFFFFFFFu, fb < 32 ? key0 : key1, fb & 31);
    if (key == kInv) break;  // pairs without a block sort last
    const bool before = fb == 0 && prev_key == key;
    const bool after = fe == kPiece && next_key == key;
    float sd = 0.f;
    if ((int)lane >= fb && (int)lane < fe) sd += d0;
    if (32 + (int)lane >= fb && 32 + (int)lane < fe) sd += d1;
    sd = warp_sum(sd);
    const int nf = fe - fb;
    if (!before && !after) {  // a whole run: apply now
      int fresh = 0;
      const int32_t row = voxel_row(mv, key, &fresh);
      if (row >= 0) {
        const float2 sw = fresh ? make_float2(0.f, 0.f) : mv.tsdf[row];
        const float Wn = sw.y + (float)nf;
        const float fm = (float)nf / Wn, fbw = sw.y * (float)nf / Wn;
        const size_t rbase = (size_t)row * L;
        float nrm = 0.f;
        for (int c0 = 0; c0 < L; c0 += 512) {
          int e[4];
          bool on[4];
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            e[g] = c0 + 128 * g + 4 * (int)lane;
            on[g] = e[g] < L;
          }
          float mean[4][4], m2[4][4];
          frag_stats_g<4>(sem, L, pt0, pt1, fb, fe, e, on, mean, m2);
#pragma unroll
          for (int g = 0; g < 4; ++g)
            if (on[g]) nrm += nig_apply4<BF16>(mv, rbase, e[g], fresh, fm, fbw, mean[g], m2[g]);
        }
        nrm = warp_sum(nrm);
        if (lane == 0) {
          mv.tsdf[row] = make_float2(sw.x + sd, Wn);
          mv.mnorm2[row] = nrm;
        }
      }
    } else {  // cut by a piece boundary: leave the statistics for the merge
      const int side = before ? 0 : 1;
      const uint32_t flags = kFragValid | (before ? 0u : (uint32_t)kFragHead) |
                             (after ? 0u : (uint32_t)kFragEnd);
      float2* dst = part + (size_t)(2 * p + side) * L;
      for (int c0 = 0; c0 < L; c0 += 512) {
        int e[4];
        bool on[4];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          e[g] = c0 + 128 * g + 4 * (int)lane;
          on[g] = e[g] < L;
        }
        float mean[4][4], m2[4][4];
        frag_stats_g<4>(sem, L, pt0, pt1, fb, fe, e, on, mean, m2);
#pragma unroll
        for (int g = 0; g < 4; ++g)
          if (on[g]) {
            float4* d4 = reinterpret_cast<float4*>(dst + e[g]);
            d4[0] = make_float4(mean[g][0], m2[g][0], mean[g][1], m2[g][1]);
            d4[1] = make_float4(mean[g][2], m2[g][2], mean[g][3], m2[g][3]);
          }
      }
      if (lane == 0) meta[2 * p + side] = make_uint4((uint32_t)nf, __float_as_uint(sd), flags, key);
    }
    fb = fe;
  }
}

// One warp per run that leaves the piece it starts in: merge its fragments
// (side 1 of the head piece, side 0 of the following pieces up to the
// fragment flagged as the run's end) and apply the run. A voxel close to
// the sensor can collect thousands of observations in one frame, so a run
// can span tens of pieces: the run's end is searched 32 pieces per step
// (one piece metadata word per lane) and the fragments' statistics are
// loaded kMergeAhead pieces at a time, so the warp's chain of dependent
// loads grows with the run length / kMergeAhead, not with the run length.
constexpr int kMergeAhead = 6;

template <int BF16>
__global__ void __launch_bounds__(256, 2) k_open_merge(MapView mv, const uint32_t* __restrict__ ctr,
                                                    int L, int64_t n_max,
                                                    const float2* __restrict__ part,
                                                    const uint4* __restrict__ meta) {
  if (*(volatile uint32_t*)&mv.ctr[kCtrStatus]) return;
  const unsigned lane = lane_id();
  const int64_t n = min(n_max, (int64_t)ctr[kOpPairs]);
  const int64_t np = (n + kPiece - 1) / kPiece;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < np; p += warps) {
    const uint4 h = meta[2 * p + 1];
    if (!(h.z & kFragHead)) continue;
    const uint32_t key = h.w;
    // the chain of pieces after p: count, sum d and the end piece
    float ntot = 0.f, sd = 0.f;
    int64_t q_end = -1;
    for (int64_t b0 = p + 1; b0 < np; b0 += 32) {
      const int64_t q = b0 + (int64_t)lane;
      const uint4 t = q < np ? meta[2 * q] : make_uint4(0u, 0u, 0u, 0u);
      const bool same = (t.z & kFragValid) && t.w == key;
      const unsigned brk = __ballot_sync(0xFFFFFFFFu, !same);
      const unsigned end = __ballot_sync(0xFFFFFFFFu, same && (t.z & kFragEnd));
      const int nb = brk ? __ffs(brk) - 1 : 32;  // first lane outside the chain
      const int ne = end ? __ffs(end) - 1 : 32;  // first lane holding the end
      const int take = ne < nb ? ne + 1 : nb;
      ntot += warp_sum((int)lane < take ? (float)t.x : 0.f);
      sd += warp_sum((int)lane < take ? __uint_as_float(t.y) : 0.f);
      if (ne < nb) {
        q_end = b0 + ne;
        break;
      }
      if (nb < 32) break;
    }
    if (q_end < 0) {  // consistency check, never expected
      if (lane == 0) raise_status(mv.ctr, kDevInternal, 13);
      continue;
    }
    ntot += (float)h.x;
    sd += __uint_as_float(h.y);
    int fresh = 0;
    const int32_t row = voxel_row(mv, key, &fresh);
    if (row < 0) continue;
    const float2 sw = fresh ? make_float2(0.f, 0.f) : mv.tsdf[row];
    const float Wn = sw.y + ntot;
    const float fm = ntot / Wn, fbw = sw.y * ntot / Wn;
    const size_t rbase = (size_t)row * L;
    float nrm = 0.f;
    for (int c0 = 0; c0 < L; c0 += 128) {
      const int e = c0 + 4 * (int)lane;
      if (e >= L) continue;
      float na = (float)h.x;
      float mean[4], m2[4], mc[4] = {0.f, 0.f, 0.f, 0.f}, vc[4] = {0.f, 0.f, 0.f, 0.f};
      {
        const float4* s4 = reinterpret_cast<const float4*>(part + (size_t)(2 * p + 1) * L + e);
        const float4 a = s4[0], b = s4[1];
        mean[0] = a.x; m2[0] = a.y; mean[1] = a.z; m2[1] = a.w;
        mean[2] = b.x; m2[2] = b.y; mean[3] = b.z; m2[3] = b.w;
      }
      for (int64_t r0 = p + 1; r0 <= q_end; r0 += kMergeAhead) {
        float nbv[kMergeAhead];
        float4 av[kMergeAhead], bv[kMergeAhead];
#pragma unroll
        for (int u = 0; u < kMergeAhead; ++u) {
          const int64_t r = r0 + u;
          if (r <= q_end) {
            nbv[u] = (float)meta[2 * r].x;
            const float4* s4 = reinterpret_cast<const float4*>(part + (size_t)(2 * r) * L + e);
            av[u] = s4[0];
            bv[u] = s4[1];
          }
        }
#pragma unroll
        for (int u = 0; u < kMergeAhead; ++u) {
          if (r0 + u > q_end) break;
          const float nb = nbv[u];
          const float mb[4] = {av[u].x, av[u].z, bv[u].x, bv[u].z};
          const float vb[4] = {av[u].y, av[u].w, bv[u].y, bv[u].w};
          const float nn = na + nb;
          const float wb = nb / nn, wab = na * nb / nn;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float dl = mb[k] - mean[k];
            // mean += dl * nb / n and M2 += M2_b + dl^2 na nb / n, compensated
            const float ym = __fsub_rn(__fmul_rn(dl, wb), mc[k]);
            const float tm = __fadd_rn(mean[k], ym);
            mc[k] = __fsub_rn(__fsub_rn(tm, mean[k]), ym);
            mean[k] = tm;
            const float yv = __fsub_rn(__fadd_rn(vb[k], __fmul_rn(__fmul_rn(dl, dl), wab)), vc[k]);
            const float tv = __fadd_rn(m2[k], yv);
            vc[k] = __fsub_rn(__fsub_rn(tv, m2[k]), yv);
            m2[k] = tv;
          }
          na = nn;
        }
      }
      nrm += nig_apply4<BF16>(mv, rbase, e, fresh, fm, fbw, mean, m2);
    }
    nrm = warp_sum(nrm);
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
  const int64_t pieces = (cap + kPiece - 1) / kPiece;
  if ((s = m->alloc(&o.part, (size_t)pieces * 2 * (size_t)m->L)) != SLIM_OK) return s;
  if ((s = m->alloc(&o.meta, (size_t)pieces * 2)) != SLIM_OK) return s;
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
  // keys of pairs without a block (0xFFFFFFFF) must sort after every valid
  // key within the sorted bits: valid keys stay below (block_cap + 1) << 9
  const int bits = 9 + ceil_log2((uint64_t)mv.block_cap + 1);
  uint32_t* skeys = nullptr;  // the sorted pairs: (keys, vals) or the ping-pong pair
  uint32_t* svals = nullptr;
  e = radix_sort_u32_devn(o.keys, o.vals, o.keys_tmp, o.vals_tmp, o.tmp, n_max, o.ctr + kOpPairs,
                          bits, st, &skeys, &svals);
  if (e != cudaSuccess) return fail(SLIM_ERR_CUDA, cudaGetErrorString(e));
  prof_end(m, tok, st);
  tok = prof_begin(m, SLIM_KERNEL_OPEN_APPLY, st);
  const int64_t pieces = (n_max + kPiece - 1) / kPiece;
  const unsigned fgrid = (unsigned)((pieces + 7) / 8);
  const unsigned mgrid = 152 * 8;
  if (bf16) {
    k_open_frag<1><<<fgrid, 256, 0, st>>>(mv, skeys, svals, o.pair_d, o.pair_pt, o.ctr, sem, L,
                                          n_max, o.part, o.meta);
    k_open_merge<1><<<mgrid, 256, 0, st>>>(mv, o.ctr, L, n_max, o.part, o.meta);
  } else {
    k_open_frag<0><<<fgrid, 256, 0, st>>>(mv, skeys, svals, o.pair_d, o.pair_pt, o.ctr, sem, L,
                                          n_max, o.part, o.meta);
    k_open_merge<0><<<mgrid, 256, 0, st>>>(mv, o.ctr, L, n_max, o.part, o.meta);
  }
  prof_end(m, tok, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(SLIM_ERR_CUDA, cudaGetErrorString(e));
  return SLIM_OK;
}

}  // namespace slim
