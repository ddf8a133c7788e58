// Open-set scan integration (Sec. III-D): per voxel and per embedding element
// the Normal-Inverse-Gamma update of Theorem 2 with lambda = W and nu = W / 2
// (the implementation simplification of Sec. III-D), applied once per scan
// to the scan's set of n observations of the voxel. With every observation
// taken about a shift vector s of the voxel (S1 = sum (z - s),
// S2 = sum (z - s)^2, W' = W + n), Eqs. norm_update_1 and norm_update_4 read
//   s = m (a voxel seen before):  m' = m + S1 / W',
//                                 beta' = beta + (S2 - S1^2 / W') / 2;
//   s = z_1 (a new voxel, W = 0): m' = s + S1 / n,
//                                 beta' = (S2 - S1^2 / n) / 2,
// the second being the batch mean and half the sum of squared deviations.
// Both are sums over observations, so partial sums from any grouping of the
// observations add up to the same update (Theorem 2 is stated for sets).
//
// Pipeline per integration call (pairs never reach HBM):
//   k_open_tile   one CTA per tile of 16 x 16 pixels of an organized frame
//                 (or 256 consecutive points): band DDA per pixel; the tile's
//                 distinct voxels in a shared-memory table with a pixel mask,
//                 count and fixed-point sum of d per voxel; blocks and voxel
//                 rows looked up or created in the map (a new row gets its
//                 shift, the embedding of one of its pixels, before it is
//                 published); the embedding rows streamed in 64-element
//                 chunks by TMA into shared memory, each read once from HBM;
//                 per (voxel, chunk) one warp sums y = z - s and y^2 over the
//                 voxel's pixels (packed FP32x2 arithmetic) and adds them to
//                 the row's accumulator with one vector reduction per lane.
//   k_open_apply  one warp per row the call touched: the update above from
//                 the accumulator, the row's state read and written once,
//                 the accumulator cleared.
#include <cuda_bf16.h>

#include <algorithm>

#include "block_sort.cuh"
#include "geometry.cuh"
#include "hash.cuh"
#include "map.h"
#include "tma.cuh"

namespace slim {

constexpr int kOT = 256;          // pixels per tile
constexpr int kORowPts = 16;      // points per staged row of unorganized tiles
constexpr int kOE = 64;           // embedding elements per staged chunk
constexpr int kOMaxTV = 256;      // distinct voxels per tile part
constexpr int kOTbl = 1024;       // voxel table entries (power of two)
constexpr int kOThreads = 256;
constexpr int32_t kPendingRow = -2;  // vox_row: being created by another CTA
constexpr int32_t kFailRow = -3;     // vox_row: creation failed (capacity)

// --------------------------------------------------------------- helpers
__device__ __forceinline__ uint64_t pack_voxel(int32_t i0, int32_t i1, int32_t i2) {
  return ((uint64_t)(uint32_t)(i0 + (1 << 20)) << 42) |
         ((uint64_t)(uint32_t)(i1 + (1 << 20)) << 21) | (uint64_t)(uint32_t)(i2 + (1 << 20));
}

__device__ __forceinline__ void unpack_voxel(uint64_t k, int32_t& i0, int32_t& i1, int32_t& i2) {
  i0 = (int32_t)((k >> 42) & 0x1FFFFF) - (1 << 20);
  i1 = (int32_t)((k >> 21) & 0x1FFFFF) - (1 << 20);
  i2 = (int32_t)(k & 0x1FFFFF) - (1 << 20);
}

// Packed FP32x2 arithmetic (each half rounded to nearest, as two scalar ops).
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ float2 f2_unpack(uint64_t a) {
  return make_float2(__uint_as_float((uint32_t)a), __uint_as_float((uint32_t)(a >> 32)));
}
__device__ __forceinline__ uint64_t f2_pack(float x, float y) {
  return (uint64_t)__float_as_uint(x) | ((uint64_t)__float_as_uint(y) << 32);
}

__device__ __forceinline__ void red_add_v4_nc(float* r, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(r), "f"(a), "f"(b),
               "f"(c), "f"(d)
               : "memory");
}

// old = *r; *r += (a, b, c, d), returning old (16-byte aligned).
__device__ __forceinline__ float4 atom_add_v4(float* r, float a, float b, float c, float d) {
  float4 o;
  asm volatile("atom.global.add.v4.f32 {%0, %1, %2, %3}, [%4], {%5, %6, %7, %8};"
               : "=f"(o.x), "=f"(o.y), "=f"(o.z), "=f"(o.w)
               : "l"(r), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
  return o;
}

// Rounding error of the addition old + x (Knuth's TwoSum with every
// operation rounded on its own): (old + x) - fl(old + x), exactly.
__device__ __forceinline__ float two_sum_err(float old, float x) {
  const float t = __fadd_rn(old, x);
  const float z = __fsub_rn(t, old);
  return __fadd_rn(__fsub_rn(old, __fsub_rn(t, z)), __fsub_rn(x, z));
}

// Compensated (Kahan) step of a packed pair of sums: sum += y with the
// running compensation c (sum - c tracks the exact sum to one rounding).
__device__ __forceinline__ void f2_kahan(uint64_t& sum, uint64_t& c, uint64_t y) {
  const uint64_t yc = f2_sub(y, c);
  const uint64_t t = f2_add(sum, yc);
  c = f2_sub(f2_sub(t, sum), yc);
  sum = t;
}

__device__ __forceinline__ void red_add_u32(uint32_t* a, uint32_t v) {
  asm volatile("red.global.add.u32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}

__device__ __forceinline__ int32_t ld_acquire_i32(const int32_t* p) {
  return (int32_t)ld_acquire(reinterpret_cast<const uint32_t*>(p));
}

// TMA 2D load with an L2 evict-first policy: the embeddings are read once.
__device__ __forceinline__ void tma_load_2d_stream(uint32_t dst, const CUtensorMap* map,
                                                   int32_t x, int32_t y, uint32_t bar,
                                                   uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      ".L2::cache_hint [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar), "l"(policy)
      : "memory");
}

__device__ __forceinline__ uint64_t evict_first_policy() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

template <int BF16>
__device__ __forceinline__ float2 load2(const void* base, size_t idx) {
  if (BF16) {
    const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(
        static_cast<const __nv_bfloat16*>(base) + idx);
    return __bfloat1622float2(v);
  }
  return *reinterpret_cast<const float2*>(static_cast<const float*>(base) + idx);
}

template <int BF16>
__device__ __forceinline__ float4 load4(const void* base, size_t idx) {
  if (BF16) {
    const uint2 u = *reinterpret_cast<const uint2*>(static_cast<const __nv_bfloat16*>(base) + idx);
    const float2 fa = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
    const float2 fb = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
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

// Pixel p of local tile lt of a job: its point index, or -1 outside the
// frame. Organized frames (width > 0): tiles of 2^tw_log2 x 256 / 2^tw_log2
// pixels of the image, pixel p at row p >> tw_log2; else 256 consecutive
// points.
__device__ __forceinline__ int64_t tile_point(const OpenJob& J, uint32_t lt, int p) {
  int64_t j;
  if (J.width > 0) {
    const uint32_t tx = lt % J.tiles_x, ty = lt / J.tiles_x;
    const int32_t u = (int32_t)(tx << J.tw_log2) + (p & ((1 << J.tw_log2) - 1));
    const int64_t v = ((int64_t)ty << (8 - J.tw_log2)) + (p >> J.tw_log2);
    if (u >= J.width) return -1;
    j = v * J.width + u;
  } else {
    j = (int64_t)lt * kOT + p;
  }
  return j < J.n ? j : -1;
}

// Points staged per row of a tile, and the first point of row r (that many
// consecutive points are copied together).
__device__ __forceinline__ int tile_row_len(const OpenJob& J) {
  return J.width > 0 ? 1 << J.tw_log2 : kORowPts;
}
__device__ __forceinline__ int64_t tile_row_point(const OpenJob& J, uint32_t lt, int r) {
  if (J.width > 0) {
    const uint32_t tx = lt % J.tiles_x, ty = lt / J.tiles_x;
    return (((int64_t)ty << (8 - J.tw_log2)) + r) * J.width + ((int64_t)tx << J.tw_log2);
  }
  return (int64_t)lt * kOT + (int64_t)r * kORowPts;
}

struct OpenTileSmem {
  float stage[kOT * kOE];          // one chunk of every pixel's embedding
  uint64_t tbl_key[kOTbl];         // voxel key table
  uint16_t tbl_tv[kOTbl];          // table entry -> dense tile voxel
  uint64_t tv_key[kOMaxTV];
  unsigned long long tv_dq[kOMaxTV];  // sum of d, fixed point 2^-32 m
  uint32_t tv_mask[kOMaxTV][kOT / 32];
  uint32_t tv_off[kOMaxTV];        // start of the voxel's pixel list in plist
  uint16_t plist[kOT * 27];        // per voxel: its pixels' stage offsets (floats / 2)
  uint32_t tv_n[kOMaxTV];
  int32_t tv_row[kOMaxTV];
  uint32_t tv_flag[kOMaxTV];       // 1: row created here, 2: wait for another CTA
  uint16_t order[kOMaxTV];         // tile voxels by decreasing pixel count
  uint32_t scan[kOThreads / 32];
  uint32_t misc[2];                // 0 status, 1 table overflow
  uint32_t work[16];               // per chunk: next tile voxel for a warp
  uint32_t rowmask;                // staged rows holding a valid pixel
  int32_t parts[2 * 16];           // pending pixel ranges
  unsigned long long bar;
};

// Insert a voxel key into the tile table; returns its entry, or -1 when the
// table is full.
__device__ __forceinline__ int tbl_insert(OpenTileSmem& s, uint64_t key) {
  uint32_t h = (uint32_t)mix64(key) & (kOTbl - 1);
  for (int it = 0; it < kOTbl; ++it) {
    const uint64_t cur = *(volatile uint64_t*)&s.tbl_key[h];
    if (cur == key) return (int)h;
    if (cur == kEmptyKey) {
      const unsigned long long prev = atomicCAS((unsigned long long*)&s.tbl_key[h],
                                                (unsigned long long)kEmptyKey,
                                                (unsigned long long)key);
      if (prev == kEmptyKey || prev == key) return (int)h;
    }
    h = (h + 1) & (kOTbl - 1);
  }
  return -1;
}

__device__ __forceinline__ int tbl_find(const OpenTileSmem& s, uint64_t key) {
  uint32_t h = (uint32_t)mix64(key) & (kOTbl - 1);
  for (int it = 0; it < kOTbl; ++it) {
    const uint64_t cur = s.tbl_key[h];
    if (cur == key) return (int)h;
    if (cur == kEmptyKey) return -1;
    h = (h + 1) & (kOTbl - 1);
  }
  return -1;
}

// Issue the TMA copies of chunk c of the tile (its rows of consecutive
// points x 64 elements) on the stage barrier.
// Rows without a valid pixel (s.rowmask bit clear) are not copied: their
// stage rows are never read.
__device__ __forceinline__ void issue_chunk(OpenTileSmem& s, const OpenJob& J, uint32_t lt, int c,
                                            uint64_t policy) {
  const uint32_t bar = smem_u32(&s.bar);
  const int rl = tile_row_len(J), nr = kOT / rl;
  const uint32_t rm = s.rowmask;
  mbar_expect_tx(bar, (uint32_t)__popc(rm) * (uint32_t)rl * kOE * 4u);
  for (int r = 0; r < nr; ++r) {
    const int64_t y = tile_row_point(J, lt, r);
    if (!((rm >> r) & 1u)) continue;
    tma_load_2d_stream(smem_u32(&s.stage[r * rl * kOE]), &J.sem_map, c * kOE, (int32_t)y, bar,
                       policy);
  }
}

template <int BF16>
__global__ void __launch_bounds__(kOThreads, 2) k_open_tile(const __grid_constant__ OpenBatch b) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  OpenTileSmem& s = *reinterpret_cast<OpenTileSmem*>(smraw);
  const uint32_t t = blockIdx.x;
  int jb = 0;
  while (jb + 1 < b.n_jobs && t >= b.job[jb + 1].tile_begin) ++jb;
  const OpenJob& J = b.job[jb];
  const MapView& mv = J.mv;
  const uint32_t lt = t - J.tile_begin;
  const int tid = threadIdx.x;
  const unsigned lane = lane_id(), warp = tid >> 5;
  const int L = J.L;
  const int nch = L / kOE;
  const uint32_t bar = smem_u32(&s.bar);
  uint64_t policy = 0;
  if (tid == 0) {
    s.misc[0] = *(volatile uint32_t*)&mv.ctr[kCtrStatus];
    s.parts[0] = 0;  // the first part: the whole tile
    s.parts[1] = kOT;
    s.rowmask = 0u;
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (s.misc[0]) return;
  // this thread's pixel and ray; the staged rows that hold a valid pixel
  const int64_t pj = tid < kOT ? tile_point(J, lt, tid) : -1;
  Ray ray0;
  const bool valid = pj >= 0 && ray_setup_at(J.g, J.pts, pj, ray0);
  if (valid) atomicOr(&s.rowmask, 1u << (tid / tile_row_len(J)));
  __syncthreads();
  // chunk 0 is fetched while the rays are walked (it serves every part)
  int cur = 0;          // chunk held or in flight in the stage
  bool inflight = true;
  uint32_t phase = 0;   // parity of the next completion of the stage barrier
  if (tid == 0) {
    policy = evict_first_policy();
    issue_chunk(s, J, lt, 0, policy);
  }

  int nparts = 1;
  bool abort = false;
  while (nparts > 0 && !abort) {
    --nparts;
    const int p0 = s.parts[2 * nparts], p1 = s.parts[2 * nparts + 1];
    const bool mine = valid && tid >= p0 && tid < p1;
    // 1. the part's distinct voxels
    for (int e = tid; e < kOTbl; e += kOThreads) s.tbl_key[e] = kEmptyKey;
    if (tid == 0) s.misc[1] = 0;
    __syncthreads();
    if (mine) {
      Ray ry = ray0;
      ray_for_each(J.g, ry, [&](int32_t i0, int32_t i1, int32_t i2, float) {
        if (tbl_insert(s, pack_voxel(i0, i1, i2)) < 0) s.misc[1] = 1;
      });
    }
    __syncthreads();
    // 2. dense ids (4 table entries per thread)
    uint32_t occ = 0;
#pragma unroll
    for (int k = 0; k < kOTbl / kOThreads; ++k) occ += s.tbl_key[tid * 4 + k] != kEmptyKey;
    uint32_t ntv;
    uint32_t off = cta_exclusive_scan(occ, s.scan, &ntv);
    if (ntv > (uint32_t)kOMaxTV || s.misc[1]) {
      // too many voxels for the tables: split the part in two
      __syncthreads();
      if (tid == 0) {
        const int mid = (p0 + p1) / 2;
        s.parts[2 * nparts] = p0;
        s.parts[2 * nparts + 1] = mid;
        s.parts[2 * nparts + 2] = mid;
        s.parts[2 * nparts + 3] = p1;
      }
      nparts += 2;
      __syncthreads();
      continue;
    }
#pragma unroll
    for (int k = 0; k < kOTbl / kOThreads; ++k) {
      const int e = tid * 4 + k;
      const uint64_t key = s.tbl_key[e];
      if (key != kEmptyKey) {
        s.tbl_tv[e] = (uint16_t)off;
        s.tv_key[off] = key;
        ++off;
      }
    }
    if (tid < 16) s.work[tid] = 0u;
    for (int v = tid; v < (int)ntv; v += kOThreads) {
      s.tv_n[v] = 0;
      s.tv_dq[v] = 0ull;
      s.tv_flag[v] = 0;
#pragma unroll
      for (int w = 0; w < kOT / 32; ++w) s.tv_mask[v][w] = 0u;
    }
    __syncthreads();
    // 3. pixel masks, counts and fixed-point sums of d
    if (mine) {
      Ray ry = ray0;
      ray_for_each(J.g, ry, [&](int32_t i0, int32_t i1, int32_t i2, float d) {
        const int e = tbl_find(s, pack_voxel(i0, i1, i2));
        const int v = s.tbl_tv[e];
        atomicOr(&s.tv_mask[v][tid >> 5], 1u << (tid & 31));
        atomicAdd(&s.tv_n[v], 1u);
        atomicAdd(&s.tv_dq[v], fx32(d));
      });
    }
    __syncthreads();
    // 4. blocks and rows: find, or create (a new row gets its shift and
    //    zero (S, W) before it is published), or wait for another CTA's
    int32_t* vr = nullptr;
    if (tid < (int)ntv) {
      int32_t i0, i1, i2;
      unpack_voxel(s.tv_key[tid], i0, i1, i2);
      const uint32_t slot = map_block_slot(mv, pack_block(i0 >> 3, i1 >> 3, i2 >> 3));
      int32_t row = kFailRow;
      if (slot < mv.block_cap) {
        vr = mv.vox_row + (size_t)slot * kBlockVoxels + local_index(i0, i1, i2);
        const int32_t r0 = atomicCAS(vr, -1, kPendingRow);
        if (r0 == -1) {
          const uint32_t r = atomicAdd(&mv.ctr[kCtrRows], 1u);
          if (r >= mv.row_cap) {
            raise_status(mv.ctr, kDevCapacity, 12);
            st_release(reinterpret_cast<uint32_t*>(vr), (uint32_t)kFailRow);
          } else {
            row = (int32_t)r;
            s.tv_flag[tid] = 1;
          }
        } else if (r0 == kPendingRow) {
          s.tv_flag[tid] = 2;
        } else if (r0 >= 0) {
          row = r0;
        }
      }
      s.tv_row[tid] = row;
    }
    __syncthreads();
    // the shift of each row created here: the embedding of its first pixel
    for (int v = (int)warp; v < (int)ntv; v += kOThreads / 32) {
      if (s.tv_flag[v] != 1) continue;
      int p = 0;
      for (int w = 0; w < kOT / 32; ++w)
        if (s.tv_mask[v][w]) {
          p = 32 * w + __ffs(s.tv_mask[v][w]) - 1;
          break;
        }
      const int64_t jp = tile_point(J, lt, p);
      const int32_t row = s.tv_row[v];
      const float* src = J.sem + (size_t)jp * L;
      for (int e = 4 * (int)lane; e < L; e += 128)
        store4<BF16>(mv.mrow, (size_t)row * L + e, *reinterpret_cast<const float4*>(src + e));
      if (lane == 0) mv.tsdf[row] = make_float2(0.f, 0.f);
    }
    __threadfence();
    __syncthreads();
    if (tid < (int)ntv) {
      if (s.tv_flag[tid] == 1) {
        st_release(reinterpret_cast<uint32_t*>(vr), (uint32_t)s.tv_row[tid]);
      } else if (s.tv_flag[tid] == 2) {
        int32_t r = ld_acquire_i32(vr);
        if (r == kPendingRow) {
          const uint64_t t0 = global_ns();
          while ((r = ld_acquire_i32(vr)) == kPendingRow) {
            if (global_ns() - t0 > kCrossCtaWaitNs) {
              raise_status(mv.ctr, kDevTimeout, 14);
              r = kFailRow;
              break;
            }
            __nanosleep(100);
          }
        }
        s.tv_row[tid] = r >= 0 ? r : kFailRow;
      }
      const int32_t row = s.tv_row[tid];
      if (row >= 0 && atomicExch(&J.acc.listed[row], 1u) == 0u)
        J.acc.list[atomicAdd(J.acc.count, 1u)] = (uint32_t)row;
      // rank by decreasing pixel count (ties by id): the longest voxels first
      const uint32_t n0 = s.tv_n[tid];
      int rank = 0;
      for (int v = 0; v < (int)ntv; ++v) {
        const uint32_t nv = s.tv_n[v];
        rank += nv > n0 || (nv == n0 && v < tid);
      }
      s.order[rank] = (uint16_t)tid;
    }
    // the pixel lists: offsets of the voxels' lists (exclusive scan of the
    // counts), then one warp per voxel expands its mask, 8 pixels per lane
    {
      uint32_t tot;
      const uint32_t o = cta_exclusive_scan(tid < (int)ntv ? s.tv_n[tid] : 0u, s.scan, &tot);
      if (tid < (int)ntv) s.tv_off[tid] = o;
      __syncthreads();
      for (int v = (int)warp; v < (int)ntv; v += kOThreads / 32) {
        const uint32_t bits = (s.tv_mask[v][lane >> 2] >> (8 * (lane & 3))) & 0xFFu;
        uint32_t x = (uint32_t)__popc(bits);
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
          if ((int)lane >= off) x += y;
        }
        uint32_t at = s.tv_off[v] + x - (uint32_t)__popc(bits);
        uint32_t b = bits;
        while (b) {
          const int p = 8 * (int)lane + __ffs(b) - 1;
          b &= b - 1;
          s.plist[at++] = (uint16_t)(p * (kOE / 2));
        }
      }
    }
    __syncthreads();
    // 5. per chunk: sums of y = z - s and y^2 over each voxel's pixels, in
    //    two alternating chains, the sums of y compensated (Kahan); warps
    //    take voxels (longest first) from a shared counter
    for (int c = 0; c < nch; ++c) {
      if (cur != c) {  // the stage is free (barrier at the end of the last chunk)
        if (tid == 0) issue_chunk(s, J, lt, c, policy);
        cur = c;
        inflight = true;
      }
      if (inflight) {
        const bool ok = mbar_wait(bar, phase);
        if (__syncthreads_or(!ok)) {  // a copy that never landed: stop, uniformly
          if (tid == 0) raise_status(mv.ctr, kDevTimeout, 15);
          abort = true;
          break;
        }
        phase ^= 1u;
        inflight = false;
      }
      const int e0 = c * kOE + 2 * (int)lane;
      for (;;) {
        uint32_t k = 0;
        if (lane == 0) k = atomicAdd(&s.work[c], 1u);
        k = __shfl_sync(0xFFFFFFFFu, k, 0);
        if (k >= ntv) break;
        const int v = s.order[k];
        const int32_t row = s.tv_row[v];
        if (row < 0) continue;
        const float2 sh = load2<BF16>(mv.mrow, (size_t)row * L + e0);
        const uint64_t s2 = f2_pack(sh.x, sh.y);
        uint64_t a1 = 0, a2 = 0, b1 = 0, b2 = 0, ca = 0, cb = 0;
        const uint64_t* st64 = reinterpret_cast<const uint64_t*>(s.stage) + lane;
        const uint32_t pb0 = s.tv_off[v], pe = pb0 + s.tv_n[v];
        uint32_t i = pb0;
        for (; i + 1 < pe; i += 2) {
          const uint64_t za = st64[s.plist[i]];
          const uint64_t zb = st64[s.plist[i + 1]];
          const uint64_t ya = f2_sub(za, s2), yb = f2_sub(zb, s2);
          f2_kahan(a1, ca, ya);
          a2 = f2_fma(ya, ya, a2);
          f2_kahan(b1, cb, yb);
          b2 = f2_fma(yb, yb, b2);
        }
        if (i < pe) {
          const uint64_t ya = f2_sub(st64[s.plist[i]], s2);
          f2_kahan(a1, ca, ya);
          a2 = f2_fma(ya, ya, a2);
        }
        const float2 S1 = f2_unpack(f2_add(f2_sub(a1, ca), f2_sub(b1, cb)));
        const float2 S2 = f2_unpack(f2_add(a2, b2));
        // across tiles, compensated: the high half of the accumulator takes
        // the sums, the low half the exact rounding error of each addition
        float* hi = J.acc.rows + (size_t)row * J.acc.stride + 4 + 2 * e0;
        const float4 old = atom_add_v4(hi, S1.x, S2.x, S1.y, S2.y);
        red_add_v4_nc(hi + 2 * L, two_sum_err(old.x, S1.x), two_sum_err(old.y, S2.x),
                      two_sum_err(old.z, S1.y), two_sum_err(old.w, S2.y));
      }
      __syncthreads();  // the stage is free again
    }
    if (abort) break;
    // 6. counts and sums of d
    if (tid < (int)ntv) {
      const int32_t row = s.tv_row[tid];
      if (row >= 0) {
        float* h = J.acc.rows + (size_t)row * J.acc.stride;
        red_add_u64(reinterpret_cast<unsigned long long*>(h), s.tv_dq[tid]);
        red_add_u32(reinterpret_cast<uint32_t*>(h) + 2, s.tv_n[tid]);
      }
    }
    __syncthreads();
  }
  if (abort && inflight) mbar_wait(bar, phase);  // let the copy land (bounded)
}

// Apply the accumulated statistics to every row the call touched (one warp
// per row), then clear the accumulators and the rows' list flags. With the
// map's status raised the rows are only cleared.
template <int BF16>
__global__ void __launch_bounds__(256) k_open_apply(const __grid_constant__ OpenApplyBatch b) {
  const unsigned lane = lane_id();
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int jb = 0; jb < b.n_jobs; ++jb) {
    const MapView& mv = b.job[jb].mv;
    const OpenAcc& A = b.job[jb].acc;
    const int L = b.job[jb].L;
    const bool live = *(volatile uint32_t*)&mv.ctr[kCtrStatus] == 0;
    const int64_t cnt = min((int64_t)*A.count, (int64_t)mv.row_cap);
    for (int64_t i = gw; i < cnt; i += nw) {
      const uint32_t row = A.list[i];
      float* h = A.rows + (size_t)row * A.stride;
      if (lane == 0) A.listed[row] = 0u;
      if (live) {
        const long long dq = *reinterpret_cast<const long long*>(h);
        const uint32_t n = reinterpret_cast<const uint32_t*>(h)[2];
        const float2 sw = mv.tsdf[row];
        const float Wn = sw.y + (float)n;
        const float inv = 1.0f / Wn;
        const bool seen = sw.y > 0.f;
        const size_t rb = (size_t)row * L;
        float nrm = 0.f, nbf = 0.f;
        for (int e = 4 * (int)lane; e < L; e += 128) {
          float4* a4 = reinterpret_cast<float4*>(h + 4 + 2 * e);          // high halves
          float4* c4 = reinterpret_cast<float4*>(h + 4 + 2 * L + 2 * e);  // low halves
          const float4 p = a4[0], q = a4[1], pc = c4[0], qc = c4[1];
          // (S1, S2) of elements e .. e + 3
          const float s1[4] = {p.x + pc.x, p.z + pc.z, q.x + qc.x, q.z + qc.z};
          const float s2[4] = {p.y + pc.y, p.w + pc.w, q.y + qc.y, q.w + qc.w};
          const float4 m4 = load4<BF16>(mv.mrow, rb + e);
          const float4 b4 = seen ? load4<BF16>(mv.brow, rb + e) : make_float4(0.f, 0.f, 0.f, 0.f);
          float mv4[4] = {m4.x, m4.y, m4.z, m4.w}, bv4[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            bv4[k] += 0.5f * fmaxf(s2[k] - s1[k] * s1[k] * inv, 0.f);
            mv4[k] += s1[k] * inv;
          }
          float4 mo = make_float4(mv4[0], mv4[1], mv4[2], mv4[3]);
          store4<BF16>(mv.mrow, rb + e, mo);
          store4<BF16>(mv.brow, rb + e, make_float4(bv4[0], bv4[1], bv4[2], bv4[3]));
          if (!BF16) {  // the query's BF16 copy of the FP32 mean, and its norm
            store4<1>(mv.mbf, rb + e, mo);
            const float4 q4 = load4<1>(mv.mbf, rb + e);
            nbf += q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w;
          }
          if (BF16) mo = load4<BF16>(mv.mrow, rb + e);  // norm of the stored values
          nrm += mo.x * mo.x + mo.y * mo.y + mo.z * mo.z + mo.w * mo.w;
          a4[0] = a4[1] = c4[0] = c4[1] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          nrm += __shfl_xor_sync(0xFFFFFFFFu, nrm, off);
          nbf += __shfl_xor_sync(0xFFFFFFFFu, nbf, off);
        }
        if (lane == 0) {
          mv.tsdf[row] = make_float2(sw.x + unfx32(dq), Wn);
          mv.mnorm2[row] = nrm;
          if (!BF16) mv.mbf_norm2[row] = nbf;
          reinterpret_cast<float4*>(h)[0] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      } else {
        for (int e = 4 * (int)lane; e < 4 * L + 4; e += 128)
          *reinterpret_cast<float4*>(h + e) = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  }
}

// ------------------------------------------------------------------ host
size_t open_tile_smem_bytes() { return sizeof(OpenTileSmem) + 1024; }

cudaError_t open_setup_attributes() {
  const int sm = (int)open_tile_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(k_open_tile<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_open_tile<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  return e;
}

slim_status open_alloc_scratch(slim_map* m, OpenScratch& o) {
  const uint64_t rc = (uint64_t)m->p.voxel_capacity;
  o.acc.stride = 4 + 4 * m->L;
  slim_status s;
  if ((s = m->alloc(&o.acc.rows, rc * (uint64_t)o.acc.stride)) != SLIM_OK) return s;
  if ((s = m->alloc(&o.acc.listed, rc)) != SLIM_OK) return s;
  if ((s = m->alloc(&o.acc.list, rc)) != SLIM_OK) return s;
  if ((s = m->alloc(&o.acc.count, (size_t)1)) != SLIM_OK) return s;
  if (cudaMemset(o.acc.rows, 0, rc * (uint64_t)o.acc.stride * sizeof(float)) != cudaSuccess ||
      cudaMemset(o.acc.listed, 0, rc * sizeof(uint32_t)) != cudaSuccess)
    return fail(SLIM_ERR_CUDA, "cudaMemset of the open-set accumulators failed");
  return SLIM_OK;
}

bool open_encode_sem(CUtensorMap* map, const float* sem, int64_t n, int L, int row_pts) {
  auto fn = get_encode();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)L, (cuuint64_t)std::max<int64_t>(n, 1)};
  cuuint64_t strides[1] = {(cuuint64_t)L * 4};
  cuuint32_t box[2] = {(cuuint32_t)kOE, (cuuint32_t)row_pts};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(sem), dims, strides,
                  box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

uint32_t open_job_tiles(OpenJob& J) {
  if (J.n <= 0) return 0;
  if (J.width > 0) {
    const int tw = 1 << J.tw_log2, th = kOT / tw;
    J.tiles_x = (uint32_t)((J.width + tw - 1) / tw);
    const int64_t rows = (J.n + J.width - 1) / J.width;
    return J.tiles_x * (uint32_t)((rows + th - 1) / th);
  }
  J.tiles_x = 0;
  return (uint32_t)((J.n + kOT - 1) / kOT);
}

cudaError_t launch_open_tiles(OpenBatch& b, int bf16, cudaStream_t st) {
  uint32_t total = 0;
  for (int k = 0; k < b.n_jobs; ++k) {
    b.job[k].tile_begin = total;
    total += open_job_tiles(b.job[k]);
  }
  b.total_tiles = total;
  if (total == 0) return cudaSuccess;
  const size_t sm = open_tile_smem_bytes();
  if (bf16)
    k_open_tile<1><<<total, kOThreads, sm, st>>>(b);
  else
    k_open_tile<0><<<total, kOThreads, sm, st>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_open_apply(const OpenApplyBatch& a, int bf16, cudaStream_t st) {
  if (a.n_jobs == 0) return cudaSuccess;
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (bf16)
    k_open_apply<1><<<(unsigned)(sms * 8), 256, 0, st>>>(a);
  else
    k_open_apply<0><<<(unsigned)(sms * 8), 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace slim

namespace slim {

__global__ void __launch_bounds__(256) k_reset_vox_rows(int4* vox_row, const uint32_t* ctr,
                                                        uint32_t block_cap) {
  const uint32_t nb = min(*(volatile const uint32_t*)&ctr[kCtrBlocks], block_cap);
  const size_t n4 = (size_t)nb * kBlockVoxels / 4;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
       i += (size_t)gridDim.x * blockDim.x)
    vox_row[i] = make_int4(-1, -1, -1, -1);
}

cudaError_t launch_reset_vox_rows(const MapView& mv, cudaStream_t st) {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  k_reset_vox_rows<<<(unsigned)(sms * 4), 256, 0, st>>>(reinterpret_cast<int4*>(mv.vox_row),
                                                         mv.ctr, mv.block_cap);
  return cudaGetLastError();
}

slim_status open_fill_job(slim_map* m, OpenJob& J, const ScanGeom& g, const float* pts,
                          const float* sem, int64_t n, int width) {
  J.mv = m->mv;
  J.g = g;
  J.acc = m->open.acc;
  J.pts = pts;
  J.sem = sem;
  J.n = n;
  J.L = m->L;
  J.width = width;
  J.tw_log2 = m->open.tw_log2;
  if (!open_encode_sem(&J.sem_map, sem, n, m->L, width > 0 ? 1 << J.tw_log2 : kORowPts))
    return fail(SLIM_ERR_CUDA, "cuTensorMapEncodeTiled failed for the embeddings");
  return SLIM_OK;
}

slim_status open_integrate(slim_map* m, const ScanGeom& g, const float* pts, const float* sem,
                           int64_t n, int width, cudaStream_t st) {
  if (n <= 0) return SLIM_OK;
  OpenBatch b;
  b.n_jobs = 1;
  slim_status s = open_fill_job(m, b.job[0], g, pts, sem, n, width);
  if (s != SLIM_OK) return s;
  cudaError_t e = cudaMemsetAsync(m->open.acc.count, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return fail(SLIM_ERR_CUDA, cudaGetErrorString(e));
  int tok = prof_begin(m, SLIM_KERNEL_OPEN_TILE, st);
  e = launch_open_tiles(b, m->bf16, st);
  prof_end(m, tok, st);
  if (e != cudaSuccess) return fail(SLIM_ERR_CUDA, cudaGetErrorString(e));
  OpenApplyBatch a;
  a.n_jobs = 1;
  a.job[0].mv = m->mv;
  a.job[0].acc = m->open.acc;
  a.job[0].L = m->L;
  tok = prof_begin(m, SLIM_KERNEL_OPEN_APPLY, st);
  e = launch_open_apply(a, m->bf16, st);
  prof_end(m, tok, st);
  if (e != cudaSuccess) return fail(SLIM_ERR_CUDA, cudaGetErrorString(e));
  return SLIM_OK;
}

// Open-set items of a batch: one tile launch per storage kind and 16 items,
// then one apply launch per storage kind and 16 maps. Items of the same map
// share the map's accumulators (one observation set).
slim_status open_integrate_batch(const std::vector<OpenItem>& items, cudaStream_t st) {
  if (items.empty()) return SLIM_OK;
  std::vector<slim_map*> maps;
  for (const OpenItem& it : items)
    if (std::find(maps.begin(), maps.end(), it.map) == maps.end()) maps.push_back(it.map);
  for (size_t k = 0; k < maps.size(); ++k) {
    cudaError_t e = cudaMemsetAsync(maps[k]->open.acc.count, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return fail(SLIM_ERR_CUDA, cudaGetErrorString(e));
  }
  for (int bf = 0; bf < 2; ++bf) {
    OpenBatch b;
    b.n_jobs = 0;
    slim_map* first = nullptr;
    auto flush = [&]() -> slim_status {
      if (b.n_jobs == 0) return SLIM_OK;
      const int tok = prof_begin(first, SLIM_KERNEL_OPEN_TILE, st);
      cudaError_t e = launch_open_tiles(b, bf, st);
      prof_end(first, tok, st);
      b.n_jobs = 0;
      first = nullptr;
      return e == cudaSuccess ? SLIM_OK : fail(SLIM_ERR_CUDA, cudaGetErrorString(e));
    };
    for (const OpenItem& it : items) {
      if (it.map->bf16 != bf || it.n <= 0) continue;
      if (!first) first = it.map;
      slim_status s = open_fill_job(it.map, b.job[b.n_jobs], it.g, it.pts, it.sem, it.n,
                                    it.width);
      if (s != SLIM_OK) return s;
      if (++b.n_jobs == kMaxOpenJobs) {
        if ((s = flush()) != SLIM_OK) return s;
      }
    }
    slim_status s = flush();
    if (s != SLIM_OK) return s;
  }
  for (int bf = 0; bf < 2; ++bf) {
    OpenApplyBatch a;
    a.n_jobs = 0;
    slim_map* first = nullptr;
    auto flush = [&]() -> slim_status {
      if (a.n_jobs == 0) return SLIM_OK;
      const int tok = prof_begin(first, SLIM_KERNEL_OPEN_APPLY, st);
      cudaError_t e = launch_open_apply(a, bf, st);
      prof_end(first, tok, st);
      a.n_jobs = 0;
      first = nullptr;
      return e == cudaSuccess ? SLIM_OK : fail(SLIM_ERR_CUDA, cudaGetErrorString(e));
    };
    for (slim_map* m : maps) {
      if (m->bf16 != bf) continue;
      if (!first) first = m;
      a.job[a.n_jobs].mv = m->mv;
      a.job[a.n_jobs].acc = m->open.acc;
      a.job[a.n_jobs].L = m->L;
      if (++a.n_jobs == kMaxOpenJobs) {
        slim_status s = flush();
        if (s != SLIM_OK) return s;
      }
    }
    slim_status s = flush();
    if (s != SLIM_OK) return s;
  }
  return SLIM_OK;
}

}  // namespace slim
