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
//   k_open_tile   one CTA per tile of 256 pixels of an organized frame
//                 (16 x 16, 8 x 32 or 32 x 8) or 256 consecutive points: band
//                 DDA per pixel; the tile's distinct voxels in a shared-memory
//                 table with their pixel lists and sums of d; blocks and voxel
//                 rows looked up or created in the map (a new row gets its
//                 shift, the embedding of one of its pixels, before it is
//                 published); the embedding rows streamed in 64-element
//                 chunks by TMA into shared memory, each read once from HBM;
//                 per chunk a warp takes four pieces (at most 64 pixels of a
//                 voxel's list each), sums y = z - s and y^2 over their
//                 pixels (packed FP32x2 arithmetic) and adds them to the
//                 rows' accumulators as exact 64-bit integer reductions.
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
constexpr int kOTbl = 512;        // voxel table entries (power of two)
constexpr int kOPList = 4096;     // pixel-list entries per part (more: the part splits)
constexpr int kOPiece = 64;       // pixels per piece of a voxel's list (a multiple of 4)
constexpr int kOMaxPc = kOMaxTV + kOPList / kOPiece;  // pieces per part
constexpr int kOThreads = 256;
// Points of one map per integration call: each piece adds at most 2^39
// units to a voxel's S1 and S2 (|z - s| <= 2B over <= 64 pixels), so 2^23
// pieces keep every exact 64-bit sum below 2^62.
constexpr int64_t kOpenMaxCallPoints = (int64_t)1 << 23;
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
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
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

// 8 (FP32) or 4 (BF16) bytes from global to shared memory, asynchronously.
template <int BYTES>
__device__ __forceinline__ void cp_async(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(dst), "l"(src), "n"(BYTES)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}
__device__ __forceinline__ uint64_t lds_u64(uint32_t a) {
  uint64_t v;
  asm volatile("ld.shared.u64 %0, [%1];" : "=l"(v) : "r"(a));
  return v;
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

// Bring a tensor-map box into L2 (no shared memory, no completion).
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap* map, int32_t x, int32_t y) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y)
               : "memory");
}

__device__ __forceinline__ uint64_t evict_first_policy() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
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
  uint32_t tbl_cnt[kOTbl];         // pixels per table entry
  uint16_t tbl_tv[kOTbl];          // table entry -> dense tile voxel
  uint64_t tv_key[kOMaxTV];
  int32_t tv_dq[kOMaxTV];          // sum of d in units of tau 2^-22 (exact: |sum| < 2^30)
  uint32_t tv_off[kOMaxTV];        // start of the voxel's pixel list (a multiple of 4)
  uint32_t tv_n[kOMaxTV];          // pixels of the voxel
  uint32_t tv_cur[kOMaxTV];        // list fill cursor
  int32_t tv_row[kOMaxTV];
  uint32_t tv_flag[kOMaxTV];       // 1: row created here, 2: wait for another CTA
  uint32_t piece[kOMaxPc];         // pieces, longest first (piece_rec)
  uint32_t pbin[kOPiece / 4];      // partial pieces per length in groups of 4
  uint32_t work[16];               // per chunk: next quad of pieces for a warp
  uint64_t shv[kOThreads / 32][4][32];  // per warp: its quad's row shifts (element pairs)
  // per voxel: its pixels' stage offsets (in 8-byte words), padded to a
  // multiple of 4 entries with the list's first pixel
  __align__(16) uint32_t plist[kOPList];
  uint32_t scan[kOThreads / 32];
  uint32_t misc[2];                // 0 status, 1 table overflow
  uint32_t rowmask;                // staged rows holding a valid pixel
  int32_t parts[2 * 16];           // pending pixel ranges
  unsigned long long bar;
};


// Two CTAs per SM: 228 KB of shared memory per SM, 1 KB reserved per CTA,
// plus the 1 KB alignment slack of the dynamic allocation.
static_assert(sizeof(OpenTileSmem) + 1024 <= (228 * 1024) / 2 - 1024,
              "k_open_tile needs two CTAs per SM");

// A piece of a voxel's pixel list: tile voxel v, first group of 4 entries
// g0, groups ng, pixels n (the last group may hold padding).
__device__ __forceinline__ uint32_t piece_rec(uint32_t v, uint32_t g0, uint32_t ng, uint32_t n) {
  return v | (g0 << 8) | (ng << 14) | (n << 19);
}

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
  // keep the next two chunks on their way into L2 (64 KB per chunk and
  // CTA): their stage copies then read L2 instead of waiting on HBM
  const int cn = c == 0 ? 1 : c + 2;
  for (int k = cn; k <= c + 2 && k * kOE < J.L; ++k)
    for (int r = 0; r < nr; ++r)
      if ((rm >> r) & 1u) tma_prefetch_2d(&J.sem_map, k * kOE, (int32_t)tile_row_point(J, lt, r));
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
  bool valid;
  {
    Ray ry;  // set up again by each walk (fewer registers held across the part)
    valid = pj >= 0 && ray_setup_at(J.g, J.pts, pj, ry);
  }
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
    // 1. the part's distinct voxels and their pixel counts
    for (int e = tid; e < kOTbl; e += kOThreads) {
      s.tbl_key[e] = kEmptyKey;
      s.tbl_cnt[e] = 0u;
    }
    if (tid == 0) s.misc[1] = 0;
    __syncthreads();
    if (mine) {
      Ray ry;
      ray_setup_at(J.g, J.pts, pj, ry);
      ray_for_each(J.g, ry, [&](int32_t i0, int32_t i1, int32_t i2, float) {
        const int e = tbl_insert(s, pack_voxel(i0, i1, i2));
        if (e < 0)
          s.misc[1] = 1;
        else
          atomicAdd(&s.tbl_cnt[e], 1u);
      });
    }
    __syncthreads();
    // 2. dense ids (2 table entries per thread)
    constexpr int kPer = kOTbl / kOThreads;
    uint32_t occ = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) occ += s.tbl_cnt[tid * kPer + k] != 0u;
    uint32_t ntv;
    uint32_t id = cta_exclusive_scan(occ, s.scan, &ntv);
    if (ntv > (uint32_t)kOMaxTV || s.misc[1]) {
      // too many voxels for the tables: split the part
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
    for (int k = 0; k < kPer; ++k) {
      const int e = tid * kPer + k;
      const uint32_t c = s.tbl_cnt[e];
      if (c) {
        s.tbl_tv[e] = (uint16_t)id;
        s.tv_key[id] = s.tbl_key[e];
        s.tv_n[id] = c;
        s.tv_cur[id] = 0u;
        s.tv_dq[id] = 0;
        s.tv_flag[id] = 0u;
        ++id;
      }
    }
    if (tid < 16) s.work[tid] = 0u;
    __syncthreads();
    // 3. list offsets (each voxel's list padded to a multiple of 4 entries)
    //    and the pieces: every list cut into pieces of at most kOPiece
    //    pixels, longest first (full pieces, then the rest by length), so
    //    that quads of consecutive pieces cost about the same
    {
      const uint32_t n = tid < (int)ntv ? s.tv_n[tid] : 0u;
      const uint32_t full = n / kOPiece, rest = n % kOPiece;
      const uint32_t packed = ((n + 3u) & ~3u) | (full << 20);
      if (tid < 16) s.pbin[tid] = 0u;
      uint32_t tot;
      const uint32_t pre = cta_exclusive_scan(packed, s.scan, &tot);
      const uint32_t nfull = tot >> 20;
      if ((tot & 0xFFFFFu) > (uint32_t)kOPList) {
        // too many list entries: split the part
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
      if (tid < (int)ntv) {
        s.tv_off[tid] = pre & 0xFFFFFu;
        for (uint32_t k = 0; k < full; ++k)
          s.piece[(pre >> 20) + k] = piece_rec(tid, k * (kOPiece / 4), kOPiece / 4, kOPiece);
        if (rest) atomicAdd(&s.pbin[(rest + 3u) / 4u - 1u], 1u);
      }
      __syncthreads();
      if (tid == 0) {  // bins of the partial pieces, longest first
        uint32_t at = nfull;
        for (int b = kOPiece / 4 - 1; b >= 0; --b) {
          const uint32_t c = s.pbin[b];
          s.pbin[b] = at;
          at += c;
        }
        s.misc[1] = at;  // pieces of the part
      }
      __syncthreads();
      if (tid < (int)ntv && rest) {
        const uint32_t g = (rest + 3u) / 4u;
        s.piece[atomicAdd(&s.pbin[g - 1u], 1u)] = piece_rec(tid, full * (kOPiece / 4), g, rest);
      }
    }
    const uint32_t npc = s.misc[1];
    __syncthreads();
    // 4. pixel lists and fixed-point sums of d
    if (mine) {
      Ray ry;
      ray_setup_at(J.g, J.pts, pj, ry);
      const uint32_t so = (uint32_t)tid * (kOE / 2);  // the pixel's stage row, 8-byte words
      const float dsc = __fdiv_rn(4194304.0f, J.g.tau);
      ray_for_each(J.g, ry, [&](int32_t i0, int32_t i1, int32_t i2, float d) {
        const int v = s.tbl_tv[tbl_find(s, pack_voxel(i0, i1, i2))];
        s.plist[s.tv_off[v] + atomicAdd(&s.tv_cur[v], 1u)] = so;
        atomicAdd(&s.tv_dq[v], __float2int_rn(__fmul_rn(d, dsc)));
      });
    }
    __syncthreads();
    // 5. list padding (with the first pixel of the list's last piece, whose
    //    deviation from that piece's shift is exactly zero); blocks and rows:
    //    find, or create (a new row gets its shift and zero (S, W) before it
    //    is published), or wait for another CTA's
    int32_t* vr = nullptr;
    if (tid < (int)ntv) {
      const uint32_t o = s.tv_off[tid], n = s.tv_n[tid];
      if (n & 3u) {
        const uint32_t f = s.plist[o + (n / kOPiece) * kOPiece];
        for (uint32_t j = n; j & 3u; ++j) s.plist[o + j] = f;
      }
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
    // the shift of each row created here: the embedding of its list's first
    // pixel
    for (int v = (int)warp; v < (int)ntv; v += kOThreads / 32) {
      if (s.tv_flag[v] != 1) continue;
      const int p = (int)(s.plist[s.tv_off[v]] / (kOE / 2));
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
    }
    __syncthreads();
    // 6. per chunk and quad of pieces: each piece's sums of y = z - s_t and
    //    y^2 over its pixels, about its first pixel s_t (in shared memory),
    //    the quad's four pieces in lockstep (four independent chains, each
    //    group of four pixels summed as a tree first); then taken about the
    //    row's shift s (d = s_t - s, n pixels):
    //      S1 = S1_t + n d,   S2 = S2_t + d (2 S1_t + n d),
    //    and added to the row's accumulator exactly, as 64-bit integer
    //    reductions (no return value, so no round trip holds the warp; the
    //    quad's four shift loads travel while the sums run). Warps take
    //    quads (longest first) from a shared counter.
    const uint32_t nq = (npc + 3u) >> 2;
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
      const uint64_t* st64 = reinterpret_cast<const uint64_t*>(s.stage) + lane;
      for (;;) {
        uint32_t q = 0;
        if (lane == 0) q = atomicAdd(&s.work[c], 1u);
        q = __shfl_sync(0xFFFFFFFFu, q, 0);
        if (q >= nq) break;
        int32_t row[4];
        uint32_t pr[4];
        const uint4* pl[4];
        uint64_t sl[4], a1[4], a2[4];
        const uint32_t ng = (s.piece[4 * q] >> 14) & 0x1Fu;  // the quad's longest
        // the rows' shifts travel to shared memory while the sums run
        const uint32_t shb = smem_u32(&s.shv[warp][0][lane]);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint32_t k = 4 * q + j;
          pr[j] = k < npc ? s.piece[k] : 0u;  // none: a piece of no groups
          const int v = (int)(pr[j] & 0xFFu);
          row[j] = k < npc ? s.tv_row[v] : -1;
          pl[j] = reinterpret_cast<const uint4*>(s.plist + s.tv_off[v]) + ((pr[j] >> 8) & 0x3Fu);
          sl[j] = st64[pl[j][0].x];
          if (row[j] >= 0) {
            if (BF16)
              cp_async<4>(shb + 256u * j,
                          static_cast<const __nv_bfloat16*>(mv.mrow) + (size_t)row[j] * L + e0);
            else
              cp_async<8>(shb + 256u * j,
                          static_cast<const float*>(mv.mrow) + (size_t)row[j] * L + e0);
          }
          a1[j] = 0;
          a2[j] = 0;
        }
        for (uint32_t gi = 0; gi < ng; ++gi) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (gi >= ((pr[j] >> 14) & 0x1Fu)) continue;  // uniform over the warp
            const uint4 o = pl[j][gi];
            const uint64_t ya = f2_sub(st64[o.x], sl[j]), yb = f2_sub(st64[o.y], sl[j]);
            const uint64_t yc = f2_sub(st64[o.z], sl[j]), yd = f2_sub(st64[o.w], sl[j]);
            // the group's four terms summed as a tree, then added to the
            // voxel's running sums (chains of at most 64 additions)
            a1[j] = f2_add(a1[j], f2_add(f2_add(ya, yb), f2_add(yc, yd)));
            a2[j] = f2_add(a2[j], f2_add(f2_fma(yb, yb, f2_mul(ya, ya)),
                                         f2_fma(yd, yd, f2_mul(yc, yc))));
          }
        }
        cp_async_wait_all();
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (row[j] < 0) continue;  // uniform over the warp
          uint64_t sg;
          if (BF16) {
            const uint32_t w = (uint32_t)lds_u64(shb + 256u * j);
            const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w));
            sg = f2_pack(f.x, f.y);
          } else {
            sg = lds_u64(shb + 256u * j);
          }
          const uint64_t dl = f2_sub(sl[j], sg);
          const float nf = (float)(pr[j] >> 19);
          const uint64_t n2 = f2_pack(nf, nf);
          const float2 S1 = f2_unpack(f2_fma(n2, dl, a1[j]));
          const float2 S2 = f2_unpack(f2_fma(dl, f2_fma(n2, dl, f2_add(a1[j], a1[j])), a2[j]));
          // lane l takes elements c 64 + l and c 64 + 32 + l (held by lanes
          // l / 2 and 16 + l / 2), so that each reduction below covers 256
          // contiguous bytes
          const int h0 = (int)(lane >> 1), h1 = 16 + (int)(lane >> 1);
          const bool odd = lane & 1u;
          const float p0x = __shfl_sync(0xFFFFFFFFu, S1.x, h0);
          const float p0y = __shfl_sync(0xFFFFFFFFu, S1.y, h0);
          const float p1x = __shfl_sync(0xFFFFFFFFu, S1.x, h1);
          const float p1y = __shfl_sync(0xFFFFFFFFu, S1.y, h1);
          const float r0x = __shfl_sync(0xFFFFFFFFu, S2.x, h0);
          const float r0y = __shfl_sync(0xFFFFFFFFu, S2.y, h0);
          const float r1x = __shfl_sync(0xFFFFFFFFu, S2.x, h1);
          const float r1y = __shfl_sync(0xFFFFFFFFu, S2.y, h1);
          const float p0 = odd ? p0y : p0x, p1 = odd ? p1y : p1x;
          const float r0 = odd ? r0y : r0x, r1 = odd ? r1y : r1x;
          // exact across tiles: 64-bit integers in units of B 2^-32 (S1) and
          // B^2 2^-31 (S2); a piece adds at most 2^39 units when every
          // element lies within the bound B (anything else, NaN included,
          // raises the range status and is not added)
          const float x0 = __fmul_rn(p0, J.fx1), x1 = __fmul_rn(p1, J.fx1);
          const float y0 = __fmul_rn(r0, J.fx2), y1 = __fmul_rn(r1, J.fx2);
          const bool ok = fabsf(x0) <= 0x1p39f && fabsf(x1) <= 0x1p39f && fabsf(y0) <= 0x1p39f &&
                          fabsf(y1) <= 0x1p39f;
          if (__any_sync(0xFFFFFFFFu, !ok)) {
            if (lane == 0) raise_status(mv.ctr, kDevRange, 16);
            continue;
          }
          unsigned long long* P1 = reinterpret_cast<unsigned long long*>(
                                       J.acc.rows + (size_t)row[j] * J.acc.stride + 4) +
                                   c * kOE + lane;
          unsigned long long* P2 = P1 + L;
          red_add_u64(P1, (unsigned long long)f2ll_fast(x0));
          red_add_u64(P1 + 32, (unsigned long long)f2ll_fast(x1));
          red_add_u64(P2, (unsigned long long)f2ll_fast(y0));
          red_add_u64(P2 + 32, (unsigned long long)f2ll_fast(y1));
        }
      }
      __syncthreads();  // the stage is free again
    }
    if (abort) break;
    // 7. counts and sums of d
    if (tid < (int)ntv) {
      const int32_t row = s.tv_row[tid];
      if (row >= 0) {
        float* h = J.acc.rows + (size_t)row * J.acc.stride;
        red_add_u64(reinterpret_cast<unsigned long long*>(h),
                    (unsigned long long)(long long)s.tv_dq[tid]);
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
    const float dunit = b.job[jb].dunit;
    const float u1 = b.job[jb].u1, u2 = b.job[jb].u2;
    const bool live = *(volatile uint32_t*)&mv.ctr[kCtrStatus] == 0;
    const int64_t cnt = min((int64_t)*A.count, (int64_t)mv.row_cap);
    for (int64_t i = gw; i < cnt; i += nw) {
      const uint32_t row = A.list[i];
      float* h = A.rows + (size_t)row * A.stride;
      longlong2* P1 = reinterpret_cast<longlong2*>(h + 4);  // S1 plane
      longlong2* P2 = P1 + L / 2;                          // S2 plane
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
          // (S1, S2) of elements e .. e + 3, from their exact integer sums
          const longlong2 qa = P1[e / 2], qb = P1[e / 2 + 1];
          const longlong2 ra = P2[e / 2], rb2 = P2[e / 2 + 1];
          const float s1[4] = {__fmul_rn(ll2f_fast(qa.x), u1), __fmul_rn(ll2f_fast(qa.y), u1),
                               __fmul_rn(ll2f_fast(qb.x), u1), __fmul_rn(ll2f_fast(qb.y), u1)};
          const float s2[4] = {__fmul_rn(ll2f_fast(ra.x), u2), __fmul_rn(ll2f_fast(ra.y), u2),
                               __fmul_rn(ll2f_fast(rb2.x), u2), __fmul_rn(ll2f_fast(rb2.y), u2)};
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
          const longlong2 z = make_longlong2(0, 0);
          P1[e / 2] = z;
          P1[e / 2 + 1] = z;
          P2[e / 2] = z;
          P2[e / 2 + 1] = z;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          nrm += __shfl_xor_sync(0xFFFFFFFFu, nrm, off);
          nbf += __shfl_xor_sync(0xFFFFFFFFu, nbf, off);
        }
        if (lane == 0) {
          mv.tsdf[row] = make_float2(__fadd_rn(sw.x, __fmul_rn(ll2f_fast(dq), dunit)), Wn);
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

// Units of the accumulated S1 and S2 (the reciprocals of the tile kernel's
// scales, each rounded once).
static void open_units(const slim_map* m, OpenApplyJob& a) {
  const double B = (double)m->p.embed_bound;
  a.u1 = (float)(B / 4294967296.0);
  a.u2 = (float)(B * B / 2147483648.0);
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
  const double B = (double)m->p.embed_bound;
  J.fx1 = (float)(4294967296.0 / B);
  J.fx2 = (float)(2147483648.0 / (B * B));
  if (!open_encode_sem(&J.sem_map, sem, n, m->L, width > 0 ? 1 << J.tw_log2 : kORowPts))
    return fail(SLIM_ERR_CUDA, "cuTensorMapEncodeTiled failed for the embeddings");
  return SLIM_OK;
}

slim_status open_integrate(slim_map* m, const ScanGeom& g, const float* pts, const float* sem,
                           int64_t n, int width, cudaStream_t st) {
  if (n <= 0) return SLIM_OK;
  if (n > kOpenMaxCallPoints)
    return fail(SLIM_ERR_ARG, "open set: at most 2^23 points per map and call");
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
  a.job[0].dunit = (float)m->p.trunc * 0x1p-22f;
  open_units(m, a.job[0]);
  tok = prof_begin(m, SLIM_KERNEL_OPEN_APPLY, st);
  e = launch_open_apply(a, m->bf16, st);
  prof_end(m, tok, st);
  if (e != cudaSuccess) return fail(SLIM_ERR_CUDA, cudaGetErrorString(e));
  return SLIM_OK;
}

// Open-set items of a batch: one tile launch per storage kind and 48 items,
// then one apply launch per storage kind and 48 maps. Items of the same map
// share the map's accumulators (one observation set).
slim_status open_integrate_batch(const std::vector<OpenItem>& items, cudaStream_t st) {
  if (items.empty()) return SLIM_OK;
  std::vector<slim_map*> maps;
  std::vector<int64_t> npts;
  for (const OpenItem& it : items) {
    const size_t k = std::find(maps.begin(), maps.end(), it.map) - maps.begin();
    if (k == maps.size()) {
      maps.push_back(it.map);
      npts.push_back(0);
    }
    npts[k] += std::max<int64_t>(it.n, 0);
    if (npts[k] > kOpenMaxCallPoints)
      return fail(SLIM_ERR_ARG, "open set: at most 2^23 points per map and call");
  }
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
      a.job[a.n_jobs].dunit = (float)m->p.trunc * 0x1p-22f;
      open_units(m, a.job[a.n_jobs]);
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
