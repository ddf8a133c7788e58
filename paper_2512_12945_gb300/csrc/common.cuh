// Shared device-side definitions of the scan-integration library.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace slim {

constexpr uint64_t kEmptyKey = ~0ull;     // empty hash entry
constexpr uint32_t kNoSlot = 0xFFFFFFFFu; // hash entry without a block slot (yet)
constexpr uint32_t kFailSlot = 0xFFFFFFFEu; // block could not get a slot (capacity)
constexpr int kBlockVoxels = 512;         // 8^3 voxels per block
// Closed-set record layouts (MapView::layout).
enum RecLayout : int32_t {
  kRecLatest = 0,  // latest label: {S, W, stamp (u64)} in FP32 / u64
  kRecSplit = 1,   // one-hot: {S_0, c_0, ..., S_{K-1}, c_{K-1}} in FP32
  kRecSoftFx = 2   // soft counts: {S, W, c_0 .. c_{K-1}} as 64-bit fixed point
};
// Fixed-point unit of soft-count records: 2^-32 (metres for S, observations
// for W and the class counts). Scaling a float by 2^32 is exact, so a value
// of magnitude >= 2^-8 converts without rounding; smaller ones round to
// 2^-33 at most. Integer sums are exact and independent of their order.
constexpr float kFxScale = 4294967296.0f;

// Device counters held by each map.
enum Counter : int {
  kCtrBlocks = 0,   // allocated blocks
  kCtrRows = 1,     // open set: allocated voxel rows
  kCtrStatus = 2,   // sticky status (slim_status value of the first fault)
  kCtrAux = 3,      // diagnostic: where the first fault came from
  kCtrWork = 5,     // persistent kernels: next tile, finished CTAs (2 words)
  kNumCounters = 8
};

// Device status codes (same values as slim_status).
enum DevStatus : uint32_t {
  kDevOk = 0,
  kDevCapacity = 3,
  kDevTimeout = 4,
  kDevInternal = 7,
  kDevRange = 8
};

// Record the first device fault of a map (later faults keep the first).
__device__ __forceinline__ void raise_status(uint32_t* ctr, uint32_t code, uint32_t where) {
  if (atomicCAS(&ctr[kCtrStatus], 0u, code) == 0u) ctr[kCtrAux] = where;
}

// Everything a kernel needs to reach one map's storage.
struct MapView {
  uint64_t* hkeys;      // [n_entries] block keys
  uint32_t* hvals;      // [n_entries] block slots
  uint32_t entry_mask;  // n_entries - 1 (power of two)
  int32_t max_probe;    // entries probed before giving up
  uint64_t* blk_key;    // [block_cap] key of each allocated slot
  uint32_t block_cap;
  uint32_t* ctr;        // kNumCounters counters
  // closed set: AoS records of rs floats per voxel (layout: RecLayout).
  //   one-hot (kRecSplit): {S_0, c_0, S_1, c_1, ..., S_{K-1}, c_{K-1}, pad}
  //     with c_k the count of class k and S_k the sum of the SDF of those
  //     observations; W = sum c_k and S = W D = sum S_k at read-out.
  //   soft (kRecSoftFx): int64 {S, W, c_0 .. c_{K-1}} in units of 2^-32
  //   latest (kRecLatest): {S, W, stamp}
  float* rec;
  // closed set: per block slot, one bit per 2 x 2 x 2 sub-block whose
  // records an integration has written since the last reset (the reset
  // zeroes those records only; the rest of the pool stays zero)
  uint64_t* blk_mask;
  int32_t rs;
  int32_t K;
  int32_t layout;
  // open set
  int32_t* vox_row;     // [block_cap * 512] voxel row or -1
  float2* tsdf;         // [row_cap] (S = W*D, W)
  void* mrow;           // [row_cap * L] f32 or bf16 NIG mean
  void* brow;           // [row_cap * L] f32 or bf16 NIG beta
  float* mnorm2;        // [row_cap] |m|^2 of the stored mean (query read-out)
  void* mbf;            // FP32 storage: [row_cap * L] bf16 copy of m (query operand)
  float* mbf_norm2;     // FP32 storage: [row_cap] |bf16(m)|^2
  uint32_t row_cap;
};

// Per-scan geometry: the pose rounded once to float32 and the band.
struct ScanGeom {
  float R[9];
  float t[3];
  float v;      // voxel size
  float tau;    // truncation
  float rmin, rmax;
  float lim;    // |coordinate| bound: 2^19 voxels
  int32_t cap;  // DDA step cap: 3 * ceil(2 tau / v) + 3
  uint32_t scan_no;  // the map's scan count at this scan (latest-label stamps)
  // depth front end: when depth is set, point j is back-projected from the
  // row-major z-depth image (dw pixels per row) instead of read from pts
  const float* depth;
  int32_t dw;
  float fx, fy, cx, cy;
  // per-observation weight w~ (Sec. III-A): 0 for w~ = 1, 1 for the linear
  // decay behind the surface (closed-set maps, direct reductions)
  int32_t weighting;
  float weight_eps;
};

// w~ of an observation with SDF d under the linear decay behind the surface
// (Bylow et al., RSS 2013; d > 0 in front of the surface here): 1 for
// d >= -eps, (tau + d) / (tau - eps) below, 0 at d = -tau.
__device__ __forceinline__ float obs_weight(const ScanGeom& g, float d) {
  return d >= -g.weight_eps ? 1.f : __fdiv_rn(__fadd_rn(g.tau, d), __fsub_rn(g.tau, g.weight_eps));
}

// Block key: each block coordinate offset by 2^20 into 21 bits, x highest,
// so the numeric order of keys is the lexicographic order of (bx, by, bz).
__device__ __forceinline__ uint64_t pack_block(int32_t bx, int32_t by, int32_t bz) {
  return ((uint64_t)(uint32_t)(bx + (1 << 20)) << 42) |
         ((uint64_t)(uint32_t)(by + (1 << 20)) << 21) |
         (uint64_t)(uint32_t)(bz + (1 << 20));
}

__device__ __forceinline__ void unpack_block(uint64_t k, int32_t& bx, int32_t& by, int32_t& bz) {
  bx = (int32_t)((k >> 42) & 0x1FFFFF) - (1 << 20);
  by = (int32_t)((k >> 21) & 0x1FFFFF) - (1 << 20);
  bz = (int32_t)(k & 0x1FFFFF) - (1 << 20);
}

__device__ __forceinline__ int local_index(int32_t ix, int32_t iy, int32_t iz) {
  return ((ix & 7) * 8 + (iy & 7)) * 8 + (iz & 7);
}

// The bit of a block's touched mask for the 2 x 2 x 2 sub-block holding
// local voxel `local` (bits 6-8 x, 3-5 y, 0-2 z).
__device__ __forceinline__ uint64_t sub_bit(uint32_t local) {
  return 1ull << ((((local >> 7) & 3u) << 4) | (((local >> 4) & 3u) << 2) | ((local >> 1) & 3u));
}

// *a |= v (64-bit, no return value).
__device__ __forceinline__ void red_or_u64(uint64_t* a, uint64_t v) {
  asm volatile("red.global.or.b64 [%0], %1;" ::"l"(a), "l"(v) : "memory");
}

// Add `bits` to a block's touched mask unless `seen` (an earlier read of the
// mask) already holds them: bits are only added until the next reset, so a
// stale read costs at most a redundant reduction, and most writers of a
// block (hundreds of rays per scan) skip the same-address reduction.
__device__ __forceinline__ void mark_touched(uint64_t* mask, uint64_t bits, uint64_t seen) {
  if (bits & ~seen) red_or_u64(mask, bits);
}

// 64-bit finaliser (splitmix64 style) for bucket selection.
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x ^= x >> 31;
  x *= 0x7FB5D329728EA185ull;
  x ^= x >> 27;
  x *= 0x81DADEF4BC2DD44Dull;
  x ^= x >> 33;
  return x;
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Relaxed (non-caching, coherent at gpu scope) 32-bit load and store: for a
// slot published to readers that only use it as an address into records
// the pool already holds zeroed, so no ordering with other data is needed.
__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}


// addr[0] += a, addr[1] += b as one vector reduction (addr 8-byte aligned).
__device__ __forceinline__ void red_add_v2(float* addr, float a, float b) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(addr), "f"(a), "f"(b) : "memory");
}

// r[0..3] += (a, b, c, d) without a return value (16-byte aligned).
__device__ __forceinline__ void red_add_v4(float* r, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(r), "f"(a), "f"(b), "f"(c),
               "f"(d)
               : "memory");
}

// *a += v (64-bit integer reduction, no return value; a 8-byte aligned).
__device__ __forceinline__ void red_add_u64(unsigned long long* a, unsigned long long v) {
  asm volatile("red.global.add.u64 [%0], %1;" ::"l"(a), "l"(v) : "memory");
}

// x rounded to the nearest integer (ties to even), as int64: the same value
// as __float2ll_rn(x), from FP32 additions and 32-bit integer operations
// (the hardware 64-bit conversion runs at the FP64 rate, about 2 per clock
// per SM on this part). With M = 1.5 2^23, adding M to a float of magnitude
// below 2^22 leaves its nearest integer in the low mantissa bits; x splits
// exactly as h 2^20 + l with h = rint(x 2^-20) and |l| <= 2^19, so rint(x) =
// h 2^20 + rint(l). Values of magnitude 2^41 or more take the hardware path.
__device__ __forceinline__ long long f2ll_fast(float x) {
  if (!(fabsf(x) < 0x1p41f)) return __float2ll_rn(x);
  const float M = 12582912.0f;
  const float hs = __fadd_rn(__fmul_rn(x, 0x1p-20f), M);
  const float l = __fmaf_rn(-__fsub_rn(hs, M), 1048576.0f, x);
  const int ih = __float_as_int(hs) - 0x4B400000;
  const int il = __float_as_int(__fadd_rn(l, M)) - 0x4B400000;
  return (long long)ih * 1048576ll + (long long)il;
}

// v as float from two 32-bit conversions and one FMA: v = h 2^32 + l with l
// the signed low word (-2^31 <= l < 2^31), so values below 2^31 in
// magnitude convert exactly rounded and larger ones within about 2^-22
// relative (not always the nearest float).
__device__ __forceinline__ float ll2f_fast(long long v) {
  const int l = (int)(unsigned)v;
  const int h = (int)((v - (long long)l) >> 32);
  return __fmaf_rn(__int2float_rn(h), 4294967296.0f, __int2float_rn(l));
}

// x in fixed point of unit 2^-32 (two's complement bits).
__device__ __forceinline__ unsigned long long fx32(float x) {
  return (unsigned long long)f2ll_fast(__fmul_rn(x, kFxScale));
}
__device__ __forceinline__ float unfx32(long long q) {
  return __fmul_rn(__ll2float_rn(q), 1.0f / kFxScale);
}
__device__ __forceinline__ const long long* rec_fx(const float* r) {
  return reinterpret_cast<const long long*>(r);
}

// (S, W) of a closed-set voxel record (S = W D).
__device__ __forceinline__ float2 rec_sw(const float* r, int K, int layout) {
  if (layout == kRecSoftFx) {
    const long long* q = rec_fx(r);
    return make_float2(unfx32(q[0]), unfx32(q[1]));
  }
  if (layout == kRecLatest) return make_float2(r[0], r[1]);
  float s = 0.f, w = 0.f;
  for (int k = 0; k < K; ++k) {
    s += r[2 * k];
    w += r[2 * k + 1];
  }
  return make_float2(s, w);
}

// D = S / W of a closed-set record (0 where W = 0); soft records divide the
// exact fixed-point sums.
__device__ __forceinline__ float rec_sdf(const float* r, int K, int layout) {
  if (layout == kRecSoftFx) {
    const long long* q = rec_fx(r);
    return q[1] > 0 ? __ll2float_rn(q[0]) / __ll2float_rn(q[1]) : 0.f;
  }
  const float2 sw = rec_sw(r, K, layout);
  return sw.y > 0.f ? sw.x / sw.y : 0.f;
}

// Weight W of a closed-set voxel record.
__device__ __forceinline__ float rec_weight(const float* r, int K, int layout) {
  return rec_sw(r, K, layout).y;
}

// Count of class k (one-hot and soft records).
__device__ __forceinline__ float rec_count(const float* r, int k, int layout) {
  if (layout == kRecSoftFx) return unfx32(rec_fx(r)[2 + k]);
  return r[2 * k + 1];
}

// Sum of the class counts (soft: the exact integer sum, rounded once).
__device__ __forceinline__ float rec_count_sum(const float* r, int K, int layout) {
  if (layout == kRecSoftFx) {
    long long t = 0;
    for (int k = 0; k < K; ++k) t += rec_fx(r)[2 + k];
    return unfx32(t);
  }
  float t = 0.f;
  for (int k = 0; k < K; ++k) t += r[2 * k + 1];
  return t;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Longest time a kernel waits on another CTA before giving up (then it raises
// kDevTimeout and skips the dependent work).
constexpr uint64_t kCrossCtaWaitNs = 500ull * 1000 * 1000;

}  // namespace slim
