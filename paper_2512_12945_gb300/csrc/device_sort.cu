// Device-wide primitives: exclusive scan of uint32 counts and a stable LSD
// radix sort of (key, value) pairs with 8- or 9-bit digits (histogram per
// 4096-item tile -> scan of the [digit][tile] table -> stable scatter ranked
// with __match_any_sync inside each warp's contiguous sub-tile). A key of b
// bits takes ceil(b / 9) passes when that is fewer than ceil(b / 8) (25-bit
// open-set voxel keys: 3 passes instead of 4), the bits spread evenly.
#include "block_sort.cuh"
#include "internal.h"

namespace slim {

constexpr int kScanChunk = 4096;  // entries per CTA in the scan
constexpr int kSortItems = 16;
constexpr int kSortTile = kCtaThreads * kSortItems;  // 4096 items per CTA
constexpr int kWarpSpan = kSortTile / kCtaWarps;     // 512 items per warp

__global__ void __launch_bounds__(256) k_scan_partials(const uint32_t* __restrict__ in,
                                                       int64_t n, uint32_t* partial) {
  __shared__ uint32_t wt[kCtaWarps];
  const int64_t base = (int64_t)blockIdx.x * kScanChunk;
  uint32_t s = 0;
  for (int k = threadIdx.x; k < kScanChunk; k += kCtaThreads) {
    const int64_t i = base + k;
    if (i < n) s += in[i];
  }
  uint32_t tot;
  cta_exclusive_scan(s, wt, &tot);
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

// Exclusive scan of the per-CTA partials by one CTA (n_part small).
__global__ void __launch_bounds__(256) k_scan_top(uint32_t* partial, int64_t n_part,
                                                  uint32_t* total_out) {
  __shared__ uint32_t wt[kCtaWarps];
  uint32_t carry = 0;
  for (int64_t b = 0; b < n_part; b += kCtaThreads) {
    const int64_t i = b + threadIdx.x;
    const uint32_t v = i < n_part ? partial[i] : 0u;
    uint32_t tot;
    const uint32_t ex = cta_exclusive_scan(v, wt, &tot);
    if (i < n_part) partial[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) *total_out = carry;
}

__global__ void __launch_bounds__(256) k_scan_apply(const uint32_t* __restrict__ in, int64_t n,
                                                    const uint32_t* __restrict__ partial,
                                                    uint32_t* out) {
  __shared__ uint32_t wt[kCtaWarps];
  constexpr int kPer = kScanChunk / kCtaThreads;  // 16 consecutive entries per thread
  const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kPer;
  uint32_t v[kPer];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0u;
    s += v[k];
  }
  uint32_t tot;
  uint32_t off = cta_exclusive_scan(s, wt, &tot) + partial[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    if (base + k < n) out[base + k] = off;
    off += v[k];
  }
}

static int64_t scan_ctas(int64_t n) { return (n + kScanChunk - 1) / kScanChunk; }

cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, void* tmp,
                               cudaStream_t st) {
  if (n <= 0) return cudaMemsetAsync(out, 0, sizeof(uint32_t), st);
  const int64_t nc = scan_ctas(n);
  uint32_t* partial = static_cast<uint32_t*>(tmp);
  k_scan_partials<<<(unsigned)nc, kCtaThreads, 0, st>>>(in, n, partial);
  k_scan_top<<<1, kCtaThreads, 0, st>>>(partial, nc, out + n);
  k_scan_apply<<<(unsigned)nc, kCtaThreads, 0, st>>>(in, n, partial, out);
  return cudaGetLastError();
}

// RADIX: histogram bins (256 or 512, at least 2^nbits).
template <typename K, int RADIX>
__global__ void __launch_bounds__(256) k_digit_hist(const K* __restrict__ keys, int64_t n_max,
                                                    const uint32_t* __restrict__ n_dev, int shift,
                                                    uint32_t mask, uint32_t* hist,
                                                    int64_t ntiles) {
  __shared__ uint32_t c[RADIX];
  const int64_t n = n_dev ? min(n_max, (int64_t)*n_dev) : n_max;
  for (int d = threadIdx.x; d < RADIX; d += kCtaThreads) c[d] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll 4
  for (int k = 0; k < kSortItems; ++k) {
    const int64_t i = base + (int64_t)k * kCtaThreads + threadIdx.x;
    if (i < n) atomicAdd(&c[(uint32_t)(keys[i] >> shift) & mask], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < RADIX; d += kCtaThreads)
    hist[(int64_t)d * ntiles + blockIdx.x] = c[d];
}

template <typename K, int RADIX>
__global__ void __launch_bounds__(256) k_scatter(const K* __restrict__ kin,
                                                 const uint32_t* __restrict__ vin, K* kout,
                                                 uint32_t* vout, int64_t n_max,
                                                 const uint32_t* __restrict__ n_dev, int shift,
                                                 uint32_t mask, const uint32_t* __restrict__ offs,
                                                 int64_t ntiles) {
  __shared__ uint32_t wh[RADIX * kCtaWarps];  // [digit][warp]
  const int64_t n = n_dev ? min(n_max, (int64_t)*n_dev) : n_max;
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  const int64_t beg = (int64_t)blockIdx.x * kSortTile + (int64_t)warp * kWarpSpan;
  const int64_t end = min(n, beg + kWarpSpan);
  for (int i = threadIdx.x; i < RADIX * kCtaWarps; i += kCtaThreads) wh[i] = 0;
  __syncthreads();
  for (int64_t b = beg; b < end; b += 32) {
    const int64_t i = b + lane;
    const bool act = i < end;
    const uint32_t dig = act ? ((uint32_t)(kin[i] >> shift) & mask) : 0xFFFFFFFFu;
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, dig);
    if (act && (int)lane == __ffs(peers) - 1) wh[dig * kCtaWarps + warp] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  for (int d = threadIdx.x; d < RADIX; d += kCtaThreads) {
    uint32_t s = offs[(int64_t)d * ntiles + blockIdx.x];
#pragma unroll
    for (int w = 0; w < kCtaWarps; ++w) {
      const uint32_t t = wh[d * kCtaWarps + w];
      wh[d * kCtaWarps + w] = s;
      s += t;
    }
  }
  __syncthreads();
  for (int64_t b = beg; b < end; b += 32) {
    const int64_t i = b + lane;
    const bool act = i < end;
    K key = 0;
    uint32_t val = 0;
    if (act) {
      key = kin[i];
      val = vin[i];
    }
    const uint32_t dig = act ? ((uint32_t)(key >> shift) & mask) : 0xFFFFFFFFu;
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, dig);
    if (act) {
      const uint32_t pos = wh[dig * kCtaWarps + warp] + __popc(peers & ((1u << lane) - 1u));
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncwarp();
    if (act && (int)lane == __ffs(peers) - 1) wh[dig * kCtaWarps + warp] += __popc(peers);
    __syncwarp();
  }
}

constexpr int kMaxRadix = 512;

size_t radix_sort_temp_bytes(int64_t n) {
  const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
  const int64_t nh = kMaxRadix * ntiles;
  // hist + scanned hist (+1) + scan partials
  return (size_t)(2 * nh + 1 + scan_ctas(nh) + 64) * sizeof(uint32_t);
}

// kres / vres non-null: the result stays in whichever buffer pair the last
// pass wrote (returned there); otherwise it is copied back into keys / vals.
template <typename K>
static cudaError_t radix_sort_impl(K* keys, uint32_t* vals, K* ktmp, uint32_t* vtmp, void* tmp,
                                   int64_t n, const uint32_t* n_dev, int bits,
                                   cudaStream_t st, K** kres = nullptr,
                                   uint32_t** vres = nullptr) {
  if (kres) *kres = keys;
  if (vres) *vres = vals;
  if (n <= 1) return cudaSuccess;
  const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
  // the [digit][tile] tables are laid out for the largest radix; a pass of
  // `radix` bins uses the first radix * ntiles entries
  uint32_t* hist = static_cast<uint32_t*>(tmp);
  uint32_t* offs = hist + kMaxRadix * ntiles;
  uint32_t* partial = offs + kMaxRadix * ntiles + 1;
  K* ka = keys;
  K* kb = ktmp;
  uint32_t* va = vals;
  uint32_t* vb = vtmp;
  // passes of at most 9 bits when that saves a pass over 8-bit digits
  int npass = (bits + 7) / 8;
  if ((bits + 8) / 9 < npass) npass = (bits + 8) / 9;
  int passes = 0;
  for (int shift = 0; passes < npass; ++passes) {
    const int width = (bits - shift + (npass - passes) - 1) / (npass - passes);
    const uint32_t mask = (1u << width) - 1u;
    const int radix = width > 8 ? 512 : 256;
    const int64_t nh = (int64_t)radix * ntiles;
    if (radix == 512)
      k_digit_hist<K, 512><<<(unsigned)ntiles, kCtaThreads, 0, st>>>(ka, n, n_dev, shift, mask,
                                                                     hist, ntiles);
    else
      k_digit_hist<K, 256><<<(unsigned)ntiles, kCtaThreads, 0, st>>>(ka, n, n_dev, shift, mask,
                                                                     hist, ntiles);
    cudaError_t e = exclusive_scan_u32(hist, offs, nh, partial, st);
    if (e != cudaSuccess) return e;
    if (radix == 512)
      k_scatter<K, 512><<<(unsigned)ntiles, kCtaThreads, 0, st>>>(ka, va, kb, vb, n, n_dev,
                                                                 shift, mask, offs, ntiles);
    else
      k_scatter<K, 256><<<(unsigned)ntiles, kCtaThreads, 0, st>>>(ka, va, kb, vb, n, n_dev,
                                                                 shift, mask, offs, ntiles);
    shift += width;
    K* t = ka;
    ka = kb;
    kb = t;
    uint32_t* tv = va;
    va = vb;
    vb = tv;
  }
  if (kres && vres) {
    *kres = ka;
    *vres = va;
  } else if (passes & 1) {  // the result is in the tmp buffers: copy back (bounded by n_max)
    cudaMemcpyAsync(keys, ka, n * sizeof(K), cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
  }
  return cudaGetLastError();
}

cudaError_t radix_sort_u64(uint64_t* keys, uint32_t* vals, uint64_t* keys_tmp,
                           uint32_t* vals_tmp, void* tmp, int64_t n, int bits,
                           cudaStream_t st) {
  return radix_sort_impl<uint64_t>(keys, vals, keys_tmp, vals_tmp, tmp, n, nullptr, bits, st);
}

cudaError_t radix_sort_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp,
                           uint32_t* vals_tmp, void* tmp, int64_t n, int bits,
                           cudaStream_t st) {
  return radix_sort_impl<uint32_t>(keys, vals, keys_tmp, vals_tmp, tmp, n, nullptr, bits, st);
}

cudaError_t radix_sort_u32_devn(uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp,
                                uint32_t* vals_tmp, void* tmp, int64_t n_max,
                                const uint32_t* n_dev, int bits, cudaStream_t st,
                                uint32_t** keys_out, uint32_t** vals_out) {
  return radix_sort_impl<uint32_t>(keys, vals, keys_tmp, vals_tmp, tmp, n_max, n_dev, bits, st,
                                   keys_out, vals_out);
}

}  // namespace slim
