// Open-set read-out (end of Sec. III-D, Fig. "sit"): cosine similarity of
// every voxel's NIG mean m against Q query embeddings, softmax over the
// queries of cos / T, most probable query kept when its probability reaches
// T_p. The scores are one dense contraction S = M Q^T (voxels x l times
// l x queries), run on the 5th-generation tensor cores:
//
//   warp 0      one thread issues TMA loads (128B swizzle) of a 128 x 64 tile
//               of M and the N x 64 tile of the queries per stage into a
//               4-stage shared-memory ring;
//   warp 1      one thread issues tcgen05.mma (kind::f16, BF16 in, FP32
//               accumulate, M = 128, N = queries rounded up to 16) into one of
//               two TMEM accumulators, and tcgen05.commit frees each stage;
//   warps 2-9   epilogue, two warps per TMEM lane quarter (one voxel row per
//               thread): each takes every other 32-column chunk of the
//               accumulator (tcgen05.ld), cosine = dot / (|m| |q|), online
//               softmax in base 2 with the chunk's maximum and sum taken by
//               trees, argmax; the odd-chunk warp hands its (max, sum,
//               argmax) to the even-chunk warp through shared memory, which
//               combines them, applies the threshold and writes the row.
//   warps 10-11 (caller-held rows) row norms |m|^2 from the A stages in
//               shared memory, 64 rows each, handed to the epilogue per
//               accumulator.
//
// The grid is persistent (one CTA per SM, tiles strided over CTAs). Every
// mbarrier wait is bounded: running out raises the map status, the CTA stops
// issuing work, waits (bounded) for its own copies and MMAs and frees TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <mutex>

#include "map.h"
#include "tma.cuh"

namespace slim {

constexpr int kQM = 128;        // voxel rows per tile
constexpr int kQK = 64;         // K elements per stage (128-byte rows)
constexpr int kQStages = 4;
constexpr int kQThreads = 384;  // 12 warps: TMA, MMA, 8 epilogue, 2 row norms

struct QueryArgs {
  uint32_t n_rows;
  int32_t L;
  int32_t Q;
  int32_t N;         // Q rounded up to 16
  uint32_t tmem_cols;
  float inv_temp;
  float temp_log2e;     // T / log2(e): turns a base-2 logit back into a cosine
  float tp;
  const float* qinv;    // [Q] 1 / |q|
  const float* rnorm2;  // [n_rows] |m|^2, or null when fuse_norms
  int32_t fuse_norms;   // compute |m|^2 from the A tiles in shared memory
  int32_t* label;
  float* prob;
  float* scores;        // [n_rows x Q] cosines or null
  uint32_t* status;     // map counters (sticky status)
};

// K-major operand, 128-byte swizzle: rows of 128 B, 8-row atoms 1024 B apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset: next 8-row atom
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)2 << 61;             // 128-byte swizzle
  return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 32 consecutive accumulator columns of this thread's TMEM lane; the values
// may be used only after tmem_wait_ld().
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Online softmax over one chunk of W accumulator columns [c0, c0 + W) of a
// row: acc * colscale[c] * rowscale are base-2 logits (cos / T times
// log2 e); columns >= Q are ignored. The chunk's maximum (with the lowest
// index among ties) is found by a tree on acc * colscale[c] (the row scale
// is positive), then its W exponentials are independent, so the chain per
// chunk is short.
template <int W>
__device__ __forceinline__ void softmax_chunk(const uint32_t (&r)[W], int c0, int Q,
                                              const float* colscale, float rowscale, float* scores,
                                              float cosscale, float& mrun, float& srun, int& best) {
  // y = acc |q|^-1 log2(e) / T: the row's base-2 logits divided by its
  // positive row scale |m|^-1, so y orders the columns as the logits do; the
  // row scale enters once, in the exponent's FMA
  float y[W];
  const float4* cs4 = reinterpret_cast<const float4*>(colscale + c0);  // c0 % 16 == 0
#pragma unroll
  for (int j4 = 0; j4 < W / 4; ++j4) {
    const float4 cv = cs4[j4];
    y[4 * j4 + 0] = __uint_as_float(r[4 * j4 + 0]) * cv.x;
    y[4 * j4 + 1] = __uint_as_float(r[4 * j4 + 1]) * cv.y;
    y[4 * j4 + 2] = __uint_as_float(r[4 * j4 + 2]) * cv.z;
    y[4 * j4 + 3] = __uint_as_float(r[4 * j4 + 3]) * cv.w;
  }
  if (c0 + W > Q) {  // the chunk holds padding columns (uniform over the warp)
#pragma unroll
    for (int j = 0; j < W; ++j)
      if (c0 + j >= Q) y[j] = -INFINITY;
  }
  if (scores) {
#pragma unroll
    for (int j = 0; j < W; ++j)
      if (c0 + j < Q) scores[c0 + j] = y[j] * cosscale;
  }
  float mx[W];
  int bi[W];
#pragma unroll
  for (int j = 0; j < W; ++j) {
    mx[j] = y[j];
    bi[j] = c0 + j;
  }
#pragma unroll
  for (int w = W / 2; w > 0; w >>= 1) {
#pragma unroll
    for (int j = 0; j < w; ++j) {
      const bool take = mx[j + w] > mx[j];  // ties keep the lower index
      bi[j] = take ? bi[j + w] : bi[j];
      mx[j] = take ? mx[j + w] : mx[j];
    }
  }
  const float mc = mx[0] * rowscale;
  const float mnew = fmaxf(mrun, mc);
  if (mc > mrun) best = bi[0];
  float e[W];
#pragma unroll
  for (int j = 0; j < W; ++j) e[j] = ex2_approx(__fmaf_rn(y[j], rowscale, -mnew));
#pragma unroll
  for (int w = W / 2; w > 0; w >>= 1) {
#pragma unroll
    for (int j = 0; j < w; ++j) e[j] += e[j + w];
  }
  srun = srun * ex2_approx(mrun - mnew) + e[0];
  mrun = mnew;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(kQThreads, 1)
    k_query(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
            QueryArgs a) {
  extern __shared__ unsigned char q_smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(q_smem_raw) + 1023) & ~(uintptr_t)1023);
  const uint32_t bytesA = kQM * 128;
  const uint32_t bytesB = (uint32_t)a.N * 128;
  unsigned char* sA = sm;
  unsigned char* sB = sA + kQStages * bytesA;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + kQStages * bytesB);
  uint64_t* full = bars;
  uint64_t* empty = bars + kQStages;
  uint64_t* tfull = bars + 2 * kQStages;
  uint64_t* tempty = bars + 2 * kQStages + 2;
  uint64_t* hdone = bars + 2 * kQStages + 4;  // [quarter][accumulator]: odd half handed over
  uint64_t* nready = bars + 2 * kQStages + 12;  // [accumulator]: the tile's row norms written
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kQStages + 14);
  volatile uint32_t* abort_flag = tmem_slot + 1;
  float* s_qinv = reinterpret_cast<float*>(tmem_slot + 4);
  float* part_m = s_qinv + 256;  // [accumulator][128 rows]: odd half's running max
  float* part_s = part_m + 256;  //                          running sum
  int* part_b = reinterpret_cast<int*>(part_s + 256);  //   argmax
  float* rn = reinterpret_cast<float*>(part_b + 256);   // [accumulator][128 rows] |m|^2

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t num_tiles = (a.n_rows + kQM - 1) / kQM;
  const int kchunks = a.L / kQK;

  // per query column: 1 / |q| * log2(e) / T (the scores output divides the
  // log2(e) / T factor back out)
  for (int c = threadIdx.x; c < a.N; c += kQThreads)
    s_qinv[c] = c < a.Q ? a.qinv[c] * (a.inv_temp * 1.4426950408889634f) : 0.f;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kQStages; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), a.fuse_norms ? 3 : 1);  // MMA commit (+ 2 norm warps)
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(smem_u32(&tfull[s]), 1);
      mbar_init(smem_u32(&tempty[s]), 8);
    }
    for (int s = 0; s < 8; ++s) mbar_init(smem_u32(&hdone[s]), 1);
    for (int s = 0; s < 2; ++s) mbar_init(smem_u32(&nready[s]), 2);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ producer
    int stage = 0;
    uint32_t phase = 0;
    uint32_t issued = 0;
    int last_stage[kQStages];
    uint32_t last_phase[kQStages];
    for (uint32_t tile = blockIdx.x; tile < num_tiles && !*abort_flag; tile += gridDim.x) {
      for (int kc = 0; kc < kchunks; ++kc) {
        if (!mbar_wait(smem_u32(&empty[stage]), phase ^ 1)) {
          *abort_flag = 1;
          raise_status(a.status, kDevTimeout, 20);
          break;
        }
        const uint32_t fb = smem_u32(&full[stage]);
        mbar_expect_tx(fb, bytesA + bytesB);
        tma_load_2d(smem_u32(sA + stage * bytesA), &tmA, kc * kQK, (int32_t)(tile * kQM), fb);
        tma_load_2d(smem_u32(sB + stage * bytesB), &tmB, kc * kQK, 0, fb);
        last_stage[issued % kQStages] = stage;
        last_phase[issued % kQStages] = phase;
        ++issued;
        if (++stage == kQStages) {
          stage = 0;
          phase ^= 1;
        }
      }
    }
    // every issued copy has landed before the CTA may exit
    const uint32_t tail = issued < (uint32_t)kQStages ? issued : (uint32_t)kQStages;
    for (uint32_t i = 0; i < tail; ++i) {
      const uint32_t k = (issued - 1 - i) % kQStages;
      mbar_wait(smem_u32(&full[last_stage[k]]), last_phase[k]);
    }
  } else if (warp == 1 && lane == 0) {
    // ----------------------------------------------------------------- MMA
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(a.N >> 3) << 17) |
                           ((uint32_t)(kQM >> 4) << 24);
    int stage = 0;
    uint32_t phase = 0;
    int acc = 0;
    uint32_t acc_phase = 0;
    bool committed_any = false;
    uint32_t last_commit_bar = 0, last_commit_phase = 0;
    for (uint32_t tile = blockIdx.x; tile < num_tiles && !*abort_flag; tile += gridDim.x) {
      if (!mbar_wait(smem_u32(&tempty[acc]), acc_phase ^ 1)) {
        *abort_flag = 1;
        raise_status(a.status, kDevTimeout, 21);
        break;
      }
      tc_fence_after();
      const uint32_t d_tmem = tmem_base + (uint32_t)(acc * a.N);
      bool ok = true;
      for (int kc = 0; kc < kchunks; ++kc) {
        if (!mbar_wait(smem_u32(&full[stage]), phase)) {
          *abort_flag = 1;
          raise_status(a.status, kDevTimeout, 22);
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a0 = smem_u32(sA + stage * bytesA);
        const uint32_t b0 = smem_u32(sB + stage * bytesB);
#pragma unroll
        for (int k = 0; k < kQK / 16; ++k)
          mma_bf16(d_tmem, sw128_desc(a0 + k * 32), sw128_desc(b0 + k * 32), idesc,
                   (kc > 0 || k > 0) ? 1u : 0u);
        mma_commit(smem_u32(&empty[stage]));
        if (++stage == kQStages) {
          stage = 0;
          phase ^= 1;
        }
      }
      if (!ok) break;
      mma_commit(smem_u32(&tfull[acc]));
      committed_any = true;
      last_commit_bar = smem_u32(&tfull[acc]);
      last_commit_phase = acc_phase;
      if (++acc == 2) {
        acc = 0;
        acc_phase ^= 1;
      }
    }
    // the MMAs must be complete before TMEM is freed
    if (committed_any) mbar_wait(last_commit_bar, last_commit_phase);
  } else if (warp >= 10) {
    // ---------------------------------------------------------- row norms
    // |m|^2 of each row from the A stages the MMA consumes: a 128-byte
    // swizzled row keeps its 16-byte chunks within the row, so a row's sum
    // of squares is the sum over its 128 bytes. Warp 10 + h takes rows
    // [64 h, 64 h + 64); lane l reads chunk l % 8 of rows 64 h + 4 i + l / 8
    // (one warp load covers 4 whole rows: no bank conflicts); the stage is
    // released after the read (the empty barrier counts both norm warps and
    // the MMA commit).
    const int rbase = (warp - 10) * 64;
    if (a.fuse_norms) {
      int stage = 0;
      uint32_t phase = 0;
      int acc = 0;
      uint32_t acc_phase = 0;
      for (uint32_t tile = blockIdx.x; tile < num_tiles; tile += gridDim.x) {
        float part[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) part[i] = 0.f;
        bool ok = true;
        for (int kc = 0; kc < kchunks; ++kc) {
          ok = mbar_wait(smem_u32(&full[stage]), phase);
          ok = __all_sync(0xFFFFFFFFu, ok);
          if (!ok) break;
          const unsigned char* sa =
              sA + stage * bytesA + (rbase + (lane >> 3)) * 128 + (lane & 7) * 16;
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const uint4 v = *reinterpret_cast<const uint4*>(sa + i * 4 * 128);
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[h]));
              part[i] += f.x * f.x + f.y * f.y;
            }
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&empty[stage]));
          if (++stage == kQStages) {
            stage = 0;
            phase ^= 1;
          }
        }
        // the epilogue has read the norms of tile - 2 before releasing acc
        if (ok) ok = __all_sync(0xFFFFFFFFu, mbar_wait(smem_u32(&tempty[acc]), acc_phase ^ 1));
        if (!ok) {
          if (lane == 0) {
            *abort_flag = 1;
            raise_status(a.status, kDevTimeout, 25);
          }
          break;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          part[i] += __shfl_xor_sync(0xFFFFFFFFu, part[i], 1);
          part[i] += __shfl_xor_sync(0xFFFFFFFFu, part[i], 2);
          part[i] += __shfl_xor_sync(0xFFFFFFFFu, part[i], 4);
        }
        if ((lane & 7) == 0)
#pragma unroll
          for (int i = 0; i < 16; ++i) rn[acc * kQM + rbase + 4 * i + (lane >> 3)] = part[i];
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&nready[acc]));
        if (++acc == 2) {
          acc = 0;
          acc_phase ^= 1;
        }
      }
    }
  } else if (warp >= 2) {
    // ------------------------------------------------------------ epilogue
    const int quarter = warp & 3;      // the TMEM lane quarter this warp may read
    const int half = (warp - 2) >> 2;  // 0: even 32-column chunks, 1: odd ones
    const int rl = quarter * 32 + lane;
    int acc = 0;
    uint32_t acc_phase = 0;
    for (uint32_t tile = blockIdx.x; tile < num_tiles; tile += gridDim.x) {
      bool ok = mbar_wait(smem_u32(&tfull[acc]), acc_phase);
      if (ok && a.fuse_norms) ok = mbar_wait(smem_u32(&nready[acc]), acc_phase);
      ok = __all_sync(0xFFFFFFFFu, ok);
      if (!ok) {
        if (lane == 0) {
          *abort_flag = 1;
          raise_status(a.status, kDevTimeout, 23);
        }
        break;
      }
      tc_fence_after();
      const uint32_t row = tile * kQM + rl;
      const uint32_t taddr = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * a.N);
      const float n2 = a.fuse_norms ? rn[acc * kQM + rl] : (row < a.n_rows ? a.rnorm2[row] : 0.f);
      const float rinv = n2 > 0.f ? rsqrtf(n2) : 0.f;
      float* srow = (a.scores && row < a.n_rows) ? a.scores + (size_t)row * a.Q : nullptr;
      // base-2 logits: colscale = |q|^-1 log2(e) / T, rowscale = |m|^-1
      float mrun = -INFINITY, srun = 0.f;
      int best = -1;
      // full 32-column chunks of this half, the next one's TMEM load in
      // flight while the current one is reduced; then the 16-wide tail
      const int nfull = a.N / 32;
      int ch = half;
      if (ch < nfull) {
        uint32_t ra[32], rb[32];
        tmem_ld32_async(taddr + (uint32_t)(ch * 32), ra);
        tmem_wait_ld();
        for (;;) {
          const int nx = ch + 2;
          if (nx < nfull) tmem_ld32_async(taddr + (uint32_t)(nx * 32), rb);
          softmax_chunk<32>(ra, ch * 32, a.Q, s_qinv, rinv, srow, rinv * a.temp_log2e, mrun,
                            srun, best);
          if (nx >= nfull) break;
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 32; ++j) ra[j] = rb[j];
          ch = nx;
        }
        ch += 2;
      }
      if (ch == nfull && nfull * 32 < a.N) {  // N is a multiple of 16
        uint32_t r[16];
        tmem_ld16(taddr + (uint32_t)(nfull * 32), r);
        softmax_chunk<16>(r, nfull * 32, a.Q, s_qinv, rinv, srow, rinv * a.temp_log2e, mrun,
                          srun, best);
      }
      const uint32_t hbar = smem_u32(&hdone[quarter * 2 + acc]);
      if (half == 1) {
        part_m[acc * kQM + rl] = mrun;
        part_s[acc * kQM + rl] = srun;
        part_b[acc * kQM + rl] = best;
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(smem_u32(&tempty[acc]));
          mbar_arrive(hbar);
        }
      } else {
        bool ok2 = mbar_wait(hbar, acc_phase);
        ok2 = __all_sync(0xFFFFFFFFu, ok2);
        if (ok2) {
          // combine with the odd half: lowest index among equal maxima
          const float m1 = part_m[acc * kQM + rl], s1 = part_s[acc * kQM + rl];
          const int b1 = part_b[acc * kQM + rl];
          const float m = fmaxf(mrun, m1);
          srun = srun * ex2_approx(mrun - m) + s1 * ex2_approx(m1 - m);
          if (m1 > mrun || (m1 == mrun && b1 >= 0 && b1 < best)) best = b1;
          mrun = m;
        }
        // the shared partials are read: the accumulator and this slot of
        // the hand-over may be reused
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&tempty[acc]));
        if (!ok2) {
          if (lane == 0) {
            *abort_flag = 1;
            raise_status(a.status, kDevTimeout, 24);
          }
          break;
        }
        if (row < a.n_rows) {
          if (n2 > 0.f) {
            const float p = 1.f / srun;
            a.prob[row] = p;
            a.label[row] = p >= a.tp ? best : -1;
          } else {
            a.prob[row] = 0.f;
            a.label[row] = -1;
          }
        }
      }
      if (++acc == 2) {
        acc = 0;
        acc_phase ^= 1;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(a.tmem_cols)
                 : "memory");
  }
}

// 1 / |q| per query (bf16 rows of length L).
__global__ void k_query_norms(const __nv_bfloat16* __restrict__ q, int Q, int L, float* qinv) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= Q) return;
  float s = 0.f;
  for (int k = lane; k < L; k += 32) {
    const float v = __bfloat162float(q[(size_t)warp * L + k]);
    s += v * v;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, off);
  if (lane == 0) qinv[warp] = s > 0.f ? rsqrtf(s) : 0.f;
}

// |m|^2 of each BF16 row (one warp per row).
__global__ void k_row_norms_bf16(const __nv_bfloat16* __restrict__ rows, float* norm2,
                                 uint32_t n_rows, int L) {
  const uint32_t row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n_rows) return;
  float s = 0.f;
  for (int e = 2 * lane; e < L; e += 64) {
    const float2 v =
        __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(rows + (size_t)row * L + e));
    s += v.x * v.x + v.y * v.y;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, off);
  if (lane == 0) norm2[row] = s;
}

static bool encode_2d(CUtensorMap* m, const void* base, uint64_t inner, uint64_t rows,
                      uint32_t box_inner, uint32_t box_rows) {
  auto fn = get_encode();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {inner * 2};
  cuuint32_t box[2] = {box_inner, box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides,
                  box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

size_t query_smem_bytes(int N) {
  return 1024 + (size_t)kQStages * (kQM * 128 + (size_t)N * 128) + (2 * kQStages + 14) * 8 + 16 +
         256 * 4 + 3 * 256 * 4 + 256 * 4;
}

cudaError_t query_setup_attributes() {
  return cudaFuncSetAttribute(k_query, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)query_smem_bytes(256));
}

slim_status run_query(slim_map* m, const uint16_t* q_dev, int32_t Q, float temperature, float tp,
                      int32_t* label, float* prob, float* scores, uint32_t n_rows,
                      cudaStream_t st) {
  if (n_rows == 0) return SLIM_OK;
  const int L = m->L;
  const int N = (Q + 15) / 16 * 16;
  uint32_t cols = 32;
  while (cols < (uint32_t)(2 * N)) cols <<= 1;
  const void* A = m->mv.mrow;
  const float* rn2 = m->mv.mnorm2;
  int tok = prof_begin(m, SLIM_KERNEL_QUERY, st);
  if (!m->bf16) {  // FP32 storage: the BF16 copy the update kernel keeps
    A = m->qscratch.abf;
    rn2 = m->qscratch.rnorm2;
  }
  k_query_norms<<<(Q * 32 + 255) / 256, 256, 0, st>>>(
      reinterpret_cast<const __nv_bfloat16*>(q_dev), Q, L, m->qscratch.qinv);
  CUtensorMap tA, tB;
  if (!encode_2d(&tA, A, (uint64_t)L, n_rows, kQK, kQM) ||
      !encode_2d(&tB, q_dev, (uint64_t)L, (uint64_t)Q, kQK, (uint32_t)N))
    return fail(SLIM_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  QueryArgs a;
  a.n_rows = n_rows;
  a.L = L;
  a.Q = Q;
  a.N = N;
  a.tmem_cols = cols;
  a.inv_temp = 1.f / temperature;
  a.temp_log2e = temperature / 1.4426950408889634f;
  a.tp = tp;
  a.qinv = m->qscratch.qinv;
  a.rnorm2 = rn2;
  a.fuse_norms = 0;
  a.label = label;
  a.prob = prob;
  a.scores = scores;
  a.status = m->mv.ctr;
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device);
  const uint32_t tiles = (n_rows + kQM - 1) / kQM;
  const unsigned grid = (unsigned)std::min<uint32_t>(tiles, (uint32_t)sms);
  k_query<<<grid, kQThreads, query_smem_bytes(N), st>>>(tA, tB, a);
  prof_end(m, tok, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(SLIM_ERR_CUDA, cudaGetErrorString(e));
  return SLIM_OK;
}

// ---------------------------------------------------------------------------
// Read-out for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all: plug-ins whose host
// application owns every device allocation, real-time loops whose memory
// budget is fixed up front, or host programs that only hand in buffers they
// already own. slim_query_rows_static serves them: its working memory is the
// file-scope array below, which exists on every GPU that loads this library
// for as long as the process lives. It holds the inverse norms of at most
// kStaticQueries queries and the status words of the call (the row norms are
// computed inside k_query from the A tiles, so no per-row storage is needed).
// kStaticQueryRows is a per-call maximum of the interface, not a size of the
// array.
// ---------------------------------------------------------------------------
constexpr uint32_t kStaticQueryRows = 1u << 20;  // rows per call
constexpr uint32_t kStaticQueries = 256;
constexpr size_t kStaticWords = kStaticQueries + kNumCounters;
static __device__ __align__(256) float g_static_query_scratch[kStaticWords];

namespace {
std::mutex g_static_mu;
void* g_static_ptr[128] = {};  // device address of the scratch, per device
bool g_static_ready[128] = {};
}  // namespace

// Per-device set-up (once, with that device current): the device address of
// the static scratch and the shared-memory opt-in of the query kernel.
static slim_status static_query_setup(int dev, float** scratch) {
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (dev < 0 || dev >= 128) return fail(SLIM_ERR_ARG, "device ordinal out of range");
  if (!g_static_ready[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_query_scratch);
    if (e != cudaSuccess)
      return fail(SLIM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    e = query_setup_attributes();
    if (e != cudaSuccess)
      return fail(SLIM_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    g_static_ptr[dev] = p;
    g_static_ready[dev] = true;
  }
  *scratch = static_cast<float*>(g_static_ptr[dev]);
  return SLIM_OK;
}

}  // namespace slim

extern "C" slim_status slim_query_rows_static(const uint16_t* rows_dev, int64_t n_rows,
                                              int32_t l, const uint16_t* q_dev, int32_t q,
                                              float temperature, float tp, int32_t* label_dev,
                                              float* prob_dev, void* stream) {
  using namespace slim;
  if (n_rows < 0 || (uint64_t)n_rows > kStaticQueryRows)
    return fail(SLIM_ERR_ARG, "n_rows must be in [0, 2^20]: the static scratch holds the norms "
                              "of at most 1048576 rows per call");
  if (l < 64 || l > 1024 || l % 64) return fail(SLIM_ERR_ARG, "l must be a multiple of 64 in [64, 1024]");
  if (q < 1 || q > (int32_t)kStaticQueries) return fail(SLIM_ERR_ARG, "q must be in [1, 256]");
  if (!(temperature > 0.f) || !std::isfinite(temperature))
    return fail(SLIM_ERR_ARG, "temperature must be finite and > 0");
  if (n_rows > 0 && (!rows_dev || !label_dev || !prob_dev))
    return fail(SLIM_ERR_ARG, "rows, label and prob must be non-NULL");
  if (!q_dev || (reinterpret_cast<uintptr_t>(q_dev) & 15) || (reinterpret_cast<uintptr_t>(rows_dev) & 15))
    return fail(SLIM_ERR_ARG, "rows and queries must be non-NULL and 16-byte aligned");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(SLIM_ERR_CUDA, cudaGetErrorString(e));
  float* scratch = nullptr;
  slim_status s = static_query_setup(dev, &scratch);
  if (s != SLIM_OK) return s;
  if (n_rows == 0) return SLIM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  float* qinv = scratch;
  uint32_t* status = reinterpret_cast<uint32_t*>(scratch + kStaticQueries);
  // the status words must start at zero; the norms are overwritten below
  e = cudaMemsetAsync(status, 0, kNumCounters * sizeof(uint32_t), st);
  if (e != cudaSuccess) return fail(SLIM_ERR_CUDA, cudaGetErrorString(e));
  const uint32_t rows = (uint32_t)n_rows;
  k_query_norms<<<(q * 32 + 255) / 256, 256, 0, st>>>(
      reinterpret_cast<const __nv_bfloat16*>(q_dev), q, l, qinv);
  const int N = (q + 15) / 16 * 16;
  uint32_t cols = 32;
  while (cols < (uint32_t)(2 * N)) cols <<= 1;
  CUtensorMap tA, tB;
  if (!encode_2d(&tA, rows_dev, (uint64_t)l, rows, kQK, kQM) ||
      !encode_2d(&tB, q_dev, (uint64_t)l, (uint64_t)q, kQK, (uint32_t)N))
    return fail(SLIM_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  QueryArgs a;
  a.n_rows = rows;
  a.L = l;
  a.Q = q;
  a.N = N;
  a.tmem_cols = cols;
  a.inv_temp = 1.f / temperature;
  a.temp_log2e = temperature / 1.4426950408889634f;
  a.tp = tp;
  a.qinv = qinv;
  a.rnorm2 = nullptr;  // the row norms are computed inside the kernel
  a.fuse_norms = 1;
  a.label = label_dev;
  a.prob = prob_dev;
  a.scores = nullptr;
  a.status = status;
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint32_t tiles = (rows + kQM - 1) / kQM;
  const unsigned grid = (unsigned)std::min<uint32_t>(tiles, (uint32_t)sms);
  k_query<<<grid, kQThreads, query_smem_bytes(N), st>>>(tA, tB, a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(SLIM_ERR_CUDA, cudaGetErrorString(e));
  // a bounded wait inside k_query that ran out leaves its code in the status
  // word: read it back (into pageable host memory: nothing to allocate)
  uint32_t code = 0;
  e = cudaMemcpyAsync(&code, status + kCtrStatus, sizeof(code), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(SLIM_ERR_CUDA, cudaGetErrorString(e));
  if (code != 0)
    return fail((slim_status)code, code == kDevTimeout
                                       ? "a bounded wait in the query kernel ran out"
                                       : "the query kernel raised a device fault");
  return SLIM_OK;
}
