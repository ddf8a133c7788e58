// C ABI of the scan-integration library (declared in include/slim_gb300.h).
// Host side only: argument checks, FP64 pose composition, device memory of
// each map, and the launch sequence of every entry point.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "map.h"

using namespace slim;

namespace slim {
thread_local std::string g_err = "no error";

slim_status fail(slim_status s, const std::string& msg) {
  g_err = msg;
  return s;
}
}  // namespace slim

namespace {

slim_status cuda_fail(cudaError_t e, const char* where) {
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  return SLIM_ERR_CUDA;
}

#define SLIM_CUDA(call)                                   \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
  } while (0)

uint64_t next_pow2(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}
}  // namespace

namespace slim {
int prof_begin(slim_map* m, int kind, cudaStream_t st) {
  if (!m->prof_on) return -1;
  const size_t k = m->prof_used;
  if (2 * k + 1 >= m->prof_ev.size()) {
    for (int i = 0; i < 2; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      m->prof_ev.push_back(e);
    }
    m->prof_kind.push_back(kind);
  }
  m->prof_kind[k] = kind;
  m->prof_used = k + 1;
  cudaEventRecord(m->prof_ev[2 * k], st);
  return (int)k;
}

void prof_end(slim_map* m, int token, cudaStream_t st) {
  if (token >= 0) cudaEventRecord(m->prof_ev[2 * token + 1], st);
}
}  // namespace slim

namespace {

int sem_width(const slim_map* m) { return m->mode == SLIM_OPEN ? m->L : m->K; }

void compose_pose(const double pose[16], const double ext[16], ScanGeom& g, float v, float tau,
                  float rmin, float rmax, int cap, int weighting, float weight_eps) {
  double M[16];
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      double s = 0.0;
      for (int k = 0; k < 4; ++k) s += pose[r * 4 + k] * ext[k * 4 + c];
      M[r * 4 + c] = s;
    }
  for (int a = 0; a < 3; ++a) {
    for (int b = 0; b < 3; ++b) g.R[a * 3 + b] = (float)M[a * 4 + b];
    g.t[a] = (float)M[a * 4 + 3];
  }
  g.v = v;
  g.tau = tau;
  g.rmin = rmin;
  g.rmax = rmax;
  volatile float lim = 524288.0f * v;  // float product, as in the geometry spec
  g.lim = lim;
  g.cap = cap;
  g.scan_no = 0;
  g.depth = nullptr;
  g.dw = 0;
  g.fx = g.fy = 1.f;
  g.cx = g.cy = 0.f;
  g.weighting = weighting;
  g.weight_eps = weight_eps;
}

bool finite_pose(const double* p) {
  for (int k = 0; k < 16; ++k)
    if (!std::isfinite(p[k])) return false;
  return true;
}

slim_status read_counters(slim_map* m, cudaStream_t st) {
  SLIM_CUDA(cudaMemcpyAsync(m->pinned, m->mv.ctr, kNumCounters * sizeof(uint32_t),
                            cudaMemcpyDeviceToHost, st));
  SLIM_CUDA(cudaStreamSynchronize(st));
  return SLIM_OK;
}

slim_status status_of(uint32_t s) {
  if (s == 0) return SLIM_OK;
  const char* what = s == kDevCapacity ? "device capacity exhausted (blocks, voxels or hash)"
                     : s == kDevTimeout ? "a bounded device wait ran out"
                     : s == kDevRange   ? "an embedding element beyond the map's embed_bound"
                                        : "device consistency check failed";
  g_err = std::string("sticky map status: ") + what;
  return (slim_status)s;
}

slim_status check_params(const slim_map_params* p) {
  if (!p) return fail(SLIM_ERR_ARG, "params is NULL");
  if (!(p->voxel_size > 0.f) || !std::isfinite(p->voxel_size))
    return fail(SLIM_ERR_ARG, "voxel_size must be finite and > 0");
  if (!(p->trunc > 0.f) || !(p->trunc <= 4.f * p->voxel_size))
    return fail(SLIM_ERR_ARG, "trunc must be in (0, 4 * voxel_size]");
  if (!(p->min_range >= 0.f) || !(p->max_range > p->min_range))
    return fail(SLIM_ERR_ARG, "need 0 <= min_range < max_range");
  if (p->mode < 0 || p->mode > 3) return fail(SLIM_ERR_ARG, "mode must be 0, 1, 2 or 3");
  if (p->mode != SLIM_OPEN && (p->num_classes < 1 || p->num_classes > 64))
    return fail(SLIM_ERR_ARG, "num_classes must be in [1, 64]");
  if (p->mode == SLIM_OPEN) {
    if (p->embed_dim < 64 || p->embed_dim > 1024 || p->embed_dim % 64)
      return fail(SLIM_ERR_ARG, "embed_dim must be a multiple of 64 in [64, 1024]");
    if (p->embed_storage != SLIM_STORE_F32 && p->embed_storage != SLIM_STORE_BF16)
      return fail(SLIM_ERR_ARG, "embed_storage must be 0 (f32) or 1 (bf16)");
    if (p->voxel_capacity < 1 || p->voxel_capacity > (int64_t)0x7FFFFFFF)
      return fail(SLIM_ERR_ARG, "voxel_capacity must be in [1, 2^31)");
    if (!(p->embed_bound >= 0x1p-16f && p->embed_bound <= 0x1p16f))
      return fail(SLIM_ERR_ARG, "embed_bound must be in [2^-16, 2^16]");
  }
  if (!(p->alpha0 >= 0.0) || !std::isfinite(p->alpha0))
    return fail(SLIM_ERR_ARG, "alpha0 must be finite and >= 0");
  if (!finite_pose(p->body_from_sensor)) return fail(SLIM_ERR_ARG, "extrinsic not finite");
  if (p->block_capacity < 1 || p->block_capacity >= (int64_t)(1u << 23))
    return fail(SLIM_ERR_ARG, "block_capacity must be in [1, 2^23)");
  if (p->hash_capacity < 32 || p->hash_capacity > ((int64_t)1 << 32))
    return fail(SLIM_ERR_ARG, "hash_capacity must be in [32, 2^32]");
  if (p->max_points < 0 || p->max_points > ((int64_t)1 << 31))
    return fail(SLIM_ERR_ARG, "max_points must be in [0, 2^31]");
  if (p->mode == SLIM_OPEN) {
    if (p->tile_points != 0 && p->tile_points != 8 && p->tile_points != 16 &&
        p->tile_points != 32)
      return fail(SLIM_ERR_ARG, "open set: tile_points (tile width) must be 0, 8, 16 or 32");
  } else if (p->tile_points != 0 && p->tile_points != 64 && p->tile_points != 128 &&
             p->tile_points != 256) {
    return fail(SLIM_ERR_ARG, "tile_points must be 0 (default), 64, 128 or 256");
  }
  if (p->aggregation < 0 || p->aggregation > 3)
    return fail(SLIM_ERR_ARG, "aggregation must be 0 (auto), 1 (sort), 2 (hash) or 3 (direct)");
  if (p->aggregation == SLIM_AGG_HASH && p->mode != SLIM_CLOSED_ONEHOT)
    return fail(SLIM_ERR_ARG, "hash aggregation serves the closed one-hot mode only");
  if (p->aggregation == SLIM_AGG_DIRECT && p->mode == SLIM_OPEN)
    return fail(SLIM_ERR_ARG, "direct aggregation serves the closed-set modes");
  if (p->mode == SLIM_CLOSED_LATEST && p->aggregation != SLIM_AGG_AUTO &&
      p->aggregation != SLIM_AGG_DIRECT)
    return fail(SLIM_ERR_ARG, "the latest-label mode uses direct reductions only");
  if (p->weighting != SLIM_WEIGHT_CONSTANT && p->weighting != SLIM_WEIGHT_LINEAR)
    return fail(SLIM_ERR_ARG, "weighting must be 0 (constant) or 1 (linear)");
  if (p->weighting == SLIM_WEIGHT_LINEAR) {
    if (p->mode == SLIM_OPEN)
      return fail(SLIM_ERR_ARG, "the linear weighting serves the closed-set modes");
    if (p->aggregation != SLIM_AGG_AUTO && p->aggregation != SLIM_AGG_DIRECT)
      return fail(SLIM_ERR_ARG, "the linear weighting uses direct reductions");
    if (!(p->weight_eps >= 0.f) || !(p->weight_eps < p->trunc))
      return fail(SLIM_ERR_ARG, "weight_eps must be in [0, trunc)");
  }
  if (p->image_width < 0 || p->image_width > 65536)
    return fail(SLIM_ERR_ARG, "image_width must be in [0, 65536]");

  return SLIM_OK;
}

}  // namespace

extern "C" {

const char* slim_last_error(void) { return g_err.c_str(); }

slim_status slim_map_params_default(slim_map_params* p) {
  if (!p) return fail(SLIM_ERR_ARG, "params is NULL");
  std::memset(p, 0, sizeof(*p));
  p->voxel_size = 0.1f;
  p->trunc = 0.3f;
  p->min_range = 0.0f;
  p->max_range = 1e30f;
  p->mode = SLIM_CLOSED_ONEHOT;
  p->num_classes = 20;
  p->embed_dim = 512;
  p->embed_storage = SLIM_STORE_F32;
  p->alpha0 = 1.0;
  for (int k = 0; k < 4; ++k) p->body_from_sensor[k * 5] = 1.0;
  p->block_capacity = 100000;
  p->hash_capacity = 262144;
  p->voxel_capacity = 1000000;
  p->max_points = 1 << 18;
  p->embed_bound = 1.0f;
  return SLIM_OK;
}

slim_status slim_map_create(const slim_map_params* p, slim_map** out) {
  if (!out) return fail(SLIM_ERR_ARG, "out is NULL");
  *out = nullptr;
  slim_status s = check_params(p);
  if (s != SLIM_OK) return s;
  slim_map* m = new slim_map();
  m->p = *p;
  SLIM_CUDA(cudaGetDevice(&m->device));
  m->mode = p->mode;
  m->K = p->mode == SLIM_OPEN ? 0 : p->num_classes;
  m->L = p->mode == SLIM_OPEN ? p->embed_dim : 0;
  m->bf16 = (p->mode == SLIM_OPEN && p->embed_storage == SLIM_STORE_BF16) ? 1 : 0;
  // record floats: one-hot {S_k, c_k} per class (FP32); soft {S, W, c_k}
  // as 64-bit fixed point (exact sums); latest {S, W, stamp}
  m->rs = p->mode == SLIM_CLOSED_ONEHOT  ? (2 * m->K + 3) / 4 * 4
          : p->mode == SLIM_CLOSED_LATEST ? 4
                                          : 2 * (2 + m->K);
  const double q = 2.0 * (double)p->trunc / (double)p->voxel_size;
  m->cap = 3 * (int)std::ceil(q) + 3;
  const int span = (int)std::ceil(q) + 2;
  const int per_axis = (span + 6) / 8 + 1;
  m->band_blocks = 1 + 3 * (per_axis - 1);
  if (m->band_blocks > max_band_blocks()) {
    delete m;
    return fail(SLIM_ERR_ARG, "trunc / voxel_size too large");
  }
  m->tile_points = closed_tile_points(m->cap, m->band_blocks);
  m->hash_tile = p->tile_points > 0 ? p->tile_points : 256;
  // soft counts: the sort tiles sum each voxel's pairs of a tile on chip
  // before their 2 + K integer reductions (AUTO); direct only on request or
  // for the weighted variant
  m->direct = p->mode == SLIM_CLOSED_LATEST || p->weighting == SLIM_WEIGHT_LINEAR ||
              (p->mode == SLIM_CLOSED_SOFT && p->aggregation == SLIM_AGG_DIRECT) ||
              (p->mode == SLIM_CLOSED_ONEHOT &&
               (p->aggregation == SLIM_AGG_DIRECT ||
                (p->aggregation == SLIM_AGG_AUTO && p->tile_points == 0)));
  m->n_entries = next_pow2((uint64_t)p->hash_capacity);
  const uint64_t nh = m->n_entries;
  const uint64_t bc = (uint64_t)p->block_capacity;

  auto bail = [&](slim_status st) {
    m->release();
    delete m;
    return st;
  };
  MapView& mv = m->mv;
  if ((s = m->alloc(&mv.hkeys, nh)) != SLIM_OK) return bail(s);
  if ((s = m->alloc(&mv.hvals, nh)) != SLIM_OK) return bail(s);
  if ((s = m->alloc(&mv.blk_key, bc)) != SLIM_OK) return bail(s);
  if ((s = m->alloc(&mv.ctr, (size_t)kNumCounters)) != SLIM_OK) return bail(s);
  if ((s = m->alloc(&m->render_bounds, (size_t)6)) != SLIM_OK) return bail(s);
  mv.entry_mask = (uint32_t)(m->n_entries - 1);
  mv.max_probe = (int32_t)std::min<uint64_t>(m->n_entries, 512);
  mv.block_cap = (uint32_t)bc;
  mv.rs = m->rs;
  mv.K = m->K;
  mv.layout = p->mode == SLIM_CLOSED_ONEHOT ? kRecSplit
              : p->mode == SLIM_CLOSED_SOFT ? kRecSoftFx
                                            : kRecLatest;
  if (m->mode != SLIM_OPEN) {
    // the pool stays zero outside the sub-blocks written since the last
    // reset (each block's touched mask names them; the reset re-zeroes
    // those), so kernels never zero a block they create
    if ((s = m->alloc(&mv.rec, bc * kBlockVoxels * (uint64_t)m->rs)) != SLIM_OK) return bail(s);
    if ((s = m->alloc(&mv.blk_mask, bc)) != SLIM_OK) return bail(s);
    if (cudaMemset(mv.rec, 0, bc * kBlockVoxels * (uint64_t)m->rs * sizeof(float)) != cudaSuccess ||
        cudaMemset(mv.blk_mask, 0, bc * sizeof(uint64_t)) != cudaSuccess)
      return bail(cuda_fail(cudaGetLastError(), "cudaMemset"));
  } else {
    const uint64_t rc = (uint64_t)p->voxel_capacity;
    const size_t esz = m->bf16 ? 2 : 4;
    unsigned char* mr = nullptr;
    unsigned char* br = nullptr;
    if ((s = m->alloc(&mv.vox_row, bc * kBlockVoxels)) != SLIM_OK) return bail(s);
    // every voxel-row table starts empty (-1); reset restores the used ones
    if (cudaMemset(mv.vox_row, 0xFF, bc * kBlockVoxels * sizeof(int32_t)) != cudaSuccess)
      return bail(cuda_fail(cudaGetLastError(), "cudaMemset"));
    if ((s = m->alloc(&mv.tsdf, rc)) != SLIM_OK) return bail(s);
    if ((s = m->alloc(&mr, rc * m->L * esz)) != SLIM_OK) return bail(s);
    if ((s = m->alloc(&br, rc * m->L * esz)) != SLIM_OK) return bail(s);
    mv.mrow = mr;
    mv.brow = br;
    mv.row_cap = (uint32_t)rc;
    if ((s = m->alloc(&mv.mnorm2, rc)) != SLIM_OK) return bail(s);
    if ((s = m->alloc(&m->qscratch.qinv, (size_t)256)) != SLIM_OK) return bail(s);
    if (!m->bf16) {
      unsigned char* abf = nullptr;
      if ((s = m->alloc(&abf, rc * m->L * 2)) != SLIM_OK) return bail(s);
      m->qscratch.abf = abf;
      if ((s = m->alloc(&m->qscratch.rnorm2, rc)) != SLIM_OK) return bail(s);
      // the update kernel keeps the BF16 copy of every mean it writes
      mv.mbf = abf;
      mv.mbf_norm2 = m->qscratch.rnorm2;
    }
    if ((s = open_alloc_scratch(m, m->open)) != SLIM_OK) return bail(s);
    m->open.tw_log2 = p->tile_points == 8 ? 3 : (p->tile_points == 32 ? 5 : 4);
  }
  const int64_t mp = std::max<int64_t>(p->max_points, 1);
  for (int k = 0; k < 2; ++k) {
    if ((s = m->alloc(&m->stage_pts[k], (size_t)mp * 3)) != SLIM_OK) return bail(s);
    if ((s = m->alloc(&m->stage_sem[k], (size_t)mp * sem_width(m))) != SLIM_OK) return bail(s);
    if (cudaEventCreateWithFlags(&m->stage_copied[k], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&m->stage_free[k], cudaEventDisableTiming) != cudaSuccess)
      return bail(cuda_fail(cudaGetLastError(), "cudaEventCreate"));
  }
  if (cudaStreamCreateWithFlags(&m->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
    return bail(cuda_fail(cudaGetLastError(), "cudaStreamCreate"));
  if ((s = m->alloc(&m->ex_keys, bc)) != SLIM_OK) return bail(s);
  if ((s = m->alloc(&m->ex_keys_tmp, bc)) != SLIM_OK) return bail(s);
  if ((s = m->alloc(&m->ex_slots, bc)) != SLIM_OK) return bail(s);
  if ((s = m->alloc(&m->ex_slots_tmp, bc)) != SLIM_OK) return bail(s);
  if ((s = m->alloc(&m->ex_counts, bc)) != SLIM_OK) return bail(s);
  if ((s = m->alloc(&m->ex_offs, bc + 1)) != SLIM_OK) return bail(s);
  unsigned char* tmp = nullptr;
  if ((s = m->alloc(&tmp, radix_sort_temp_bytes((int64_t)bc))) != SLIM_OK) return bail(s);
  m->ex_tmp = tmp;
  if (cudaMallocHost(&m->pinned, kPinnedWords * sizeof(uint32_t)) != cudaSuccess) {
    cudaGetLastError();
    m->pinned = nullptr;
    return bail(fail(SLIM_ERR_NOMEM, "cudaMallocHost failed"));
  }
  std::memset(m->pinned, 0, kPinnedWords * sizeof(uint32_t));
  if (cudaMemset(mv.ctr, 0, kNumCounters * sizeof(uint32_t)) != cudaSuccess)
    return bail(cuda_fail(cudaGetLastError(), "cudaMemset"));
  cudaError_t e = cudaSuccess;
  if (m->mode != SLIM_OPEN) e = closed_setup_attributes(m->mode, m->K, m->tile_points);
  else {
    e = open_setup_attributes();
    if (e == cudaSuccess) e = query_setup_attributes();
  }
  if (e != cudaSuccess) return bail(cuda_fail(e, "cudaFuncSetAttribute"));
  if ((s = slim_map_reset(m, nullptr)) != SLIM_OK) return bail(s);
  if (cudaDeviceSynchronize() != cudaSuccess) return bail(cuda_fail(cudaGetLastError(), "sync"));
  *out = m;
  return SLIM_OK;
}

slim_status slim_map_destroy(slim_map* m) {
  if (!m) return fail(SLIM_ERR_ARG, "map is NULL");
  cudaDeviceSynchronize();
  m->release();
  delete m;
  return SLIM_OK;
}

// Closed one-hot map integrated by direct per-pair reductions.
static bool uses_direct(const slim_map* m) {
  return m->mode != SLIM_OPEN && m->direct;
}

// Closed one-hot map integrated by the shared-memory hash tiles.
static bool uses_hash(const slim_map* m) {
  return m->mode == SLIM_CLOSED_ONEHOT && !m->direct && m->p.aggregation != SLIM_AGG_SORT;
}

slim_status slim_map_reset(slim_map* m, void* stream) {
  if (!m) return fail(SLIM_ERR_ARG, "map is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nh = (size_t)m->n_entries;
  const int tok = prof_begin(m, SLIM_KERNEL_RESET, st);
  if (m->mode != SLIM_OPEN)
    SLIM_CUDA(launch_zero_touched_blocks(m->mv.rec, m->mv.blk_mask, m->mv.ctr + kCtrBlocks,
                                         m->mv.block_cap, m->rs, st));
  else
    SLIM_CUDA(launch_reset_vox_rows(m->mv, st));
  prof_end(m, tok, st);
  SLIM_CUDA(cudaMemsetAsync(m->mv.hkeys, 0xFF, nh * sizeof(uint64_t), st));
  SLIM_CUDA(cudaMemsetAsync(m->mv.hvals, 0xFF, nh * sizeof(uint32_t), st));
  SLIM_CUDA(cudaMemsetAsync(m->mv.ctr, 0, kNumCounters * sizeof(uint32_t), st));
  m->scans = 0;
  return SLIM_OK;
}

slim_status slim_integrate(slim_map* m, const float* pts_dev, int64_t n,
                           const double pose_host[16], const void* sem_dev, void* stream) {
  if (!m) return fail(SLIM_ERR_ARG, "map is NULL");
  if (n < 0 || n > m->p.max_points) return fail(SLIM_ERR_ARG, "n must be in [0, max_points]");
  if (!pose_host || !finite_pose(pose_host)) return fail(SLIM_ERR_ARG, "pose missing or not finite");
  if (n > 0 && (!pts_dev || !sem_dev)) return fail(SLIM_ERR_ARG, "pts/sem NULL with n > 0");
  if ((reinterpret_cast<uintptr_t>(pts_dev) & 3) || (reinterpret_cast<uintptr_t>(sem_dev) & 3))
    return fail(SLIM_ERR_ARG, "pts/sem must be 4-byte aligned");
  if (m->mode == SLIM_OPEN && (reinterpret_cast<uintptr_t>(sem_dev) & 15))
    return fail(SLIM_ERR_ARG, "open-set embeddings must be 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  ScanGeom g;
  compose_pose(pose_host, m->p.body_from_sensor, g, m->p.voxel_size, m->p.trunc,
               m->p.min_range, m->p.max_range, m->cap, m->p.weighting,
               m->p.weight_eps);
  m->scans++;
  g.scan_no = (uint32_t)m->scans;
  if (n == 0) return SLIM_OK;
  const float* sem = static_cast<const float*>(sem_dev);
  if (m->mode != SLIM_OPEN) {
    const int tok = prof_begin(m, SLIM_KERNEL_FUSE_CLOSED, st);
    if (uses_direct(m))
      SLIM_CUDA(launch_fuse_direct(m->mv, g, pts_dev, sem, n, m->K,
                                   m->mode == SLIM_CLOSED_LATEST ? 1 : 0,
                                   m->mode == SLIM_CLOSED_SOFT ? 1 : 0, st));
    else if (uses_hash(m))
      SLIM_CUDA(launch_fuse_hash(m->mv, g, pts_dev, sem, n, m->K, m->hash_tile, m->band_blocks,
                                 st));
    else
      SLIM_CUDA(launch_fuse_closed(m->mv, g, pts_dev, sem, n, m->mode, m->K, m->tile_points, st));
    prof_end(m, tok, st);
    return SLIM_OK;
  }
  return open_integrate(m, g, pts_dev, sem, n, m->p.image_width, st);
}

slim_status slim_integrate_depth(slim_map* m, const float* depth_dev, int32_t width,
                                 int32_t height, float fx, float fy, float cx, float cy,
                                 const double pose_host[16], const void* sem_dev, void* stream) {
  if (!m) return fail(SLIM_ERR_ARG, "map is NULL");
  if (width < 1 || height < 1) return fail(SLIM_ERR_ARG, "width and height must be >= 1");
  const int64_t n = (int64_t)width * height;
  if (n > m->p.max_points) return fail(SLIM_ERR_ARG, "width * height must be <= max_points");
  if (!pose_host || !finite_pose(pose_host)) return fail(SLIM_ERR_ARG, "pose missing or not finite");
  if (!(fx > 0.f) || !(fy > 0.f) || !std::isfinite(fx) || !std::isfinite(fy) ||
      !std::isfinite(cx) || !std::isfinite(cy))
    return fail(SLIM_ERR_ARG, "fx, fy must be finite and > 0; cx, cy finite");
  if (!depth_dev || !sem_dev) return fail(SLIM_ERR_ARG, "depth/sem NULL");
  if ((reinterpret_cast<uintptr_t>(depth_dev) & 3) || (reinterpret_cast<uintptr_t>(sem_dev) & 3))
    return fail(SLIM_ERR_ARG, "depth/sem must be 4-byte aligned");
  if (m->mode == SLIM_OPEN && (reinterpret_cast<uintptr_t>(sem_dev) & 15))
    return fail(SLIM_ERR_ARG, "open-set embeddings must be 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  ScanGeom g;
  compose_pose(pose_host, m->p.body_from_sensor, g, m->p.voxel_size, m->p.trunc,
               m->p.min_range, m->p.max_range, m->cap, m->p.weighting,
               m->p.weight_eps);
  m->scans++;
  g.scan_no = (uint32_t)m->scans;
  g.depth = depth_dev;
  g.dw = width;
  g.fx = fx;
  g.fy = fy;
  g.cx = cx;
  g.cy = cy;
  const float* sem = static_cast<const float*>(sem_dev);
  if (m->mode != SLIM_OPEN) {
    // one-hot and latest maps take the direct kernel (the hash tiles read
    // point arrays); soft counts the sort tiles
    const int tok = prof_begin(m, SLIM_KERNEL_FUSE_CLOSED, st);
    if (m->mode == SLIM_CLOSED_SOFT && !m->direct)
      SLIM_CUDA(launch_fuse_closed(m->mv, g, nullptr, sem, n, m->mode, m->K, m->tile_points, st));
    else
      SLIM_CUDA(launch_fuse_direct(m->mv, g, nullptr, sem, n, m->K,
                                   m->mode == SLIM_CLOSED_LATEST ? 1 : 0,
                                   m->mode == SLIM_CLOSED_SOFT ? 1 : 0, st));
    prof_end(m, tok, st);
    return SLIM_OK;
  }
  return open_integrate(m, g, nullptr, sem, n, width, st);
}

slim_status slim_integrate_host(slim_map* m, const float* pts_host, int64_t n,
                                const double pose_host[16], const void* sem_host,
                                void* stream) {
  if (!m) return fail(SLIM_ERR_ARG, "map is NULL");
  if (n < 0 || n > m->p.max_points) return fail(SLIM_ERR_ARG, "n must be in [0, max_points]");
  if (n > 0 && (!pts_host || !sem_host)) return fail(SLIM_ERR_ARG, "pts/sem NULL with n > 0");
  if (!pose_host || !finite_pose(pose_host)) return fail(SLIM_ERR_ARG, "pose missing or not finite");
  cudaStream_t st = (cudaStream_t)stream;
  if (n == 0) return slim_integrate(m, nullptr, 0, pose_host, nullptr, stream);
  // staging buffer b is free once the integration that last read it (two
  // calls ago) has run; its copies go on the map's copy stream, so they
  // overlap the previous call's integration on `stream`
  const int b = m->stage_next;
  m->stage_next ^= 1;
  SLIM_CUDA(cudaStreamWaitEvent(m->copy_stream, m->stage_free[b], 0));
  SLIM_CUDA(cudaMemcpyAsync(m->stage_pts[b], pts_host, (size_t)n * 3 * sizeof(float),
                            cudaMemcpyHostToDevice, m->copy_stream));
  SLIM_CUDA(cudaMemcpyAsync(m->stage_sem[b], sem_host, (size_t)n * sem_width(m) * sizeof(float),
                            cudaMemcpyHostToDevice, m->copy_stream));
  SLIM_CUDA(cudaEventRecord(m->stage_copied[b], m->copy_stream));
  SLIM_CUDA(cudaStreamWaitEvent(st, m->stage_copied[b], 0));
  const slim_status s = slim_integrate(m, m->stage_pts[b], n, pose_host, m->stage_sem[b], stream);
  SLIM_CUDA(cudaEventRecord(m->stage_free[b], st));
  return s;
}

// Open-set maps of organized frames: time the tile shapes 8 x 32, 16 x 16
// and 32 x 8 pixels on the caller's scan (3 integration calls each after 2
// untimed ones, CUDA events) and keep the fastest.
static slim_status open_autotune(slim_map* m, const float* pts_dev, int64_t n,
                                 const double pose_host[16], const void* sem_dev,
                                 cudaStream_t st, int32_t* best_tile) {
  if (m->p.image_width <= 0) {  // unorganized points: one tiling only
    if (best_tile) *best_tile = 0;
    return SLIM_OK;
  }
  ScanGeom g;
  compose_pose(pose_host, m->p.body_from_sensor, g, m->p.voxel_size, m->p.trunc,
               m->p.min_range, m->p.max_range, m->cap, m->p.weighting, m->p.weight_eps);
  g.scan_no = 1;
  const bool prof = m->prof_on;
  m->prof_on = false;
  const int saved = m->open.tw_log2;
  cudaEvent_t e0, e1;
  SLIM_CUDA(cudaEventCreate(&e0));
  SLIM_CUDA(cudaEventCreate(&e1));
  float best_ms = 1e30f;
  int best = saved;
  slim_status s = SLIM_OK;
  for (int tw = 3; tw <= 5 && s == SLIM_OK; ++tw) {
    m->open.tw_log2 = tw;
    if ((s = slim_map_reset(m, st)) != SLIM_OK) break;
    for (int r = 0; r < 5 && s == SLIM_OK; ++r) {
      if (r == 2 && cudaEventRecord(e0, st) != cudaSuccess) s = cuda_fail(cudaGetLastError(), "event");
      if (s == SLIM_OK)
        s = open_integrate(m, g, pts_dev, static_cast<const float*>(sem_dev), n,
                           m->p.image_width, st);
    }
    if (s != SLIM_OK) break;
    cudaError_t e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      s = cuda_fail(e, "autotune");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      best = tw;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  m->prof_on = prof;
  m->open.tw_log2 = s == SLIM_OK ? best : saved;
  const slim_status r = slim_map_reset(m, st);
  if (s != SLIM_OK) return s;
  if (r != SLIM_OK) return r;
  SLIM_CUDA(cudaStreamSynchronize(st));
  if (best_tile) *best_tile = 1 << m->open.tw_log2;
  return SLIM_OK;
}

slim_status slim_autotune(slim_map* m, const float* pts_dev, int64_t n,
                          const double pose_host[16], const void* sem_dev, void* stream,
                          int32_t* best_tile) {
  if (!m) return fail(SLIM_ERR_ARG, "map is NULL");
  if (m->mode == SLIM_OPEN) {
    if (n < 1 || n > m->p.max_points) return fail(SLIM_ERR_ARG, "n must be in [1, max_points]");
    if (!pts_dev || !sem_dev || !pose_host || !finite_pose(pose_host))
      return fail(SLIM_ERR_ARG, "pts, sem or pose missing");
    if (reinterpret_cast<uintptr_t>(sem_dev) & 15)
      return fail(SLIM_ERR_ARG, "open-set embeddings must be 16-byte aligned");
    return open_autotune(m, pts_dev, n, pose_host, sem_dev, (cudaStream_t)stream, best_tile);
  }
  if (m->mode != SLIM_CLOSED_ONEHOT || m->p.aggregation == SLIM_AGG_SORT)
    return fail(SLIM_ERR_UNSUPPORTED, "autotune serves closed one-hot maps (hash or direct)");
  if (n < 1 || n > m->p.max_points) return fail(SLIM_ERR_ARG, "n must be in [1, max_points]");
  if (!pts_dev || !sem_dev || !pose_host || !finite_pose(pose_host))
    return fail(SLIM_ERR_ARG, "pts, sem or pose missing");
  cudaStream_t st = (cudaStream_t)stream;
  // candidates: 0 = direct reductions, else hash tiles of that many points
  int cand[4];
  int nc = 0;
  if (m->p.aggregation != SLIM_AGG_HASH) cand[nc++] = 0;
  if (m->p.aggregation != SLIM_AGG_DIRECT && m->p.weighting == SLIM_WEIGHT_CONSTANT) {
    cand[nc++] = 64;
    cand[nc++] = 128;
    cand[nc++] = 256;
  }
  const int saved_tile = m->hash_tile;
  const bool saved_direct = m->direct;
  // each candidate integrates 8 copies of the scan per launch: the batched
  // form in which the persistent and grid kernels run
  HashBatch b;
  b.n_jobs = 8;
  b.work = m->mv.ctr + kCtrWork;
  for (int k = 0; k < b.n_jobs; ++k) {
    compose_pose(pose_host, m->p.body_from_sensor, b.job[k].g, m->p.voxel_size, m->p.trunc,
                 m->p.min_range, m->p.max_range, m->cap, m->p.weighting,
               m->p.weight_eps);
    b.job[k].mv = m->mv;
    b.job[k].pts = pts_dev;
    b.job[k].sem = static_cast<const float*>(sem_dev);
    b.job[k].n = n;
    b.job[k].K = m->K;
    b.job[k].band_blocks = m->band_blocks;
    b.job[k].latest = 0;
    b.job[k].soft = 0;
    b.job[k].g.scan_no = 1;
  }
  const bool prof = m->prof_on;
  m->prof_on = false;
  cudaEvent_t e0, e1;
  SLIM_CUDA(cudaEventCreate(&e0));
  SLIM_CUDA(cudaEventCreate(&e1));
  float best_ms = 1e30f;
  int best = saved_direct ? 0 : saved_tile;
  slim_status s = SLIM_OK;
  for (int c = 0; c < nc && s == SLIM_OK; ++c) {
    if ((s = slim_map_reset(m, stream)) != SLIM_OK) break;
    const int tile = cand[c];
    auto launch = [&]() {
      return tile == 0 ? launch_direct_batch(b, m->p.weighting ? 3 : 0, st)
                       : launch_hash_batch(b, tile, 0, st);
    };
    cudaError_t e = cudaSuccess;
    for (int w = 0; w < 2 && e == cudaSuccess; ++w) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      s = cuda_fail(e, "autotune");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      best = tile;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  m->prof_on = prof;
  if (s == SLIM_OK) {
    m->direct = best == 0;
    if (best) m->hash_tile = best;
  } else {
    m->direct = saved_direct;
    m->hash_tile = saved_tile;
  }
  const slim_status r = slim_map_reset(m, stream);
  if (s != SLIM_OK) return s;
  if (r != SLIM_OK) return r;
  SLIM_CUDA(cudaStreamSynchronize(st));
  if (best_tile) *best_tile = m->direct ? 0 : m->hash_tile;
  return SLIM_OK;
}

slim_status slim_profile_enable(slim_map* m, int32_t on) {
  if (!m) return fail(SLIM_ERR_ARG, "map is NULL");
  m->prof_on = on != 0;
  m->prof_used = 0;
  return SLIM_OK;
}

slim_status slim_profile_read(slim_map* m, int64_t* launches, double* ms) {
  if (!m || !launches || !ms) return fail(SLIM_ERR_ARG, "map, launches or ms is NULL");
  for (int k = 0; k < SLIM_KERNEL_KINDS; ++k) {
    launches[k] = 0;
    ms[k] = 0.0;
  }
  for (size_t k = 0; k < m->prof_used; ++k) {
    SLIM_CUDA(cudaEventSynchronize(m->prof_ev[2 * k + 1]));
    float t = 0.f;
    SLIM_CUDA(cudaEventElapsedTime(&t, m->prof_ev[2 * k], m->prof_ev[2 * k + 1]));
    const int kind = m->prof_kind[k];
    launches[kind] += 1;
    ms[kind] += (double)t;
  }
  m->prof_used = 0;
  return SLIM_OK;
}

slim_status slim_map_sync(slim_map* m, void* stream) {
  if (!m) return fail(SLIM_ERR_ARG, "map is NULL");
  slim_status s = read_counters(m, (cudaStream_t)stream);
  if (s != SLIM_OK) return s;
  return status_of(m->pinned[kCtrStatus]);
}

slim_status slim_map_stats(slim_map* m, slim_stats* out, void* stream) {
  if (!m || !out) return fail(SLIM_ERR_ARG, "map or out is NULL");
  slim_status s = read_counters(m, (cudaStream_t)stream);
  if (s != SLIM_OK) return s;
  out->blocks = std::min<int64_t>(m->pinned[kCtrBlocks], m->p.block_capacity);
  out->voxels = m->mode == SLIM_OPEN ? std::min<int64_t>(m->pinned[kCtrRows], m->p.voxel_capacity)
                                     : -1;
  out->device_bytes = (int64_t)m->bytes;
  out->scans = m->scans;
  out->status = m->pinned[kCtrStatus];
  return SLIM_OK;
}

}  // extern "C"

// The shared read-out pipeline: sort the allocated blocks by key, count the
// voxels per block, scan, then write the requested outputs (a) in order.
static slim_status extract_impl(slim_map* m, ExtractArgs a, int64_t cap, int64_t* n_out,
                                cudaStream_t st) {
  slim_status s = read_counters(m, st);
  if (s != SLIM_OK) return s;
  if (m->pinned[kCtrStatus]) return status_of(m->pinned[kCtrStatus]);
  const int64_t nb = std::min<int64_t>(m->pinned[kCtrBlocks], m->p.block_capacity);
  const bool open = m->mode == SLIM_OPEN;
  SLIM_CUDA(launch_gather_keys(m->mv, nb, m->ex_keys, m->ex_slots, st));
  SLIM_CUDA(radix_sort_u64(m->ex_keys, m->ex_slots, m->ex_keys_tmp, m->ex_slots_tmp, m->ex_tmp,
                           nb, 63, st));
  SLIM_CUDA(launch_extract_count(m->mv, m->ex_slots, nb, open, m->ex_counts, st));
  SLIM_CUDA(exclusive_scan_u32(m->ex_counts, m->ex_offs, nb, m->ex_tmp, st));
  SLIM_CUDA(cudaMemcpyAsync(m->pinned + kCtrAux + 1, m->ex_offs + nb, sizeof(uint32_t),
                            cudaMemcpyDeviceToHost, st));
  SLIM_CUDA(cudaStreamSynchronize(st));
  const uint32_t total = m->pinned[kCtrAux + 1];
  *n_out = total;
  if (cap == 0) return SLIM_OK;
  if (cap < (int64_t)total) return fail(SLIM_ERR_CAPACITY, "cap smaller than the voxel count");
  a.mode = m->mode;
  a.K = m->K;
  a.L = m->L;
  a.bf16 = m->bf16;
  a.alpha0 = (float)m->p.alpha0;
  SLIM_CUDA(launch_extract_write(m->mv, m->ex_slots, m->ex_keys, nb, m->ex_offs, a, st));
  SLIM_CUDA(cudaStreamSynchronize(st));
  return SLIM_OK;
}

extern "C" {

slim_status slim_extract_tsdf(slim_map* m, int32_t* ijk_dev, float* D_dev, float* W_dev,
                              float* sem_dev, float* beta_dev, int32_t* index_dev, int64_t cap,
                              int64_t* n_out, int32_t flags, void* stream) {
  if (!m || !n_out) return fail(SLIM_ERR_ARG, "map or n_out is NULL");
  if (cap < 0) return fail(SLIM_ERR_ARG, "cap must be >= 0");
  ExtractArgs a{};
  a.ijk = ijk_dev;
  a.D = D_dev;
  a.W = W_dev;
  a.sem = sem_dev;
  a.beta = m->mode == SLIM_OPEN ? beta_dev : nullptr;
  a.index = index_dev;
  a.unc = nullptr;
  a.flags = flags;
  return extract_impl(m, a, cap, n_out, (cudaStream_t)stream);
}

slim_status slim_render(slim_map* m, const double world_from_camera[16], float fx, float fy,
                        float cx, float cy, int32_t width, int32_t height, float near_t,
                        float far_t, const float* q_dev, float* depth_dev, int32_t* ijk_dev,
                        int32_t* label_dev, float* sim_dev, void* stream) {
  if (!m) return fail(SLIM_ERR_ARG, "map is NULL");
  if (!world_from_camera || !finite_pose(world_from_camera))
    return fail(SLIM_ERR_ARG, "world_from_camera missing or not finite");
  if (width < 1 || height < 1 || width > 16384 || height > 16384)
    return fail(SLIM_ERR_ARG, "width and height must be in [1, 16384]");
  if (!(fx > 0.f) || !(fy > 0.f) || !std::isfinite(fx) || !std::isfinite(fy) ||
      !std::isfinite(cx) || !std::isfinite(cy))
    return fail(SLIM_ERR_ARG, "fx, fy must be finite and > 0; cx, cy finite");
  if (!(near_t >= 0.f) || !(far_t > near_t) || !std::isfinite(far_t))
    return fail(SLIM_ERR_ARG, "need 0 <= near_t < far_t < inf");
  if (((double)far_t - (double)near_t) / m->p.voxel_size > 1e6)
    return fail(SLIM_ERR_ARG, "far_t - near_t spans more than 10^6 voxels");
  if (!depth_dev) return fail(SLIM_ERR_ARG, "depth_dev is NULL");
  if (sim_dev && m->mode == SLIM_OPEN && !q_dev)
    return fail(SLIM_ERR_ARG, "sim_dev needs q_dev for an open-set map");
  return run_render(m, world_from_camera, fx, fy, cx, cy, width, height, near_t, far_t, q_dev,
                    depth_dev, ijk_dev, label_dev, sim_dev, (cudaStream_t)stream);
}

slim_status slim_extract_uncertainty(slim_map* m, float* unc_dev, int64_t cap, int64_t* n_out,
                                     void* stream) {
  if (!m || !n_out) return fail(SLIM_ERR_ARG, "map or n_out is NULL");
  if (cap < 0) return fail(SLIM_ERR_ARG, "cap must be >= 0");
  if (cap > 0 && !unc_dev) return fail(SLIM_ERR_ARG, "unc_dev is NULL");
  if (m->mode == SLIM_CLOSED_LATEST)
    return fail(SLIM_ERR_UNSUPPORTED, "the latest-label mode keeps no distribution");
  ExtractArgs a{};
  a.unc = unc_dev;
  return extract_impl(m, a, cap, n_out, (cudaStream_t)stream);
}

}  // extern "C"

extern "C" {

slim_status slim_query(slim_map* m, const uint16_t* q_dev, int32_t q, float temperature,
                       float tp, int32_t* label_dev, float* prob_dev, float* scores_dev,
                       void* stream) {
  if (!m) return fail(SLIM_ERR_ARG, "map is NULL");
  if (m->mode != SLIM_OPEN) return fail(SLIM_ERR_UNSUPPORTED, "query needs an open-set map");
  if (q < 1 || q > 256) return fail(SLIM_ERR_ARG, "q must be in [1, 256]");
  if (!q_dev || (reinterpret_cast<uintptr_t>(q_dev) & 15))
    return fail(SLIM_ERR_ARG, "q_dev must be non-NULL and 16-byte aligned");
  if (!(temperature > 0.f) || !std::isfinite(temperature))
    return fail(SLIM_ERR_ARG, "temperature must be finite and > 0");
  if (!label_dev || !prob_dev) return fail(SLIM_ERR_ARG, "label/prob NULL");
  cudaStream_t st = (cudaStream_t)stream;
  slim_status s = read_counters(m, st);
  if (s != SLIM_OK) return s;
  if (m->pinned[kCtrStatus]) return status_of(m->pinned[kCtrStatus]);
  const uint32_t rows = std::min<uint32_t>(m->pinned[kCtrRows], m->mv.row_cap);
  return run_query(m, q_dev, q, temperature, tp, label_dev, prob_dev, scores_dev, rows, st);
}

slim_status slim_backward(slim_map* m, const float* pts_dev, int64_t n,
                          const double pose_host[16], const void* sem_dev, const float* gD_dev,
                          const float* gS_dev, const float* gB_dev, float* gsem_dev,
                          float* gxyz_dev, void* stream) {
  if (!m) return fail(SLIM_ERR_ARG, "map is NULL");
  if (n < 0 || n > m->p.max_points) return fail(SLIM_ERR_ARG, "n must be in [0, max_points]");
  if (!pose_host || !finite_pose(pose_host)) return fail(SLIM_ERR_ARG, "pose missing or not finite");
  if (n > 0 && (!pts_dev || !sem_dev || !gD_dev || !gsem_dev || !gxyz_dev))
    return fail(SLIM_ERR_ARG, "pts, sem, gD, gsem and gxyz are required");
  if (m->mode == SLIM_CLOSED_LATEST)
    return fail(SLIM_ERR_UNSUPPORTED, "the latest-label mode has no adjoint");
  if (m->p.weighting != SLIM_WEIGHT_CONSTANT)
    return fail(SLIM_ERR_UNSUPPORTED, "the adjoint is for maps with w~ = 1");
  if (n > 0 && m->mode != SLIM_CLOSED_ONEHOT && !gS_dev)
    return fail(SLIM_ERR_ARG, "gS is required in the soft and open modes");
  ScanGeom g;
  compose_pose(pose_host, m->p.body_from_sensor, g, m->p.voxel_size, m->p.trunc,
               m->p.min_range, m->p.max_range, m->cap, m->p.weighting,
               m->p.weight_eps);
  return run_backward(m, g, pts_dev, static_cast<const float*>(sem_dev), n, gD_dev, gS_dev,
                      m->mode == SLIM_OPEN ? gB_dev : nullptr, gsem_dev, gxyz_dev,
                      (cudaStream_t)stream);
}

// Arguments shared by the stored-pair calls; returns SLIM_OK or the failure.
static slim_status check_pair_call(slim_map* m, const float* pts_dev, int64_t n,
                                   const double* pose_host) {
  if (!m) return fail(SLIM_ERR_ARG, "map is NULL");
  if (n < 0 || n > m->p.max_points) return fail(SLIM_ERR_ARG, "n must be in [0, max_points]");
  if (!pose_host || !finite_pose(pose_host)) return fail(SLIM_ERR_ARG, "pose missing or not finite");
  if (n > 0 && !pts_dev) return fail(SLIM_ERR_ARG, "pts is NULL with n > 0");
  if (m->mode != SLIM_CLOSED_ONEHOT && m->mode != SLIM_CLOSED_SOFT)
    return fail(SLIM_ERR_UNSUPPORTED, "stored pair lists serve the one-hot and soft modes");
  if (m->p.weighting != SLIM_WEIGHT_CONSTANT)
    return fail(SLIM_ERR_UNSUPPORTED, "the adjoint is for maps with w~ = 1");
  return SLIM_OK;
}

slim_status slim_record_pairs(slim_map* m, const float* pts_dev, int64_t n,
                              const double pose_host[16], uint32_t* offsets_dev,
                              uint32_t* vox_dev, int64_t cap, int64_t* n_pairs, void* stream) {
  slim_status s = check_pair_call(m, pts_dev, n, pose_host);
  if (s != SLIM_OK) return s;
  if (!offsets_dev || !n_pairs) return fail(SLIM_ERR_ARG, "offsets and n_pairs are required");
  if (cap < 0) return fail(SLIM_ERR_ARG, "cap must be >= 0");
  if (cap > 0 && !vox_dev) return fail(SLIM_ERR_ARG, "vox is NULL with cap > 0");
  ScanGeom g;
  compose_pose(pose_host, m->p.body_from_sensor, g, m->p.voxel_size, m->p.trunc,
               m->p.min_range, m->p.max_range, m->cap, m->p.weighting, m->p.weight_eps);
  return run_record_pairs(m, g, pts_dev, n, offsets_dev, vox_dev, cap, n_pairs,
                          (cudaStream_t)stream);
}

slim_status slim_backward_pairs(slim_map* m, const float* pts_dev, int64_t n,
                                const double pose_host[16], const uint32_t* offsets_dev,
                                const uint32_t* vox_dev, const float* gD_dev,
                                const float* gS_dev, float* gsem_dev, float* gxyz_dev,
                                void* stream) {
  slim_status s = check_pair_call(m, pts_dev, n, pose_host);
  if (s != SLIM_OK) return s;
  if (n > 0 && (!offsets_dev || !vox_dev || !gD_dev || !gsem_dev || !gxyz_dev))
    return fail(SLIM_ERR_ARG, "offsets, vox, gD, gsem and gxyz are required");
  if (n > 0 && m->mode == SLIM_CLOSED_SOFT && !gS_dev)
    return fail(SLIM_ERR_ARG, "gS is required in the soft mode");
  ScanGeom g;
  compose_pose(pose_host, m->p.body_from_sensor, g, m->p.voxel_size, m->p.trunc,
               m->p.min_range, m->p.max_range, m->cap, m->p.weighting, m->p.weight_eps);
  return run_backward_pairs(m, g, pts_dev, n, offsets_dev, vox_dev, gD_dev, gS_dev, gsem_dev,
                            gxyz_dev, (cudaStream_t)stream);
}

slim_status slim_integrate_batch(const slim_batch_item* items, int32_t n_items, void* stream) {
  if (n_items < 0) return fail(SLIM_ERR_ARG, "n_items must be >= 0");
  if (n_items > 0 && !items) return fail(SLIM_ERR_ARG, "items is NULL");
  for (int32_t k = 0; k < n_items; ++k) {
    const slim_batch_item& it = items[k];
    const slim_map* m = it.map;
    if (!m) return fail(SLIM_ERR_ARG, "item " + std::to_string(k) + ": map is NULL");
    if (it.n < 0 || it.n > m->p.max_points)
      return fail(SLIM_ERR_ARG, "item " + std::to_string(k) + ": n must be in [0, max_points]");
    if (!finite_pose(it.pose)) return fail(SLIM_ERR_ARG, "item " + std::to_string(k) + ": pose");
    if (it.n > 0 && (!it.pts_dev || !it.sem_dev))
      return fail(SLIM_ERR_ARG, "item " + std::to_string(k) + ": pts/sem NULL with n > 0");
    if ((reinterpret_cast<uintptr_t>(it.pts_dev) & 3) ||
        (reinterpret_cast<uintptr_t>(it.sem_dev) & (m->mode == SLIM_OPEN ? 15 : 3)))
      return fail(SLIM_ERR_ARG, "item " + std::to_string(k) + ": misaligned pts/sem");
  }
  {  // open-set maps: at most 2^23 points per map and call (checked before
     // anything is queued)
    std::vector<std::pair<const slim_map*, int64_t>> per_map;
    for (int32_t k = 0; k < n_items; ++k) {
      if (items[k].map->mode != SLIM_OPEN) continue;
      auto f = std::find_if(per_map.begin(), per_map.end(),
                            [&](const std::pair<const slim_map*, int64_t>& e) {
                              return e.first == items[k].map;
                            });
      if (f == per_map.end()) {
        per_map.emplace_back(items[k].map, 0);
        f = per_map.end() - 1;
      }
      if ((f->second += items[k].n) > ((int64_t)1 << 23))
        return fail(SLIM_ERR_ARG, "open set: at most 2^23 points per map and call");
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  // closed one-hot scans with hash aggregation share persistent launches
  HashBatch b;
  b.n_jobs = 0;
  int tile = 0;
  auto flush = [&]() -> slim_status {
    if (b.n_jobs == 0) return SLIM_OK;
    slim_map* m0 = items[0].map;
    for (int32_t k = 0; k < n_items; ++k)
      if (uses_hash(items[k].map)) {
        m0 = items[k].map;
        break;
      }
    const int tok = prof_begin(m0, SLIM_KERNEL_BATCH, st);
    cudaError_t e = launch_hash_batch(b, tile, 0, st);
    prof_end(m0, tok, st);
    b.n_jobs = 0;
    return e == cudaSuccess ? SLIM_OK : cuda_fail(e, "launch_hash_batch");
  };
  // direct-reduction maps share one grid per 64 scans, mode and weighting
  HashBatch nb[6];
  slim_map* direct0[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  for (int q = 0; q < 6; ++q) nb[q].n_jobs = 0;
  auto flush_direct = [&](int q) -> slim_status {
    if (nb[q].n_jobs == 0) return SLIM_OK;
    const int tok = prof_begin(direct0[q], SLIM_KERNEL_BATCH, st);
    cudaError_t e = launch_direct_batch(nb[q], q, st);
    prof_end(direct0[q], tok, st);
    nb[q].n_jobs = 0;
    return e == cudaSuccess ? SLIM_OK : cuda_fail(e, "launch_direct_batch");
  };
  std::vector<OpenItem> open_items;
  for (int32_t k = 0; k < n_items; ++k) {
    const slim_batch_item& it = items[k];
    slim_map* m = it.map;
    m->scans++;
    if (it.n == 0) continue;
    if (uses_direct(m)) {
      const int q = (m->mode == SLIM_CLOSED_SOFT ? 1 : (m->mode == SLIM_CLOSED_LATEST ? 2 : 0)) +
                    (m->p.weighting ? 3 : 0);
      if (!direct0[q]) direct0[q] = m;
      HashJob& J = nb[q].job[nb[q].n_jobs++];
      compose_pose(it.pose, m->p.body_from_sensor, J.g, m->p.voxel_size, m->p.trunc,
                   m->p.min_range, m->p.max_range, m->cap, m->p.weighting,
               m->p.weight_eps);
      J.g.scan_no = (uint32_t)m->scans;
      J.mv = m->mv;
      J.pts = it.pts_dev;
      J.sem = static_cast<const float*>(it.sem_dev);
      J.n = it.n;
      J.K = m->K;
      J.band_blocks = m->band_blocks;
      J.latest = m->mode == SLIM_CLOSED_LATEST ? 1 : 0;
      J.soft = m->mode == SLIM_CLOSED_SOFT ? 1 : 0;
      if (nb[q].n_jobs == kMaxHashJobs) {
        slim_status s = flush_direct(q);
        if (s != SLIM_OK) return s;
      }
    } else if (uses_hash(m)) {
      if (b.n_jobs == 0) {
        b.work = m->mv.ctr + kCtrWork;
        tile = m->hash_tile;
      }
      HashJob& J = b.job[b.n_jobs++];
      compose_pose(it.pose, m->p.body_from_sensor, J.g, m->p.voxel_size, m->p.trunc,
                   m->p.min_range, m->p.max_range, m->cap, m->p.weighting,
               m->p.weight_eps);
      J.g.scan_no = (uint32_t)m->scans;
      J.latest = 0;
      J.soft = 0;
      J.mv = m->mv;
      J.pts = it.pts_dev;
      J.sem = static_cast<const float*>(it.sem_dev);
      J.n = it.n;
      J.K = m->K;
      J.band_blocks = m->band_blocks;
      if (b.n_jobs == kMaxHashJobs) {
        slim_status s = flush();
        if (s != SLIM_OK) return s;
      }
    } else if (m->mode == SLIM_OPEN) {
      OpenItem oi;
      oi.map = m;
      compose_pose(it.pose, m->p.body_from_sensor, oi.g, m->p.voxel_size, m->p.trunc,
                   m->p.min_range, m->p.max_range, m->cap, m->p.weighting, m->p.weight_eps);
      oi.g.scan_no = (uint32_t)m->scans;
      oi.pts = it.pts_dev;
      oi.sem = static_cast<const float*>(it.sem_dev);
      oi.n = it.n;
      oi.width = m->p.image_width;
      open_items.push_back(oi);
    } else {
      m->scans--;  // counted again by slim_integrate
      slim_status s = slim_integrate(m, it.pts_dev, it.n, it.pose, it.sem_dev, stream);
      if (s != SLIM_OK) return s;
    }
  }
  for (int q = 0; q < 6; ++q) {
    slim_status s = flush_direct(q);
    if (s != SLIM_OK) return s;
  }
  slim_status s = flush();
  if (s != SLIM_OK) return s;
  return open_integrate_batch(open_items, st);
}

}  // extern "C"
