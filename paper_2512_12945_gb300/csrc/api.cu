// C ABI of the scan-integration library (declared in include/slim_gb300.h).
// Host side only: argument checks, FP64 pose composition, device memory of
// each map, and the launch sequence of every entry point.
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

namespace {

int sem_width(const slim_map* m) { return m->mode == SLIM_OPEN ? m->L : m->K; }

void compose_pose(const double pose[16], const double ext[16], ScanGeom& g, float v, float tau,
                  float rmin, float rmax, int cap) {
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
  if (p->mode < 0 || p->mode > 2) return fail(SLIM_ERR_ARG, "mode must be 0, 1 or 2");
  if (p->mode != SLIM_OPEN && (p->num_classes < 1 || p->num_classes > 64))
    return fail(SLIM_ERR_ARG, "num_classes must be in [1, 64]");
  if (p->mode == SLIM_OPEN) {
    if (p->embed_dim < 64 || p->embed_dim > 1024 || p->embed_dim % 64)
      return fail(SLIM_ERR_ARG, "embed_dim must be a multiple of 64 in [64, 1024]");
    if (p->embed_storage != SLIM_STORE_F32 && p->embed_storage != SLIM_STORE_BF16)
      return fail(SLIM_ERR_ARG, "embed_storage must be 0 (f32) or 1 (bf16)");
    if (p->voxel_capacity < 1 || p->voxel_capacity > (int64_t)0x7FFFFFFF)
      return fail(SLIM_ERR_ARG, "voxel_capacity must be in [1, 2^31)");
  }
  if (!(p->alpha0 >= 0.0) || !std::isfinite(p->alpha0))
    return fail(SLIM_ERR_ARG, "alpha0 must be finite and >= 0");
  if (!finite_pose(p->body_from_sensor)) return fail(SLIM_ERR_ARG, "extrinsic not finite");
  if (p->block_capacity < 1 || p->block_capacity > (int64_t)(1u << 23))
    return fail(SLIM_ERR_ARG, "block_capacity must be in [1, 2^23]");
  if (p->hash_capacity < 32 || p->hash_capacity > ((int64_t)1 << 32))
    return fail(SLIM_ERR_ARG, "hash_capacity must be in [32, 2^32]");
  if (p->max_points < 0 || p->max_points > ((int64_t)1 << 31))
    return fail(SLIM_ERR_ARG, "max_points must be in [0, 2^31]");
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
  m->rs = ((2 + m->K) + 3) / 4 * 4;
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
  m->n_buckets = (uint32_t)next_pow2((uint64_t)((p->hash_capacity + 31) / 32));
  const uint64_t nh = (uint64_t)m->n_buckets * kBucket;
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
  mv.bucket_mask = m->n_buckets - 1;
  mv.max_probe = (int32_t)std::min<uint64_t>(m->n_buckets, 64);
  mv.block_cap = (uint32_t)bc;
  mv.rs = m->rs;
  if (m->mode != SLIM_OPEN) {
    if ((s = m->alloc(&mv.rec, bc * kBlockVoxels * (uint64_t)m->rs)) != SLIM_OK) return bail(s);
  } else {
    const uint64_t rc = (uint64_t)p->voxel_capacity;
    const size_t esz = m->bf16 ? 2 : 4;
    unsigned char* mr = nullptr;
    unsigned char* br = nullptr;
    if ((s = m->alloc(&mv.vox_row, bc * kBlockVoxels)) != SLIM_OK) return bail(s);
    if ((s = m->alloc(&mv.tsdf, rc)) != SLIM_OK) return bail(s);
    if ((s = m->alloc(&mr, rc * m->L * esz)) != SLIM_OK) return bail(s);
    if ((s = m->alloc(&br, rc * m->L * esz)) != SLIM_OK) return bail(s);
    mv.mrow = mr;
    mv.brow = br;
    mv.row_cap = (uint32_t)rc;
    if ((s = open_alloc_scratch(m, m->open, p->max_points)) != SLIM_OK) return bail(s);
  }
  const int64_t mp = std::max<int64_t>(p->max_points, 1);
  if ((s = m->alloc(&m->stage_pts, (size_t)mp * 3)) != SLIM_OK) return bail(s);
  if ((s = m->alloc(&m->stage_sem, (size_t)mp * sem_width(m))) != SLIM_OK) return bail(s);
  if ((s = m->alloc(&m->ex_keys, bc)) != SLIM_OK) return bail(s);
  if ((s = m->alloc(&m->ex_keys_tmp, bc)) != SLIM_OK) return bail(s);
  if ((s = m->alloc(&m->ex_slots, bc)) != SLIM_OK) return bail(s);
  if ((s = m->alloc(&m->ex_slots_tmp, bc)) != SLIM_OK) return bail(s);
  if ((s = m->alloc(&m->ex_counts, bc)) != SLIM_OK) return bail(s);
  if ((s = m->alloc(&m->ex_offs, bc + 1)) != SLIM_OK) return bail(s);
  unsigned char* tmp = nullptr;
  if ((s = m->alloc(&tmp, radix_sort_temp_bytes((int64_t)bc))) != SLIM_OK) return bail(s);
  m->ex_tmp = tmp;
  if (cudaMallocHost(&m->pinned, kNumCounters * sizeof(uint32_t)) != cudaSuccess) {
    cudaGetLastError();
    m->pinned = nullptr;
    return bail(fail(SLIM_ERR_NOMEM, "cudaMallocHost failed"));
  }
  std::memset(m->pinned, 0, kNumCounters * sizeof(uint32_t));
  cudaError_t e = cudaSuccess;
  if (m->mode != SLIM_OPEN) e = closed_setup_attributes(m->mode, m->K, m->tile_points);
  else e = open_setup_attributes(m);
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

slim_status slim_map_reset(slim_map* m, void* stream) {
  if (!m) return fail(SLIM_ERR_ARG, "map is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nh = (size_t)m->n_buckets * kBucket;
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
  cudaStream_t st = (cudaStream_t)stream;
  ScanGeom g;
  compose_pose(pose_host, m->p.body_from_sensor, g, m->p.voxel_size, m->p.trunc,
               m->p.min_range, m->p.max_range, m->cap);
  m->scans++;
  if (n == 0) return SLIM_OK;
  const float* sem = static_cast<const float*>(sem_dev);
  SLIM_CUDA(launch_traverse_alloc(m->mv, g, pts_dev, n, m->mode == SLIM_OPEN, st));
  if (m->mode != SLIM_OPEN) {
    SLIM_CUDA(launch_fuse_closed(m->mv, g, pts_dev, sem, n, m->mode, m->K, m->tile_points, st));
    return SLIM_OK;
  }
  return open_integrate(m, m->mv, m->open, g, pts_dev, sem, n, m->L, m->bf16, st);
}

slim_status slim_integrate_host(slim_map* m, const float* pts_host, int64_t n,
                                const double pose_host[16], const void* sem_host,
                                void* stream) {
  if (!m) return fail(SLIM_ERR_ARG, "map is NULL");
  if (n < 0 || n > m->p.max_points) return fail(SLIM_ERR_ARG, "n must be in [0, max_points]");
  if (n > 0 && (!pts_host || !sem_host)) return fail(SLIM_ERR_ARG, "pts/sem NULL with n > 0");
  cudaStream_t st = (cudaStream_t)stream;
  if (n > 0) {
    SLIM_CUDA(cudaMemcpyAsync(m->stage_pts, pts_host, (size_t)n * 3 * sizeof(float),
                              cudaMemcpyHostToDevice, st));
    SLIM_CUDA(cudaMemcpyAsync(m->stage_sem, sem_host, (size_t)n * sem_width(m) * sizeof(float),
                              cudaMemcpyHostToDevice, st));
  }
  return slim_integrate(m, m->stage_pts, n, pose_host, m->stage_sem, stream);
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

slim_status slim_extract_tsdf(slim_map* m, int32_t* ijk_dev, float* D_dev, float* W_dev,
                              float* sem_dev, float* beta_dev, int32_t* index_dev, int64_t cap,
                              int64_t* n_out, int32_t flags, void* stream) {
  if (!m || !n_out) return fail(SLIM_ERR_ARG, "map or n_out is NULL");
  if (cap < 0) return fail(SLIM_ERR_ARG, "cap must be >= 0");
  cudaStream_t st = (cudaStream_t)stream;
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
  uint32_t total = 0;
  SLIM_CUDA(cudaMemcpyAsync(m->pinned + kCtrAux + 1, m->ex_offs + nb, sizeof(uint32_t),
                            cudaMemcpyDeviceToHost, st));
  SLIM_CUDA(cudaStreamSynchronize(st));
  total = m->pinned[kCtrAux + 1];
  *n_out = total;
  if (cap == 0) return SLIM_OK;
  if (cap < (int64_t)total) return fail(SLIM_ERR_CAPACITY, "cap smaller than the voxel count");
  ExtractArgs a;
  a.ijk = ijk_dev;
  a.D = D_dev;
  a.W = W_dev;
  a.sem = sem_dev;
  a.beta = open ? beta_dev : nullptr;
  a.index = index_dev;
  a.flags = flags;
  a.mode = m->mode;
  a.K = m->K;
  a.L = m->L;
  a.bf16 = m->bf16;
  a.alpha0 = (float)m->p.alpha0;
  SLIM_CUDA(launch_extract_write(m->mv, m->ex_slots, m->ex_keys, nb, m->ex_offs, a, st));
  SLIM_CUDA(cudaStreamSynchronize(st));
  return SLIM_OK;
}

}  // extern "C"

extern "C" {

slim_status slim_query(slim_map* m, const uint16_t*, int32_t, float, float, int32_t*, float*,
                       float*, void*) {
  if (!m) return fail(SLIM_ERR_ARG, "map is NULL");
  return fail(SLIM_ERR_UNSUPPORTED, "query not built yet");
}

slim_status slim_backward(slim_map* m, const float*, int64_t, const double*, const void*,
                          const float*, const float*, const float*, float*, float*, void*) {
  if (!m) return fail(SLIM_ERR_ARG, "map is NULL");
  return fail(SLIM_ERR_UNSUPPORTED, "backward not built yet");
}

slim_status slim_integrate_batch(const slim_batch_item* items, int32_t n_items, void*) {
  if (!items && n_items) return fail(SLIM_ERR_ARG, "items is NULL");
  return fail(SLIM_ERR_UNSUPPORTED, "batched integration not built yet");
}

}  // extern "C"
