// The map handle behind the C ABI, shared by the host-side translation units.
#pragma once
#include <algorithm>
#include <string>
#include <vector>

#include "internal.h"

namespace slim {
// Words of a map's pinned host block: the device counters and, at
// kNumCounters, the pair total read back by slim_record_pairs.
constexpr int kPinnedWords = kNumCounters + 8;
// Record a failure message for slim_last_error() and return s.
slim_status fail(slim_status s, const std::string& msg);

// Scratch of the open-set path: per-row accumulators of one integration
// call and the list of the rows it touched.
struct OpenScratch {
  OpenAcc acc{};
  int32_t tw_log2 = 4;  // tile width of organized frames: 16 x 16 pixels (slim_autotune)
};
// Scratch of the open-set query.
struct QueryScratch {
  void* abf = nullptr;     // FP32 storage: BF16 copy of the means [row_cap x L]
  float* rnorm2 = nullptr; // FP32 storage: |m|^2 of the BF16 copy [row_cap]
  float* qinv = nullptr;   // [256] 1 / |q|
};
}  // namespace slim

struct slim_map {
  slim_map_params p;
  int device = 0;
  int K = 0, L = 0, mode = 0, bf16 = 0, rs = 0;
  int cap = 0, band_blocks = 0, tile_points = 0;
  int hash_tile = 256;  // threads (points) per CTA of the hash-aggregation kernel
  bool direct = false;  // closed one-hot: direct per-pair reductions instead of hash tiles
  int32_t* render_bounds = nullptr;  // slim_render: block bounding box (6 ints)

  uint64_t n_entries = 0;
  slim::MapView mv{};
  std::vector<void*> allocs;
  size_t bytes = 0;
  // slim_integrate_host: two device staging buffers, filled on the map's own
  // copy stream while the previous call's integration runs
  float* stage_pts[2] = {nullptr, nullptr};
  float* stage_sem[2] = {nullptr, nullptr};
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t stage_copied[2] = {nullptr, nullptr};
  cudaEvent_t stage_free[2] = {nullptr, nullptr};
  int stage_next = 0;
  // extract scratch
  uint64_t* ex_keys = nullptr;
  uint64_t* ex_keys_tmp = nullptr;
  uint32_t* ex_slots = nullptr;
  uint32_t* ex_slots_tmp = nullptr;
  uint32_t* ex_counts = nullptr;
  uint32_t* ex_offs = nullptr;
  void* ex_tmp = nullptr;
  uint32_t* pinned = nullptr;  // host copy of the device counters, then spare words
  // slim_record_pairs scratch (allocated by its first call)
  uint32_t* pr_counts = nullptr;  // [max_points] pairs per point
  uint32_t* pr_tmp = nullptr;     // scan partials
  slim::OpenScratch open{};
  slim::QueryScratch qscratch{};
  // kernel timing (slim_profile_enable)
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_ev;  // pairs: [2k] start, [2k+1] end
  std::vector<int> prof_kind;
  size_t prof_used = 0;
  int64_t scans = 0;

  template <class T>
  slim_status alloc(T** out, size_t count) {
    void* p = nullptr;
    const size_t b = count * sizeof(T);
    if (b == 0) {
      *out = nullptr;
      return SLIM_OK;
    }
    cudaError_t e = cudaMalloc(&p, b);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return slim::fail(SLIM_ERR_NOMEM, "cudaMalloc of " + std::to_string(b) + " bytes failed: " +
                                      cudaGetErrorString(e));
    }
    allocs.push_back(p);
    bytes += b;
    *out = static_cast<T*>(p);
    return SLIM_OK;
  }
  void release() {
    for (cudaEvent_t e : prof_ev) cudaEventDestroy(e);
    prof_ev.clear();
    for (int k = 0; k < 2; ++k) {
      if (stage_copied[k]) cudaEventDestroy(stage_copied[k]);
      if (stage_free[k]) cudaEventDestroy(stage_free[k]);
      stage_copied[k] = stage_free[k] = nullptr;
    }
    if (copy_stream) cudaStreamDestroy(copy_stream);
    copy_stream = nullptr;
    for (void* p : allocs) cudaFree(p);
    allocs.clear();
    if (pinned) cudaFreeHost(pinned);
    pinned = nullptr;
  }
};


namespace slim {
// Bracket one kernel launch with timing events when profiling is on.
// prof_begin returns a token for prof_end (-1 when off).
int prof_begin(slim_map* m, int kind, cudaStream_t st);
void prof_end(slim_map* m, int token, cudaStream_t st);
slim_status open_alloc_scratch(slim_map* m, OpenScratch& o);
cudaError_t open_setup_attributes();
cudaError_t query_setup_attributes();
slim_status run_render(slim_map* m, const double world_from_camera[16], float fx, float fy,
                       float cx, float cy, int32_t width, int32_t height, float near_t,
                       float far_t, const float* q, float* depth, int32_t* ijk, int32_t* label,
                       float* sim, cudaStream_t st);
slim_status run_backward(slim_map* m, const ScanGeom& g, const float* pts, const float* sem,
                         int64_t n, const float* gD, const float* gS, const float* gB,
                         float* gsem, float* gxyz, cudaStream_t st);
slim_status run_record_pairs(slim_map* m, const ScanGeom& g, const float* pts, int64_t n,
                             uint32_t* offsets, uint32_t* vox, int64_t cap, int64_t* n_pairs,
                             cudaStream_t st);
slim_status run_backward_pairs(slim_map* m, const ScanGeom& g, const float* pts, int64_t n,
                               const uint32_t* offsets, const uint32_t* vox, const float* gD,
                               const float* gS, float* gsem, float* gxyz, cudaStream_t st);
slim_status run_query(slim_map* m, const uint16_t* q_dev, int32_t Q, float temperature, float tp,
                      int32_t* label, float* prob, float* scores, uint32_t n_rows,
                      cudaStream_t st);
// Integrate one scan (or z-depth frame, g.depth set) of an open-set map:
// width = pixels per image row of an organized frame, 0 for unorganized
// points.
slim_status open_integrate(slim_map* m, const ScanGeom& g, const float* pts, const float* sem,
                           int64_t n, int width, cudaStream_t st);
// One open-set item of a batched integration.
struct OpenItem {
  slim_map* map;
  ScanGeom g;
  const float* pts;
  const float* sem;
  int64_t n;
  int width;
};
slim_status open_integrate_batch(const std::vector<OpenItem>& items, cudaStream_t st);
}  // namespace slim
