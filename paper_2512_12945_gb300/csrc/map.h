// The map handle behind the C ABI, shared by the host-side translation units.
#pragma once
#include <algorithm>
#include <string>
#include <vector>

#include "internal.h"

namespace slim {
// Record a failure message for slim_last_error() and return s.
slim_status fail(slim_status s, const std::string& msg);

// Scratch of the open-set path, sized by max_points at map creation.
struct OpenScratch {
  int64_t pair_cap = 0;          // (voxel, point) pairs per scan
  uint32_t* keys = nullptr;      // voxel key per pair (slot << 9 | local)
  uint32_t* vals = nullptr;      // pair index, permuted with the keys
  uint32_t* keys_tmp = nullptr;  // sort ping-pong buffers
  uint32_t* vals_tmp = nullptr;
  float* pair_d = nullptr;       // SDF of each pair, by pair index
  uint32_t* pair_pt = nullptr;   // point of each pair, by pair index
  float2* part = nullptr;        // per piece and side: (mean, M2) per element
  uint4* meta = nullptr;         // per piece and side: (n, sum d, flags, key)
  uint32_t* ctr = nullptr;       // device counters: pairs, runs
  void* tmp = nullptr;           // sort / scan temp
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
  float* stage_pts = nullptr;
  float* stage_sem = nullptr;
  // extract scratch
  uint64_t* ex_keys = nullptr;
  uint64_t* ex_keys_tmp = nullptr;
  uint32_t* ex_slots = nullptr;
  uint32_t* ex_slots_tmp = nullptr;
  uint32_t* ex_counts = nullptr;
  uint32_t* ex_offs = nullptr;
  void* ex_tmp = nullptr;
  uint32_t* pinned = nullptr;  // host copy of the device counters
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
slim_status open_alloc_scratch(slim_map* m, OpenScratch& o, int64_t max_points);
cudaError_t open_setup_attributes(slim_map* m);
cudaError_t query_setup_attributes();
slim_status run_render(slim_map* m, const double world_from_camera[16], float fx, float fy,
                       float cx, float cy, int32_t width, int32_t height, float near_t,
                       float far_t, const float* q, float* depth, int32_t* ijk, int32_t* label,
                       float* sim, cudaStream_t st);
slim_status run_backward(slim_map* m, const ScanGeom& g, const float* pts, const float* sem,
                         int64_t n, const float* gD, const float* gS, const float* gB,
                         float* gsem, float* gxyz, cudaStream_t st);
slim_status run_query(slim_map* m, const uint16_t* q_dev, int32_t Q, float temperature, float tp,
                      int32_t* label, float* prob, float* scores, uint32_t n_rows,
                      cudaStream_t st);
slim_status open_integrate(slim_map* m, const MapView& mv, OpenScratch& o, const ScanGeom& g,
                           const float* pts, const float* sem, int64_t n, int L, int bf16,
                           cudaStream_t st);
}  // namespace slim
