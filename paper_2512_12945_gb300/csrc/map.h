// The map handle behind the C ABI, shared by the host-side translation units.
#pragma once
#include <string>
#include <vector>

#include "internal.h"

namespace slim {
// Record a failure message for slim_last_error() and return s.
slim_status fail(slim_status s, const std::string& msg);

// Scratch of the open-set path, sized by max_points at map creation.
struct OpenScratch {
  int64_t pair_cap = 0;     // (voxel, point) pairs per scan
  uint32_t* keys = nullptr; // voxel key per pair (slot << 9 | local)
  uint32_t* vals = nullptr; // pair index -> (point << 5 | step)
  uint32_t* keys_tmp = nullptr;
  uint32_t* vals_tmp = nullptr;
  float* pair_d = nullptr;  // d per pair, by pair index
  uint32_t* npairs = nullptr;  // device counter
  uint32_t* seg_flag = nullptr;  // segment heads
  uint32_t* seg_off = nullptr;   // segment starts (scan of heads)
  void* tmp = nullptr;      // sort / scan temp
};
}  // namespace slim

struct slim_map {
  slim_map_params p;
  int device = 0;
  int K = 0, L = 0, mode = 0, bf16 = 0, rs = 0;
  int cap = 0, band_blocks = 0, tile_points = 0;
  uint32_t n_buckets = 0;
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
    for (void* p : allocs) cudaFree(p);
    allocs.clear();
    if (pinned) cudaFreeHost(pinned);
    pinned = nullptr;
  }
};


namespace slim {
slim_status open_alloc_scratch(slim_map* m, OpenScratch& o, int64_t max_points);
cudaError_t open_setup_attributes(slim_map* m);
slim_status open_integrate(slim_map* m, const MapView& mv, OpenScratch& o, const ScanGeom& g,
                           const float* pts, const float* sem, int64_t n, int L, int bf16,
                           cudaStream_t st);
}  // namespace slim
