// Open-set scan integration (Sec. III-D): placeholder until the kernels land.
#include "map.h"

namespace slim {

slim_status open_alloc_scratch(slim_map*, OpenScratch&, int64_t) { return SLIM_OK; }

cudaError_t open_setup_attributes(slim_map*) { return cudaSuccess; }

slim_status open_integrate(slim_map*, const MapView&, OpenScratch&, const ScanGeom&,
                           const float*, const float*, int64_t, int, int, cudaStream_t) {
  return fail(SLIM_ERR_UNSUPPORTED, "open-set integration not built yet");
}

}  // namespace slim
