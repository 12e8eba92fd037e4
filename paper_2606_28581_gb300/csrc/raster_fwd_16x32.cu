// Rasterizer fwd kernels for 16 x 32 pixel tiles (see raster_impl.cuh).
#include "raster_impl.cuh"

namespace ss {
SS_RASTER_FWD_DISPATCH(16, 32)
}  // namespace ss
