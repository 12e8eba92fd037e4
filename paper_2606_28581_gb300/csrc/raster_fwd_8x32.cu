// Rasterizer fwd kernels for 8 x 32 pixel tiles (see raster_impl.cuh).
#include "raster_impl.cuh"

namespace ss {
SS_RASTER_FWD_DISPATCH(8, 32)
}  // namespace ss
