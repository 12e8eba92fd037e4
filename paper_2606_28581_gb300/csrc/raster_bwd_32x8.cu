// Rasterizer bwd kernels for 32 x 8 pixel tiles (see raster_impl.cuh).
#include "raster_impl.cuh"

namespace ss {
SS_RASTER_BWD_DISPATCH(32, 8)
}  // namespace ss
