// Rasterizer bwd kernels for 16 x 32 pixel tiles (see raster_impl.cuh).
#include "raster_impl.cuh"

namespace ss {
SS_RASTER_BWD_DISPATCH(16, 32)
}  // namespace ss
