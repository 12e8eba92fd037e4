// Rasterizer bwd kernels for 16 x 16 pixel tiles (see raster_impl.cuh).
#include "raster_impl.cuh"

namespace ss {
SS_RASTER_BWD_DISPATCH(16, 16)
}  // namespace ss
