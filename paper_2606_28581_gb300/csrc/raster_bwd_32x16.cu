// Rasterizer bwd kernels for 32 x 16 pixel tiles (see raster_impl.cuh).
#include "raster_impl.cuh"

namespace ss {
SS_RASTER_BWD_DISPATCH(32, 16)
}  // namespace ss
