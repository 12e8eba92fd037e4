// Rasterizer kernels for 32 x 8 pixel tiles (see raster_impl.cuh).
#include "raster_impl.cuh"

namespace ss {
SS_RASTER_DISPATCH(fwd, 32, 8)
SS_RASTER_DISPATCH(bwd, 32, 8)
}  // namespace ss
