// Rasterizer kernels for 8 x 32 pixel tiles (see raster_impl.cuh).
#include "raster_impl.cuh"

namespace ss {
SS_RASTER_DISPATCH(fwd, 8, 32)
SS_RASTER_DISPATCH(bwd, 8, 32)
}  // namespace ss
