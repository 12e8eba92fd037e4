// Rasterizer kernels for 16 x 16 pixel tiles (see raster_impl.cuh).
#include "raster_impl.cuh"

namespace ss {
SS_RASTER_DISPATCH(fwd, 16, 16)
SS_RASTER_DISPATCH(bwd, 16, 16)
}  // namespace ss
