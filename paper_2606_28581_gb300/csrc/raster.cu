// Dispatch of the rasterizer launches by tile shape (kernels in raster_<W>x<H>.cu).
#include "kernels.cuh"

namespace ss {

cudaError_t launch_raster_fwd_16x16(const RasterParams&, int, bool, int, cudaStream_t);
cudaError_t launch_raster_bwd_16x16(const RasterParams&, int, bool, int, cudaStream_t);
cudaError_t launch_raster_fwd_32x8(const RasterParams&, int, bool, int, cudaStream_t);
cudaError_t launch_raster_bwd_32x8(const RasterParams&, int, bool, int, cudaStream_t);
cudaError_t launch_raster_fwd_8x32(const RasterParams&, int, bool, int, cudaStream_t);
cudaError_t launch_raster_bwd_8x32(const RasterParams&, int, bool, int, cudaStream_t);
cudaError_t launch_raster_fwd_32x16(const RasterParams&, int, bool, int, cudaStream_t);
cudaError_t launch_raster_bwd_32x16(const RasterParams&, int, bool, int, cudaStream_t);
cudaError_t launch_raster_fwd_16x32(const RasterParams&, int, bool, int, cudaStream_t);
cudaError_t launch_raster_bwd_16x32(const RasterParams&, int, bool, int, cudaStream_t);

cudaError_t launch_raster_fwd(const RasterParams& p, int tile_w, int tile_h, int batch, bool persistent, int num_sms,
                              cudaStream_t st) {
  if (tile_w == 16 && tile_h == 16) return launch_raster_fwd_16x16(p, batch, persistent, num_sms, st);
  if (tile_w == 32 && tile_h == 8) return launch_raster_fwd_32x8(p, batch, persistent, num_sms, st);
  if (tile_w == 8 && tile_h == 32) return launch_raster_fwd_8x32(p, batch, persistent, num_sms, st);
  if (tile_w == 32 && tile_h == 16) return launch_raster_fwd_32x16(p, batch, persistent, num_sms, st);
  if (tile_w == 16 && tile_h == 32) return launch_raster_fwd_16x32(p, batch, persistent, num_sms, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_raster_bwd(const RasterParams& p, int tile_w, int tile_h, int batch, bool persistent, int num_sms,
                              cudaStream_t st) {
  if (tile_w == 16 && tile_h == 16) return launch_raster_bwd_16x16(p, batch, persistent, num_sms, st);
  if (tile_w == 32 && tile_h == 8) return launch_raster_bwd_32x8(p, batch, persistent, num_sms, st);
  if (tile_w == 8 && tile_h == 32) return launch_raster_bwd_8x32(p, batch, persistent, num_sms, st);
  if (tile_w == 32 && tile_h == 16) return launch_raster_bwd_32x16(p, batch, persistent, num_sms, st);
  if (tile_w == 16 && tile_h == 32) return launch_raster_bwd_16x32(p, batch, persistent, num_sms, st);
  return cudaErrorInvalidValue;
}

}  // namespace ss
