// Forward render of one view without any device allocation.
//
// For callers that cannot call cudaMalloc: host applications whose device memory is reserved once
// at start-up (a real-time viewer, an inference service under a fixed memory budget), or plug-ins
// that are handed a stream but no allocator.  The call synchronises its stream once, to read the
// view's intersection count.  The frame's workspace is a
// file-scope static device array of kNoAllocScratchBytes; every GPU that loads this library holds
// that much memory until the process exits.  Every call shares the array and leaves its contents
// behind; the calls below clear what has to start at zero (the status block and the per-tile
// ranges), and calls that overlap on the GPU (two streams, or two threads) race on the array.
#include <atomic>
#include <cmath>

#include "kernels.cuh"

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;  // 64 MiB

// The shared scratch.  In host code this name is only a stand-in: its device address comes from
// cudaGetSymbolAddress, per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kMaxDevices = 64;

// Device address of the scratch array, looked up once per device (with that device current).
// Atomic, so that host threads making their first calls at once do not race on the cache (they
// look up the same address).  The cached address belongs to the device's context of the time:
// after a cudaDeviceReset the process must not call this entry point again on that device.
std::atomic<void*> g_scratch_ptr[kMaxDevices];

ss_status scratch_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SS_ERR_CUDA;
  void* p = g_scratch_ptr[dev].load(std::memory_order_acquire);
  if (p == nullptr) {
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return SS_ERR_CUDA;
    g_scratch_ptr[dev].store(p, std::memory_order_release);
  }
  *out = p;
  return SS_OK;
}

}  // namespace

extern "C" {

size_t ss_noalloc_scratch_bytes(void) { return kNoAllocScratchBytes; }

ss_status ss_render_fwd_noalloc(const ss_splats* splats, const ss_camera* cam, const float* dF, const float* color,
                                const ss_raster_opts* opts, const ss_target_io* io, int64_t* needed,
                                ss_stream_t stream) {
  if (!splats || !cam || !opts || !io) return SS_ERR_INVALID_ARG;
  // the intersection capacity that fits the array (workspace bytes grow linearly with it)
  size_t base = 0, probe = 0;
  ss_status e = ss_workspace_size(splats, cam, 1, SS_PASS_MAIN, opts, 0, &base);
  if (e != SS_OK) return e;
  if (base >= kNoAllocScratchBytes) return SS_ERR_INVALID_ARG;  // too many splats for the array
  const int64_t step = 1 << 20;
  e = ss_workspace_size(splats, cam, 1, SS_PASS_MAIN, opts, step, &probe);
  if (e != SS_OK) return e;
  const double per_isect = (double)(probe - base) / (double)step;
  int64_t capacity = (int64_t)((double)(kNoAllocScratchBytes - base) / per_isect);
  size_t bytes = 0;
  for (int i = 0; i < 64; ++i) {
    if ((e = ss_workspace_size(splats, cam, 1, SS_PASS_MAIN, opts, capacity, &bytes)) != SS_OK) return e;
    if (bytes <= kNoAllocScratchBytes) break;
    capacity -= capacity / 32 + 1;
  }
  if (bytes > kNoAllocScratchBytes || capacity < 1) return SS_ERR_INVALID_ARG;
  void* ws = nullptr;
  if ((e = scratch_for_current_device(&ws)) != SS_OK) return e;
  // projection clears the status block; binning clears the per-tile ranges
  e = ss_project_splats(splats, cam, 1, SS_PASS_MAIN, dF, color, opts, ws, kNoAllocScratchBytes, capacity,
                        stream);
  if (e != SS_OK) return e;
  int64_t need = 0;
  e = ss_bin_and_sort(splats, cam, 1, SS_PASS_MAIN, opts, ws, kNoAllocScratchBytes, capacity, &need, stream);
  if (needed) *needed = need;
  if (e != SS_OK) return e;
  return ss_rasterize_fwd(splats, cam, 1, SS_PASS_MAIN, opts, io, ws, kNoAllocScratchBytes, capacity,
                          stream);
}

}  // extern "C"
