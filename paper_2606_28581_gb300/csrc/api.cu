// C ABI of the rasterizer: host-side validation, workspace layout and launch sequencing.
#include <atomic>
#include <cmath>
#include <cstring>

#include "kernels.cuh"

using namespace ss;

namespace ss {
static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int device_sm_count() {
  static int dev_sms[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (dev_sms[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
    dev_sms[dev] = v;
  }
  return dev_sms[dev];
}
}  // namespace ss

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Layout {
  size_t status, tcams, geom, feat, rect, grad;
  size_t hk_a, hv_a, hk_b, hv_b;  // height sort
  size_t counts, offsets, scan_scratch;
  size_t keys_a, vals_a, keys_b, vals_b;
  size_t hist, hist_off;
  size_t segs;
  size_t ranges;
  size_t total;
  int64_t T, n, n_pad, total_tiles, capacity;
  int local_bits;  // bits of the largest target's tile ids, relative to its first tile
  int hbit_lo;
  ScanPlan count_scan;
  RadixPlan rp_tiles, rp_height;
  bool tiles_in_b, height_in_b;
  TargetStatic tg[kMaxTargets];
};


bool finite(float x) { return std::isfinite(x); }

ss_status check_opts(const ss_raster_opts* o) {
  if (!o) return SS_ERR_INVALID_ARG;
  const bool shape = (o->tile_w == 16 && o->tile_h == 16) || (o->tile_w == 32 && o->tile_h == 8) ||
                     (o->tile_w == 8 && o->tile_h == 32) || (o->tile_w == 32 && o->tile_h == 16) ||
                     (o->tile_w == 16 && o->tile_h == 32);
  if (!shape) return SS_ERR_INVALID_ARG;
  if (o->batch != 256) return SS_ERR_INVALID_ARG;
  if (o->pixels_per_thread != 4) return SS_ERR_INVALID_ARG;
  if (o->count_pairs != 0 && o->count_pairs != 1) return SS_ERR_INVALID_ARG;
  if (o->persistent != 0 && o->persistent != 1) return SS_ERR_INVALID_ARG;
  if (o->subblock_cull != 0 && o->subblock_cull != 1) return SS_ERR_INVALID_ARG;
  if (!finite(o->sigma_px) || !(o->sigma_px > 0.0f)) return SS_ERR_INVALID_ARG;
  if (!finite(o->det_eps) || !(o->det_eps >= 0.0f)) return SS_ERR_INVALID_ARG;
  if (!finite(o->alpha_min) || !finite(o->alpha_max) || !(o->alpha_min > 0.0f) ||
      !(o->alpha_max >= o->alpha_min) || !(o->alpha_max < 1.0f))
    return SS_ERR_INVALID_ARG;
  if (!finite(o->t_min) || !(o->t_min > 0.0f) || !(o->t_min < 1.0f)) return SS_ERR_INVALID_ARG;
  return SS_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

ss_status check_splats(const ss_splats* s) {
  if (!s) return SS_ERR_INVALID_ARG;
  if (s->n < 0 || s->n_pad < s->n || (s->n_pad % 8) != 0) return SS_ERR_INVALID_ARG;
  if (s->n > 0x7fffffffLL || s->n_pad > 0x7fffffffLL) return SS_ERR_INVALID_ARG;
  if (s->dtype != SS_F32 && s->dtype != SS_BF16) return SS_ERR_INVALID_ARG;
  if (s->n > 0) {
    const void* ps[5] = {s->means, s->scales, s->quats, s->opacity, s->rgb};
    for (const void* p : ps)
      if (!p || !aligned16(p)) return SS_ERR_INVALID_ARG;
  }
  return SS_OK;
}

ss_status check_cams(const ss_camera* cams, int32_t n_cams, int32_t passes) {
  if (!cams || n_cams < 1 || n_cams > kMaxCams) return SS_ERR_INVALID_ARG;
  if (passes < 1 || passes > 3) return SS_ERR_INVALID_ARG;
  for (int c = 0; c < n_cams; ++c) {
    const ss_camera& k = cams[c];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 4; ++j)
        if (!finite(k.F_xy[i][j])) return SS_ERR_INVALID_ARG;
    if (!finite(k.max_alt)) return SS_ERR_INVALID_ARG;
    if ((passes & SS_PASS_MAIN) && (k.width < 1 || k.height < 1 || k.width > 16384 || k.height > 16384))
      return SS_ERR_INVALID_ARG;
    if (passes & SS_PASS_SUN) {
      if (k.shadow_w < 1 || k.shadow_h < 1 || k.shadow_w > 16384 || k.shadow_h > 16384)
        return SS_ERR_INVALID_ARG;
      if (!finite(k.sun_phi) || !finite(k.sun_theta) || !(k.sun_theta > 0.0f) || !(k.sun_theta <= 1.5707964f))
        return SS_ERR_INVALID_ARG;
      if (!finite(k.shadow_scale) || !(k.shadow_scale > 0.0f)) return SS_ERR_INVALID_ARG;
    }
  }
  return SS_OK;
}

int targets_of(int32_t n_cams, int32_t passes) {
  return n_cams * (((passes & SS_PASS_MAIN) ? 1 : 0) + ((passes & SS_PASS_SUN) ? 1 : 0));
}

ss_status make_layout(const ss_splats* s, const ss_camera* cams, int32_t n_cams, int32_t passes,
                      const ss_raster_opts* o, int64_t capacity, Layout* L) {
  ss_status e;
  if ((e = check_splats(s)) != SS_OK) return e;
  if ((e = check_cams(cams, n_cams, passes)) != SS_OK) return e;
  if ((e = check_opts(o)) != SS_OK) return e;
  if (capacity < 0 || capacity > 0x7fffffffLL) return SS_ERR_INVALID_ARG;
  std::memset(L, 0, sizeof(Layout));
  L->T = targets_of(n_cams, passes);
  L->n = s->n;
  L->n_pad = s->n_pad;
  L->capacity = capacity;
  int64_t tiles = 0;
  int ti = 0;
  for (int pass = 0; pass < 2; ++pass) {
    const bool sun = pass == 1;
    if (!(passes & (sun ? SS_PASS_SUN : SS_PASS_MAIN))) continue;
    for (int c = 0; c < n_cams; ++c) {
      TargetStatic& t = L->tg[ti++];
      t.W = sun ? cams[c].shadow_w : cams[c].width;
      t.H = sun ? cams[c].shadow_h : cams[c].height;
      t.tiles_x = (t.W + o->tile_w - 1) / o->tile_w;
      t.tiles_y = (t.H + o->tile_h - 1) / o->tile_h;
      t.tile_base = (int32_t)tiles;
      t.cam = c;
      t.sun = sun ? 1 : 0;
      t.S = sun ? cams[c].shadow_scale : 1.0f;
      tiles += (int64_t)t.tiles_x * t.tiles_y;
      if (tiles > 0x7fffffffLL) return SS_ERR_INVALID_ARG;
    }
  }
  L->total_tiles = tiles;
  // The emission leaves each target's overlaps contiguous, so the tile sort orders each target's
  // segment by its local tile id: as many bits as the largest target's tile count needs.
  int lb = 1;
  for (int t = 0; t < (int)L->T; ++t)
    while ((1LL << lb) < (int64_t)L->tg[t].tiles_x * L->tg[t].tiles_y) ++lb;
  L->local_bits = lb;
  L->hbit_lo = (s->dtype == SS_BF16) ? 16 : 0;
  L->count_scan = plan_scan(L->T * L->n);
  L->rp_tiles = plan_radix(capacity, segment_digit_bits(lb), (int)L->T);
  L->rp_height = plan_radix(s->n);
  L->tiles_in_b = radix_pass_count(0, lb, segment_digit_bits(lb)) % 2 == 1;
  L->height_in_b = radix_pass_count(L->hbit_lo, 32, 8) % 2 == 1;

  const size_t TN = (size_t)L->T * (size_t)L->n_pad;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off = align_up(off + bytes);
    return at;
  };
  L->status = take(sizeof(StatusBlock));
  L->tcams = take(sizeof(TargetCam) * kMaxTargets);
  L->geom = take(TN * 48);
  L->feat = take(TN * 32);
  L->rect = take(TN * 16);
  L->grad = take(TN * 64);
  const size_t np4 = (size_t)L->n_pad * 4;
  L->hk_a = take(np4);
  L->hv_a = take(np4);
  L->hk_b = take(np4);
  L->hv_b = take(np4);
  const size_t tn4 = (size_t)L->T * (size_t)L->n * 4;
  L->counts = take(tn4);
  L->offsets = take(tn4);
  size_t scr = L->count_scan.scratch_elems;
  const size_t hs1 = L->rp_tiles.hist_scan.scratch_elems, hs2 = L->rp_height.hist_scan.scratch_elems;
  if (hs1 > scr) scr = hs1;
  if (hs2 > scr) scr = hs2;
  L->scan_scratch = take((scr + 2) * 8);
  const size_t cap4 = (size_t)capacity * 4;
  L->keys_a = take(cap4);
  L->vals_a = take(cap4);
  L->keys_b = take(cap4);
  L->vals_b = take(cap4);
  const int64_t hb_t = L->rp_tiles.nblocks << L->rp_tiles.digit_bits, hb_h = L->rp_height.nblocks << 8;
  const int64_t hb = hb_t > hb_h ? hb_t : hb_h;  // histogram entries of the larger sort
  L->hist = take((size_t)hb * 4);
  L->hist_off = take((size_t)hb * 4);
  L->segs = take(sizeof(SortSeg) * (kMaxTargets + 1));
  L->ranges = take((size_t)tiles * 8);
  L->total = off;
  return SS_OK;
}

template <typename T>
T* at(void* ws, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(ws) + off);
}

ss_status check_ws(const Layout& L, void* ws, size_t ws_bytes) {
  if (!ws || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0) return SS_ERR_INVALID_ARG;
  if (ws_bytes < L.total) return SS_ERR_INVALID_ARG;
  return SS_OK;
}

int num_sms_cached() { return device_sm_count(); }

ProjectCommon common_of(const ss_splats* s, const Layout& L, void* ws) {
  ProjectCommon c;
  c.means = s->means;
  c.scales = s->scales;
  c.quats = s->quats;
  c.opacity = s->opacity;
  c.rgb = s->rgb;
  c.n = s->n;
  c.n_pad = s->n_pad;
  c.n_targets = (int32_t)L.T;
  c.tcams = at<TargetCam>(ws, L.tcams);
  return c;
}

ss_status fill_raster(RasterParams& rp, const ss_splats* s, const Layout& L, const ss_raster_opts* o,
                      const ss_target_io* io, void* ws, bool bwd) {
  std::memset(&rp, 0, sizeof(rp));
  if (!io) return SS_ERR_INVALID_ARG;
  for (int t = 0; t < L.T; ++t) {
    const ss_target_io& a = io[t];
    if (!a.T_final || !a.last) return SS_ERR_INVALID_ARG;
    if (L.tg[t].sun && (a.rgb || a.normal || (bwd && (a.d_rgb || a.d_normal)))) return SS_ERR_INVALID_ARG;
    TargetIO& b = rp.io[t];
    b.rgb = a.rgb;
    b.depth = a.depth;
    b.normal = a.normal;
    b.alpha = a.alpha;
    b.T_final = a.T_final;
    b.last = a.last;
    b.d_rgb = bwd ? a.d_rgb : nullptr;
    b.d_depth = bwd ? a.d_depth : nullptr;
    b.d_normal = bwd ? a.d_normal : nullptr;
    b.d_alpha = bwd ? a.d_alpha : nullptr;
    b.distort = bwd ? nullptr : a.distort;
    b.d_distort = bwd ? a.d_distort : nullptr;
    // the distortion adjoint reads the forward's depth plane (the weighted depth of the whole ray)
    if (bwd && a.d_distort && !a.depth) return SS_ERR_INVALID_ARG;
    rp.distort |= (b.distort || b.d_distort) ? 1 : 0;
  }
  rp.tcams = at<TargetCam>(ws, L.tcams);
  rp.geom = at<float4>(ws, L.geom);
  rp.feat = at<float4>(ws, L.feat);
  rp.vals = at<uint32_t>(ws, L.tiles_in_b ? L.vals_b : L.vals_a);
  rp.ranges = at<uint2>(ws, L.ranges);
  rp.items = nullptr;
  rp.status = at<StatusBlock>(ws, L.status);
  rp.grad = at<float>(ws, L.grad);
  rp.n_pad = s->n_pad;
  rp.n_targets = (int32_t)L.T;
  rp.total_tiles = (int32_t)L.total_tiles;
  const float sig = o->sigma_px;
  rp.k.inv2s2 = 1.0f / (2.0f * sig * sig);
  rp.k.c_uv = -0.5f * kLog2e;
  rp.k.c_xy = -kLog2e * rp.k.inv2s2;
  rp.k.amin = o->alpha_min;
  rp.k.amax = o->alpha_max;
  rp.cull.ln_amin = logf(o->alpha_min);
  rp.cull.sigma2 = sig * sig;
  rp.t_min = o->t_min;
  rp.subblock_cull = o->subblock_cull;
  rp.count_pairs = bwd ? 0 : o->count_pairs;
  return SS_OK;
}

ss_status check_grads(const ss_splats* s, const ss_splat_grads* g) {
  if (!g || g->n_pad < s->n) return SS_ERR_INVALID_ARG;
  if (s->n > 0 && (!g->means || !g->scales || !g->quats || !g->opacity || !g->rgb)) return SS_ERR_INVALID_ARG;
  return SS_OK;
}

ss_status run_project_bwd(const ss_splats* splats, const Layout& L, const ss_raster_opts* opts,
                          const ss_splat_grads* grads, float* d_dF, float* d_color, void* ws, cudaStream_t st) {
  ProjectBwdParams pb;
  pb.c = common_of(splats, L, ws);
  pb.rect = at<uint4>(ws, L.rect);
  pb.grad = at<float>(ws, L.grad);
  pb.g.means = grads->means;
  pb.g.scales = grads->scales;
  pb.g.quats = grads->quats;
  pb.g.opacity = grads->opacity;
  pb.g.rgb = grads->rgb;
  pb.g.n_pad = grads->n_pad;
  pb.d_dF = d_dF;
  pb.d_color = d_color;
  pb.amin = opts->alpha_min;
  pb.det_eps = opts->det_eps;
  SS_CUDA_TRY(launch_project_bwd(pb, splats->dtype, st));
  return SS_OK;
}

}  // namespace

extern "C" {

void ss_default_opts(ss_raster_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tile_w = 16;
  o->tile_h = 16;
  o->batch = 256;
  o->persistent = 0;
  o->sigma_px = 0.70710678f;
  o->det_eps = 1e-6f;
  o->alpha_min = 1.0f / 255.0f;
  o->alpha_max = 0.99f;
  o->t_min = 1e-4f;
  o->pixels_per_thread = 4;
  o->subblock_cull = 1;
  o->count_pairs = 0;
}

void ss_staging_batches(int32_t* fwd, int32_t* bwd) {
  if (fwd) *fwd = ss::kFwdBatch;
  if (bwd) *bwd = ss::kBwdBatch;
}

const char* ss_status_string(ss_status s) {
  switch (s) {
    case SS_OK: return "ok";
    case SS_ERR_INVALID_ARG: return "invalid argument";
    case SS_ERR_CAPACITY: return "intersection capacity exceeded";
    case SS_ERR_CUDA: return "CUDA error";
    case SS_ERR_TIMEOUT: return "device wait timed out";
    case SS_ERR_NONFINITE: return "non-finite input";
  }
  return "unknown status";
}

ss_status ss_workspace_size(const ss_splats* splats, const ss_camera* cams, int32_t n_cams, int32_t passes,
                            const ss_raster_opts* opts, int64_t capacity, size_t* bytes) {
  if (!bytes) return SS_ERR_INVALID_ARG;
  Layout L;
  ss_status e = make_layout(splats, cams, n_cams, passes, opts, capacity, &L);
  if (e != SS_OK) return e;
  *bytes = L.total;
  return SS_OK;
}

ss_status ss_project_splats(const ss_splats* splats, const ss_camera* cams, int32_t n_cams, int32_t passes,
                            const float* dF, const float* color, const ss_raster_opts* opts, void* ws,
                            size_t ws_bytes,
                            int64_t capacity, ss_stream_t stream) {
  Layout L;
  ss_status e = make_layout(splats, cams, n_cams, passes, opts, capacity, &L);
  if (e != SS_OK) return e;
  if ((e = check_ws(L, ws, ws_bytes)) != SS_OK) return e;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  SS_CUDA_TRY(cudaMemsetAsync(at<char>(ws, L.status), 0, sizeof(StatusBlock), st));
  AssembleParams ap;
  std::memset(&ap, 0, sizeof(ap));
  for (int c = 0; c < n_cams; ++c) {
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 4; ++j) ap.cams[c].F[4 * i + j] = cams[c].F_xy[i][j];
    ap.cams[c].max_alt = cams[c].max_alt;
    ap.cams[c].phi = cams[c].sun_phi;
    ap.cams[c].theta = cams[c].sun_theta;
  }
  for (int t = 0; t < L.T; ++t) ap.tg[t] = L.tg[t];
  ap.n_targets = (int32_t)L.T;
  ap.dF = dF;
  ap.color = color;
  ap.out = at<TargetCam>(ws, L.tcams);
  SS_CUDA_TRY(launch_assemble(ap, st));
  ProjectParams pp;
  pp.c = common_of(splats, L, ws);
  pp.geom = at<float4>(ws, L.geom);
  pp.feat = at<float4>(ws, L.feat);
  pp.rect = at<uint4>(ws, L.rect);
  pp.grad = at<float4>(ws, L.grad);
  pp.status = at<StatusBlock>(ws, L.status);
  pp.amin = opts->alpha_min;
  pp.ln_amin = logf(opts->alpha_min);
  pp.sigma = opts->sigma_px;
  pp.det_eps = opts->det_eps;
  pp.cull.ln_amin = pp.ln_amin;
  pp.cull.sigma2 = opts->sigma_px * opts->sigma_px;
  pp.tile_w = opts->tile_w;
  pp.tile_h = opts->tile_h;
  SS_CUDA_TRY(launch_project(pp, splats->dtype, st));
  return SS_OK;
}

ss_status ss_bin_and_sort(const ss_splats* splats, const ss_camera* cams, int32_t n_cams, int32_t passes,
                          const ss_raster_opts* opts, void* ws, size_t ws_bytes, int64_t capacity,
                          int64_t* needed, ss_stream_t stream) {
  Layout L;
  ss_status e = make_layout(splats, cams, n_cams, passes, opts, capacity, &L);
  if (e != SS_OK) return e;
  if ((e = check_ws(L, ws, ws_bytes)) != SS_OK) return e;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  StatusBlock* status = at<StatusBlock>(ws, L.status);
  unsigned long long* scratch = at<unsigned long long>(ws, L.scan_scratch);
  // 1. visibility order: stable sort by height, descending
  uint32_t* hk_a = at<uint32_t>(ws, L.hk_a);
  uint32_t* hv_a = at<uint32_t>(ws, L.hv_a);
  uint32_t* hk_b = at<uint32_t>(ws, L.hk_b);
  uint32_t* hv_b = at<uint32_t>(ws, L.hv_b);
  SS_CUDA_TRY(launch_height_keys(splats->means, splats->dtype, L.n, L.n_pad, hk_a, hv_a, st));
  bool hin_b = false;
  SS_CUDA_TRY(radix_sort_pairs(hk_a, hv_a, hk_b, hv_b, L.n, nullptr, L.hbit_lo, 32, at<uint32_t>(ws, L.hist),
                               at<uint32_t>(ws, L.hist_off), scratch, L.rp_height, &hin_b, st));
  const uint32_t* order = hin_b ? hv_b : hv_a;
  // 2. per (target, rank) tile counts, their scan, and the emission in visibility order
  BinParams bp;
  bp.tcams = at<TargetCam>(ws, L.tcams);
  bp.n_targets = (int32_t)L.T;
  bp.n = L.n;
  bp.n_pad = L.n_pad;
  bp.rect = at<uint4>(ws, L.rect);
  bp.order = order;
  bp.counts = at<uint32_t>(ws, L.counts);
  bp.offsets = at<uint32_t>(ws, L.offsets);
  bp.keys = at<uint32_t>(ws, L.keys_a);
  bp.vals = at<uint32_t>(ws, L.vals_a);
  bp.capacity = capacity;
  bp.status = status;
  SS_CUDA_TRY(launch_counts(bp, st));
  unsigned long long* total = scratch + L.count_scan.scratch_elems;  // one past the scan's own total
  SS_CUDA_TRY(exclusive_scan_u32(bp.counts, at<uint32_t>(ws, L.offsets), L.T * L.n, scratch, L.count_scan,
                                 total, st));
  SS_CUDA_TRY(launch_finish_count(status, nullptr, nullptr, total, capacity, st));
  SS_CUDA_TRY(launch_emit(bp, st));
  // 3. stable sort of each target's overlaps by tile id, then per-tile ranges
  bool tin_b = false;
  SortSeg* segs = at<SortSeg>(ws, L.segs);
  SS_CUDA_TRY(launch_sort_segments(at<uint32_t>(ws, L.offsets), L.n, (int)L.T, bp.tcams, status,
                                   radix_tile(L.rp_tiles.digit_bits), segs, st));
  SS_CUDA_TRY(radix_sort_segments(at<uint32_t>(ws, L.keys_a), at<uint32_t>(ws, L.vals_a), at<uint32_t>(ws, L.keys_b),
                                  at<uint32_t>(ws, L.vals_b), segs, (int)L.T, L.local_bits, at<uint32_t>(ws, L.hist),
                                  at<uint32_t>(ws, L.hist_off), scratch, L.rp_tiles, &tin_b, st));
  const uint32_t* keys = at<uint32_t>(ws, tin_b ? L.keys_b : L.keys_a);
  SS_CUDA_TRY(cudaMemsetAsync(at<char>(ws, L.ranges), 0, (size_t)L.total_tiles * 8, st));
  SS_CUDA_TRY(launch_ranges(keys, status, at<uint2>(ws, L.ranges), capacity, st));
  if (needed) {
    StatusBlock hs;
    SS_CUDA_TRY(cudaMemcpyAsync(&hs, status, sizeof(hs), cudaMemcpyDeviceToHost, st));
    SS_CUDA_TRY(cudaStreamSynchronize(st));
    *needed = (int64_t)hs.n_isect;
    if (hs.n_isect > (unsigned long long)capacity) return SS_ERR_CAPACITY;
  }
  return SS_OK;
}

ss_status ss_rasterize_fwd(const ss_splats* splats, const ss_camera* cams, int32_t n_cams, int32_t passes,
                           const ss_raster_opts* opts, const ss_target_io* io, void* ws,
                           size_t ws_bytes, int64_t capacity, ss_stream_t stream) {
  Layout L;
  ss_status e = make_layout(splats, cams, n_cams, passes, opts, capacity, &L);
  if (e != SS_OK) return e;
  if ((e = check_ws(L, ws, ws_bytes)) != SS_OK) return e;
  RasterParams* rp = new RasterParams;
  e = fill_raster(*rp, splats, L, opts, io, ws, false);
  if (e != SS_OK) {
    delete rp;
    return e;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t ce = cudaSuccess;
  if (opts->persistent)
    ce = cudaMemsetAsync(&at<StatusBlock>(ws, L.status)->work_fwd, 0, sizeof(unsigned int), st);
  if (ce == cudaSuccess)
    ce = launch_raster_fwd(*rp, opts->tile_w, opts->tile_h, opts->batch,
                           opts->persistent != 0, num_sms_cached(), st);
  delete rp;
  return ce == cudaSuccess ? SS_OK : SS_ERR_CUDA;
}

ss_status ss_rasterize_bwd(const ss_splats* splats, const ss_camera* cams, int32_t n_cams, int32_t passes,
                           const ss_raster_opts* opts, const ss_target_io* io, const ss_splat_grads* grads,
                           float* d_dF, float* d_color,
                           void* ws, size_t ws_bytes, int64_t capacity, ss_stream_t stream) {
  Layout L;
  ss_status e = make_layout(splats, cams, n_cams, passes, opts, capacity, &L);
  if (e != SS_OK) return e;
  if ((e = check_ws(L, ws, ws_bytes)) != SS_OK) return e;
  if (grads && (e = check_grads(splats, grads)) != SS_OK) return e;
  RasterParams* rp = new RasterParams;
  e = fill_raster(*rp, splats, L, opts, io, ws, true);
  if (e != SS_OK) {
    delete rp;
    return e;
  }
  rp->d_color = d_color;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t ce = cudaSuccess;
  if (opts->persistent)
    ce = cudaMemsetAsync(&at<StatusBlock>(ws, L.status)->work_bwd, 0, sizeof(unsigned int), st);
  if (ce == cudaSuccess)
    ce = launch_raster_bwd(*rp, opts->tile_w, opts->tile_h, opts->batch,
                           opts->persistent != 0, num_sms_cached(), st);
  delete rp;
  if (ce != cudaSuccess) return SS_ERR_CUDA;
  if (!grads) return SS_OK;
  return run_project_bwd(splats, L, opts, grads, d_dF, d_color, ws, st);
}

ss_status ss_project_bwd(const ss_splats* splats, const ss_camera* cams, int32_t n_cams, int32_t passes,
                         const ss_raster_opts* opts, const ss_splat_grads* grads, float* d_dF, float* d_color,
                         void* ws,
                         size_t ws_bytes, int64_t capacity, ss_stream_t stream) {
  Layout L;
  ss_status e = make_layout(splats, cams, n_cams, passes, opts, capacity, &L);
  if (e != SS_OK) return e;
  if ((e = check_ws(L, ws, ws_bytes)) != SS_OK) return e;
  if ((e = check_grads(splats, grads)) != SS_OK) return e;
  return run_project_bwd(splats, L, opts, grads, d_dF, d_color, ws, reinterpret_cast<cudaStream_t>(stream));
}

ss_status ss_shadow_depth(const ss_splats* splats, const ss_camera* cams, int32_t n_cams, const float* dF,
                          const ss_raster_opts* opts, const ss_target_io* io, void* ws, size_t ws_bytes,
                          int64_t capacity, int64_t* needed, ss_stream_t stream) {
  ss_status e =
      ss_project_splats(splats, cams, n_cams, SS_PASS_SUN, dF, nullptr, opts, ws, ws_bytes, capacity, stream);
  if (e != SS_OK) return e;
  e = ss_bin_and_sort(splats, cams, n_cams, SS_PASS_SUN, opts, ws, ws_bytes, capacity, needed, stream);
  if (e != SS_OK) return e;
  return ss_rasterize_fwd(splats, cams, n_cams, SS_PASS_SUN, opts, io, ws, ws_bytes, capacity, stream);
}

ss_status ss_frame_status(const void* ws, size_t ws_bytes, int64_t* needed, int64_t* nonfinite, int64_t* walked,
                          int32_t* flags, ss_stream_t stream) {
  if (!ws || ws_bytes < sizeof(StatusBlock)) return SS_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  StatusBlock hs;
  SS_CUDA_TRY(cudaMemcpyAsync(&hs, ws, sizeof(hs), cudaMemcpyDeviceToHost, st));
  SS_CUDA_TRY(cudaStreamSynchronize(st));
  if (needed) *needed = (int64_t)hs.n_isect;
  if (nonfinite) *nonfinite = (int64_t)hs.nonfinite;
  if (walked) *walked = (int64_t)hs.n_walked;
  if (flags) *flags = (int32_t)hs.flags;
  if (hs.flags & FLAG_OVERFLOW) return SS_ERR_CAPACITY;
  if (hs.flags & FLAG_TIMEOUT) return SS_ERR_TIMEOUT;
  if (hs.nonfinite) return SS_ERR_NONFINITE;
  return SS_OK;
}

int64_t ss_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int32_t ss_device_info(int32_t* num_sms, int32_t* arch) {
  if (num_sms) *num_sms = num_sms_cached();
  if (arch) {
#if defined(SS_ARCH)
    *arch = SS_ARCH;
#else
    *arch = 0;
#endif
  }
  return 0;
}

}  // extern "C"
