// Geometry-aware initialisation (Sec. 3.4): area-weighted sampling of splat centres from a DSM,
// orientation from the DSM's local normal by Gram-Schmidt, and scales from the mean distance to
// the k nearest samples (a uniform 2-D grid of cells, searched ring by ring).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "kernels.cuh"

using namespace ss;

namespace {

constexpr unsigned long long kPhiloxM0 = 0xD2E7470EE14C6C93ull;
constexpr unsigned long long kPhiloxM1 = 0xCA5A826395121157ull;
constexpr unsigned long long kPhiloxW0 = 0x9E3779B97F4A7C15ull;
constexpr unsigned long long kPhiloxW1 = 0xBB67AE8584CAA73Bull;
constexpr unsigned long long kStreamInit = 2ull;
constexpr int kMaxK = 8;

struct U64x4 {
  unsigned long long x, y, z, w;
};

// Philox4x64-10 (Salmon et al., SC'11)
__device__ __forceinline__ U64x4 philox(U64x4 c, unsigned long long k0, unsigned long long k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += kPhiloxW0;
      k1 += kPhiloxW1;
    }
    const unsigned long long hi0 = __umul64hi(kPhiloxM0, c.x), lo0 = kPhiloxM0 * c.x;
    const unsigned long long hi1 = __umul64hi(kPhiloxM1, c.z), lo1 = kPhiloxM1 * c.z;
    c = U64x4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
  }
  return c;
}

__device__ __forceinline__ float uniform24(unsigned long long x) {
  return ((float)(x >> 40) + 0.5f) * 5.9604644775390625e-8f;
}

struct InitParams {
  const float* Z;    // [H][W]
  const float* rgb;  // [3][H][W] or null
  int32_t W, H;
  float x0, y0, g, kscale;  // kscale = 2^16 / g (float)
  int64_t n;
  int32_t K;
  float opacity;
  unsigned long long seed;
  uint32_t* w;                // [H W] integer weights
  unsigned long long* excl;   // [H W] exclusive prefix sums
  const unsigned long long* total;
  float* pts;                 // [3][n] sample positions (FP32) for the kNN
  // kNN grid
  float gx0, gy0, h;          // west edge, north edge, cell size
  int32_t NX, NY;
  uint32_t* keys;             // [n] cell of each sample
  uint32_t* idx;              // [n] sample index
  const uint32_t* skeys;      // sorted
  const uint32_t* sidx;
  float* spts;                // [3][n] the positions in cell order
  uint32_t* cstart;           // [NX NY]
  uint32_t* cend;
  // outputs
  void* st[5];  // means, scales, quats, opacity, rgb
  int32_t dtype;
  int64_t n_pad;
};

__device__ __forceinline__ void put(void* base, int32_t dtype, int64_t i, float v) {
  if (dtype == SS_F32) static_cast<float*>(base)[i] = v;
  else static_cast<__nv_bfloat16*>(base)[i] = __float2bfloat16_rn(v);
}

// dz toward +x (next column) and toward +y (previous row), one pixel each: central differences
// inside, one-sided on the border, with IEEE operations in a fixed order (no contraction)
__device__ __forceinline__ void dz_at(const InitParams& p, int i, int j, float& dzx, float& dzy) {
  const float* Z = p.Z;
  const int64_t r = (int64_t)j * p.W;
  if (p.W < 2) dzx = 0.0f;
  else if (i == 0) dzx = __fsub_rn(Z[r + 1], Z[r]);
  else if (i == p.W - 1) dzx = __fsub_rn(Z[r + i], Z[r + i - 1]);
  else dzx = __fmul_rn(__fsub_rn(Z[r + i + 1], Z[r + i - 1]), 0.5f);
  if (p.H < 2) dzy = 0.0f;
  else if (j == 0) dzy = __fsub_rn(Z[i], Z[p.W + i]);
  else if (j == p.H - 1) dzy = __fsub_rn(Z[r - p.W + i], Z[r + i]);
  else dzy = __fmul_rn(__fsub_rn(Z[r - p.W + i], Z[r + p.W + i]), 0.5f);
}

// w = floor(sqrt(dz_x^2 + dz_y^2 + g^2) 2^16 / g): |dx x dy| in units of a flat pixel's area
__global__ void __launch_bounds__(256) init_weights_kernel(const __grid_constant__ InitParams p) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (int64_t)p.W * p.H) return;
  const int i = (int)(k % p.W), j = (int)(k / p.W);
  float dzx, dzy;
  dz_at(p, i, j, dzx, dzy);
  const float q = __fadd_rn(__fadd_rn(__fmul_rn(dzx, dzx), __fmul_rn(dzy, dzy)), __fmul_rn(p.g, p.g));
  const float a = floorf(__fmul_rn(__fsqrt_rn(q), p.kscale));
  p.w[k] = a >= 2147483647.0f ? 2147483647u : (uint32_t)a;
}

// quaternion (w, x, y, z), w >= 0, of the rotation with columns c0, c1, c2 (Shepperd's method)
__device__ void quat_of(const float c0[3], const float c1[3], const float c2[3], float q[4]) {
  const float m00 = c0[0], m11 = c1[1], m22 = c2[2];
  const float tr = m00 + m11 + m22;
  if (tr > 0.0f) {
    const float s = sqrtf(tr + 1.0f) * 2.0f;
    q[0] = 0.25f * s;
    q[1] = (c1[2] - c2[1]) / s;
    q[2] = (c2[0] - c0[2]) / s;
    q[3] = (c0[1] - c1[0]) / s;
  } else if (m00 > m11 && m00 > m22) {
    const float s = sqrtf(1.0f + m00 - m11 - m22) * 2.0f;
    q[0] = (c1[2] - c2[1]) / s;
    q[1] = 0.25f * s;
    q[2] = (c1[0] + c0[1]) / s;
    q[3] = (c2[0] + c0[2]) / s;
  } else if (m11 > m22) {
    const float s = sqrtf(1.0f + m11 - m00 - m22) * 2.0f;
    q[0] = (c2[0] - c0[2]) / s;
    q[1] = (c1[0] + c0[1]) / s;
    q[2] = 0.25f * s;
    q[3] = (c2[1] + c1[2]) / s;
  } else {
    const float s = sqrtf(1.0f + m22 - m00 - m11) * 2.0f;
    q[0] = (c0[1] - c1[0]) / s;
    q[1] = (c2[0] + c0[2]) / s;
    q[2] = (c2[1] + c1[2]) / s;
    q[3] = 0.25f * s;
  }
  if (q[0] < 0.0f)
    for (int t = 0; t < 4; ++t) q[t] = -q[t];
}

// the kNN cell of a position (the same arithmetic wherever it is evaluated)
__device__ __forceinline__ uint32_t cell_of(const InitParams& p, float x, float y) {
  const int cx = min(max((int)floorf((x - p.gx0) / p.h), 0), p.NX - 1);
  const int cy = min(max((int)floorf((p.gy0 - y) / p.h), 0), p.NY - 1);
  return (uint32_t)(cy * p.NX + cx);
}

// one sample: the pixel (exact integer draw), the jittered centre, the Gram-Schmidt basis, the
// colour, and its kNN cell
__global__ void __launch_bounds__(256) init_sample_kernel(const __grid_constant__ InitParams p) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= p.n) return;
  const U64x4 x = philox(U64x4{(unsigned long long)s, 0ull, kStreamInit, 0ull}, p.seed, 0ull);
  const unsigned long long r = __umul64hi(x.x, *p.total);
  int64_t lo = 0, hi = (int64_t)p.W * p.H;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (p.excl[mid] <= r) lo = mid + 1;
    else hi = mid;
  }
  const int64_t pix = lo - 1;
  const int i = (int)(pix % p.W), j = (int)(pix / p.W);
  const float u = uniform24(x.y) - 0.5f, v = uniform24(x.z) - 0.5f;
  float dzx, dzy;
  dz_at(p, i, j, dzx, dzy);
  const float g = p.g;
  const float px = p.x0 + ((float)i + u) * g;
  const float py = p.y0 - (float)j * g + v * g;
  const float pz = p.Z[pix] + u * dzx + v * dzy;
  // t_u = dx / |dx|; t_v = the residual of dy against t_u, normalised; n = t_u x t_v
  const float inu = rsqrtf(g * g + dzx * dzx);
  const float tu[3] = {g * inu, 0.0f, dzx * inu};
  const float dyt = dzy * tu[2];  // dy . t_u, dy = (0, g, dz_y)
  float rv[3] = {-dyt * tu[0], g, dzy - dyt * tu[2]};
  const float inv = rsqrtf(rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2]);
  const float tv[3] = {rv[0] * inv, rv[1] * inv, rv[2] * inv};
  const float nn[3] = {tu[1] * tv[2] - tu[2] * tv[1], tu[2] * tv[0] - tu[0] * tv[2], tu[0] * tv[1] - tu[1] * tv[0]};
  float q[4];
  quat_of(tu, tv, nn, q);
  const int64_t np = p.n_pad;
  put(p.st[0], p.dtype, s, px);
  put(p.st[0], p.dtype, np + s, py);
  put(p.st[0], p.dtype, 2 * np + s, pz);
  for (int t = 0; t < 4; ++t) put(p.st[2], p.dtype, t * np + s, q[t]);
  put(p.st[3], p.dtype, s, p.opacity);
  for (int c = 0; c < 3; ++c)
    put(p.st[4], p.dtype, c * np + s, p.rgb ? p.rgb[(int64_t)c * p.W * p.H + pix] : 0.5f);
  p.pts[s] = px;
  p.pts[p.n + s] = py;
  p.pts[2 * p.n + s] = pz;
  p.keys[s] = cell_of(p, px, py);
  p.idx[s] = (uint32_t)s;
}

// cell ranges of the sorted samples, and their positions gathered into cell order
__global__ void __launch_bounds__(256) init_cells_kernel(const __grid_constant__ InitParams p) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= p.n) return;
  const uint32_t k = p.skeys[s];
  if (s == 0 || p.skeys[s - 1] != k) p.cstart[k] = (uint32_t)s;
  if (s == p.n - 1 || p.skeys[s + 1] != k) p.cend[k] = (uint32_t)(s + 1);
  const uint32_t o = p.sidx[s];
  p.spts[s] = p.pts[o];
  p.spts[p.n + s] = p.pts[p.n + o];
  p.spts[2 * p.n + s] = p.pts[2 * p.n + o];
}

// mean distance to the K nearest other samples: rings of cells around the sample's cell until
// the K-th distance is within the searched radius (every unsearched sample is at least r h away).
// Threads take the samples in cell order, so a warp searches the same few cells.
template <int K>
__global__ void __launch_bounds__(256) init_knn_kernel(const __grid_constant__ InitParams p) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.n) return;
  const int64_t s = p.sidx[t];
  const float x = p.spts[t], y = p.spts[p.n + t], z = p.spts[2 * p.n + t];
  const uint32_t key = p.skeys[t];
  const int cx = (int)(key % (uint32_t)p.NX), cy = (int)(key / (uint32_t)p.NX);
  float best[K];
#pragma unroll
  for (int t = 0; t < K; ++t) best[t] = INFINITY;
  const int rmax = max(p.NX, p.NY);
  for (int r = 0; r <= rmax; ++r) {
    for (int dy = -r; dy <= r; ++dy) {
      const int yy = cy + dy;
      if (yy < 0 || yy >= p.NY) continue;
      const bool edge = dy == -r || dy == r;
      for (int dx = -r; dx <= r; dx += (edge || r == 0) ? 1 : 2 * r) {
        const int xx = cx + dx;
        if (xx < 0 || xx >= p.NX) continue;
        const int c = yy * p.NX + xx;
        const uint32_t b = p.cstart[c], e = p.cend[c];
        for (uint32_t u = b; u < e; ++u) {
          if (u == (uint32_t)t) continue;
          const float ex = p.spts[u] - x, ey = p.spts[p.n + u] - y, ez = p.spts[2 * p.n + u] - z;
          float d2 = ex * ex + ey * ey + ez * ez;
          if (d2 < best[K - 1]) {
#pragma unroll
            for (int q = 0; q < K; ++q) {
              if (d2 < best[q]) {
                const float tmp = best[q];
                best[q] = d2;
                d2 = tmp;
              }
            }
          }
        }
        if (r == 0) break;
      }
    }
    const float rad = (float)r * p.h;
    if (best[K - 1] <= rad * rad) break;
  }
  float m = 0.0f;
#pragma unroll
  for (int t = 0; t < K; ++t) m += sqrtf(best[t]);
  m *= 1.0f / (float)K;
  put(p.st[1], p.dtype, s, m);
  put(p.st[1], p.dtype, p.n_pad + s, m);
}

constexpr size_t kAl = 256;
size_t up(size_t x) { return (x + kAl - 1) / kAl * kAl; }

struct InitLayout {
  size_t w, excl, scan, total, pts, spts, keys_a, vals_a, keys_b, vals_b, hist, hist_off, rscan, cstart, cend, bytes;
  ScanPlan wplan;
  RadixPlan rplan;
  int NX, NY;
  float h;
};

bool grid_of(int32_t W, int32_t H, float g, int64_t n, int& NX, int& NY, float& h) {
  // cells of about four samples where the DSM is flat
  const double ex = (double)W * g, ey = (double)H * g;
  double hh = 2.0 * std::sqrt(ex * ey / (double)std::max<int64_t>(n, 1));
  const double lim = 4096.0;
  hh = std::max(hh, std::max(ex, ey) / lim);
  NX = (int)std::ceil(ex / hh);
  NY = (int)std::ceil(ey / hh);
  NX = std::max(1, std::min(NX, (int)lim));
  NY = std::max(1, std::min(NY, (int)lim));
  h = (float)hh;
  return std::isfinite(hh) && hh > 0.0;
}

bool layout_of(int32_t W, int32_t H, float g, int64_t n, InitLayout& L) {
  if (W < 1 || H < 1 || n < 1 || (int64_t)W * H >= (1LL << 31) || n >= (1LL << 31) || !(g > 0.0f)) return false;
  if (!grid_of(W, H, g, n, L.NX, L.NY, L.h)) return false;
  const int64_t hw = (int64_t)W * H, cells = (int64_t)L.NX * L.NY;
  L.wplan = plan_scan(hw);
  L.rplan = plan_radix(n);
  size_t o = 0;
  auto take = [&](size_t b) { const size_t at = o; o = up(o + b); return at; };
  L.w = take(4 * (size_t)hw);
  L.excl = take(8 * (size_t)hw);
  L.scan = take(8 * L.wplan.scratch_elems);
  L.total = take(8);
  L.pts = take(12 * (size_t)n);
  L.spts = take(12 * (size_t)n);
  L.keys_a = take(4 * (size_t)n);
  L.vals_a = take(4 * (size_t)n);
  L.keys_b = take(4 * (size_t)n);
  L.vals_b = take(4 * (size_t)n);
  L.hist = take(4 * 256 * (size_t)L.rplan.nblocks);
  L.hist_off = take(4 * 256 * (size_t)L.rplan.nblocks);
  L.rscan = take(8 * L.rplan.hist_scan.scratch_elems);
  L.cstart = take(4 * (size_t)cells);
  L.cend = take(4 * (size_t)cells);
  L.bytes = o;
  return true;
}

template <class T>
T* at_(void* b, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(b) + off);
}

unsigned nblk(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

extern "C" {

void ss_default_init_opts(ss_init_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->knn_k = 3;
  o->opacity = 0.1f;
  o->seed = 0;
}

ss_status ss_init_workspace_size(const ss_dsm* dsm, int64_t n, size_t* bytes) {
  if (!dsm || !bytes) return SS_ERR_INVALID_ARG;
  InitLayout L;
  if (!layout_of(dsm->width, dsm->height_px, dsm->gsd, n, L)) return SS_ERR_INVALID_ARG;
  *bytes = L.bytes;
  return SS_OK;
}

ss_status ss_dsm_init(const ss_dsm* dsm, const ss_init_opts* opts, const ss_splats* out, void* ws, size_t ws_bytes,
                      ss_stream_t stream) {
  if (!dsm || !opts || !out || !dsm->heights) return SS_ERR_INVALID_ARG;
  if (opts->knn_k < 1 || opts->knn_k > kMaxK || !(opts->opacity > 0.0f && opts->opacity < 1.0f))
    return SS_ERR_INVALID_ARG;
  if (!std::isfinite(dsm->x0) || !std::isfinite(dsm->y0) || !std::isfinite(dsm->gsd)) return SS_ERR_INVALID_ARG;
  if (out->dtype != SS_F32 && out->dtype != SS_BF16) return SS_ERR_INVALID_ARG;
  if (out->n < 1 || out->n_pad < out->n || (out->n_pad % 8) != 0 || out->n <= opts->knn_k) return SS_ERR_INVALID_ARG;
  const void* ps[5] = {out->means, out->scales, out->quats, out->opacity, out->rgb};
  for (const void* x : ps)
    if (!x || (reinterpret_cast<uintptr_t>(x) & 15u)) return SS_ERR_INVALID_ARG;
  InitLayout L;
  if (!layout_of(dsm->width, dsm->height_px, dsm->gsd, out->n, L)) return SS_ERR_INVALID_ARG;
  if (!ws || ws_bytes < L.bytes || (reinterpret_cast<uintptr_t>(ws) & 255u)) return SS_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  InitParams p;
  std::memset(&p, 0, sizeof(p));
  p.Z = dsm->heights;
  p.rgb = dsm->rgb;
  p.W = dsm->width;
  p.H = dsm->height_px;
  p.x0 = dsm->x0;
  p.y0 = dsm->y0;
  p.g = dsm->gsd;
  p.kscale = (float)(65536.0 / (double)dsm->gsd);
  p.n = out->n;
  p.K = opts->knn_k;
  p.opacity = opts->opacity;
  p.seed = opts->seed;
  p.w = at_<uint32_t>(ws, L.w);
  p.excl = at_<unsigned long long>(ws, L.excl);
  unsigned long long* total = at_<unsigned long long>(ws, L.total);
  p.total = total;
  p.pts = at_<float>(ws, L.pts);
  p.spts = at_<float>(ws, L.spts);
  p.gx0 = dsm->x0 - 0.5f * dsm->gsd;
  p.gy0 = dsm->y0 + 0.5f * dsm->gsd;
  p.h = L.h;
  p.NX = L.NX;
  p.NY = L.NY;
  p.keys = at_<uint32_t>(ws, L.keys_a);
  p.idx = at_<uint32_t>(ws, L.vals_a);
  p.cstart = at_<uint32_t>(ws, L.cstart);
  p.cend = at_<uint32_t>(ws, L.cend);
  p.st[0] = const_cast<void*>(out->means);
  p.st[1] = const_cast<void*>(out->scales);
  p.st[2] = const_cast<void*>(out->quats);
  p.st[3] = const_cast<void*>(out->opacity);
  p.st[4] = const_cast<void*>(out->rgb);
  p.dtype = out->dtype;
  p.n_pad = out->n_pad;
  const int64_t hw = (int64_t)p.W * p.H;
  count_launch();
  init_weights_kernel<<<nblk(hw), 256, 0, st>>>(p);
  if (cudaGetLastError() != cudaSuccess) return SS_ERR_CUDA;
  if (exclusive_scan_u32_u64(p.w, p.excl, hw, at_<unsigned long long>(ws, L.scan), L.wplan, total, st) !=
      cudaSuccess)
    return SS_ERR_CUDA;
  count_launch();
  init_sample_kernel<<<nblk(p.n), 256, 0, st>>>(p);
  if (cudaGetLastError() != cudaSuccess) return SS_ERR_CUDA;
  // samples by kNN cell
  int bits = 1;
  while ((1LL << bits) < (int64_t)L.NX * L.NY) ++bits;
  bool in_b = false;
  if (radix_sort_pairs(p.keys, p.idx, at_<uint32_t>(ws, L.keys_b), at_<uint32_t>(ws, L.vals_b), p.n, nullptr, 0,
                       bits, at_<uint32_t>(ws, L.hist), at_<uint32_t>(ws, L.hist_off),
                       at_<unsigned long long>(ws, L.rscan), L.rplan, &in_b, st) != cudaSuccess)
    return SS_ERR_CUDA;
  p.skeys = in_b ? at_<uint32_t>(ws, L.keys_b) : p.keys;
  p.sidx = in_b ? at_<uint32_t>(ws, L.vals_b) : p.idx;
  const size_t cells = (size_t)L.NX * L.NY;
  if (cudaMemsetAsync(p.cstart, 0, 4 * cells, st) != cudaSuccess ||
      cudaMemsetAsync(p.cend, 0, 4 * cells, st) != cudaSuccess)
    return SS_ERR_CUDA;
  count_launch();
  init_cells_kernel<<<nblk(p.n), 256, 0, st>>>(p);
  count_launch();
  switch (p.K) {
    case 1: init_knn_kernel<1><<<nblk(p.n), 256, 0, st>>>(p); break;
    case 2: init_knn_kernel<2><<<nblk(p.n), 256, 0, st>>>(p); break;
    case 3: init_knn_kernel<3><<<nblk(p.n), 256, 0, st>>>(p); break;
    case 4: init_knn_kernel<4><<<nblk(p.n), 256, 0, st>>>(p); break;
    case 5: init_knn_kernel<5><<<nblk(p.n), 256, 0, st>>>(p); break;
    case 6: init_knn_kernel<6><<<nblk(p.n), 256, 0, st>>>(p); break;
    case 7: init_knn_kernel<7><<<nblk(p.n), 256, 0, st>>>(p); break;
    default: init_knn_kernel<8><<<nblk(p.n), 256, 0, st>>>(p); break;
  }
  return cudaGetLastError() == cudaSuccess ? SS_OK : SS_ERR_CUDA;
}

}  // extern "C"
