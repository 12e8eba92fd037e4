// Sun visibility and image formation (K7), Sec. 3.1 Eq. image_formation with the shadow mapping
// of Sec. 3.1 / Sec. 3.3 (sun camera of Supp. A).
//
// One thread per main-view pixel, every view in one launch (blockIdx.y = view).  The receiver
// (alpha-normalised rendered depth z, height h = max_alt - z) is moved along the sun ray into
// the view's sun view at u = S (x - h B' s); the occluder depth z_o is the bilinear sample of
// the sun view's alpha-normalised depth there; V = exp(-k max(z - z_o - bias, 0)) and
// I = (C A + c) (V + (1 - V) L_a).  The pass is HBM-bound: per pixel it reads 5 planes (and
// four sun texels, mostly from L2) and writes 3 or 4.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "kernels.cuh"

namespace ss {

struct ShadeView {
  float B[2][3];  // F_xy[:, 0:3] (host values; dF is added on the device)
  float s[3];     // sun direction (cos phi / tan theta, sin phi / tan theta, 1)
  float S, maxalt;
  int32_t W, H, Ws, Hs;
  bool vec4;  // pixel count and every plane address are multiples of 4 floats: 16-byte accesses
  ss_shade_io io;
};

struct ShadeParams {
  ShadeView v[kMaxCams];
  const float* dF;  // [V][8] or null
  const float* La;  // [V][3]
  float* d_La;      // [V][3] or null
  float* d_dF;      // [V][8] or null
  float k, bias, eps;
};

// The per-pixel geometry shared by the forward and the backward.
struct ShadeGeom {
  bool shadowed;        // a valid sample with z - z_o - bias > 0
  float V;              // visibility
  float z, h, a, D;     // receiver
  float fx, fy;         // bilinear offsets
  int64_t t00;          // first tap (row-major index into the sun planes)
  float zs[4], as[4], Ds[4];  // taps (00, 10, 01, 11)
  float Bs0, Bs1;       // B' s
};

__device__ __forceinline__ ShadeGeom shade_geom(const ShadeParams& p, const ShadeView& v, int cam, int px, int py,
                                                float alpha, float depth) {
  ShadeGeom g;
  const float* dF = p.dF ? p.dF + 8 * cam : nullptr;
  g.Bs0 = 0.0f;
  g.Bs1 = 0.0f;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float b0 = v.B[0][j] + (dF ? dF[j] : 0.0f);
    const float b1 = v.B[1][j] + (dF ? dF[4 + j] : 0.0f);
    g.Bs0 = fmaf(b0, v.s[j], g.Bs0);
    g.Bs1 = fmaf(b1, v.s[j], g.Bs1);
  }
  g.shadowed = false;
  g.V = 1.0f;
  g.a = alpha;
  g.D = depth;
  g.z = 0.0f;
  g.h = 0.0f;
  g.fx = g.fy = 0.0f;
  g.t00 = 0;
  if (g.a >= p.eps) {
    g.z = g.D / g.a;
    g.h = v.maxalt - g.z;
    const float tx = v.S * (((float)px + 0.5f) - g.h * g.Bs0) - 0.5f;
    const float ty = v.S * (((float)py + 0.5f) - g.h * g.Bs1) - 0.5f;
    if (tx >= 0.0f && tx < (float)(v.Ws - 1) && ty >= 0.0f && ty < (float)(v.Hs - 1)) {
      const float fi = floorf(tx), fj = floorf(ty);
      g.fx = tx - fi;
      g.fy = ty - fj;
      g.t00 = (int64_t)fj * v.Ws + (int64_t)fi;
      const int64_t tap[4] = {g.t00, g.t00 + 1, g.t00 + v.Ws, g.t00 + v.Ws + 1};
      bool ok = true;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        g.as[t] = v.io.sun_alpha[tap[t]];
        g.Ds[t] = v.io.sun_depth[tap[t]];
        ok = ok && g.as[t] >= p.eps;
        g.zs[t] = g.as[t] >= p.eps ? g.Ds[t] / g.as[t] : 0.0f;
      }
      if (ok) {
        const float zo = (1.0f - g.fx) * (1.0f - g.fy) * g.zs[0] + g.fx * (1.0f - g.fy) * g.zs[1] +
                         (1.0f - g.fx) * g.fy * g.zs[2] + g.fx * g.fy * g.zs[3];
        const float delta = g.z - zo - p.bias;
        if (delta > 0.0f) {
          g.shadowed = true;
          g.V = expf(-p.k * delta);
        }
      }
    }
  }
  return g;
}

// Four consecutive pixels (of the flattened view) per thread: their plane reads and writes are
// 16-byte accesses when the view allows it (vec4: pixel count and plane addresses multiples of
// 4 floats), and their independent sun samples overlap.
constexpr int kShadePix = 4;

__device__ __forceinline__ float4 ld4(const float* p, int64_t i, bool vec, int64_t hw) {
  if (vec) return *reinterpret_cast<const float4*>(p + i);
  float4 r;
  r.x = p[i];
  r.y = i + 1 < hw ? p[i + 1] : 0.0f;
  r.z = i + 2 < hw ? p[i + 2] : 0.0f;
  r.w = i + 3 < hw ? p[i + 3] : 0.0f;
  return r;
}
__device__ __forceinline__ void st4(float* p, int64_t i, float4 v, bool vec, int64_t hw) {
  if (vec) {
    *reinterpret_cast<float4*>(p + i) = v;
    return;
  }
  p[i] = v.x;
  if (i + 1 < hw) p[i + 1] = v.y;
  if (i + 2 < hw) p[i + 2] = v.z;
  if (i + 3 < hw) p[i + 3] = v.w;
}
__device__ __forceinline__ float comp(const float4& v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }
__device__ __forceinline__ void set_comp(float4& v, int k, float x) {
  if (k == 0) v.x = x; else if (k == 1) v.y = x; else if (k == 2) v.z = x; else v.w = x;
}

// Both shading kernels are latency-bound: the forward at eight blocks per SM (32 registers, a few
// spilled) measured 15-20 % faster than the four that its natural register count allows; the
// backward, which loads all of a pixel's planes before its stores, is fastest at six.
__global__ void __launch_bounds__(256, 8) shade_fwd_kernel(const __grid_constant__ ShadeParams p) {
  const int cam = blockIdx.y;
  const ShadeView& v = p.v[cam];
  const int64_t hw = (int64_t)v.W * v.H;
  const int64_t pix0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * kShadePix;
  if (pix0 >= hw) return;
  const bool vec = v.vec4;
  // the planes first: their loads do not wait on the geometry
  const float4 a4 = ld4(v.io.alpha, pix0, vec, hw), d4 = ld4(v.io.depth, pix0, vec, hw);
  float4 rgb4[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) rgb4[c] = ld4(v.io.rgb, c * hw + pix0, vec, hw);
  float4 V4;
  // the first pixel's row and column (a view has fewer than 2^31 pixels: 32-bit division), then
  // step along the row
  int py = (int)((uint32_t)pix0 / (uint32_t)v.W), px = (int)pix0 - py * v.W;
#pragma unroll
  for (int k = 0; k < kShadePix; ++k) {
    const int64_t pix = pix0 + k;
    float Vk = 1.0f;
    if (pix < hw) Vk = shade_geom(p, v, cam, px, py, comp(a4, k), comp(d4, k)).V;
    set_comp(V4, k, Vk);
    if (++px == v.W) {
      px = 0;
      ++py;
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float La = p.La[3 * cam + c];
    float4 o;
    o.x = rgb4[c].x * (La + V4.x * (1.0f - La));
    o.y = rgb4[c].y * (La + V4.y * (1.0f - La));
    o.z = rgb4[c].z * (La + V4.z * (1.0f - La));
    o.w = rgb4[c].w * (La + V4.w * (1.0f - La));
    st4(v.io.image, c * hw + pix0, o, vec, hw);
  }
  if (v.io.vis) st4(v.io.vis, pix0, V4, vec, hw);
}

// One pixel per thread: four per thread measured slower here (its sun-view atomics serialise).
__global__ void __launch_bounds__(256, 6) shade_bwd_kernel(const __grid_constant__ ShadeParams p) {
  __shared__ float red[8][10];
  const int cam = blockIdx.y;
  const ShadeView& v = p.v[cam];
  const int64_t hw = (int64_t)v.W * v.H;
  const int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // per-view sums: d La (3) and d B'[:, 0:3] (6); threads past the view add zeros
  float acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (pix < hw) {
    const int py = (int)((uint32_t)pix / (uint32_t)v.W), px = (int)pix - py * v.W;  // fewer than 2^31 pixels
    // every plane value of the pixel is loaded before any gradient is stored: a store could alias
    // a later load, so loads interleaved with the read-modify-writes would wait on each other
    const float alpha = v.io.alpha[pix], depth = v.io.depth[pix];
    float dI[3], R[3], gR[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      dI[c] = v.io.d_image[c * hw + pix];
      R[c] = v.io.rgb[c * hw + pix];
      if (v.io.d_rgb) gR[c] = v.io.d_rgb[c * hw + pix];
    }
    // the depth and alpha gradients of a pixel with a surface (only those can be in shadow)
    float gz = 0.0f, ga = 0.0f;
    if (alpha >= p.eps) {
      if (v.io.d_depth) gz = v.io.d_depth[pix];
      if (v.io.d_alpha) ga = v.io.d_alpha[pix];
    }
    const ShadeGeom g = shade_geom(p, v, cam, px, py, alpha, depth);
    float dV = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float La = p.La[3 * cam + c];
      if (v.io.d_rgb) v.io.d_rgb[c * hw + pix] = gR[c] + dI[c] * (La + g.V * (1.0f - La));
      dV = fmaf(dI[c] * R[c], 1.0f - La, dV);
      acc[c] = dI[c] * R[c] * (1.0f - g.V);
    }
    if (g.shadowed) {
      // V = exp(-k delta), delta = z - z_o - bias
      const float d_delta = -p.k * g.V * dV;
      const float dzo = -d_delta;
      const float dzo_dux = (1.0f - g.fy) * (g.zs[1] - g.zs[0]) + g.fy * (g.zs[3] - g.zs[2]);
      const float dzo_duy = (1.0f - g.fx) * (g.zs[2] - g.zs[0]) + g.fx * (g.zs[3] - g.zs[1]);
      const float dux = dzo * dzo_dux, duy = dzo * dzo_duy;
      const float w[4] = {(1.0f - g.fx) * (1.0f - g.fy), g.fx * (1.0f - g.fy), (1.0f - g.fx) * g.fy, g.fx * g.fy};
      const int64_t tap[4] = {g.t00, g.t00 + 1, g.t00 + v.Ws, g.t00 + v.Ws + 1};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        // z_s = D_s / alpha_s
        const float dzs = w[t] * dzo;
        // gradient-only quotients: the fast division (within 2 ulp; alpha_s >= eps)
        const float dD = __fdividef(dzs, g.as[t]);
        if (v.io.d_sun_depth) atomicAdd(v.io.d_sun_depth + tap[t], dD);
        if (v.io.d_sun_alpha) atomicAdd(v.io.d_sun_alpha + tap[t], -dD * g.zs[t]);
      }
      // u = S (x - h B' s): du/dh = -S B' s, du/dB'_ij = -S h s_j
      const float dh = -v.S * (dux * g.Bs0 + duy * g.Bs1);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        acc[3 + j] = -v.S * g.h * v.s[j] * dux;
        acc[6 + j] = -v.S * g.h * v.s[j] * duy;
      }
      // h = max_alt - z, z = D / alpha
      const float dz = d_delta - dh;
      const float dDp = __fdividef(dz, g.a);  // gradient only; alpha >= eps
      if (v.io.d_depth) v.io.d_depth[pix] = gz + dDp;
      if (v.io.d_alpha) v.io.d_alpha[pix] = ga + -dDp * g.z;
    }
  }
  // block sums, one atomic per field and block
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  {
    // the nine warp sums by the transposed butterfly (15 shuffles instead of 45): even lane 2f
    // ends with field f
    float v16[16];
#pragma unroll
    for (int f = 0; f < 16; ++f) v16[f] = f < 9 ? acc[f] : 0.0f;
    const float tot = warp_reduce16_transposed(v16);
    if (!(lane & 1) && (lane >> 1) < 9) red[warp][lane >> 1] = tot;
  }
  __syncthreads();
  if (threadIdx.x < 9) {
    float s = 0.0f;
    for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) s += red[w2][threadIdx.x];
    const int f = threadIdx.x;
    if (s != 0.0f) {
      if (f < 3) {
        if (p.d_La) atomicAdd(p.d_La + 3 * cam + f, s);
      } else if (p.d_dF) {
        const int i = (f - 3) / 3, j = (f - 3) % 3;
        atomicAdd(p.d_dF + 8 * cam + 4 * i + j, s);
      }
    }
  }
}

namespace {

bool fin(float x) { return std::isfinite(x); }

ss_status fill_shade(ShadeParams& p, const ss_camera* cams, int32_t n_cams, const float* dF, const float* La,
                     const ss_shade_opts* o, const ss_shade_io* io, bool bwd) {
  if (!cams || !io || !o || !La || n_cams < 1 || n_cams > kMaxCams) return SS_ERR_INVALID_ARG;
  if (!fin(o->esm_k) || !(o->esm_k >= 0.0f) || !fin(o->esm_bias) || !fin(o->alpha_eps) || !(o->alpha_eps > 0.0f))
    return SS_ERR_INVALID_ARG;
  std::memset(&p, 0, sizeof(p));
  for (int c = 0; c < n_cams; ++c) {
    const ss_camera& k = cams[c];
    const ss_shade_io& q = io[c];
    if (k.width < 1 || k.height < 1 || k.width > 16384 || k.height > 16384) return SS_ERR_INVALID_ARG;
    if (k.shadow_w < 2 || k.shadow_h < 2 || k.shadow_w > 16384 || k.shadow_h > 16384) return SS_ERR_INVALID_ARG;
    if (!fin(k.sun_phi) || !fin(k.sun_theta) || !(k.sun_theta > 0.0f) || !(k.sun_theta <= 1.5707964f))
      return SS_ERR_INVALID_ARG;
    if (!fin(k.shadow_scale) || !(k.shadow_scale > 0.0f) || !fin(k.max_alt)) return SS_ERR_INVALID_ARG;
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 4; ++j)
        if (!fin(k.F_xy[i][j])) return SS_ERR_INVALID_ARG;
    if (!q.rgb || !q.depth || !q.alpha || !q.sun_depth || !q.sun_alpha) return SS_ERR_INVALID_ARG;
    if (!bwd && !q.image) return SS_ERR_INVALID_ARG;
    if (bwd && !q.d_image) return SS_ERR_INVALID_ARG;
    ShadeView& v = p.v[c];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 3; ++j) v.B[i][j] = k.F_xy[i][j];
    const double ct = 1.0 / std::tan((double)k.sun_theta);
    v.s[0] = (float)(std::cos((double)k.sun_phi) * ct);
    v.s[1] = (float)(std::sin((double)k.sun_phi) * ct);
    v.s[2] = 1.0f;
    v.S = k.shadow_scale;
    v.maxalt = k.max_alt;
    v.W = k.width;
    v.H = k.height;
    v.Ws = k.shadow_w;
    v.Hs = k.shadow_h;
    v.io = q;
    auto al = [](const void* ptr) { return ptr == nullptr || (reinterpret_cast<uintptr_t>(ptr) & 15u) == 0; };
    v.vec4 = ((int64_t)k.width * k.height) % 4 == 0 && al(q.rgb) && al(q.depth) && al(q.alpha) && al(q.image) &&
             al(q.vis) && al(q.d_image) && al(q.d_rgb);
  }
  p.dF = dF;
  p.La = La;
  p.k = o->esm_k;
  p.bias = o->esm_bias;
  p.eps = o->alpha_eps;
  return SS_OK;
}

dim3 shade_grid(const ss_camera* cams, int32_t n_cams, int pix_per_thread) {
  int64_t most = 0;
  for (int c = 0; c < n_cams; ++c) most = std::max(most, (int64_t)cams[c].width * cams[c].height);
  const int64_t threads = (most + pix_per_thread - 1) / pix_per_thread;
  return dim3((unsigned)((threads + 255) / 256), (unsigned)n_cams);
}

}  // namespace
}  // namespace ss

using namespace ss;

extern "C" {

void ss_default_shade_opts(ss_shade_opts* o) {
  if (!o) return;
  o->esm_k = 2000.0f;
  o->esm_bias = 0.0f;
  o->alpha_eps = 1e-3f;
}

ss_status ss_shade_fwd(const ss_camera* cams, int32_t n_cams, const float* dF, const float* La,
                       const ss_shade_opts* opts, const ss_shade_io* io, ss_stream_t stream) {
  ShadeParams p;
  ss_status e = fill_shade(p, cams, n_cams, dF, La, opts, io, false);
  if (e != SS_OK) return e;
  count_launch();
  shade_fwd_kernel<<<shade_grid(cams, n_cams, kShadePix), 256, 0, (cudaStream_t)stream>>>(p);
  return cudaGetLastError() == cudaSuccess ? SS_OK : SS_ERR_CUDA;
}

ss_status ss_shade_bwd(const ss_camera* cams, int32_t n_cams, const float* dF, const float* La,
                       const ss_shade_opts* opts, const ss_shade_io* io, float* d_La, float* d_dF,
                       ss_stream_t stream) {
  ShadeParams p;
  ss_status e = fill_shade(p, cams, n_cams, dF, La, opts, io, true);
  if (e != SS_OK) return e;
  p.d_La = d_La;
  p.d_dF = d_dF;
  count_launch();
  shade_bwd_kernel<<<shade_grid(cams, n_cams, 1), 256, 0, (cudaStream_t)stream>>>(p);
  return cudaGetLastError() == cudaSuccess ? SS_OK : SS_ERR_CUDA;
}

}  // extern "C"
