// Depth-gradient surface normal (K8), Sec. 3.2 Eq. surface_normal, and its adjoint.
//
// Blocks of 32 x 8 threads over tiles of 32 x 32 pixels; every view in one launch (blockIdx.y =
// view), and each block loops over tiles of its view, about as many blocks as the SMs hold at
// once (one block per tile measured slower).  The point map
// p_s = (X, Y, h) is affine in the pixel and in the height, so its central differences are
//   grad_x p_s = a1 + (h(i+1) - h(i-1)) G,  grad_y p_s = a2 + (h(j+1) - h(j-1)) G,
// with per-view a1 = (2 A^-1 e1, 0), a2 = (2 A^-1 e2, 0), G = (-A^-1 B'[:, 2], 1), A = B'[:, 0:2].
// Forming them this way never subtracts two absolute world positions (which FP32 would round at
// ~1e-7 of the scene size, far above a pixel's footprint).  Per pixel the forward reads depth and
// alpha once (a halo from L2) and writes 3 values: HBM-bound.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "kernels.cuh"

namespace ss {
int device_sm_count();  // SMs of the current device (cached)

struct NormalView {
  float F[2][4];  // host F_xy; dF is added on the device
  float maxalt;
  int32_t W, H;
  ss_dnormal_io io;
};

struct NormalParams {
  NormalView v[kMaxCams];
  const float* dF;  // [V][8] or null
  float* d_dF;      // [V][8] or null
  float eps;
};

// Per-view constants from B' = F'[:, 0:3].
struct NormalCam {
  float Ai[2][2];  // A^-1
  float B2[2];     // B'[:, 2]
  float Gx, Gy;    // G_xy = -A^-1 B'[:, 2]
  float sgn;       // sign(det A)
};

__device__ __forceinline__ NormalCam normal_cam(const NormalParams& p, const NormalView& v, int cam) {
  const float* dF = p.dF ? p.dF + 8 * cam : nullptr;
  float B[2][3];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) B[i][j] = v.F[i][j] + (dF ? dF[4 * i + j] : 0.0f);
  NormalCam c;
  const float det = B[0][0] * B[1][1] - B[0][1] * B[1][0];
  const float id = 1.0f / det;
  c.Ai[0][0] = B[1][1] * id;
  c.Ai[0][1] = -B[0][1] * id;
  c.Ai[1][0] = -B[1][0] * id;
  c.Ai[1][1] = B[0][0] * id;
  c.B2[0] = B[0][2];
  c.B2[1] = B[1][2];
  c.Gx = -(c.Ai[0][0] * c.B2[0] + c.Ai[0][1] * c.B2[1]);
  c.Gy = -(c.Ai[1][0] * c.B2[0] + c.Ai[1][1] * c.B2[1]);
  c.sgn = det < 0.0f ? -1.0f : 1.0f;
  return c;
}

// Tiles of kNX x kNY pixels per block of kNX x 8 threads, kRows rows per thread.  The
// alpha-normalised depth z of the tile and a halo is staged in shared memory (NaN where there is
// no surface or no pixel), so each pixel's z is formed once instead of once per neighbour that
// needs it.  A thread issues all its staging loads of a phase (about five slots, alpha and
// depth together) before it uses any: these passes are bound by the bytes each SM keeps in
// flight, and a tile of 32 x 8 pixels with one load pair per thread kept too few.
constexpr int kNX = 32, kNY = 32, kThreads = kNX * 8, kRows = kNY / 8;
// resident blocks of the backward: its threads hold five slots of d_normal in registers
constexpr int kNormalBwdBlocks = 4;

template <int HALO>
struct Slots {
  static constexpr int W = kNX + 2 * HALO, N = (kNY + 2 * HALO) * W, PER = (N + kThreads - 1) / kThreads;
};

// z of the tile at (x0, y0) and its halo of HALO pixels into sz (and alpha into sa when given)
template <int HALO, int SX>
__device__ __forceinline__ void stage_z(const NormalView& v, int x0, int y0, float eps, float (*sz)[SX],
                                        float (*sa)[SX] = nullptr) {
  constexpr int PER = Slots<HALO>::PER;
  float a[PER], d[PER];
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const int k = threadIdx.x + r * kThreads;
    a[r] = 0.0f;  // no pixel: no surface
    d[r] = 0.0f;
    if (k < Slots<HALO>::N) {
      const int ty = k / Slots<HALO>::W, tx = k - ty * Slots<HALO>::W;
      const int x = x0 - HALO + tx, y = y0 - HALO + ty;
      if (x >= 0 && y >= 0 && x < v.W && y < v.H) {
        const int64_t i = (int64_t)y * v.W + x;
        a[r] = v.io.alpha[i];
        d[r] = v.io.depth[i];
      }
    }
  }
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const int k = threadIdx.x + r * kThreads;
    if (k < Slots<HALO>::N) {
      const int ty = k / Slots<HALO>::W, tx = k - ty * Slots<HALO>::W;
      sz[ty][tx] = a[r] >= eps ? d[r] / a[r] : __int_as_float(0x7fc00000);
      if (sa) sa[ty][tx] = a[r];
    }
  }
}

// u = grad_x p_s and v = grad_y p_s from the height differences dhx = z(i-1) - z(i+1) and
// dhy = z(j-1) - z(j+1) (h = max_alt - z).
struct NormalUV {
  float ux, uy, uz, vx, vy, vz;
};
__device__ __forceinline__ NormalUV normal_uv(const NormalCam& c, float dhx, float dhy) {
  NormalUV r;
  r.ux = 2.0f * c.Ai[0][0] + dhx * c.Gx;
  r.uy = 2.0f * c.Ai[1][0] + dhx * c.Gy;
  r.uz = dhx;
  r.vx = 2.0f * c.Ai[0][1] + dhy * c.Gx;
  r.vy = 2.0f * c.Ai[1][1] + dhy * c.Gy;
  r.vz = dhy;
  return r;
}

__global__ void __launch_bounds__(kThreads) depth_normal_fwd_kernel(const __grid_constant__ NormalParams p) {
  __shared__ float sz[kNY + 2][kNX + 3];
  const int cam = blockIdx.y;
  const NormalView& v = p.v[cam];
  const int bxs = (v.W + kNX - 1) / kNX;
  const int ntiles = bxs * ((v.H + kNY - 1) / kNY);
  const NormalCam c = normal_cam(p, v, cam);
  const int64_t hw = (int64_t)v.W * v.H;
  const int tx = threadIdx.x % kNX, ty0 = threadIdx.x / kNX;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int by = tile / bxs, bx = tile - by * bxs;
    const int x0 = bx * kNX, y0 = by * kNY;
    __syncthreads();  // the previous tile's reads of sz are done
    stage_z<1>(v, x0, y0, p.eps, sz);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kRows; ++j) {
      const int ty = ty0 + 8 * j;
      const int px = x0 + tx, py = y0 + ty;
      if (px >= v.W || py >= v.H) continue;
      const float zc = sz[ty + 1][tx + 1], zl = sz[ty + 1][tx], zr = sz[ty + 1][tx + 2], zu = sz[ty][tx + 1],
                  zd = sz[ty + 2][tx + 1];
      float n[3] = {0.0f, 0.0f, 0.0f};
      // a NaN (no surface, or outside the view) anywhere leaves the normal at 0
      if (!(isnan(zc) || isnan(zl) || isnan(zr) || isnan(zu) || isnan(zd))) {
        const NormalUV q = normal_uv(c, zl - zr, zu - zd);
        n[0] = q.uy * q.vz - q.uz * q.vy;
        n[1] = q.uz * q.vx - q.ux * q.vz;
        n[2] = q.ux * q.vy - q.uy * q.vx;
        const float sc = c.sgn * rsqrtf(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        n[0] *= sc;
        n[1] *= sc;
        n[2] *= sc;
      }
      const int64_t pix = (int64_t)py * v.W + px;
#pragma unroll
      for (int k = 0; k < 3; ++k) v.io.normal[k * hw + pix] = n[k];
    }
  }
}

// Gather form of the backward: a pixel's depth enters the normals of its four neighbours
// (dhx = z(i-1) - z(i+1), dhy = z(j-1) - z(j+1)), so its gradient is
// ddhx(i+1) - ddhx(i-1) + ddhy(j+1) - ddhy(j-1).  The block forms ddhx, ddhy once for the tile
// and a halo of one pixel (from z staged with a halo of two), then every pixel gathers.  Each
// block loops over several tiles of its view (blockIdx.x, + gridDim.x, ...) and adds its
// per-view sums to the camera gradient once.
__global__ void __launch_bounds__(kThreads, kNormalBwdBlocks) depth_normal_bwd_kernel(
    const __grid_constant__ NormalParams p) {
  __shared__ float sz[kNY + 4][kNX + 5], sa[kNY + 4][kNX + 5];
  __shared__ float sdx[kNY + 2][kNX + 3], sdy[kNY + 2][kNX + 3];
  __shared__ float red[kThreads / 32][8];
  const int cam = blockIdx.y;
  const NormalView& v = p.v[cam];
  const int bxs = (v.W + kNX - 1) / kNX;
  const int ntiles = bxs * ((v.H + kNY - 1) / kNY);
  const int64_t hw = (int64_t)v.W * v.H;
  const NormalCam c = normal_cam(p, v, cam);
  // per-view sums over the tiles' own pixels: d A^-1 (4) and d G_xy (2)
  float acc[6] = {0, 0, 0, 0, 0, 0};
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
  const int by = tile / bxs, bx = tile - by * bxs;
  const int x0 = bx * kNX, y0 = by * kNY;
  __syncthreads();  // the previous tile's reads of the shared planes are done
  // d_normal at the thread's halo-1 positions, issued with the staging loads below (both are
  // in flight together) and loaded before any is used
  constexpr int PER1 = Slots<1>::PER;
  float dn[PER1][3];
#pragma unroll
  for (int r = 0; r < PER1; ++r) {
    const int k = threadIdx.x + r * kThreads;
    dn[r][0] = dn[r][1] = dn[r][2] = 0.0f;
    if (k < Slots<1>::N) {
      const int ty = k / Slots<1>::W, tx = k - ty * Slots<1>::W;
      const int px = x0 - 1 + tx, py = y0 - 1 + ty;
      if (px >= 0 && py >= 0 && px < v.W && py < v.H) {
        const int64_t pix = (int64_t)py * v.W + px;
#pragma unroll
        for (int j = 0; j < 3; ++j) dn[r][j] = v.io.d_normal[j * hw + pix];
      }
    }
  }
  stage_z<2>(v, x0, y0, p.eps, sz, sa);
  __syncthreads();
#pragma unroll
  for (int r = 0; r < PER1; ++r) {
    const int k = threadIdx.x + r * kThreads;
    if (k >= Slots<1>::N) break;
    const int ty = k / Slots<1>::W, tx = k - ty * Slots<1>::W;  // halo-1 coordinates
    const float zc = sz[ty + 1][tx + 1], zl = sz[ty + 1][tx], zr = sz[ty + 1][tx + 2], zu = sz[ty][tx + 1],
                zd = sz[ty + 2][tx + 1];
    float ddhx = 0.0f, ddhy = 0.0f;
    if (!(isnan(zc) || isnan(zl) || isnan(zr) || isnan(zu) || isnan(zd))) {
      const float dhx = zl - zr, dhy = zu - zd;
      const NormalUV q = normal_uv(c, dhx, dhy);
      const float n[3] = {q.uy * q.vz - q.uz * q.vy, q.uz * q.vx - q.ux * q.vz, q.ux * q.vy - q.uy * q.vx};
      const float inv = rsqrtf(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
      const float N[3] = {n[0] * inv, n[1] * inv, n[2] * inv};  // unsigned unit normal
      const float* dN = dn[r];
      // N_out = sgn n / |n|: dn = sgn (dN - N (N . dN)) / |n|
      const float nd = N[0] * dN[0] + N[1] * dN[1] + N[2] * dN[2];
      float dc[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) dc[j] = c.sgn * (dN[j] - N[j] * nd) * inv;
      // n = u x v: du = v x dc, dv = dc x u
      const float dux = q.vy * dc[2] - q.vz * dc[1], duy = q.vz * dc[0] - q.vx * dc[2],
                  duz = q.vx * dc[1] - q.vy * dc[0];
      const float dvx = dc[1] * q.uz - dc[2] * q.uy, dvy = dc[2] * q.ux - dc[0] * q.uz,
                  dvz = dc[0] * q.uy - dc[1] * q.ux;
      // u = a1 + dhx G, v = a2 + dhy G, G = (Gx, Gy, 1)
      ddhx = dux * c.Gx + duy * c.Gy + duz;
      ddhy = dvx * c.Gx + dvy * c.Gy + dvz;
      if (tx >= 1 && tx <= kNX && ty >= 1 && ty <= kNY) {
        // the tile's own pixel: a1 = 2 A^-1[:, 0], a2 = 2 A^-1[:, 1]
        acc[0] += 2.0f * dux;  // d A^-1[0][0]
        acc[1] += 2.0f * dvx;  // d A^-1[0][1]
        acc[2] += 2.0f * duy;  // d A^-1[1][0]
        acc[3] += 2.0f * dvy;  // d A^-1[1][1]
        acc[4] += dhx * dux + dhy * dvx;  // d G_x
        acc[5] += dhx * duy + dhy * dvy;  // d G_y
      }
    }
    sdx[ty][tx] = ddhx;
    sdy[ty][tx] = ddhy;
  }
  __syncthreads();
  {
    // the thread's kRows pixels: every load first, then the read-modify-writes (a store could
    // alias a later row's loads, so loads interleaved with stores would wait on each other).
    // z = D / alpha (a pixel that feeds a normal has a surface): dD = dz / alpha and
    // d alpha = -dz D / alpha^2 = -dD z, with alpha and z from the staged tile
    const int tx = threadIdx.x % kNX, ty0 = threadIdx.x / kNX;
    float dz[kRows], gd[kRows], ga[kRows];
#pragma unroll
    for (int j = 0; j < kRows; ++j) {
      const int ty = ty0 + 8 * j;
      const int px = x0 + tx, py = y0 + ty;
      dz[j] = 0.0f;
      if (px < v.W && py < v.H)
        dz[j] = sdx[ty + 1][tx + 2] - sdx[ty + 1][tx] + sdy[ty + 2][tx + 1] - sdy[ty][tx + 1];
      gd[j] = ga[j] = 0.0f;
      if (dz[j] != 0.0f) {
        const int64_t pix = (int64_t)py * v.W + px;
        if (v.io.d_depth) gd[j] = v.io.d_depth[pix];
        if (v.io.d_alpha) ga[j] = v.io.d_alpha[pix];
      }
    }
#pragma unroll
    for (int j = 0; j < kRows; ++j) {
      if (dz[j] == 0.0f) continue;
      const int ty = ty0 + 8 * j;
      const int64_t pix = (int64_t)(y0 + ty) * v.W + x0 + tx;
      const float dD = __fdividef(dz[j], sa[ty + 2][tx + 2]);  // gradient only; alpha >= eps
      if (v.io.d_depth) v.io.d_depth[pix] = gd[j] + dD;
      if (v.io.d_alpha) v.io.d_alpha[pix] = ga[j] + -dD * sz[ty + 2][tx + 2];
    }
  }
  }  // tiles
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    float x = acc[f];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[warp][f] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0 && p.d_dF) {
    float s[6] = {0, 0, 0, 0, 0, 0};
    for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2)
      for (int f = 0; f < 6; ++f) s[f] += red[w2][f];
    // G_xy = -A^-1 B2: d A^-1 -= dG B2^T, d B2 = -A^-T dG
    float dAi[2][2] = {{s[0] - s[4] * c.B2[0], s[1] - s[4] * c.B2[1]},
                       {s[2] - s[5] * c.B2[0], s[3] - s[5] * c.B2[1]}};
    const float dB2[2] = {-(c.Ai[0][0] * s[4] + c.Ai[1][0] * s[5]), -(c.Ai[0][1] * s[4] + c.Ai[1][1] * s[5])};
    // A^-1 = inv(A): dA = -A^-T dA^-1 A^-T
    float t[2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) t[i][j] = c.Ai[0][i] * dAi[0][j] + c.Ai[1][i] * dAi[1][j];
    float* d = p.d_dF + 8 * cam;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const float dA = -(t[i][0] * c.Ai[j][0] + t[i][1] * c.Ai[j][1]);
        if (dA != 0.0f) atomicAdd(d + 4 * i + j, dA);
      }
      if (dB2[i] != 0.0f) atomicAdd(d + 4 * i + 2, dB2[i]);
    }
  }
}

namespace {

ss_status fill_normal(NormalParams& p, const ss_camera* cams, int32_t n_cams, const float* dF, float eps,
                      const ss_dnormal_io* io, bool bwd) {
  if (!cams || !io || n_cams < 1 || n_cams > kMaxCams || !std::isfinite(eps) || !(eps > 0.0f))
    return SS_ERR_INVALID_ARG;
  std::memset(&p, 0, sizeof(p));
  for (int c = 0; c < n_cams; ++c) {
    const ss_camera& k = cams[c];
    const ss_dnormal_io& q = io[c];
    if (k.width < 1 || k.height < 1 || k.width > 16384 || k.height > 16384 || !std::isfinite(k.max_alt))
      return SS_ERR_INVALID_ARG;
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 4; ++j) {
        if (!std::isfinite(k.F_xy[i][j])) return SS_ERR_INVALID_ARG;
        p.v[c].F[i][j] = k.F_xy[i][j];
      }
    if (!q.depth || !q.alpha) return SS_ERR_INVALID_ARG;
    if (!bwd && !q.normal) return SS_ERR_INVALID_ARG;
    if (bwd && !q.d_normal) return SS_ERR_INVALID_ARG;
    p.v[c].maxalt = k.max_alt;
    p.v[c].W = k.width;
    p.v[c].H = k.height;
    p.v[c].io = q;
  }
  p.dF = dF;
  p.eps = eps;
  return SS_OK;
}

dim3 normal_grid(const ss_camera* cams, int32_t n_cams) {
  int64_t most = 0;
  for (int c = 0; c < n_cams; ++c)
    most = std::max(most, (int64_t)((cams[c].width + kNX - 1) / kNX) * ((cams[c].height + kNY - 1) / kNY));
  return dim3((unsigned)most, (unsigned)n_cams);
}

// as many blocks in all as the SMs hold at once, each looping over tiles of its view
template <class K>
dim3 normal_loop_grid(const ss_camera* cams, int32_t n_cams, K kernel, int& per_sm) {
  if (per_sm == 0) {
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kernel, kThreads, 0) != cudaSuccess || v < 1) v = 1;
    per_sm = v;
  }
  const dim3 full = normal_grid(cams, n_cams);
  const int64_t want = ((int64_t)device_sm_count() * per_sm + n_cams - 1) / n_cams;
  return dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>(full.x, want)), (unsigned)n_cams);
}

}  // namespace
}  // namespace ss

using namespace ss;

extern "C" {

ss_status ss_depth_normal_fwd(const ss_camera* cams, int32_t n_cams, const float* dF, float alpha_eps,
                              const ss_dnormal_io* io, ss_stream_t stream) {
  NormalParams p;
  ss_status e = fill_normal(p, cams, n_cams, dF, alpha_eps, io, false);
  if (e != SS_OK) return e;
  count_launch();
  static int per_sm = 0;
  depth_normal_fwd_kernel<<<normal_loop_grid(cams, n_cams, depth_normal_fwd_kernel, per_sm), kThreads, 0,
                            (cudaStream_t)stream>>>(p);
  return cudaGetLastError() == cudaSuccess ? SS_OK : SS_ERR_CUDA;
}

ss_status ss_depth_normal_bwd(const ss_camera* cams, int32_t n_cams, const float* dF, float alpha_eps,
                              const ss_dnormal_io* io, float* d_dF, ss_stream_t stream) {
  NormalParams p;
  ss_status e = fill_normal(p, cams, n_cams, dF, alpha_eps, io, true);
  if (e != SS_OK) return e;
  p.d_dF = d_dF;
  count_launch();
  static int per_sm = 0;
  depth_normal_bwd_kernel<<<normal_loop_grid(cams, n_cams, depth_normal_bwd_kernel, per_sm), kThreads, 0,
                            (cudaStream_t)stream>>>(p);
  return cudaGetLastError() == cudaSuccess ? SS_OK : SS_ERR_CUDA;
}

}  // extern "C"
