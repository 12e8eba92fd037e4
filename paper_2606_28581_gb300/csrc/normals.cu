// Depth-gradient surface normal (K8), Sec. 3.2 Eq. surface_normal, and its adjoint.
//
// One thread per main-view pixel, every view in one launch (blockIdx.y = view).  The point map
// p_s = (X, Y, h) is affine in the pixel and in the height, so its central differences are
//   grad_x p_s = a1 + (h(i+1) - h(i-1)) G,  grad_y p_s = a2 + (h(j+1) - h(j-1)) G,
// with per-view a1 = (2 A^-1 e1, 0), a2 = (2 A^-1 e2, 0), G = (-A^-1 B'[:, 2], 1), A = B'[:, 0:2].
// Forming them this way never subtracts two absolute world positions (which FP32 would round at
// ~1e-7 of the scene size, far above a pixel's footprint).  Reads 5 depth and 5 alpha values per
// pixel (neighbours from L1/L2), writes 3: HBM-bound.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "kernels.cuh"

namespace ss {

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

// The normal's inputs at pixel (px, py): whether it is defined, and the two height differences.
struct NormalPix {
  bool ok;
  float dhx, dhy;   // h(i+1) - h(i-1), h(j+1) - h(j-1)
  float ux, uy, uz, vx, vy, vz;  // grad_x p_s, grad_y p_s
};

__device__ __forceinline__ NormalPix normal_pix(const NormalParams& p, const NormalView& v, const NormalCam& c,
                                                int px, int py) {
  NormalPix r;
  r.ok = false;
  r.dhx = r.dhy = 0.0f;
  if (px < 1 || py < 1 || px >= v.W - 1 || py >= v.H - 1) return r;
  const int64_t W = v.W;
  const int64_t i = (int64_t)py * W + px;
  const int64_t nb[5] = {i, i + 1, i - 1, i + W, i - W};
  float z[5];
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const float a = v.io.alpha[nb[k]];
    ok = ok && a >= p.eps;
    z[k] = a >= p.eps ? v.io.depth[nb[k]] / a : 0.0f;
  }
  if (!ok) return r;
  r.ok = true;
  // h = max_alt - z: the differences of h are the negated differences of z
  r.dhx = z[2] - z[1];
  r.dhy = z[4] - z[3];
  r.ux = 2.0f * c.Ai[0][0] + r.dhx * c.Gx;
  r.uy = 2.0f * c.Ai[1][0] + r.dhx * c.Gy;
  r.uz = r.dhx;
  r.vx = 2.0f * c.Ai[0][1] + r.dhy * c.Gx;
  r.vy = 2.0f * c.Ai[1][1] + r.dhy * c.Gy;
  r.vz = r.dhy;
  return r;
}

__global__ void __launch_bounds__(256) depth_normal_fwd_kernel(const __grid_constant__ NormalParams p) {
  const int cam = blockIdx.y;
  const NormalView& v = p.v[cam];
  const int64_t hw = (int64_t)v.W * v.H;
  const int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= hw) return;
  const int py = (int)(pix / v.W), px = (int)(pix - (int64_t)py * v.W);
  const NormalCam c = normal_cam(p, v, cam);
  const NormalPix q = normal_pix(p, v, c, px, py);
  float n[3] = {0.0f, 0.0f, 0.0f};
  if (q.ok) {
    n[0] = q.uy * q.vz - q.uz * q.vy;
    n[1] = q.uz * q.vx - q.ux * q.vz;
    n[2] = q.ux * q.vy - q.uy * q.vx;
    const float s = c.sgn * rsqrtf(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    n[0] *= s;
    n[1] *= s;
    n[2] *= s;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) v.io.normal[k * hw + pix] = n[k];
}

__global__ void __launch_bounds__(256) depth_normal_bwd_kernel(const __grid_constant__ NormalParams p) {
  __shared__ float red[8][8];
  const int cam = blockIdx.y;
  const NormalView& v = p.v[cam];
  const int64_t hw = (int64_t)v.W * v.H;
  const int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const NormalCam c = normal_cam(p, v, cam);
  // per-view sums: d A^-1 (4) and d G_xy (2), chained through A^-1 once per block
  float acc[6] = {0, 0, 0, 0, 0, 0};
  if (pix < hw) {
    const int py = (int)(pix / v.W), px = (int)(pix - (int64_t)py * v.W);
    const NormalPix q = normal_pix(p, v, c, px, py);
    if (q.ok) {
      float n[3] = {q.uy * q.vz - q.uz * q.vy, q.uz * q.vx - q.ux * q.vz, q.ux * q.vy - q.uy * q.vx};
      const float inv = rsqrtf(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
      float N[3] = {n[0] * inv, n[1] * inv, n[2] * inv};  // unsigned unit normal
      float dN[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) dN[k] = v.io.d_normal[k * hw + pix];
      // N_out = sgn n / |n|: dn = sgn (dN - N (N . dN)) / |n|
      const float nd = N[0] * dN[0] + N[1] * dN[1] + N[2] * dN[2];
      float dc[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) dc[k] = c.sgn * (dN[k] - N[k] * nd) * inv;
      // n = u x v: du = v x dc, dv = dc x u
      const float dux = q.vy * dc[2] - q.vz * dc[1], duy = q.vz * dc[0] - q.vx * dc[2],
                  duz = q.vx * dc[1] - q.vy * dc[0];
      const float dvx = dc[1] * q.uz - dc[2] * q.uy, dvy = dc[2] * q.ux - dc[0] * q.uz,
                  dvz = dc[0] * q.uy - dc[1] * q.ux;
      // u = a1 + dhx G, v = a2 + dhy G, G = (Gx, Gy, 1)
      const float ddhx = dux * c.Gx + duy * c.Gy + duz;
      const float ddhy = dvx * c.Gx + dvy * c.Gy + dvz;
      // a1 = 2 A^-1[:, 0], a2 = 2 A^-1[:, 1]
      acc[0] = 2.0f * dux;  // d A^-1[0][0]
      acc[1] = 2.0f * dvx;  // d A^-1[0][1]
      acc[2] = 2.0f * duy;  // d A^-1[1][0]
      acc[3] = 2.0f * dvy;  // d A^-1[1][1]
      acc[4] = q.dhx * dux + q.dhy * dvx;  // d G_x
      acc[5] = q.dhx * duy + q.dhy * dvy;  // d G_y
      // dhx = z(i-1) - z(i+1), dhy = z(j-1) - z(j+1); z = D / alpha
      const int64_t W = v.W;
      const int64_t nb[4] = {pix - 1, pix + 1, pix - W, pix + W};
      const float dz[4] = {ddhx, -ddhx, ddhy, -ddhy};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float a = v.io.alpha[nb[k]], D = v.io.depth[nb[k]];
        if (v.io.d_depth) atomicAdd(v.io.d_depth + nb[k], dz[k] / a);
        if (v.io.d_alpha) atomicAdd(v.io.d_alpha + nb[k], -dz[k] * D / (a * a));
      }
    }
  }
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
  for (int c = 0; c < n_cams; ++c) most = std::max(most, (int64_t)cams[c].width * cams[c].height);
  return dim3((unsigned)((most + 255) / 256), (unsigned)n_cams);
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
  depth_normal_fwd_kernel<<<normal_grid(cams, n_cams), 256, 0, (cudaStream_t)stream>>>(p);
  return cudaGetLastError() == cudaSuccess ? SS_OK : SS_ERR_CUDA;
}

ss_status ss_depth_normal_bwd(const ss_camera* cams, int32_t n_cams, const float* dF, float alpha_eps,
                              const ss_dnormal_io* io, float* d_dF, ss_stream_t stream) {
  NormalParams p;
  ss_status e = fill_normal(p, cams, n_cams, dF, alpha_eps, io, true);
  if (e != SS_OK) return e;
  p.d_dF = d_dF;
  count_launch();
  depth_normal_bwd_kernel<<<normal_grid(cams, n_cams), 256, 0, (cudaStream_t)stream>>>(p);
  return cudaGetLastError() == cudaSuccess ? SS_OK : SS_ERR_CUDA;
}

}  // extern "C"
