// Shared device-side definitions of the GB300 affine 2DGS rasterizer.
//
// Data layout in HBM (one frame = one workspace):
//   TargetCam   [T]                 assembled camera of every render target
//   geom        [T][n_pad] 3 x f4   cx, cy, cx_lo, cy_lo | Q00 Q01 Q10 Q11 | lno, ex(sign=degenerate), ey, zc
//   feat        [T][n_pad] 2 x f4   dzdu, dzdv, nx, ny | nz, C rgb
//               (degenerate splats: Q = kDegenerateQ I, dzdu = dzdv = 0)
//   rect        [T][n_pad] 4 x u16  tile rectangle x0, y0, x1, y1 (empty: x0 > x1)
//   grad        [T][n_pad] 16 f32   d(loss)/d of the projected quantities (see GradField)
//   lists       capacity x (tile key u32, splat index u32), sorted by tile, then front to back
//   ranges      [total tiles] uint2 [start, end) into the lists
// The projected centre is kept as an unevaluated float pair (hi + lo): it is about
// 10^3 px in magnitude while the per-pixel offset x - c must be accurate to ~1e-7 px.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "satsplat.h"

namespace ss {

constexpr int kMaxCams = 64;
constexpr int kMaxTargets = 2 * kMaxCams;
constexpr int kGradFields = 16;

// Per-(target, splat) gradient record fields.
enum GradField {
  GF_Q00 = 0, GF_Q01, GF_Q10, GF_Q11,  // d/dQ
  GF_CX, GF_CY,                        // d/dc (projected centre)
  GF_LNO,                              // d/d(log opacity)
  GF_ZC, GF_DZDU, GF_DZDV,             // d/d(depth at centre, depth slopes)
  GF_NX, GF_NY, GF_NZ,                 // d/d(normal after the flip)
  GF_R, GF_G, GF_B                     // d/d(rgb)
};

// Status block at the start of the workspace (256 bytes).
struct StatusBlock {
  unsigned long long n_isect;    // intersections the frame needs
  unsigned long long nonfinite;  // splats culled for non-finite values
  unsigned int flags;            // bit 0 overflow, bit 1 timeout
  unsigned int work_fwd;         // persistent work-queue counters
  unsigned int work_bwd;
  unsigned int n_isect32;        // min(n_isect, capacity): the count the sort kernels use
  unsigned long long n_walked;   // (pixel, splat) pairs the forward walked with alpha >= alpha_min
  unsigned int pad[54];
};
static_assert(sizeof(StatusBlock) == 256, "status block size");

enum { FLAG_OVERFLOW = 1, FLAG_TIMEOUT = 2 };

// Assembled camera of one render target (written on the device by the assembly kernel).
struct __align__(16) TargetCam {
  float B[2][3];    // F'_xy screen block, rounded
  float Blo[2][3];  // rounding residual of F + dF
  float b[2];
  float blo[2];
  float maxalt;     // b_z
  float vs[3];      // unit viewing direction toward the sensor (z >= 0)
  float S;          // sun view: pixels per main-view pixel (1 for main views)
  float s[3];       // sun view: flattening direction (cos phi/tan th, sin phi/tan th, 1); 0 for main
  int32_t W, H, tiles_x, tiles_y;
  int32_t tile_base;
  int32_t cam, sun, pad;
  float C[12];      // colour correction [C | c] row-major (identity for sun views)
};

// Host-known static part of a target.
struct TargetStatic {
  int32_t W, H, tiles_x, tiles_y, tile_base, cam, sun;
  float S;
};

struct CamRaw {
  float F[8];
  float max_alt, phi, theta;
};

struct TargetIO {
  float* rgb;
  float* depth;
  float* normal;
  float* alpha;
  float* T_final;
  uint32_t* last;
  const float* d_rgb;
  const float* d_depth;
  const float* d_normal;
  const float* d_alpha;
  float* distort;            // distortion of the blending weights (forward output)
  const float* d_distort;    // its upstream (backward)
};

// ---------------------------------------------------------------- error-free transforms
// Knuth's two-sum and the FMA two-product (exact rounding residuals).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}
// (hi, lo) += a * b for a float-float accumulator, a = ah + al, b = bh + bl
__device__ __forceinline__ void ff_fma(float& hi, float& lo, float ah, float al, float bh, float bl) {
  float p, pe;
  two_prod(ah, bh, p, pe);
  float s, se;
  two_sum(hi, p, s, se);
  lo = __fadd_rn(lo, __fadd_rn(se, __fadd_rn(pe, __fmaf_rn(ah, bl, __fmul_rn(al, bh)))));
  hi = s;
}
__device__ __forceinline__ void ff_renorm(float& hi, float& lo) {
  float s, e;
  two_sum(hi, lo, s, e);
  hi = s;
  lo = e;
}

// 2x2 determinant a*d - b*c with Kahan's FMA scheme (error ~1.5 ulp even under cancellation).
__device__ __forceinline__ float det2(float a, float b, float c, float d) {
  float w = __fmul_rn(b, c);
  float e = __fmaf_rn(-b, c, w);
  float f = __fmaf_rn(a, d, -w);
  return __fadd_rn(f, e);
}

// ---------------------------------------------------------------- storage loads
__device__ __forceinline__ float load_attr(const float* p, int64_t i) { return __ldg(p + i); }
__device__ __forceinline__ float load_attr(const __nv_bfloat16* p, int64_t i) {
  return __bfloat162float(p[i]);
}

// Order-preserving map of a float to uint32 (ascending).
__device__ __forceinline__ uint32_t float_order(float x) {
  uint32_t u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// ---------------------------------------------------------------- per-pixel evaluation
// The one definition of a splat's alpha at a pixel, shared by the forward and the
// backward kernels so that both take every threshold decision identically.
//
// A degenerate splat (|det M| below det_eps) is drawn by the screen-space term alone.  Its
// projected record carries Q = kDegenerateQ I and zero depth slopes instead of a flag: then
// |Q (x - c)|^2 is at least 10^36 |x - c|^2 (or +inf), so the uv term never exceeds the
// screen term, and at x = c, where both are 0, either choice gives the same alpha.  u and v
// stay finite (|x - c| is bounded by the splat's extent), so w * u never forms inf * 0.
constexpr float kDegenerateQ = 1e18f;

struct EvalConsts {
  float inv2s2;   // 1 / (2 sigma^2)
  float amin, amax;
  float c_uv;     // -log2(e) / 2: log2 G(u) = c_uv |u|^2
  float c_xy;     // -log2(e) / (2 sigma^2): log2 of the screen-space term = c_xy |x - c|^2
};

constexpr float kLog2e = 1.4426950408889634f;

// 2^x and 1/x on the MUFU unit (PTX ex2.approx.ftz / rcp.approx.ftz, a few ulp): o G^ is formed
// as 2^(log2 o + log2 G^), using e^y = 2^(y log2 e); subnormal results flush to zero, far below
// alpha_min.  The reciprocal is taken of 1 - alpha in [1 - alpha_max, 1].
__device__ __forceinline__ float ex2_ftz(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_ftz(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// sqrt(x) on the MUFU unit (PTX sqrt.approx.ftz), a few ulp: the footprint tests' slack covers it.
__device__ __forceinline__ float sqrt_ftz(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ---------------------------------------------------------------- warp reductions
// Transposed warp reduction of 16 values: lanes 2f and 2f + 1 end with the warp sum of field f
// (16 shuffles instead of 80 for 16 separate reductions).
__device__ __forceinline__ float warp_reduce16_transposed(float v[16]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const bool up = lane & 16;
    const float send = up ? v[i] : v[i + 8];
    const float keep = up ? v[i + 8] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const bool up = lane & 8;
    const float send = up ? v[i] : v[i + 4];
    const float keep = up ? v[i + 4] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const bool up = lane & 4;
    const float send = up ? v[i] : v[i + 2];
    const float keep = up ? v[i + 2] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  {
    const bool up = lane & 2;
    const float send = up ? v[0] : v[1];
    const float keep = up ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
  return v[0];
}

// ---------------------------------------------------------------- footprint culling
// The support of a splat is {alpha >= alpha_min}: the ellipse |Q (x - c)|^2 <= r2 united with the
// disc |x - c|^2 <= sigma^2 r2, r2 = 2 (ln o - ln alpha_min).  The binning keeps the tiles of a
// splat's rectangle that the support can reach, and the rasterizer the sub-blocks of a tile; both
// test the support conservatively, with slack far above the FP32 error of the pair evaluation,
// so that no pair the evaluation accepts is ever dropped.
struct CullConsts {
  float ln_amin;
  float sigma2;  // sigma^2
};

// Slices of the support through bands of rows.  For a band of rows yl <= y - cy <= yh, range()
// gives an x-range, relative to cx, that holds the support's slice through the band: exact for
// the ellipse and for the disc, their union bounded by the hull of the two ranges; empty
// (lo > hi) when the band misses both.  A convex set meets a rectangle exactly when its slice
// through the rectangle's rows meets the rectangle's columns, so this tests a row of rectangles
// at once.  On the ellipse's boundary at height y, x = (-A01 y +- sqrt(A00 r2 - det(Q)^2 y^2)) / A00
// with A = Q^T Q, extreme at y = -+A01 X / A11.  Conservative: r2 is inflated by 0.2 % (far above
// the FP32 error of the slice formulas, whose square roots and quotients take the MUFU
// approximations of a few ulp, and of the pair evaluation); callers pad the rectangles by 2e-3 px
// (the centre's low part is ignored).  Degenerate splats (record ex < 0) have the disc only.
struct SupportSlices {
  float Ar2, dA, A01, iA00, Xe, Ye, yr, rd2;
  bool ell;
  __device__ __forceinline__ void init(const float4 g1, const float4 g2, const CullConsts& cc) {
    const float r2 = fmaxf(2.0f * (g2.x - cc.ln_amin), 0.0f) * 1.002f + 1e-4f;
    rd2 = r2 * cc.sigma2;
    ell = g2.y >= 0.0f;
    const float Q00 = g1.x, Q01 = g1.y, Q10 = g1.z, Q11 = g1.w;
    const float A00 = Q00 * Q00 + Q10 * Q10, A11 = Q01 * Q01 + Q11 * Q11;
    A01 = Q00 * Q01 + Q10 * Q11;
    const float dq = fabsf(det2(Q00, Q01, Q10, Q11));
    dA = dq * dq;
    Ar2 = A00 * r2;
    const float idq = rcp_ftz(dq);
    Xe = sqrt_ftz(r2 * A11) * idq;  // x half-extent of the ellipse
    Ye = sqrt_ftz(Ar2) * idq;       // y half-extent
    yr = -A01 * Xe * rcp_ftz(A11);  // height of the rightmost point (leftmost: -yr)
    iA00 = rcp_ftz(A00);
  }
  __device__ __forceinline__ void range(float yl, float yh, float& lo, float& hi) const {
    lo = INFINITY;
    hi = -INFINITY;
    if (ell && yh >= -Ye && yl <= Ye) {
      const float er = fminf(fmaxf(yr, yl), yh), el = fminf(fmaxf(-yr, yl), yh);
      const float hr = sqrt_ftz(fmaxf(Ar2 - dA * er * er, 0.0f)), hl = sqrt_ftz(fmaxf(Ar2 - dA * el * el, 0.0f));
      hi = er == yr ? Xe : (hr - A01 * er) * iA00;
      lo = el == -yr ? -Xe : (-hl - A01 * el) * iA00;
    }
    const float dy = fminf(fmaxf(0.0f, yl), yh);
    if (dy * dy <= rd2) {
      const float hw = sqrt_ftz(rd2 - dy * dy);
      lo = fminf(lo, -hw);
      hi = fmaxf(hi, hw);
    }
  }
};

// Host-side count of the kernels this library has launched (or captured into a graph).
void count_launch();

#define SS_CUDA_TRY(expr)                            \
  do {                                                 \
    cudaError_t _e = (expr);                           \
    if (_e != cudaSuccess) return SS_ERR_CUDA;         \
  } while (0)

}  // namespace ss
