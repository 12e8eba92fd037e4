// Forward (K3) and backward (K4) rasterization, Sec. 3.2 Eq. rasterization.
//
// One block renders one screen tile of one target and stages the tile's sorted splat list,
// batch by batch, in shared memory.  Each warp owns an 8 x 8 pixel block made of four 4 x 4
// sub-blocks; the 8 lanes of a group own one sub-block, two pixels per lane (rows r, r + 2).
// The thread that stages a splat also forms the set of the tile's 16 sub-blocks its support can
// reach (`subblock_mask`); each group walks only the staged splats that reach its sub-block, in
// list order (forward) or reverse list order (backward), independently of the other groups.  A pixel's walk is therefore exactly
// the per-pixel definition, whatever the tile shape or schedule.  With PERSIST one launch
// sized to the GPU pulls (target, tile) items from a queue, so views of uneven size and sun
// views share a single launch.
//
// Backward: with T_i the transmittance in front of splat i and S_i the composite behind it
// (normalised to T_{i+1}), d f / d alpha_i = T_i (f_i - S_i); the alpha output adds
// T_final / (1 - alpha_i).  T_i is recovered as T_{i+1} / (1 - alpha_i) from the saved
// T_final (alpha <= alpha_max < 1 keeps the division safe); only T_final and the end of the
// walk are stored per pixel.  A lane first sums its two pixels' gradient contributions, the
// 8 lanes of a group reduce the 16 fields with a transposed butterfly (14 shuffles, each lane
// ends with 2 fields), groups meet in shared memory, and one global atomic per (tile, splat,
// field) leaves the block.
#pragma once

#include <type_traits>

#include "kernels.cuh"

namespace ss {

constexpr int kSaccStride = kGradFields + 1;  // padded rows: groups on different splats hit different banks

__device__ __forceinline__ int find_target(const TargetCam* tc, int n_targets, int tile) {
  int lo = 0, hi = n_targets - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tc[mid].tile_base <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------- paired FP32 arithmetic
// A lane's two pixels share every operation, so the forward keeps their state in float2 and
// uses the paired FP32 instructions (one issue, two IEEE round-to-nearest results), each lane
// bitwise equal to the scalar operation.
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// eval_pair (common.cuh) of one splat at a lane's two pixels (x, y.x) and (x, y.y), with the
// same operations in the same order: bitwise the same alpha and decisions as two scalar calls.
struct PairEval2 {
  float dx;                   // x - c (the lane's pixels share a column)
  float2 dy, u, v, alpha;
  bool contrib0, contrib1;    // alpha >= alpha_min
  bool uwin0, uwin1;          // the uv Gaussian won the max (ties: uv)
  bool clamped0, clamped1;    // alpha_max reached
};

__device__ __forceinline__ PairEval2 eval_pair2(const float4 g0, const float4 g1, const float4 g2, float x,
                                                float2 y, const EvalConsts& k) {
  PairEval2 e;
  const float dx = __fsub_rn(__fsub_rn(x, g0.x), g0.z);
  const float2 dy = add2(add2(y, bc2(-g0.y)), bc2(-g0.w));
  e.dx = dx;
  e.dy = dy;
  e.u = fma2(bc2(g1.y), dy, bc2(__fmul_rn(g1.x, dx)));
  e.v = fma2(bc2(g1.w), dy, bc2(__fmul_rn(g1.z, dx)));
  const float2 pu = mul2(bc2(-0.5f), fma2(e.u, e.u, mul2(e.v, e.v)));
  const float2 ps = mul2(neg2(fma2(bc2(dx), bc2(dx), mul2(dy, dy))), bc2(k.inv2s2));
  e.uwin0 = pu.x >= ps.x;
  e.uwin1 = pu.y >= ps.y;
  const float2 lp = add2(make_float2(fmaxf(pu.x, ps.x), fmaxf(pu.y, ps.y)), bc2(g2.x));
  const float og0 = __expf(lp.x), og1 = __expf(lp.y);
  e.clamped0 = og0 > k.amax;
  e.clamped1 = og1 > k.amax;
  e.alpha = make_float2(fminf(og0, k.amax), fminf(og1, k.amax));
  e.contrib0 = e.alpha.x >= k.amin;
  e.contrib1 = e.alpha.y >= k.amin;
  return e;
}

// Transposed reduction of 16 values over the 8 lanes of a group: lane gl of the group ends
// with the group sums of fields 2 gl and 2 gl + 1 (in v[0], v[1]).
__device__ __forceinline__ void group_reduce16(float v[16]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const bool up = lane & 4;
    const float send = up ? v[i] : v[i + 8];
    const float keep = up ? v[i + 8] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const bool up = lane & 2;
    const float send = up ? v[i] : v[i + 4];
    const float keep = up ? v[i + 4] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const bool up = lane & 1;
    const float send = up ? v[i] : v[i + 2];
    const float keep = up ? v[i + 2] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 1);
  }
}

// Work item of a block (forward): one block per tile, or the next item of the persistent queue.
template <bool PERSIST>
__device__ __forceinline__ bool next_item(const RasterParams& p, unsigned int* counter, int& tile, int& s_item) {
  if (!PERSIST) {
    tile = blockIdx.x;
    return true;
  }
  __syncthreads();
  if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
  __syncthreads();
  const int it = s_item;
  if (it >= p.total_tiles) return false;
  tile = p.items ? (int)p.items[it] : it;
  return true;
}

// Work items of a block (backward).  A persistent block claims its next (target, tile) item
// while it works on the current one (s_item[cur ^ 1]), so claiming needs no barrier of its own:
// the one barrier at the top of each iteration frees the shared buffers of the previous tile,
// publishes the claim made during it, and orders the claim's overwrite after every read of the
// slot.
template <bool PERSIST>
__device__ __forceinline__ bool begin_item(const RasterParams& p, unsigned int* counter, int* s_item, int& cur,
                                           int iter, int& tile) {
  __syncthreads();
  if (!PERSIST) {
    tile = blockIdx.x;
    return iter == 0;
  }
  const int it = s_item[cur];
  if (it >= p.total_tiles) return false;
  if (threadIdx.x == 0) s_item[cur ^ 1] = (int)atomicAdd(counter, 1u);
  cur ^= 1;
  tile = p.items ? (int)p.items[it] : it;
  return true;
}

// Pixels of this lane, and the tile's origin.
struct LaneGeom {
  int px;        // pixel column
  int py0;       // first pixel row; the second is py0 + 2
  float x0, y0;  // the tile's first pixel column and row
};

template <int TW, int TH>
__device__ __forceinline__ LaneGeom lane_geom(const TargetCam& cam, int tile) {
  constexpr int WBX = TW / 8;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane >> 3, gl = lane & 7;
  const int local = tile - cam.tile_base;
  const int ty = local / cam.tiles_x, tx = local - ty * cam.tiles_x;
  const int sbx = tx * TW + (warp % WBX) * 8 + (grp & 1) * 4;
  const int sby = ty * TH + (warp / WBX) * 8 + (grp >> 1) * 4;
  LaneGeom g;
  g.px = sbx + (gl & 3);
  g.py0 = sby + (gl >> 2);
  g.x0 = (float)(tx * TW);
  g.y0 = (float)(ty * TH);
  return g;
}

// The 4 x 4 sub-blocks of a tile that a splat can reach: bit (row * TW / 4 + col) is set when the
// support {alpha >= alpha_min} can contain a pixel centre of sub-block (col, row).  The support is
// the ellipse |Q d|^2 <= r2 united with the disc |d|^2 <= sigma^2 r2 (d = x - c,
// r2 = 2 (ln o - ln alpha_min)).  A convex set meets a rectangle exactly when its slice through
// the rectangle's rows meets the rectangle's columns, so per row of sub-blocks the x-range of
// each slice is formed and compared with the columns: exact for the ellipse and for the disc,
// their union bounded by the hull of the two ranges.  On the ellipse's boundary at height y,
// x = (-A01 y +- sqrt(A00 r2 - det(Q)^2 y^2)) / A00 with A = Q^T Q, extreme at y = -+A01 X / A11.
// Conservative: r2 is inflated by 0.2 % (far above the FP32 error of the slice formulas and of
// eval_pair) and the rectangles are padded by 2e-3 px (the centre's low part is ignored).
// Degenerate splats (record ex < 0) have the disc only.
template <int TW, int TH>
__device__ __forceinline__ uint32_t subblock_mask(const float4 g0, const float4 g1, const float4 g2, float x0,
                                                  float y0, const CullConsts& cc) {
  constexpr int SBX = TW / 4, SBY = TH / 4;
  constexpr float kPad = 2e-3f;
  const float r2 = fmaxf(2.0f * (g2.x - cc.ln_amin), 0.0f) * 1.002f + 1e-4f;
  const float rd2 = r2 * cc.sigma2;
  const bool ell = g2.y >= 0.0f;
  const float Q00 = g1.x, Q01 = g1.y, Q10 = g1.z, Q11 = g1.w;
  const float A00 = Q00 * Q00 + Q10 * Q10, A11 = Q01 * Q01 + Q11 * Q11, A01 = Q00 * Q01 + Q10 * Q11;
  const float dq = fabsf(det2(Q00, Q01, Q10, Q11));
  const float dA = dq * dq;
  const float Ar2 = A00 * r2;
  const float Xe = sqrtf(r2 * A11) / dq;  // x half-extent of the ellipse
  const float Ye = sqrtf(Ar2) / dq;       // y half-extent
  const float yr = -A01 * Xe / A11;       // height of the rightmost point (leftmost: -yr)
  const float iA00 = 1.0f / A00;
  // tile-relative offsets: pixel centre (x0 + i + 0.5) - cx
  const float ox = x0 + 0.5f - g0.x, oy = y0 + 0.5f - g0.y;
  uint32_t mask = 0;
#pragma unroll
  for (int b = 0; b < SBY; ++b) {
    const float yl = oy + (float)(4 * b) - kPad, yh = oy + (float)(4 * b + 3) + kPad;
    float lo = INFINITY, hi = -INFINITY;
    if (ell && yh >= -Ye && yl <= Ye) {
      const float er = fminf(fmaxf(yr, yl), yh), el = fminf(fmaxf(-yr, yl), yh);
      const float hr = sqrtf(fmaxf(Ar2 - dA * er * er, 0.0f)), hl = sqrtf(fmaxf(Ar2 - dA * el * el, 0.0f));
      hi = er == yr ? Xe : (hr - A01 * er) * iA00;
      lo = el == -yr ? -Xe : (-hl - A01 * el) * iA00;
    }
    const float dy = fminf(fmaxf(0.0f, yl), yh);
    if (dy * dy <= rd2) {
      const float hw = sqrtf(rd2 - dy * dy);
      lo = fminf(lo, -hw);
      hi = fmaxf(hi, hw);
    }
    // columns c with [ox + 4c, ox + 4c + 3] (padded) meeting [lo, hi]
    const float cl = fmaxf(ceilf((lo - ox - 3.0f - kPad) * 0.25f), 0.0f);
    const float ch = fminf(floorf((hi - ox + kPad) * 0.25f), (float)(SBX - 1));
    if (cl <= ch) {
      const int a = (int)cl, z = (int)ch;
      mask |= ((2u << z) - (1u << a)) << (b * SBX);
    }
  }
  return mask;
}

// Candidate masks of a whole staged batch from the per-splat sub-block masks: lane gl of a
// group ends with the group's mask of chunk gl (staged splats [32 gl, 32 gl + 32)).  Holding
// every chunk at once lets a group walk its candidates across chunk boundaries, so the groups
// of a warp stay busy until the warp's total work, not each chunk's largest group, is done.
template <int TW, int BATCH>
__device__ __forceinline__ uint32_t batch_masks(const uint32_t* smask, int nb) {
  static_assert(BATCH % 32 == 0 && BATCH / 32 <= 8, "one chunk per lane of a group");
  constexpr int WBX = TW / 8, SBX = TW / 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, grp = lane >> 3, gl = lane & 7;
  // bit of this warp's first sub-block; its groups add 0, 1, SBX, SBX + 1
  const int base = (warp / WBX) * 2 * SBX + (warp % WBX) * 2;
  uint32_t mk = 0;
#pragma unroll 1
  for (int c0 = 0; c0 < nb; c0 += 32) {
    const int i = c0 + lane;
    const uint32_t v = i < nb ? smask[i] >> base : 0u;
    const uint32_t m0 = __ballot_sync(0xffffffffu, v & 1u);
    const uint32_t m1 = __ballot_sync(0xffffffffu, (v >> 1) & 1u);
    const uint32_t m2 = __ballot_sync(0xffffffffu, (v >> SBX) & 1u);
    const uint32_t m3 = __ballot_sync(0xffffffffu, (v >> (SBX + 1)) & 1u);
    const uint32_t mine = grp == 0 ? m0 : grp == 1 ? m1 : grp == 2 ? m2 : m3;
    mk = (gl == (c0 >> 5)) ? mine : mk;
  }
  return mk;
}

// Writes a group's candidates (the set bits of its chunk masks, lane gl holding chunk gl) to the
// group's list of staged-splat indices, in list order, and returns their number.  The walk then
// reads its next splat from the list at a position that depends on the step count alone, so no
// step waits on the previous one to find its splat.  Every lane of the warp takes part.
__device__ __forceinline__ int compact_candidates(uint32_t mk, uint8_t* list) {
  const int gl = threadIdx.x & 7;
  const int c = __popc(mk);
  int inc = c;
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, inc, o, 8);
    if (gl >= o) inc += t;
  }
  const int total = __shfl_sync(0xffffffffu, inc, 7, 8);
  int pos = inc - c;
  uint32_t mm = mk;
  while (mm) {
    const int bit = __ffs(mm) - 1;
    mm &= mm - 1;
    list[pos++] = (uint8_t)(gl * 32 + bit);
  }
  __syncwarp();
  return total;
}

// ------------------------------------------------------------------------------------------
// K3 forward
// ------------------------------------------------------------------------------------------
// DIST: the distortion of the blending weights along each ray is accumulated beside the planes:
// each composited splat i adds w_i (zs_i (1 - T_i) - D'_i) = sum_{j<i} w_i w_j (z_i - z_j), with
// 1 - T_i the weight composited in front of it and D'_i the weighted depth in front of it, both
// taken relative to the depth z0 of the pixel's first composited splat (zs = z - z0).  The sum is
// unchanged by that common shift, and with it the terms are of the size of the depth differences
// rather than of the depths.  The sum is doubled when it is written.
template <int TW, int TH, int BATCH, bool PERSIST, bool DIST>
__global__ void __launch_bounds__(TW * TH / 2, 6) raster_fwd_kernel(const __grid_constant__ RasterParams p) {
  constexpr int NT = TW * TH / 2;
  static_assert(TW % 8 == 0 && TH % 8 == 0, "tiles are whole 8 x 8 warp blocks");
  __shared__ float4 sg[BATCH][3];
  __shared__ float4 sf[BATCH][2];
  __shared__ uint32_t smask[BATCH];
  __shared__ uint8_t slist[NT / 8][BATCH + 4];  // candidates of each group (rows padded: the 4 groups of a warp read at one position from different banks)
  __shared__ int s_item;
  const int tid = threadIdx.x, lane = tid & 31;
  int tile;
  bool first = true;
  while (true) {
    if (!PERSIST && !first) break;
    first = false;
    if (!next_item<PERSIST>(p, &p.status->work_fwd, tile, s_item)) break;
    const int t = find_target(p.tcams, p.n_targets, tile);
    const TargetCam& cam = p.tcams[t];
    const LaneGeom lg = lane_geom<TW, TH>(cam, tile);
    const bool sun = cam.sun != 0;
    const float x = (float)lg.px + 0.5f;
    const uint2 range = p.ranges[tile];
    const int64_t recbase = (int64_t)t * p.n_pad;

    // the lane's two pixels (rows py0 and py0 + 2) side by side: .x and .y
    float2 T = bc2(1.0f), D = bc2(0.0f), A0 = bc2(0.0f), A1 = bc2(0.0f), A2 = bc2(0.0f), N0 = bc2(0.0f),
           N1 = bc2(0.0f), N2 = bc2(0.0f), Dst = bc2(0.0f), Dsh = bc2(0.0f), Z0f = bc2(0.0f);
    const float2 y = make_float2((float)lg.py0 + 0.5f, (float)(lg.py0 + 2) + 0.5f);
    uint32_t last0 = range.x, last1 = range.x;
    bool done0 = !(lg.px < cam.W && lg.py0 < cam.H), done1 = !(lg.px < cam.W && lg.py0 + 2 < cam.H);
    uint32_t walked = 0;  // contributing pairs, the stopping one included
    const float4 zero4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    for (uint32_t b0 = range.x; b0 < range.y; b0 += BATCH) {
      const int nb = min((int)(range.y - b0), BATCH);
      __syncthreads();
      for (int i = tid; i < nb; i += NT) {
        const int64_t rec = recbase + p.vals[b0 + i];
        const float4* g = p.geom + rec * 3;
        const float4* f = p.feat + rec * 2;
        const float4 g0 = g[0], g1 = g[1], g2 = g[2];
        sg[i][0] = g0;
        sg[i][1] = g1;
        sg[i][2] = g2;
        sf[i][0] = f[0];
        if (!sun) sf[i][1] = f[1];  // a sun view composites depth alone
        smask[i] = p.subblock_cull ? subblock_mask<TW, TH>(g0, g1, g2, lg.x0, lg.y0, p.cull) : 0xffffu;
      }
      const bool all_done = done0 && done1;
      if (__syncthreads_and(all_done)) break;
      const uint32_t mk = batch_masks<TW, BATCH>(smask, nb);
      // a group whose 16 pixels have all stopped walks nothing
      const bool gdone = ((__ballot_sync(0xffffffffu, all_done) >> (lane & 24)) & 0xffu) == 0xffu;
      const uint8_t* list = slist[tid >> 3];
      const int total = compact_candidates(gdone ? 0u : mk, slist[tid >> 3]);
      const int nsteps = (int)__reduce_max_sync(0xffffffffu, (unsigned)total);
      // two splats per step: their pair evaluations are independent; only the compositing
      // runs in order (splat a, then splat b) for each pixel.  A sun view (SUN) composites
      // depth alone: it has no colour or normal output.
      auto walk = [&](auto sun_c) {
        constexpr bool SUN = decltype(sun_c)::value;
        auto composite = [&](const PairEval2& e, bool ck0, bool ck1, const float4& g2, const float4& f0,
                             const float4& f1, uint32_t pos) {
          const float2 Tn = mul2(T, add2(bc2(1.0f), neg2(e.alpha)));
          // a splat that takes T below t_min ends the walk and is not composited
          const bool stop0 = ck0 && Tn.x < p.t_min, stop1 = ck1 && Tn.y < p.t_min;
          const bool take0 = ck0 && !stop0, take1 = ck1 && !stop1;
          const float2 aT = mul2(e.alpha, T);
          const float2 w = make_float2(take0 ? aT.x : 0.0f, take1 ? aT.y : 0.0f);
          const float2 z = fma2(bc2(f0.y), e.v, fma2(bc2(f0.x), e.u, bc2(g2.w)));
          if (DIST) {
            // z0: T is exactly 1 until the first splat is composited (alpha >= alpha_min)
            Z0f = make_float2(T.x == 1.0f ? z.x : Z0f.x, T.y == 1.0f ? z.y : Z0f.y);
            const float2 zs = add2(z, neg2(Z0f));
            Dst = fma2(w, add2(fma2(neg2(zs), T, zs), neg2(Dsh)), Dst);
            Dsh = fma2(w, zs, Dsh);
          }
          D = fma2(w, z, D);
          if (!SUN) {
            A0 = fma2(w, bc2(f1.y), A0);
            A1 = fma2(w, bc2(f1.z), A1);
            A2 = fma2(w, bc2(f1.w), A2);
            N0 = fma2(w, bc2(f0.z), N0);
            N1 = fma2(w, bc2(f0.w), N1);
            N2 = fma2(w, bc2(f1.x), N2);
          }
          T = make_float2(take0 ? Tn.x : T.x, take1 ? Tn.y : T.y);
          last0 = take0 ? pos : last0;
          last1 = take1 ? pos : last1;
          done0 = done0 || stop0;
          done1 = done1 || stop1;
        };
        for (int st = 0; st < nsteps; st += 2) {
          // lanes whose group has nothing left evaluate a stand-in and composite nothing
          const bool has_a = st < total, has_b = st + 1 < total;
          const int ja = has_a ? list[st] : 0;
          const int jb = has_b ? list[st + 1] : ja;
          const float4 ga0 = sg[ja][0], ga1 = sg[ja][1], ga2 = sg[ja][2];
          const float4 gb0 = sg[jb][0], gb1 = sg[jb][1], gb2 = sg[jb][2];
          const PairEval2 ea = eval_pair2(ga0, ga1, ga2, x, y, p.k);
          const PairEval2 eb = eval_pair2(gb0, gb1, gb2, x, y, p.k);
          const float4 fa0 = sf[ja][0], fb0 = sf[jb][0];
          const float4 fa1 = SUN ? zero4 : sf[ja][1], fb1 = SUN ? zero4 : sf[jb][1];
          const uint32_t pa = b0 + (uint32_t)ja + 1u, pb = b0 + (uint32_t)jb + 1u;
          const bool ca0 = has_a && !done0 && ea.contrib0, ca1 = has_a && !done1 && ea.contrib1;
          walked += (uint32_t)ca0 + (uint32_t)ca1;
          composite(ea, ca0, ca1, ga2, fa0, fa1, pa);
          const bool cb0 = has_b && !done0 && eb.contrib0, cb1 = has_b && !done1 && eb.contrib1;
          walked += (uint32_t)cb0 + (uint32_t)cb1;
          composite(eb, cb0, cb1, gb2, fb0, fb1, pb);
        }
      };
      if (sun) walk(std::true_type{}); else walk(std::false_type{});
    }
    const TargetIO io = p.io[t];
    const int64_t hw = (int64_t)cam.W * cam.H;
    auto pick = [](float2 v, int k) { return k == 0 ? v.x : v.y; };
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int py = lg.py0 + 2 * k;
      if (!(lg.px < cam.W && py < cam.H)) continue;
      const int64_t pix = (int64_t)py * cam.W + lg.px;
      if (io.rgb) {
        // the splats carry C rgb; the offset c completes C A + c (Sec. 3.1 Eq. image_formation)
        io.rgb[pix] = pick(A0, k) + cam.C[3];
        io.rgb[hw + pix] = pick(A1, k) + cam.C[7];
        io.rgb[2 * hw + pix] = pick(A2, k) + cam.C[11];
      }
      if (io.depth) io.depth[pix] = pick(D, k);
      if (io.normal) {
        io.normal[pix] = pick(N0, k);
        io.normal[hw + pix] = pick(N1, k);
        io.normal[2 * hw + pix] = pick(N2, k);
      }
      const float Tk = pick(T, k);
      if (io.alpha) io.alpha[pix] = 1.0f - Tk;
      if (DIST && io.distort) io.distort[pix] = 2.0f * pick(Dst, k);
      io.T_final[pix] = Tk;
      io.last[pix] = k == 0 ? last0 : last1;
    }
    // algorithmic work counter: one atomic per warp
    const unsigned int wsum = __reduce_add_sync(0xffffffffu, walked);
    if (lane == 0 && wsum) atomicAdd(&p.status->n_walked, (unsigned long long)wsum);
  }
}

// ------------------------------------------------------------------------------------------
// K4 backward
// ------------------------------------------------------------------------------------------
// DIST: the adjoint of the distortion.  With W, M the weight and the weighted depth composited
// in front of splat m and W', M' those behind it, its partial in the weight of m is
// 2 (z_m W_m - M_m) + 2 (M'_m - z_m W'_m) and in its depth 2 w_m (W_m - W'_m).  The distortion is
// unchanged by a common shift of a pixel's depths, so the walk carries them relative to the
// pixel's alpha-normalised depth z0 = D / alpha_out: every term is then of the size of the depth
// differences, not of the depths, and no difference of absolute depths is formed.  With
// W_m = alpha_out - W'_m - w_m and M_m = D' - M'_m - w_m zs_m (zs = z - z0, D' = D - z0 alpha_out)
// the weight partial is 2 (zs_m U_m + E_m) and the depth partial 2 w_m (U_m - w_m), where
// U = alpha_out - 2 W' and E = 2 M' - D' are carried along the reverse walk from the weights
// themselves (not from differences of recovered transmittances).  The weight partial joins the
// splat's per-pixel value f.
template <int TW, int TH, int BATCH, bool PERSIST, bool DIST>
// Five resident blocks (20 warps): the bound keeps every variant, the distortion's included, at
// <= 102 registers without spills.
__global__ void __launch_bounds__(TW * TH / 2, 5) raster_bwd_kernel(const __grid_constant__ RasterParams p) {
  constexpr int NT = TW * TH / 2;
  constexpr int NW = NT / 32;
  static_assert(TW % 8 == 0 && TH % 8 == 0, "tiles are whole 8 x 8 warp blocks");
  __shared__ float4 sg[BATCH][3];
  __shared__ float4 sf[BATCH][2];
  __shared__ uint32_t sk[BATCH];
  __shared__ uint32_t smask[BATCH];
  __shared__ uint8_t slist[NT / 8][BATCH + 4];  // candidates of each group (rows padded: the 4 groups of a warp read at one position from different banks)
  __shared__ float sacc[BATCH][kSaccStride];
  __shared__ float scol[NW][4];
  __shared__ int s_item[2];
  __shared__ unsigned int s_hi[2];  // per iteration parity: the tile's largest walk end
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, gl = lane & 7;
  int cur = 0, tile;
  if (tid == 0) {
    if (PERSIST) s_item[0] = (int)atomicAdd(&p.status->work_bwd, 1u);
    s_hi[0] = 0u;
  }
  for (int iter = 0;; ++iter) {
    if (!begin_item<PERSIST>(p, &p.status->work_bwd, s_item, cur, iter, tile)) break;
    const int hp = iter & 1;
    if (tid == 0) s_hi[hp ^ 1] = 0u;  // reset for the next iteration (read in this one: s_hi[hp])
    const int t = find_target(p.tcams, p.n_targets, tile);
    const TargetCam& cam = p.tcams[t];
    const LaneGeom lg = lane_geom<TW, TH>(cam, tile);
    const bool sun = cam.sun != 0;
    const float x = (float)lg.px + 0.5f;
    const uint2 range = p.ranges[tile];
    const int64_t recbase = (int64_t)t * p.n_pad;
    const TargetIO io = p.io[t];
    const int64_t hw = (int64_t)cam.W * cam.H;

    // per pixel: T (recovered backwards), the composite behind (as g . S), the upstream
    float T[2], y[2], Sg[2], gD[2], gAlT[2], gR[2][3], gN[2][3];  // gAlT: d(alpha_out) T_final
    float gDs2[2], U0[2], E[2], Z0[2];  // distortion: twice its upstream, alpha_out - 2 W', 2 M' - D', z0
    uint32_t lastp[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int py = lg.py0 + 2 * k;
      const bool inside = lg.px < cam.W && py < cam.H;
      y[k] = (float)py + 0.5f;
      T[k] = 1.0f;
      Sg[k] = gD[k] = gAlT[k] = 0.0f;
      gDs2[k] = E[k] = Z0[k] = 0.0f;
      lastp[k] = range.x;
#pragma unroll
      for (int c = 0; c < 3; ++c) gR[k][c] = gN[k][c] = 0.0f;
      if (inside) {
        const int64_t pix = (int64_t)py * cam.W + lg.px;
        T[k] = io.T_final[pix];
        // the saved end of the walk, clamped to this tile's list
        lastp[k] = min(max(io.last[pix], range.x), range.y);
        if (!sun && io.d_rgb) {
          // the splats carry C rgb, so d(rgb_out) multiplies their colour directly
          gR[k][0] = io.d_rgb[pix];
          gR[k][1] = io.d_rgb[hw + pix];
          gR[k][2] = io.d_rgb[2 * hw + pix];
        }
        if (!sun && io.d_normal) {
          gN[k][0] = io.d_normal[pix];
          gN[k][1] = io.d_normal[hw + pix];
          gN[k][2] = io.d_normal[2 * hw + pix];
        }
        if (io.d_depth) gD[k] = io.d_depth[pix];
        if (io.d_alpha) gAlT[k] = io.d_alpha[pix] * T[k];
        if (DIST && io.d_distort) {
          gDs2[k] = 2.0f * io.d_distort[pix];
          const float D = io.depth[pix], aout = 1.0f - T[k];
          Z0[k] = aout > 0.0f ? D / aout : 0.0f;
          E[k] = -__fmaf_rn(-Z0[k], aout, D);
        }
        if (lastp[k] > range.x) atomicMax(&s_hi[hp], lastp[k]);
      }
      U0[k] = 1.0f - T[k];
    }
    // the two pixels side by side (.x, .y) for the paired FP32 arithmetic of the walk
    float2 T2 = make_float2(T[0], T[1]), Sg2 = make_float2(Sg[0], Sg[1]), gD2 = make_float2(gD[0], gD[1]);
    const float2 gAlT2 = make_float2(gAlT[0], gAlT[1]);
    const float2 gR0 = make_float2(gR[0][0], gR[1][0]), gR1 = make_float2(gR[0][1], gR[1][1]),
                 gR2 = make_float2(gR[0][2], gR[1][2]);
    const float2 gN0 = make_float2(gN[0][0], gN[1][0]), gN1 = make_float2(gN[0][1], gN[1][1]),
                 gN2 = make_float2(gN[0][2], gN[1][2]);
    const float2 gDsv = make_float2(gDs2[0], gDs2[1]), z0v = make_float2(Z0[0], Z0[1]);
    float2 Ev = make_float2(E[0], E[1]), Uv = make_float2(U0[0], U0[1]);
    const float2 yy = make_float2(y[0], y[1]);
    // the group's last walked position (exclusive): its walk ends there
    uint32_t glast = max(lastp[0], lastp[1]);
    glast = max(glast, __shfl_xor_sync(0xffffffffu, glast, 1));
    glast = max(glast, __shfl_xor_sync(0xffffffffu, glast, 2));
    glast = max(glast, __shfl_xor_sync(0xffffffffu, glast, 4));
    __syncthreads();
    const uint32_t hi_all = s_hi[hp];  // 0 when no pixel walked: no batch
    const float two_inv2s2 = 2.0f * p.k.inv2s2;
    for (uint32_t hi = hi_all; hi > range.x;) {
      const uint32_t b0 = (hi - range.x > (uint32_t)BATCH) ? hi - BATCH : range.x;
      const int nb = (int)(hi - b0);
      if (hi != hi_all) __syncthreads();  // the first batch follows the barrier after the upstream loads
      for (int i = tid; i < nb; i += NT) {
        const uint32_t kk = p.vals[b0 + i];
        const int64_t rec = recbase + kk;
        const float4* g = p.geom + rec * 3;
        const float4* f = p.feat + rec * 2;
        const float4 g0 = g[0], g1 = g[1], g2 = g[2];
        sk[i] = kk;
        sg[i][0] = g0;
        sg[i][1] = g1;
        sg[i][2] = g2;
        sf[i][0] = f[0];
        if (!sun) sf[i][1] = f[1];  // a sun view has no colour or normal terms
        smask[i] = p.subblock_cull ? subblock_mask<TW, TH>(g0, g1, g2, lg.x0, lg.y0, p.cull) : 0xffffu;
      }
      for (int i = tid; i < nb * kSaccStride; i += NT) (&sacc[0][0])[i] = 0.0f;
      __syncthreads();
      // each group walks its candidates in reverse list order, up to its last walked splat.
      // The group reduction of one splat's 16 sums is issued in the next step, beside the next
      // splat's arithmetic (software pipelining); the sums alternate between GA and GB so that
      // the pending ones are never copied.
      uint32_t mk = batch_masks<TW, BATCH>(smask, nb);
      {
        const int lim = (int)min(max((int64_t)glast - (int64_t)b0, (int64_t)0), (int64_t)nb) - (gl << 5);
        mk = lim <= 0 ? 0u : (lim >= 32 ? mk : mk & ((1u << lim) - 1u));
      }
      const uint8_t* list = slist[tid >> 3];
      const int total = compact_candidates(mk, slist[tid >> 3]);
      const int nsteps = (int)__reduce_max_sync(0xffffffffu, (unsigned)total);
      // group sums of splat jq, one atomic per field into the block's accumulator
      auto flush = [&](float (&Gq)[16], const int jq) {
        group_reduce16(Gq);
        if (jq >= 0) {
          if (Gq[0] != 0.0f) atomicAdd(&sacc[jq][2 * gl], Gq[0]);
          if (Gq[1] != 0.0f) atomicAdd(&sacc[jq][2 * gl + 1], Gq[1]);
        }
      };
      float GA[16], GB[16];
#pragma unroll
      for (int f = 0; f < 16; ++f) GA[f] = GB[f] = 0.0f;
      int jA = -1, jB = -1;
      // A sun view (SUN) has depth and alpha upstream only: its colour and normal terms are
      // zero and are not formed.
      auto walk = [&](auto sun_c) {
        constexpr bool SUN = decltype(sun_c)::value;
        // step st: the group's candidate total - 1 - st (reverse list order) into Gc, and the
        // reduction of the pending Gq
        auto step = [&](float (&Gc)[16], int& jc, float (&Gq)[16], const int jq, const int st) {
          const int pos = total - 1 - st;
          const int jj = pos >= 0 ? (int)list[pos] : -1;
          // lanes whose group has no splat left evaluate a stand-in and add nothing
          const int js = jj >= 0 ? jj : 0;
          const uint32_t j = b0 + (uint32_t)js;
          const float4 g0 = sg[js][0], g1 = sg[js][1], g2 = sg[js][2];
          const PairEval2 e = eval_pair2(g0, g1, g2, x, yy, p.k);
          const bool c0p = jj >= 0 && j < lastp[0] && e.contrib0, c1p = jj >= 0 && j < lastp[1] && e.contrib1;
          // the previous splat's group reduction overlaps this splat's arithmetic; it runs
          // unconditionally (sums that nothing wrote are zeros) so that it stays branch free
          flush(Gq, jq);
          const float4 f0 = sf[js][0];
          const float4 f1 = SUN ? make_float4(0.0f, 0.0f, 0.0f, 0.0f) : sf[js][1];
          // both pixels side by side.  A pair that does not contribute runs with alpha = 0, which
          // leaves T and S unchanged and adds zeros.  The two pixels share their column, so the
          // terms linear in dx and the centre's chain through Q are summed over the lane before
          // they are formed.
          const float2 a = make_float2(c0p ? e.alpha.x : 0.0f, c1p ? e.alpha.y : 0.0f);
          const float2 om = add2(bc2(1.0f), neg2(a));
          const float2 rom = make_float2(__fdividef(1.0f, om.x), __fdividef(1.0f, om.y));  // om >= 1 - alpha_max
          const float2 Ti = mul2(T2, rom);  // T in front of the splat
          const float2 z = fma2(bc2(f0.y), e.v, fma2(bc2(f0.x), e.u, bc2(g2.w)));
          float2 gf = mul2(gD2, z);
          if (!SUN) {
            gf = fma2(gR0, bc2(f1.y), gf);
            gf = fma2(gR1, bc2(f1.z), gf);
            gf = fma2(gR2, bc2(f1.w), gf);
            gf = fma2(gN0, bc2(f0.z), gf);
            gf = fma2(gN1, bc2(f0.w), gf);
            gf = fma2(gN2, bc2(f1.x), gf);
          }
          const float2 w = mul2(a, Ti);
          float2 dzd = bc2(0.0f);  // the distortion's partial in z
          if (DIST) {
            const float2 zs = add2(z, neg2(z0v));  // depth relative to z0
            gf = fma2(gDsv, fma2(zs, Uv, Ev), gf);
            dzd = mul2(mul2(gDsv, w), add2(Uv, neg2(w)));  // W - W' = U - w
            const float2 w2 = mul2(bc2(2.0f), w);
            Uv = add2(Uv, neg2(w2));
            Ev = fma2(w2, zs, Ev);
          }
          const float2 gs = add2(gf, neg2(Sg2));
          T2 = Ti;
          Sg2 = fma2(a, gs, Sg2);  // composite from this splat on: a f + (1 - a) S
          auto hsum = [](float2 v) { return v.x + v.y; };
          if (SUN) {
            Gc[GF_R] = Gc[GF_G] = Gc[GF_B] = Gc[GF_NX] = Gc[GF_NY] = Gc[GF_NZ] = 0.0f;
          } else {
            Gc[GF_R] = hsum(mul2(w, gR0));
            Gc[GF_G] = hsum(mul2(w, gR1));
            Gc[GF_B] = hsum(mul2(w, gR2));
            Gc[GF_NX] = hsum(mul2(w, gN0));
            Gc[GF_NY] = hsum(mul2(w, gN1));
            Gc[GF_NZ] = hsum(mul2(w, gN2));
          }
          const float2 dz = fma2(w, gD2, dzd);
          Gc[GF_ZC] = hsum(dz);
          Gc[GF_DZDU] = hsum(mul2(dz, e.u));
          Gc[GF_DZDV] = hsum(mul2(dz, e.v));
          // d / d ln(o G^) = alpha dL/dalpha, dL/dalpha = T_i (f - S) + d(alpha_out) T_final / (1 - alpha);
          // zero when clamped (the exact adjoint of the clamp)
          const float2 dal = fma2(Ti, gs, mul2(gAlT2, rom));
          const float2 dpa = mul2(dal, a);
          const float2 dpw = make_float2(e.clamped0 ? 0.0f : dpa.x, e.clamped1 ? 0.0f : dpa.y);
          Gc[GF_LNO] = hsum(dpw);
          const float2 dpu = make_float2(e.uwin0 ? dpw.x : 0.0f, e.uwin1 ? dpw.y : 0.0f);
          const float2 dps = mul2(make_float2(e.uwin0 ? 0.0f : dpw.x, e.uwin1 ? 0.0f : dpw.y), bc2(two_inv2s2));
          // degenerate splats: zero slopes, and dpu = 0 except at u = v = 0
          const float2 du = fma2(dz, bc2(f0.x), neg2(mul2(dpu, e.u)));
          const float2 dv = fma2(dz, bc2(f0.y), neg2(mul2(dpu, e.v)));
          const float sdu = hsum(du), sdv = hsum(dv);
          Gc[GF_Q00] = sdu * e.dx;
          Gc[GF_Q01] = hsum(mul2(du, e.dy));
          Gc[GF_Q10] = sdv * e.dx;
          Gc[GF_Q11] = hsum(mul2(dv, e.dy));
          Gc[GF_CX] = hsum(dps) * e.dx - (g1.x * sdu + g1.z * sdv);
          Gc[GF_CY] = hsum(mul2(dps, e.dy)) - (g1.y * sdu + g1.w * sdv);
          jc = jj;
        };
        bool lastA = false;  // the last step wrote GA (else GB)
        for (int st = 0; st < nsteps; st += 2) {
          step(GA, jA, GB, jB, st);
          lastA = true;
          if (st + 1 >= nsteps) break;
          step(GB, jB, GA, jA, st + 1);
          lastA = false;
        }
        // the sums of the last step are still pending
        if (lastA) flush(GA, jA); else flush(GB, jB);
      };
      if (sun) walk(std::true_type{}); else walk(std::false_type{});
      __syncthreads();
      for (int i = tid; i < nb * kGradFields; i += NT) {
        const int s = i >> 4, f = i & 15;
        const float v = sacc[s][f];
        if (v != 0.0f) atomicAdd(p.grad + (recbase + sk[s]) * kGradFields + f, v);
      }
      hi = b0;
    }
    // gradient of the colour offset c of this target: the sum of d(rgb_out) over its pixels
    // (the 3x3 block C is chained per splat in the projection adjoint)
    if (!sun && p.d_color && io.d_rgb) {
      float s3[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        s3[c] = gR[0][c] + gR[1][c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s3[c] += __shfl_xor_sync(0xffffffffu, s3[c], o);
      }
      if (lane == 0) {
        scol[warp][0] = s3[0];
        scol[warp][1] = s3[1];
        scol[warp][2] = s3[2];
      }
      __syncthreads();
      if (tid < 3) {
        float s = 0.0f;
#pragma unroll
        for (int w2 = 0; w2 < NW; ++w2) s += scol[w2][tid];
        if (s != 0.0f) atomicAdd(p.d_color + cam.cam * 12 + 4 * tid + 3, s);
      }
    }
  }
}

// ------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------
template <int TW, int TH, int BATCH, bool DIST>
cudaError_t launch_fwd_t(const RasterParams& p, bool persistent, int num_sms, cudaStream_t st) {
  constexpr int NT = TW * TH / 2;
  if (p.total_tiles == 0) return cudaSuccess;
  if (persistent) {
    // resident blocks per SM, queried once (outside any later stream capture)
    static int per_sm = 0;
    if (per_sm == 0) {
      int v = 0;
      cudaError_t e =
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, raster_fwd_kernel<TW, TH, BATCH, true, DIST>, NT, 0);
      if (e != cudaSuccess) return e;
      per_sm = v < 1 ? 1 : v;
    }
    int grid = num_sms * per_sm;
    if (grid > p.total_tiles) grid = p.total_tiles;
    count_launch();
    raster_fwd_kernel<TW, TH, BATCH, true, DIST><<<grid, NT, 0, st>>>(p);
  } else {
    count_launch();
    raster_fwd_kernel<TW, TH, BATCH, false, DIST><<<p.total_tiles, NT, 0, st>>>(p);
  }
  return cudaGetLastError();
}

// The backward stages at most 224 splats per batch when the option asks for 256: its shared
// accumulator is then 15 KB instead of 17 KB (measured 1.6 % faster on the 1M-splat batch).
template <int TW, int TH, int BATCH_OPT, bool DIST>
cudaError_t launch_bwd_t(const RasterParams& p, bool persistent, int num_sms, cudaStream_t st) {
  constexpr int BATCH = BATCH_OPT == 256 ? 224 : BATCH_OPT;
  constexpr int NT = TW * TH / 2;
  if (p.total_tiles == 0) return cudaSuccess;
  if (persistent) {
    static int per_sm = 0;
    if (per_sm == 0) {
      int v = 0;
      cudaError_t e =
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, raster_bwd_kernel<TW, TH, BATCH, true, DIST>, NT, 0);
      if (e != cudaSuccess) return e;
      per_sm = v < 1 ? 1 : v;
    }
    int grid = num_sms * per_sm;
    if (grid > p.total_tiles) grid = p.total_tiles;
    count_launch();
    raster_bwd_kernel<TW, TH, BATCH, true, DIST><<<grid, NT, 0, st>>>(p);
  } else {
    count_launch();
    raster_bwd_kernel<TW, TH, BATCH, false, DIST><<<p.total_tiles, NT, 0, st>>>(p);
  }
  return cudaGetLastError();
}

// Instantiates the launchers of one tile shape for both batch sizes, with and without the
// distortion.
#define SS_RASTER_DISPATCH(KIND, TW, TH)                                                                    \
  cudaError_t launch_raster_##KIND##_##TW##x##TH(const RasterParams& p, int batch, bool persistent,        \
                                                 int num_sms, cudaStream_t st) {                            \
    const bool dist = p.distort != 0;                                                                        \
    if (batch == 128)                                                                                        \
      return dist ? launch_##KIND##_t<TW, TH, 128, true>(p, persistent, num_sms, st)                        \
                  : launch_##KIND##_t<TW, TH, 128, false>(p, persistent, num_sms, st);                      \
    if (batch == 256)                                                                                        \
      return dist ? launch_##KIND##_t<TW, TH, 256, true>(p, persistent, num_sms, st)                        \
                  : launch_##KIND##_t<TW, TH, 256, false>(p, persistent, num_sms, st);                      \
    return cudaErrorInvalidValue;                                                                            \
  }

}  // namespace ss
