// Forward (K3) and backward (K4) rasterization, Sec. 3.2 Eq. rasterization.
//
// Work decomposition.  A screen tile (16 x 16, 32 x 8, 8 x 32, 32 x 16 or 16 x 32 px) is rendered
// by one block of one warp per 128 pixels (a 16 x 8 part, or 8 x 16 in 8-wide tiles).  A warp's
// pixels are split into sub-blocks of GL columns by 4 rows, one per group of GL lanes (GL = 2 in
// both directions, kernels.cuh: sixteen groups per warp).  Lane l of a group owns column l of its
// sub-block, four pixels, kept as two pairs (rows 0-1 and 2-3) so that the paired FP32
// instructions of sm_100-family GPUs compute two pixels in one issue.  The block stages the tile's
// sorted splat list in shared memory in batches of records copied with cp.async (the next batch's
// splat indices are loaded while a batch is walked); large batches keep the groups of a warp,
// which walk their own candidate lists in lockstep, evenly loaded.
//
// The thread that stages a splat forms the set of the tile's sub-blocks its support can reach
// (`subblock_mask`); each group walks only the staged splats that reach its sub-block, in list
// order (forward) or reverse list order (backward).  A pixel's walk is therefore exactly the
// per-pixel definition, whatever the tile shape, grouping or schedule, and every pixel runs the
// same FP32 operations in both kernels, so the backward retraces the forward's alpha decisions
// bit for bit.
//
// Backward: with T_i the transmittance in front of splat i and S_i the composite behind it
// (normalised to T_{i+1}), d f / d alpha_i = T_i (f_i - S_i); the alpha output adds
// T_final / (1 - alpha_i).  T_i is recovered as T_{i+1} / (1 - alpha_i) from the saved T_final
// (alpha <= alpha_max < 1 keeps the division safe); only T_final and the end of the walk are
// stored per pixel.  A lane sums its four pixels' contributions to the 16 gradient fields of the
// splat, the lanes of the group reduce them with a transposed butterfly (each of the two lanes
// ends with eight fields), and each lane adds its fields to the (target, splat) gradient record
// with vector reductions in L2 (red.global.add.v4.f32).
#pragma once

#include <type_traits>

#include "kernels.cuh"

namespace ss {

constexpr int kWarpPixels = 128;  // pixels of one warp
// warps of a tile block: one per 128 pixels of the tile
template <int TW, int TH>
__host__ __device__ constexpr int tile_warps() { return TW * TH / kWarpPixels; }
// Lanes of a group (GL, two or four): a group owns a sub-block of GL pixel columns by 4 rows, one
// column per lane; a warp holds 32 / GL groups.
template <int TW, int TH, int GL>
__host__ __device__ constexpr int tile_subblocks() { return TW * TH / (4 * GL); }
// A tile's sub-block mask: one bit per sub-block.
template <int TW, int TH, int GL>
using SubMask = std::conditional_t<(tile_subblocks<TW, TH, GL>() > 32), unsigned long long, uint32_t>;

__device__ __forceinline__ int find_target(const TargetCam* tc, int n_targets, int tile) {
  int lo = 0, hi = n_targets - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tc[mid].tile_base <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------- paired FP32 arithmetic
// Two pixels share every operation: their state is a float2 and the paired FP32 instructions
// (one issue, two IEEE round-to-nearest results) compute both halves, each bitwise equal to the
// scalar operation.
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float hsum(float2 v) { return v.x + v.y; }

// Evaluation of one splat at two pixels (x, y.x) and (x, y.y) of one column (Eq. rasterization):
// the offset from the float-pair centre, the uv coordinates u = Q (x - c), the log2 of the two
// Gaussians of the lower-bounded max, and alpha = min(alpha_max, 2^(log2 o + log2 G^)).  Branch
// free: the kernels evaluate several pairs side by side.  ex2 is accurate to a few ulp, so
// alpha >= alpha_min decides the same as log2(o G^) >= log2(alpha_min) except within that error of
// the threshold, and both kernels take every decision from this same function, so the backward
// retraces the forward's decisions bit for bit.
struct PairEval2 {
  float dx;                   // x - c (the two pixels share a column)
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
  const float2 pu = mul2(bc2(k.c_uv), fma2(e.u, e.u, mul2(e.v, e.v)));
  const float2 ps = mul2(bc2(k.c_xy), fma2(bc2(dx), bc2(dx), mul2(dy, dy)));
  e.uwin0 = pu.x >= ps.x;
  e.uwin1 = pu.y >= ps.y;
  const float2 lp = add2(make_float2(fmaxf(pu.x, ps.x), fmaxf(pu.y, ps.y)), bc2(__fmul_rn(g2.x, kLog2e)));
  const float og0 = ex2_ftz(lp.x), og1 = ex2_ftz(lp.y);
  e.clamped0 = og0 > k.amax;
  e.clamped1 = og1 > k.amax;
  e.alpha = make_float2(fminf(og0, k.amax), fminf(og1, k.amax));
  e.contrib0 = e.alpha.x >= k.amin;
  e.contrib1 = e.alpha.y >= k.amin;
  return e;
}

// Transposed reduction of 16 values over the lanes of a group: lane gl of the group ends with the
// group sums of fields F gl .. F gl + F - 1 (F = 16 / GL) in v[0 .. F - 1].  Each exchange
// sends the half of the values that the partner keeps (8 shuffles for two lanes, 12 for four).
// LOW12: only fields 0 .. 11 are wanted (a sun view's fields 12 .. 15 are zero and not added);
// with two lanes, the upper lane's slots for fields 12 .. 15 then need no exchange of their own.
template <int GL, bool LOW12 = false>
__device__ __forceinline__ void group_reduce16(float v[16]) {
  static_assert(GL == 2 || GL == 4, "groups of two or four lanes");
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int s = GL / 2, n = 16; s >= 1; s >>= 1, n >>= 1) {
    const bool up = lane & s;
#pragma unroll
    for (int i = 0; i < n / 2; ++i) {
      if (LOW12 && GL == 2 && i >= 4) {
        v[i] += __shfl_xor_sync(0xffffffffu, v[i], s);  // the lower lane's field i
        continue;
      }
      const float send = up ? v[i] : v[i + n / 2];
      const float keep = up ? v[i + n / 2] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
}

// One vector reduction of four floats into global memory (16-byte aligned), performed in L2.
__device__ __forceinline__ void red_add_v4(float* p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
}

// ---------------------------------------------------------------- asynchronous staging
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Shared memory of one tile block: one or two buffers of B staged records (geometry 48 B, features
// 32 B, the splat index), the sub-block masks of the current batch and each group's candidates.
// Batches of up to 128 records are double-buffered (the next batch copied while one is walked);
// larger ones fit shared memory once.
template <int B>
__host__ __device__ constexpr int stage_bufs() { return B > 128 ? 1 : 2; }
// 32-entry chunks of a batch held per lane of a group
template <int B, int GL>
__host__ __device__ constexpr int mask_chunks() { return (B + 32 * GL - 1) / (32 * GL); }
// entries of a batch that each thread of a block of NT threads copies
template <int B, int NT>
__host__ __device__ constexpr int per_thread() { return (B + NT - 1) / NT; }

template <int B, int NW, typename M, int GL>
struct TileStage {
  float4 g[stage_bufs<B>()][B][3];
  float4 f[stage_bufs<B>()][B][2];
  uint32_t k[stage_bufs<B>()][B];
  // per sub-block of the tile, its candidate masks of the batch's 32-entry chunks (rows padded
  // by a word so that a warp's stores of one chunk fall in different banks)
  uint32_t words[8 * sizeof(M)][B / 32 + 1];
  uint8_t list[32 / GL * NW][B + 4];  // per group its candidates' slots (buffer * B + index); rows
                                        // padded so that the groups read at one position from
                                        // different banks
};

// Pixels of this lane and the tile's origin.  A warp's 128 pixels are 16 x 8 (8 x 16 for 8-wide
// tiles); its sub-blocks go to its groups in row-major order.
struct LaneGeom {
  int px;        // pixel column
  int py0;       // first of the lane's four pixel rows
  int sub;       // bit of the lane's sub-block in the tile's sub-block mask
  float x0, y0;  // the tile's first pixel column and row
};

template <int TW, int TH, int GL>
__device__ __forceinline__ int group_sub(int half, int grp) {
  constexpr int WW = TW >= 16 ? 16 : 8, WH = kWarpPixels / WW;
  constexpr int WX = TW / WW, GX = WW / GL, SBX = TW / GL;
  const int wx = half % WX, wy = half / WX;
  const int sbx = wx * GX + grp % GX, sby = wy * (WH / 4) + grp / GX;
  return sby * SBX + sbx;
}

template <int TW, int TH, int GL>
__device__ __forceinline__ LaneGeom lane_geom(const TargetCam& cam, int tile, int half) {
  constexpr int SBX = TW / GL;
  const int lane = threadIdx.x & 31, grp = lane / GL, gl = lane % GL;
  const int local = tile - cam.tile_base;
  const int ty = local / cam.tiles_x, tx = local - ty * cam.tiles_x;
  LaneGeom g;
  g.sub = group_sub<TW, TH, GL>(half, grp);
  const int sby = g.sub / SBX, sbx = g.sub - sby * SBX;
  g.px = tx * TW + sbx * GL + gl;
  g.py0 = ty * TH + sby * 4;
  g.x0 = (float)(tx * TW);
  g.y0 = (float)(ty * TH);
  return g;
}

// The GL x 4 sub-blocks of a tile that a splat can reach: bit (row * TW / GL + col) is set when the
// support {alpha >= alpha_min} can contain a pixel centre of sub-block (col, row), tested a row of
// sub-blocks at a time against the support's slice through its rows (SupportSlices), with the
// sub-blocks padded by 2e-3 px.
template <int TW, int TH, int GL>
__device__ __forceinline__ SubMask<TW, TH, GL> subblock_mask(const float4 g0, const float4 g1, const float4 g2,
                                                            float x0, float y0, const CullConsts& cc) {
  using M = SubMask<TW, TH, GL>;
  constexpr int SW = GL, SBX = TW / SW, SBY = TH / 4;
  constexpr float kInvSW = 1.0f / SW;
  constexpr float kPad = 2e-3f;
  SupportSlices sl;
  sl.init(g1, g2, cc);
  // tile-relative offsets: pixel centre (x0 + i + 0.5) - cx
  const float ox = x0 + 0.5f - g0.x, oy = y0 + 0.5f - g0.y;
  M mask = 0;
#pragma unroll
  for (int b = 0; b < SBY; ++b) {
    float lo, hi;
    sl.range(oy + (float)(4 * b) - kPad, oy + (float)(4 * b + 3) + kPad, lo, hi);
    // columns c with [ox + SW c, ox + SW c + SW - 1] (padded) meeting [lo, hi]
    const float cl = fmaxf(ceilf((lo - ox - (float)(SW - 1) - kPad) * kInvSW), 0.0f);
    const float ch = fminf(floorf((hi - ox + kPad) * kInvSW), (float)(SBX - 1));
    if (cl <= ch) {
      const int a = (int)cl, z = (int)ch;
      mask |= ((M(2) << z) - (M(1) << a)) << (b * SBX);
    }
  }
  return mask;
}

// Candidate masks of a staged batch: lane gl of a group reads the group's masks of chunks
// gl, gl + GL, ... (staged splats [32 c, 32 c + 32)).  Holding every chunk at once lets a group
// walk its candidates across chunk boundaries.
template <int B, int GL, int ROWS>
__device__ __forceinline__ void batch_masks(const uint32_t (&words)[ROWS][B / 32 + 1], int sub,
                                            uint32_t (&mk)[mask_chunks<B, GL>()]) {
  static_assert(B % 32 == 0 && B / 32 <= GL * mask_chunks<B, GL>(), "chunks per lane of a group");
  const int gl = threadIdx.x % GL;
#pragma unroll
  for (int q = 0; q < mask_chunks<B, GL>(); ++q) {
    const int c = q * GL + gl;
    mk[q] = c < B / 32 ? words[sub][c] : 0u;
  }
}

// Transpose of a 32 x 32 bit matrix held one row per lane (bit c of lane r's word is entry
// (r, c)): returns column `lane`.  Each level swaps the off-diagonal blocks of every 2j x 2j block,
// from j = 16 down to 1.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x) {
  const int lane = threadIdx.x & 31;
  constexpr uint32_t kLo[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int l = 0; l < 5; ++l) {
    const int j = 16 >> l;
    const uint32_t lo = kLo[l];  // the columns c with c & j == 0
    const uint32_t t = __shfl_xor_sync(0xffffffffu, x, j);
    x = (lane & j) ? (((t >> j) & lo) | (x & ~lo)) : ((x & lo) | ((t << j) & ~lo));
  }
  return x;
}

// Writes a group's candidates of a staged batch (the set bits of its chunk masks) to the group's
// list as shared-memory slots (slot_base + index), in list order or, with `desc`, in reverse list
// order, and returns their number.  The walk then reads its next splat from the list at a
// position that depends on the step count alone, so no step waits on the previous one to find
// its splat.  Every lane of the warp takes part.
template <int GL, int CH>
__device__ __forceinline__ int compact_candidates(const uint32_t (&mk)[CH], uint8_t* list, int slot_base,
                                                  bool desc) {
  const int gl = threadIdx.x % GL;
  int before[CH], total = 0;
#pragma unroll
  for (int q = 0; q < CH; ++q) {
    const int c = __popc(mk[q]);
    int inc = c;
#pragma unroll
    for (int d = 1; d < GL; d <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, inc, d, GL);
      if (gl >= d) inc += t;
    }
    before[q] = total + inc - c;
    total += __shfl_sync(0xffffffffu, inc, GL - 1, GL);
  }
#pragma unroll
  for (int q = 0; q < CH; ++q) {
    int k = before[q];
    uint32_t mm = mk[q];
    while (mm) {
      const int bit = __ffs(mm) - 1;
      mm &= mm - 1;
      list[desc ? total - 1 - k : k] = (uint8_t)(slot_base + (q * GL + gl) * 32 + bit);
      ++k;
    }
  }
  __syncwarp();
  return total;
}

// Splat indices of a batch (thread t holds entries t, t + kTileThreads, ...), loaded one batch
// ahead of their copies.
template <int B, int NT>
__device__ __forceinline__ void load_vals(uint32_t (&kv)[per_thread<B, NT>()], const uint32_t* vals, uint32_t b0,
                                          int nb) {
#pragma unroll
  for (int c = 0; c < per_thread<B, NT>(); ++c) {
    const int i = c * NT + threadIdx.x;
    kv[c] = i < nb ? __ldg(vals + b0 + i) : 0u;
  }
}

// Issues the asynchronous copies of a batch's records into buffer `buf` (one commit group).
// A sun view composites depth alone and needs only the first feature vector.
template <int B, int NW, typename M, int GL>
__device__ __forceinline__ void stage_issue(TileStage<B, NW, M, GL>& S, int buf,
                                            const uint32_t (&kv)[per_thread<B, 32 * NW>()],
                                            int nb, const RasterParams& p, int64_t recbase, bool sun) {
#pragma unroll
  for (int c = 0; c < per_thread<B, 32 * NW>(); ++c) {
    const int i = c * (32 * NW) + threadIdx.x;
    if (i < nb) {
      const int64_t rec = recbase + kv[c];
      const float4* g = p.geom + rec * 3;
      const float4* f = p.feat + rec * 2;
      cp_async16(&S.g[buf][i][0], g);
      cp_async16(&S.g[buf][i][1], g + 1);
      cp_async16(&S.g[buf][i][2], g + 2);
      cp_async16(&S.f[buf][i][0], f);
      if (!sun) cp_async16(&S.f[buf][i][1], f + 1);
      S.k[buf][i] = kv[c];
    }
  }
  cp_async_commit();
}

// Sub-block masks of a landed batch: each thread forms the masks of the records it copied itself
// (before the barrier that publishes copies and masks to the block).  A warp's records of one pass
// are one 32-entry chunk, one record per lane, so transposing the warp's masks as a bit matrix gives
// lane s the chunk's candidate mask of sub-block s.
template <int TW, int TH, int B, int NW, int GL>
__device__ __forceinline__ void stage_masks(TileStage<B, NW, SubMask<TW, TH, GL>, GL>& S, int buf, int nb,
                                            const LaneGeom& lg, const RasterParams& p) {
  using M = SubMask<TW, TH, GL>;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int c = 0; c < per_thread<B, 32 * NW>(); ++c) {
    const int i = c * (32 * NW) + threadIdx.x;
    const int chunk = i >> 5;  // the same for the whole warp
    if (chunk >= B / 32) break;
    M m = 0;
    if (i < nb)
      m = p.subblock_cull ? subblock_mask<TW, TH, GL>(S.g[buf][i][0], S.g[buf][i][1], S.g[buf][i][2], lg.x0, lg.y0,
                                                     p.cull)
                          : ~M(0);
    S.words[lane][chunk] = warp_transpose32((uint32_t)m);
    if (sizeof(M) == 8) S.words[32 + lane][chunk] = warp_transpose32((uint32_t)((unsigned long long)m >> 32));
  }
}

// Work item of a block: one tile per block, or the next tile of the persistent queue, claimed one
// item ahead by thread 0 so that the claim's latency overlaps the current item.  The barriers
// around each read of the shared slot order it against thread 0's next claim, and the one that
// ends an item also frees the staging buffers for the next.
template <bool PERSIST>
struct ItemQueue {
  unsigned int* counter;
  int* slot;  // shared
  int item;
  __device__ __forceinline__ void begin(unsigned int* c, int* s) {
    counter = c;
    slot = s;
    if (PERSIST) {
      if (threadIdx.x == 0) *slot = (int)atomicAdd(counter, 1u);
      __syncthreads();
      item = *slot;
      __syncthreads();
    } else {
      item = blockIdx.x;
    }
  }
  __device__ __forceinline__ void claim_next() {
    if (PERSIST && threadIdx.x == 0) *slot = (int)atomicAdd(counter, 1u);
  }
  // false when this block has no item left
  __device__ __forceinline__ bool advance() {
    if (!PERSIST) return false;
    __syncthreads();
    item = *slot;
    __syncthreads();
    return true;
  }
};

// ------------------------------------------------------------------------------------------
// K3 forward
// ------------------------------------------------------------------------------------------
// DIST: the distortion of the blending weights along each ray is accumulated beside the planes:
// each composited splat i adds w_i (zs_i (1 - T_i) - D'_i) = sum_{j<i} w_i w_j (z_i - z_j), with
// 1 - T_i the weight composited in front of it and D'_i the weighted depth in front of it, both
// taken relative to the depth z0 of the pixel's first composited splat (zs = z - z0).  The sum is
// unchanged by that common shift, and with it the terms are of the size of the depth differences
// rather than of the depths.  The sum is doubled when it is written.

// Compositing state of one pixel pair of a lane.
struct FwdPair {
  float2 T, D, A0, A1, A2, N0, N1, N2, Dst, Dsh, Z0;
  uint32_t last0, last1;
  bool done0, done1;
};

__device__ __forceinline__ void fwd_init(FwdPair& s, uint32_t start, bool out0, bool out1) {
  s.T = bc2(1.0f);
  s.D = s.A0 = s.A1 = s.A2 = s.N0 = s.N1 = s.N2 = s.Dst = s.Dsh = s.Z0 = bc2(0.0f);
  s.last0 = s.last1 = start;
  s.done0 = out0;
  s.done1 = out1;
}

// Composites one splat into a pixel pair (Eq. rasterization, front to back); returns the number
// of walked pairs (contributing, the stopping one included).  A sun view composites depth alone.
template <bool SUN, bool DIST>
__device__ __forceinline__ uint32_t composite(FwdPair& s, const PairEval2& e, bool has, const float4& g2,
                                              const float4& f0, const float4& f1, uint32_t pos, float t_min) {
  const bool ck0 = has && !s.done0 && e.contrib0, ck1 = has && !s.done1 && e.contrib1;
  // T after the splat: T - alpha T (the weight is alpha T)
  const float2 aT = mul2(e.alpha, s.T);
  const float2 Tn = add2(s.T, neg2(aT));
  // a splat that takes T below t_min ends the walk and is not composited
  const bool stop0 = ck0 && Tn.x < t_min, stop1 = ck1 && Tn.y < t_min;
  const bool take0 = ck0 && !stop0, take1 = ck1 && !stop1;
  const float2 w = make_float2(take0 ? aT.x : 0.0f, take1 ? aT.y : 0.0f);
  const float2 z = fma2(bc2(f0.y), e.v, fma2(bc2(f0.x), e.u, bc2(g2.w)));
  if (DIST) {
    // z0: T is exactly 1 until the first splat is composited (alpha >= alpha_min)
    s.Z0 = make_float2(s.T.x == 1.0f ? z.x : s.Z0.x, s.T.y == 1.0f ? z.y : s.Z0.y);
    const float2 zs = add2(z, neg2(s.Z0));
    s.Dst = fma2(w, add2(fma2(neg2(zs), s.T, zs), neg2(s.Dsh)), s.Dst);
    s.Dsh = fma2(w, zs, s.Dsh);
  }
  s.D = fma2(w, z, s.D);
  if (!SUN) {
    s.A0 = fma2(w, bc2(f1.y), s.A0);
    s.A1 = fma2(w, bc2(f1.z), s.A1);
    s.A2 = fma2(w, bc2(f1.w), s.A2);
    s.N0 = fma2(w, bc2(f0.z), s.N0);
    s.N1 = fma2(w, bc2(f0.w), s.N1);
    s.N2 = fma2(w, bc2(f1.x), s.N2);
  }
  s.T = add2(s.T, neg2(w));  // Tn where the splat is taken, else T unchanged (w = 0)
  s.last0 = take0 ? pos : s.last0;
  s.last1 = take1 ? pos : s.last1;
  s.done0 = s.done0 || stop0;
  s.done1 = s.done1 || stop1;
  return (uint32_t)ck0 + (uint32_t)ck1;
}

// COUNT: the launch also counts the walked pairs (the algorithmic work of the roofline) into the
// status block; the training step runs without it.
template <int TW, int TH, int B, int GL, bool PERSIST, bool DIST, bool COUNT>
__global__ void __launch_bounds__(32 * tile_warps<TW, TH>(), 16 / tile_warps<TW, TH>())
    raster_fwd_kernel(const __grid_constant__ RasterParams p) {
  constexpr int NW = tile_warps<TW, TH>(), NT = 32 * NW;
  static_assert(TW * TH == NW * kWarpPixels, "whole warps per tile");
  constexpr int kBufs = stage_bufs<B>();
  __shared__ TileStage<B, NW, SubMask<TW, TH, GL>, GL> S;
  __shared__ int s_item;
  const int lane = threadIdx.x & 31, grp = lane / GL, half = threadIdx.x >> 5;
  const float4 zero4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  ItemQueue<PERSIST> q;
  q.begin(&p.status->work_fwd, &s_item);
  while (q.item < p.total_tiles) {
    q.claim_next();
    const int tile = q.item;
    const int t = find_target(p.tcams, p.n_targets, tile);
    const TargetCam& cam = p.tcams[t];
    const LaneGeom lg = lane_geom<TW, TH, GL>(cam, tile, half);
    const bool sun = cam.sun != 0;
    const float x = (float)lg.px + 0.5f;
    const float yb = (float)lg.py0 + 0.5f;
    const float2 yA = make_float2(yb, yb + 1.0f), yB = make_float2(yb + 2.0f, yb + 3.0f);
    const uint2 range = p.ranges[tile];
    const int64_t recbase = (int64_t)t * p.n_pad;
    const bool inx = lg.px < cam.W;
    FwdPair sA, sB;
    fwd_init(sA, range.x, !(inx && lg.py0 < cam.H), !(inx && lg.py0 + 1 < cam.H));
    fwd_init(sB, range.x, !(inx && lg.py0 + 2 < cam.H), !(inx && lg.py0 + 3 < cam.H));
    uint32_t walked = 0;
    // batches of B list entries in list order; batch k is copied into buffer k & 1 while batch
    // k - 1 is walked
    const int n = (int)(range.y - range.x), nbat = (n + B - 1) / B;
    auto nb_of = [&](int k) { return min(n - k * B, B); };
    uint8_t* list = S.list[half * (32 / GL) + grp];
    uint32_t kv[per_thread<B, NT>()];  // splat indices of the next batch to copy
    if (nbat > 0) {
      load_vals<B, NT>(kv, p.vals, range.x, nb_of(0));
      if (kBufs == 2) {
        stage_issue(S, 0, kv, nb_of(0), p, recbase, sun);
        if (nbat > 1) load_vals<B, NT>(kv, p.vals, range.x + B, nb_of(1));
      }
    }
    for (int bi = 0; bi < nbat; ++bi) {
      const int buf = kBufs == 2 ? (bi & 1) : 0;
      const uint32_t b0 = range.x + (uint32_t)(bi * B);
      const int nb = nb_of(bi);
      const bool all_done = sA.done0 && sA.done1 && sB.done0 && sB.done1;
      // both warps are done with the previous batch's buffer (refilled next), or with the tile
      if (__syncthreads_and(all_done)) break;
      if (kBufs == 1) {
        // one buffer: this batch's copies, the next batch's indices loaded meanwhile
        stage_issue(S, 0, kv, nb, p, recbase, sun);
        if (bi + 1 < nbat) load_vals<B, NT>(kv, p.vals, range.x + (uint32_t)((bi + 1) * B), nb_of(bi + 1));
        cp_async_wait_all();
      } else if (bi + 1 < nbat) {
        // the next batch's copies overlap this batch's walk
        stage_issue(S, buf ^ 1, kv, nb_of(bi + 1), p, recbase, sun);
        if (bi + 2 < nbat) load_vals<B, NT>(kv, p.vals, range.x + (uint32_t)((bi + 2) * B), nb_of(bi + 2));
        cp_async_wait_prev();
      } else {
        cp_async_wait_all();
      }
      stage_masks<TW, TH, B, NW, GL>(S, buf, nb, lg, p);
      __syncthreads();  // every thread's copies and masks of this batch are visible to the block
      uint32_t mk[mask_chunks<B, GL>()];
      batch_masks<B, GL>(S.words, lg.sub, mk);
      // a group whose 16 pixels have all stopped walks nothing
      constexpr uint32_t kGroupBits = (1u << GL) - 1u;
      if (((__ballot_sync(0xffffffffu, all_done) >> (lane & ~(GL - 1))) & kGroupBits) == kGroupBits) {
#pragma unroll
        for (int q = 0; q < mask_chunks<B, GL>(); ++q) mk[q] = 0u;
      }
      const int total = compact_candidates<GL>(mk, list, buf * B, false);
      const int nsteps = (int)__reduce_max_sync(0xffffffffu, (unsigned)total);
      auto walk = [&](auto sun_c) {
        constexpr bool SUN = decltype(sun_c)::value;
        for (int st = 0; st < nsteps; ++st) {
          // lanes whose group has nothing left evaluate a stand-in and composite nothing
          const bool has = st < total;
          const int slot = has ? (int)list[st] : buf * B;
          const float4* gs = &S.g[0][0][0] + slot * 3;
          const float4* fs = &S.f[0][0][0] + slot * 2;
          const float4 g0 = gs[0], g1 = gs[1], g2 = gs[2];
          const float4 f0 = fs[0];
          const float4 f1 = SUN ? zero4 : fs[1];
          const PairEval2 eA = eval_pair2(g0, g1, g2, x, yA, p.k);
          const PairEval2 eB = eval_pair2(g0, g1, g2, x, yB, p.k);
          const uint32_t pos = b0 + (uint32_t)(kBufs == 1 ? slot : (slot & (B - 1))) + 1u;
          const uint32_t wa = composite<SUN, DIST>(sA, eA, has, g2, f0, f1, pos, p.t_min);
          const uint32_t wb = composite<SUN, DIST>(sB, eB, has, g2, f0, f1, pos, p.t_min);
          if (COUNT) walked += wa + wb;
        }
      };
      if (sun) walk(std::true_type{}); else walk(std::false_type{});
    }
    cp_async_wait_all();  // no copy is left in flight when the walk ends early
    const TargetIO& io = p.io[t];
    const int64_t hw = (int64_t)cam.W * cam.H;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const FwdPair& s = k < 2 ? sA : sB;
      const bool hi = k & 1;
      const int py = lg.py0 + k;
      if (!(inx && py < cam.H)) continue;
      const int64_t pix = (int64_t)py * cam.W + lg.px;
      auto pick = [hi](float2 v) { return hi ? v.y : v.x; };
      if (io.rgb) {
        // the splats carry C rgb; the offset c completes C A + c (Sec. 3.1 Eq. image_formation)
        io.rgb[pix] = pick(s.A0) + cam.C[3];
        io.rgb[hw + pix] = pick(s.A1) + cam.C[7];
        io.rgb[2 * hw + pix] = pick(s.A2) + cam.C[11];
      }
      if (io.depth) io.depth[pix] = pick(s.D);
      if (io.normal) {
        io.normal[pix] = pick(s.N0);
        io.normal[hw + pix] = pick(s.N1);
        io.normal[2 * hw + pix] = pick(s.N2);
      }
      const float Tk = pick(s.T);
      if (io.alpha) io.alpha[pix] = 1.0f - Tk;
      if (DIST && io.distort) io.distort[pix] = 2.0f * pick(s.Dst);
      io.T_final[pix] = Tk;
      io.last[pix] = hi ? s.last1 : s.last0;
    }
    if (COUNT) {
      const unsigned int wsum = __reduce_add_sync(0xffffffffu, walked);
      if (lane == 0 && wsum) atomicAdd(&p.status->n_walked, (unsigned long long)wsum);
    }
    if (!q.advance()) break;
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

// Reverse-walk state of one pixel pair of a lane: T (recovered backwards), the composite behind
// (as g . S), the upstream gradients (gAlT = d(alpha_out) T_final), and for the distortion twice
// its upstream, z0, E and U.
struct BwdPair {
  float2 T, Sg, gD, gAlT, gR0, gR1, gR2, gN0, gN1, gN2;
  float2 gDs, Z0, E, U;
  uint32_t last0, last1;
};

template <bool DIST>
__device__ __forceinline__ void bwd_load_pixel(BwdPair& s, bool hi, const TargetIO& io, int64_t hw, int64_t pix,
                                               bool inside, bool sun, uint2 range) {
  float T = 1.0f, gD = 0.0f, gAlT = 0.0f, r0 = 0.0f, r1 = 0.0f, r2 = 0.0f, n0 = 0.0f, n1 = 0.0f, n2 = 0.0f;
  float gDs = 0.0f, Z0 = 0.0f, E = 0.0f;
  uint32_t last = range.x;
  if (inside) {
    T = io.T_final[pix];
    // the saved end of the walk, clamped to this tile's list
    last = min(max(io.last[pix], range.x), range.y);
    if (!sun && io.d_rgb) {
      // the splats carry C rgb, so d(rgb_out) multiplies their colour directly
      r0 = io.d_rgb[pix];
      r1 = io.d_rgb[hw + pix];
      r2 = io.d_rgb[2 * hw + pix];
    }
    if (!sun && io.d_normal) {
      n0 = io.d_normal[pix];
      n1 = io.d_normal[hw + pix];
      n2 = io.d_normal[2 * hw + pix];
    }
    if (io.d_depth) gD = io.d_depth[pix];
    if (io.d_alpha) gAlT = io.d_alpha[pix] * T;
    if (DIST && io.d_distort) {
      gDs = 2.0f * io.d_distort[pix];
      const float D = io.depth[pix], aout = 1.0f - T;
      Z0 = aout > 0.0f ? D / aout : 0.0f;
      E = -__fmaf_rn(-Z0, aout, D);
    }
  }
  auto put = [hi](float2& v, float a) { if (hi) v.y = a; else v.x = a; };
  put(s.T, T);
  put(s.Sg, 0.0f);
  put(s.gD, gD);
  put(s.gAlT, gAlT);
  put(s.gR0, r0);
  put(s.gR1, r1);
  put(s.gR2, r2);
  put(s.gN0, n0);
  put(s.gN1, n1);
  put(s.gN2, n2);
  put(s.gDs, gDs);
  put(s.Z0, Z0);
  put(s.E, E);
  put(s.U, 1.0f - T);
  if (hi) s.last1 = last; else s.last0 = last;
}

// Partials of one splat at a pixel pair, for the gradient fields.
struct BwdTerms {
  float2 w, dz, dpw, du, dv, dps;
};

// One step of the reverse walk for a pixel pair: the adjoint of compositing splat j (position j in
// the tile's list, contributing where j < last) into the pair.  A pair that does not contribute
// runs with alpha = 0, which leaves T and S unchanged and gives zero partials.
template <bool SUN, bool DIST>
__device__ __forceinline__ BwdTerms bwd_pair(BwdPair& s, const PairEval2& e, uint32_t j, const float4& g2,
                                             const float4& f0, const float4& f1, float two_inv2s2, bool& c0,
                                             bool& c1) {
  c0 = j < s.last0 && e.contrib0;  // a stand-in step carries j = ~0
  c1 = j < s.last1 && e.contrib1;
  const float2 a = make_float2(c0 ? e.alpha.x : 0.0f, c1 ? e.alpha.y : 0.0f);
  const float2 om = add2(bc2(1.0f), neg2(a));
  const float2 rom = make_float2(rcp_ftz(om.x), rcp_ftz(om.y));  // om >= 1 - alpha_max
  const float2 Ti = mul2(s.T, rom);  // T in front of the splat
  const float2 z = fma2(bc2(f0.y), e.v, fma2(bc2(f0.x), e.u, bc2(g2.w)));
  float2 gf = mul2(s.gD, z);
  if (!SUN) {
    gf = fma2(s.gR0, bc2(f1.y), gf);
    gf = fma2(s.gR1, bc2(f1.z), gf);
    gf = fma2(s.gR2, bc2(f1.w), gf);
    gf = fma2(s.gN0, bc2(f0.z), gf);
    gf = fma2(s.gN1, bc2(f0.w), gf);
    gf = fma2(s.gN2, bc2(f1.x), gf);
  }
  BwdTerms r;
  r.w = mul2(a, Ti);
  float2 dzd = bc2(0.0f);  // the distortion's partial in z
  if (DIST) {
    const float2 zs = add2(z, neg2(s.Z0));  // depth relative to z0
    gf = fma2(s.gDs, fma2(zs, s.U, s.E), gf);
    dzd = mul2(mul2(s.gDs, r.w), add2(s.U, neg2(r.w)));  // W - W' = U - w
    const float2 w2 = mul2(bc2(2.0f), r.w);
    s.U = add2(s.U, neg2(w2));
    s.E = fma2(w2, zs, s.E);
  }
  const float2 gs = add2(gf, neg2(s.Sg));
  s.T = Ti;
  s.Sg = fma2(a, gs, s.Sg);  // composite from this splat on: a f + (1 - a) S
  r.dz = fma2(r.w, s.gD, dzd);
  // d / d ln(o G^) = alpha dL/dalpha, dL/dalpha = T_i (f - S) + d(alpha_out) T_final / (1 - alpha);
  // zero when clamped (the exact adjoint of the clamp)
  const float2 dpa = mul2(fma2(Ti, gs, mul2(s.gAlT, rom)), a);
  r.dpw = make_float2(e.clamped0 ? 0.0f : dpa.x, e.clamped1 ? 0.0f : dpa.y);
  const float2 dpu = make_float2(e.uwin0 ? r.dpw.x : 0.0f, e.uwin1 ? r.dpw.y : 0.0f);
  r.dps = mul2(add2(r.dpw, neg2(dpu)), bc2(two_inv2s2));  // dpw - dpu is exact: dpw or 0
  // degenerate splats: zero slopes, and dpu = 0 except at u = v = 0
  r.du = fma2(r.dz, bc2(f0.x), neg2(mul2(dpu, e.u)));
  r.dv = fma2(r.dz, bc2(f0.y), neg2(mul2(dpu, e.v)));
  return r;
}

// The distortion's per-pixel state needs more registers: that variant runs 12 warps per SM.
template <int TW, int TH, int B, int GL, bool PERSIST, bool DIST>
__global__ void __launch_bounds__(32 * tile_warps<TW, TH>(), (DIST ? 12 : 16) / tile_warps<TW, TH>())
    raster_bwd_kernel(const __grid_constant__ RasterParams p) {
  constexpr int NW = tile_warps<TW, TH>(), NT = 32 * NW;
  static_assert(TW * TH == NW * kWarpPixels, "whole warps per tile");
  constexpr int kBufs = stage_bufs<B>();
  __shared__ TileStage<B, NW, SubMask<TW, TH, GL>, GL> S;
  __shared__ int s_item;
  __shared__ uint32_t s_hi[NW];
  const int lane = threadIdx.x & 31, grp = lane / GL, gl = lane % GL, half = threadIdx.x >> 5;
  const float4 zero4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  const float two_inv2s2 = 2.0f * p.k.inv2s2;
  ItemQueue<PERSIST> q;
  q.begin(&p.status->work_bwd, &s_item);
  while (q.item < p.total_tiles) {
    q.claim_next();
    const int tile = q.item;
    const int t = find_target(p.tcams, p.n_targets, tile);
    const TargetCam& cam = p.tcams[t];
    const LaneGeom lg = lane_geom<TW, TH, GL>(cam, tile, half);
    const bool sun = cam.sun != 0;
    const float x = (float)lg.px + 0.5f;
    const float yb = (float)lg.py0 + 0.5f;
    const float2 yA = make_float2(yb, yb + 1.0f), yB = make_float2(yb + 2.0f, yb + 3.0f);
    const uint2 range = p.ranges[tile];
    const int64_t recbase = (int64_t)t * p.n_pad;
    const TargetIO& io = p.io[t];
    // this lane's fields of the target's gradient records
    float* const gtile = p.grad + recbase * kGradFields + (16 / GL) * gl;
    const int64_t hw = (int64_t)cam.W * cam.H;
    const bool inx = lg.px < cam.W;
    BwdPair sA, sB;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int py = lg.py0 + k;
      bwd_load_pixel<DIST>(k < 2 ? sA : sB, k & 1, io, hw, (int64_t)py * cam.W + lg.px, inx && py < cam.H, sun,
                           range);
    }
    // the group's last walked position (exclusive): its walk ends there; the warp's batches start
    // at the largest one
    uint32_t glast = max(max(sA.last0, sA.last1), max(sB.last0, sB.last1));
#pragma unroll
    for (int d = 1; d < GL; d <<= 1) glast = max(glast, __shfl_xor_sync(0xffffffffu, glast, d));
    // the tile's largest last walked position: the block's batches start there
    const uint32_t whi = __reduce_max_sync(0xffffffffu, glast);
    if (lane == 0) s_hi[half] = whi;
    __syncthreads();
    uint32_t hi_all = s_hi[0];
#pragma unroll
    for (int w = 1; w < NW; ++w) hi_all = max(hi_all, s_hi[w]);
    // batches of B list entries from the warp's last walked position down; batch k is copied into
    // buffer k & 1 while batch k - 1 is walked
    const int nbat = (int)((hi_all - range.x + B - 1) / B);
    auto lo_of = [&](int k) -> uint32_t {
      const uint32_t top = hi_all - (uint32_t)(k * B);
      return top - range.x > (uint32_t)B ? top - B : range.x;
    };
    auto nb_of = [&](int k) { return (int)(hi_all - (uint32_t)(k * B) - lo_of(k)); };
    uint8_t* list = S.list[half * (32 / GL) + grp];
    uint32_t kv[per_thread<B, NT>()];  // splat indices of the next batch to copy
    if (nbat > 0) {
      load_vals<B, NT>(kv, p.vals, lo_of(0), nb_of(0));
      if (kBufs == 2) {
        stage_issue(S, 0, kv, nb_of(0), p, recbase, sun);
        if (nbat > 1) load_vals<B, NT>(kv, p.vals, lo_of(1), nb_of(1));
      }
    }
    for (int bi = 0; bi < nbat; ++bi) {
      const int buf = kBufs == 2 ? (bi & 1) : 0;
      const uint32_t b0 = lo_of(bi);
      const int nb = nb_of(bi);
      if (bi > 0) __syncthreads();  // both warps are done with the buffer refilled next
      if (kBufs == 1) {
        stage_issue(S, 0, kv, nb, p, recbase, sun);
        if (bi + 1 < nbat) load_vals<B, NT>(kv, p.vals, lo_of(bi + 1), nb_of(bi + 1));
        cp_async_wait_all();
      } else if (bi + 1 < nbat) {
        // the next (lower) batch's copies overlap this batch's walk
        stage_issue(S, buf ^ 1, kv, nb_of(bi + 1), p, recbase, sun);
        if (bi + 2 < nbat) load_vals<B, NT>(kv, p.vals, lo_of(bi + 2), nb_of(bi + 2));
        cp_async_wait_prev();
      } else {
        cp_async_wait_all();
      }
      stage_masks<TW, TH, B, NW, GL>(S, buf, nb, lg, p);
      __syncthreads();  // every thread's copies and masks of this batch are visible to the block
      uint32_t mk[mask_chunks<B, GL>()];
      batch_masks<B, GL>(S.words, lg.sub, mk);
#pragma unroll
      for (int q = 0; q < mask_chunks<B, GL>(); ++q) {
        // candidates at or after the group's last walked position are not walked
        const int lim = (int)min(max((int64_t)glast - (int64_t)b0, (int64_t)0), (int64_t)nb) - ((q * GL + gl) << 5);
        mk[q] = lim <= 0 ? 0u : (lim >= 32 ? mk[q] : mk[q] & ((1u << lim) - 1u));
      }
      const int total = compact_candidates<GL>(mk, list, buf * B, true);
      const int nsteps = (int)__reduce_max_sync(0xffffffffu, (unsigned)total);
      auto walk = [&](auto sun_c) {
        constexpr bool SUN = decltype(sun_c)::value;
        for (int st = 0; st < nsteps; ++st) {
          // reverse list order; lanes whose group has nothing left evaluate a stand-in and add
          // nothing (j = ~0 is never below a pixel's last walked position)
          const bool ok = st < total;
          const int slot = ok ? (int)list[st] : buf * B;
          const uint32_t j = ok ? b0 + (uint32_t)(kBufs == 1 ? slot : (slot & (B - 1))) : 0xffffffffu;
          const float4* gs = &S.g[0][0][0] + slot * 3;
          const float4* fs = &S.f[0][0][0] + slot * 2;
          const float4 g0 = gs[0], g1 = gs[1], g2 = gs[2];
          const float4 f0 = fs[0];
          const float4 f1 = SUN ? zero4 : fs[1];
          const uint32_t kk = (&S.k[0][0])[slot];
          const PairEval2 eA = eval_pair2(g0, g1, g2, x, yA, p.k);
          const PairEval2 eB = eval_pair2(g0, g1, g2, x, yB, p.k);
          bool cA0, cA1, cB0, cB1;
          const BwdTerms rA = bwd_pair<SUN, DIST>(sA, eA, j, g2, f0, f1, two_inv2s2, cA0, cA1);
          const BwdTerms rB = bwd_pair<SUN, DIST>(sB, eB, j, g2, f0, f1, two_inv2s2, cB0, cB1);
          // the lane's four pixels summed; terms linear in the shared column offset dx are summed
          // before they are formed
          float v[16];
          if (SUN) {
            v[GF_R] = v[GF_G] = v[GF_B] = v[GF_NX] = v[GF_NY] = v[GF_NZ] = 0.0f;
          } else {
            v[GF_R] = hsum(fma2(rB.w, sB.gR0, mul2(rA.w, sA.gR0)));
            v[GF_G] = hsum(fma2(rB.w, sB.gR1, mul2(rA.w, sA.gR1)));
            v[GF_B] = hsum(fma2(rB.w, sB.gR2, mul2(rA.w, sA.gR2)));
            v[GF_NX] = hsum(fma2(rB.w, sB.gN0, mul2(rA.w, sA.gN0)));
            v[GF_NY] = hsum(fma2(rB.w, sB.gN1, mul2(rA.w, sA.gN1)));
            v[GF_NZ] = hsum(fma2(rB.w, sB.gN2, mul2(rA.w, sA.gN2)));
          }
          v[GF_ZC] = hsum(add2(rA.dz, rB.dz));
          v[GF_DZDU] = hsum(fma2(rB.dz, eB.u, mul2(rA.dz, eA.u)));
          v[GF_DZDV] = hsum(fma2(rB.dz, eB.v, mul2(rA.dz, eA.v)));
          v[GF_LNO] = hsum(add2(rA.dpw, rB.dpw));
          const float sdu = hsum(add2(rA.du, rB.du)), sdv = hsum(add2(rA.dv, rB.dv));
          const float dx = eA.dx;
          v[GF_Q00] = sdu * dx;
          v[GF_Q01] = hsum(fma2(rB.du, eB.dy, mul2(rA.du, eA.dy)));
          v[GF_Q10] = sdv * dx;
          v[GF_Q11] = hsum(fma2(rB.dv, eB.dy, mul2(rA.dv, eA.dy)));
          v[GF_CX] = hsum(add2(rA.dps, rB.dps)) * dx - (g1.x * sdu + g1.z * sdv);
          v[GF_CY] = hsum(fma2(rB.dps, eB.dy, mul2(rA.dps, eA.dy))) - (g1.y * sdu + g1.w * sdv);
          // a real step adds its sums even where no pixel of the group contributed (zeros; 0.5 % of
          // the steps): only the stand-ins add nothing
          group_reduce16<GL, SUN>(v);
          constexpr int F = 16 / GL;  // fields summed by each lane
          float* dst = gtile + (size_t)kk * kGradFields;
#pragma unroll
          for (int r = 0; r < F / 4; ++r) {
            // a sun view's fields 12 .. 15 (normal z, colour) are zero
            if (ok && !(SUN && F * gl + 4 * r >= 12)) red_add_v4(dst + 4 * r, v[4 * r], v[4 * r + 1], v[4 * r + 2], v[4 * r + 3]);
          }
        }
      };
      if (sun) walk(std::true_type{}); else walk(std::false_type{});
    }
    cp_async_wait_all();
    // gradient of the colour offset c of this target: the sum of d(rgb_out) over its pixels
    // (the 3x3 block C is chained per splat in the projection adjoint)
    if (!sun && p.d_color && io.d_rgb) {
      float s3[3] = {hsum(add2(sA.gR0, sB.gR0)), hsum(add2(sA.gR1, sB.gR1)), hsum(add2(sA.gR2, sB.gR2))};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s3[c] += __shfl_xor_sync(0xffffffffu, s3[c], o);
      }
      if (lane == 0) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (s3[c] != 0.0f) atomicAdd(p.d_color + cam.cam * 12 + 4 * c + 3, s3[c]);
      }
    }
    if (!q.advance()) break;
  }
}

// ------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------
// One two-warp block per tile.  Persistent: as many blocks as fit on the GPU pull tiles from the
// queue; otherwise one block per tile.  Resident blocks per SM are queried once per kernel
// (outside any later stream capture).
template <typename K>
cudaError_t launch_items(K kernel, int threads, const RasterParams& p, bool persistent, int num_sms, int& per_sm,
                         cudaStream_t st) {
  const int n_items = p.total_tiles;
  if (n_items == 0) return cudaSuccess;
  int grid = n_items;
  if (persistent) {
    if (per_sm == 0) {
      int v = 0;
      const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kernel, threads, 0);
      if (e != cudaSuccess) return e;
      per_sm = v < 1 ? 1 : v;
    }
    grid = min(num_sms * per_sm, n_items);
  }
  count_launch();
  kernel<<<grid, threads, 0, st>>>(p);
  return cudaGetLastError();
}

template <int TW, int TH, bool DIST, bool COUNT>
cudaError_t launch_fwd_t(const RasterParams& p, bool persistent, int num_sms, cudaStream_t st) {
  constexpr int B = kFwdBatch, GL = kFwdGroupLanes, NT = 32 * tile_warps<TW, TH>();
  static int per_sm = 0;
  if (persistent) return launch_items(raster_fwd_kernel<TW, TH, B, GL, true, DIST, COUNT>, NT, p, true, num_sms, per_sm, st);
  return launch_items(raster_fwd_kernel<TW, TH, B, GL, false, DIST, COUNT>, NT, p, false, num_sms, per_sm, st);
}

template <int TW, int TH, bool DIST>
cudaError_t launch_bwd_t(const RasterParams& p, bool persistent, int num_sms, cudaStream_t st) {
  constexpr int B = kBwdBatch, GL = kBwdGroupLanes, NT = 32 * tile_warps<TW, TH>();
  static int per_sm = 0;
  if (persistent) return launch_items(raster_bwd_kernel<TW, TH, B, GL, true, DIST>, NT, p, true, num_sms, per_sm, st);
  return launch_items(raster_bwd_kernel<TW, TH, B, GL, false, DIST>, NT, p, false, num_sms, per_sm, st);
}

// Instantiates the launchers of one tile shape (the staging of kernels.cuh; the options' batch of
// 256 selects it), with and without the distortion, and (forward) with and without the
// walked-pair count.
#define SS_RASTER_FWD_DISPATCH(TW, TH)                                                                      \
  cudaError_t launch_raster_fwd_##TW##x##TH(const RasterParams& p, int batch, bool persistent, int num_sms, \
                                            cudaStream_t st) {                                              \
    if (batch != 256) return cudaErrorInvalidValue;                                                         \
    const bool dist = p.distort != 0, cnt = p.count_pairs != 0;                                             \
    if (dist) return cnt ? launch_fwd_t<TW, TH, true, true>(p, persistent, num_sms, st)                     \
                         : launch_fwd_t<TW, TH, true, false>(p, persistent, num_sms, st);                   \
    return cnt ? launch_fwd_t<TW, TH, false, true>(p, persistent, num_sms, st)                              \
               : launch_fwd_t<TW, TH, false, false>(p, persistent, num_sms, st);                            \
  }
#define SS_RASTER_BWD_DISPATCH(TW, TH)                                                                      \
  cudaError_t launch_raster_bwd_##TW##x##TH(const RasterParams& p, int batch, bool persistent, int num_sms, \
                                            cudaStream_t st) {                                              \
    if (batch != 256) return cudaErrorInvalidValue;                                                         \
    return p.distort ? launch_bwd_t<TW, TH, true>(p, persistent, num_sms, st)                               \
                     : launch_bwd_t<TW, TH, false>(p, persistent, num_sms, st);                             \
  }

}  // namespace ss
