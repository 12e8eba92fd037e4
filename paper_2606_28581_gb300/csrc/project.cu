// Camera assembly (a1), per-splat projection (K1) and its adjoint (K5).
//
// Sec. 3.2 Eq. affine2dgs_Qq: Q = (B_xy R S')^-1, q = -Q (B_xy p + b_xy); the kernels keep
// the projected centre c = B_xy p + b_xy instead of q (u = Q (x - c) = Q x + q).
// Sec. 3.2 Eq. depth_affine_camera: depth = max_alt - height.
// Sec. 3.3: F'_xy = F_xy + dF_xy; sun camera B_sun = B'_xy (I - [0 0 s]) (Eq. sun_camera_Bxy),
// applied here as "flatten along s, then project with S B'" (Supp. A).
#include "kernels.cuh"

namespace ss {

// ------------------------------------------------------------------------------------------
// a1: assembled cameras
// ------------------------------------------------------------------------------------------
__global__ void assemble_kernel(AssembleParams p) {
  const int t = threadIdx.x;
  if (t >= p.n_targets) return;
  const TargetStatic st = p.tg[t];
  const CamRaw cr = p.cams[st.cam];
  TargetCam tc;
  float dF[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) dF[i] = p.dF ? p.dF[st.cam * 8 + i] : 0.0f;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j) two_sum(cr.F[4 * i + j], dF[4 * i + j], tc.B[i][j], tc.Blo[i][j]);
    two_sum(cr.F[4 * i + 3], dF[4 * i + 3], tc.b[i], tc.blo[i]);
  }
  // viewing direction: the null space of B'_xy, B_x x B_y, oriented upward (toward the sensor)
  float d0 = tc.B[0][1] * tc.B[1][2] - tc.B[0][2] * tc.B[1][1];
  float d1 = tc.B[0][2] * tc.B[1][0] - tc.B[0][0] * tc.B[1][2];
  float d2 = tc.B[0][0] * tc.B[1][1] - tc.B[0][1] * tc.B[1][0];
  float inv = rsqrtf(d0 * d0 + d1 * d1 + d2 * d2) * (d2 < 0.0f ? -1.0f : 1.0f);
  tc.vs[0] = d0 * inv;
  tc.vs[1] = d1 * inv;
  tc.vs[2] = d2 * inv;
  tc.maxalt = cr.max_alt;
  if (st.sun) {
    const float ct = 1.0f / tanf(cr.theta);
    tc.s[0] = cosf(cr.phi) * ct;
    tc.s[1] = sinf(cr.phi) * ct;
    tc.s[2] = 1.0f;
    tc.S = st.S;
  } else {
    tc.s[0] = tc.s[1] = tc.s[2] = 0.0f;
    tc.S = 1.0f;
  }
  tc.W = st.W;
  tc.H = st.H;
  tc.tiles_x = st.tiles_x;
  tc.tiles_y = st.tiles_y;
  tc.tile_base = st.tile_base;
  tc.cam = st.cam;
  tc.sun = st.sun;
  tc.pad = 0;
  // colour correction [C | c] of main views (Sec. 3.1 Eq. image_formation); sun views carry none
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    const float id = (i % 4 == i / 4) ? 1.0f : 0.0f;
    tc.C[i] = (!st.sun && p.color) ? p.color[st.cam * 12 + i] : id;
  }
  p.out[t] = tc;
}

// ------------------------------------------------------------------------------------------
// Per-splat state shared by K1 and K5
// ------------------------------------------------------------------------------------------
struct SplatIn {
  float p[3], su, sv, q[4], o, rgb[3];
  float R[3][3];
  float qn[4], inv_qnorm;
  bool ok;
};

template <typename Tst>
__device__ __forceinline__ SplatIn load_splat(const ProjectCommon& pc, int64_t k) {
  SplatIn s;
  const Tst* m = static_cast<const Tst*>(pc.means);
  const Tst* sc = static_cast<const Tst*>(pc.scales);
  const Tst* qq = static_cast<const Tst*>(pc.quats);
  const Tst* op = static_cast<const Tst*>(pc.opacity);
  const Tst* cl = static_cast<const Tst*>(pc.rgb);
  const int64_t np = pc.n_pad;
#pragma unroll
  for (int i = 0; i < 3; ++i) s.p[i] = load_attr(m, i * np + k);
  s.su = load_attr(sc, k);
  s.sv = load_attr(sc, np + k);
#pragma unroll
  for (int i = 0; i < 4; ++i) s.q[i] = load_attr(qq, i * np + k);
  s.o = load_attr(op, k);
#pragma unroll
  for (int i = 0; i < 3; ++i) s.rgb[i] = load_attr(cl, i * np + k);
  float n2 = s.q[0] * s.q[0] + s.q[1] * s.q[1] + s.q[2] * s.q[2] + s.q[3] * s.q[3];
  bool fin = isfinite(s.p[0]) && isfinite(s.p[1]) && isfinite(s.p[2]) && isfinite(s.su) &&
             isfinite(s.sv) && isfinite(n2) && isfinite(s.o) && isfinite(s.rgb[0]) &&
             isfinite(s.rgb[1]) && isfinite(s.rgb[2]);
  s.ok = fin && s.su > 0.0f && s.sv > 0.0f && n2 > 0.0f;
  s.inv_qnorm = rsqrtf(n2);
  const float w = s.q[0] * s.inv_qnorm, x = s.q[1] * s.inv_qnorm, y = s.q[2] * s.inv_qnorm,
              z = s.q[3] * s.inv_qnorm;
  s.qn[0] = w; s.qn[1] = x; s.qn[2] = y; s.qn[3] = z;
  // rotation matrix of the unit quaternion (w, x, y, z); columns are t_u, t_v, n
  s.R[0][0] = 1.0f - 2.0f * (y * y + z * z);
  s.R[0][1] = 2.0f * (x * y - w * z);
  s.R[0][2] = 2.0f * (x * z + w * y);
  s.R[1][0] = 2.0f * (x * y + w * z);
  s.R[1][1] = 1.0f - 2.0f * (x * x + z * z);
  s.R[1][2] = 2.0f * (y * z - w * x);
  s.R[2][0] = 2.0f * (x * z - w * y);
  s.R[2][1] = 2.0f * (y * z + w * x);
  s.R[2][2] = 1.0f - 2.0f * (x * x + y * y);
  return s;
}

// Projection of one splat into one target.
struct SplatProj {
  float RSf[3][2];   // S' axes, flattened along s for sun targets
  float ph[3], pl[3];// centre, flattened for sun targets, as a float pair
  float M[2][2], det, Q[2][2];
  float chi[2], clo[2];
  bool deg;
  float flip;
};

__device__ __forceinline__ SplatProj project_one(const SplatIn& s, const TargetCam& cam, float det_eps) {
  SplatProj r;
  float RS[3][2];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    RS[j][0] = s.su * s.R[j][0];
    RS[j][1] = s.sv * s.R[j][1];
  }
  if (cam.sun) {
    // flatten onto z = 0 along s (s_z = 1): p' = p - p_z s, axes a' = a - a_z s
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      float t, te, h, l;
      two_prod(s.p[2], cam.s[j], t, te);
      two_sum(s.p[j], -t, h, l);
      r.ph[j] = h;
      r.pl[j] = __fsub_rn(l, te);
      r.RSf[j][0] = __fmaf_rn(-cam.s[j], RS[2][0], RS[j][0]);
      r.RSf[j][1] = __fmaf_rn(-cam.s[j], RS[2][1], RS[j][1]);
    }
    r.ph[2] = 0.0f; r.pl[2] = 0.0f;
    r.RSf[2][0] = 0.0f; r.RSf[2][1] = 0.0f;
  } else {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      r.ph[j] = s.p[j];
      r.pl[j] = 0.0f;
      r.RSf[j][0] = RS[j][0];
      r.RSf[j][1] = RS[j][1];
    }
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      float m = __fmul_rn(cam.B[i][0], r.RSf[0][c]);
      m = __fmaf_rn(cam.B[i][1], r.RSf[1][c], m);
      m = __fmaf_rn(cam.B[i][2], r.RSf[2][c], m);
      r.M[i][c] = __fmul_rn(cam.S, m);
    }
    // c = S (B' p' + b') as a float pair
    float hi = cam.b[i], lo = cam.blo[i];
#pragma unroll
    for (int j = 0; j < 3; ++j) ff_fma(hi, lo, cam.B[i][j], cam.Blo[i][j], r.ph[j], r.pl[j]);
    ff_renorm(hi, lo);
    if (cam.sun) {
      float h2, e2;
      two_prod(hi, cam.S, h2, e2);
      lo = __fmaf_rn(lo, cam.S, e2);
      hi = h2;
      ff_renorm(hi, lo);
    }
    r.chi[i] = hi;
    r.clo[i] = lo;
  }
  r.det = det2(r.M[0][0], r.M[0][1], r.M[1][0], r.M[1][1]);
  r.deg = !(fabsf(r.det) >= det_eps);
  if (!r.deg) {
    const float id = 1.0f / r.det;
    r.Q[0][0] = r.M[1][1] * id;
    r.Q[0][1] = -r.M[0][1] * id;
    r.Q[1][0] = -r.M[1][0] * id;
    r.Q[1][1] = r.M[0][0] * id;
  } else {
    // drawn by the screen-space term alone (see kDegenerateQ)
    r.Q[0][0] = r.Q[1][1] = kDegenerateQ;
    r.Q[0][1] = r.Q[1][0] = 0.0f;
  }
  const float nd = s.R[0][2] * cam.vs[0] + s.R[1][2] * cam.vs[1] + s.R[2][2] * cam.vs[2];
  r.flip = nd < 0.0f ? -1.0f : 1.0f;
  return r;
}

// ------------------------------------------------------------------------------------------
// K1: projection of every splat into every target
// ------------------------------------------------------------------------------------------
template <typename Tst>
__global__ void __launch_bounds__(256, 3) project_kernel(ProjectParams p) {
  __shared__ TargetCam scam[kMaxTargets];
  for (int t = threadIdx.x; t < p.c.n_targets; t += blockDim.x) scam[t] = p.c.tcams[t];
  __syncthreads();
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= p.c.n) return;
  const SplatIn s = load_splat<Tst>(p.c, k);
  if (!s.ok) atomicAdd(&p.status->nonfinite, 1ull);
  const bool alive = s.ok && (s.o >= p.amin);
  const float lno = logf(s.o);
  const float r = sqrtf(fmaxf(2.0f * (lno - p.ln_amin), 0.0f));
  const int64_t np = p.c.n_pad;
  for (int t = 0; t < p.c.n_targets; ++t) {
    const TargetCam& cam = scam[t];
    const int64_t rec = (int64_t)t * np + k;
    uint4 trec = make_uint4(0u, 0u, 0u, 0u);
    if (alive) {
      const SplatProj sp = project_one(s, cam, p.det_eps);
      const float m0 = sp.deg ? 0.0f : sqrtf(sp.M[0][0] * sp.M[0][0] + sp.M[0][1] * sp.M[0][1]);
      const float m1 = sp.deg ? 0.0f : sqrtf(sp.M[1][0] * sp.M[1][0] + sp.M[1][1] * sp.M[1][1]);
      // conservative half extents of {alpha >= alpha_min}: r max(|M_i,:|, sigma), padded
      const float ex = r * fmaxf(m0, p.sigma) * 1.0001f + 0.01f;
      const float ey = r * fmaxf(m1, p.sigma) * 1.0001f + 0.01f;
      const float cx = sp.chi[0], cy = sp.chi[1];
      const bool fin = isfinite(cx) && isfinite(cy) && isfinite(sp.det) && isfinite(ex) && isfinite(ey);
      if (fin) {
        // pixels i with |i + 0.5 - cx| <= ex
        float ilo = fmaxf(ceilf(cx - ex - 0.5f), 0.0f);
        float ihi = fminf(floorf(cx + ex - 0.5f), (float)(cam.W - 1));
        float jlo = fmaxf(ceilf(cy - ey - 0.5f), 0.0f);
        float jhi = fminf(floorf(cy + ey - 0.5f), (float)(cam.H - 1));
        const float4 g0 = make_float4(sp.chi[0], sp.chi[1], sp.clo[0], sp.clo[1]);
        const float4 g1 = make_float4(sp.Q[0][0], sp.Q[0][1], sp.Q[1][0], sp.Q[1][1]);
        const float4 g2 = make_float4(lno, sp.deg ? -ex : ex, ey, cam.maxalt - s.p[2]);
        uint32_t count = 0, mask = 0;
        int tx0 = 0, ty0 = 0, tx1 = -1, ty1 = -1;
        if (ilo <= ihi && jlo <= jhi) {
          tx0 = (int)ilo / p.tile_w; tx1 = (int)ihi / p.tile_w;
          ty0 = (int)jlo / p.tile_h; ty1 = (int)jhi / p.tile_h;
          const int ntx = tx1 - tx0 + 1, nty = ty1 - ty0 + 1;
          if (ntx * nty > 32) {
            // large footprint: keep every tile of the rectangle
            mask = 0xffffffffu;
            count = (uint32_t)(ntx * nty);
          } else {
            // per row of the rectangle, the tiles whose pixel-centre rectangles (padded by
            // 2e-3 px) meet the support's slice through the row's pixel rows
            constexpr float kPad = 2e-3f;
            const float inv_tw = 1.0f / (float)p.tile_w;  // tile widths are powers of two
            SupportSlices sl;
            sl.init(g1, g2, p.cull);
            for (int ty = ty0; ty <= ty1; ++ty) {
              const float yl = ((float)(ty * p.tile_h) + 0.5f - cy) - kPad;
              const float yh = ((float)(min((ty + 1) * p.tile_h, cam.H) - 1) + 0.5f - cy) + kPad;
              float lo, hi;
              sl.range(yl, yh, lo, hi);
              // tiles tx with [tx w + 0.5, tx w + w - 0.5] - cx (padded) meeting [lo, hi]
              const float cl = fmaxf(ceilf(((lo + cx) - 0.5f - kPad - (float)(p.tile_w - 1)) * inv_tw), (float)tx0);
              const float ch = fminf(floorf(((hi + cx) - 0.5f + kPad) * inv_tw), (float)tx1);
              if (cl <= ch) {
                const int a = (int)cl - tx0, z = (int)ch - tx0;
                mask |= ((2u << z) - (1u << a)) << ((ty - ty0) * ntx);
              }
            }
            count = (uint32_t)__popc(mask);
          }
        }
        if (count > 0) {
          trec = make_uint4((uint32_t)tx0 | ((uint32_t)ty0 << 16), (uint32_t)tx1 | ((uint32_t)ty1 << 16), mask,
                            count);
          float4* g = p.geom + rec * 3;
          g[0] = g0;
          g[1] = g1;
          g[2] = g2;
          float4* f = p.feat + rec * 2;
          // a degenerate splat's depth is zc at every pixel (u = v = 0 in the per-pixel definition)
          f[0] = make_float4(sp.deg ? 0.0f : -s.su * s.R[2][0], sp.deg ? 0.0f : -s.sv * s.R[2][1],
                             sp.flip * s.R[0][2], sp.flip * s.R[1][2]);
          // C (sum w rgb) = sum w (C rgb): main views composite the corrected splat colour
          const float* C = cam.C;
          f[1] = make_float4(sp.flip * s.R[2][2], C[0] * s.rgb[0] + C[1] * s.rgb[1] + C[2] * s.rgb[2],
                             C[4] * s.rgb[0] + C[5] * s.rgb[1] + C[6] * s.rgb[2],
                             C[8] * s.rgb[0] + C[9] * s.rgb[1] + C[10] * s.rgb[2]);
          float4* gz = p.grad + rec * 4;
          const float4 z4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
          gz[0] = z4;
          gz[1] = z4;
          gz[2] = z4;
          gz[3] = z4;
        }
      }
    }
    p.rect[rec] = trec;
  }
}

// ------------------------------------------------------------------------------------------
// K5: chain the per-(target, splat) gradient records through the projection
// ------------------------------------------------------------------------------------------
// AHEAD: each target's gradient record is loaded one target ahead, at two blocks per SM (the
// registers it takes); without it, three blocks per SM load each record in its own iteration,
// which suits frames of few targets.
template <typename Tst, bool AHEAD>
__global__ void __launch_bounds__(256, AHEAD ? 2 : 3) project_bwd_kernel(ProjectBwdParams p) {
  __shared__ TargetCam scam[kMaxTargets];
  // the block's camera-delta and colour sums per target: d/d[B' | b'] (8) and d/dC (9)
  __shared__ float sred[kMaxTargets][17];
  for (int t = threadIdx.x; t < p.c.n_targets; t += blockDim.x) scam[t] = p.c.tcams[t];
  for (int i = threadIdx.x; i < p.c.n_targets * 17; i += blockDim.x) (&sred[0][0])[i] = 0.0f;
  __syncthreads();
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = k < p.c.n;
  SplatIn s;
  if (valid) s = load_splat<Tst>(p.c, k);
  const bool alive = valid && s.ok && (s.o >= p.amin);
  float dp[3] = {0, 0, 0}, dsu = 0, dsv = 0, dlno = 0, drgb[3] = {0, 0, 0};
  float dR[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  const int64_t np = p.c.n_pad;
  const int lane = threadIdx.x & 31;
  // with AHEAD a target's gradient record is loaded one target ahead; its tile count is loaded two
  // ahead, so that each request goes out before its use
  const int nt = p.c.n_targets;
  const float4 z4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  auto load_rec = [&](int64_t rec, float4 (&r)[4]) {
    const float4* gp = reinterpret_cast<const float4*>(p.grad + rec * kGradFields);
    r[0] = gp[0]; r[1] = gp[1]; r[2] = gp[2]; r[3] = gp[3];
  };
  uint32_t count_cur = alive ? p.rect[k].w : 0u;
  uint32_t count_next = (alive && nt > 1) ? p.rect[np + k].w : 0u;
  float4 rnext[4] = {z4, z4, z4, z4};
  if (AHEAD && count_cur > 0u) load_rec(k, rnext);
  for (int t = 0; t < p.c.n_targets; ++t) {
    const TargetCam& cam = scam[t];
    // per target: d/d[B' | b'] (8) and d/dC of the colour correction's 3x3 block (9)
    float dBp[16] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    float dC22 = 0.0f;
    const int64_t rec = (int64_t)t * np + k;
    const bool live = count_cur > 0u;  // the pair was emitted to at least one tile
    if (!AHEAD && live) load_rec(rec, rnext);
    const float4 a = rnext[0], b = rnext[1], c = rnext[2], d = rnext[3];
    if (t + 1 < nt) {
      if (AHEAD && count_next > 0u) load_rec(rec + np, rnext);
      count_cur = count_next;
      count_next = (alive && t + 2 < nt) ? p.rect[rec + 2 * np].w : 0u;
    }
    if (live) {
      const float g[16] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w, d.x, d.y, d.z, d.w};
      const SplatProj sp = project_one(s, cam, p.det_eps);
      // Q = M^-1: dM = -Q^T dQ Q^T
      float dM[2][2] = {{0, 0}, {0, 0}};
      if (!sp.deg) {
        const float dQ[2][2] = {{g[GF_Q00], g[GF_Q01]}, {g[GF_Q10], g[GF_Q11]}};
        float tq[2][2];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int j = 0; j < 2; ++j) tq[i][j] = sp.Q[0][i] * dQ[0][j] + sp.Q[1][i] * dQ[1][j];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int j = 0; j < 2; ++j) dM[i][j] = -(tq[i][0] * sp.Q[j][0] + tq[i][1] * sp.Q[j][1]);
      }
      const float dc[2] = {g[GF_CX], g[GF_CY]};
      const float S = cam.S;
      // c = S (B' p' + b'),  M = S B' RSf
      float dpf[3] = {0, 0, 0}, dRSf[3][2] = {{0, 0}, {0, 0}, {0, 0}};
#pragma unroll
      for (int i = 0; i < 2; ++i) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const float pj = sp.ph[j] + sp.pl[j];
          dBp[4 * i + j] += S * (dc[i] * pj + dM[i][0] * sp.RSf[j][0] + dM[i][1] * sp.RSf[j][1]);
          dpf[j] += S * cam.B[i][j] * dc[i];
          dRSf[j][0] += S * cam.B[i][j] * dM[i][0];
          dRSf[j][1] += S * cam.B[i][j] * dM[i][1];
        }
        dBp[4 * i + 3] += S * dc[i];
      }
      float dRS[3][2];
      if (cam.sun) {
        // p'_j = p_j - p_z s_j (j < 2), p'_z = 0; the same flattening for the axes
        dp[0] += dpf[0];
        dp[1] += dpf[1];
        dp[2] += -(cam.s[0] * dpf[0] + cam.s[1] * dpf[1]);
#pragma unroll
        for (int c2 = 0; c2 < 2; ++c2) {
          dRS[0][c2] = dRSf[0][c2];
          dRS[1][c2] = dRSf[1][c2];
          dRS[2][c2] = -(cam.s[0] * dRSf[0][c2] + cam.s[1] * dRSf[1][c2]);
        }
      } else {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          dp[j] += dpf[j];
          dRS[j][0] = dRSf[j][0];
          dRS[j][1] = dRSf[j][1];
        }
      }
      // depth at the centre zc = max_alt - p_z and its slopes dzdu = -s_u R20, dzdv = -s_v R21
      dp[2] -= g[GF_ZC];
      if (!sp.deg) {  // a degenerate splat's depth has no slope term (its u, v fields are meaningless)
        dRS[2][0] -= g[GF_DZDU];
        dRS[2][1] -= g[GF_DZDV];
      }
      // RS' = [s_u R[:,0], s_v R[:,1]]
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        dsu += dRS[j][0] * s.R[j][0];
        dsv += dRS[j][1] * s.R[j][1];
        dR[j][0] += s.su * dRS[j][0];
        dR[j][1] += s.sv * dRS[j][1];
      }
      // normal = flip R[:,2]
      dR[0][2] += sp.flip * g[GF_NX];
      dR[1][2] += sp.flip * g[GF_NY];
      dR[2][2] += sp.flip * g[GF_NZ];
      dlno += g[GF_LNO];
      if (!cam.sun) {
        // the record holds H = sum_px w d(rgb_out): the splat composited C rgb, so
        // d rgb = C^T H and dC = H rgb^T (Sec. 3.1 Eq. image_formation)
        const float H[3] = {g[GF_R], g[GF_G], g[GF_B]};
#pragma unroll
        for (int j = 0; j < 3; ++j) drgb[j] += cam.C[j] * H[0] + cam.C[4 + j] * H[1] + cam.C[8 + j] * H[2];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            if (3 * i + j < 8) dBp[8 + 3 * i + j] = H[i] * s.rgb[j];
          }
        dC22 = H[2] * s.rgb[2];
      }
    }
    // camera-delta and colour gradients of this target: warp sums into the block's per-target
    // sums (no block barrier per target)
    if (p.d_dF != nullptr || (p.d_color != nullptr && !cam.sun)) {
      const float tot = warp_reduce16_transposed(dBp);
      float t22 = dC22;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t22 += __shfl_xor_sync(0xffffffffu, t22, o);
      if (!(lane & 1) && tot != 0.0f) atomicAdd(&sred[t][lane >> 1], tot);
      if (lane == 0 && t22 != 0.0f) atomicAdd(&sred[t][16], t22);
    }
  }
  // one atomic per target and field for the block
  __syncthreads();
  for (int i = threadIdx.x; i < p.c.n_targets * 17; i += blockDim.x) {
    const int t = i / 17, f = i - t * 17;
    const float acc = sred[t][f];
    if (acc == 0.0f) continue;
    const TargetCam& cam = scam[t];
    if (f < 8) {
      if (p.d_dF) atomicAdd(p.d_dF + cam.cam * 8 + f, acc);
    } else if (p.d_color && !cam.sun) {
      const int ij = f - 8, i2 = ij / 3, j = ij % 3;  // dC[i2][j], row-major [C | c]
      atomicAdd(p.d_color + cam.cam * 12 + 4 * i2 + j, acc);
    }
  }
  if (!alive) return;
  // R(q_n) -> d q_n, through the normalisation -> d q
  const float w = s.qn[0], x = s.qn[1], y = s.qn[2], z = s.qn[3];
  // dR entries weighted by the partials of each R entry with respect to (w, x, y, z)
  const float A01 = dR[0][1] - dR[1][0];  // antisymmetric parts carry w
  const float A02 = dR[0][2] - dR[2][0];
  const float A12 = dR[1][2] - dR[2][1];
  const float S01 = dR[0][1] + dR[1][0];  // symmetric parts
  const float S02 = dR[0][2] + dR[2][0];
  const float S12 = dR[1][2] + dR[2][1];
  float gq[4];
  gq[0] = 2.0f * (-z * A01 + y * A02 - x * A12);
  gq[1] = 2.0f * (y * S01 + z * S02 - w * A12) - 4.0f * x * (dR[1][1] + dR[2][2]);
  gq[2] = 2.0f * (x * S01 + w * A02 + z * S12) - 4.0f * y * (dR[0][0] + dR[2][2]);
  gq[3] = 2.0f * (-w * A01 + x * S02 + y * S12) - 4.0f * z * (dR[0][0] + dR[1][1]);
  const float dot = gq[0] * w + gq[1] * x + gq[2] * y + gq[3] * z;
  float* dq = p.g.quats;
#pragma unroll
  for (int i = 0; i < 4; ++i) dq[i * p.g.n_pad + k] += (gq[i] - s.qn[i] * dot) * s.inv_qnorm;
#pragma unroll
  for (int i = 0; i < 3; ++i) p.g.means[i * p.g.n_pad + k] += dp[i];
  p.g.scales[k] += dsu;
  p.g.scales[p.g.n_pad + k] += dsv;
  p.g.opacity[k] += dlno / s.o;  // lno = log(o)
#pragma unroll
  for (int i = 0; i < 3; ++i) p.g.rgb[i * p.g.n_pad + k] += drgb[i];
}

// ------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------
cudaError_t launch_assemble(const AssembleParams& p, cudaStream_t st) {
  count_launch();
  assemble_kernel<<<1, kMaxTargets, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_project(const ProjectParams& p, int dtype, cudaStream_t st) {
  const int64_t nb = (p.c.n + 255) / 256;
  if (nb == 0) return cudaSuccess;
  if (dtype == SS_BF16) {
    count_launch();
    project_kernel<__nv_bfloat16><<<(unsigned)nb, 256, 0, st>>>(p);
  } else {
    count_launch();
    project_kernel<float><<<(unsigned)nb, 256, 0, st>>>(p);
  }
  return cudaGetLastError();
}

cudaError_t launch_project_bwd(const ProjectBwdParams& p, int dtype, cudaStream_t st) {
  const int64_t nb = (p.c.n + 255) / 256;
  if (nb == 0) return cudaSuccess;
  // records loaded a target ahead pay off over many targets (0.69 -> 0.53 ms at 32 targets); with
  // two (a view and its sun view) the occupancy they cost weighs more (0.069 -> 0.080 ms)
  const bool ahead = p.c.n_targets > 4;
  if (dtype == SS_BF16) {
    count_launch();
    if (ahead) project_bwd_kernel<__nv_bfloat16, true><<<(unsigned)nb, 256, 0, st>>>(p);
    else project_bwd_kernel<__nv_bfloat16, false><<<(unsigned)nb, 256, 0, st>>>(p);
  } else {
    count_launch();
    if (ahead) project_bwd_kernel<float, true><<<(unsigned)nb, 256, 0, st>>>(p);
    else project_bwd_kernel<float, false><<<(unsigned)nb, 256, 0, st>>>(p);
  }
  return cudaGetLastError();
}

}  // namespace ss
