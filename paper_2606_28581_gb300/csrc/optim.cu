// Optimiser step of the splats: fused Adam with the 3DGS-MCMC position noise, and the
// 3DGS-MCMC relocation of dead splats with growth toward a fixed budget (Sec. 3.5, Sec. 4.4;
// learning rates of Supp. B).  Random numbers: Philox4x64-10 (Salmon et al., SC'11).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "kernels.cuh"

using namespace ss;

namespace {

// ------------------------------------------------------------------------------------------
// Philox4x64-10: the multipliers and Weyl key increments of the published generator
// ------------------------------------------------------------------------------------------
constexpr unsigned long long kPhiloxM0 = 0xD2E7470EE14C6C93ull;
constexpr unsigned long long kPhiloxM1 = 0xCA5A826395121157ull;
constexpr unsigned long long kPhiloxW0 = 0x9E3779B97F4A7C15ull;
constexpr unsigned long long kPhiloxW1 = 0xBB67AE8584CAA73Bull;
constexpr unsigned long long kStreamNoise = 0ull;
constexpr unsigned long long kStreamRelocate = 1ull;

struct U64x4 {
  unsigned long long x, y, z, w;
};

__device__ __forceinline__ U64x4 philox4x64_10(U64x4 c, unsigned long long k0, unsigned long long k1) {
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

// a uniform in (0, 1) from the top 24 bits (exact in float)
__device__ __forceinline__ float uniform24(unsigned long long x) {
  return ((float)(x >> 40) + 0.5f) * 5.9604644775390625e-8f;
}

// ------------------------------------------------------------------------------------------
// storage of the activated values (fp32 or bf16, round to nearest even)
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void store_act(void* base, int32_t dtype, int64_t idx, float a) {
  if (dtype == SS_F32)
    static_cast<float*>(base)[idx] = a;
  else
    static_cast<__nv_bfloat16*>(base)[idx] = __float2bfloat16_rn(a);
}

__device__ __forceinline__ float sigmoid_f(float x) { return 1.0f / (1.0f + expf(-x)); }

// ------------------------------------------------------------------------------------------
// fused Adam + position noise: each thread owns four consecutive splats (16-byte accesses)
// ------------------------------------------------------------------------------------------
enum { G_MEANS = 0, G_SCALES = 1, G_QUATS = 2, G_OPAC = 3, G_RGB = 4 };

struct AdamParams {
  float* p[5];        // raw rows: means, log_scales, quats, logit_opacity, rgb
  float* m[5];
  float* v[5];
  const float* g[5];  // gradients with respect to the activated values, same rows
  void* st[5];        // storage arrays (activated values)
  int32_t dtype;
  int64_t n, n_pad;
  float lr[5];
  float beta1, beta2, eps, inv_bc1, inv_bc2;
  float noise_coef;  // lr_means * noise_lr (0: no noise)
  float noise_k, noise_t;
  unsigned long long step, seed;
};

struct Lanes {
  float v[4];
};

__device__ __forceinline__ Lanes load4(const float* p, bool full, int cnt) {
  Lanes r;
  if (full) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w;
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) r.v[k] = k < cnt ? p[k] : 0.0f;
  }
  return r;
}

__device__ __forceinline__ void store4(float* p, const Lanes& a, bool full, int cnt) {
  if (full) {
    *reinterpret_cast<float4*>(p) = make_float4(a.v[0], a.v[1], a.v[2], a.v[3]);
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k < cnt) p[k] = a.v[k];
  }
}

__device__ __forceinline__ void store_act4(void* base, int32_t dtype, int64_t idx, const Lanes& a, bool full,
                                           int cnt) {
  if (full && dtype == SS_F32) {
    *reinterpret_cast<float4*>(static_cast<float*>(base) + idx) = make_float4(a.v[0], a.v[1], a.v[2], a.v[3]);
  } else if (full) {
    __nv_bfloat162 lo = __floats2bfloat162_rn(a.v[0], a.v[1]), hi = __floats2bfloat162_rn(a.v[2], a.v[3]);
    uint2 u;
    u.x = *reinterpret_cast<uint32_t*>(&lo);
    u.y = *reinterpret_cast<uint32_t*>(&hi);
    *reinterpret_cast<uint2*>(static_cast<__nv_bfloat16*>(base) + idx) = u;
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k < cnt) store_act(base, dtype, idx + k, a.v[k]);
  }
}

// Adam on one row of four splats; the incoming gradient is multiplied by `chain` (the
// derivative of the activation) when CHAIN.  Returns the updated raw values.
template <bool CHAIN>
__device__ __forceinline__ Lanes adam_row(const AdamParams& a, int grp, int row, int64_t i0, const Lanes& chain,
                                          bool full, int cnt) {
  const int64_t idx = (int64_t)row * a.n_pad + i0;
  const Lanes g = load4(a.g[grp] + idx, full, cnt);
  Lanes x = load4(a.p[grp] + idx, full, cnt), m = load4(a.m[grp] + idx, full, cnt),
        v = load4(a.v[grp] + idx, full, cnt);
  const float lr = a.lr[grp];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float gk = CHAIN ? g.v[k] * chain.v[k] : g.v[k];
    m.v[k] = a.beta1 * m.v[k] + (1.0f - a.beta1) * gk;
    v.v[k] = a.beta2 * v.v[k] + (1.0f - a.beta2) * gk * gk;
    x.v[k] = x.v[k] - lr * (m.v[k] * a.inv_bc1) / (sqrtf(v.v[k] * a.inv_bc2) + a.eps);
  }
  store4(a.m[grp] + idx, m, full, cnt);
  store4(a.v[grp] + idx, v, full, cnt);
  return x;
}

// four blocks per SM (64 registers) measured 12 % faster than the three of 72 registers
__global__ void __launch_bounds__(256, 4) adam_kernel(const __grid_constant__ AdamParams a) {
  const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (i0 >= a.n) return;
  const int cnt = (int)min((int64_t)4, a.n - i0);
  const bool full = cnt == 4;
  const Lanes none{};
  // opacity: d logit = o (1 - o) d o, with o from the raw value before the step
  Lanes op;
  {
    const Lanes x = load4(a.p[G_OPAC] + i0, full, cnt);
    Lanes ch;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float o = sigmoid_f(x.v[k]);
      ch.v[k] = o * (1.0f - o);
    }
    const Lanes xn = adam_row<true>(a, G_OPAC, 0, i0, ch, full, cnt);
    store4(a.p[G_OPAC] + i0, xn, full, cnt);
#pragma unroll
    for (int k = 0; k < 4; ++k) op.v[k] = sigmoid_f(xn.v[k]);
    store_act4(a.st[G_OPAC], a.dtype, i0, op, full, cnt);
  }
  // scales: d log s = s d s
  Lanes sc[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int64_t idx = (int64_t)r * a.n_pad + i0;
    const Lanes x = load4(a.p[G_SCALES] + idx, full, cnt);
    Lanes ch;
#pragma unroll
    for (int k = 0; k < 4; ++k) ch.v[k] = expf(x.v[k]);
    const Lanes xn = adam_row<true>(a, G_SCALES, r, i0, ch, full, cnt);
    store4(a.p[G_SCALES] + idx, xn, full, cnt);
#pragma unroll
    for (int k = 0; k < 4; ++k) sc[r].v[k] = expf(xn.v[k]);
    store_act4(a.st[G_SCALES], a.dtype, idx, sc[r], full, cnt);
  }
  // quaternions, rgb: identity activations
  Lanes q[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t idx = (int64_t)r * a.n_pad + i0;
    q[r] = adam_row<false>(a, G_QUATS, r, i0, none, full, cnt);
    store4(a.p[G_QUATS] + idx, q[r], full, cnt);
    store_act4(a.st[G_QUATS], a.dtype, idx, q[r], full, cnt);
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const int64_t idx = (int64_t)r * a.n_pad + i0;
    const Lanes xn = adam_row<false>(a, G_RGB, r, i0, none, full, cnt);
    store4(a.p[G_RGB] + idx, xn, full, cnt);
    store_act4(a.st[G_RGB], a.dtype, idx, xn, full, cnt);
  }
  // means, then the position noise from the updated opacity, scales and rotation:
  // Sigma eta = s_u^2 (t_u . eta) t_u + s_v^2 (t_v . eta) t_v, t_u and t_v the first two
  // columns of R
  Lanes mu[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) mu[r] = adam_row<false>(a, G_MEANS, r, i0, none, full, cnt);
  if (a.noise_coef != 0.0f) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (k >= cnt) continue;
      const U64x4 x = philox4x64_10(U64x4{(unsigned long long)(i0 + k), a.step, kStreamNoise, 0ull}, a.seed, 0ull);
      const float u0 = uniform24(x.x), u1 = uniform24(x.y), u2 = uniform24(x.z), u3 = uniform24(x.w);
      const float r0 = sqrtf(-2.0f * logf(u0)), r1 = sqrtf(-2.0f * logf(u2));
      float s1, c1;
      sincospif(2.0f * u1, &s1, &c1);
      const float e0 = r0 * c1, e1 = r0 * s1, e2 = r1 * cospif(2.0f * u3);
      float qw = q[0].v[k], qx = q[1].v[k], qy = q[2].v[k], qz = q[3].v[k];
      const float inv = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
      qw *= inv; qx *= inv; qy *= inv; qz *= inv;
      const float tu0 = 1.0f - 2.0f * (qy * qy + qz * qz), tu1 = 2.0f * (qx * qy + qw * qz),
                  tu2 = 2.0f * (qx * qz - qw * qy);
      const float tv0 = 2.0f * (qx * qy - qw * qz), tv1 = 1.0f - 2.0f * (qx * qx + qz * qz),
                  tv2 = 2.0f * (qy * qz + qw * qx);
      const float su = sc[0].v[k], sv = sc[1].v[k];
      const float cu = su * su * (tu0 * e0 + tu1 * e1 + tu2 * e2);
      const float cv = sv * sv * (tv0 * e0 + tv1 * e1 + tv2 * e2);
      const float gate = 1.0f / (1.0f + expf(a.noise_k * (op.v[k] - a.noise_t)));
      const float coef = a.noise_coef * gate;
      mu[0].v[k] += coef * (cu * tu0 + cv * tv0);
      mu[1].v[k] += coef * (cu * tu1 + cv * tv1);
      mu[2].v[k] += coef * (cu * tu2 + cv * tv2);
    }
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const int64_t idx = (int64_t)r * a.n_pad + i0;
    store4(a.p[G_MEANS] + idx, mu[r], full, cnt);
    store_act4(a.st[G_MEANS], a.dtype, idx, mu[r], full, cnt);
  }
}

struct FlatAdam {
  float* p;
  float* m;
  float* v;
  const float* g;
  int64_t n;
  float lr, beta1, beta2, eps, inv_bc1, inv_bc2;
};

__global__ void __launch_bounds__(256) adam_flat_kernel(const __grid_constant__ FlatAdam a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const float g = a.g[i];
  const float m = a.beta1 * a.m[i] + (1.0f - a.beta1) * g;
  const float v = a.beta2 * a.v[i] + (1.0f - a.beta2) * g * g;
  a.m[i] = m;
  a.v[i] = v;
  a.p[i] = a.p[i] - a.lr * (m * a.inv_bc1) / (sqrtf(v * a.inv_bc2) + a.eps);
}

// ------------------------------------------------------------------------------------------
// 3DGS-MCMC relocation
// ------------------------------------------------------------------------------------------
struct Params13 {
  float* row[13];  // the 13 raw rows in the order means(3), log_scales(2), quats(4), opacity, rgb(3)
};

struct McmcParams {
  Params13 p, m, v;
  void* st[5];
  int32_t dtype;
  int64_t n_pad, n_active, n_targets, n_dead;
  const void* stored_opacity;
  float min_opacity;
  int32_t n_max;
  unsigned long long step, seed, W;
  uint32_t* w;       // [n_active] integer weights
  uint32_t* dead;    // [n_active] 0/1
  uint32_t* dpos;    // [n_active] exclusive scan of dead
  unsigned long long* excl;  // [n_active] exclusive scan of w
  uint32_t* counts;  // [n_active] times each splat was drawn
  uint32_t* tgt;     // [n_targets]
  uint32_t* src;     // [n_targets]
  uint32_t* ulist;   // the distinct sources, in no particular order
  uint32_t* n_ulist; // their count
  int64_t* d_stats;  // optional
  const unsigned long long* totals;  // [2]: dead count, total weight
};

__device__ __forceinline__ float load_opacity(const void* p, int32_t dtype, int64_t i) {
  return dtype == SS_F32 ? static_cast<const float*>(p)[i]
                         : __bfloat162float(static_cast<const __nv_bfloat16*>(p)[i]);
}

__global__ void __launch_bounds__(256) mcmc_weights_kernel(const __grid_constant__ McmcParams q) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= q.n_active) return;
  const float o = load_opacity(q.stored_opacity, q.dtype, i);
  const bool dead = o <= q.min_opacity;
  // o <= 1, so o 2^24 is exact and its floor fits 25 bits
  q.w[i] = dead ? 0u : (uint32_t)floorf(o * 16777216.0f);
  q.dead[i] = dead ? 1u : 0u;
  q.counts[i] = 0u;
}

__global__ void __launch_bounds__(256) mcmc_compact_kernel(const __grid_constant__ McmcParams q) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && q.d_stats) {
    q.d_stats[0] = (int64_t)q.totals[0];
    q.d_stats[1] = (int64_t)q.totals[1];
  }
  if (i >= q.n_active || !q.dead[i]) return;
  q.tgt[q.dpos[i]] = (uint32_t)i;
}

__global__ void __launch_bounds__(256) mcmc_draw_kernel(const __grid_constant__ McmcParams q) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= q.n_targets) return;
  const int64_t t = j < q.n_dead ? (int64_t)q.tgt[j] : q.n_active + (j - q.n_dead);
  const U64x4 x = philox4x64_10(U64x4{(unsigned long long)j, q.step, kStreamRelocate, 0ull}, q.seed, 0ull);
  const unsigned long long r = __umul64hi(x.x, q.W);  // floor(x W / 2^64) < W
  // the last splat whose exclusive prefix sum is <= r (a live one: a zero-weight splat shares
  // its prefix sum with the next splat, and the last prefix sum of a trailing run is W > r)
  int64_t lo = 0, hi = q.n_active;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (q.excl[mid] <= r) lo = mid + 1;
    else hi = mid;
  }
  const int64_t s = lo - 1;
  q.tgt[j] = (uint32_t)t;
  q.src[j] = (uint32_t)s;
  // the first draw of a source lists it once, so that the split rule runs densely over them
  if (atomicAdd(&q.counts[s], 1u) == 0u) q.ulist[atomicAdd(q.n_ulist, 1u)] = (uint32_t)s;
}

// the activation of raw row r, as the Adam step stores it
__device__ __forceinline__ float activate_row(int r, float x) {
  if (r == 3 || r == 4) return expf(x);  // log-scales
  if (r == 9) return sigmoid_f(x);       // logit-opacity
  return x;
}

// storage row of raw row r: (group, row within the group)
__device__ __forceinline__ void storage_slot(int r, int& grp, int& row) {
  if (r < 3) { grp = 0; row = r; }
  else if (r < 5) { grp = 1; row = r - 3; }
  else if (r < 9) { grp = 2; row = r - 5; }
  else if (r == 9) { grp = 3; row = 0; }
  else { grp = 4; row = r - 10; }
}

// the sources: o' = 1 - (1 - o)^(1/N) and s' = s o / sum_{j=1}^{N} (-1)^(j-1) C(N, j) o'^j / sqrt(j),
// in FP64; moments zeroed, storage rewritten
__global__ void __launch_bounds__(256) mcmc_sources_kernel(const __grid_constant__ McmcParams q) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= q.n_targets || k >= (int64_t)*q.n_ulist) return;
  const int64_t i = q.ulist[k];
  const uint32_t c = q.counts[i];
  const int N = (int)min((uint32_t)q.n_max, c + 1u);
  const double x = (double)q.p.row[9][i];
  const double o = 1.0 / (1.0 + exp(-x));
  double o_new = -expm1(log1p(-o) / (double)N);
  o_new = fmin(fmax(o_new, (double)q.min_opacity), 1.0 - 1.0 / 8388608.0);
  double den = 0.0, binom = 1.0, pw = 1.0;
  for (int j = 1; j <= N; ++j) {
    binom = binom * (double)(N - j + 1) / (double)j;  // C(N, j), exact for N <= 51
    pw *= o_new;
    den += ((j & 1) ? 1.0 : -1.0) * binom * pw / sqrt((double)j);
  }
  const double lf = log(o / den);
  q.p.row[9][i] = (float)log(o_new / (1.0 - o_new));
  q.p.row[3][i] = (float)((double)q.p.row[3][i] + lf);
  q.p.row[4][i] = (float)((double)q.p.row[4][i] + lf);
#pragma unroll
  for (int r = 0; r < 13; ++r) {
    q.m.row[r][i] = 0.0f;
    q.v.row[r][i] = 0.0f;
  }
  const int rs[3] = {3, 4, 9};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    int grp, row;
    storage_slot(rs[k], grp, row);
    store_act(q.st[grp], q.dtype, (int64_t)row * q.n_pad + i, activate_row(rs[k], q.p.row[rs[k]][i]));
  }
}

// the targets copy their (updated) source: raw rows and storage; moments zeroed
__global__ void __launch_bounds__(256) mcmc_copy_kernel(const __grid_constant__ McmcParams q) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= q.n_targets) return;
  const int64_t t = q.tgt[j], s = q.src[j];
#pragma unroll
  for (int r = 0; r < 13; ++r) {
    const float x = q.p.row[r][s];
    q.p.row[r][t] = x;
    q.m.row[r][t] = 0.0f;
    q.v.row[r][t] = 0.0f;
    int grp, row;
    storage_slot(r, grp, row);
    store_act(q.st[grp], q.dtype, (int64_t)row * q.n_pad + t, activate_row(r, x));
  }
}

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
bool aligned16(const void* p) { return p && (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

bool check_params(const ss_splat_params* p, int64_t n_pad) {
  if (!p || p->n_pad != n_pad) return false;
  const float* ps[5] = {p->means, p->log_scales, p->quats, p->logit_opacity, p->rgb};
  for (const float* x : ps)
    if (!aligned16(x)) return false;
  return true;
}

bool check_storage(const ss_splats* s) {
  if (!s || s->n < 0 || s->n_pad < s->n || (s->n_pad % 8) != 0) return false;
  if (s->dtype != SS_F32 && s->dtype != SS_BF16) return false;
  const void* ps[5] = {s->means, s->scales, s->quats, s->opacity, s->rgb};
  for (const void* x : ps)
    if (!aligned16(x)) return false;
  return true;
}

bool check_adam(const ss_adam_opts* o) {
  if (!o) return false;
  const float v[11] = {o->lr_means, o->lr_scales, o->lr_quats, o->lr_opacity, o->lr_rgb, o->beta1, o->beta2,
                       o->eps, o->noise_lr, o->noise_k, o->noise_t};
  for (float x : v)
    if (!std::isfinite(x)) return false;
  if (!(o->beta1 >= 0.0f && o->beta1 < 1.0f && o->beta2 >= 0.0f && o->beta2 < 1.0f)) return false;
  if (!(o->eps >= 0.0f) || o->step < 1) return false;
  return true;
}

void bias_corrections(const ss_adam_opts* o, float& inv_bc1, float& inv_bc2) {
  inv_bc1 = (float)(1.0 / (1.0 - std::pow((double)o->beta1, (double)o->step)));
  inv_bc2 = (float)(1.0 / (1.0 - std::pow((double)o->beta2, (double)o->step)));
}

Params13 rows13(const ss_splat_params* p) {
  Params13 r;
  const int64_t np = p->n_pad;
  for (int k = 0; k < 3; ++k) r.row[k] = p->means + k * np;
  for (int k = 0; k < 2; ++k) r.row[3 + k] = p->log_scales + k * np;
  for (int k = 0; k < 4; ++k) r.row[5 + k] = p->quats + k * np;
  r.row[9] = p->logit_opacity;
  for (int k = 0; k < 3; ++k) r.row[10 + k] = p->rgb + k * np;
  return r;
}

constexpr size_t kAlignMc = 256;
size_t up(size_t x) { return (x + kAlignMc - 1) / kAlignMc * kAlignMc; }

struct McmcLayout {
  size_t w, dead, dpos, excl, counts, tgt, src, ulist, nlist, scratch_a, scratch_b, totals, total;
  ScanPlan plan;
};

McmcLayout mcmc_layout(int64_t cap) {
  McmcLayout L;
  L.plan = plan_scan(cap);
  size_t o = 0;
  auto take = [&](size_t bytes) { const size_t at = o; o = up(o + bytes); return at; };
  L.w = take(4 * (size_t)cap);
  L.dead = take(4 * (size_t)cap);
  L.dpos = take(4 * (size_t)cap);
  L.excl = take(8 * (size_t)cap);
  L.counts = take(4 * (size_t)cap);
  L.tgt = take(4 * (size_t)cap);
  L.src = take(4 * (size_t)cap);
  L.ulist = take(4 * (size_t)cap);
  L.nlist = take(16);
  L.scratch_a = take(8 * L.plan.scratch_elems);
  L.scratch_b = take(8 * L.plan.scratch_elems);
  L.totals = take(16);
  L.total = o;
  return L;
}

template <class T>
T* at_(void* base, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(base) + off);
}

unsigned blocks_for(int64_t n, int per_thread = 1) {
  return (unsigned)((n + 256LL * per_thread - 1) / (256LL * per_thread));
}

}  // namespace

extern "C" {

void ss_default_adam_opts(ss_adam_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->lr_means = 0.075f;
  o->lr_scales = 0.001f;
  o->lr_quats = 0.001f;
  o->lr_opacity = 0.05f;
  o->lr_rgb = 0.0025f;
  o->beta1 = 0.9f;
  o->beta2 = 0.999f;
  o->eps = 1e-15f;
  o->noise_lr = 5e5f;
  o->noise_k = 100.0f;
  o->noise_t = 0.005f;
  o->step = 1;
  o->seed = 0;
}

ss_status ss_adam_step(const ss_splat_params* params, const ss_splat_params* exp_avg,
                       const ss_splat_params* exp_avg_sq, const ss_splat_grads* grads, const ss_splats* storage,
                       const ss_adam_opts* opts, ss_stream_t stream) {
  if (!check_storage(storage) || !check_adam(opts)) return SS_ERR_INVALID_ARG;
  const int64_t np = storage->n_pad;
  if (!check_params(params, np) || !check_params(exp_avg, np) || !check_params(exp_avg_sq, np))
    return SS_ERR_INVALID_ARG;
  if (!grads || grads->n_pad != np) return SS_ERR_INVALID_ARG;
  {
    const float* gs[5] = {grads->means, grads->scales, grads->quats, grads->opacity, grads->rgb};
    for (const float* x : gs)
      if (!aligned16(x)) return SS_ERR_INVALID_ARG;
  }
  if (storage->n == 0) return SS_OK;
  AdamParams a;
  std::memset(&a, 0, sizeof(a));
  const ss_splat_params* ps[3] = {params, exp_avg, exp_avg_sq};
  float** dst[3] = {a.p, a.m, a.v};
  for (int k = 0; k < 3; ++k) {
    dst[k][0] = ps[k]->means;
    dst[k][1] = ps[k]->log_scales;
    dst[k][2] = ps[k]->quats;
    dst[k][3] = ps[k]->logit_opacity;
    dst[k][4] = ps[k]->rgb;
  }
  a.g[0] = grads->means;
  a.g[1] = grads->scales;
  a.g[2] = grads->quats;
  a.g[3] = grads->opacity;
  a.g[4] = grads->rgb;
  // the storage arrays are the rasterizer's inputs, written here
  a.st[0] = const_cast<void*>(storage->means);
  a.st[1] = const_cast<void*>(storage->scales);
  a.st[2] = const_cast<void*>(storage->quats);
  a.st[3] = const_cast<void*>(storage->opacity);
  a.st[4] = const_cast<void*>(storage->rgb);
  a.dtype = storage->dtype;
  a.n = storage->n;
  a.n_pad = np;
  a.lr[0] = opts->lr_means;
  a.lr[1] = opts->lr_scales;
  a.lr[2] = opts->lr_quats;
  a.lr[3] = opts->lr_opacity;
  a.lr[4] = opts->lr_rgb;
  a.beta1 = opts->beta1;
  a.beta2 = opts->beta2;
  a.eps = opts->eps;
  bias_corrections(opts, a.inv_bc1, a.inv_bc2);
  a.noise_coef = opts->lr_means * opts->noise_lr;
  a.noise_k = opts->noise_k;
  a.noise_t = opts->noise_t;
  a.step = (unsigned long long)opts->step;
  a.seed = opts->seed;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  count_launch();
  adam_kernel<<<blocks_for(a.n, 4), 256, 0, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? SS_OK : SS_ERR_CUDA;
}

ss_status ss_adam_flat(float* param, float* exp_avg, float* exp_avg_sq, const float* grad, int64_t n, float lr,
                       const ss_adam_opts* opts, ss_stream_t stream) {
  if (!check_adam(opts) || n < 0 || !std::isfinite(lr)) return SS_ERR_INVALID_ARG;
  if (n == 0) return SS_OK;
  if (!param || !exp_avg || !exp_avg_sq || !grad) return SS_ERR_INVALID_ARG;
  FlatAdam a{param, exp_avg, exp_avg_sq, grad, n, lr, opts->beta1, opts->beta2, opts->eps, 0.0f, 0.0f};
  bias_corrections(opts, a.inv_bc1, a.inv_bc2);
  count_launch();
  adam_flat_kernel<<<blocks_for(n), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(a);
  return cudaGetLastError() == cudaSuccess ? SS_OK : SS_ERR_CUDA;
}

void ss_default_mcmc_opts(ss_mcmc_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->min_opacity = 0.005f;
  o->growth = 0.05f;
  o->n_max = 51;
  o->step = 0;
  o->seed = 0;
}

ss_status ss_mcmc_workspace_size(int64_t cap, size_t* bytes) {
  if (!bytes || cap < 1 || cap >= (1LL << 31)) return SS_ERR_INVALID_ARG;
  *bytes = mcmc_layout(cap).total;
  return SS_OK;
}

ss_status ss_mcmc_relocate(const ss_splat_params* params, const ss_splat_params* exp_avg,
                           const ss_splat_params* exp_avg_sq, const ss_splats* storage, int64_t cap,
                           const ss_mcmc_opts* opts, void* ws, size_t ws_bytes, int64_t* n_after, int64_t* d_stats,
                           ss_stream_t stream) {
  if (!opts || !n_after || !check_storage(storage)) return SS_ERR_INVALID_ARG;
  if (cap < 1 || cap >= (1LL << 31) || storage->n > cap || storage->n_pad < cap) return SS_ERR_INVALID_ARG;
  if (!(opts->min_opacity >= 0.0f && opts->min_opacity < 1.0f) || !std::isfinite(opts->growth) ||
      !(opts->growth >= 0.0f) || opts->n_max < 1 || opts->n_max > 51)
    return SS_ERR_INVALID_ARG;
  const int64_t np = storage->n_pad;
  if (!check_params(params, np) || !check_params(exp_avg, np) || !check_params(exp_avg_sq, np))
    return SS_ERR_INVALID_ARG;
  const McmcLayout L = mcmc_layout(cap);
  if (!ws || ws_bytes < L.total || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0) return SS_ERR_INVALID_ARG;
  const int64_t n = storage->n;
  *n_after = n;
  if (n == 0) return SS_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  McmcParams q;
  std::memset(&q, 0, sizeof(q));
  q.p = rows13(params);
  q.m = rows13(exp_avg);
  q.v = rows13(exp_avg_sq);
  q.st[0] = const_cast<void*>(storage->means);
  q.st[1] = const_cast<void*>(storage->scales);
  q.st[2] = const_cast<void*>(storage->quats);
  q.st[3] = const_cast<void*>(storage->opacity);
  q.st[4] = const_cast<void*>(storage->rgb);
  q.dtype = storage->dtype;
  q.n_pad = np;
  q.n_active = n;
  q.stored_opacity = storage->opacity;
  q.min_opacity = opts->min_opacity;
  q.n_max = opts->n_max;
  q.step = (unsigned long long)(uint32_t)opts->step;
  q.seed = opts->seed;
  q.w = at_<uint32_t>(ws, L.w);
  q.dead = at_<uint32_t>(ws, L.dead);
  q.dpos = at_<uint32_t>(ws, L.dpos);
  q.excl = at_<unsigned long long>(ws, L.excl);
  q.counts = at_<uint32_t>(ws, L.counts);
  q.tgt = at_<uint32_t>(ws, L.tgt);
  q.src = at_<uint32_t>(ws, L.src);
  q.ulist = at_<uint32_t>(ws, L.ulist);
  q.n_ulist = at_<uint32_t>(ws, L.nlist);
  q.d_stats = d_stats;
  unsigned long long* totals = at_<unsigned long long>(ws, L.totals);
  q.totals = totals;
  const ScanPlan plan = plan_scan(n);
  count_launch();
  mcmc_weights_kernel<<<blocks_for(n), 256, 0, st>>>(q);
  if (cudaGetLastError() != cudaSuccess) return SS_ERR_CUDA;
  if (exclusive_scan_u32(q.dead, q.dpos, n, at_<unsigned long long>(ws, L.scratch_a), plan, totals, st) !=
      cudaSuccess)
    return SS_ERR_CUDA;
  if (exclusive_scan_u32_u64(q.w, q.excl, n, at_<unsigned long long>(ws, L.scratch_b), plan, totals + 1, st) !=
      cudaSuccess)
    return SS_ERR_CUDA;
  count_launch();
  mcmc_compact_kernel<<<blocks_for(n), 256, 0, st>>>(q);
  if (cudaGetLastError() != cudaSuccess) return SS_ERR_CUDA;
  // the dead count and the total weight size the draws
  unsigned long long h_tot[2] = {0ull, 0ull};
  if (cudaMemcpyAsync(h_tot, totals, sizeof(h_tot), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return SS_ERR_CUDA;
  if (h_tot[1] == 0ull) return SS_OK;  // no live splat: nothing to draw from
  const int64_t grown = n + std::min<int64_t>(cap - n, (int64_t)std::floor((double)n * (double)opts->growth));
  q.n_dead = (int64_t)h_tot[0];
  q.W = h_tot[1];
  q.n_targets = q.n_dead + (grown - n);
  *n_after = grown;
  if (q.n_targets == 0) return SS_OK;
  if (cudaMemsetAsync(q.n_ulist, 0, sizeof(uint32_t), st) != cudaSuccess) return SS_ERR_CUDA;
  count_launch();
  mcmc_draw_kernel<<<blocks_for(q.n_targets), 256, 0, st>>>(q);
  count_launch();
  mcmc_sources_kernel<<<blocks_for(q.n_targets), 256, 0, st>>>(q);
  count_launch();
  mcmc_copy_kernel<<<blocks_for(q.n_targets), 256, 0, st>>>(q);
  return cudaGetLastError() == cudaSuccess ? SS_OK : SS_ERR_CUDA;
}

}  // extern "C"
