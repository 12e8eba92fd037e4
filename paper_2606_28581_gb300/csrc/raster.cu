// Forward (K3) and backward (K4) rasterization, Sec. 3.2 Eq. rasterization.
//
// One block renders one screen tile of one target: it stages the tile's sorted splat batch in
// shared memory, and each thread walks its pixel front to back (forward) or back to front
// (backward).  With `persistent`, one launch sized to the GPU pulls (target, tile) items from
// a queue, so views of uneven size and sun views share a single launch.
//
// Backward: with T_i the transmittance in front of splat i and S_i the composite behind it
// (normalised to T_{i+1}), d f / d alpha_i = T_i (f_i - S_i); the alpha output adds
// T_final / (1 - alpha_i).  T_i is recovered as T_{i+1} / (1 - alpha_i) from the saved
// T_final (alpha <= alpha_max < 1 keeps the division safe); only T_final and the end of the
// walk are stored per pixel.
#include "kernels.cuh"

namespace ss {

__device__ __forceinline__ int find_target(const TargetCam* tc, int n_targets, int tile) {
  int lo = 0, hi = n_targets - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tc[mid].tile_base <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Transposed warp reduction of 16 values: lanes 2f and 2f + 1 end with the warp sum of field f.
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

// ------------------------------------------------------------------------------------------
// K3 forward
// ------------------------------------------------------------------------------------------
template <int TW, int TH, int BATCH, bool PERSIST>
__global__ void __launch_bounds__(TW * TH) raster_fwd_kernel(const __grid_constant__ RasterParams p) {
  constexpr int NT = TW * TH;
  __shared__ float4 sg[BATCH][3];
  __shared__ float4 sf[BATCH][2];
  __shared__ int s_item;
  const int tid = threadIdx.x;
  int tile;
  bool first = true;
  while (true) {
    if (!PERSIST && !first) break;
    first = false;
    if (!next_item<PERSIST>(p, &p.status->work_fwd, tile, s_item)) break;
    const int t = find_target(p.tcams, p.n_targets, tile);
    const TargetCam& cam = p.tcams[t];
    const int local = tile - cam.tile_base;
    const int ty = local / cam.tiles_x, tx = local - ty * cam.tiles_x;
    const int px = tx * TW + (tid % TW), py = ty * TH + (tid / TW);
    const bool inside = px < cam.W && py < cam.H;
    const bool sun = cam.sun != 0;
    const float x = (float)px + 0.5f, y = (float)py + 0.5f;
    const uint2 range = p.ranges[tile];
    const int64_t recbase = (int64_t)t * p.n_pad;

    float T = 1.0f, D = 0.0f, A0 = 0.0f, A1 = 0.0f, A2 = 0.0f, N0 = 0.0f, N1 = 0.0f, N2 = 0.0f;
    uint32_t last = range.x;
    uint32_t walked = 0;  // contributing pairs, the stopping one included
    bool done = !inside;
    for (uint32_t b0 = range.x; b0 < range.y; b0 += BATCH) {
      const int nb = min((int)(range.y - b0), BATCH);
      __syncthreads();
      for (int i = tid; i < nb; i += NT) {
        const int64_t rec = recbase + p.vals[b0 + i];
        const float4* g = p.geom + rec * 3;
        const float4* f = p.feat + rec * 2;
        sg[i][0] = g[0];
        sg[i][1] = g[1];
        sg[i][2] = g[2];
        sf[i][0] = f[0];
        if (!sun) sf[i][1] = f[1];
      }
      if (__syncthreads_and(done)) break;
      if (!done) {
        for (int j = 0; j < nb; ++j) {
          const float4 g2 = sg[j][2];
          const PairEval e = eval_pair(sg[j][0], sg[j][1], g2, x, y, p.k);
          if (!e.contrib) continue;
          ++walked;
          const float Tn = T * (1.0f - e.alpha);
          if (Tn < p.t_min) {
            done = true;
            break;
          }
          const float w = e.alpha * T;
          const float4 f0 = sf[j][0];
          D += w * (g2.w + f0.x * e.u + f0.y * e.v);
          if (!sun) {
            const float4 f1 = sf[j][1];
            A0 += w * f1.y;
            A1 += w * f1.z;
            A2 += w * f1.w;
            N0 += w * f0.z;
            N1 += w * f0.w;
            N2 += w * f1.x;
          }
          T = Tn;
          last = b0 + j + 1;
        }
      }
    }
    if (inside) {
      const TargetIO io = p.io[t];
      const int64_t pix = (int64_t)py * cam.W + px;
      const int64_t hw = (int64_t)cam.W * cam.H;
      if (io.rgb) {
        float C[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0};
        if (p.color) {
#pragma unroll
          for (int i = 0; i < 12; ++i) C[i] = p.color[cam.cam * 12 + i];
        }
        io.rgb[pix] = C[0] * A0 + C[1] * A1 + C[2] * A2 + C[3];
        io.rgb[hw + pix] = C[4] * A0 + C[5] * A1 + C[6] * A2 + C[7];
        io.rgb[2 * hw + pix] = C[8] * A0 + C[9] * A1 + C[10] * A2 + C[11];
      }
      if (io.depth) io.depth[pix] = D;
      if (io.normal) {
        io.normal[pix] = N0;
        io.normal[hw + pix] = N1;
        io.normal[2 * hw + pix] = N2;
      }
      if (io.alpha) io.alpha[pix] = 1.0f - T;
      io.T_final[pix] = T;
      io.last[pix] = last;
    }
    // algorithmic work counter: one atomic per warp
    const unsigned int wsum = __reduce_add_sync(0xffffffffu, walked);
    if ((tid & 31) == 0 && wsum) atomicAdd(&p.status->n_walked, (unsigned long long)wsum);
  }
}

// ------------------------------------------------------------------------------------------
// K4 backward
// ------------------------------------------------------------------------------------------
template <int TW, int TH, int BATCH, bool PERSIST>
__global__ void __launch_bounds__(TW * TH) raster_bwd_kernel(const __grid_constant__ RasterParams p) {
  constexpr int NT = TW * TH;
  constexpr int NW = NT / 32;
  __shared__ float4 sg[BATCH][3];
  __shared__ float4 sf[BATCH][2];
  __shared__ uint32_t sk[BATCH];
  __shared__ float sacc[BATCH][kGradFields];
  __shared__ float scol[NW][16];
  __shared__ int s_item;
  __shared__ unsigned int s_hi;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int tile;
  bool first = true;
  while (true) {
    if (!PERSIST && !first) break;
    first = false;
    if (!next_item<PERSIST>(p, &p.status->work_bwd, tile, s_item)) break;
    const int t = find_target(p.tcams, p.n_targets, tile);
    const TargetCam& cam = p.tcams[t];
    const int local = tile - cam.tile_base;
    const int ty = local / cam.tiles_x, tx = local - ty * cam.tiles_x;
    const int px = tx * TW + (tid % TW), py = ty * TH + (tid / TW);
    const bool inside = px < cam.W && py < cam.H;
    const bool sun = cam.sun != 0;
    const float x = (float)px + 0.5f, y = (float)py + 0.5f;
    const uint2 range = p.ranges[tile];
    const int64_t recbase = (int64_t)t * p.n_pad;
    const TargetIO io = p.io[t];
    const int64_t pix = (int64_t)py * cam.W + px;
    const int64_t hw = (int64_t)cam.W * cam.H;

    float T = 1.0f, Tfin = 1.0f;
    uint32_t lastp = range.x;
    float gR[3] = {0, 0, 0}, gA[3] = {0, 0, 0}, gN[3] = {0, 0, 0}, gD = 0.0f, gAl = 0.0f;
    if (inside) {
      T = io.T_final[pix];
      Tfin = T;
      // the saved end of the walk, clamped to this tile's list
      lastp = min(max(io.last[pix], range.x), range.y);
      if (!sun && io.d_rgb) {
        gR[0] = io.d_rgb[pix];
        gR[1] = io.d_rgb[hw + pix];
        gR[2] = io.d_rgb[2 * hw + pix];
        // rgb_out = C A + c  ->  dA = C^T d(rgb_out)
        if (p.color) {
          const float* C = p.color + cam.cam * 12;
#pragma unroll
          for (int j = 0; j < 3; ++j) gA[j] = C[j] * gR[0] + C[4 + j] * gR[1] + C[8 + j] * gR[2];
        } else {
          gA[0] = gR[0]; gA[1] = gR[1]; gA[2] = gR[2];
        }
      }
      if (!sun && io.d_normal) {
        gN[0] = io.d_normal[pix];
        gN[1] = io.d_normal[hw + pix];
        gN[2] = io.d_normal[2 * hw + pix];
      }
      if (io.d_depth) gD = io.d_depth[pix];
      if (io.d_alpha) gAl = io.d_alpha[pix];
    }
    if (tid == 0) s_hi = range.x;
    __syncthreads();
    if (inside && lastp > range.x) atomicMax(&s_hi, lastp);
    __syncthreads();
    const uint32_t hi_all = s_hi;
    float Sg = 0.0f;  // g . S_i
    float Aacc[3] = {0, 0, 0};
    const float two_inv2s2 = 2.0f * p.k.inv2s2;
    for (uint32_t hi = hi_all; hi > range.x;) {
      const uint32_t b0 = (hi - range.x > (uint32_t)BATCH) ? hi - BATCH : range.x;
      const int nb = (int)(hi - b0);
      __syncthreads();
      for (int i = tid; i < nb; i += NT) {
        const uint32_t kk = p.vals[b0 + i];
        const int64_t rec = recbase + kk;
        const float4* g = p.geom + rec * 3;
        const float4* f = p.feat + rec * 2;
        sk[i] = kk;
        sg[i][0] = g[0];
        sg[i][1] = g[1];
        sg[i][2] = g[2];
        sf[i][0] = f[0];
        if (!sun) sf[i][1] = f[1];
      }
      for (int i = tid; i < nb * kGradFields; i += NT) (&sacc[0][0])[i] = 0.0f;
      __syncthreads();
      for (int jj = nb - 1; jj >= 0; --jj) {
        const uint32_t j = b0 + jj;
        float g[16];
#pragma unroll
        for (int f = 0; f < 16; ++f) g[f] = 0.0f;
        bool c = false;
        if (j < lastp) {
          const float4 g0 = sg[jj][0], g1 = sg[jj][1], g2 = sg[jj][2];
          const PairEval e = eval_pair(g0, g1, g2, x, y, p.k);
          if (e.contrib) {
            c = true;
            const float4 f0 = sf[jj][0];
            const bool deg = g2.y < 0.0f;
            const float om = 1.0f - e.alpha;
            const float Ti = T / om;
            const float w = e.alpha * Ti;
            const float z = g2.w + f0.x * e.u + f0.y * e.v;
            float gf = gD * z;
            float4 f1 = make_float4(0, 0, 0, 0);
            if (!sun) {
              f1 = sf[jj][1];
              gf += gA[0] * f1.y + gA[1] * f1.z + gA[2] * f1.w + gN[0] * f0.z + gN[1] * f0.w + gN[2] * f1.x;
            }
            const float dal = Ti * (gf - Sg) + gAl * Tfin / om;
            Sg = e.alpha * gf + om * Sg;
            T = Ti;
            if (!sun) {
              Aacc[0] += w * f1.y;
              Aacc[1] += w * f1.z;
              Aacc[2] += w * f1.w;
              g[GF_R] = w * gA[0];
              g[GF_G] = w * gA[1];
              g[GF_B] = w * gA[2];
              g[GF_NX] = w * gN[0];
              g[GF_NY] = w * gN[1];
              g[GF_NZ] = w * gN[2];
            }
            const float dz = w * gD;
            g[GF_ZC] = dz;
            g[GF_DZDU] = dz * e.u;
            g[GF_DZDV] = dz * e.v;
            float du = deg ? 0.0f : dz * f0.x;
            float dv = deg ? 0.0f : dz * f0.y;
            if (!e.clamped) {
              const float dpw = dal * e.alpha;  // d/d ln(o G^)
              g[GF_LNO] = dpw;
              if (e.uwin) {
                du -= dpw * e.u;
                dv -= dpw * e.v;
              } else {
                g[GF_CX] = dpw * e.dx * two_inv2s2;
                g[GF_CY] = dpw * e.dy * two_inv2s2;
              }
            }
            if (!deg) {
              g[GF_Q00] = du * e.dx;
              g[GF_Q01] = du * e.dy;
              g[GF_Q10] = dv * e.dx;
              g[GF_Q11] = dv * e.dy;
              g[GF_CX] -= g1.x * du + g1.z * dv;
              g[GF_CY] -= g1.y * du + g1.w * dv;
            }
          }
        }
        if (__any_sync(0xffffffffu, c)) {
          const float r = warp_reduce16_transposed(g);
          if (!(lane & 1) && r != 0.0f) atomicAdd(&sacc[jj][lane >> 1], r);
        }
      }
      __syncthreads();
      for (int i = tid; i < nb * kGradFields; i += NT) {
        const float v = (&sacc[0][0])[i];
        if (v != 0.0f) atomicAdd(p.grad + (recbase + sk[i >> 4]) * kGradFields + (i & 15), v);
      }
      hi = b0;
    }
    // colour correction gradient of this target: dC = sum g A^T, dc = sum g
    if (!sun && p.d_color && io.d_rgb) {
      float cv[16];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        cv[4 * a + 0] = gR[a] * Aacc[0];
        cv[4 * a + 1] = gR[a] * Aacc[1];
        cv[4 * a + 2] = gR[a] * Aacc[2];
        cv[4 * a + 3] = gR[a];
      }
      cv[12] = cv[13] = cv[14] = cv[15] = 0.0f;
      const float r = warp_reduce16_transposed(cv);
      if (!(lane & 1)) scol[warp][lane >> 1] = r;
      __syncthreads();
      if (tid < 12) {
        float s = 0.0f;
#pragma unroll
        for (int w2 = 0; w2 < NW; ++w2) s += scol[w2][tid];
        if (s != 0.0f) atomicAdd(p.d_color + cam.cam * 12 + tid, s);
      }
    }
  }
}

// ------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------
template <int TW, int TH, int BATCH>
static cudaError_t launch_fwd_t(const RasterParams& p, bool persistent, int num_sms, cudaStream_t st) {
  if (p.total_tiles == 0) return cudaSuccess;
  if (persistent) {
    // resident blocks per SM, queried once (outside any later stream capture)
    static int per_sm = 0;
    if (per_sm == 0) {
      int v = 0;
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, raster_fwd_kernel<TW, TH, BATCH, true>,
                                                                    TW * TH, 0);
      if (e != cudaSuccess) return e;
      per_sm = v < 1 ? 1 : v;
    }
    int grid = num_sms * per_sm;
    if (grid > p.total_tiles) grid = p.total_tiles; {
    count_launch();
    raster_fwd_kernel<TW, TH, BATCH, true><<<grid, TW * TH, 0, st>>>(p);
  }
  } else {
    count_launch();
    raster_fwd_kernel<TW, TH, BATCH, false><<<p.total_tiles, TW * TH, 0, st>>>(p);
  }
  return cudaGetLastError();
}

template <int TW, int TH, int BATCH>
static cudaError_t launch_bwd_t(const RasterParams& p, bool persistent, int num_sms, cudaStream_t st) {
  if (p.total_tiles == 0) return cudaSuccess;
  if (persistent) {
    // resident blocks per SM, queried once (outside any later stream capture)
    static int per_sm = 0;
    if (per_sm == 0) {
      int v = 0;
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, raster_bwd_kernel<TW, TH, BATCH, true>,
                                                                    TW * TH, 0);
      if (e != cudaSuccess) return e;
      per_sm = v < 1 ? 1 : v;
    }
    int grid = num_sms * per_sm;
    if (grid > p.total_tiles) grid = p.total_tiles; {
    count_launch();
    raster_bwd_kernel<TW, TH, BATCH, true><<<grid, TW * TH, 0, st>>>(p);
  }
  } else {
    count_launch();
    raster_bwd_kernel<TW, TH, BATCH, false><<<p.total_tiles, TW * TH, 0, st>>>(p);
  }
  return cudaGetLastError();
}

#define SS_DISPATCH_SHAPE(FN, ...)                                                   \
  do {                                                                               \
    if (tile_w == 16 && tile_h == 16) {                                              \
      if (batch == 64) return FN<16, 16, 64>(__VA_ARGS__);                           \
      if (batch == 128) return FN<16, 16, 128>(__VA_ARGS__);                         \
      return FN<16, 16, 256>(__VA_ARGS__);                                           \
    }                                                                                \
    if (tile_w == 32 && tile_h == 8) {                                               \
      if (batch == 64) return FN<32, 8, 64>(__VA_ARGS__);                            \
      if (batch == 128) return FN<32, 8, 128>(__VA_ARGS__);                          \
      return FN<32, 8, 256>(__VA_ARGS__);                                            \
    }                                                                                \
    if (tile_w == 8 && tile_h == 32) {                                               \
      if (batch == 64) return FN<8, 32, 64>(__VA_ARGS__);                            \
      if (batch == 128) return FN<8, 32, 128>(__VA_ARGS__);                          \
      return FN<8, 32, 256>(__VA_ARGS__);                                            \
    }                                                                                \
    return cudaErrorInvalidValue;                                                    \
  } while (0)

cudaError_t launch_raster_fwd(const RasterParams& p, int tile_w, int tile_h, int batch, bool persistent,
                              int num_sms, cudaStream_t st) {
  SS_DISPATCH_SHAPE(launch_fwd_t, p, persistent, num_sms, st);
}

cudaError_t launch_raster_bwd(const RasterParams& p, int tile_w, int tile_h, int batch, bool persistent,
                              int num_sms, cudaStream_t st) {
  SS_DISPATCH_SHAPE(launch_bwd_t, p, persistent, num_sms, st);
}

}  // namespace ss
