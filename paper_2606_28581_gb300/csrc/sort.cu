// Tile binning and sorting (K2), Sec. 3.2 rasterization paragraph.
//
// The visibility key is the height-based depth of a splat's centre (Eq. depth_affine_camera),
// which is the same for every view, so one stable sort of the splats by height (descending,
// ties by index) serves all targets.  Every (target, splat, tile) overlap is then emitted in
// that order, target after target, and each target's overlaps are stably sorted by tile id:
// within a tile the list stays front to back, and since the targets' tile ids are consecutive
// ranges the whole array ends sorted by global tile id.  Both sorts are a hand-written stable
// LSD radix sort (per-block digit histograms, a device-wide exclusive scan, and a stable scatter
// that ranks equal digits with warp match masks in element order).  The height sort takes 8-bit
// digits.  The tile sort works on each target's segment with the digits of the tile id relative
// to the target's first tile (14 bits for a 2048^2 view of 16 x 16 tiles): two 7-bit passes where
// the global ids of 16 views (18 bits) took two 9-bit ones, and 4M splats over 32 views
// (20 bits) three 8-bit ones.  Its blocks never straddle two segments, and its histograms are
// laid out segment after segment, so one scan gives each block its positions in its segment.
#include "kernels.cuh"

namespace ss {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// ------------------------------------------------------------------------------------------
// exclusive scan (uint32 in, uint32 out saturated, uint64 block sums)
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long block_exclusive_scan(unsigned long long v,
                                                                   unsigned long long* total) {
  __shared__ unsigned long long warp_tot[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    unsigned long long w = lane < kScanThreads / 32 ? warp_tot[lane] : 0ull;
    unsigned long long wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = wi - w;
    if (lane == kScanThreads / 32 - 1) *total = wi;
  }
  __syncthreads();
  unsigned long long r = warp_tot[warp] + inc - v;
  __syncthreads();
  return r;
}

// A thread's kScanItems consecutive elements: two 16-byte loads for a 32-bit input that starts
// 16-byte aligned when all of them are in range, else element by element.
template <typename Tin>
__device__ __forceinline__ void scan_load(const Tin* in, int64_t base, int64_t n, unsigned long long (&v)[kScanItems]) {
  if (sizeof(Tin) == 4 && base + kScanItems <= n && (reinterpret_cast<uintptr_t>(in) & 15u) == 0) {
    static_assert(kScanItems == 8, "two 16-byte loads per thread");
    const uint4 a = reinterpret_cast<const uint4*>(in + base)[0], b = reinterpret_cast<const uint4*>(in + base)[1];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  } else {
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) v[i] = (base + i < n) ? (unsigned long long)in[base + i] : 0ull;
  }
}

template <typename Tin>
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const Tin* in, int64_t n,
                                                                    unsigned long long* sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  unsigned long long v[kScanItems];
  scan_load(in, base, n, v);
  unsigned long long s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) s += v[i];
  __shared__ unsigned long long tot;
  (void)block_exclusive_scan(s, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kScanThreads) scan_down_kernel(const Tin* in, Tout* out, int64_t n,
                                                                  const unsigned long long* offs,
                                                                  unsigned long long* total) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  unsigned long long v[kScanItems];
  scan_load(in, base, n, v);
  unsigned long long s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) s += v[i];
  __shared__ unsigned long long tot;
  unsigned long long run = block_exclusive_scan(s, &tot);
  if (offs) run += offs[blockIdx.x];
  else if (threadIdx.x == 0 && total) *total = tot;
  if (sizeof(Tout) == 4 && base + kScanItems <= n && (reinterpret_cast<uintptr_t>(out) & 15u) == 0) {
    // two 16-byte stores of the saturated 32-bit prefixes
    uint32_t o[kScanItems];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
      o[i] = (uint32_t)(run > 0xffffffffull ? 0xffffffffull : run);
      run += v[i];
    }
    uint4* dst = reinterpret_cast<uint4*>(out + base);
    dst[0] = make_uint4(o[0], o[1], o[2], o[3]);
    dst[1] = make_uint4(o[4], o[5], o[6], o[7]);
    return;
  }
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) {
      if (sizeof(Tout) == 4)
        out[base + i] = (Tout)(run > 0xffffffffull ? 0xffffffffull : run);
      else
        out[base + i] = (Tout)run;
    }
    run += v[i];
  }
}

ScanPlan plan_scan(int64_t n) {
  ScanPlan p{};
  p.n = n;
  int64_t s = n;
  size_t off = 0;
  p.levels = 0;
  // level l >= 1 holds the block sums of level l - 1
  while (s > kScanTile) {
    s = (s + kScanTile - 1) / kScanTile;
    p.level_n[p.levels] = s;
    p.level_off[p.levels] = off;
    off += (size_t)s;
    ++p.levels;
  }
  p.scratch_elems = off + 1;  // + the total
  return p;
}

namespace {
// uint32 in; Tout = uint32 (saturated) or uint64 out
template <typename Tout>
cudaError_t exclusive_scan_t(const uint32_t* in, Tout* out, int64_t n, unsigned long long* scratch,
                             const ScanPlan& plan, unsigned long long* total, cudaStream_t st) {
  if (n == 0) return cudaMemsetAsync(total, 0, sizeof(unsigned long long), st);
  const int L = plan.levels;
  if (L == 0) {
    count_launch();
    scan_down_kernel<uint32_t, Tout><<<1, kScanThreads, 0, st>>>(in, out, n, nullptr, total);
    return cudaGetLastError();
  }
  // up: block sums
  count_launch();
  scan_reduce_kernel<uint32_t><<<(unsigned)plan.level_n[0], kScanThreads, 0, st>>>(
      in, n, scratch + plan.level_off[0]);
  for (int l = 1; l < L; ++l) {
    count_launch();
    scan_reduce_kernel<unsigned long long><<<(unsigned)plan.level_n[l], kScanThreads, 0, st>>>(
        scratch + plan.level_off[l - 1], plan.level_n[l - 1], scratch + plan.level_off[l]);
  }
  // top level fits one block
  count_launch();
  scan_down_kernel<unsigned long long, unsigned long long><<<1, kScanThreads, 0, st>>>(
      scratch + plan.level_off[L - 1], scratch + plan.level_off[L - 1], plan.level_n[L - 1], nullptr,
      total);
  for (int l = L - 2; l >= 0; --l) {
    count_launch();
    scan_down_kernel<unsigned long long, unsigned long long><<<(unsigned)plan.level_n[l + 1], kScanThreads, 0, st>>>(
        scratch + plan.level_off[l], scratch + plan.level_off[l], plan.level_n[l],
        scratch + plan.level_off[l + 1], nullptr);
  }
  count_launch();
  scan_down_kernel<uint32_t, Tout><<<(unsigned)plan.level_n[0], kScanThreads, 0, st>>>(
      in, out, n, scratch + plan.level_off[0], nullptr);
  return cudaGetLastError();
}
}  // namespace

cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, unsigned long long* scratch,
                               const ScanPlan& plan, unsigned long long* total, cudaStream_t st) {
  return exclusive_scan_t<uint32_t>(in, out, n, scratch, plan, total, st);
}

cudaError_t exclusive_scan_u32_u64(const uint32_t* in, unsigned long long* out, int64_t n,
                                   unsigned long long* scratch, const ScanPlan& plan, unsigned long long* total,
                                   cudaStream_t st) {
  return exclusive_scan_t<unsigned long long>(in, out, n, scratch, plan, total, st);
}

// ------------------------------------------------------------------------------------------
// stable LSD radix sort of (key, value) pairs
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ int64_t radix_count(int64_t n_host, const uint32_t* n_dev) {
  return n_dev ? (int64_t)(*n_dev) : n_host;
}

// The elements a block of the sort takes.  Whole-array sort (SEG false): block b takes
// [b TILE, b TILE + TILE) of the n elements, and its count of digit d goes to d nblocks + b.
// Segmented sort (SEG true): the block belongs to the segment s whose blocks include b, takes
// the segment's elements from its start, and its count of digit d goes to
// blk0 2^RB + d nblk + (b - blk0), so that one exclusive scan of the histograms, segment after
// segment, gives every block its output positions inside its own segment; digits are taken from
// key - key_base.
struct BlockSpan {
  int64_t base;      // first element
  int count;         // elements (0: none)
  int64_t hbase;     // histogram entry of digit 0
  int64_t hstride;   // step between digits
  uint32_t key_base;
};

template <bool SEG, int RB, int TILE>
__device__ __forceinline__ bool block_span(int64_t b, int64_t n, int64_t nblocks, const SortSeg* segs, int nseg,
                                           BlockSpan& sp) {
  if (!SEG) {
    sp.base = b * TILE;
    sp.count = sp.base < n ? (int)min((int64_t)TILE, n - sp.base) : 0;
    sp.hbase = b;
    sp.hstride = nblocks;
    sp.key_base = 0u;
    return true;
  }
  if (b >= (int64_t)segs[nseg].blk0) return false;
  int lo = 0, hi = nseg - 1;  // the last segment whose first block is at or before b
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((int64_t)segs[mid].blk0 <= b) lo = mid; else hi = mid - 1;
  }
  const SortSeg g = segs[lo];
  const int64_t bis = b - (int64_t)g.blk0;
  sp.base = (int64_t)g.start + bis * TILE;
  sp.count = (int)min((int64_t)TILE, (int64_t)g.len - bis * TILE);
  sp.hbase = ((int64_t)g.blk0 << RB) + bis;
  sp.hstride = g.nblk;
  sp.key_base = g.key_base;
  return true;
}

// Digit histograms of one block's elements, RB-bit digits.
template <int RB, int ITEMS, bool SEG>
__global__ void __launch_bounds__(kRadixThreads) radix_upsweep_kernel(const uint32_t* keys, int64_t n_host,
                                                                       const uint32_t* n_dev, int shift,
                                                                       uint32_t mask, uint32_t* hist,
                                                                       int64_t nblocks, const SortSeg* segs,
                                                                       int nseg) {
  constexpr int NB = 1 << RB, TILE = kRadixThreads * ITEMS;
  __shared__ uint32_t h[NB];
  const int64_t n = SEG ? 0 : radix_count(n_host, n_dev);
  BlockSpan sp;
  if (!block_span<SEG, RB, TILE>(blockIdx.x, n, nblocks, segs, nseg, sp)) return;
  for (int d = threadIdx.x; d < NB; d += kRadixThreads) h[d] = 0;
  __syncthreads();
#pragma unroll 4
  for (int i = 0; i < ITEMS; ++i) {
    const int j = i * kRadixThreads + threadIdx.x;
    if (j < sp.count) atomicAdd(&h[((keys[sp.base + j] - sp.key_base) >> shift) & mask], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < NB; d += kRadixThreads) hist[sp.hbase + (int64_t)d * sp.hstride] = h[d];
}

// Stable scatter of one block's tile: ranks within the block (warps own consecutive
// sub-chunks, equal digits ranked in element order with warp match masks), the tile reordered
// by digit in shared memory, then written out in runs that are contiguous in the output.
template <int RB, int ITEMS, bool SEG>
__global__ void __launch_bounds__(kRadixThreads) radix_downsweep_kernel(
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in, uint32_t* __restrict__ keys_out,
    uint32_t* __restrict__ vals_out, int64_t n_host, const uint32_t* n_dev, int shift, uint32_t mask,
    const uint32_t* hist_off, int64_t nblocks, const SortSeg* segs, int nseg) {
  constexpr int kWarps = kRadixThreads / 32;
  constexpr int NB = 1 << RB, TILE = kRadixThreads * ITEMS;
  // digits per thread; with fewer digits than threads, thread d < NB owns digit d
  constexpr int DPT = NB >= kRadixThreads ? NB / kRadixThreads : 1;
  static_assert(NB < kRadixThreads || NB % kRadixThreads == 0, "whole digits per thread");
  __shared__ uint32_t whist[kWarps][NB];
  __shared__ uint32_t dbase[NB];   // output position of the block's first element of each digit
  __shared__ uint32_t dstart[NB];  // block-local position of the first element of each digit
  __shared__ uint32_t sk[TILE], sv[TILE];
  const int64_t n = SEG ? 0 : radix_count(n_host, n_dev);
  BlockSpan sp;
  if (!block_span<SEG, RB, TILE>(blockIdx.x, n, nblocks, segs, nseg, sp) || sp.count <= 0) return;
  const int64_t base = sp.base;
  const int count = sp.count;
  const uint32_t kb = sp.key_base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kWarps * NB; i += kRadixThreads) (&whist[0][0])[i] = 0;
  for (int d = threadIdx.x; d < NB; d += kRadixThreads) dbase[d] = hist_off[sp.hbase + (int64_t)d * sp.hstride];
  __syncthreads();
  const uint32_t lt = (1u << lane) - 1u;
  const int wbase = warp * (ITEMS * 32);
  uint32_t k[ITEMS], v[ITEMS], rk[ITEMS];
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const int idx = wbase + i * 32 + lane;
    const bool valid = idx < count;
    k[i] = valid ? keys_in[base + idx] : 0u;
    v[i] = valid ? vals_in[base + idx] : 0u;
    const uint32_t d = valid ? (((k[i] - kb) >> shift) & mask) : (uint32_t)NB;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    uint32_t before = 0;
    if (valid) before = whist[warp][d];
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) whist[warp][d] = before + __popc(peers);
    __syncwarp();
    rk[i] = before + __popc(peers & lt);
  }
  __syncthreads();
  {
    // per digit: exclusive scan of the warps' counts; then over the digits (each thread owns
    // DPT consecutive digits)
    const bool owns = NB >= kRadixThreads || threadIdx.x < NB;
    uint32_t tsum = 0, dsum[DPT];
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
      const int d = threadIdx.x * DPT + q;
      uint32_t run = 0;
      if (owns) {
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
          const uint32_t c = whist[w][d];
          whist[w][d] = run;
          run += c;
        }
      }
      dsum[q] = run;
      tsum += run;
    }
    unsigned long long tot;
    uint32_t pre = (uint32_t)block_exclusive_scan((unsigned long long)tsum, &tot);
    if (owns) {
#pragma unroll
      for (int q = 0; q < DPT; ++q) {
        dstart[threadIdx.x * DPT + q] = pre;
        pre += dsum[q];
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const int idx = wbase + i * 32 + lane;
    if (idx < count) {
      const uint32_t d = ((k[i] - kb) >> shift) & mask;
      const uint32_t lp = dstart[d] + whist[warp][d] + rk[i];
      sk[lp] = k[i];
      sv[lp] = v[i];
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < count; j += kRadixThreads) {
    const uint32_t kk = sk[j];
    const uint32_t d = ((kk - kb) >> shift) & mask;
    const uint32_t pos = dbase[d] + (uint32_t)j - dstart[d];
    keys_out[pos] = kk;
    vals_out[pos] = sv[j];
  }
}

// Elements per block for a digit width: 7- and 8-bit digits take 16 per thread, 9-bit digits 12
// (their 512-bucket rank tables leave less shared memory for the tile).
int radix_tile(int digit_bits) { return kRadixThreads * (digit_bits == 9 ? 12 : kRadixItems); }

int radix_pass_count(int bit_lo, int bit_hi, int digit_bits) {
  return (bit_hi - bit_lo + digit_bits - 1) / digit_bits;
}

RadixPlan plan_radix(int64_t capacity, int digit_bits, int segments) {
  RadixPlan p{};
  p.capacity = capacity;
  p.digit_bits = digit_bits;
  // a segment's last block may be partial: one block more per segment
  p.nblocks = (capacity + radix_tile(digit_bits) - 1) / radix_tile(digit_bits) + segments;
  if (p.nblocks < 1) p.nblocks = 1;
  p.hist_scan = plan_scan((int64_t)(1 << digit_bits) * p.nblocks);
  return p;
}

int segment_digit_bits(int key_bits) {
  const int passes = (key_bits + 8) / 9;
  const int rb = (key_bits + passes - 1) / passes;
  return rb < 7 ? 7 : rb;
}

namespace {
template <int RB, int ITEMS, bool SEG>
cudaError_t radix_pass(const uint32_t* ki, const uint32_t* vi, uint32_t* ko, uint32_t* vo, int64_t n_host,
                       const uint32_t* n_dev, int shift, uint32_t mask, uint32_t* hist, uint32_t* hist_off,
                       unsigned long long* scan_scratch, const ScanPlan& hs, int64_t nblocks, const SortSeg* segs,
                       int nseg, cudaStream_t st) {
  count_launch();
  radix_upsweep_kernel<RB, ITEMS, SEG><<<(unsigned)nblocks, kRadixThreads, 0, st>>>(
      ki, n_host, n_dev, shift, mask, hist, nblocks, segs, nseg);
  cudaError_t e = exclusive_scan_u32(hist, hist_off, (int64_t)(1 << RB) * nblocks, scan_scratch, hs,
                                     scan_scratch + hs.scratch_elems - 1, st);
  if (e != cudaSuccess) return e;
  count_launch();
  radix_downsweep_kernel<RB, ITEMS, SEG><<<(unsigned)nblocks, kRadixThreads, 0, st>>>(
      ki, vi, ko, vo, n_host, n_dev, shift, mask, hist_off, nblocks, segs, nseg);
  return cudaGetLastError();
}
}  // namespace

cudaError_t radix_sort_pairs(uint32_t* keys_a, uint32_t* vals_a, uint32_t* keys_b, uint32_t* vals_b,
                             int64_t n_host, const uint32_t* n_dev, int bit_lo, int bit_hi,
                             uint32_t* hist, uint32_t* hist_off, unsigned long long* scan_scratch,
                             const RadixPlan& plan, bool* in_b, cudaStream_t st) {
  *in_b = false;
  const int db = plan.digit_bits;
  const int64_t tile = radix_tile(db);
  const int64_t nblocks = n_dev ? plan.nblocks : (n_host + tile - 1) / tile;
  if (nblocks == 0) return cudaSuccess;
  const ScanPlan hs = n_dev ? plan.hist_scan : plan_scan((int64_t)(1 << db) * nblocks);
  uint32_t *ki = keys_a, *vi = vals_a, *ko = keys_b, *vo = vals_b;
  for (int shift = bit_lo; shift < bit_hi; shift += db) {
    const int bits = (bit_hi - shift) < db ? (bit_hi - shift) : db;
    const uint32_t mask = (1u << bits) - 1u;
    const cudaError_t e =
        db == 9 ? radix_pass<9, 12, false>(ki, vi, ko, vo, n_host, n_dev, shift, mask, hist, hist_off, scan_scratch,
                                           hs, nblocks, nullptr, 0, st)
                : radix_pass<8, kRadixItems, false>(ki, vi, ko, vo, n_host, n_dev, shift, mask, hist, hist_off,
                                                    scan_scratch, hs, nblocks, nullptr, 0, st);
    if (e != cudaSuccess) return e;
    uint32_t* t;
    t = ki; ki = ko; ko = t;
    t = vi; vi = vo; vo = t;
    *in_b = !*in_b;
  }
  return cudaGetLastError();
}

cudaError_t radix_sort_segments(uint32_t* keys_a, uint32_t* vals_a, uint32_t* keys_b, uint32_t* vals_b,
                                const SortSeg* segs, int nseg, int key_bits, uint32_t* hist, uint32_t* hist_off,
                                unsigned long long* scan_scratch, const RadixPlan& plan, bool* in_b,
                                cudaStream_t st) {
  *in_b = false;
  const int db = plan.digit_bits;
  if (nseg == 0 || plan.nblocks == 0) return cudaSuccess;
  uint32_t *ki = keys_a, *vi = vals_a, *ko = keys_b, *vo = vals_b;
  for (int shift = 0; shift < key_bits; shift += db) {
    const int bits = (key_bits - shift) < db ? (key_bits - shift) : db;
    const uint32_t mask = (1u << bits) - 1u;
    cudaError_t e;
    if (db == 7)
      e = radix_pass<7, kRadixItems, true>(ki, vi, ko, vo, 0, nullptr, shift, mask, hist, hist_off, scan_scratch,
                                           plan.hist_scan, plan.nblocks, segs, nseg, st);
    else if (db == 8)
      e = radix_pass<8, kRadixItems, true>(ki, vi, ko, vo, 0, nullptr, shift, mask, hist, hist_off, scan_scratch,
                                           plan.hist_scan, plan.nblocks, segs, nseg, st);
    else if (db == 9)
      e = radix_pass<9, 12, true>(ki, vi, ko, vo, 0, nullptr, shift, mask, hist, hist_off, scan_scratch,
                                  plan.hist_scan, plan.nblocks, segs, nseg, st);
    else
      return cudaErrorInvalidValue;
    if (e != cudaSuccess) return e;
    uint32_t* t;
    t = ki; ki = ko; ko = t;
    t = vi; vi = vo; vo = t;
    *in_b = !*in_b;
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// binning kernels
// ------------------------------------------------------------------------------------------
template <typename Tst>
__global__ void height_keys_kernel(const Tst* means, int64_t n, int64_t n_pad, uint32_t* keys, uint32_t* vals) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  // +0.0f maps -0 to +0 so that equal heights compare equal
  const float z = __fadd_rn(load_attr(means, 2 * n_pad + k), 0.0f);
  keys[k] = ~float_order(z);  // ascending key = descending height
  vals[k] = (uint32_t)k;
}

cudaError_t launch_height_keys(const void* means, int dtype, int64_t n, int64_t n_pad, uint32_t* keys,
                               uint32_t* vals, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const unsigned nb = (unsigned)((n + 255) / 256);
  if (dtype == SS_BF16) {
    count_launch();
    height_keys_kernel<__nv_bfloat16><<<nb, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(means), n, n_pad,
                                                           keys, vals);
  } else {
    count_launch();
    height_keys_kernel<float><<<nb, 256, 0, st>>>(static_cast<const float*>(means), n, n_pad, keys, vals);
  }
  return cudaGetLastError();
}

// Tile record of a (target, splat) (written by the projection): x = x0 | y0 << 16,
// y = x1 | y1 << 16 (tile rectangle), z = bitmask of the tiles of the rectangle, in row-major
// order, that the footprint touches (all ones when the rectangle has more than 32 tiles),
// w = number of tiles kept (0: culled).
// Both binning kernels run on a grid of (splats, targets): blockIdx.y is the target, so no
// thread divides its flat index.
__global__ void counts_kernel(BinParams p) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, t = blockIdx.y;
  if (r >= p.n) return;
  const int64_t idx = t * p.n + r;
  const uint32_t k = p.order[r];
  p.counts[idx] = p.rect[t * p.n_pad + k].w;
}

__global__ void emit_kernel(BinParams p) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, t = blockIdx.y;
  if (r >= p.n) return;
  const int64_t idx = t * p.n + r;
  const uint32_t k = p.order[r];
  const uint4 rc = p.rect[t * p.n_pad + k];
  if (rc.w == 0u) return;
  const int x0 = (int)(rc.x & 0xffffu), y0 = (int)(rc.x >> 16), x1 = (int)(rc.y & 0xffffu), y1 = (int)(rc.y >> 16);
  const int ntx = x1 - x0 + 1, nty = y1 - y0 + 1;
  const TargetCam& cam = p.tcams[t];
  int64_t pos = p.offsets[idx];
  uint32_t row_key = (uint32_t)(cam.tile_base + y0 * cam.tiles_x + x0);
  if (ntx * nty <= 32) {
    // the kept tiles only: each row's bits of the mask, lowest first
    uint32_t m = rc.z;
    const uint32_t row_bits = ntx >= 32 ? 0xffffffffu : ((1u << ntx) - 1u);
    for (int r = 0; r < nty && m != 0u; ++r, row_key += (uint32_t)cam.tiles_x) {
      uint32_t b = m & row_bits;
      m = ntx >= 32 ? 0u : m >> ntx;
      while (b != 0u) {
        const int c = __ffs(b) - 1;
        b &= b - 1u;
        if (pos >= p.capacity) return;
        p.keys[pos] = row_key + (uint32_t)c;
        p.vals[pos] = k;
        ++pos;
      }
    }
    return;
  }
  for (int ty = 0; ty < nty; ++ty, row_key += (uint32_t)cam.tiles_x) {
    for (int tx = 0; tx < ntx; ++tx) {
      if (pos >= p.capacity) return;
      p.keys[pos] = row_key + (uint32_t)tx;
      p.vals[pos] = k;
      ++pos;
    }
  }
}

cudaError_t launch_counts(const BinParams& p, cudaStream_t st) {
  const int64_t m = (int64_t)p.n_targets * p.n;
  if (m == 0) return cudaSuccess;
  count_launch();
  counts_kernel<<<dim3((unsigned)((p.n + 255) / 256), (unsigned)p.n_targets), 256, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_emit(const BinParams& p, cudaStream_t st) {
  const int64_t m = (int64_t)p.n_targets * p.n;
  if (m == 0) return cudaSuccess;
  count_launch();
  emit_kernel<<<dim3((unsigned)((p.n + 255) / 256), (unsigned)p.n_targets), 256, 0, st>>>(p);
  return cudaGetLastError();
}

__global__ void finish_count_kernel(StatusBlock* status, const unsigned long long* total, int64_t capacity) {
  const unsigned long long t = *total;
  status->n_isect = t;
  status->n_isect32 = (unsigned int)(t > (unsigned long long)capacity ? (unsigned long long)capacity : t);
  if (t > (unsigned long long)capacity) atomicOr(&status->flags, (unsigned int)FLAG_OVERFLOW);
}

cudaError_t launch_finish_count(StatusBlock* status, const uint32_t*, const uint32_t*,
                                const unsigned long long* total, int64_t capacity, cudaStream_t st) {
  count_launch();
  finish_count_kernel<<<1, 1, 0, st>>>(status, total, capacity);
  return cudaGetLastError();
}

// The tile sort's segments: target t's overlaps are [offsets[t n], offsets[(t + 1) n]) of the
// emitted array (the emission is target-major), clipped to the count the sort takes; each
// segment gets the blocks its elements fill, in target order.  One thread: there are at most a
// few hundred targets.
__global__ void sort_segments_kernel(const uint32_t* offsets, int64_t n, int nt, const TargetCam* tcams,
                                     const StatusBlock* status, int tile, SortSeg* segs) {
  if (threadIdx.x != 0) return;
  const uint32_t total = status->n_isect32;
  uint32_t blk = 0;
  for (int t = 0; t < nt; ++t) {
    const uint32_t s0 = n > 0 ? min(offsets[(int64_t)t * n], total) : 0u;
    const uint32_t s1 = (t + 1 < nt && n > 0) ? min(offsets[(int64_t)(t + 1) * n], total) : total;
    SortSeg g;
    g.start = s0;
    g.len = s1 > s0 ? s1 - s0 : 0u;
    g.blk0 = blk;
    g.nblk = (g.len + (uint32_t)tile - 1u) / (uint32_t)tile;
    g.key_base = (uint32_t)tcams[t].tile_base;
    g.pad[0] = g.pad[1] = g.pad[2] = 0u;
    segs[t] = g;
    blk += g.nblk;
  }
  SortSeg e;
  e.start = total;
  e.len = 0u;
  e.blk0 = blk;
  e.nblk = 0u;
  e.key_base = 0u;
  e.pad[0] = e.pad[1] = e.pad[2] = 0u;
  segs[nt] = e;
}

cudaError_t launch_sort_segments(const uint32_t* offsets, int64_t n, int nt, const TargetCam* tcams,
                                 const StatusBlock* status, int tile, SortSeg* segs, cudaStream_t st) {
  count_launch();
  sort_segments_kernel<<<1, 32, 0, st>>>(offsets, n, nt, tcams, status, tile, segs);
  return cudaGetLastError();
}

// [start, end) of every tile's run in the sorted keys.  Each thread reads four consecutive keys
// (one 16-byte load) and takes its neighbours' boundary keys from the adjacent lanes; the
// boundary lanes of a warp read them from memory.  Tiles without a run keep the zeros the
// caller wrote.
__global__ void ranges_kernel(const uint32_t* keys, const StatusBlock* status, uint2* ranges) {
  const int64_t n = status->n_isect32;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // quad index
  const int64_t i0 = q * 4;
  const int lane = threadIdx.x & 31;
  uint32_t k[4];
  if (i0 + 3 < n) {
    const uint4 v = reinterpret_cast<const uint4*>(keys)[q];
    k[0] = v.x; k[1] = v.y; k[2] = v.z; k[3] = v.w;
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) k[j] = i0 + j < n ? keys[i0 + j] : 0xffffffffu;
  }
  uint32_t prev = __shfl_up_sync(0xffffffffu, k[3], 1);
  uint32_t next = __shfl_down_sync(0xffffffffu, k[0], 1);
  if (lane == 0) prev = (i0 > 0 && i0 - 1 < n) ? keys[i0 - 1] : 0xffffffffu;
  if (lane == 31) next = i0 + 4 < n ? keys[i0 + 4] : 0xffffffffu;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int64_t i = i0 + j;
    if (i >= n) break;
    const uint32_t before = j == 0 ? prev : k[j - 1];
    const uint32_t after = (j == 3 || i + 1 >= n) ? (i + 1 >= n ? 0xffffffffu : next) : k[j + 1];
    if (i == 0 || before != k[j]) ranges[k[j]].x = (uint32_t)i;
    if (i + 1 == n || after != k[j]) ranges[k[j]].y = (uint32_t)(i + 1);
  }
}

cudaError_t launch_ranges(const uint32_t* keys, const StatusBlock* status, uint2* ranges, int64_t capacity,
                          cudaStream_t st) {
  if (capacity == 0) return cudaSuccess;
  const int64_t quads = (capacity + 3) / 4;
  count_launch();
  ranges_kernel<<<(unsigned)((quads + 255) / 256), 256, 0, st>>>(keys, status, ranges);
  return cudaGetLastError();
}

}  // namespace ss
