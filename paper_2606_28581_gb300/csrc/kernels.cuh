// Kernel parameter blocks and launcher declarations (internal to the library).
#pragma once

#include "common.cuh"

namespace ss {

struct AssembleParams {
  CamRaw cams[kMaxCams];
  TargetStatic tg[kMaxTargets];
  int32_t n_targets;
  const float* dF;     // [n_cams][8] or null
  const float* color;  // [n_cams][12] or null (identity)
  TargetCam* out;
};

struct ProjectCommon {
  const void* means;
  const void* scales;
  const void* quats;
  const void* opacity;
  const void* rgb;
  int64_t n, n_pad;
  int32_t n_targets;
  const TargetCam* tcams;
};

struct ProjectParams {
  ProjectCommon c;
  float4* geom;  // [T][n_pad][3]
  float4* feat;  // [T][n_pad][2]
  uint4* rect;   // [T][n_pad] tile records (see emit_kernel)
  float4* grad;  // [T][n_pad][4]: zeroed for visible pairs
  StatusBlock* status;
  float amin, ln_amin, sigma, det_eps;
  CullConsts cull;
  int32_t tile_w, tile_h;
};

struct GradOut {
  float* means;
  float* scales;
  float* quats;
  float* opacity;
  float* rgb;
  int64_t n_pad;
};

struct ProjectBwdParams {
  ProjectCommon c;
  const uint4* rect;
  const float* grad;  // [T][n_pad][16]
  GradOut g;
  float* d_dF;        // [n_cams][8] or null
  float* d_color;     // [n_cams][12] or null: the 3x3 block C
  float amin, det_eps;
};

// Binning (K2) -----------------------------------------------------------------------
struct BinParams {
  const TargetCam* tcams;
  int32_t n_targets;
  int64_t n, n_pad;
  const uint4* rect;        // [T][n_pad] tile records
  const uint32_t* order;    // [n] splat indices, front to back
  uint32_t* counts;         // [T * n]
  const uint32_t* offsets;  // [T * n] exclusive scan of counts (saturated)
  uint32_t* keys;           // [capacity] global tile id
  uint32_t* vals;           // [capacity] splat index
  int64_t capacity;
  StatusBlock* status;
};

// Rasterization (K3 / K4) ----------------------------------------------------------------
// Staging and grouping of the rasterizer (raster_impl.cuh).  Both directions walk 2 x 4 pixel
// sub-blocks, one per group of two lanes: on the 16-view workload they evaluate 1.41 pairs per
// walked pair where 4 x 4 sub-blocks evaluate 1.66, at the price (in the backward) of two L2 vector
// reductions per lane and step instead of one.  The forward stages batches of 192 records and the
// backward of 224: with their candidate lists they leave eight blocks per SM, and larger batches
// measured no faster.
constexpr int kFwdBatch = 192, kFwdGroupLanes = 2;
constexpr int kBwdBatch = 224, kBwdGroupLanes = 2;

struct RasterParams {
  const TargetCam* tcams;
  const float4* geom;
  const float4* feat;
  const uint32_t* vals;    // sorted splat indices
  const uint2* ranges;     // [total_tiles]
  const uint32_t* items;   // optional work order of global tile ids (persistent)
  StatusBlock* status;
  float* grad;             // [T][n_pad][16] (backward)
  float* d_color;          // [n_cams][12] or null: the offset column c receives sum d(rgb_out)
  int64_t n_pad;
  int32_t n_targets, total_tiles;
  EvalConsts k;
  CullConsts cull;
  float t_min;
  int32_t subblock_cull;   // 0: every staged splat is a candidate of every sub-block
  int32_t distort;         // some target writes (forward) or back-propagates (backward) the distortion
  int32_t count_pairs;     // the forward also counts its walked pairs into the status block
  TargetIO io[kMaxTargets];
};

cudaError_t launch_assemble(const AssembleParams& p, cudaStream_t st);
cudaError_t launch_project(const ProjectParams& p, int dtype, cudaStream_t st);
cudaError_t launch_project_bwd(const ProjectBwdParams& p, int dtype, cudaStream_t st);

// radix sort / scan primitives (sort.cu)
struct ScanPlan {
  int64_t n;
  int levels;
  int64_t level_n[8];
  size_t level_off[8];  // offsets (elements, uint64) into the scratch
  size_t scratch_elems; // uint64 elements
};
ScanPlan plan_scan(int64_t n);
cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, unsigned long long* scratch,
                               const ScanPlan& plan, unsigned long long* total, cudaStream_t st);
// the same scan with 64-bit (unsaturated) outputs
cudaError_t exclusive_scan_u32_u64(const uint32_t* in, unsigned long long* out, int64_t n,
                                   unsigned long long* scratch, const ScanPlan& plan, unsigned long long* total,
                                   cudaStream_t st);

struct RadixPlan {
  int64_t capacity;     // max elements
  int digit_bits;       // 8 or 9
  int64_t nblocks;      // blocks of radix_tile(digit_bits) elements
  ScanPlan hist_scan;   // over 2^digit_bits * nblocks histogram entries
};
constexpr int kRadixThreads = 256;
constexpr int kRadixItems = 16;
constexpr int kRadixTile = kRadixThreads * kRadixItems;
int radix_tile(int digit_bits);
int radix_pass_count(int bit_lo, int bit_hi, int digit_bits);
// segments > 0: the plan of a segmented sort over that many segments (radix_sort_segments)
RadixPlan plan_radix(int64_t capacity, int digit_bits = 8, int segments = 0);
// Digit width of a segmented sort of key_bits-bit keys: as few passes as 9-bit digits allow, the
// bits shared evenly among them, at least 7.
int segment_digit_bits(int key_bits);
// Stable LSD radix sort of (key, value) pairs on key bits [bit_lo, bit_hi).  The element
// count is n_host, or *n_dev when n_dev is not null (device-resident count).  Returns in
// *in_b whether the sorted result ended in the b buffers.
cudaError_t radix_sort_pairs(uint32_t* keys_a, uint32_t* vals_a, uint32_t* keys_b, uint32_t* vals_b,
                             int64_t n_host, const uint32_t* n_dev, int bit_lo, int bit_hi,
                             uint32_t* hist, uint32_t* hist_off, unsigned long long* scan_scratch,
                             const RadixPlan& plan, bool* in_b, cudaStream_t st);

// A segment of a segmented sort: elements [start, start + len), sorted among themselves on the
// bits of key - key_base, by blocks [blk0, blk0 + nblk) of the sort's grid.  An array of nseg + 1
// entries, the last holding in blk0 the number of blocks in use.
struct SortSeg {
  uint32_t start, len;
  uint32_t blk0, nblk;
  uint32_t key_base;
  uint32_t pad[3];
};
// Stable LSD radix sort of each segment on bits [0, key_bits) of key - key_base; the segments
// (device array, filled by launch_sort_segments) stay where they are.
cudaError_t radix_sort_segments(uint32_t* keys_a, uint32_t* vals_a, uint32_t* keys_b, uint32_t* vals_b,
                                const SortSeg* segs, int nseg, int key_bits, uint32_t* hist, uint32_t* hist_off,
                                unsigned long long* scan_scratch, const RadixPlan& plan, bool* in_b,
                                cudaStream_t st);
// The tile sort's segments: one per target, from the scanned per-(target, splat) tile counts.
cudaError_t launch_sort_segments(const uint32_t* offsets, int64_t n, int nt, const TargetCam* tcams,
                                 const StatusBlock* status, int tile, SortSeg* segs, cudaStream_t st);

cudaError_t launch_height_keys(const void* means, int dtype, int64_t n, int64_t n_pad, uint32_t* keys,
                               uint32_t* vals, cudaStream_t st);
cudaError_t launch_counts(const BinParams& p, cudaStream_t st);
cudaError_t launch_emit(const BinParams& p, cudaStream_t st);
cudaError_t launch_finish_count(StatusBlock* status, const uint32_t* counts_last,
                                const uint32_t* offsets_last, const unsigned long long* total,
                                int64_t capacity, cudaStream_t st);
cudaError_t launch_ranges(const uint32_t* keys, const StatusBlock* status, uint2* ranges,
                          int64_t capacity, cudaStream_t st);

// raster (raster.cu)
cudaError_t launch_raster_fwd(const RasterParams& p, int tile_w, int tile_h, int batch, bool persistent,
                              int num_sms, cudaStream_t st);
cudaError_t launch_raster_bwd(const RasterParams& p, int tile_w, int tile_h, int batch, bool persistent,
                              int num_sms, cudaStream_t st);

}  // namespace ss
