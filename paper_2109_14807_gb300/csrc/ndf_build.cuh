// Internal interface of the footprint-histogram kernels (binning.cu), used by
// the CP operand preparation in als.cu.
#pragma once

#include <cuda_fp16.h>

#include "common.cuh"

namespace gsp {

// Where one level slice of counts goes.  Any pointer may be null.
//  h:     int32 counts [N][N][B][B]
//  f32:   counts * scale as FP32 (exact; on the TF32 grid when tf32 is set)
//  bf16:  counts * scale rounded to BF16
//  sumsq: one 64-bit counter receiving sum of counts^2 (exact)
// BF16 and TF32 values are rounded without bias (dither_round), the dither
// indexed by base + the element's index in the slice.
struct LevelSink {
  int32_t* h;
  float* f32;
  __nv_bfloat16* bf16;
  float scale;
  unsigned long long* sumsq;
  int tf32;
  long long base;
};

// Outputs of the all-level histogram build; any pointer may be null.  Arrays
// are the full [levels][N][N][B][B] tensors; sumsq has one counter per level.
// Rounding as for LevelSink, the dither indexed by the element's index in the
// full tensor.
struct HistOut {
  int32_t* h;
  float* f32;
  __nv_bfloat16* bf16;
  unsigned long long* sumsq;
  const uint32_t* groups;  // occupied 16-bin groups (bitmask) or null
  float scale[16];         // counts -> operand value, per level
  int tf32;                // f32 values rounded to the TF32 grid without bias
  // Optional scratch of col_prefix_bytes(N, B2) (null: none).  With it the
  // window counts of the coarse levels start from column prefix sums over
  // blocks of rows instead of from the 2^l map rows of the window.
  __half* colp;
};

// Bytes of the column-prefix scratch of launch_box_hist: N / 32 + 1 rows of
// N x B2 FP16 counts; 0 when N < 64 (no window starts on a 32-row block).
size_t col_prefix_bytes(int N, int B2);

// Bytes of the occupied-bin-group bitmask (one bit per 16 bins, B <= 128).
constexpr size_t kGroupBytes = 128 * 128 / 16 / 8;

// Bin the normal map; when d_groups is non-null also mark the occupied
// 16-bin groups there (kGroupBytes, cleared first).
int launch_bins(const float* d_normal_xy, int N, int bins, uint16_t* d_bins,
                uint32_t* d_status, uint32_t* d_groups, cudaStream_t s);
// Histograms of every footprint of every level 0..levels-1 from the bin map,
// whose codes lie in [0, B2) (B2 columns per footprint, a multiple of 16).
int launch_box_hist(const uint16_t* d_bins, int N, int levels, int B2, const HistOut& o,
                    cudaStream_t s);
// Copy / convert an existing int32 slice into a sink.
int launch_cast(const int32_t* d_in, int N, int bins, LevelSink o, cudaStream_t s);

}  // namespace gsp
