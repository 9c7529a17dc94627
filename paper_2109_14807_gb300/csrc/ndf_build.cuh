// Internal interface of the footprint-histogram kernels (binning.cu), used by
// the CP operand preparation in als.cu.
#pragma once

#include "common.cuh"

namespace gsp {

// Where one level slice of counts goes.  Any pointer may be null.
//  h:     int32 counts [N][N][B][B]
//  f32:   counts * scale as FP32
//  bf16:  counts * scale rounded to BF16 (round to nearest even)
//  sumsq: one 64-bit counter receiving sum of counts^2 (exact)
struct LevelSink {
  int32_t* h;
  float* f32;
  __nv_bfloat16* bf16;
  float scale;
  unsigned long long* sumsq;
};

int launch_bins(const float* d_normal_xy, int N, int bins, uint16_t* d_bins,
                uint32_t* d_status, cudaStream_t s);
// Level 0: one-hot counts of every texel's own bin.
int launch_level0(const uint16_t* d_bins, int N, int bins, LevelSink o, cudaStream_t s);
// Level l+1 from level l (l = level_in) by the doubling identity
// W_{l+1}(x) = W_l(x - d) u W_l(x + d), d = 2^(l-1) (W_1(x) = W_0(x-1) u W_0(x)),
// applied along x and along y: four shifted adds per count.
int launch_double(const int32_t* d_in, int N, int bins, int level_in, LevelSink o,
                  cudaStream_t s);
// Copy / convert an existing int32 slice into a sink.
int launch_cast(const int32_t* d_in, int N, int bins, LevelSink o, cudaStream_t s);

}  // namespace gsp
