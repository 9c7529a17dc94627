// Shared helpers of the CUDA library (host and device).  No method arithmetic.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "gsp.h"

namespace gsp {

// Last failing cudaError_t of this host thread (read by gsp_last_cuda_error).
int& last_cuda_error();

inline int cuda_fail(cudaError_t e) {
  last_cuda_error() = static_cast<int>(e);
  return GSP_ERR_CUDA;
}

#define GSP_CUDA(call)                                   \
  do {                                                   \
    cudaError_t gsp_e_ = (call);                         \
    if (gsp_e_ != cudaSuccess) return gsp::cuda_fail(gsp_e_); \
  } while (0)

// Every kernel launch is followed by GSP_CHECK_LAUNCH(): it counts the launch
// and turns a launch error into GSP_ERR_CUDA.
void count_launch();
#define GSP_CHECK_LAUNCH() \
  do {                     \
    gsp::count_launch();   \
    GSP_CUDA(cudaGetLastError()); \
  } while (0)

enum ProfId {
  PROF_BINS = 0, PROF_LEVEL0, PROF_DOUBLE, PROF_CAST, PROF_MTTKRP_XY, PROF_MTTKRP_LST,
  PROF_ALS_SMALL, PROF_TABLES, PROF_QUERY, PROF_QUERY_BWD, PROF_ADAM, PROF_STRUCT_TABLES,
  PROF_STRUCT_SIDE, PROF_STRUCT_BINS, PROF_SOLVE, PROF_COUNT
};
// Event pair around one launch (no-ops unless profiling is enabled).
void prof_begin(int id, cudaStream_t s);
void prof_end(int id, cudaStream_t s);

#define GSP_TRY(expr)               \
  do {                              \
    int gsp_rc_ = (expr);           \
    if (gsp_rc_ != GSP_OK) return gsp_rc_; \
  } while (0)

inline bool is_pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }

inline int ilog2(long long v) {
  int l = 0;
  while ((1LL << (l + 1)) <= v) ++l;
  return l;
}

inline cudaStream_t to_stream(gsp_stream s) { return reinterpret_cast<cudaStream_t>(s); }

// Streaming-multiprocessor count of the current device (cached per device).
int sm_count();

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

inline unsigned grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  return static_cast<unsigned>(b < 1 ? 1 : b);
}

// Checks shared by the NDF-building calls.
inline bool valid_map(int N, int levels, int bins) {
  return is_pow2(N) && N >= 2 && N <= 1024 && levels >= 1 && levels <= ilog2(N) + 1 &&
         is_pow2(bins) && bins >= 4 && bins <= 128;
}

// Round an FP32 value to the nearest TF32 value (ties away from zero), so the
// tensor core, which drops the low 13 mantissa bits, sees an unbiased operand.
__device__ __forceinline__ float round_tf32(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r);
}

// Unbiased rounding of the NDF operand tensor to fewer significand bits.
// Round-to-nearest of counts drawn from a decreasing distribution (most
// footprint counts are small) errs low on average, and that bias, not the
// rounding noise, is what moves an ALS fit.  Instead a dither d in [0, 2^drop)
// is added below the kept bits and the sum truncated, so that a value between
// two representable neighbours goes up with probability equal to its distance
// from the lower one.  The dithers come from the Weyl sequence frac(i * phi)
// (32-bit fixed point, phi = golden ratio; Knuth, TAOCP vol. 3, Sec. 6.4):
// equidistributed, cheap and the same wherever an element is produced.  TF32
// element e takes the top bits of the Weyl value of e; BF16 elements 2p and
// 2p + 1 take the low and the high 16 bits of the Weyl value of their pair p.
// Representable values (low bits zero) are unchanged, so counts with at most
// 8 (BF16) or 11 (TF32) significant bits stay exact.
constexpr uint32_t kWeyl = 0x9E3779B9u;

__device__ __forceinline__ uint32_t weyl_dither(unsigned long long i) {
  return static_cast<uint32_t>(i) * kWeyl;
}

// FP32 bits of v >= 0 rounded to keep 32 - drop bits, dither d (full 32 bits).
__device__ __forceinline__ uint32_t dither_round(float v, uint32_t d, int drop) {
  return (__float_as_uint(v) + (d >> (32 - drop))) & ~((1u << drop) - 1u);
}

// The two 16-bit BF16 dithers of the element pair that starts at even e.
__device__ __forceinline__ uint32_t bf16_pair_bits(unsigned long long e) {
  return static_cast<uint32_t>(e >> 1) * kWeyl;
}

// The 16-bit BF16 dither of element e.
__device__ __forceinline__ uint32_t bf16_dither16(unsigned long long e) {
  const uint32_t r = bf16_pair_bits(e);
  return (e & 1) ? r >> 16 : r & 0xFFFFu;
}

// BF16 bits of v >= 0 rounded without bias, dither d16 < 2^16.
__device__ __forceinline__ uint32_t bf16_dither(float v, uint32_t d16) {
  return (__float_as_uint(v) + d16) >> 16;
}

// Two BF16 values (element 0 in the low half) as one 32-bit word, rounded
// without bias with the dithers in the low and high halves of rbits: the
// stochastic-rounding convert adds each half below the kept bits of its value
// and truncates, the same as bf16_dither (the CP operand prepared from
// histograms takes bf16_dither and the one from the normal map this form; the
// GPU tests require the two to agree).
__device__ __forceinline__ uint32_t bf16_pair_dither(float v0, float v1, uint32_t rbits) {
  uint32_t r;
  asm("cvt.rs.satfinite.bf16x2.f32 %0, %1, %2, %3;" : "=r"(r) : "f"(v1), "f"(v0), "r"(rbits));
  return r;
}

// v >= 0 on the TF32 grid (10 fraction bits), rounded without bias.
__device__ __forceinline__ float tf32_dither(float v, uint32_t d) {
  return __uint_as_float(dither_round(v, d, 13));
}

__device__ __forceinline__ void set_status(uint32_t* status, uint32_t bits) {
  if (status) atomicOr(status, bits);
}

}  // namespace gsp
