// Internal interface of the two MTTKRP contractions of a CP-ALS sweep.
//
// The sweep uses the dimension tree {x, y} | {l, s, t}: both passes stream the
// operand tensor T [l][xy][st] (xy = y * N + x, st = s * B + t) once.
//   Y'[xy][r]    = sum_{l, st} T[l][xy][st] * fl[l][r] fs[s][r] ft[t][r]
//                  (then M_x, M_y are small contractions of Y' with fy, fx)
//   Z'[l][st][r] = sum_{xy} T[l][xy][st] * fx[x][r] fy[y][r]
//                  (then M_l, M_s, M_t are small contractions of Z')
// Each mode update of plain ALS (Kolda & Bader) needs exactly these sums, so
// the sweep is the textbook one, only associated differently.
#pragma once

#include "common.cuh"

namespace gsp {

struct MttkrpDims {
  int N, L, B, R;
  long long N2() const { return static_cast<long long>(N) * N; }
  int B2() const { return B * B; }
};

// Number of split-K chunks per level used by the Z' pass (partials [L*C][B2][R]).
int lst_chunks(const MttkrpDims& d, int precision);

// FP32 CUDA-core path.  KR: [L*B2][R] fp32 (fl*fs*ft).  T: fp32.
int simt_mttkrp_xy(const float* T, const float* KR, float* Yp, const MttkrpDims& d,
                   cudaStream_t s);
int simt_mttkrp_lst(const float* T, const float* fx, const float* fy, float* Zpart,
                    const MttkrpDims& d, int chunks, cudaStream_t s);

// tcgen05 path.  KRt: [R][L*B2] in the operand type (bf16 or fp32 read as tf32).
// Returns GSP_ERR_UNSUPPORTED when the shape is outside the kernel's support.
// `err` (device word, may be null) receives GSP_DEV_TIMEOUT if a bounded wait
// inside the kernel gave up.
int tc_mttkrp_xy(const void* T, const void* KRt, float* Yp, const MttkrpDims& d, int precision,
                 uint32_t* err, cudaStream_t s);
// Z' pass: builds the fx operand in FXt (2 * R * N operand elements at most),
// writes per-CTA partial slices to Zpart (at most kLstMaxRanges * 2 * B2 * R
// floats) and reduces them into Zp [L][B2][R].
int tc_mttkrp_lst(const void* T, const float* fx, const float* fy, void* FXt, float* Zpart,
                  float* Zp, const MttkrpDims& d, int precision, uint32_t* err, cudaStream_t s);
bool tc_supported(const MttkrpDims& d, int precision);
constexpr int kLstMaxRanges = 256;

}  // namespace gsp
