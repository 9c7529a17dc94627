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

// Bk: bin columns per footprint seen by the MTTKRP passes.  0 means all B * B
// bins; the CP-ALS prepare sets it to the occupied bins of the map rounded up
// to 128 (see als.cu, bin compaction).  Bt: columns stored per operand row
// (0: Bk).  The tensor-core passes store the occupied bins rounded up to 16
// only and read columns Bt .. Bk-1 as zeros through the TMA tensor bounds.
struct MttkrpDims {
  int N, L, B, R;
  int Bk = 0;
  int Bt = 0;
  long long N2() const { return static_cast<long long>(N) * N; }
  int B2() const { return Bk ? Bk : B * B; }
  int B2t() const { return Bt ? Bt : B2(); }
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
constexpr int kLstMaxRanges = 320;  // >= 2 CTAs per SM x 152 SMs

// Structured path (structured.cu): exact MTTKRPs from the bin map, the footprint
// windows moved onto the spatial factors.  Buffers, all device, caller-owned:
struct StructWs {
  float* part;    // [splits][N][L][R]  side-pass partials
  double* pre;    // [L][N + 1][R]      FP64 prefix along the pass's columns
  float* sig;     // [N][L][R]          the pass's reduced sums (sigma for mode l)
  double* sig64;  // [N][L][R]          the same in FP64
  double* segtot; // [L][N / 32][R]     prefix segment totals
  double* off;    // [L][N / 32][R]     prefix segment offsets
  float* stpart;  // [ctas][B][R]       bin-pass partials
  const double* lscale;  // [L]         c_l: counts -> tensor values
  float* gw = nullptr;   // [L][N]      Gaussian footprint weights (null: box footprints)
  float* conv = nullptr; // [N][L][R]   Gaussian-weighted sums of the side pass
};
struct StructSizes {
  size_t table_floats, part_floats, pre_doubles, seg_doubles, stpart_floats;
  size_t gauss_floats, autocorr_ints, normpart_doubles;
};
bool struct_supported(const MttkrpDims& d);
StructSizes struct_sizes(const MttkrpDims& d);
// out[u][l][r] = sum_{i < 2^l} f[(u + a_l - i) mod N][r]  (the window's adjoint)
int struct_window_tables(const float* f, float* out, const StructWs& w, const MttkrpDims& d,
                         cudaStream_t s);
// Side pass over bm [rows][cols] (rows = the reduction index, win its window
// table) into w.pre; with M non-null also M[col][r] of the mode (FP64, and FP32
// into Mf when non-null).
int struct_side(const uint16_t* bm, const float* win, const float* fs, const float* ft,
                const float* fl, const StructWs& w, const MttkrpDims& d, double* M, float* Mf,
                cudaStream_t s);
// M_l from w.sig of the y side pass and the beta table.
int struct_level(const float* be, const StructWs& w, const MttkrpDims& d, double* M, float* Mf,
                 cudaStream_t s);
// Bin pass: mode s (mode_t 0, tab = ft) or t (mode_t 1, tab = fs).
int struct_bins(const uint16_t* bm, const float* al, const float* be, const float* fl,
                const float* tab, int mode_t, const StructWs& w, const MttkrpDims& d, double* M,
                float* Mf, cudaStream_t s);
// lscale[l] = B^2 / (4 * 4^l), or 1 with raw counts
int struct_level_scales(int L, int B, int raw, int gauss, double* lscale, cudaStream_t s);
// Gaussian footprints: the weights (w.gw, and FP64 in gw64 [L][N]) and ||T||^2
// into *norm2 from the same-bin autocorrelation A [N][N] of the bin map and the
// weights' autocorrelation K [L][N]; normpart [N][L] scratch.  Needs w.lscale.
int struct_gauss_prepare(const uint16_t* bins, const StructWs& w, const MttkrpDims& d,
                         double* gw64, double* K, int32_t* A, double* normpart, double* norm2,
                         cudaStream_t s);
int struct_transpose_bins(const uint16_t* in, uint16_t* out, int N, cudaStream_t s);
int struct_bins_from_level0(const int32_t* h0, int N, int B, uint16_t* bins, uint32_t* status,
                            cudaStream_t s);

}  // namespace gsp
