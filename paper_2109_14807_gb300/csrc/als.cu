// Rows a3-a4: CP decomposition of the footprint NDF tensor by alternating
// least squares (Sec. 4.2, Eq. 3; CP-ALS of Kolda & Bader 2009).
//
// Per sweep, modes in the order x, y, l, s, t:
//   Y'  = T contracted with fl (.) fs (.) ft          (one pass over T)
//   x:  M_x = sum_y Y' fy      -> solve -> normalise
//   y:  M_y = sum_x Y' fx_new  -> solve -> normalise
//   Z'  = T contracted with fx_new (.) fy_new         (one pass over T)
//   l:  M_l = sum_st Z' fs ft           -> solve -> normalise
//   s:  M_s = sum_{l,t} Z' fl_new ft    -> solve -> normalise
//   t:  M_t = sum_{l,s} Z' fl_new fs_new-> solve -> normalise -> fit
// "solve" is A_n = M_n V^-1 with V the Hadamard product of the other four FP64
// Gram matrices (FP64 Cholesky; pseudo-inverse by Jacobi eigendecomposition
// when V is not numerically positive definite); "normalise" divides every
// column by its 2-norm, which becomes lambda.  All small linear algebra is
// FP64; the two passes over T are the MTTKRP kernels (FP32 FFMA or tcgen05).
#include <math.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "mttkrp.cuh"
#include "ndf_build.cuh"
#include "solve.cuh"

namespace gsp {
namespace {

constexpr int kMaxCpRank = 64;
constexpr int kJacobiMaxRank = 64;
constexpr int kGramRows = 64;  // rows of a factor per partial Gram matrix

// Workspace layout.  The head (bin map, column tables, the small FP64 ALS
// arrays and flags) depends only on the shape and precision and comes first,
// so that the operand's columns can be counted into it before the rest is
// laid out; the operand and the arrays sized by its columns follow.
struct CpLayout {
  size_t T, bins, Yp, Zp, Zpart, KR, FX, M, G, Gpart, W, lam, fit, sumsq, norm2, flags, cols, head,
      total;
  // GSP_PREC_STRUCTURED only (zero-sized otherwise)
  size_t binsT, AL, BE, part, pre, sig, sig64, segtot, off, stpart, lscale;
  // GSP_PREC_STRUCTURED_GAUSSIAN only
  size_t gw, gw64, K, conv, A, normpart;
};

size_t esize(int prec) { return prec == GSP_PREC_BF16 || prec == GSP_PREC_BF16_1X ? 2 : 4; }
bool is_bf16(int prec) { return prec == GSP_PREC_BF16 || prec == GSP_PREC_BF16_1X; }
bool is_structured(int prec) {
  return prec == GSP_PREC_STRUCTURED || prec == GSP_PREC_STRUCTURED_GAUSSIAN;
}

// Bytes of the bin map (+ the occupied-group mask) and of the column tables
// {count, Bk, Bt, 0}, column -> bin [B2], bin -> column [B2], occupancy mask
// [B2 / 32]: the first two entries of every CP workspace.
size_t bins_bytes(int N) { return static_cast<size_t>(N) * N * sizeof(uint16_t) + kGroupBytes; }
size_t cols_bytes(int B) {
  const size_t B2 = static_cast<size_t>(B) * B;
  return (4 + 2 * B2 + (B2 + 31) / 32) * sizeof(int32_t);
}
size_t count_ws_bytes(int N, int B) { return align_up(bins_bytes(N), 256) + align_up(cols_bytes(B), 256); }

// Stored columns per operand row: the FP32 CUDA-core pass reads T with its
// own tile grid and stores all Bk columns; the tensor-core passes store the
// occupied bins rounded up to 16 (Bt16 from the column table).
int stored_cols(int prec, int Bk, int Bt16) { return prec == GSP_PREC_FP32 ? Bk : Bt16; }

// Walked (Bk) and stored (Bt) operand columns for `count` occupied bins: the
// rule k_bin_compact applies on the device.
void cols_for(int B2, int count, int prec, int* Bk, int* Bt) {
  const bool ident = B2 < 256;
  int bk = ident ? B2 : ((count + 127) / 128) * 128;
  if (bk < 128 && !ident) bk = 128;
  if (bk > B2) bk = B2;
  int bt16 = ident ? B2 : (count + 15) / 16 * 16;
  if (bt16 < 16) bt16 = 16;
  if (bt16 > bk) bt16 = bk;
  *Bk = bk;
  *Bt = stored_cols(prec, bk, bt16);
}

// FP32 split-K partials of the Z' pass: L * chunks * Bk * R floats for the
// walked columns Bk; with the columns unknown (d.Bk == 0) the largest over
// every column count the compaction can produce.
size_t simt_part_floats(const MttkrpDims& d) {
  auto part = [&](int bk) {
    MttkrpDims e = d;
    e.Bk = bk;
    e.Bt = bk;
    return static_cast<size_t>(d.L) * lst_chunks(e, GSP_PREC_FP32) * bk * d.R;
  };
  if (d.Bk) return part(d.Bk);
  const int B2 = d.B * d.B;
  if (B2 < 256) return part(B2);
  size_t best = 0;
  for (int bk = 128; bk <= B2; bk += 128) best = std::max(best, part(bk));
  return best;
}

CpLayout cp_layout(const MttkrpDims& d, int prec) {
  CpLayout o;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off = align_up(off + bytes, 256);
    return at;
  };
  const size_t N2 = static_cast<size_t>(d.N2()), B2 = static_cast<size_t>(d.B2());
  const size_t L = d.L, R = d.R;
  const bool st = prec == GSP_PREC_STRUCTURED || prec == GSP_PREC_STRUCTURED_GAUSSIAN;
  const bool ga = prec == GSP_PREC_STRUCTURED_GAUSSIAN;
  const size_t dense = st ? 0 : 1;  // the structured path builds no tensor
  // ---- head: fixed by (N, L, B, R, precision)
  o.bins = take(bins_bytes(d.N));
  o.cols = take(cols_bytes(d.B));
  size_t imax = static_cast<size_t>(d.N > d.B ? (d.N > d.L ? d.N : d.L) : (d.B > d.L ? d.B : d.L));
  o.M = take(imax * R * sizeof(double));
  o.G = take(5 * R * R * sizeof(double));
  o.Gpart = take((imax + kGramRows - 1) / kGramRows * R * R * sizeof(double));
  o.W = take((3 * R * R + R) * sizeof(double) + 16);  // L, Z^T, 1/diag(L), mode, then W
  o.lam = take(R * sizeof(double));
  o.fit = take(GSP_MAX_SWEEPS * sizeof(double));
  o.sumsq = take(L * sizeof(unsigned long long));
  o.norm2 = take(sizeof(double));
  o.flags = take(16);
  o.head = off;
  // ---- the operand (B2t() stored columns) and the arrays sized by its columns
  o.T = take(dense * N2 * L * static_cast<size_t>(d.B2t()) * esize(prec));
  o.Yp = take(dense * N2 * R * sizeof(float));
  o.Zp = take(dense * L * B2 * R * sizeof(float));
  const size_t tc_part = static_cast<size_t>(kLstMaxRanges) * 2 * B2 * R;
  o.Zpart = take(dense * (prec == GSP_PREC_FP32 ? simt_part_floats(d) : tc_part) * sizeof(float));
  o.KR = take(dense * 2 * R * L * B2 * sizeof(float));  // FP32 rows, or a hi + lo operand pair
  o.FX = take(dense * 2 * R * static_cast<size_t>(d.N) * sizeof(float));  // Z' fx operand
  const StructSizes z = st ? struct_sizes(d) : StructSizes{0, 0, 0, 0, 0, 0, 0, 0};
  o.binsT = take(st ? N2 * sizeof(uint16_t) : 0);
  o.AL = take(z.table_floats * sizeof(float));
  o.BE = take(z.table_floats * sizeof(float));
  o.part = take(z.part_floats * sizeof(float));
  o.pre = take(z.pre_doubles * sizeof(double));
  o.sig = take(z.table_floats * sizeof(float));
  o.sig64 = take(z.table_floats * sizeof(double));
  o.segtot = take(z.seg_doubles * sizeof(double));
  o.off = take(z.seg_doubles * sizeof(double));
  o.stpart = take(z.stpart_floats * sizeof(float));
  o.lscale = take(st ? L * sizeof(double) : 0);
  o.gw = take(ga ? z.gauss_floats * sizeof(float) : 0);
  o.gw64 = take(ga ? z.gauss_floats * sizeof(double) : 0);
  o.K = take(ga ? z.gauss_floats * sizeof(double) : 0);
  o.conv = take(ga ? z.table_floats * sizeof(float) : 0);
  o.A = take(ga ? z.autocorr_ints * sizeof(int32_t) : 0);
  o.normpart = take(ga ? z.normpart_doubles * sizeof(double) : 0);
  o.total = off;
  return o;
}

bool valid_cp(int N, int L, int B, int R, int prec) {
  return valid_map(N, L, B) && N >= 8 && B >= 8 && is_pow2(R) && R >= 8 && R <= kMaxCpRank &&
         prec >= GSP_PREC_FP32 && prec <= GSP_PREC_STRUCTURED_GAUSSIAN;
}

// --------------------------------------------------------------- kernels --

// Dense bin of operand column c: cols (column -> dense bin, -1 for padding)
// or the identity when the operand holds all B * B bins.
__device__ __forceinline__ int col_bin(const int32_t* cols, int c) { return cols ? cols[c] : c; }

// KR[(l*K1 + c)][r] = fl[l][r] fs[s][r] ft[t][r], (s, t) the bin of column c
// (0 for a padding column); row layout, FP32.  K1 = operand columns.
__global__ void k_kr_rows(const float* __restrict__ fl, const float* __restrict__ fs,
                          const float* __restrict__ ft, int L, int B, int K1, int R,
                          const int32_t* __restrict__ cols, float* __restrict__ out) {
  long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  long long total = static_cast<long long>(L) * K1 * R;
  if (i >= total) return;
  int r = static_cast<int>(i % R);
  long long k = i / R;
  const int cidx = static_cast<int>(k % K1);
  const int l = static_cast<int>(k / K1);
  const int b = col_bin(cols, cidx);
  out[i] = b < 0 ? 0.0f : fl[l * R + r] * fs[(b / B) * R + r] * ft[(b % B) * R + r];
}

// KRt[r][l*K1 + c] in the operand type (the K-major B operand of the
// tensor-core pass): BF16, or FP32 rounded to the nearest TF32; with `split`
// rows R..2R-1 hold the remainder v - hi of rows 0..R-1, rounded the same way.
template <typename OutT>
__global__ void k_kr_cols(const float* __restrict__ fl, const float* __restrict__ fs,
                          const float* __restrict__ ft, int L, int B, int K1, int R, int split,
                          const int32_t* __restrict__ cols, OutT* __restrict__ out) {
  long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  long long K = static_cast<long long>(L) * K1;
  if (i >= K * R) return;
  long long k = i % K;
  int r = static_cast<int>(i / K);
  const int cidx = static_cast<int>(k % K1);
  const int l = static_cast<int>(k / K1);
  const int b = col_bin(cols, cidx);
  float v = b < 0 ? 0.0f : fl[l * R + r] * fs[(b / B) * R + r] * ft[(b % B) * R + r];
  if constexpr (sizeof(OutT) == 2) {
    __nv_bfloat16 hi = __float2bfloat16_rn(v);
    out[i] = hi;
    if (split) out[i + K * R] = __float2bfloat16_rn(v - __bfloat162float(hi));
  } else {
    const float hi = round_tf32(v);
    out[i] = hi;
    if (split) out[i + K * R] = round_tf32(v - hi);
  }
}

// ------------------------------------------------------- bin compaction --
// Bins that no texel of the map falls in are zero in every footprint of every
// level: the dense operand's columns for them carry nothing (Sec. 4.2 drops
// blank NDF blocks for the same reason).  The operand keeps the occupied bins
// only, in increasing order: the MTTKRP passes see Bk columns (the count
// padded with zero columns to a multiple of 128, the tensor-core tile), and
// the tensor-core precisions store only Bt of them (the count rounded up to
// 16), the TMA tensor bounds supplying the zeros past Bt.  The bin map is
// renumbered to those columns, so the histogram and MTTKRP kernels just see a
// smaller bin axis, and only the Khatri-Rao operand and the (l, s, t)
// contractions map a column back to its (s, t).  All results are those of
// the dense operand up to the order of FP32 accumulation.

// occ bit b: bin b occurs in the map.  Lanes holding the same bin elect one
// shared-memory OR; every CTA ORs its mask into the global one.
__global__ void k_bin_occupancy(const uint16_t* __restrict__ bins, long long n, int B2,
                                uint32_t* __restrict__ occ) {
  __shared__ uint32_t m[512];  // B2 <= 16384
  const int words = (B2 + 31) / 32;
  for (int i = threadIdx.x; i < words; i += blockDim.x) m[i] = 0u;
  __syncthreads();
  for (long long u = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; u < n;
       u += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int b = bins[u];
    const unsigned peers = __match_any_sync(__activemask(), b);
    if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicOr(m + (b >> 5), 1u << (b & 31));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < words; i += blockDim.x)
    if (m[i]) atomicOr(occ + i, m[i]);
}

// cols = {count, Bk, Bt, 0, col -> bin [Bk] (-1: padding), bin -> col [B2]
// (-1: absent)}.  Bk = B2 (identity columns) when B2 < 256, else the occupied
// count rounded up to 128, at most B2; Bt = the count rounded up to 16 (B2 for
// identity columns), the columns the tensor-core precisions store.  One CTA of
// 512 threads, one word each.
__global__ void __launch_bounds__(512) k_bin_compact(const uint32_t* __restrict__ occ, int B2,
                                                     int32_t* __restrict__ cols) {
  __shared__ int wbase[512];
  const int words = (B2 + 31) / 32;
  const int w = threadIdx.x;
  const uint32_t bits = w < words ? occ[w] : 0u;
  wbase[w] = __popc(bits);
  __syncthreads();
  for (int off = 1; off < 512; off <<= 1) {  // inclusive scan of the word counts
    const int v = w >= off ? wbase[w - off] : 0;
    __syncthreads();
    wbase[w] += v;
    __syncthreads();
  }
  const int count = wbase[511];
  const bool ident = B2 < 256;
  int Bk = ident ? B2 : ((count + 127) / 128) * 128;
  if (Bk < 128 && !ident) Bk = 128;
  if (Bk > B2) Bk = B2;
  int32_t* col_bin_t = cols + 4;
  int32_t* bin_col_t = cols + 4 + B2;
  if (w == 0) {
    cols[0] = ident ? B2 : count;
    cols[1] = Bk;
    cols[2] = ident ? B2 : min(Bk, max(16, (count + 15) / 16 * 16));
    cols[3] = 0;
  }
  if (w < words) {
    int rank = wbase[w] - __popc(bits);
    for (int k = 0; k < 32; ++k) {
      const int b = w * 32 + k;
      if (b >= B2) break;
      if (ident) {
        bin_col_t[b] = b;
        col_bin_t[b] = b;
      } else if ((bits >> k) & 1u) {
        bin_col_t[b] = rank;
        col_bin_t[rank] = b;
        ++rank;
      } else {
        bin_col_t[b] = -1;
      }
    }
  }
  __syncthreads();
  if (!ident)
    for (int c = count + w; c < Bk; c += 512) col_bin_t[c] = -1;
}

// bins[u] <- column of bins[u]
__global__ void k_bin_remap(uint16_t* __restrict__ bins, long long n, const int32_t* __restrict__ cols,
                            int B2) {
  const long long u = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (u < n) bins[u] = static_cast<uint16_t>(cols[4 + B2 + bins[u]]);
}

// groups bit g: column group g (16 columns) holds an occupied bin
__global__ void k_col_groups(const int32_t* __restrict__ cols, uint32_t* __restrict__ groups) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= static_cast<int>(kGroupBytes * 8)) return;
  const int count = cols[0];
  if ((g & 31) == 0) {
    uint32_t wbits = 0u;
    for (int k = 0; k < 32; ++k)
      if ((g + k) * 16 < count) wbits |= 1u << k;
    groups[g >> 5] = wbits;
  }
}

// The operand from int32 histograms [N][N][B2] of one level: column c takes
// the count of its bin (0 for padding), times scale, rounded like the
// histogram sink (exact FP32; TF32 / BF16 without bias, the dither indexed by
// the element's index base + i in the operand); Sigma count^2 into *sumsq.
template <typename OutT>
__global__ void k_cast_cols(const int32_t* __restrict__ h, long long fps, int B2, int Bk,
                            const int32_t* __restrict__ cols, float scale, int tf32,
                            long long base, OutT* __restrict__ out,
                            unsigned long long* __restrict__ sumsq) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  unsigned long long q = 0;
  if (i < fps * Bk) {
    const long long fp = i / Bk;
    const int c = static_cast<int>(i % Bk);
    const int b = cols[4 + c];
    const int v = b < 0 ? 0 : h[fp * B2 + b];
    q = static_cast<unsigned long long>(static_cast<long long>(v) * v);
    const float f = static_cast<float>(v) * scale;
    const unsigned long long e = static_cast<unsigned long long>(base + i);
    if constexpr (sizeof(OutT) == 2) {
      out[i] = __ushort_as_bfloat16(static_cast<unsigned short>(bf16_dither(f, bf16_dither16(e))));
    } else {
      out[i] = tf32 ? tf32_dither(f, weyl_dither(e)) : f;
    }
  }
  for (int off = 16; off > 0; off >>= 1) q += __shfl_down_sync(0xffffffffu, q, off);
  if ((threadIdx.x & 31) == 0 && q) atomicAdd(sumsq, q);
}

// M_l, M_s or M_t (mode 2, 3, 4) from Z' [L][K1][R] over the operand columns:
//   l: M[l][r] = sum_c Z'[l][c][r] fs[s_c][r] ft[t_c][r]
//   s: M[s][r] = sum_{l, c : s_c = s} Z'[l][c][r] fl[l][r] ft[t_c][r]
//   t: M[t][r] = sum_{l, c : t_c = t} Z'[l][c][r] fl[l][r] fs[s_c][r]
// (s_c, t_c) the bin of column c (padding columns skipped).  One CTA per output
// row; thread (part, r) sums every 256/R-th term with compensated FP32, the
// parts are added in FP64 in a fixed order.
__global__ void __launch_bounds__(256) k_contract_cols(const float* __restrict__ Zp, int L, int B,
                                                       int K1, int R, const int32_t* __restrict__ colbin,
                                                       const float* __restrict__ fl,
                                                       const float* __restrict__ fs,
                                                       const float* __restrict__ ft, int mode,
                                                       double* __restrict__ M,
                                                       float* __restrict__ Mf) {
  __shared__ double red[256];
  const int i = blockIdx.x;
  const int r = threadIdx.x % R, part = threadIdx.x / R, P = blockDim.x / R;
  float hi = 0.0f, lo = 0.0f;
  auto add = [&](float x) {
    const float t = __fadd_rn(hi, x);
    const float bp = __fsub_rn(t, hi);
    lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(x, bp)));
    hi = t;
  };
  if (part < P) {
    if (mode == 2) {
      for (int c = part; c < K1; c += P) {
        const int b = colbin[c];
        if (b >= 0)
          add(Zp[(static_cast<size_t>(i) * K1 + c) * R + r] * fs[(b / B) * R + r] * ft[(b % B) * R + r]);
      }
    } else {
      for (int c = part; c < K1; c += P) {
        const int b = colbin[c];
        if (b < 0 || (mode == 3 ? b / B : b % B) != i) continue;
        const float o = mode == 3 ? ft[(b % B) * R + r] : fs[(b / B) * R + r];
        for (int l = 0; l < L; ++l) add(Zp[(static_cast<size_t>(l) * K1 + c) * R + r] * fl[l * R + r] * o);
      }
    }
  }
  red[threadIdx.x] = part < P ? static_cast<double>(hi) + static_cast<double>(lo) : 0.0;
  __syncthreads();
  if (threadIdx.x < R) {
    double acc = 0.0;
    for (int q = 0; q < P; ++q) acc += red[q * R + threadIdx.x];
    if (M) M[i * R + threadIdx.x] = acc;
    if (Mf) Mf[i * R + threadIdx.x] = static_cast<float>(acc);
  }
}

// Zp[l][st][r] = sum_c Zpart[l*C + c][st][r], fixed order
__global__ void k_zreduce(const float* __restrict__ Zpart, float* __restrict__ Zp, int L, int C,
                          long long per_level) {
  long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (e >= per_level * L) return;
  long long l = e / per_level, rem = e % per_level;
  const float* p = Zpart + (l * C) * per_level + rem;
  float acc = 0.0f;
  for (int c = 0; c < C; ++c) acc += p[static_cast<long long>(c) * per_level];
  Zp[e] = acc;
}

// M[i][r] = sum_{j1 < J1, j2 < J2} W[(i*wi + j1*w1 + j2*w2)][r] * A1[j1][r] * A2[j2][r]
struct CParams {
  const float* W;
  long long wi, w1, w2;
  int J1, J2;
  const float* A1;
  const float* A2;
  int R;
  double* M;
  float* Mf;
};

__global__ void __launch_bounds__(256) k_contract(CParams p) {
  __shared__ double red[256];
  const int i = blockIdx.x;
  const int R = p.R;
  const int r = threadIdx.x % R;
  const int jl = threadIdx.x / R;
  const int JL = blockDim.x / R;
  const long long J = static_cast<long long>(p.J1) * p.J2;
  // FP32 (the operands are FP32 tensor-core / FFMA sums); 4 independent chains.
  // J2 is a power of two, so j splits into (j1, j2) by shift and mask.
  const int j2_log = 31 - __clz(p.J2);
  const int j2_mask = p.J2 - 1;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  int j = jl;
  const int Ji = static_cast<int>(J);
  for (; j + 3 * JL < Ji; j += 4 * JL) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int jj = j + u * JL;
      const int j1 = jj >> j2_log, j2 = jj & j2_mask;
      float v = p.W[(i * p.wi + j1 * p.w1 + j2 * p.w2) * R + r];
      if (p.A1) v *= p.A1[j1 * R + r];
      if (p.A2) v *= p.A2[j2 * R + r];
      acc[u] += v;
    }
  }
  for (; j < Ji; j += JL) {
    const int j1 = j >> j2_log, j2 = j & j2_mask;
    float v = p.W[(i * p.wi + j1 * p.w1 + j2 * p.w2) * R + r];
    if (p.A1) v *= p.A1[j1 * R + r];
    if (p.A2) v *= p.A2[j2 * R + r];
    acc[0] += v;
  }
  red[threadIdx.x] = static_cast<double>((acc[0] + acc[1]) + (acc[2] + acc[3]));
  __syncthreads();
  for (int w = JL / 2; w > 0; w >>= 1) {
    if (jl < w) red[threadIdx.x] += red[threadIdx.x + w * R];
    __syncthreads();
  }
  if (jl == 0) {
    if (p.M) p.M[i * R + r] = red[threadIdx.x];
    if (p.Mf) p.Mf[i * R + r] = static_cast<float>(red[threadIdx.x]);
  }
}

// M[i][r] = sum_j W[i * wi + j * w1][r] * A1[j][r] (the x and y contractions
// of Y'), rows of R floats read as float4: one CTA per i, its threads = groups
// of j x R / 4 runs of 4 ranks, 4 row pairs in flight per thread (16-byte
// loads: one 4-byte load per thread and row left these passes at half the HBM
// rate); the group sums are combined in shared memory in a fixed order.
// R % 4 == 0, W and A1 16-byte aligned.
__global__ void __launch_bounds__(256) k_contract4(const float* __restrict__ W, long long wi,
                                                   long long w1, int J, const float* __restrict__ A1,
                                                   int R, double* __restrict__ M,
                                                   float* __restrict__ Mf) {
  __shared__ float4 part[256];
  const int RV = R >> 2;
  const int G = blockDim.x / RV;
  const int i = blockIdx.x;
  const int gj = threadIdx.x / RV, r4 = threadIdx.x % RV;
  const float4* W4 = reinterpret_cast<const float4*>(W);
  const float4* A4 = reinterpret_cast<const float4*>(A1);
  float4 acc[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) acc[u] = make_float4(0.f, 0.f, 0.f, 0.f);
  auto fma4 = [](float4& c, float4 a, float4 b) {
    c.x = fmaf(a.x, b.x, c.x);
    c.y = fmaf(a.y, b.y, c.y);
    c.z = fmaf(a.z, b.z, c.z);
    c.w = fmaf(a.w, b.w, c.w);
  };
  if (gj < G) {
    int j = gj;
    for (; j + 3 * G < J; j += 4 * G) {
      float4 w[4], a[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const long long jj = j + u * G;
        w[u] = __ldg(W4 + (i * wi + jj * w1) * RV + r4);
        a[u] = __ldg(A4 + jj * RV + r4);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) fma4(acc[u], w[u], a[u]);
    }
    for (; j < J; j += G)
      fma4(acc[0], __ldg(W4 + (i * wi + static_cast<long long>(j) * w1) * RV + r4),
           __ldg(A4 + static_cast<long long>(j) * RV + r4));
    part[threadIdx.x] = make_float4((acc[0].x + acc[1].x) + (acc[2].x + acc[3].x),
                                    (acc[0].y + acc[1].y) + (acc[2].y + acc[3].y),
                                    (acc[0].z + acc[1].z) + (acc[2].z + acc[3].z),
                                    (acc[0].w + acc[1].w) + (acc[2].w + acc[3].w));
  }
  __syncthreads();
  if (gj == 0) {
    float4 t = part[r4];
    for (int k = 1; k < G; ++k) {
      const float4 v = part[k * RV + r4];
      t.x += v.x; t.y += v.y; t.z += v.z; t.w += v.w;
    }
    const float tv[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (M) M[i * R + 4 * r4 + c] = static_cast<double>(tv[c]);
      if (Mf) Mf[i * R + 4 * r4 + c] = tv[c];
    }
  }
}

// M[i][r] = sum_j W[(i + j*w1)][r] * A1[j][r] for rows i of stride 1: one CTA
// per row i, its 256 threads = 256/R groups of j (j = g, g + G, ...) x R
// ranks, 8 loads in flight per thread; the group sums are combined in shared
// memory in a fixed order.
__global__ void __launch_bounds__(256) k_contract_rows(const float* __restrict__ W, long long w1,
                                                       int J, const float* __restrict__ A1,
                                                       int R, double* __restrict__ M,
                                                       float* __restrict__ Mf) {
  __shared__ float part[256];
  const int G = blockDim.x / R;
  const int i = blockIdx.x;
  const int gj = threadIdx.x / R, r = threadIdx.x % R;
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  int j = gj;
  for (; j + 7 * G < J; j += 8 * G) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const long long jj = j + u * G;
      acc[u] = fmaf(W[(i + jj * w1) * R + r], A1[jj * R + r], acc[u]);
    }
  }
  for (; j < J; j += G) acc[0] = fmaf(W[(i + static_cast<long long>(j) * w1) * R + r], A1[j * R + r], acc[0]);
  part[threadIdx.x] = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
  __syncthreads();
  if (gj == 0) {
    float t = part[r];
    for (int k = 1; k < G; ++k) t += part[k * R + r];
    if (M) M[i * R + r] = static_cast<double>(t);
    if (Mf) Mf[i * R + r] = t;
  }
}

// G[r1][r2] = sum_i A[i][r1] A[i][r2], FP64; 256/R row slices per output row,
// combined in a fixed order

// Gpart[chunk][r1][r2] = sum over the chunk's rows of A[i][r1] A[i][r2]: FP32
// dot products over 32 rows, added in FP64.  One CTA per 64-row chunk, the
// chunk staged in shared memory.
__global__ void __launch_bounds__(256) k_gram_part(const float* __restrict__ A, int I, int R,
                                                   double* __restrict__ Gpart) {
  __shared__ float As[kGramRows * kMaxCpRank];
  const int i0 = blockIdx.x * kGramRows;
  const int rows = min(kGramRows, I - i0);
  for (int e = threadIdx.x; e < rows * R; e += blockDim.x) As[e] = A[static_cast<size_t>(i0) * R + e];
  __syncthreads();
  double* out = Gpart + static_cast<size_t>(blockIdx.x) * R * R;
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
    const int r1 = e / R, r2 = e % R;
    double acc = 0.0;
    for (int c0 = 0; c0 < rows; c0 += 32) {
      float chunk = 0.0f;
      const int c1 = min(rows, c0 + 32);
      for (int i = c0; i < c1; ++i) chunk = fmaf(As[i * R + r1], As[i * R + r2], chunk);
      acc += static_cast<double>(chunk);
    }
    out[e] = acc;
  }
}

// G[e] = sum_chunk Gpart[chunk][e], FP64 in chunk order.
__global__ void k_gram_sum(const double* __restrict__ Gpart, int chunks, int R2,
                           double* __restrict__ G) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= R2) return;
  double acc = 0.0;
  for (int c = 0; c < chunks; ++c) acc += Gpart[static_cast<size_t>(c) * R2 + e];
  G[e] = acc;
}

// Hadamard product of the four Gram matrices other than `skip`.
// V (row stride ld) = Hadamard product of the Gram matrices of all modes but `skip`.
__device__ void hadamard_v(const double* __restrict__ G, int R, int skip, double* V, int ld) {
  // four elements per thread and pass, their 16 Gram loads issued together
  const int RR = R * R;
  for (int e0 = threadIdx.x; e0 < RR; e0 += 4 * blockDim.x) {
    double v[4] = {1.0, 1.0, 1.0, 1.0};
#pragma unroll
    for (int m = 0; m < 5; ++m) {
      if (m == skip) continue;
      double g[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int e = e0 + k * static_cast<int>(blockDim.x);
        g[k] = e < RR ? G[m * RR + e] : 1.0;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] *= g[k];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int e = e0 + k * static_cast<int>(blockDim.x);
      if (e < RR) V[(e / R) * ld + e % R] = v[k];
    }
  }
}


// Right-looking Cholesky of V in shared memory (lower triangle, row-major).
// Returns false when a pivot is not above thresh; block-uniform result.
// In place on V (row stride ld = R + 1, so that the column reads of the
// trailing update fall on distinct banks).

// Layout of the solve scratch `fac` (doubles): L [R][R], Z^T [R][R] with
// Z = L^-1, 1/diag(L) [R], the mode word (int, padded to 16 bytes), W [R][R].
struct SolveScratch {
  double *L, *Zt, *invd, *W;
  int* mode;
};
__host__ __device__ inline SolveScratch solve_scratch(double* fac, int R) {
  SolveScratch s;
  s.L = fac;
  s.Zt = fac + R * R;
  s.invd = fac + 2 * R * R;
  s.mode = reinterpret_cast<int*>(fac + 2 * R * R + R);
  s.W = fac + 2 * R * R + R + 2;
  return s;
}

// Threads of k_chol (1024 made its latency-bound FP64 steps slower: the
// steps' barriers span more warps).
constexpr int kCholThreads = 256;

// One CTA: factor V (Hadamard product of the other modes' Grams) for the
// least-squares update: L and 1/diag(L), mode 0.  When V is not numerically
// positive definite: W = V^+ from a Jacobi eigendecomposition, mode 1, and
// GSP_DEV_NUMERIC.
__global__ void __launch_bounds__(kCholThreads) k_chol(const double* __restrict__ G, int R, int skip,
                                              double* __restrict__ out, uint32_t* flags) {
  extern __shared__ double smem[];
  __shared__ double invd_s[kMaxCpRank];
  const int ld = R + 1;
  double* V = smem;               // [R][R + 1] for the Cholesky, [R][R] for the fallback
  double* Q = smem + R * ld;      // [R][R] (eigenvectors, R <= 64 only)
  const SolveScratch ss = solve_scratch(out, R);
  double* L = ss.L;
  double* invd = ss.invd;
  int* mode = ss.mode;
  const double eps = 2.220446049250313e-16;
  hadamard_v(G, R, skip, V, ld);
  __syncthreads();
  const double mx = max_diag(V, R, ld);
  bool ok = cholesky_packed(V, R, ld, R * eps * mx, invd_s);
  if (!ok) {
    if (threadIdx.x == 0 && flags) atomicOr(flags, GSP_DEV_NUMERIC);
    if (R <= kJacobiMaxRank) {
      hadamard_v(G, R, skip, V, R);
      __syncthreads();
      jacobi_eigen(V, Q, R);
      const double lmax = max_diag(V, R, R);
      const double cutoff = R * eps * lmax;
      for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
        const int a = e / R, b = e % R;
        double acc = 0.0;
        for (int k = 0; k < R; ++k) {
          const double lam = V[k * R + k];
          if (lam > cutoff) acc += Q[a * R + k] * Q[b * R + k] / lam;
        }
        ss.W[e] = acc;
      }
      if (threadIdx.x == 0) *mode = 1;
      return;
    }
    const double deltas[3] = {1e-12, 1e-9, 1e-6};
    for (int t = 0; t < 3 && !ok; ++t) {
      hadamard_v(G, R, skip, V, ld);
      __syncthreads();
      if (threadIdx.x == 0)
        for (int k = 0; k < R; ++k) V[k * ld + k] += deltas[t] * mx;
      __syncthreads();
      ok = cholesky_packed(V, R, ld, R * eps * mx, invd_s);
    }
    if (!ok) {  // give up on this update: A = 0, lambda = 0 for the mode
      for (int e = threadIdx.x; e < R * R; e += blockDim.x) ss.W[e] = 0.0;
      if (threadIdx.x == 0) *mode = 1;
      return;
    }
  }
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
    const int i = e / R, k = e % R;
    L[e] = k <= i ? V[i * ld + k] : 0.0;
  }
  for (int k = threadIdx.x; k < R; k += blockDim.x) invd[k] = invd_s[k];
  if (threadIdx.x == 0) *mode = 0;
}

// Column c of Z = L^-1 by forward substitution in column (axpy) form, one warp
// per column: lane q holds b_k for rows k = c + q and c + q + 32; for j = c ..
// R - 1, z_j = b_j / L_jj is broadcast from its owner and every later row does
// b_k -= L_kj z_j.  No block barriers on the sequential chain.  Writes Z^T[c][:].
// Skipped in mode 1.
__global__ void __launch_bounds__(128) k_inv_cols(double* __restrict__ fac, int R) {
  const SolveScratch ss = solve_scratch(fac, R);
  if (*ss.mode != 0) return;
  const int c = blockIdx.x * 4 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (c >= R) return;
  const int k0 = c + lane, k1 = k0 + 32;
  double b0 = lane == 0 ? 1.0 : 0.0, b1 = 0.0;
  for (int j = c; j < R; ++j) {
    const int q = j - c;
    const double bj = __shfl_sync(0xffffffffu, q >= 32 ? b1 : b0, q & 31);
    const double z = bj * ss.invd[j];
    if (lane == 0) ss.Zt[c * R + j] = z;
    if (k0 > j && k0 < R) b0 = fma(-ss.L[k0 * R + j], z, b0);
    if (k1 > j && k1 < R) b1 = fma(-ss.L[k1 * R + j], z, b1);
  }
  for (int j = lane; j < c; j += 32) ss.Zt[c * R + j] = 0.0;
}

// W = Z^T Z = V^-1: W[a][b] = sum_{k >= max(a, b)} Z^T[a][k] Z^T[b][k]; one CTA
// per row a.  Skipped in mode 1 (W already holds V^+).
__global__ void __launch_bounds__(kMaxCpRank) k_gram_inv(double* __restrict__ fac, int R) {
  const SolveScratch ss = solve_scratch(fac, R);
  if (*ss.mode != 0) return;
  const int a = blockIdx.x, b = threadIdx.x;
  if (b >= R) return;
  double acc = 0.0;
  for (int k = a > b ? a : b; k < R; ++k) acc += ss.Zt[a * R + k] * ss.Zt[b * R + k];
  ss.W[a * R + b] = acc;
}

// A[i][c] = sum_k M[i][k] W[k][c]   (FP64 accumulate, FP32 out)
__global__ void k_apply(const double* __restrict__ M, double* __restrict__ fac, int I, int R,
                        float* __restrict__ A) {
  const SolveScratch ss = solve_scratch(fac, R);
  long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (e >= static_cast<long long>(I) * R) return;
  const int i = static_cast<int>(e / R), c = static_cast<int>(e % R);
  double acc = 0.0;
  for (int k = 0; k < R; ++k) acc += M[i * R + k] * ss.W[k * R + c];
  A[e] = static_cast<float>(acc);
}

// lambda_c = ||A[:, c]||_2; A[:, c] /= lambda_c (left alone if zero)
__global__ void __launch_bounds__(256) k_colnorm(float* __restrict__ A, int I, int R,
                                                 double* __restrict__ lam64,
                                                 float* __restrict__ lam32) {
  __shared__ double red[256];
  __shared__ double nrm;
  const int c = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < I; i += blockDim.x) {
    double v = A[i * R + c];
    acc += v * v;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    nrm = sqrt(red[0]);
    lam64[c] = nrm;
    if (lam32) lam32[c] = static_cast<float>(nrm);
  }
  __syncthreads();
  if (nrm > 0.0) {
    for (int i = threadIdx.x; i < I; i += blockDim.x)
      A[i * R + c] = static_cast<float>(static_cast<double>(A[i * R + c]) / nrm);
  }
}

__global__ void k_norm2(const unsigned long long* __restrict__ sumsq, int L, int B, int raw,
                        double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double acc = 0.0;
  for (int l = 0; l < L; ++l) {
    double sc = raw ? 1.0 : static_cast<double>(B) * B / (4.0 * ldexp(1.0, 2 * l));
    acc += static_cast<double>(sumsq[l]) * sc * sc;
  }
  *out = acc;
}

// fit = 1 - sqrt(max(0, ||T||^2 + ||T_hat||^2 - 2 <T, T_hat>)) / ||T||
__global__ void __launch_bounds__(256) k_fit(const double* __restrict__ Mt,
                                             const float* __restrict__ ft,
                                             const double* __restrict__ lam,
                                             const double* __restrict__ G, int B, int R,
                                             const double* __restrict__ norm2,
                                             double* __restrict__ fit_out) {
  __shared__ double ri[256], rh[256];
  double inner = 0.0, hat = 0.0;
  for (int e = threadIdx.x; e < B * R; e += blockDim.x) {
    int r = e % R;
    inner += lam[r] * Mt[e] * static_cast<double>(ft[e]);
  }
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
    int a = e / R, b = e % R;
    double g = 1.0;
    for (int m = 0; m < 5; ++m) g *= G[m * R * R + e];
    hat += lam[a] * lam[b] * g;
  }
  ri[threadIdx.x] = inner;
  rh[threadIdx.x] = hat;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      ri[threadIdx.x] += ri[threadIdx.x + w];
      rh[threadIdx.x] += rh[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double n2 = *norm2;
    double res = n2 + rh[0] - 2.0 * ri[0];
    *fit_out = 1.0 - sqrt(res > 0.0 ? res : 0.0) / sqrt(n2);
  }
}

// ------------------------------------------------------------ host side --

struct Ctx {
  MttkrpDims d;
  int prec;
  CpLayout lay;
  char* ws;
  size_t ws_bytes;
  cudaStream_t s;
  // Side stream for the part of a mode update that does not need the mode's
  // MTTKRP (null: everything runs on s).
  cudaStream_t side = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  template <typename T>
  T* at(size_t off) const { return reinterpret_cast<T*>(ws + off); }
};

// Owns the side stream and the fork / join events of one gsp_cp_sweeps call.
struct SideStream {
  Ctx& c;
  explicit SideStream(Ctx& ctx) : c(ctx) {}
  int open() {
    // while c.s is being captured into a graph everything stays on c.s
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    GSP_CUDA(cudaStreamIsCapturing(c.s, &cap));
    if (cap != cudaStreamCaptureStatusNone) return GSP_OK;
    GSP_CUDA(cudaStreamCreateWithFlags(&c.side, cudaStreamNonBlocking));
    GSP_CUDA(cudaEventCreateWithFlags(&c.fork_ev, cudaEventDisableTiming));
    GSP_CUDA(cudaEventCreateWithFlags(&c.join_ev, cudaEventDisableTiming));
    return GSP_OK;
  }
  ~SideStream() {
    if (c.join_ev) cudaEventDestroy(c.join_ev);
    if (c.fork_ev) cudaEventDestroy(c.fork_ev);
    if (c.side) cudaStreamDestroy(c.side);  // deferred until its work completes
    c.side = nullptr;
    c.fork_ev = c.join_ev = nullptr;
  }
};

int ensure_smem_attr() {
  static int done_dev = -1;
  int dev = 0;
  GSP_CUDA(cudaGetDevice(&dev));
  if (done_dev != dev) {
    // k_chol: V (R*(R+1) doubles) plus eigenvectors for R <= 64
    GSP_CUDA(cudaFuncSetAttribute(k_chol, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (2 * kMaxCpRank + 1) * kMaxCpRank * static_cast<int>(sizeof(double))));
    done_dev = dev;
  }
  return GSP_OK;
}

int run_xy(const Ctx& c, const float* fl, const float* fs, const float* ft) {
  const MttkrpDims& d = c.d;
  long long K = static_cast<long long>(d.L) * d.B2();
  const int32_t* cb = c.at<int32_t>(c.lay.cols) + 4;
  if (c.prec == GSP_PREC_FP32) {
    k_kr_rows<<<grid_for(K * d.R, 256), 256, 0, c.s>>>(fl, fs, ft, d.L, d.B, d.B2(), d.R, cb,
                                                       c.at<float>(c.lay.KR));
    GSP_CHECK_LAUNCH();
    return simt_mttkrp_xy(c.at<float>(c.lay.T), c.at<float>(c.lay.KR), c.at<float>(c.lay.Yp), d, c.s);
  }
  if (is_bf16(c.prec))
    k_kr_cols<__nv_bfloat16><<<grid_for(K * d.R, 256), 256, 0, c.s>>>(
        fl, fs, ft, d.L, d.B, d.B2(), d.R, c.prec == GSP_PREC_BF16 ? 1 : 0, cb,
        c.at<__nv_bfloat16>(c.lay.KR));
  else
    k_kr_cols<float><<<grid_for(K * d.R, 256), 256, 0, c.s>>>(fl, fs, ft, d.L, d.B, d.B2(), d.R, 1,
                                                               cb, c.at<float>(c.lay.KR));
  GSP_CHECK_LAUNCH();
  return tc_mttkrp_xy(c.ws + c.lay.T, c.ws + c.lay.KR, c.at<float>(c.lay.Yp), d, c.prec,
                      c.at<uint32_t>(c.lay.flags), c.s);
}

int run_lst(const Ctx& c, const float* fx, const float* fy) {
  const MttkrpDims& d = c.d;
  if (c.prec != GSP_PREC_FP32)
    return tc_mttkrp_lst(c.ws + c.lay.T, fx, fy, c.ws + c.lay.FX, c.at<float>(c.lay.Zpart),
                         c.at<float>(c.lay.Zp), d, c.prec, c.at<uint32_t>(c.lay.flags), c.s);
  // split-K chunks (the partial buffer is laid out for this many)
  const int C = lst_chunks(d, c.prec);
  GSP_TRY(simt_mttkrp_lst(c.at<float>(c.lay.T), fx, fy, c.at<float>(c.lay.Zpart), d, C, c.s));
  long long per_level = static_cast<long long>(d.B2()) * d.R;
  k_zreduce<<<grid_for(per_level * d.L, 256), 256, 0, c.s>>>(c.at<float>(c.lay.Zpart),
                                                             c.at<float>(c.lay.Zp), d.L, C, per_level);
  GSP_CHECK_LAUNCH();
  return GSP_OK;
}

// mode 0..4 = x, y, l, s, t
int contract(const Ctx& c, int mode, const gsp_cp_factors& f, double* M, float* Mf) {
  const MttkrpDims& d = c.d;
  CParams p{};
  p.R = d.R;
  p.M = M;
  p.Mf = Mf;
  int I = 0;
  const long long B = d.B, B2 = d.B2(), N = d.N;
  switch (mode) {
    case 0:  // x: W = Y'[(y*N + x)]
      p.W = c.at<float>(c.lay.Yp); p.wi = 1; p.w1 = N; p.w2 = 0; p.J1 = d.N; p.J2 = 1;
      p.A1 = f.fy; p.A2 = nullptr; I = d.N;
      break;
    case 1:  // y
      p.W = c.at<float>(c.lay.Yp); p.wi = N; p.w1 = 1; p.w2 = 0; p.J1 = d.N; p.J2 = 1;
      p.A1 = f.fx; p.A2 = nullptr; I = d.N;
      break;
    case 2:  // l: W = Z'[l][s*B + t]
      p.W = c.at<float>(c.lay.Zp); p.wi = B2; p.w1 = B; p.w2 = 1; p.J1 = d.B; p.J2 = d.B;
      p.A1 = f.fs; p.A2 = f.ft; I = d.L;
      break;
    case 3:  // s
      p.W = c.at<float>(c.lay.Zp); p.wi = B; p.w1 = B2; p.w2 = 1; p.J1 = d.L; p.J2 = d.B;
      p.A1 = f.fl; p.A2 = f.ft; I = d.B;
      break;
    default:  // t
      p.W = c.at<float>(c.lay.Zp); p.wi = 1; p.w1 = B2; p.w2 = B; p.J1 = d.L; p.J2 = d.B;
      p.A1 = f.fl; p.A2 = f.fs; I = d.B;
      break;
  }
  prof_begin(PROF_ALS_SMALL, c.s);
  const bool v4 = d.R % 4 == 0 && d.R <= 256 &&
                  ((reinterpret_cast<uintptr_t>(p.W) | reinterpret_cast<uintptr_t>(p.A1)) & 15) == 0;
  if (mode <= 1 && v4)
    k_contract4<<<I, 256, 0, c.s>>>(p.W, p.wi, p.w1, p.J1, p.A1, d.R, M, Mf);
  else if (mode == 0)
    k_contract_rows<<<I, 256, 0, c.s>>>(p.W, p.w1, p.J1, p.A1, d.R, M, Mf);
  else if (mode == 1)
    k_contract<<<I, 256, 0, c.s>>>(p);
  else
    k_contract_cols<<<I, 256, 0, c.s>>>(c.at<float>(c.lay.Zp), d.L, d.B, d.B2(), d.R,
                                        c.at<int32_t>(c.lay.cols) + 4, f.fl, f.fs, f.ft, mode, M, Mf);
  prof_end(PROF_ALS_SMALL, c.s);
  GSP_CHECK_LAUNCH();
  return GSP_OK;
}

float* factor_ptr(const gsp_cp_factors& f, int mode) {
  switch (mode) {
    case 0: return f.fx;
    case 1: return f.fy;
    case 2: return f.fl;
    case 3: return f.fs;
    default: return f.ft;
  }
}

int mode_rows(const MttkrpDims& d, int mode) {
  return mode < 2 ? d.N : mode == 2 ? d.L : d.B;
}

int gram(const Ctx& c, const gsp_cp_factors& f, int mode) {
  const int R = c.d.R;
  const int I = mode_rows(c.d, mode);
  const int chunks = (I + kGramRows - 1) / kGramRows;
  double* G = c.at<double>(c.lay.G) + static_cast<size_t>(mode) * R * R;
  double* Gpart = c.at<double>(c.lay.Gpart);
  k_gram_part<<<chunks, 256, 0, c.s>>>(factor_ptr(f, mode), I, R, chunks > 1 ? Gpart : G);
  GSP_CHECK_LAUNCH();
  if (chunks > 1) {
    k_gram_sum<<<grid_for(R * R, 256), 256, 0, c.s>>>(Gpart, chunks, R * R, G);
    GSP_CHECK_LAUNCH();
  }
  return GSP_OK;
}

// First half of a mode update, independent of the mode's MTTKRP: factor V (the
// Hadamard product of the other modes' Grams) and form W = V^-1 (or V^+), on
// stream st.
int solve_factor(const Ctx& c, int mode, cudaStream_t st) {
  const int R = c.d.R;
  size_t smem = static_cast<size_t>(R) * (R + 1) * sizeof(double) +
                (R <= kJacobiMaxRank ? static_cast<size_t>(R) * R * sizeof(double) : 0);
  double* fac = c.at<double>(c.lay.W);
  prof_begin(PROF_SOLVE, st);
  k_chol<<<1, kCholThreads, smem, st>>>(c.at<double>(c.lay.G), R, mode, fac,
                                       c.at<uint32_t>(c.lay.flags));
  GSP_CHECK_LAUNCH();
  k_inv_cols<<<(R + 3) / 4, 128, 0, st>>>(fac, R);
  GSP_CHECK_LAUNCH();
  k_gram_inv<<<R, kMaxCpRank, 0, st>>>(fac, R);
  GSP_CHECK_LAUNCH();
  prof_end(PROF_SOLVE, st);
  return GSP_OK;
}

// Second half, on the main stream once M_n is there: A_n = M_n W, column norms
// into lambda, the new Gram matrix of the mode.
int solve_apply(const Ctx& c, const gsp_cp_factors& f, int mode) {
  const int R = c.d.R;
  const int I = mode_rows(c.d, mode);
  float* A = factor_ptr(f, mode);
  prof_begin(PROF_ALS_SMALL, c.s);
  k_apply<<<grid_for(static_cast<long long>(I) * R, 256), 256, 0, c.s>>>(c.at<double>(c.lay.M),
                                                                         c.at<double>(c.lay.W), I,
                                                                         R, A);
  GSP_CHECK_LAUNCH();
  k_colnorm<<<R, 256, 0, c.s>>>(A, I, R, c.at<double>(c.lay.lam), f.lambda);
  GSP_CHECK_LAUNCH();
  GSP_TRY(gram(c, f, mode));
  prof_end(PROF_ALS_SMALL, c.s);
  return GSP_OK;
}

// Start the first half of mode `mode`'s update: on the side stream after
// everything already queued on the main stream, or inline without one.  Call
// it before the mode's MTTKRP so the two run concurrently.
int fork_solve(const Ctx& c, int mode) {
  if (!c.side) return GSP_OK;
  GSP_CUDA(cudaEventRecord(c.fork_ev, c.s));
  GSP_CUDA(cudaStreamWaitEvent(c.side, c.fork_ev, 0));
  GSP_TRY(solve_factor(c, mode, c.side));
  GSP_CUDA(cudaEventRecord(c.join_ev, c.side));
  return GSP_OK;
}

// Finish mode `mode`'s update once its MTTKRP (in c.lay.M) is queued.
int join_solve(const Ctx& c, const gsp_cp_factors& f, int mode) {
  if (c.side)
    GSP_CUDA(cudaStreamWaitEvent(c.s, c.join_ev, 0));
  else
    GSP_TRY(solve_factor(c, mode, c.s));
  return solve_apply(c, f, mode);
}

// Operand columns of prepared workspaces, kept on the host so that sweeps and
// MTTKRPs launch without reading the device (and can be graph-captured).
struct ColsEntry {
  const void* ws;
  int N, L, B, R, prec, Bk, Bt;
};
std::mutex g_cols_mu;
std::vector<ColsEntry> g_cols;

void remember_cols(const void* ws, const MttkrpDims& d, int prec, int Bk, int Bt) {
  std::lock_guard<std::mutex> lk(g_cols_mu);
  for (auto& e : g_cols)
    if (e.ws == ws) {
      e = ColsEntry{ws, d.N, d.L, d.B, d.R, prec, Bk, Bt};
      return;
    }
  if (g_cols.size() >= 256) g_cols.erase(g_cols.begin());
  g_cols.push_back(ColsEntry{ws, d.N, d.L, d.B, d.R, prec, Bk, Bt});
}

bool recall_cols(const void* ws, const MttkrpDims& d, int prec, int* Bk, int* Bt) {
  std::lock_guard<std::mutex> lk(g_cols_mu);
  for (const auto& e : g_cols)
    if (e.ws == ws && e.N == d.N && e.L == d.L && e.B == d.B && e.R == d.R && e.prec == prec) {
      *Bk = e.Bk;
      *Bt = e.Bt;
      return true;
    }
  return false;
}

bool valid_cols(const MttkrpDims& d, int Bk, int Bt) {
  const int B2 = d.B * d.B;
  if (B2 < 256) return Bk == B2 && Bt == B2;
  return Bk >= 128 && Bk <= B2 && Bk % 128 == 0 && Bt >= 16 && Bt <= Bk && Bt % 16 == 0;
}

bool path_supported(const MttkrpDims& d, int prec) {
  if (prec == GSP_PREC_FP32) return true;
  if (is_structured(prec)) return struct_supported(d);
  return tc_supported(d, prec);
}

// A context whose head offsets are valid; the dense-path arrays behind the
// head are laid out once the operand's columns are known (set_cols).  The
// structured path's layout is complete at once.
int make_ctx(int N, int L, int B, int R, int prec, void* d_ws, size_t ws_bytes, gsp_stream st,
             Ctx& c) {
  if (!valid_cp(N, L, B, R, prec)) return GSP_ERR_INVALID_ARG;
  c.d = MttkrpDims{N, L, B, R};
  c.prec = prec;
  if (!path_supported(c.d, prec)) return GSP_ERR_UNSUPPORTED;
  c.lay = cp_layout(c.d, prec);
  const size_t need = is_structured(prec) ? c.lay.total : c.lay.head;
  if (!d_ws || ws_bytes < need) return GSP_ERR_WORKSPACE;
  c.ws = static_cast<char*>(d_ws);
  c.ws_bytes = ws_bytes;
  c.s = to_stream(st);
  return ensure_smem_attr();
}

// Lay out the operand of Bk walked / Bt stored columns behind the head; the
// workspace must hold it.
int set_cols(Ctx& c, int Bk, int Bt) {
  c.d.Bk = Bk;
  c.d.Bt = Bt;
  c.lay = cp_layout(c.d, c.prec);
  return c.ws_bytes < c.lay.total ? GSP_ERR_WORKSPACE : GSP_OK;
}

// The operand columns of a prepared dense-path workspace: from the host record
// of its prepare, else read from the workspace; then the full layout.
int resolve_cols(Ctx& c) {
  if (is_structured(c.prec)) return GSP_OK;
  int Bk = 0, Bt = 0;
  if (!recall_cols(c.ws, c.d, c.prec, &Bk, &Bt)) {
    int32_t h[3] = {0, 0, 0};
    GSP_CUDA(cudaMemcpyAsync(h, c.ws + c.lay.cols, sizeof(h), cudaMemcpyDeviceToHost, c.s));
    GSP_CUDA(cudaStreamSynchronize(c.s));
    Bk = h[1];
    Bt = stored_cols(c.prec, h[1], h[2]);
    if (!valid_cols(c.d, Bk, Bt)) return GSP_ERR_INVALID_ARG;  // not a prepared workspace
    GSP_TRY(set_cols(c, Bk, Bt));
    remember_cols(c.ws, c.d, c.prec, Bk, Bt);
    return GSP_OK;
  }
  return set_cols(c, Bk, Bt);
}

bool valid_factors(const gsp_cp_factors* f) {
  return f && f->fx && f->fy && f->fl && f->fs && f->ft && f->lambda;
}

// One sweep over the prepared operand: the xy pass, modes x and y, the (l, s, t)
// pass, modes l, s and t.
int dense_sweep(const Ctx& c, const gsp_cp_factors& f) {
  double* M = c.at<double>(c.lay.M);
  GSP_TRY(fork_solve(c, 0));
  GSP_TRY(run_xy(c, f.fl, f.fs, f.ft));
  GSP_TRY(contract(c, 0, f, M, nullptr));
  GSP_TRY(join_solve(c, f, 0));
  GSP_TRY(fork_solve(c, 1));
  GSP_TRY(contract(c, 1, f, M, nullptr));
  GSP_TRY(join_solve(c, f, 1));
  GSP_TRY(fork_solve(c, 2));
  GSP_TRY(run_lst(c, f.fx, f.fy));
  for (int m = 2; m < 5; ++m) {
    if (m > 2) GSP_TRY(fork_solve(c, m));
    GSP_TRY(contract(c, m, f, M, nullptr));
    GSP_TRY(join_solve(c, f, m));
  }
  return GSP_OK;
}

StructWs struct_ws(const Ctx& c) {
  StructWs w;
  w.part = c.at<float>(c.lay.part);
  w.pre = c.at<double>(c.lay.pre);
  w.sig = c.at<float>(c.lay.sig);
  w.sig64 = c.at<double>(c.lay.sig64);
  w.segtot = c.at<double>(c.lay.segtot);
  w.off = c.at<double>(c.lay.off);
  w.stpart = c.at<float>(c.lay.stpart);
  w.lscale = c.at<double>(c.lay.lscale);
  if (c.prec == GSP_PREC_STRUCTURED_GAUSSIAN) {
    w.gw = c.at<float>(c.lay.gw);
    w.conv = c.at<float>(c.lay.conv);
  }
  return w;
}

// Structured operand: the bin map (and its transpose), the level scales and
// ||T||^2; no tensor.
int prepare_structured(const int32_t* d_hist, const float* d_normal_xy, int raw,
                       uint32_t* d_status, const Ctx& c) {
  const MttkrpDims& d = c.d;
  const bool gauss = c.prec == GSP_PREC_STRUCTURED_GAUSSIAN;
  if (gauss && d_hist) return GSP_ERR_INVALID_ARG;  // box histograms hold no Gaussian weights
  uint16_t* bm = c.at<uint16_t>(c.lay.bins);
  uint32_t* groups = reinterpret_cast<uint32_t*>(c.ws + c.lay.bins + d.N2() * sizeof(uint16_t));
  unsigned long long* sumsq = c.at<unsigned long long>(c.lay.sumsq);
  GSP_TRY(struct_level_scales(d.L, d.B, raw, gauss ? 1 : 0, c.at<double>(c.lay.lscale), c.s));
  if (d_hist) {
    const long long slice = d.N2() * d.B2();
    GSP_TRY(struct_bins_from_level0(d_hist, d.N, d.B, bm, d_status, c.s));
    for (int l = 0; l < d.L; ++l) {
      LevelSink o{nullptr, nullptr, nullptr, 1.0f, sumsq + l, 0, 0};
      GSP_TRY(launch_cast(d_hist + slice * l, d.N, d.B, o, c.s));
    }
  } else {
    GSP_TRY(launch_bins(d_normal_xy, d.N, d.B, bm, d_status, groups, c.s));
    if (!gauss) {
      HistOut o{};
      o.sumsq = sumsq;
      o.groups = groups;
      GSP_TRY(launch_box_hist(bm, d.N, d.L, d.B * d.B, o, c.s));
    }
  }
  GSP_TRY(struct_transpose_bins(bm, c.at<uint16_t>(c.lay.binsT), d.N, c.s));
  if (gauss)
    return struct_gauss_prepare(bm, struct_ws(c), d, c.at<double>(c.lay.gw64), c.at<double>(c.lay.K),
                                c.at<int32_t>(c.lay.A), c.at<double>(c.lay.normpart),
                                c.at<double>(c.lay.norm2), c.s);
  k_norm2<<<1, 32, 0, c.s>>>(sumsq, d.L, d.B, raw, c.at<double>(c.lay.norm2));
  GSP_CHECK_LAUNCH();
  return GSP_OK;
}

// One structured sweep, modes x, y, l, s, t.  BE holds beta of f.fy on entry
// and on exit; AL holds alpha of f.fx on exit.
int structured_sweep(const Ctx& c, const gsp_cp_factors& f) {
  const MttkrpDims& d = c.d;
  const StructWs w = struct_ws(c);
  const uint16_t* bm = c.at<uint16_t>(c.lay.bins);
  const uint16_t* bt = c.at<uint16_t>(c.lay.binsT);
  float* al = c.at<float>(c.lay.AL);
  float* be = c.at<float>(c.lay.BE);
  double* M = c.at<double>(c.lay.M);
  GSP_TRY(fork_solve(c, 0));
  GSP_TRY(struct_side(bm, be, f.fs, f.ft, f.fl, w, d, M, nullptr, c.s));
  GSP_TRY(join_solve(c, f, 0));
  GSP_TRY(fork_solve(c, 1));
  GSP_TRY(struct_window_tables(f.fx, al, w, d, c.s));
  GSP_TRY(struct_side(bt, al, f.fs, f.ft, f.fl, w, d, M, nullptr, c.s));
  GSP_TRY(join_solve(c, f, 1));
  GSP_TRY(fork_solve(c, 2));
  GSP_TRY(struct_window_tables(f.fy, be, w, d, c.s));
  GSP_TRY(struct_level(be, w, d, M, nullptr, c.s));
  GSP_TRY(join_solve(c, f, 2));
  GSP_TRY(fork_solve(c, 3));
  GSP_TRY(struct_bins(bm, al, be, f.fl, f.ft, 0, w, d, M, nullptr, c.s));
  GSP_TRY(join_solve(c, f, 3));
  GSP_TRY(fork_solve(c, 4));
  GSP_TRY(struct_bins(bm, al, be, f.fl, f.fs, 1, w, d, M, nullptr, c.s));
  return join_solve(c, f, 4);
}

// Bin map into bm, the occupied bins and the column tables into cols (the
// first two entries of a CP workspace), then {count, Bk, Bt16} read back into
// hc (synchronises s).
int count_columns(const int32_t* d_hist, const float* d_normal_xy, int N, int bins, uint16_t* bm,
                  int32_t* cols, uint32_t* d_status, cudaStream_t s, int32_t* hc) {
  const int B2 = bins * bins;
  uint32_t* occ = reinterpret_cast<uint32_t*>(cols + 4 + 2 * B2);
  if (d_hist)
    GSP_TRY(struct_bins_from_level0(d_hist, N, bins, bm, d_status, s));
  else
    GSP_TRY(launch_bins(d_normal_xy, N, bins, bm, d_status, nullptr, s));
  GSP_CUDA(cudaMemsetAsync(occ, 0, (B2 + 31) / 32 * sizeof(uint32_t), s));
  k_bin_occupancy<<<sm_count() * 2, 256, 0, s>>>(bm, static_cast<long long>(N) * N, B2, occ);
  GSP_CHECK_LAUNCH();
  k_bin_compact<<<1, 512, 0, s>>>(occ, B2, cols);
  GSP_CHECK_LAUNCH();
  GSP_CUDA(cudaMemcpyAsync(hc, cols, 3 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  GSP_CUDA(cudaStreamSynchronize(s));
  return GSP_OK;
}

}  // namespace
}  // namespace gsp

using namespace gsp;

namespace gsp {
namespace {
__global__ void k_selftest_recip(const double* __restrict__ in, long long n, double* __restrict__ out) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i < n) out[i] = recip_newton(in[i]);
}
}  // namespace
}  // namespace gsp

extern "C" int gsp_selftest_recip(const double* d_in, int64_t n, double* d_out, gsp_stream stream) {
  if (n < 0 || (n > 0 && (!d_in || !d_out))) return GSP_ERR_INVALID_ARG;
  if (n == 0) return GSP_OK;
  k_selftest_recip<<<grid_for(n, 256), 256, 0, to_stream(stream)>>>(d_in, n, d_out);
  GSP_CHECK_LAUNCH();
  return GSP_OK;
}

extern "C" size_t gsp_cp_workspace_bytes(int N, int levels, int bins, int rank, int precision) {
  if (!valid_cp(N, levels, bins, rank, precision)) return 0;
  MttkrpDims d{N, levels, bins, rank};
  if (!path_supported(d, precision)) return 0;
  return cp_layout(d, precision).total;
}

extern "C" size_t gsp_cp_workspace_bytes_for_bins(int N, int levels, int bins, int rank,
                                                  int precision, int occupied_bins) {
  if (!valid_cp(N, levels, bins, rank, precision)) return 0;
  MttkrpDims d{N, levels, bins, rank};
  if (!path_supported(d, precision)) return 0;
  if (is_structured(precision)) return cp_layout(d, precision).total;
  const int B2 = bins * bins;
  if (occupied_bins < 1 || occupied_bins > B2) return 0;
  int Bk = 0, Bt = 0;
  cols_for(B2, occupied_bins, precision, &Bk, &Bt);
  d.Bk = Bk;
  d.Bt = Bt;
  return cp_layout(d, precision).total;
}

extern "C" size_t gsp_cp_operand_offset(int N, int levels, int bins, int rank, int precision) {
  if (!valid_cp(N, levels, bins, rank, precision) || is_structured(precision)) return 0;
  return cp_layout(MttkrpDims{N, levels, bins, rank}, precision).T;
}

extern "C" size_t gsp_cp_count_bins_workspace_bytes(int N, int bins) {
  if (!valid_map(N, 1, bins) || N < 8 || bins < 8) return 0;
  return count_ws_bytes(N, bins);
}

extern "C" int gsp_cp_count_bins(const int32_t* d_hist, const float* d_normal_xy, int N,
                                 int levels, int bins, void* d_ws, size_t ws_bytes,
                                 int32_t* h_occupied, uint32_t* d_status, gsp_stream stream) {
  if (!h_occupied || (d_hist == nullptr) == (d_normal_xy == nullptr)) return GSP_ERR_INVALID_ARG;
  if (!valid_map(N, levels, bins) || N < 8 || bins < 8) return GSP_ERR_INVALID_ARG;
  if (!d_ws || ws_bytes < count_ws_bytes(N, bins)) return GSP_ERR_WORKSPACE;
  char* w = static_cast<char*>(d_ws);
  int32_t hc[3] = {0, 0, 0};
  GSP_TRY(count_columns(d_hist, d_normal_xy, N, bins, reinterpret_cast<uint16_t*>(w),
                        reinterpret_cast<int32_t*>(w + align_up(bins_bytes(N), 256)), d_status,
                        to_stream(stream), hc));
  *h_occupied = hc[0];
  return GSP_OK;
}

extern "C" int gsp_cp_prepare(const int32_t* d_hist, const float* d_normal_xy, int N, int levels,
                              int bins, int rank, const gsp_als_opts* opts, void* d_ws,
                              size_t ws_bytes, uint32_t* d_status, gsp_stream stream) {
  if (!opts || (d_hist == nullptr) == (d_normal_xy == nullptr)) return GSP_ERR_INVALID_ARG;
  Ctx c;
  GSP_TRY(make_ctx(N, levels, bins, rank, opts->precision, d_ws, ws_bytes, stream, c));
  const MttkrpDims& d = c.d;
  unsigned long long* sumsq = c.at<unsigned long long>(c.lay.sumsq);
  GSP_CUDA(cudaMemsetAsync(sumsq, 0, sizeof(unsigned long long) * levels, c.s));
  GSP_CUDA(cudaMemsetAsync(c.ws + c.lay.flags, 0, 16, c.s));
  if (is_structured(c.prec)) return prepare_structured(d_hist, d_normal_xy, opts->raw_counts, d_status, c);
  // bin map (dense bins), occupied bins, operand columns
  const int B2 = bins * bins;
  uint16_t* bm = c.at<uint16_t>(c.lay.bins);
  uint32_t* groups = reinterpret_cast<uint32_t*>(c.ws + c.lay.bins + d.N2() * sizeof(uint16_t));
  int32_t* cols = c.at<int32_t>(c.lay.cols);
  int32_t hc[3] = {0, 0, 0};
  GSP_TRY(count_columns(d_hist, d_normal_xy, N, bins, bm, cols, d_status, c.s, hc));
  const int Bk = hc[1], Bt = stored_cols(c.prec, hc[1], hc[2]);
  if (!valid_cols(d, Bk, Bt)) return GSP_ERR_INVALID_ARG;
  GSP_TRY(set_cols(c, Bk, Bt));  // the workspace must hold the operand of these columns
  remember_cols(c.ws, d, c.prec, Bk, Bt);
  const long long slice = d.N2() * Bt;  // operand elements per level (Bt stored columns)
  if (d_hist) {
    for (int l = 0; l < levels; ++l) {
      const float scale =
          opts->raw_counts ? 1.0f : static_cast<float>(bins * bins) / (4.0f * ldexpf(1.0f, 2 * l));
      const int32_t* hl = d_hist + d.N2() * B2 * l;
      if (is_bf16(c.prec))
        k_cast_cols<__nv_bfloat16><<<grid_for(slice, 256), 256, 0, c.s>>>(
            hl, d.N2(), B2, Bt, cols, scale, 0, slice * l, c.at<__nv_bfloat16>(c.lay.T) + slice * l,
            sumsq + l);
      else
        k_cast_cols<float><<<grid_for(slice, 256), 256, 0, c.s>>>(
            hl, d.N2(), B2, Bt, cols, scale, c.prec == GSP_PREC_TF32, slice * l,
            c.at<float>(c.lay.T) + slice * l, sumsq + l);
      GSP_CHECK_LAUNCH();
    }
  } else {
    k_bin_remap<<<grid_for(d.N2(), 256), 256, 0, c.s>>>(bm, d.N2(), cols, B2);
    GSP_CHECK_LAUNCH();
    k_col_groups<<<grid_for(kGroupBytes * 8, 256), 256, 0, c.s>>>(cols, groups);
    GSP_CHECK_LAUNCH();
    HistOut o{};
    o.sumsq = sumsq;
    o.groups = groups;
    for (int l = 0; l < levels; ++l)
      o.scale[l] = opts->raw_counts ? 1.0f : static_cast<float>(bins * bins) / (4.0f * ldexpf(1.0f, 2 * l));
    if (is_bf16(c.prec))
      o.bf16 = c.at<__nv_bfloat16>(c.lay.T);
    else
      o.f32 = c.at<float>(c.lay.T);
    o.tf32 = c.prec == GSP_PREC_TF32;
    // the Y' array is not read before the first sweep: it holds the column
    // prefix scratch of the histogram build when that fits
    const size_t yp_bytes = static_cast<size_t>(N) * N * static_cast<size_t>(d.R) * sizeof(float);
    const size_t cp_bytes = col_prefix_bytes(N, Bt);
    if (cp_bytes > 0 && cp_bytes <= yp_bytes) o.colp = c.at<__half>(c.lay.Yp);
    GSP_TRY(launch_box_hist(bm, N, levels, Bt, o, c.s));
  }
  k_norm2<<<1, 32, 0, c.s>>>(sumsq, levels, bins, opts->raw_counts, c.at<double>(c.lay.norm2));
  GSP_CHECK_LAUNCH();
  return GSP_OK;
}

extern "C" int gsp_cp_operand_cols(int N, int levels, int bins, int rank, int precision,
                                   const void* d_ws, size_t ws_bytes, int32_t* h_cols,
                                   gsp_stream stream) {
  if (!h_cols || is_structured(precision)) return GSP_ERR_INVALID_ARG;
  Ctx c;
  GSP_TRY(make_ctx(N, levels, bins, rank, precision, const_cast<void*>(d_ws), ws_bytes, stream, c));
  int32_t h[3] = {0, 0, 0};
  GSP_CUDA(cudaMemcpyAsync(h, c.ws + c.lay.cols, sizeof(h), cudaMemcpyDeviceToHost, c.s));
  GSP_CUDA(cudaStreamSynchronize(c.s));
  const int Bt = stored_cols(precision, h[1], h[2]);
  if (!valid_cols(c.d, h[1], Bt)) return GSP_ERR_INVALID_ARG;
  h_cols[0] = h[0];
  h_cols[1] = Bt;
  return GSP_OK;
}

extern "C" int gsp_cp_sweeps(int N, int levels, int bins, int rank, const gsp_als_opts* opts,
                             const gsp_cp_factors* f, gsp_als_report* h_report, void* d_ws,
                             size_t ws_bytes, gsp_stream stream) {
  if (!opts || !valid_factors(f) || opts->sweeps < 1 || opts->sweeps > GSP_MAX_SWEEPS ||
      !(opts->tol >= 0.0))
    return GSP_ERR_INVALID_ARG;
  Ctx c;
  GSP_TRY(make_ctx(N, levels, bins, rank, opts->precision, d_ws, ws_bytes, stream, c));
  GSP_TRY(resolve_cols(c));
  SideStream side(c);
  GSP_TRY(side.open());
  double* M = c.at<double>(c.lay.M);
  double* fits = c.at<double>(c.lay.fit);
  GSP_CUDA(cudaMemsetAsync(c.ws + c.lay.flags, 0, 16, c.s));
  for (int m = 0; m < 5; ++m) GSP_TRY(gram(c, *f, m));
  const bool st = is_structured(c.prec);
  if (st) GSP_TRY(struct_window_tables(f->fy, c.at<float>(c.lay.BE), struct_ws(c), c.d, c.s));
  int done = 0;
  double prev = 0.0;
  for (int sweep = 0; sweep < opts->sweeps; ++sweep) {
    GSP_TRY(st ? structured_sweep(c, *f) : dense_sweep(c, *f));
    k_fit<<<1, 256, 0, c.s>>>(M, f->ft, c.at<double>(c.lay.lam), c.at<double>(c.lay.G), bins,
                              rank, c.at<double>(c.lay.norm2), fits + sweep);
    GSP_CHECK_LAUNCH();
    done = sweep + 1;
    if (opts->tol > 0.0) {
      double cur = 0.0;
      GSP_CUDA(cudaMemcpyAsync(&cur, fits + sweep, sizeof(double), cudaMemcpyDeviceToHost, c.s));
      GSP_CUDA(cudaStreamSynchronize(c.s));
      if (sweep > 0 && fabs(cur - prev) < opts->tol) break;
      prev = cur;
    }
  }
  if (h_report) {
    h_report->sweeps_done = done;
    uint32_t flags = 0;
    GSP_CUDA(cudaMemcpyAsync(h_report->fit, fits, sizeof(double) * done, cudaMemcpyDeviceToHost, c.s));
    GSP_CUDA(cudaMemcpyAsync(&flags, c.ws + c.lay.flags, sizeof(uint32_t), cudaMemcpyDeviceToHost, c.s));
    GSP_CUDA(cudaStreamSynchronize(c.s));
    h_report->numeric_fallbacks = (flags & GSP_DEV_NUMERIC) ? 1 : 0;
    if (flags & GSP_DEV_TIMEOUT) return GSP_ERR_TIMEOUT;
  }
  return GSP_OK;
}

extern "C" int gsp_cp_decompose(const int32_t* d_hist, const float* d_normal_xy, int N,
                                int levels, int bins, int rank, const gsp_als_opts* opts,
                                const gsp_cp_factors* f, gsp_als_report* h_report, void* d_ws,
                                size_t ws_bytes, uint32_t* d_status, gsp_stream stream) {
  GSP_TRY(gsp_cp_prepare(d_hist, d_normal_xy, N, levels, bins, rank, opts, d_ws, ws_bytes,
                         d_status, stream));
  return gsp_cp_sweeps(N, levels, bins, rank, opts, f, h_report, d_ws, ws_bytes, stream);
}

extern "C" int gsp_cp_mttkrp(int N, int levels, int bins, int rank, int precision,
                             const gsp_cp_factors* f, float* const d_m[5], void* d_ws,
                             size_t ws_bytes, gsp_stream stream) {
  if (!f || !f->fx || !f->fy || !f->fl || !f->fs || !f->ft || !d_m) return GSP_ERR_INVALID_ARG;
  for (int m = 0; m < 5; ++m)
    if (!d_m[m]) return GSP_ERR_INVALID_ARG;
  Ctx c;
  GSP_TRY(make_ctx(N, levels, bins, rank, precision, d_ws, ws_bytes, stream, c));
  GSP_TRY(resolve_cols(c));
  if (is_structured(precision)) {
    const StructWs w = struct_ws(c);
    const uint16_t* bm = c.at<uint16_t>(c.lay.bins);
    float* al = c.at<float>(c.lay.AL);
    float* be = c.at<float>(c.lay.BE);
    double* M = c.at<double>(c.lay.M);
    GSP_TRY(struct_window_tables(f->fx, al, w, c.d, c.s));
    GSP_TRY(struct_window_tables(f->fy, be, w, c.d, c.s));
    GSP_TRY(struct_side(bm, be, f->fs, f->ft, f->fl, w, c.d, M, d_m[0], c.s));
    GSP_TRY(struct_side(c.at<uint16_t>(c.lay.binsT), al, f->fs, f->ft, f->fl, w, c.d, M, d_m[1], c.s));
    GSP_TRY(struct_level(be, w, c.d, M, d_m[2], c.s));
    GSP_TRY(struct_bins(bm, al, be, f->fl, f->ft, 0, w, c.d, M, d_m[3], c.s));
    return struct_bins(bm, al, be, f->fl, f->fs, 1, w, c.d, M, d_m[4], c.s);
  }
  GSP_TRY(run_xy(c, f->fl, f->fs, f->ft));
  GSP_TRY(contract(c, 0, *f, nullptr, d_m[0]));
  GSP_TRY(contract(c, 1, *f, nullptr, d_m[1]));
  GSP_TRY(run_lst(c, f->fx, f->fy));
  for (int m = 2; m < 5; ++m) GSP_TRY(contract(c, m, *f, nullptr, d_m[m]));
  return GSP_OK;
}
