// Structured MTTKRP of the footprint NDF tensor: exact, from the bin map, never
// materialising the tensor.
//
// Every level slice of the tensor is a box sum of the texel -> bin one-hot
// (Sec. 4.1): T[x, y, l, s, t] = c_l * #{u in W_l(x, y) : bin(u) = (s, t)} with
// c_l = B^2 / (4 * 4^l) (1 for raw counts) and W_l(x, y) the 2^l x 2^l window
// at offset a_l = floor(2^l / 2), wrapping.  Texel u lies in the window of
// column x exactly when x = u + a_l - i (mod N) for an i < 2^l, so contracting
// T with a spatial factor moves the window onto the factor:
//   alpha_l(u, r) = sum_{i < 2^l} fx[(u + a_l - i) mod N][r]      (beta_l: fy).
// With h(u, r) = fs[s_u][r] ft[t_u][r] the five MTTKRPs of a CP-ALS sweep
// (Sec. 4.2, Eq. 3) become
//   x: rho_l(u_x, r) = sum_{u_y} h(u, r) beta_l(u_y, r)           (side pass)
//      M_x[x, r] = sum_l c_l fl[l][r] sum_{i < 2^l} rho_l((x - a_l + i) mod N, r)
//   y: the same with x and y exchanged: sigma_l(u_y, r) from alpha_l
//   l: M_l[l, r] = c_l sum_{u_y} beta_l(u_y, r) sigma_l(u_y, r)
//   s: M_s[s, r] = sum_{u : s_u = s} ft[t_u][r] P(u, r)             (bin pass)
//      P(u, r) = sum_l c_l fl[l][r] alpha_l(u_x, r) beta_l(u_y, r)
//   t: M_t[t, r] = sum_{u : t_u = t} fs[s_u][r] P(u, r)
// O(N^2 L R) multiply-adds per mode instead of O(N^2 L B^2 R) over the dense
// tensor; at 1024^2 texels, 11 levels, 32^2 bins and rank 64 that is a
// 1024-fold reduction, and the workspace shrinks from the tensor (23.6 GB in
// BF16) to tens of MB.
//
// Kernels (FP32 products on the CUDA cores, FP64 wherever sums get long):
//   k_window_tables  alpha / beta from an FP64 cyclic prefix sum of the factor
//   k_side_pass<L>   rho or sigma: a thread owns one rank and 8 columns and keeps
//                    8 x L FP32 accumulators over a split of the rows; partials
//                    per row split
//   k_side_reduce / _offsets / _fix
//                    sum over row splits (compensated FP32), FP64 prefix along
//                    the columns in 32-row segments, then the segment offsets
//   k_side_window    M_x / M_y: footprint windows as prefix differences, FP64
//   k_level_mode     M_l from sigma and beta (compensated FP32, FP64 at the end)
//   k_bin_pass<L>    P recomputed per texel from alpha (registers) and beta, then
//                    added into warp-private [B][rank] tables in shared memory
//                    (plain read-modify-write: a lane owns its rank's column);
//                    per-CTA partials
//   k_bin_reduce     sum of the per-CTA partials in a fixed order (compensated)
// Every sum has a fixed order, so results are bit-reproducible.
#include <algorithm>

#include "mttkrp.cuh"

namespace gsp {
namespace {

constexpr int kSC = 8;        // columns per thread (one 16-byte load of bins)
constexpr int kSW = 4;        // warps per CTA of the side and bin passes
constexpr int kSideTargetCtas = 912;  // six CTAs on each of 152 SMs
constexpr int kMaxLevels = 11;        // maps up to 1024^2

__host__ __device__ inline int rank_lanes(int R) { return R < 32 ? R : 32; }
__device__ __forceinline__ int ilog2_dev(int v) { return 31 - __clz(v); }

// out[u][l][r] = sum_{i < 2^l} f[(u + a_l - i) mod N][r].  One CTA per (8 ranks,
// level): warp w scans rank r0 + w into an FP64 prefix P[k] = sum_{j < k} f[j]
// (lane-sequential chunks, then a warp scan of the chunk totals); every window
// is then a difference of two (three when it wraps) prefix values.
constexpr int kWinRanks = 8;
__global__ void __launch_bounds__(256) k_window_tables(const float* __restrict__ f, int N, int L,
                                                       int R, float* __restrict__ out) {
  extern __shared__ double pre[];  // [N + 1][kWinRanks]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = blockIdx.x * kWinRanks;
  const int r = r0 + warp;
  const int chunk = (N + 31) / 32;
  const int k0 = lane * chunk, k1 = min(N, k0 + chunk);
  double run = 0.0;
  for (int k = k0; k < k1; ++k) run += static_cast<double>(f[static_cast<size_t>(k) * R + r]);
  double incl = run;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const double v = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += v;
  }
  double acc = incl - run;  // exclusive prefix of this lane's chunk
  for (int k = k0; k < k1; ++k) {
    acc += static_cast<double>(f[static_cast<size_t>(k) * R + r]);
    pre[(k + 1) * kWinRanks + warp] = acc;
  }
  if (lane == 0) pre[warp] = 0.0;
  __syncthreads();
  const int l = blockIdx.y, w = 1 << l, a = w >> 1;
  for (int e = threadIdx.x; e < N * kWinRanks; e += blockDim.x) {
    const int rr = e & (kWinRanks - 1), u = e / kWinRanks;
    const int start = (u + a - w + 1 + N) & (N - 1);
    double v;
    if (start + w <= N)
      v = pre[(start + w) * kWinRanks + rr] - pre[start * kWinRanks + rr];
    else
      v = pre[N * kWinRanks + rr] - pre[start * kWinRanks + rr] + pre[(start + w - N) * kWinRanks + rr];
    out[(static_cast<size_t>(u) * L + l) * R + r0 + rr] = static_cast<float>(v);
  }
}

// Compensated FP32 summation (Knuth's TwoSum): hi + lo carries the running sum
// to about twice FP32 precision, so long sums need no FP64 arithmetic (GB300's
// FP64 rate is a small fraction of its FP32 rate).
__device__ __forceinline__ void sum2_add(float& hi, float& lo, float x) {
  const float t = hi + x;
  const float bp = t - hi;
  lo += (hi - (t - bp)) + (x - bp);
  hi = t;
}

// Eight bins (uint16 s * B + t) of one 16-byte load.
__device__ __forceinline__ int bin_of(const uint4& q, int c) {
  const uint32_t w = c < 2 ? q.x : c < 4 ? q.y : c < 6 ? q.z : q.w;
  return static_cast<int>((w >> (16 * (c & 1))) & 0xffffu);
}

// Rows of a side or bin pass staged in shared memory: the window-table rows
// [row][l][RL] of the CTA's rank chunk and the CTA's columns of the bin map,
// copied with cp.async (global -> shared without a register round trip, every
// thread's 16-byte pieces in flight at once) into one of two buffers while the
// other one is consumed.
constexpr int kChunkRows = 16;

__host__ __device__ inline int cta_cols(int R) { return kSW * (32 / rank_lanes(R)) * kSC; }

__device__ __forceinline__ void cp_async16(void* dst, const void* src, int bytes) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int Pending>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(Pending) : "memory");
}

// Issue the copies of rows [u, u + n) (ranks rbase .. rbase + RL - 1 of table
// [N][L][R]; bin-map columns [cbase, cbase + ncols), zero past column N).
// lrl = log2(RL / 4): 16-byte pieces per (row, level) segment.
template <int L>
__device__ __forceinline__ void stage_rows(const float* __restrict__ tab,
                                           const uint16_t* __restrict__ bm, int N, int R, int lrl,
                                           int rbase, int u, int n, int cbase, int ncols,
                                           float* __restrict__ ws, uint16_t* __restrict__ bs) {
  const int pieces = (n * L) << lrl;
  for (int i = threadIdx.x; i < pieces; i += blockDim.x) {
    const int seg = i >> lrl, k4 = (i - (seg << lrl)) * 4;
    const int row = seg / L, l = seg - row * L;  // L is a compile-time constant
    cp_async16(ws + (seg << (lrl + 2)) + k4,
               tab + (static_cast<size_t>(u + row) * L + l) * R + rbase + k4, 16);
  }
  const int q = ncols >> 3;  // 16-byte pieces per row of the bin map
  for (int i = threadIdx.x; i < n * q; i += blockDim.x) {
    const int row = i / q, col = cbase + (i - row * q) * 8;
    const bool in = col < N;
    cp_async16(bs + i * 8, in ? bm + static_cast<size_t>(u + row) * N + col : bm, in ? 16 : 0);
  }
  cp_async_commit();
}

// part[split][col][l][r] = sum over the split's rows u of h(u, col, r) * win[u][l][r]
// with bm[u][col] the bin of (row u, column col).  blockIdx: x column block,
// y row split, z rank chunk of min(R, 32) ranks.  Lane = (sub, rank): the
// 32 / RL sub-groups of a warp take consecutive 8-column groups.
template <int L>
__global__ void __launch_bounds__(kSW * 32, 3) k_side_pass(const uint16_t* __restrict__ bm,
                                                        const float* __restrict__ win,
                                                        const float* __restrict__ fs,
                                                        const float* __restrict__ ft, int N,
                                                        int logB, int R, int rows_per_split,
                                                        float* __restrict__ part) {
  extern __shared__ float sm[];  // fs [B][RL], ft [B][RL], two row buffers, two bin buffers
  const int B = 1 << logB;
  const int RL = rank_lanes(R), G = 32 / RL;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rr = lane % RL, sub = lane / RL;
  const int rbase = blockIdx.z * RL;
  const int r = rbase + rr;
  const int ncols = cta_cols(R);
  const int lrl = ilog2_dev(RL) - 2;
  const int wrows = kChunkRows * L * RL;        // floats per staged buffer
  float* ws = sm + 2 * B * RL;                  // [2][kChunkRows][L][RL]
  uint16_t* bs = reinterpret_cast<uint16_t*>(ws + 2 * wrows);  // [2][kChunkRows][ncols]
  for (int i = threadIdx.x; i < B * RL; i += blockDim.x) {
    const int b = i / RL, k = i - b * RL;
    sm[i] = fs[b * R + rbase + k];
    sm[B * RL + i] = ft[b * R + rbase + k];
  }
  const int cbase = blockIdx.x * ncols;
  const int cl = (warp * G + sub) * kSC;  // first of my columns within the CTA's
  const int col0 = cbase + cl;
  const bool active = col0 < N;
  const int u0 = blockIdx.y * rows_per_split;
  const int u1 = min(N, u0 + rows_per_split);
  const float* fsr = sm + rr;
  const float* ftr = sm + B * RL + rr;
  float acc[kSC][L];
#pragma unroll
  for (int c = 0; c < kSC; ++c)
#pragma unroll
    for (int l = 0; l < L; ++l) acc[c][l] = 0.0f;
  if (u0 < u1) stage_rows<L>(win, bm, N, R, lrl, rbase, u0, min(kChunkRows, u1 - u0), cbase, ncols, ws, bs);
  int buf = 0;
  for (int cu = u0; cu < u1; cu += kChunkRows, buf ^= 1) {
    const int n = min(kChunkRows, u1 - cu);
    const int nx = cu + kChunkRows;
    __syncthreads();  // buffer buf ^ 1 is no longer read
    if (nx < u1) {
      stage_rows<L>(win, bm, N, R, lrl, rbase, nx, min(kChunkRows, u1 - nx), cbase, ncols,
                    ws + (buf ^ 1) * wrows, bs + (buf ^ 1) * kChunkRows * ncols);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();  // buffer buf complete for every thread
    const float* wb = ws + buf * wrows;
    const uint16_t* bb = bs + buf * kChunkRows * ncols;
    if (active) {
      for (int row = 0; row < n; ++row) {
        const uint4 q = reinterpret_cast<const uint4*>(bb + row * ncols + cl)[0];
        float wc[L];
#pragma unroll
        for (int l = 0; l < L; ++l) wc[l] = wb[(row * L + l) * RL + rr];
#pragma unroll
        for (int c = 0; c < kSC; ++c) {
          const int b = bin_of(q, c);
          const float h = fsr[(b >> logB) * RL] * ftr[(b & (B - 1)) * RL];
#pragma unroll
          for (int l = 0; l < L; ++l) acc[c][l] = fmaf(h, wc[l], acc[c][l]);
        }
      }
    }
  }
  if (!active) return;
  float* dst = part + (static_cast<size_t>(blockIdx.y) * N + col0) * L * R + r;
#pragma unroll
  for (int c = 0; c < kSC; ++c)
#pragma unroll
    for (int l = 0; l < L; ++l) dst[(static_cast<size_t>(c) * L + l) * R] = acc[c][l];
}

// Row-split reduction and prefix, in three steps so that every step spreads
// over the whole GPU.  With sigma(u, l, r) = sum_split part[split][u][l][r]:
//   k_side_reduce   sigma (compensated FP32, one thread per element) -> sig
//                   [N][L][R] in FP32 and FP64
//   k_side_segments the FP64 prefix of sigma inside u's 32-row segment ->
//                   pre[l][u + 1][r], the segment totals -> segtot[l][seg][r]
//   k_side_offsets  off[l][seg][r] = sum of the earlier segments' totals
//   k_side_fix      pre[l][k][r] += off[l][(k - 1) / 32][r]; pre[l][0][r] = 0
// after which pre[l][k][r] = sum_{u < k} sigma(u, l, r), FP64.
constexpr int kSeg = 32;
__host__ __device__ inline int seg_count(int N) { return (N + kSeg - 1) / kSeg; }

__global__ void __launch_bounds__(256) k_side_reduce(const float* __restrict__ part, int S,
                                                     long long n, float* __restrict__ sig,
                                                     double* __restrict__ sig64) {
  const long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (idx >= n) return;
  float hi = 0.0f, lo = 0.0f;
  for (int sp = 0; sp < S; ++sp) sum2_add(hi, lo, part[idx + sp * n]);
  const double v = static_cast<double>(hi) + static_cast<double>(lo);
  sig[idx] = static_cast<float>(v);
  sig64[idx] = v;
}

// FP64 prefix of sigma inside each 32-row segment: a warp per (segment, level,
// 32-rank chunk), lanes = ranks.
__global__ void __launch_bounds__(256) k_side_segments(const double* __restrict__ sig64, int N,
                                                       int L, int R, double* __restrict__ pre,
                                                       double* __restrict__ segtot) {
  const long long gw = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int nseg = seg_count(N), chunks = (R + 31) / 32;
  if (gw >= static_cast<long long>(nseg) * L * chunks) return;
  const int ch = static_cast<int>(gw % chunks);
  const int l = static_cast<int>((gw / chunks) % L);
  const int seg = static_cast<int>(gw / (static_cast<long long>(chunks) * L));
  const int r = ch * 32 + lane;
  if (r >= R) return;
  const int u0 = seg * kSeg, u1 = min(N, u0 + kSeg);
  double run = 0.0;
  for (int u = u0; u < u1; ++u) {
    run += sig64[(static_cast<size_t>(u) * L + l) * R + r];
    pre[(static_cast<size_t>(l) * (N + 1) + u + 1) * R + r] = run;
  }
  segtot[(static_cast<size_t>(l) * nseg + seg) * R + r] = run;
}

__global__ void k_side_offsets(const double* __restrict__ segtot, int N, int L, int R,
                               double* __restrict__ off) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= L * R) return;
  const int l = e / R, r = e % R, nseg = seg_count(N);
  double acc = 0.0;
  for (int sg = 0; sg < nseg; ++sg) {
    off[(static_cast<size_t>(l) * nseg + sg) * R + r] = acc;
    acc += segtot[(static_cast<size_t>(l) * nseg + sg) * R + r];
  }
}

__global__ void k_side_fix(const double* __restrict__ off, int N, int L, int R,
                           double* __restrict__ pre) {
  const long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (e >= static_cast<long long>(L) * (N + 1) * R) return;
  const int r = static_cast<int>(e % R);
  const long long lk = e / R;
  const int k = static_cast<int>(lk % (N + 1)), l = static_cast<int>(lk / (N + 1));
  if (k == 0)
    pre[e] = 0.0;
  else
    pre[e] += off[(static_cast<size_t>(l) * seg_count(N) + (k - 1) / kSeg) * R + r];
}

// M[x][r] = sum_l c_l fl[l][r] * (sum of the level's prefix over the footprint
// window of x: columns (x - a_l + i) mod N, i < 2^l), FP64.
__global__ void k_side_window(const double* __restrict__ pre, const float* __restrict__ fl, int N,
                              int L, int R, const double* __restrict__ lscale,
                              double* __restrict__ M, float* __restrict__ Mf) {
  const long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (e >= static_cast<long long>(N) * R) return;
  const int x = static_cast<int>(e / R), r = static_cast<int>(e % R);
  double acc = 0.0;
  for (int l = 0; l < L; ++l) {
    const int w = 1 << l, a = w >> 1;
    const int start = (x - a + N) & (N - 1);
    const double* P = pre + static_cast<size_t>(l) * (N + 1) * R + r;
    double win;
    if (start + w <= N)
      win = P[static_cast<size_t>(start + w) * R] - P[static_cast<size_t>(start) * R];
    else
      win = P[static_cast<size_t>(N) * R] - P[static_cast<size_t>(start) * R] +
            P[static_cast<size_t>(start + w - N) * R];
    acc += lscale[l] * static_cast<double>(fl[l * R + r]) * win;
  }
  M[e] = acc;
  if (Mf) Mf[e] = static_cast<float>(acc);
}

// M[l][r] = c_l sum_u be[u][l][r] * sig[u][l][r] (sigma of the y side pass).
// One CTA per (level, 32-rank chunk); warp w sums rows w, w + 32, ... with
// compensated FP32, the warps' sums are added in FP64 in a fixed order.
__global__ void __launch_bounds__(1024) k_level_mode(const float* __restrict__ sig,
                                                     const float* __restrict__ be, int N, int L,
                                                     int R, const double* __restrict__ lscale,
                                                     double* __restrict__ M, float* __restrict__ Mf) {
  __shared__ double red[32][32];
  const int l = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = blockIdx.y * 32 + lane;
  float hi = 0.0f, lo = 0.0f;
  if (r < R) {
    for (int u = warp; u < N; u += 32) {
      const size_t idx = (static_cast<size_t>(u) * L + l) * R + r;
      sum2_add(hi, lo, be[idx] * sig[idx]);
    }
  }
  red[warp][lane] = static_cast<double>(hi) + static_cast<double>(lo);
  __syncthreads();
  if (warp != 0 || r >= R) return;
  double sacc = 0.0;
  for (int w = 0; w < 32; ++w) sacc += red[w][lane];
  M[l * R + r] = lscale[l] * sacc;
  if (Mf) Mf[l * R + r] = static_cast<float>(lscale[l] * sacc);
}

// Bin pass of mode s (mode_t = 0: key s, multiplier ft[t]) or t (mode_t = 1: key
// t, multiplier fs[s]).  A thread holds alpha of its 8 columns for all levels
// in registers; per staged row wv_l = c_l fl[l][r] beta_l(u_y, r), so
// P = sum_l alpha_l wv_l per texel, and mult * P is added into the thread's
// private [B] column of its warp's table in shared memory.  stpart[cta][key][r]
// gets the CTA's table sum.
template <int L>
__global__ void __launch_bounds__(kSW * 32) k_bin_pass(const uint16_t* __restrict__ bm,
                                                       const float* __restrict__ al,
                                                       const float* __restrict__ be,
                                                       const float* __restrict__ fl,
                                                       const float* __restrict__ tab, int N,
                                                       int logB, int R,
                                                       const double* __restrict__ lscale, int mode_t,
                                                       int rows_per_split,
                                                       float* __restrict__ stpart) {
  // tab [B][RL]; private tables [kSW * G][B][RL]; two row buffers; two bin buffers
  extern __shared__ float sm[];
  const int B = 1 << logB;
  const int RL = rank_lanes(R), G = 32 / RL;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rr = lane % RL, sub = lane / RL;
  const int rbase = blockIdx.z * RL;
  const int r = rbase + rr;
  const int ncols = cta_cols(R);
  const int lrl = ilog2_dev(RL) - 2;
  const int wrows = kChunkRows * L * RL;
  float* priv = sm + B * RL;
  float* ws = priv + kSW * 32 * B;              // [2][kChunkRows][L][RL]
  uint16_t* bs = reinterpret_cast<uint16_t*>(ws + 2 * wrows);
  for (int i = threadIdx.x; i < B * RL; i += blockDim.x) {
    const int b = i / RL, k = i - b * RL;
    sm[i] = tab[b * R + rbase + k];
  }
  for (int i = threadIdx.x; i < kSW * 32 * B; i += blockDim.x) priv[i] = 0.0f;
  const int cbase = blockIdx.x * ncols;
  const int cl = (warp * G + sub) * kSC;
  const int col0 = cbase + cl;
  const bool active = col0 < N;
  float* mine = priv + (warp * G + sub) * B * RL + rr;
  const float* tabr = sm + rr;
  float alpha[kSC][L], cf[L];
#pragma unroll
  for (int c = 0; c < kSC; ++c)
#pragma unroll
    for (int l = 0; l < L; ++l)
      alpha[c][l] = active ? __ldg(al + (static_cast<size_t>(col0 + c) * L + l) * R + r) : 0.0f;
#pragma unroll
  for (int l = 0; l < L; ++l) cf[l] = static_cast<float>(lscale[l]) * __ldg(fl + l * R + r);
  const int u0 = blockIdx.y * rows_per_split;
  const int u1 = min(N, u0 + rows_per_split);
  if (u0 < u1) stage_rows<L>(be, bm, N, R, lrl, rbase, u0, min(kChunkRows, u1 - u0), cbase, ncols, ws, bs);
  int buf = 0;
  for (int cu = u0; cu < u1; cu += kChunkRows, buf ^= 1) {
    const int n = min(kChunkRows, u1 - cu);
    const int nx = cu + kChunkRows;
    __syncthreads();  // buffer buf ^ 1 is no longer read (first time: tables staged)
    if (nx < u1) {
      stage_rows<L>(be, bm, N, R, lrl, rbase, nx, min(kChunkRows, u1 - nx), cbase, ncols,
                    ws + (buf ^ 1) * wrows, bs + (buf ^ 1) * kChunkRows * ncols);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const float* wb = ws + buf * wrows;
    const uint16_t* bb = bs + buf * kChunkRows * ncols;
    if (active) {
      for (int row = 0; row < n; ++row) {
        const uint4 q = reinterpret_cast<const uint4*>(bb + row * ncols + cl)[0];
        float wv[L];
#pragma unroll
        for (int l = 0; l < L; ++l) wv[l] = cf[l] * wb[(row * L + l) * RL + rr];
#pragma unroll
        for (int c = 0; c < kSC; ++c) {
          float p = 0.0f;
#pragma unroll
          for (int l = 0; l < L; ++l) p = fmaf(alpha[c][l], wv[l], p);
          const int b = bin_of(q, c);
          const int hi = b >> logB, lo = b & (B - 1);
          const int key = mode_t ? lo : hi, oth = mode_t ? hi : lo;
          mine[key * RL] = fmaf(tabr[oth * RL], p, mine[key * RL]);
        }
      }
    }
  }
  __syncthreads();
  const size_t cta = static_cast<size_t>(blockIdx.y) * gridDim.x + blockIdx.x;
  const int nt = kSW * G;
  for (int i = threadIdx.x; i < B * RL; i += blockDim.x) {
    float acc = 0.0f;
    for (int t = 0; t < nt; ++t) acc += priv[t * B * RL + i];
    const int key = i / RL, k = i - key * RL;
    stpart[(cta * B + key) * R + rbase + k] = acc;
  }
}

// M[key][r] = sum_cta stpart[cta][key][r] in a fixed order.  One CTA per (key,
// 32-rank chunk); warp w sums ctas w, w + 8, ... with compensated FP32, the
// warps' sums are added in FP64.
__global__ void __launch_bounds__(256) k_bin_reduce(const float* __restrict__ stpart, int ctas,
                                                    int B, int R, double* __restrict__ M,
                                                    float* __restrict__ Mf) {
  __shared__ double red[8][32];
  const int key = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = blockIdx.y * 32 + lane;
  float hi = 0.0f, lo = 0.0f;
  if (r < R)
    for (int c = warp; c < ctas; c += 8)
      sum2_add(hi, lo, stpart[(static_cast<size_t>(c) * B + key) * R + r]);
  red[warp][lane] = static_cast<double>(hi) + static_cast<double>(lo);
  __syncthreads();
  if (warp != 0 || r >= R) return;
  double s = 0.0;
  for (int w = 0; w < 8; ++w) s += red[w][lane];
  M[key * R + r] = s;
  if (Mf) Mf[key * R + r] = static_cast<float>(s);
}

// lscale[l] = B^2 / (4 * 4^l), the counts -> NDF density factor of level l
// (Eq. 2 normalises the footprint; a bin covers (2/B)^2), or 1 for raw counts
// (box counts; a Gaussian footprint's weights already sum to 1: B^2 / 4)
__global__ void k_level_scales(int L, int B, int raw, int gauss, double* __restrict__ lscale) {
  const int l = threadIdx.x;
  if (l < L)
    lscale[l] = raw ? 1.0 : static_cast<double>(B) * B / (4.0 * (gauss ? 1.0 : ldexp(1.0, 2 * l)));
}

// bins_t[x][y] = bins[y][x]
__global__ void k_transpose_bins(const uint16_t* __restrict__ in, int N, uint16_t* __restrict__ out) {
  __shared__ uint16_t tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int y = by + j, x = bx + threadIdx.x;
    if (y < N && x < N) tile[j][threadIdx.x] = in[static_cast<size_t>(y) * N + x];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int x = bx + j, y = by + threadIdx.x;
    if (y < N && x < N) out[static_cast<size_t>(x) * N + y] = tile[threadIdx.x][j];
  }
}

// bins[u] = the bin of texel u from the level-0 histogram slice (one count of 1
// per texel); a texel whose slice is not a single 1 keeps bin 0 and sets
// GSP_DEV_BAD_QUERY in status.  One warp per texel.
__global__ void k_bins_from_level0(const int32_t* __restrict__ h0, int N, int B2,
                                   uint16_t* __restrict__ bins, uint32_t* status) {
  const long long u = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (u >= static_cast<long long>(N) * N) return;
  const int32_t* p = h0 + u * B2;
  int ones = 0, found = -1, bad = 0;
  for (int b = lane; b < B2; b += 32) {
    const int v = p[b];
    if (v == 1) {
      ++ones;
      found = b;
    } else if (v != 0) {
      bad = 1;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) ones += __shfl_xor_sync(0xffffffffu, ones, off);
  bad = __any_sync(0xffffffffu, bad) || ones != 1;
  const unsigned m = __ballot_sync(0xffffffffu, found >= 0);
  const int b = __shfl_sync(0xffffffffu, found, m ? __ffs(m) - 1 : 0);
  if (lane == 0) {
    bins[u] = static_cast<uint16_t>(bad ? 0 : b);
    if (bad) set_status(status, GSP_DEV_BAD_QUERY);
  }
}

// ------------------------------------------------ Gaussian footprints --
// Eq. geom weighs the footprint's texels by a Gaussian G_p instead of a box.
// Level l here: a separable Gaussian of sigma_l = 1.5 * 2^l / sqrt(12) (the
// paper's 1.5 s / sqrt(12) with the box width 2^l as the stride s), truncated
// to |d| <= rho_l = min(ceil(3 sigma_l), (N - 1) / 2) (never overlapping itself
// on the periodic map) and normalised to sum 1.  The structured MTTKRPs keep
// their form with the weights g_l(u - x) in place of the box indicator: the
// window tables and the mode-x / mode-y window step become Gaussian-weighted
// sums over the support (k_gauss_conv), and T = B^2/4 times the weight sums.

__host__ __device__ inline double gauss_sigma(int l) { return 1.5 * ldexp(1.0, l) / sqrt(12.0); }
__host__ __device__ inline int gauss_radius(int l, int N) {
  const int r = static_cast<int>(ceil(3.0 * gauss_sigma(l)));
  const int m = (N - 1) / 2;
  return r < m ? r : m;
}

// gw[l][d mod N] (FP32) and gw64 (FP64): one CTA per level, the normalising sum
// in a fixed order.
__global__ void __launch_bounds__(256) k_gauss_weights(int N, float* __restrict__ gw,
                                                       double* __restrict__ gw64) {
  __shared__ double red[256];
  const int l = blockIdx.x;
  const double sig = gauss_sigma(l);
  const int rho = gauss_radius(l, N);
  double part = 0.0;
  for (int d = -rho + static_cast<int>(threadIdx.x); d <= rho; d += blockDim.x)
    part += exp(-static_cast<double>(d) * d / (2.0 * sig * sig));
  red[threadIdx.x] = part;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const double z = red[0];
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int d = i <= N / 2 ? i : i - N;  // the cyclic offset of slot i
    const double v = (d >= -rho && d <= rho) ? exp(-static_cast<double>(d) * d / (2.0 * sig * sig)) / z : 0.0;
    gw64[static_cast<size_t>(l) * N + i] = v;
    gw[static_cast<size_t>(l) * N + i] = static_cast<float>(v);
  }
}

// out[u][l][r] = sum_{|d| <= rho_l} g_l(d) src[(u - d) mod N] (level l's slice of
// src when lstride = 1, else the level-independent src [N][R]), compensated
// FP32.  CTA: 64 outputs u x (up to) 32 ranks of one level; the 64 + 2 rho rows
// it reads and the weights staged in shared memory.
constexpr int kConvRows = 64;
__global__ void __launch_bounds__(256) k_gauss_conv(const float* __restrict__ src, int lstride,
                                                    const float* __restrict__ gw, int N, int L,
                                                    int R, float* __restrict__ out) {
  extern __shared__ float cs[];  // weights [2 rho + 1], rows [kConvRows + 2 rho][RL]
  const int l = blockIdx.y;
  const int RL = rank_lanes(R);
  const int rbase = blockIdx.z * RL;
  const int rho = gauss_radius(l, N);
  const int u0 = blockIdx.x * kConvRows;
  const int nw = 2 * rho + 1;
  const int nrows = kConvRows + 2 * rho;
  float* wts = cs;
  float* rows = cs + ((nw + 3) & ~3);
  for (int i = threadIdx.x; i < nw; i += blockDim.x)
    wts[i] = gw[static_cast<size_t>(l) * N + ((i - rho + N) % N)];
  const size_t rs = lstride ? static_cast<size_t>(L) * R : static_cast<size_t>(R);
  const size_t lo = lstride ? static_cast<size_t>(l) * R : 0;
  for (int i = threadIdx.x; i < nrows * RL; i += blockDim.x) {
    const int j = i / RL, k = i - j * RL;
    const int u = ((u0 - rho + j) % N + N) % N;
    rows[i] = src[u * rs + lo + rbase + k];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kConvRows * RL; i += blockDim.x) {
    const int iu = i / RL, k = i - iu * RL;
    if (u0 + iu >= N) continue;
    float hi = 0.0f, lo2 = 0.0f;
    // output u0 + iu reads rows j = iu + rho - d, d = -rho .. rho
    for (int t = 0; t < nw; ++t) sum2_add(hi, lo2, wts[t] * rows[(iu + 2 * rho - t) * RL + k]);
    out[(static_cast<size_t>(u0 + iu) * L + l) * R + rbase + k] = hi + lo2;
  }
}

// M[x][r] = sum_l c_l fl[l][r] conv[x][l][r], FP64.
__global__ void k_level_combine(const float* __restrict__ conv, const float* __restrict__ fl, int N,
                                int L, int R, const double* __restrict__ lscale,
                                double* __restrict__ M, float* __restrict__ Mf) {
  const long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (e >= static_cast<long long>(N) * R) return;
  const int x = static_cast<int>(e / R), r = static_cast<int>(e % R);
  double acc = 0.0;
  for (int l = 0; l < L; ++l)
    acc += lscale[l] * static_cast<double>(fl[l * R + r]) *
           static_cast<double>(conv[(static_cast<size_t>(x) * L + l) * R + r]);
  M[e] = acc;
  if (Mf) Mf[e] = static_cast<float>(acc);
}

// A[ey][ex] = #{u : bin(u) = bin(u + (ex, ey))} (cyclic): the same-bin
// autocorrelation of the map.  The sum of squared Gaussian footprint weights of
// a level is sum_e K(ex) K(ey) A[ey][ex] with K the weights' autocorrelation
// (the texel pairs of a bin weighed by how much a footprint covers both).  One
// CTA per ey; warp w takes rows y = w, w + 8, ...: the row y + ey is staged
// twice (as is and shifted by one bin) so that every lane reads its two
// neighbouring shifts ex = 2j, 2j + 1 as one aligned 32-bit word and compares
// both with one SIMD 16-bit compare; matches are counted in 16-bit halves and
// flushed to 32 bits every 32 rows.
constexpr int kAcWarps = 8;
constexpr int kAcPairs = 16;  // 32-bit words (bin pairs) per lane: N <= 1024
__global__ void __launch_bounds__(kAcWarps * 32) k_match_autocorr(const uint16_t* __restrict__ bm,
                                                                  int N, int32_t* __restrict__ A) {
  extern __shared__ uint16_t acs[];  // per warp: row y [N], shifted rows R0, R1 [N + 64]; then red
  const int ey = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int P = (N + 63) / 64;  // words per lane
  const int span = N + 64 * P;  // a lane reads up to element ux + 2 (32 P - 1) + 1
  uint16_t* ry = acs + warp * (N + 2 * span);
  uint16_t* r0 = ry + N;
  uint16_t* r1 = r0 + span;
  uint32_t packed[kAcPairs];
  uint32_t cnt[2 * kAcPairs];
#pragma unroll
  for (int k = 0; k < kAcPairs; ++k) packed[k] = 0u;
#pragma unroll
  for (int k = 0; k < 2 * kAcPairs; ++k) cnt[k] = 0u;
  int rows_since = 0;
  for (int y = warp; y < N; y += kAcWarps) {
    const int ys = (y + ey) & (N - 1);
    for (int i = lane; i < N; i += 32) ry[i] = bm[static_cast<size_t>(y) * N + i];
    for (int i = lane; i < span; i += 32) {
      r0[i] = bm[static_cast<size_t>(ys) * N + (i & (N - 1))];
      r1[i] = bm[static_cast<size_t>(ys) * N + ((i + 1) & (N - 1))];
    }
    __syncwarp();
    const uint32_t* w0 = reinterpret_cast<const uint32_t*>(r0);
    const uint32_t* w1 = reinterpret_cast<const uint32_t*>(r1);
    for (int ux = 0; ux < N; ++ux) {
      const uint32_t a = ry[ux] * 0x00010001u;
      const uint32_t* wsrc = (ux & 1) ? w1 : w0;
      const int base = ux >> 1;
#pragma unroll
      for (int k = 0; k < kAcPairs; ++k) {
        if (k < P) {
          const int j = lane + 32 * k;  // shifts ex = 2j, 2j + 1
          const uint32_t m = __vcmpeq2(wsrc[base + j], a);
          packed[k] += m & 0x00010001u;
        }
      }
    }
    __syncwarp();
    if (++rows_since == 32) {  // at most 32 * N <= 32768 per 16-bit half
#pragma unroll
      for (int k = 0; k < kAcPairs; ++k) {
        cnt[2 * k] += packed[k] & 0xffffu;
        cnt[2 * k + 1] += packed[k] >> 16;
        packed[k] = 0u;
      }
      rows_since = 0;
    }
  }
#pragma unroll
  for (int k = 0; k < kAcPairs; ++k) {
    cnt[2 * k] += packed[k] & 0xffffu;
    cnt[2 * k + 1] += packed[k] >> 16;
  }
  __syncthreads();
  int32_t* red = reinterpret_cast<int32_t*>(acs);  // [kAcWarps][N]
#pragma unroll
  for (int k = 0; k < kAcPairs; ++k) {
    const int ex = 2 * (lane + 32 * k);
    if (k < P && ex < N) {
      red[warp * N + ex] = static_cast<int32_t>(cnt[2 * k]);
      if (ex + 1 < N) red[warp * N + ex + 1] = static_cast<int32_t>(cnt[2 * k + 1]);
    }
  }
  __syncthreads();
  for (int ex = threadIdx.x; ex < N; ex += blockDim.x) {
    int32_t t = 0;
    for (int w = 0; w < kAcWarps; ++w) t += red[w * N + ex];
    A[static_cast<size_t>(ey) * N + ex] = t;
  }
}

// K[l][e] = sum_d g_l(d) g_l((d + e) mod N), FP64.
__global__ void k_gauss_autocorr(const double* __restrict__ gw64, int N, int L, double* __restrict__ K) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i >= static_cast<long long>(N) * L) return;
  const int l = static_cast<int>(i / N), e = static_cast<int>(i % N);
  const int rho = gauss_radius(l, N);
  const double* g = gw64 + static_cast<size_t>(l) * N;
  double acc = 0.0;
  for (int d = -rho; d <= rho; ++d) acc += g[(d + N) % N] * g[((d + e) % N + N) % N];
  K[i] = acc;
}

// part[ey][l] = K_l[ey] sum_ex K_l[ex] A[ey][ex]; one CTA per ey, fixed order.
__global__ void __launch_bounds__(256) k_gauss_norm_rows(const int32_t* __restrict__ A,
                                                         const double* __restrict__ K, int N, int L,
                                                         double* __restrict__ part) {
  __shared__ double red[256];
  const int ey = blockIdx.x;
  for (int l = 0; l < L; ++l) {
    const double* Kl = K + static_cast<size_t>(l) * N;
    double acc = 0.0;
    for (int ex = threadIdx.x; ex < N; ex += blockDim.x)
      acc += Kl[ex] * static_cast<double>(A[static_cast<size_t>(ey) * N + ex]);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[static_cast<size_t>(ey) * L + l] = Kl[ey] * red[0];
    __syncthreads();
  }
}

// norm2 = sum_l lscale[l]^2 sum_ey part[ey][l], fixed order.
__global__ void __launch_bounds__(256) k_gauss_norm_final(const double* __restrict__ part, int N,
                                                          int L, const double* __restrict__ lscale,
                                                          double* __restrict__ norm2) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < N * L; i += blockDim.x) {
    const double c = lscale[i % L];
    acc += c * c * part[i];
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *norm2 = red[0];
}

size_t conv_smem(int l, int N, int RL) {
  const int rho = gauss_radius(l, N);
  return (static_cast<size_t>((2 * rho + 1 + 3) & ~3) + static_cast<size_t>(kConvRows + 2 * rho) * RL) *
         sizeof(float);
}

size_t autocorr_smem(int N) {
  const size_t span = static_cast<size_t>(N) + 64 * ((N + 63) / 64);
  const size_t rows = static_cast<size_t>(kAcWarps) * (N + 2 * span) * sizeof(uint16_t);
  const size_t red = static_cast<size_t>(kAcWarps) * N * sizeof(int32_t);
  return rows > red ? rows : red;
}

int launch_gauss_conv(const float* src, int lstride, const float* gw, const MttkrpDims& d, float* out,
                      cudaStream_t s) {
  const int RL = rank_lanes(d.R);
  size_t smem = 0;
  for (int l = 0; l < d.L; ++l) smem = std::max(smem, conv_smem(l, d.N, RL));
  k_gauss_conv<<<dim3((d.N + kConvRows - 1) / kConvRows, d.L, d.R / RL), 256, smem, s>>>(
      src, lstride, gw, d.N, d.L, d.R, out);
  GSP_CHECK_LAUNCH();
  return GSP_OK;
}

// Row splits of a side or bin pass: about kSideTargetCtas CTAs, at least 16 rows each.
int row_splits(const MttkrpDims& d) {
  const int G = 32 / rank_lanes(d.R);
  const int colblocks = (d.N + kSW * G * kSC - 1) / (kSW * G * kSC);
  const int chunks = (d.R + 31) / 32;
  int S = (kSideTargetCtas + colblocks * chunks - 1) / (colblocks * chunks);
  const int smax = d.N >= 16 ? d.N / 16 : 1;
  if (S > smax) S = smax;
  if (S < 1) S = 1;
  const int rows = (d.N + S - 1) / S;
  return (d.N + rows - 1) / rows;
}

dim3 pass_grid(const MttkrpDims& d, int S) {
  const int G = 32 / rank_lanes(d.R);
  return dim3((d.N + kSW * G * kSC - 1) / (kSW * G * kSC), S, (d.R + 31) / 32);
}

size_t rows_smem(const MttkrpDims& d) {  // two buffers
  return 2 * (static_cast<size_t>(kChunkRows) * d.L * rank_lanes(d.R) * sizeof(float) +
              static_cast<size_t>(kChunkRows) * cta_cols(d.R) * sizeof(uint16_t));
}
size_t side_smem(const MttkrpDims& d) {
  return 2u * d.B * rank_lanes(d.R) * sizeof(float) + rows_smem(d);
}
size_t bin_smem(const MttkrpDims& d) {
  return (static_cast<size_t>(d.B) * rank_lanes(d.R) + static_cast<size_t>(kSW) * 32 * d.B) *
             sizeof(float) + rows_smem(d);
}

#define GSP_LEVELS_1_TO_11(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11)

int ensure_struct_attrs(const MttkrpDims& d) {
  static int done_dev = -1;
  int dev = 0;
  GSP_CUDA(cudaGetDevice(&dev));
  if (done_dev == dev) return GSP_OK;
  // the largest shapes: 128 bins, 11 levels, 32 rank lanes (8 rank lanes: 128 columns)
  const MttkrpDims big{1024, kMaxLevels, 128, 32}, wide{1024, kMaxLevels, 128, 8};
  const int side = static_cast<int>(std::max(side_smem(big), side_smem(wide)));
  const int bin = static_cast<int>(std::max(bin_smem(big), bin_smem(wide)));
#define GSP_SET_ATTR(n)                                                                    \
  GSP_CUDA(cudaFuncSetAttribute(k_bin_pass<n>, cudaFuncAttributeMaxDynamicSharedMemorySize, bin)); \
  GSP_CUDA(cudaFuncSetAttribute(k_side_pass<n>, cudaFuncAttributeMaxDynamicSharedMemorySize, side));
  GSP_LEVELS_1_TO_11(GSP_SET_ATTR)
#undef GSP_SET_ATTR
  GSP_CUDA(cudaFuncSetAttribute(k_window_tables, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (1024 + 1) * kWinRanks * static_cast<int>(sizeof(double))));
  GSP_CUDA(cudaFuncSetAttribute(k_gauss_conv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(conv_smem(kMaxLevels - 1, 1024, 32))));
  GSP_CUDA(cudaFuncSetAttribute(k_match_autocorr, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(autocorr_smem(1024))));
  (void)d;
  done_dev = dev;
  return GSP_OK;
}

}  // namespace

bool struct_supported(const MttkrpDims& d) { return d.L >= 1 && d.L <= kMaxLevels && d.N >= 8; }

StructSizes struct_sizes(const MttkrpDims& d) {
  StructSizes z;
  const size_t NLR = static_cast<size_t>(d.N) * d.L * d.R;
  const int S = row_splits(d);
  const dim3 g = pass_grid(d, S);
  z.table_floats = NLR;
  z.part_floats = static_cast<size_t>(S) * NLR;
  z.pre_doubles = static_cast<size_t>(d.L) * (d.N + 1) * d.R;
  z.seg_doubles = static_cast<size_t>(d.L) * seg_count(d.N) * d.R;
  z.stpart_floats = static_cast<size_t>(g.x) * g.y * d.B * d.R;
  z.gauss_floats = static_cast<size_t>(d.L) * d.N;  // weights; FP64 copy and K alike
  z.autocorr_ints = static_cast<size_t>(d.N) * d.N;
  z.normpart_doubles = static_cast<size_t>(d.N) * d.L;
  return z;
}

int struct_window_tables(const float* f, float* out, const StructWs& w, const MttkrpDims& d,
                         cudaStream_t s) {
  GSP_TRY(ensure_struct_attrs(d));
  prof_begin(PROF_STRUCT_TABLES, s);
  if (w.gw) {
    GSP_TRY(launch_gauss_conv(f, 0, w.gw, d, out, s));
    prof_end(PROF_STRUCT_TABLES, s);
    return GSP_OK;
  }
  k_window_tables<<<dim3(d.R / kWinRanks, d.L), 256, (d.N + 1) * kWinRanks * sizeof(double), s>>>(
      f, d.N, d.L, d.R, out);
  prof_end(PROF_STRUCT_TABLES, s);
  GSP_CHECK_LAUNCH();
  return GSP_OK;
}

int struct_side(const uint16_t* bm, const float* win, const float* fs, const float* ft,
                const float* fl, const StructWs& w, const MttkrpDims& d, double* M, float* Mf,
                cudaStream_t s) {
  GSP_TRY(ensure_struct_attrs(d));
  const int S = row_splits(d);
  const int rows = (d.N + S - 1) / S;
  const dim3 g = pass_grid(d, S);
  prof_begin(PROF_STRUCT_SIDE, s);
  switch (d.L) {
#define GSP_SIDE_CASE(n)                                                                    \
  case n:                                                                                   \
    k_side_pass<n><<<g, kSW * 32, side_smem(d), s>>>(bm, win, fs, ft, d.N, ilog2(d.B), d.R, \
                                                     rows, w.part);                         \
    break;
    GSP_LEVELS_1_TO_11(GSP_SIDE_CASE)
#undef GSP_SIDE_CASE
    default:
      return GSP_ERR_UNSUPPORTED;
  }
  GSP_CHECK_LAUNCH();
  const int chunks = (d.R + 31) / 32, nseg = seg_count(d.N);
  const long long nel = static_cast<long long>(d.N) * d.L * d.R;
  k_side_reduce<<<grid_for(nel, 256), 256, 0, s>>>(w.part, S, nel, w.sig, w.sig64);
  GSP_CHECK_LAUNCH();
  if (w.gw) {  // Gaussian footprints: weighted sums of sigma, no prefix
    if (M) {
      GSP_TRY(launch_gauss_conv(w.sig, 1, w.gw, d, w.conv, s));
      k_level_combine<<<grid_for(static_cast<long long>(d.N) * d.R, 256), 256, 0, s>>>(
          w.conv, fl, d.N, d.L, d.R, w.lscale, M, Mf);
      GSP_CHECK_LAUNCH();
    }
    prof_end(PROF_STRUCT_SIDE, s);
    return GSP_OK;
  }
  k_side_segments<<<grid_for(static_cast<long long>(nseg) * d.L * chunks * 32, 256), 256, 0, s>>>(
      w.sig64, d.N, d.L, d.R, w.pre, w.segtot);
  GSP_CHECK_LAUNCH();
  k_side_offsets<<<grid_for(static_cast<long long>(d.L) * d.R, 128), 128, 0, s>>>(w.segtot, d.N, d.L,
                                                                                   d.R, w.off);
  GSP_CHECK_LAUNCH();
  k_side_fix<<<grid_for(static_cast<long long>(d.L) * (d.N + 1) * d.R, 256), 256, 0, s>>>(
      w.off, d.N, d.L, d.R, w.pre);
  GSP_CHECK_LAUNCH();
  if (M) {
    k_side_window<<<grid_for(static_cast<long long>(d.N) * d.R, 256), 256, 0, s>>>(
        w.pre, fl, d.N, d.L, d.R, w.lscale, M, Mf);
    GSP_CHECK_LAUNCH();
  }
  prof_end(PROF_STRUCT_SIDE, s);
  return GSP_OK;
}

int struct_level(const float* be, const StructWs& w, const MttkrpDims& d, double* M, float* Mf,
                 cudaStream_t s) {
  k_level_mode<<<dim3(d.L, (d.R + 31) / 32), 1024, 0, s>>>(w.sig, be, d.N, d.L, d.R, w.lscale, M, Mf);
  GSP_CHECK_LAUNCH();
  return GSP_OK;
}

int struct_bins(const uint16_t* bm, const float* al, const float* be, const float* fl,
                const float* tab, int mode_t, const StructWs& w, const MttkrpDims& d, double* M,
                float* Mf, cudaStream_t s) {
  GSP_TRY(ensure_struct_attrs(d));
  const int S = row_splits(d);
  const int rows = (d.N + S - 1) / S;
  const dim3 g = pass_grid(d, S);
  prof_begin(PROF_STRUCT_BINS, s);
  switch (d.L) {
#define GSP_BIN_CASE(n)                                                                     \
  case n:                                                                                   \
    k_bin_pass<n><<<g, kSW * 32, bin_smem(d), s>>>(bm, al, be, fl, tab, d.N, ilog2(d.B), d.R, \
                                                   w.lscale, mode_t, rows, w.stpart);       \
    break;
    GSP_LEVELS_1_TO_11(GSP_BIN_CASE)
#undef GSP_BIN_CASE
    default:
      return GSP_ERR_UNSUPPORTED;
  }
  GSP_CHECK_LAUNCH();
  k_bin_reduce<<<dim3(d.B, (d.R + 31) / 32), 256, 0, s>>>(w.stpart, static_cast<int>(g.x * g.y),
                                                         d.B, d.R, M, Mf);
  GSP_CHECK_LAUNCH();
  prof_end(PROF_STRUCT_BINS, s);
  return GSP_OK;
}

int struct_level_scales(int L, int B, int raw, int gauss, double* lscale, cudaStream_t s) {
  k_level_scales<<<1, 32, 0, s>>>(L, B, raw, gauss, lscale);
  GSP_CHECK_LAUNCH();
  return GSP_OK;
}

int struct_gauss_prepare(const uint16_t* bins, const StructWs& w, const MttkrpDims& d,
                         double* gw64, double* K, int32_t* A, double* normpart, double* norm2,
                         cudaStream_t s) {
  GSP_TRY(ensure_struct_attrs(d));
  if (d.N > 1024 || !is_pow2(d.N)) return GSP_ERR_UNSUPPORTED;
  k_gauss_weights<<<d.L, 256, 0, s>>>(d.N, w.gw, gw64);
  GSP_CHECK_LAUNCH();
  k_match_autocorr<<<d.N, kAcWarps * 32, autocorr_smem(d.N), s>>>(bins, d.N, A);
  GSP_CHECK_LAUNCH();
  k_gauss_autocorr<<<grid_for(static_cast<long long>(d.N) * d.L, 256), 256, 0, s>>>(gw64, d.N, d.L, K);
  GSP_CHECK_LAUNCH();
  k_gauss_norm_rows<<<d.N, 256, 0, s>>>(A, K, d.N, d.L, normpart);
  GSP_CHECK_LAUNCH();
  k_gauss_norm_final<<<1, 256, 0, s>>>(normpart, d.N, d.L, w.lscale, norm2);
  GSP_CHECK_LAUNCH();
  return GSP_OK;
}

int struct_transpose_bins(const uint16_t* in, uint16_t* out, int N, cudaStream_t s) {
  k_transpose_bins<<<dim3((N + 31) / 32, (N + 31) / 32), dim3(32, 8), 0, s>>>(in, N, out);
  GSP_CHECK_LAUNCH();
  return GSP_OK;
}

int struct_bins_from_level0(const int32_t* h0, int N, int B, uint16_t* bins, uint32_t* status,
                            cudaStream_t s) {
  k_bins_from_level0<<<grid_for(static_cast<long long>(N) * N * 32, 256), 256, 0, s>>>(
      h0, N, B * B, bins, status);
  GSP_CHECK_LAUNCH();
  return GSP_OK;
}

}  // namespace gsp
