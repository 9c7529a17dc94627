// Rows a1-a3: binning of the normal map and exhaustive multi-level footprint
// histograms (Sec. 4.1), written straight into int32 counts and/or the
// scaled MTTKRP operand.
//
// Every level is computed from the 2-byte bin map alone (it stays in L2) by
// box sums of per-bin indicators staged in shared memory, so the only HBM
// traffic is the output itself.  Every value is an integer count, exact in
// the types it passes through (FP16 <= 2^11, FP32 < 2^24), hence bit-exact.
#include <cuda_fp16.h>

#include "ndf_build.cuh"

namespace gsp {

namespace {

constexpr int kGroupWords = 128 * 128 / 16 / 32;  // one bit per 16-bin group, B <= 128

// `groups` (optional): bit g set when some texel falls in bins [16g, 16g + 16).
__global__ void k_bin_normals(const float2* __restrict__ nxy, int n, int bins,
                              uint16_t* __restrict__ out, uint32_t* status,
                              uint32_t* __restrict__ groups) {
  __shared__ uint32_t gmask[kGroupWords];
  if (groups) {
    for (int k = threadIdx.x; k < kGroupWords; k += blockDim.x) gmask[k] = 0u;
    __syncthreads();
  }
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < n;
  uint16_t code = 0;
  if (valid) {
    const float2 v = nxy[i];
    if (!isfinite(v.x) || !isfinite(v.y)) {
      set_status(status, GSP_DEV_NONFINITE_NORMAL);
    } else {
      const float half = static_cast<float>(bins >> 1);
      const float hi = static_cast<float>(bins - 1);
      // fl32(fl32(n + 1) * B/2), explicit roundings, no contraction into an FMA
      float s = floorf(__fmul_rn(__fadd_rn(v.x, 1.0f), half));
      float t = floorf(__fmul_rn(__fadd_rn(v.y, 1.0f), half));
      s = fminf(fmaxf(s, 0.0f), hi);
      t = fminf(fmaxf(t, 0.0f), hi);
      code = static_cast<uint16_t>(static_cast<int>(s) * bins + static_cast<int>(t));
    }
    out[i] = code;
  }
  if (groups) {
    if (valid) atomicOr(&gmask[(code >> 4) >> 5], 1u << ((code >> 4) & 31));
    __syncthreads();
    for (int k = threadIdx.x; k < kGroupWords; k += blockDim.x)
      if (gmask[k]) atomicOr(groups + k, gmask[k]);
  }
}

__device__ __forceinline__ void sink_store(const LevelSink& o, long long i, int4 v) {
  if (o.h) reinterpret_cast<int4*>(o.h)[i] = v;
  const float f0 = static_cast<float>(v.x) * o.scale, f1 = static_cast<float>(v.y) * o.scale;
  const float f2 = static_cast<float>(v.z) * o.scale, f3 = static_cast<float>(v.w) * o.scale;
  const uint32_t d = weyl_dither(static_cast<unsigned long long>(o.base + 4 * i));
  if (o.f32) {
    float4 f = make_float4(f0, f1, f2, f3);
    if (o.tf32)
      f = make_float4(tf32_dither(f0, d), tf32_dither(f1, d + kWeyl), tf32_dither(f2, d + 2 * kWeyl),
                      tf32_dither(f3, d + 3 * kWeyl));
    reinterpret_cast<float4*>(o.f32)[i] = f;
  }
  if (o.bf16) {
    uint2 p;
    p.x = bf16_pair_dither(f0, d, f1, d + kWeyl);
    p.y = bf16_pair_dither(f2, d + 2 * kWeyl, f3, d + 3 * kWeyl);
    reinterpret_cast<uint2*>(o.bf16)[i] = p;
  }
}

__device__ __forceinline__ void sink_sumsq(const LevelSink& o, int4 v, bool active) {
  if (!o.sumsq) return;
  unsigned long long q = 0;
  if (active) {
    q = static_cast<unsigned long long>(static_cast<long long>(v.x) * v.x) +
        static_cast<unsigned long long>(static_cast<long long>(v.y) * v.y) +
        static_cast<unsigned long long>(static_cast<long long>(v.z) * v.z) +
        static_cast<unsigned long long>(static_cast<long long>(v.w) * v.w);
  }
  for (int off = 16; off > 0; off >>= 1) q += __shfl_down_sync(0xffffffffu, q, off);
  if ((threadIdx.x & 31) == 0 && q) atomicAdd(o.sumsq, q);
}

// Sliding box sums of per-bin indicators (all levels straight from the bin map).
//
// CTA (group of 16 bins, band of `ychunk` rows, level l): shared memory holds
// V[x][b] = number of texels of bin g0 + b in column x among the window rows
// [y - a, y - a + w) (w = 2^l, a = w/2, wrapped).  Moving from row y to y+1
// removes one texel and adds one per column.  For each row the histograms of
// all N footprints are window sums of V along x, read from the prefix sum S
// over x: two look-ups per count, three across the wrap.
//  - updates: thread t owns the columns x = t, t + 512, ... (no atomics); V
//    holds FP16 counts (<= 2^10, exact), updated by exact +-1 adds;
//  - prefix: warp w covers a contiguous x range in blocks of 32 columns; the
//    inclusive prefix of a block is a lower-triangular ones matrix times the
//    block's [32 x 16] counts, six warp MMAs (m16n8k16, FP16 in, FP32 out,
//    exact since every sum is an integer below 2^24); block totals carry in
//    FP32, and S is stored (as int) once the offsets of the earlier ranges
//    are known;
//  - rows of V (48 B) are padded so that the ldmatrix row reads of consecutive
//    columns fall on distinct banks; S is kept as two planes of 8 bins (32-byte
//    rows) whose offsets differ by 16 mod 128 bytes, so the output's reads
//    (lane pairs per column, one plane each) fall on distinct banks;
//  - S is double-buffered, so the scan of row y and the output of row y - 1
//    share one phase: two barriers per row.
constexpr int kHistG = 16;
constexpr int kHistThreads = 512;
constexpr int kHistWarps = kHistThreads / 32;
constexpr int kVRow = 24;  // uint16 per column count row (16 + 8 padding)
constexpr int kSRow = 8;   // ints per prefix row of one 8-bin plane
constexpr int kMaxBlocks = 2;  // 32-column blocks per scanning warp (N <= 1024)

// Ints per S plane: N + 1 rows of 8, padded so that the second plane starts 4
// ints (16 bytes) past a multiple of 32 ints from the first.
__host__ __device__ constexpr int s_plane_ints(int N) {
  return (N + 1) * kSRow + (((4 - (N + 1) * kSRow) % 32) + 32) % 32;
}

// Four 8x8 b16 matrices from shared memory, transposed into the B-fragment
// layout of mma.m16n8k16 (lanes 8i..8i+7 give the row addresses of matrix i).
__device__ __forceinline__ void ldsm_x4_trans(uint32_t addr, uint32_t (&r)[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr)
               : "memory");
}

// D = A B + C, A 16x16 and B 16x8 FP16, C and D FP32 (warp-level MMA).
__device__ __forceinline__ void mma_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                          uint32_t b1, const float (&c)[4]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
      "{%8, %9}, {%10, %11, %12, %13};"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(c[0]), "f"(c[1]),
        "f"(c[2]), "f"(c[3]));
}

// An exact non-negative integer below 2^23 held in a float, as an int.
__device__ __forceinline__ int float_to_int_exact(float v) {
  return __float_as_int(v + 8388608.0f) - 0x4B000000;
}

__global__ void __launch_bounds__(kHistThreads, 1)
    k_box_hist(const uint16_t* __restrict__ bins_map, int logN, int B2, int ychunk,
               const __grid_constant__ HistOut o) {
  constexpr int G = kHistG;
  extern __shared__ __align__(16) uint8_t smem_b[];
  __shared__ __align__(16) float WT[kHistWarps * G];
  const int N = 1 << logN, m = N - 1;
  const int vrows = N < 32 ? 32 : N;                                          // whole 32-column blocks
  __half* V = reinterpret_cast<__half*>(smem_b);                              // [vrows][24]
  int* S = reinterpret_cast<int*>(smem_b + vrows * kVRow * sizeof(__half));  // [2][2][N + 1][8]
  const int plane = s_plane_ints(N), sbuf = 2 * plane;
  const int g0 = blockIdx.x * G;
  const int y0 = blockIdx.y * ychunk;
  const int l = gridDim.z - 1 - blockIdx.z;  // coarsest level first: its window fill is the longest
  const int w = 1 << l, a = w >> 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (o.groups && !((o.groups[blockIdx.x >> 5] >> (blockIdx.x & 31)) & 1u)) {
    // no texel of the map falls in this bin group: every count is zero
    // items of 8 bins (16-byte BF16 stores; two 16-byte stores for 32-bit outputs)
    const int row_log = logN + 1;  // N * (G / 8) items per row
    const long long items = static_cast<long long>(ychunk) << row_log;
    const uint4 z4 = make_uint4(0u, 0u, 0u, 0u);
    for (long long e = tid; e < items; e += kHistThreads) {
      const int yy = y0 + static_cast<int>(e >> row_log);
      const int rem = static_cast<int>(e & ((1LL << row_log) - 1));
      const int x = rem >> 1, h = rem & 1;
      const long long i8 = (((static_cast<long long>(l) * N + yy) * N * B2) >> 3) +
                           ((static_cast<long long>(x) * B2 + g0) >> 3) + h;
      if (o.h) {
        reinterpret_cast<uint4*>(o.h)[2 * i8] = z4;
        reinterpret_cast<uint4*>(o.h)[2 * i8 + 1] = z4;
      }
      if (o.f32) {
        reinterpret_cast<uint4*>(o.f32)[2 * i8] = z4;
        reinterpret_cast<uint4*>(o.f32)[2 * i8 + 1] = z4;
      }
      if (o.bf16) reinterpret_cast<uint4*>(o.bf16)[i8] = z4;
    }
    return;
  }
  const int scan_warps = N >= 32 * kHistWarps ? kHistWarps : (N >= 32 ? N >> 5 : 1);
  const int xr = N / scan_warps;               // columns per scanning warp
  const int nblk = xr >= 32 ? xr >> 5 : 1;     // 32-column blocks per warp
  // Prefix over a 32-column block by warp MMA: S_block = [Tri; Ones Tri] V_block
  // with Tri the 16x16 lower-triangular ones.  Counts (<= 2^10) are exact in
  // FP16 and every sum (< 2^24) in FP32, whatever the accumulation order.
  const int fr = lane >> 2, fc = 2 * (lane & 3);  // fragment row / column pair of this lane
  uint32_t aTri[4], aOne[4];
  {
    auto tri = [](int mm, int kk) -> uint32_t { return kk <= mm ? 0x3C00u : 0u; };
    aTri[0] = tri(fr, fc) | (tri(fr, fc + 1) << 16);
    aTri[1] = tri(fr + 8, fc) | (tri(fr + 8, fc + 1) << 16);
    aTri[2] = tri(fr, fc + 8) | (tri(fr, fc + 9) << 16);
    aTri[3] = tri(fr + 8, fc + 8) | (tri(fr + 8, fc + 9) << 16);
#pragma unroll
    for (int i = 0; i < 4; ++i) aOne[i] = 0x3C003C00u;
  }
  // ldmatrix row address of this lane: matrix q = lane / 8 covers k rows
  // (q & 1) * 8 .. + 7 and bins (q >> 1) * 8 .. + 7 of a 16-column half block
  const uint32_t v_lane = static_cast<uint32_t>(__cvta_generic_to_shared(V)) +
                          static_cast<uint32_t>((((lane >> 3) & 1) * 8 + (lane & 7)) * kVRow +
                                                (lane >> 4) * 8) * 2u;

  for (int i = tid; i < vrows * kVRow / 8; i += kHistThreads)
    reinterpret_cast<uint4*>(V)[i] = make_uint4(0, 0, 0, 0);
  if (tid < 8)  // S[0] = 0 in both planes of both buffers
    reinterpret_cast<int4*>(S + (tid >> 2) * sbuf + ((tid >> 1) & 1) * plane)[tid & 1] =
        make_int4(0, 0, 0, 0);
  __syncthreads();
  {
    // the window's rows for this thread's columns x = tid, tid + 512:
    // 16 rows x 2 columns of independent loads in flight (N <= 2 * kHistThreads)
    constexpr int kRows = 16;
    for (int j0 = 0; j0 < w; j0 += kRows) {
      uint16_t code[2][kRows];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int x = tid + k * kHistThreads;
#pragma unroll
        for (int u = 0; u < kRows; ++u)
          code[k][u] = (x < N && j0 + u < w) ? bins_map[(((y0 - a + j0 + u) & m) << logN) + x]
                                              : static_cast<uint16_t>(0xFFFFu);
      }
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int x = tid + k * kHistThreads;
#pragma unroll
        for (int u = 0; u < kRows; ++u) {
          const int b = static_cast<int>(code[k][u]) - g0;
          if (static_cast<unsigned>(b) < static_cast<unsigned>(G))
            V[x * kVRow + b] = __hadd(V[x * kVRow + b], __float2half(1.0f));
        }
      }
    }
  }
  const float sc = o.scale[l];
  const float nb = -8388608.0f * sc;  // -2^23 * scale, exact
  // codes leaving / entering the window at the next row step, loaded one row
  // ahead so the L2 latency overlaps this row's work (N <= 2 * kHistThreads)
  int nxt_out[2], nxt_in[2];
  auto fetch = [&](int yn) {
    const int ro = (yn - 1 - a) & m, ri = (yn - 1 - a + w) & m;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int x = tid + k * kHistThreads;
      nxt_out[k] = x < N ? static_cast<int>(bins_map[(ro << logN) + x]) : 0xFFFF;
      nxt_in[k] = x < N ? static_cast<int>(bins_map[(ri << logN) + x]) : 0xFFFF;
    }
  };
  fetch(y0 + 1);
  unsigned long long sumsq = 0;
  // The output items of this thread (x = e / 2, plane h = e % 2 for
  // e = tid + k * 512, k < 2N / 512) are the same in every row: their prefix
  // offsets within an S buffer (ints), the wrap term and the column part of
  // the output index are computed once.  S[N] + S[en - N] replaces S[en] for
  // a window that wraps (wr >= 0).
  constexpr int kMaxItems = 4;  // 2N / kHistThreads for N <= 1024
  int it_lo[kMaxItems], it_hi[kMaxItems], it_wr[kMaxItems], it_col[kMaxItems];
#pragma unroll
  for (int k = 0; k < kMaxItems; ++k) {
    const int e = tid + k * kHistThreads;
    const int h = e & 1, x = e >> 1;
    const int st = (x - a) & m, en = st + w;
    it_lo[k] = h * plane + st * kSRow;
    it_hi[k] = h * plane + (en <= N ? en : N) * kSRow;
    it_wr[k] = en <= N ? -1 : h * plane + (en - N) * kSRow;
    it_col[k] = ((x * B2 + g0) >> 3) + h;
  }
  __syncthreads();  // V of row y0 complete (columns are initialised by other warps)

  // Pipelined over rows with S double-buffered: iteration y scans row y (V
  // holds its window) while writing the counts of row y - 1 from the other S
  // buffer; after the barrier the scan's range offsets are applied, S of row y
  // is stored and V moves on to row y + 1.  Two barriers per row.
  for (int y = y0; y <= y0 + ychunk; ++y) {
    const bool scan_row = y < y0 + ychunk;
    int* Sc = S + ((y - y0) & 1) * sbuf;        // S of row y
    const int* Sp = S + ((y - y0 + 1) & 1) * sbuf;  // S of row y - 1
    // inclusive prefix of each block, per lane: [block][nt][row group][2 bins]
    float pre[kMaxBlocks][2][4][2];
    if (scan_row && warp < scan_warps) {
      float carry[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
      const int xbeg = warp * xr;
#pragma unroll
      for (int blk = 0; blk < kMaxBlocks; ++blk) {
        if (blk < nblk) {
          const int xb = xbeg + blk * 32;
          uint32_t bk0[4], bk1[4];  // B fragments of columns xb..xb+15 and xb+16..xb+31
          ldsm_x4_trans(v_lane + static_cast<uint32_t>(xb * kVRow * 2), bk0);
          ldsm_x4_trans(v_lane + static_cast<uint32_t>((xb + 16) * kVRow * 2), bk1);
          const float zero[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int nt = 0; nt < 2; ++nt) {
            float top[4], bot[4];
            mma_16816(top, aTri, bk0[2 * nt], bk0[2 * nt + 1], zero);
            mma_16816(bot, aOne, bk0[2 * nt], bk0[2 * nt + 1], zero);
            mma_16816(bot, aTri, bk1[2 * nt], bk1[2 * nt + 1], bot);
            pre[blk][nt][0][0] = top[0] + carry[nt][0];
            pre[blk][nt][0][1] = top[1] + carry[nt][1];
            pre[blk][nt][1][0] = top[2] + carry[nt][0];
            pre[blk][nt][1][1] = top[3] + carry[nt][1];
            pre[blk][nt][2][0] = bot[0] + carry[nt][0];
            pre[blk][nt][2][1] = bot[1] + carry[nt][1];
            pre[blk][nt][3][0] = bot[2] + carry[nt][0];
            pre[blk][nt][3][1] = bot[3] + carry[nt][1];
            // block total: row 31 (lanes 28..31 hold it for their bin pairs)
            carry[nt][0] = __shfl_sync(0xffffffffu, pre[blk][nt][3][0], 28 + (lane & 3));
            carry[nt][1] = __shfl_sync(0xffffffffu, pre[blk][nt][3][1], 28 + (lane & 3));
          }
        }
      }
      if (lane < 4) {  // range totals of bins fc, fc + 1 (plane 0) and fc + 8, fc + 9
        WT[warp * G + fc] = carry[0][0];
        WT[warp * G + fc + 1] = carry[0][1];
        WT[warp * G + 8 + fc] = carry[1][0];
        WT[warp * G + 8 + fc + 1] = carry[1][1];
      }
    }
    if (y > y0) {
      // counts of every footprint of row y - 1, eight bins per item; the lanes
      // of a warp take consecutive x, so their 16-byte prefix reads (80-byte
      // rows) fall on distinct banks
      const long long row8 = ((static_cast<long long>(l) * N + (y - 1)) * N * B2) >> 3;
#pragma unroll
      for (int k = 0; k < kMaxItems; ++k) {
        if (tid + k * kHistThreads >= 2 * N) break;  // lane pairs write 32 contiguous bytes
        const int4* lo4 = reinterpret_cast<const int4*>(Sp + it_lo[k]);
        const int4* hi4 = reinterpret_cast<const int4*>(Sp + it_hi[k]);
        int c[8];
        {
          const int4 l0 = lo4[0], l1 = lo4[1];
          int4 h0 = hi4[0], h1 = hi4[1];
          if (it_wr[k] >= 0) {  // window wraps: S[N] - S[st] + S[en - N]
            const int4* wr = reinterpret_cast<const int4*>(Sp + it_wr[k]);
            const int4 w0 = wr[0], w1 = wr[1];
            h0 = make_int4(h0.x + w0.x, h0.y + w0.y, h0.z + w0.z, h0.w + w0.w);
            h1 = make_int4(h1.x + w1.x, h1.y + w1.y, h1.z + w1.z, h1.w + w1.w);
          }
          c[0] = h0.x - l0.x; c[1] = h0.y - l0.y; c[2] = h0.z - l0.z; c[3] = h0.w - l0.w;
          c[4] = h1.x - l1.x; c[5] = h1.y - l1.y; c[6] = h1.z - l1.z; c[7] = h1.w - l1.w;
        }
        const long long i8 = row8 + it_col[k];
        if (o.h) {
          reinterpret_cast<int4*>(o.h)[2 * i8] = make_int4(c[0], c[1], c[2], c[3]);
          reinterpret_cast<int4*>(o.h)[2 * i8 + 1] = make_int4(c[4], c[5], c[6], c[7]);
        }
        // c * scale, exactly: 2^23 + c as a float (c < 2^23), times the
        // power-of-two scale, minus 2^23 * scale, in one rounding
        float f[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) f[k] = fmaf(__int_as_float(c[k] | 0x4B000000), sc, nb);
        const uint32_t d = weyl_dither(static_cast<unsigned long long>(i8) * 8);
        if (o.f32) {
          if (o.tf32 && l >= 6) {  // counts <= 4^5 are exact on the TF32 grid
#pragma unroll
            for (int k = 0; k < 8; ++k) f[k] = tf32_dither(f[k], d + k * kWeyl);
          }
          reinterpret_cast<float4*>(o.f32)[2 * i8] = make_float4(f[0], f[1], f[2], f[3]);
          reinterpret_cast<float4*>(o.f32)[2 * i8 + 1] = make_float4(f[4], f[5], f[6], f[7]);
        }
        if (o.bf16 && l <= 4) {  // counts <= 256: exact in BF16
          uint4 p;
          p.x = __byte_perm(__float_as_uint(f[0]), __float_as_uint(f[1]), 0x7632);
          p.y = __byte_perm(__float_as_uint(f[2]), __float_as_uint(f[3]), 0x7632);
          p.z = __byte_perm(__float_as_uint(f[4]), __float_as_uint(f[5]), 0x7632);
          p.w = __byte_perm(__float_as_uint(f[6]), __float_as_uint(f[7]), 0x7632);
          reinterpret_cast<uint4*>(o.bf16)[i8] = p;
        } else if (o.bf16) {
          uint4 p;
          p.x = bf16_pair_dither(f[0], d, f[1], d + kWeyl);
          p.y = bf16_pair_dither(f[2], d + 2 * kWeyl, f[3], d + 3 * kWeyl);
          p.z = bf16_pair_dither(f[4], d + 4 * kWeyl, f[5], d + 5 * kWeyl);
          p.w = bf16_pair_dither(f[6], d + 6 * kWeyl, f[7], d + 7 * kWeyl);
          reinterpret_cast<uint4*>(o.bf16)[i8] = p;
        }
        if (o.sumsq) {
          if (l <= 7) {  // counts <= 4^7: eight squares fit in 32 bits
            uint32_t q = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) q += static_cast<uint32_t>(c[k]) * static_cast<uint32_t>(c[k]);
            sumsq += q;
          } else {
#pragma unroll
            for (int k = 0; k < 8; ++k)
              sumsq += static_cast<unsigned long long>(static_cast<uint32_t>(c[k])) * static_cast<uint32_t>(c[k]);
          }
        }
      }
    }
    __syncthreads();  // range totals WT complete; V and S of row y - 1 no longer read
    if (scan_row) {
      if (warp < scan_warps) {
        // offset of this warp's range: lanes 0..15 sum one bin each over the earlier warps
        float my = 0.f;
        if (lane < G) {
#pragma unroll
          for (int k = 0; k < kHistWarps; ++k)  // independent loads, then the sum
            if (k < warp) my += WT[k * G + lane];
        }
        float off[2][2];
        off[0][0] = __shfl_sync(0xffffffffu, my, fc);
        off[0][1] = __shfl_sync(0xffffffffu, my, fc + 1);
        off[1][0] = __shfl_sync(0xffffffffu, my, fc + 8);
        off[1][1] = __shfl_sync(0xffffffffu, my, fc + 9);
        const int xbeg = warp * xr;
#pragma unroll
        for (int blk = 0; blk < kMaxBlocks; ++blk) {
          if (blk < nblk) {
#pragma unroll
            for (int rg = 0; rg < 4; ++rg) {
              const int x = xbeg + blk * 32 + rg * 8 + fr;  // rows fr, fr+8, 16+fr, 24+fr
              if (x < N) {
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                  int2* dst = reinterpret_cast<int2*>(Sc + nt * plane + (x + 1) * kSRow + fc);
                  *dst = make_int2(float_to_int_exact(pre[blk][nt][rg][0] + off[nt][0]),
                                   float_to_int_exact(pre[blk][nt][rg][1] + off[nt][1]));
                }
              }
            }
          }
        }
      }
      if (y + 1 < y0 + ychunk) {  // V: window of row y + 1
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int x = tid + k * kHistThreads;
          const int bo = nxt_out[k] - g0, bi = nxt_in[k] - g0;
          if (x < N && static_cast<unsigned>(bo) < static_cast<unsigned>(G))
            V[x * kVRow + bo] = __hsub(V[x * kVRow + bo], __float2half(1.0f));
          if (x < N && static_cast<unsigned>(bi) < static_cast<unsigned>(G))
            V[x * kVRow + bi] = __hadd(V[x * kVRow + bi], __float2half(1.0f));
        }
        if (y + 2 < y0 + ychunk) fetch(y + 2);
      }
    }
    __syncthreads();  // S of row y and V of row y + 1 complete; WT read
  }
  if (o.sumsq) {
    for (int off = 16; off > 0; off >>= 1) sumsq += __shfl_down_sync(0xffffffffu, sumsq, off);
    if (lane == 0 && sumsq) atomicAdd(o.sumsq + l, sumsq);
  }
}

__global__ void k_cast(const int4* __restrict__ in, long long total, LevelSink o) {
  long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  bool active = i < total;
  int4 v = make_int4(0, 0, 0, 0);
  if (active) {
    v = in[i];
    sink_store(o, i, v);
  }
  sink_sumsq(o, v, active);
}

constexpr int kThreads = 256;

}  // namespace

int launch_bins(const float* d_normal_xy, int N, int bins, uint16_t* d_bins, uint32_t* d_status,
                uint32_t* d_groups, cudaStream_t s) {
  int n = N * N;
  if (d_groups) GSP_CUDA(cudaMemsetAsync(d_groups, 0, kGroupWords * sizeof(uint32_t), s));
  prof_begin(PROF_BINS, s);
  k_bin_normals<<<grid_for(n, kThreads), kThreads, 0, s>>>(
      reinterpret_cast<const float2*>(d_normal_xy), n, bins, d_bins, d_status, d_groups);
  prof_end(PROF_BINS, s);
  GSP_CHECK_LAUNCH();
  return GSP_OK;
}

size_t box_hist_smem(int N) {
  return static_cast<size_t>(N < 32 ? 32 : N) * kVRow * sizeof(__half) +
         4 * static_cast<size_t>(s_plane_ints(N)) * sizeof(int);
}

int launch_box_hist(const uint16_t* d_bins, int N, int levels, int B2, const HistOut& o,
                    cudaStream_t s) {
  if (B2 % kHistG) return GSP_ERR_UNSUPPORTED;
  // Rows per CTA: of 256, 128 and 64 (at most N), the largest whose grid fills
  // the waves of one-CTA-per-SM residency to at least 90 %, else the best
  // filling one (the window fill, at most N rows of 2-byte L2 reads, is small
  // next to 64 rows of output).
  const int sms = sm_count();
  int ychunk = N >= 256 ? 256 : N;
  double best = -1.0;
  for (int yc = ychunk; yc >= 64; yc >>= 1) {
    const long long ctas = static_cast<long long>(B2 / kHistG) * (N / yc) * levels;
    const long long waves = (ctas + sms - 1) / sms;
    const double fill = static_cast<double>(ctas) / static_cast<double>(waves * sms);
    if (fill > best + 1e-9) {
      best = fill;
      ychunk = yc;
    }
    if (fill >= 0.9) break;
  }
  const size_t smem = box_hist_smem(N);
  if (smem > 227 * 1024) return GSP_ERR_UNSUPPORTED;
  dim3 grid(B2 / kHistG, N / ychunk, levels);
  GSP_CUDA(cudaFuncSetAttribute(k_box_hist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(smem)));
  prof_begin(PROF_DOUBLE, s);
  k_box_hist<<<grid, kHistThreads, smem, s>>>(d_bins, ilog2(N), B2, ychunk, o);
  prof_end(PROF_DOUBLE, s);
  GSP_CHECK_LAUNCH();
  return GSP_OK;
}

int launch_cast(const int32_t* d_in, int N, int bins, LevelSink o, cudaStream_t s) {
  long long total = static_cast<long long>(N) * N * bins * bins / 4;
  prof_begin(PROF_CAST, s);
  k_cast<<<grid_for(total, kThreads), kThreads, 0, s>>>(reinterpret_cast<const int4*>(d_in), total,
                                                        o);
  prof_end(PROF_CAST, s);
  GSP_CHECK_LAUNCH();
  return GSP_OK;
}

}  // namespace gsp

using namespace gsp;

extern "C" int gsp_bin_normals(const float* d_normal_xy, int N, int bins, uint16_t* d_bins,
                               uint32_t* d_status, gsp_stream stream) {
  if (!d_normal_xy || !d_bins || !is_pow2(N) || N < 2 || N > 1024 || !is_pow2(bins) ||
      bins < 4 || bins > 128)
    return GSP_ERR_INVALID_ARG;
  return launch_bins(d_normal_xy, N, bins, d_bins, d_status, nullptr, to_stream(stream));
}

extern "C" size_t gsp_build_workspace_bytes(int N, int levels, int bins) {
  if (!valid_map(N, levels, bins)) return 0;
  return align_up(static_cast<size_t>(N) * N * sizeof(uint16_t), 256) + kGroupBytes;
}

extern "C" int gsp_build_footprint_ndfs(const float* d_normal_xy, int N, int levels, int bins,
                                        int32_t* d_hist, void* d_ws, size_t ws_bytes,
                                        uint32_t* d_status, gsp_stream stream) {
  if (!d_normal_xy || !d_hist || !valid_map(N, levels, bins)) return GSP_ERR_INVALID_ARG;
  if (!d_ws || ws_bytes < gsp_build_workspace_bytes(N, levels, bins)) return GSP_ERR_WORKSPACE;
  cudaStream_t s = to_stream(stream);
  uint16_t* bins_map = static_cast<uint16_t*>(d_ws);
  uint32_t* groups = reinterpret_cast<uint32_t*>(
      static_cast<char*>(d_ws) + align_up(static_cast<size_t>(N) * N * sizeof(uint16_t), 256));
  GSP_TRY(launch_bins(d_normal_xy, N, bins, bins_map, d_status, groups, s));
  HistOut o{};
  o.h = d_hist;
  o.groups = groups;
  for (int l = 0; l < levels; ++l) o.scale[l] = 1.0f;
  return launch_box_hist(bins_map, N, levels, bins * bins, o, s);
}
