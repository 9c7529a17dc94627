// Rows a1-a3: binning of the normal map and exhaustive multi-level footprint
// histograms (Sec. 4.1), written straight into int32 counts and/or the
// scaled MTTKRP operand.
//
// Every level is computed from the 2-byte bin map alone (it stays in L2) by
// box sums of per-bin indicators staged in shared memory, so the only HBM
// traffic is the output itself.  Every value is an integer count, exact in
// the types it passes through (FP16 <= 2^11, FP32 < 2^24), hence bit-exact.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include <cstring>
#include <type_traits>

#include "ndf_build.cuh"

namespace gsp {

// The driver's tensor-map encoder (mttkrp_tc.cu), null without a driver.
PFN_cuTensorMapEncodeTiled_v12000 encode_fn();

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
    const uint32_t rb = bf16_pair_bits(static_cast<unsigned long long>(o.base + 4 * i));
    p.x = bf16_pair_dither(f0, f1, rb);
    p.y = bf16_pair_dither(f2, f3, rb + kWeyl);
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
// [y - a, y - a + w) (w = 2^l, a = w/2, wrapped), exact FP16 counts (<= 2^10).
// Moving from row y to y + 1 removes one texel and adds one per column.  The
// counts of the footprints of row y are window sums of V along x, taken by
// warp MMAs: the 16 footprints x = X0 + i (i < 16) have the window columns
// s0 + i + [0, w), s0 = X0 - a, so that
//     C = A1 V[s0, s0 + 16) + A2 V[s0 + w2, s0 + w2 + 16) + M,
//     A1[i][j] = [i <= j < i + w],  A2[i][j] = [w2 + j < i + w],  w2 = max(w, 16),
// with M the sum of V over [s0 + 16, s0 + w) (w > 16): whole 16-column tiles
// (s0 is a multiple of 16 there), added from per-tile totals TT of V.  Every
// product is a count times 0 or 1 and every partial sum an integer below
// 2^24, exact in FP32 whatever the order.  The accumulator starts at
// M + 2^23, so that the FP32 bits of the result are 0x4B000000 + count.
//  - warp w owns a contiguous range of columns: it updates their V and TT
//    (the TT by shared-memory integer reductions) and computes the footprints
//    x of that range, so one barrier separates the reads of V and TT from
//    their update and one the update from the next row's reads;
//  - V rows are 32 bytes with 16 bytes of padding after every 4 columns, so
//    that the ldmatrix row reads of 8 consecutive columns (from a multiple of
//    4) and the window updates of the lanes (each owning 1, 2 or 4 adjacent
//    columns) spread over the banks;
//  - BF16 results go by stmatrix into a per-warp staging buffer in the same
//    swizzle (the TMA 32-byte swizzle) and out by one TMA bulk store per warp
//    and row; the other outputs are stored from the accumulator fragments.
constexpr int kBhG = 16;
constexpr int kBhThreads = 256;
constexpr int kBhWarps = kBhThreads / 32;
constexpr int kBhCtasPerSm = 3;
constexpr int kTTRow = 20;     // ints per tile-total row (16 + 4 padding)
constexpr int kFillRows = 16;  // window rows loaded per batch of the fill
constexpr int kBhRows = 32;    // rows per CTA, and per block of the column prefix sums

// Columns owned by one warp (N <= 1024): N / 8 from N = 128 on, else 16 (the
// first N / 16 warps) or N (one warp, N < 16).
__host__ __device__ constexpr int bh_cols_per_warp(int N) {
  return N >= 128 ? N / kBhWarps : (N >= 16 ? 16 : N);
}

// Byte offset of column x of V (32-byte rows, 16 bytes of padding after every 4).
__host__ __device__ constexpr uint32_t v_off(int x) {
  return static_cast<uint32_t>(x) * 32u + static_cast<uint32_t>(x >> 2) * 16u;
}

// Byte offset of half h (bins 8h .. 8h + 7) of row x in a buffer of 32-byte
// rows (16 BF16 values), halves swapped on bit 2 of x: the 32-byte TMA swizzle.
__device__ __forceinline__ uint32_t row32_off(int x, int h) {
  return static_cast<uint32_t>(x) * 32u + static_cast<uint32_t>((h ^ (x >> 2)) & 1) * 16u;
}

// Position of bin b in a tile-total row: the bins fc, fc + 1, fc + 8, fc + 9
// of the accumulator lanes with fc = 2g are the 4 ints at 4g.
__device__ __forceinline__ int tt_pos(int b) { return 4 * ((b & 7) >> 1) + 2 * (b >> 3) + (b & 1); }

// Four 8x8 b16 matrices from shared memory, transposed into the B-fragment
// layout of mma.m16n8k16 (lanes 8i..8i+7 give the row addresses of matrix i).
__device__ __forceinline__ void ldsm_x4_trans(uint32_t addr, uint32_t (&r)[4]) {
  asm("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
      : "r"(addr)
      : "memory");
}

// Four 8x8 b16 matrices in the accumulator-fragment layout (lane: row lane/4,
// elements 2 (lane%4) and +1) to shared memory (lanes 8i..8i+7: rows of matrix i).
__device__ __forceinline__ void stsm_x4(uint32_t addr, uint32_t r0, uint32_t r1, uint32_t r2,
                                        uint32_t r3) {
  asm volatile("stmatrix.sync.aligned.m8n8.x4.shared.b16 [%0], {%1, %2, %3, %4};" ::"r"(addr),
               "r"(r0), "r"(r1), "r"(r2), "r"(r3)
               : "memory");
}

// D = A B + C, A 16x16 and B 16x8 FP16, C and D FP32 (warp-level MMA).
__device__ __forceinline__ void mma_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                          uint32_t b1, const float (&c)[4]) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
      "{%8, %9}, {%10, %11, %12, %13};"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(c[0]), "f"(c[1]),
        "f"(c[2]), "f"(c[3]));
}

// (x, y) * s + nb in one packed FP32 instruction, each lane rounded once.
__device__ __forceinline__ float2 fma2(float x, float y, float s, float nb) {
  unsigned long long v, sv, nv, r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(v) : "f"(x), "f"(y));
  asm("mov.b64 %0, {%1, %1};" : "=l"(sv) : "f"(s));
  asm("mov.b64 %0, {%1, %1};" : "=l"(nv) : "f"(nb));
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(v), "l"(sv), "l"(nv));
  float2 o;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(o.x), "=f"(o.y) : "l"(r));
  return o;
}

// (x, y) += (a, b) in one packed FP32 instruction, each lane rounded once.
__device__ __forceinline__ void add2(float& x, float& y, float a, float b) {
  unsigned long long v, u, r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(v) : "f"(x), "f"(y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(u) : "f"(a), "f"(b));
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(v), "l"(u));
  asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(r));
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, uint32_t src, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(src), "r"(c0), "r"(c1)
      : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// The staging buffer may be written again once the copies have read it.
__device__ __forceinline__ void bulk_wait_read0() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait0() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}
// Generic-proxy writes of shared memory made visible to the TMA (async proxy).
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// The bin codes of CPL consecutive columns (CPL = 1, 2, 4) of one row, packed
// as in memory; missing ones read 0xFFFF (no bin).
template <int CPL>
__device__ __forceinline__ uint2 load_codes(const uint16_t* p) {
  if constexpr (CPL == 1) {
    return make_uint2(0xFFFF0000u | __ldg(p), 0xFFFFFFFFu);
  } else if constexpr (CPL == 2) {
    return make_uint2(__ldg(reinterpret_cast<const unsigned int*>(p)), 0xFFFFFFFFu);
  } else {
    return __ldg(reinterpret_cast<const uint2*>(p));
  }
}
__device__ __forceinline__ int code_at(uint2 v, int c) {
  const uint32_t u = c < 2 ? v.x : v.y;
  return static_cast<int>((c & 1) ? u >> 16 : u & 0xFFFFu);
}

// V[x][b] += d (one owner thread per column x).
__device__ __forceinline__ void v_add(uint8_t* Vb, int x, int b, __half d) {
  __half* p = reinterpret_cast<__half*>(Vb + v_off(x) + 2 * b);
  *p = __hadd(*p, d);
}

// Column prefix sums over blocks of kBhRows rows, the starting windows of the
// coarse levels: P[k][x][b] = number of texels of bin b in column x among the
// rows [0, k kBhRows), k = 0 .. N / kBhRows, as exact FP16 counts (<= N <=
// 1024).  First the count of each block (thread: column x, block k, 16-bin
// group; counts of 2 bins per 32-bit word), then the running sum over k in
// place.
__global__ void k_col_blocks(const uint16_t* __restrict__ bins_map, int logN, int B2,
                             const uint32_t* __restrict__ groups, __half* __restrict__ P) {
  const int N = 1 << logN;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y, g = blockIdx.z;
  if (x >= N || (groups && !((groups[g >> 5] >> (g & 31)) & 1u))) return;
  const int g0 = g * 16;
  uint32_t cnt[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
#pragma unroll 8
  for (int r = 0; r < kBhRows; ++r) {
    const int b = static_cast<int>(__ldg(bins_map + ((kBhRows * k + r) << logN) + x)) - g0;
    const uint32_t inc = static_cast<unsigned>(b) < 16u ? 1u << ((b & 1) << 4) : 0u;
#pragma unroll
    for (int q = 0; q < 8; ++q) cnt[q] += q == (b >> 1) ? inc : 0u;
  }
  // count c (< 1024) as FP16: the bits of 1024 + c are 0x6400 + c; minus 1024
  uint32_t hw[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const __half2 v = __hsub2(__halves2half2(__ushort_as_half(static_cast<unsigned short>(0x6400u + (cnt[q] & 0xFFFFu))),
                                             __ushort_as_half(static_cast<unsigned short>(0x6400u + (cnt[q] >> 16)))),
                              __float2half2_rn(1024.0f));
    hw[q] = *reinterpret_cast<const uint32_t*>(&v);
  }
  uint4* dst = reinterpret_cast<uint4*>(P + (static_cast<long long>(k + 1) * N + x) * B2 + g0);
  dst[0] = make_uint4(hw[0], hw[1], hw[2], hw[3]);
  dst[1] = make_uint4(hw[4], hw[5], hw[6], hw[7]);
  if (k == 0) {
    uint4* z = reinterpret_cast<uint4*>(P + static_cast<long long>(x) * B2 + g0);
    z[0] = z[1] = make_uint4(0u, 0u, 0u, 0u);
  }
}

// Thread: column x, half h (8 bins) of a 16-bin group; rows k = 1 .. N / kBhRows
// in batches of 8 loads in flight.
__global__ void k_col_prefix(int logN, int B2, const uint32_t* __restrict__ groups,
                             __half* __restrict__ P) {
  const int N = 1 << logN, K = N / kBhRows;
  const int t = blockIdx.x * blockDim.x + threadIdx.x, g = blockIdx.y;
  if (t >= 2 * N || (groups && !((groups[g >> 5] >> (g & 31)) & 1u))) return;
  const int x = t >> 1, h = t & 1;
  uint4* col = reinterpret_cast<uint4*>(P + static_cast<long long>(x) * B2 + g * 16 + 8 * h);
  const long long stride = static_cast<long long>(N) * B2 / 8;  // uint4 per P row
  __half2 acc[4] = {__float2half2_rn(0.f), __float2half2_rn(0.f), __float2half2_rn(0.f),
                    __float2half2_rn(0.f)};
  for (int k0 = 1; k0 <= K; k0 += 8) {
    uint4 v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (k0 + j <= K) v[j] = col[(k0 + j) * stride];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (k0 + j <= K) {
        __half2* a = reinterpret_cast<__half2*>(&v[j]);
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = acc[i] = __hadd2(acc[i], a[i]);
        col[(k0 + j) * stride] = v[j];
      }
    }
  }
}

// Output of one launch: exactly one of int32 counts, FP32 values, BF16 values
// (through the TMA), or none (sums of squares only).
enum BhMode { kBhSumsq = 0, kBhBf16 = 1, kBhF32 = 2, kBhInt = 3 };

// Zero counts for a CTA whose 16-bin group holds no texel of the map.
__device__ void box_hist_zero(int logN, int B2, int ychunk, int y0, int l, int g0,
                              const HistOut& o) {
  const int N = 1 << logN;
  const int row_log = logN + 1;  // N * (16 / 8) items of 8 bins per row
  const long long items = static_cast<long long>(ychunk) << row_log;
  const uint4 z4 = make_uint4(0u, 0u, 0u, 0u);
  for (long long e = threadIdx.x; e < items; e += kBhThreads) {
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
}

// CPL: columns per lane (N / 256 for N >= 512, else 1).  MODE kBhInt writes
// counts only; the others add the sums of squares to o.sumsq.  kBhBf16 writes
// through `tmap`: the BF16 tensor as [levels * N * N][B2], box 16 bins x
// bh_cols_per_warp(N) rows, 32-byte swizzle.
template <int CPL, int MODE>
__global__ void __launch_bounds__(kBhThreads, kBhCtasPerSm)
    k_box_hist(const uint16_t* __restrict__ bins_map, int logN, int B2, int ychunk,
               const __grid_constant__ HistOut o, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ uint8_t smem_raw[];
  const int N = 1 << logN, m = N - 1;
  const int g0 = blockIdx.x * kBhG;
  const int y0 = blockIdx.y * ychunk;
  const int l = gridDim.z - 1 - blockIdx.z;  // coarsest level first: its window fill is the longest
  const int w = 1 << l, a = w >> 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr bool kSumsq = MODE != kBhInt;  // the counts alone carry no sums of squares
  if (o.groups && !((o.groups[blockIdx.x >> 5] >> (blockIdx.x & 31)) & 1u)) {
    if (MODE != kBhSumsq) box_hist_zero(logN, B2, ychunk, y0, l, g0, o);
    return;
  }
  const int cw = bh_cols_per_warp(N);
  const int T = N >= 16 ? N >> 4 : 1;  // 16-column tiles
  const int xw = warp * cw;            // first column of this warp
  const bool owner = xw < N;
  const bool lane_cols = owner && lane * CPL < cw;
  const int xl = xw + lane * CPL;  // first column of this lane
  const int ntile = cw >= 16 ? cw >> 4 : 1;
  const int vcols = N < 16 ? 16 : N;
  const uint32_t raw_s = static_cast<uint32_t>(__cvta_generic_to_shared(smem_raw));
  const uint32_t pad = (1024u - (raw_s & 1023u)) & 1023u;
  const uint32_t srow_bytes = static_cast<uint32_t>((cw < 16 ? 16 : cw) * 32);  // staging per warp
  const uint32_t stage_bytes = MODE == kBhBf16 ? kBhWarps * srow_bytes : 0u;
  uint8_t* Vb = smem_raw + pad + stage_bytes;
  int* TT = reinterpret_cast<int*>(Vb + v_off(vcols));  // [T][kTTRow] tile totals of V (tt_pos order)
  const uint32_t v_s = raw_s + pad + stage_bytes;
  const uint32_t st_s = raw_s + pad + static_cast<uint32_t>(warp) * srow_bytes;

  for (int i = threadIdx.x; i < static_cast<int>(v_off(vcols) / 16); i += kBhThreads)
    reinterpret_cast<uint4*>(Vb)[i] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  const __half one = __float2half(1.0f), mone = __float2half(-1.0f);
  if (lane_cols && o.colp && a >= kBhRows) {
    // window rows [s, s + w) of row y0, s a multiple of kBhRows: differences
    // of the column prefix sums (all counts <= N, exact in FP16)
    const int K = N / kBhRows;
    const int s = (y0 - a) & m, e = s + w;
    const int ks = s / kBhRows, ke = e <= N ? e / kBhRows : K, kw = e > N ? (e - N) / kBhRows : -1;
#pragma unroll 1
    for (int c = 0; c < CPL; ++c) {
      const __half* col = o.colp + static_cast<long long>(xl + c) * B2 + g0;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const long long rs = static_cast<long long>(N) * B2;
        uint4 vs = *reinterpret_cast<const uint4*>(col + ks * rs + 8 * h);
        uint4 ve = *reinterpret_cast<const uint4*>(col + ke * rs + 8 * h);
        __half2* pe = reinterpret_cast<__half2*>(&ve);
        const __half2* ps = reinterpret_cast<const __half2*>(&vs);
#pragma unroll
        for (int i = 0; i < 4; ++i) pe[i] = __hsub2(pe[i], ps[i]);
        if (kw >= 0) {
          uint4 vw = *reinterpret_cast<const uint4*>(col + kw * rs + 8 * h);
          const __half2* pw = reinterpret_cast<const __half2*>(&vw);
#pragma unroll
          for (int i = 0; i < 4; ++i) pe[i] = __hadd2(pe[i], pw[i]);
        }
        *reinterpret_cast<uint4*>(Vb + v_off(xl + c) + 16 * h) = ve;
      }
    }
  } else if (lane_cols) {
    // the window rows of row y0, kFillRows rows of loads in flight
    for (int j0 = 0; j0 < w; j0 += kFillRows) {
      uint2 raw[kFillRows];
#pragma unroll
      for (int u = 0; u < kFillRows; ++u)
        raw[u] = j0 + u < w ? load_codes<CPL>(bins_map + (((y0 - a + j0 + u) & m) << logN) + xl)
                            : make_uint2(0xFFFFFFFFu, 0xFFFFFFFFu);
#pragma unroll
      for (int u = 0; u < kFillRows; ++u) {
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          const int b = code_at(raw[u], c) - g0;
          if (static_cast<unsigned>(b) < static_cast<unsigned>(kBhG)) v_add(Vb, xl + c, b, one);
        }
      }
    }
  }

  const int fr = lane >> 2, fc = 2 * (lane & 3);  // accumulator row / column pair of this lane
  // row and half of the 8x8 matrices this lane addresses in ldmatrix /
  // stmatrix: matrix q = lane / 8 covers rows (q & 1) * 8 .. + 7 and bins
  // (q >> 1) * 8 .. + 7 of a 16 x 16 block
  const int lrow = ((lane >> 3) & 1) * 8 + (lane & 7), lhalf = lane >> 4;
  const bool need_tt = l >= 5;  // whole tiles inside the window
  const float kOff = 8388608.0f;  // 2^23
  const uint32_t kOffBits = 0x4B000000u;
  const float off4[4] = {kOff, kOff, kOff, kOff}, zero4[4] = {0.f, 0.f, 0.f, 0.f};
  if (need_tt && owner) {  // tile totals of row y0: an all-ones A times each tile
    __syncwarp();
    uint32_t ones[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) ones[i] = 0x3C003C00u;
    for (int k = 0; k < ntile; ++k) {
      const int x0 = xw + 16 * k;
      uint32_t bv[4];
      ldsm_x4_trans(v_s + v_off(x0 + lrow) + 16 * lhalf, bv);
      float t0[4], t1[4];
      mma_16816(t0, ones, bv[0], bv[1], off4);
      mma_16816(t1, ones, bv[2], bv[3], off4);
      if (lane < 4)  // bins fc, fc + 1, fc + 8, fc + 9 at tt_pos
        *reinterpret_cast<int4*>(TT + (x0 >> 4) * kTTRow + 4 * lane) =
            make_int4(static_cast<int>(__float_as_uint(t0[0]) - kOffBits),
                      static_cast<int>(__float_as_uint(t0[1]) - kOffBits),
                      static_cast<int>(__float_as_uint(t1[0]) - kOffBits),
                      static_cast<int>(__float_as_uint(t1[1]) - kOffBits));
    }
  }

  // A fragments (row-major 16 x 16 FP16; lane: rows fr, fr + 8, columns fc,
  // fc + 1 and fc + 8, fc + 9) of the two window matrices
  const int w2 = w > 16 ? w : 16;
  uint32_t A1[4], A2[4];
  {
    auto a1 = [&](int i, int j) -> uint32_t { return (i <= j && j < i + w) ? 0x3C00u : 0u; };
    auto a2 = [&](int i, int j) -> uint32_t { return (w2 + j < i + w) ? 0x3C00u : 0u; };
    A1[0] = a1(fr, fc) | (a1(fr, fc + 1) << 16);
    A1[1] = a1(fr + 8, fc) | (a1(fr + 8, fc + 1) << 16);
    A1[2] = a1(fr, fc + 8) | (a1(fr, fc + 9) << 16);
    A1[3] = a1(fr + 8, fc + 8) | (a1(fr + 8, fc + 9) << 16);
    A2[0] = a2(fr, fc) | (a2(fr, fc + 1) << 16);
    A2[1] = a2(fr + 8, fc) | (a2(fr + 8, fc + 1) << 16);
    A2[2] = a2(fr, fc + 8) | (a2(fr, fc + 9) << 16);
    A2[3] = a2(fr + 8, fc + 8) | (a2(fr + 8, fc + 9) << 16);
  }
  // This lane's ldmatrix rows of the two column ranges of the warp's first
  // tile: a byte offset into V that advances by 16 columns (v_off(16) bytes)
  // per tile, modulo the N columns (v_off(N) bytes), plus the bin half.
  const int x1 = (xw - a + lrow) & m, x2 = (xw - a + w2 + lrow) & m;
  const uint32_t vend = v_off(N), vstep = v_off(16);
  const uint32_t va = v_s + 16u * static_cast<uint32_t>(lhalf);
  const uint32_t vo1 = v_off(x1), vo2 = v_off(x2);
  // stmatrix row of this lane in the staging buffer (tile k adds 512 bytes)
  const uint32_t st_lane = st_s + row32_off(lrow, lhalf);

  // codes leaving / entering the window at the next row step, loaded one row
  // ahead so the L2 latency overlaps this row's work
  uint2 nxt_out = make_uint2(0xFFFFFFFFu, 0xFFFFFFFFu), nxt_in = nxt_out;
  auto fetch = [&](int yn) {
    if (lane_cols) {
      nxt_out = load_codes<CPL>(bins_map + (((yn - 1 - a) & m) << logN) + xl);
      nxt_in = load_codes<CPL>(bins_map + (((yn - 1 - a + w) & m) << logN) + xl);
    }
  };
  if (ychunk > 1 && w < N) fetch(y0 + 1);

  const float sc = o.scale[l];
  const float nb = -kOff * sc;  // -2^23 * scale, exact
  const uint32_t dK8r = static_cast<uint32_t>(8 * B2) * kWeyl;    // dither step of 8 rows
  const uint32_t dKtile = static_cast<uint32_t>(16 * B2) * kWeyl;  // ... and of one tile
  const uint32_t dP8r = static_cast<uint32_t>(4 * B2) * kWeyl;    // pair dither: 8 rows
  const uint32_t dPtile = static_cast<uint32_t>(8 * B2) * kWeyl;  // ... and one tile
  const int ta = a >> 4, wt = w >> 4;                              // in tiles (l >= 5)
  const int* tt_lane = TT + 2 * fc;  // this lane's 4 bins of a tile-total row
  unsigned long long sumsq = 0;
  __syncthreads();  // V and TT of row y0 complete

  const bool sliding = w < N;  // else every window is the whole map
  // One row of footprints for the level class LC of l (compile-time, so the
  // tile loop has no level branches): 0: l <= 4 (counts <= 256, exact in BF16;
  // no whole tiles in the window), 1: 5 <= l <= 7 (squares of 8 counts fit 32
  // bits), 2: l >= 8, 3: w = N >= 32 (the counts Dc of every tile).
  auto row_out = [&](int y, auto lc_tag, const float (&Dc)[2][4], unsigned long long qc) {
    constexpr int LC = decltype(lc_tag)::value;
    // middle sums of the warp's first tile: the 8 lanes of one column pair
    // take every 8th tile, then add up
    uint32_t Mb[4] = {0u, 0u, 0u, 0u};  // bins fc, fc + 1, fc + 8, fc + 9
    if constexpr (LC == 1 || LC == 2) {
      const int u0 = (xw >> 4) - ta + 1;
      for (int q = fr; q < wt - 1; q += 8) {
        const int4 p = *reinterpret_cast<const int4*>(tt_lane + ((u0 + q) & (T - 1)) * kTTRow);
        Mb[0] += p.x; Mb[1] += p.y; Mb[2] += p.z; Mb[3] += p.w;
      }
#pragma unroll
      for (int off = 4; off < 32; off <<= 1)
#pragma unroll
        for (int i = 0; i < 4; ++i) Mb[i] += __shfl_xor_sync(0xffffffffu, Mb[i], off);
    }
    // FP32 bits of 2^23 + M, added to the accumulators of both rows fr, fr + 8
#pragma unroll
    for (int i = 0; i < 4; ++i) Mb[i] += kOffBits;
    if (MODE == kBhBf16 && y > y0) {  // the previous row's store has read the staging buffer
      if (lane == 0) bulk_wait_read0();
      __syncwarp();
    }
    const long long e_row = (static_cast<long long>(l) * N + y) * N;  // footprint index of x = 0
    // element index of (x = xw + fr, bin g0 + fc), its Weyl value (TF32) and
    // that of its pair (BF16)
    const long long e_lane = (e_row + xw + fr) * B2 + g0 + fc;
    uint32_t d00 = MODE == kBhF32 ? static_cast<uint32_t>(e_lane) * kWeyl : 0u;
    uint32_t p00 = MODE == kBhBf16 ? static_cast<uint32_t>(e_lane >> 1) * kWeyl : 0u;
    (void)d00;
    (void)p00;
    uint32_t o1 = vo1, o2 = vo2;
    // 4 tiles in flight for the BF16 operand (2 in the other modes, whose
    // direct stores need the registers)
#pragma unroll(MODE == kBhBf16 ? 4 : 2)
    for (int k = 0; k < ntile; ++k) {
      float D[2][4];
      if constexpr (LC == 3) {
#pragma unroll
        for (int n = 0; n < 2; ++n)
#pragma unroll
          for (int i = 0; i < 4; ++i) D[n][i] = Dc[n][i];
      } else {
        uint32_t bA[4], bB[4];
        ldsm_x4_trans(va + o1, bA);
        ldsm_x4_trans(va + o2, bB);
        o1 += vstep;
        o2 += vstep;
        if (o1 >= vend) o1 -= vend;
        if (o2 >= vend) o2 -= vend;
        if constexpr (LC == 0) {  // no middle sums: the accumulators start at 2^23
          mma_16816(D[0], A1, bA[0], bA[1], off4);
          mma_16816(D[1], A1, bA[2], bA[3], off4);
        } else {
          mma_16816(D[0], A1, bA[0], bA[1], zero4);
          mma_16816(D[1], A1, bA[2], bA[3], zero4);
        }
        mma_16816(D[0], A2, bB[0], bB[1], D[0]);
        mma_16816(D[1], A2, bB[2], bB[3], D[1]);
        if constexpr (LC >= 1) {
          // + (2^23 + M), exact (integers below 2^24), two rows per packed add
#pragma unroll
          for (int n = 0; n < 2; ++n)
#pragma unroll
            for (int r = 0; r < 2; ++r)
              add2(D[n][2 * r], D[n][2 * r + 1], __uint_as_float(Mb[2 * n]), __uint_as_float(Mb[2 * n + 1]));
          if (k + 1 < ntile) {  // middle sums of the next tile
            const int t = (xw >> 4) + k;
            const int4 lo = *reinterpret_cast<const int4*>(tt_lane + ((t - ta + 1) & (T - 1)) * kTTRow);
            const int4 hi = *reinterpret_cast<const int4*>(tt_lane + ((t - ta + wt) & (T - 1)) * kTTRow);
            Mb[0] += hi.x - lo.x; Mb[1] += hi.y - lo.y;
            Mb[2] += hi.z - lo.z; Mb[3] += hi.w - lo.w;
          }
        }
      }
      // D[n][2r + e]: bits 0x4B000000 + count of footprint x = X0 + fr + 8r, bin g0 + 8n + fc + e
      if constexpr (kSumsq && LC == 3) {
        sumsq += qc;
      } else if constexpr (kSumsq) {
        if constexpr (LC <= 1) {
          // counts <= 4^7: the eight squares of a tile sum below 2^32, so they
          // may be formed modulo 2^32 from the FP32 bits u = K + c (K =
          // 0x4B000000): c^2 = u u - 2K u + K^2, two multiply-adds per count
          uint32_t q = 8u * (kOffBits * kOffBits);
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const uint32_t u = __float_as_uint(D[i >> 2][i & 3]);
            asm("mad.lo.u32 %0, %1, %1, %0;" : "+r"(q) : "r"(u));
            asm("mad.lo.u32 %0, %1, %2, %0;" : "+r"(q) : "r"(u), "r"(0u - 2u * kOffBits));
          }
          sumsq += q;
        } else {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const uint32_t c = __float_as_uint(D[i >> 2][i & 3]) - kOffBits;
            sumsq += static_cast<unsigned long long>(c) * c;
          }
        }
      }
      if constexpr (MODE == kBhBf16 || MODE == kBhF32) {
        // c * scale, exactly: (2^23 + c) * scale - 2^23 * scale in one rounding
        float2 f[2][2];
#pragma unroll
        for (int n = 0; n < 2; ++n)
#pragma unroll
          for (int r = 0; r < 2; ++r) f[n][r] = fma2(D[n][2 * r], D[n][2 * r + 1], sc, nb);
        // Weyl values of element (n, r, e): d00 + r * dK8r + (8n + e) * kWeyl
        // (TF32); of its pair: p00 + r * dP8r + 4n * kWeyl (BF16)
        if constexpr (MODE == kBhBf16) {
          uint32_t wd[2][2];
#pragma unroll
          for (int n = 0; n < 2; ++n)
#pragma unroll
            for (int r = 0; r < 2; ++r) {
              if constexpr (LC == 0) {  // counts <= 256: exact in BF16
                wd[n][r] = __byte_perm(__float_as_uint(f[n][r].x), __float_as_uint(f[n][r].y), 0x7632);
              } else {
                wd[n][r] = bf16_pair_dither(
                    f[n][r].x, f[n][r].y, p00 + (r ? dP8r : 0u) + static_cast<uint32_t>(4 * n) * kWeyl);
              }
            }
          stsm_x4(st_lane + 512u * static_cast<uint32_t>(k), wd[0][0], wd[0][1], wd[1][0], wd[1][1]);
        } else {
          const long long e00 = (e_row + xw + 16 * k + fr) * B2 + g0 + fc;
#pragma unroll
          for (int n = 0; n < 2; ++n)
#pragma unroll
            for (int r = 0; r < 2; ++r) {
              float2 v = f[n][r];
              if (o.tf32 && l >= 6) {  // counts <= 4^5 are exact on the TF32 grid
                const uint32_t d = d00 + (r ? dK8r : 0u) + static_cast<uint32_t>(8 * n) * kWeyl;
                v = make_float2(tf32_dither(v.x, d), tf32_dither(v.y, d + kWeyl));
              }
              if (N >= 16 || fr + 8 * r < N)
                *reinterpret_cast<float2*>(o.f32 + e00 + r * 8LL * B2 + 8 * n) = v;
            }
        }
      } else if constexpr (MODE == kBhInt) {
        const long long e00 = (e_row + xw + 16 * k + fr) * B2 + g0 + fc;
#pragma unroll
        for (int n = 0; n < 2; ++n)
#pragma unroll
          for (int r = 0; r < 2; ++r)
            if (N >= 16 || fr + 8 * r < N)
              *reinterpret_cast<int2*>(o.h + e00 + r * 8LL * B2 + 8 * n) =
                  make_int2(static_cast<int>(__float_as_uint(D[n][2 * r]) - kOffBits),
                            static_cast<int>(__float_as_uint(D[n][2 * r + 1]) - kOffBits));
      }
      if constexpr (MODE == kBhF32) d00 += dKtile;
      if constexpr (MODE == kBhBf16) p00 += dPtile;
    }
    if constexpr (MODE == kBhBf16) {  // this warp's footprints of row y: one bulk store
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) {
        tma_store_2d(&tmap, st_s, g0, static_cast<int>(e_row + xw));
        bulk_commit();
      }
    }
  };
  // V of this lane's columns: bin b of column xl + c at v_col + 32 c + 2 b
  // (the CPL columns lie within one group of 4)
  uint8_t* const v_col = Vb + v_off(xl);
  int* const tr = TT + (xl >> 4) * kTTRow;  // the lane's columns share one tile
  const int lc = !sliding && need_tt ? 3 : (l <= 4 ? 0 : (l <= 7 ? 1 : 2));

  if (lc == 3) {
    // w = N (from l = 5 on): every window is the whole map, so the count of a
    // bin is its total in every footprint, taken from the tile totals once
    if (owner) {
      uint32_t tot[4] = {0u, 0u, 0u, 0u};  // bins fc, fc + 1, fc + 8, fc + 9
      for (int q = fr; q < T; q += 8) {
        const int4 p = *reinterpret_cast<const int4*>(tt_lane + q * kTTRow);
        tot[0] += p.x; tot[1] += p.y; tot[2] += p.z; tot[3] += p.w;
      }
#pragma unroll
      for (int off = 4; off < 32; off <<= 1)
#pragma unroll
        for (int i = 0; i < 4; ++i) tot[i] += __shfl_xor_sync(0xffffffffu, tot[i], off);
      float Dc[2][4];             // accumulator values 2^23 + total of this lane
      unsigned long long qc = 0;  // the sum of their squared counts in one tile
#pragma unroll
      for (int n = 0; n < 2; ++n)
#pragma unroll
        for (int i = 0; i < 4; ++i) Dc[n][i] = __uint_as_float(kOffBits + tot[2 * n + (i & 1)]);
#pragma unroll
      for (int i = 0; i < 4; ++i) qc += 2ull * tot[i] * tot[i];  // rows fr and fr + 8
      for (int y = y0; y < y0 + ychunk; ++y) row_out(y, std::integral_constant<int, 3>{}, Dc, qc);
    }
  } else {
    float D0[2][4];  // unused outside the constant-window path
    // w = N below 32 columns: V and TT never change, no barriers
    for (int y = y0; y < y0 + ychunk; ++y) {
      if (owner) {
        if (lc == 0)
          row_out(y, std::integral_constant<int, 0>{}, D0, 0ull);
        else if (lc == 1)
          row_out(y, std::integral_constant<int, 1>{}, D0, 0ull);
        else
          row_out(y, std::integral_constant<int, 2>{}, D0, 0ull);
      }
      if (!sliding) continue;
      __syncthreads();  // V and TT of row y no longer read
      if (y + 1 < y0 + ychunk) {
        if (lane_cols) {  // V and TT: window of row y + 1
          // predicates and addresses first, then every load, then every store
          // (each column has one owner, so plain read-modify-writes; the tile
          // totals are shared by the lanes of a tile: integer atomics)
          bool po[CPL], pi[CPL];
          int bo[CPL], bi[CPL];
          __half vo[CPL], vi[CPL];
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            const int co = code_at(nxt_out, c), ci = code_at(nxt_in, c);
            bo[c] = co - g0;
            bi[c] = ci - g0;
            po[c] = co != ci && static_cast<unsigned>(bo[c]) < static_cast<unsigned>(kBhG);
            pi[c] = co != ci && static_cast<unsigned>(bi[c]) < static_cast<unsigned>(kBhG);
          }
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            if (po[c]) vo[c] = *reinterpret_cast<const __half*>(v_col + 32 * c + 2 * bo[c]);
            if (pi[c]) vi[c] = *reinterpret_cast<const __half*>(v_col + 32 * c + 2 * bi[c]);
          }
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            if (po[c]) *reinterpret_cast<__half*>(v_col + 32 * c + 2 * bo[c]) = __hadd(vo[c], mone);
            if (pi[c]) *reinterpret_cast<__half*>(v_col + 32 * c + 2 * bi[c]) = __hadd(vi[c], one);
          }
          if (need_tt) {
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
              if (po[c]) atomicAdd(tr + tt_pos(bo[c]), -1);
              if (pi[c]) atomicAdd(tr + tt_pos(bi[c]), 1);
            }
          }
        }
        if (y + 2 < y0 + ychunk) fetch(y + 2);
        __syncthreads();  // V and TT of row y + 1 complete
      }
    }
  }
  if (MODE == kBhBf16 && owner && lane == 0) bulk_wait0();
  if constexpr (kSumsq) {
    for (int off = 16; off > 0; off >>= 1) sumsq += __shfl_down_sync(0xffffffffu, sumsq, off);
    // N < 16: the 16 rows of the one tile hold each footprint 16 / N times
    if (N < 16) sumsq >>= 4 - logN;
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

int launch_col_prefix(const uint16_t* d_bins, int N, int B2, const uint32_t* groups, __half* P,
                      cudaStream_t s) {
  const int logN = ilog2(N);
  const int tb = N < 256 ? N : 256;
  k_col_blocks<<<dim3(N / tb, N / kBhRows, B2 / 16), tb, 0, s>>>(d_bins, logN, B2, groups, P);
  GSP_CHECK_LAUNCH();
  k_col_prefix<<<dim3(2 * N / tb, B2 / 16), tb, 0, s>>>(logN, B2, groups, P);
  GSP_CHECK_LAUNCH();
  return GSP_OK;
}

size_t box_hist_smem(int N, bool bf16) {
  const size_t cw = static_cast<size_t>(bh_cols_per_warp(N));
  const size_t stage = bf16 ? kBhWarps * (cw < 16 ? 16 : cw) * 32 : 0;
  const size_t v = v_off(N < 16 ? 16 : N);
  const size_t tt = static_cast<size_t>(N >= 16 ? N / 16 : 1) * kTTRow * sizeof(int);
  return 1024 + stage + v + tt;  // 1024: alignment of the staging buffers
}

// TMA store map of the BF16 tensor viewed as [rows][B2], box 16 bins x
// box_rows rows, 32-byte swizzle (the staging layout of k_box_hist).
int make_bf16_store_map(CUtensorMap* map, void* base, long long rows, int B2, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return GSP_ERR_UNSUPPORTED;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(B2), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(B2) * 2};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(kBhG), static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                  CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? GSP_OK : GSP_ERR_CUDA;
}

template <int CPL, int MODE>
int launch_box_hist_mode(const uint16_t* d_bins, int N, int B2, int ychunk, dim3 grid, size_t smem,
                         const HistOut& o, const CUtensorMap& tm, cudaStream_t s) {
  GSP_CUDA(cudaFuncSetAttribute(k_box_hist<CPL, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(smem)));
  k_box_hist<CPL, MODE><<<grid, kBhThreads, smem, s>>>(d_bins, ilog2(N), B2, ychunk, o, tm);
  GSP_CHECK_LAUNCH();
  return GSP_OK;
}

template <int CPL>
int launch_box_hist_cpl(const uint16_t* d_bins, int N, int B2, int ychunk, dim3 grid, size_t smem,
                        const HistOut& o, int mode, const CUtensorMap& tm, cudaStream_t s) {
  switch (mode) {
    case kBhBf16: return launch_box_hist_mode<CPL, kBhBf16>(d_bins, N, B2, ychunk, grid, smem, o, tm, s);
    case kBhF32: return launch_box_hist_mode<CPL, kBhF32>(d_bins, N, B2, ychunk, grid, smem, o, tm, s);
    case kBhInt: return launch_box_hist_mode<CPL, kBhInt>(d_bins, N, B2, ychunk, grid, smem, o, tm, s);
    default: return launch_box_hist_mode<CPL, kBhSumsq>(d_bins, N, B2, ychunk, grid, smem, o, tm, s);
  }
}

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

size_t col_prefix_bytes(int N, int B2) {
  if (N < 2 * kBhRows) return 0;  // no level has a window that starts on a block
  return static_cast<size_t>(N / kBhRows + 1) * N * B2 * sizeof(__half);
}

int launch_box_hist(const uint16_t* d_bins, int N, int levels, int B2, const HistOut& o,
                    cudaStream_t s) {
  if (B2 % kBhG || N > 1024) return GSP_ERR_UNSUPPORTED;
  if ((o.h != nullptr) + (o.f32 != nullptr) + (o.bf16 != nullptr) > 1) return GSP_ERR_UNSUPPORTED;
  // int32 counts come without sums of squares, the other modes with them
  if ((o.h != nullptr) == (o.sumsq != nullptr)) return GSP_ERR_UNSUPPORTED;
  const int mode = o.h ? kBhInt : o.f32 ? kBhF32 : o.bf16 ? kBhBf16 : kBhSumsq;
  CUtensorMap tm;
  memset(&tm, 0, sizeof(tm));
  if (mode == kBhBf16) {
    if (reinterpret_cast<uintptr_t>(o.bf16) & 15) return GSP_ERR_UNSUPPORTED;
    GSP_TRY(make_bf16_store_map(&tm, o.bf16, static_cast<long long>(levels) * N * N, B2,
                                bh_cols_per_warp(N)));
  }
  // Rows per CTA: kBhRows (at most N).  The coarsest levels are launched
  // first; with their windows started from the column prefix sums every CTA
  // is kBhRows rows of output plus at most 32 rows of window fill, and the
  // ~4 waves of kBhCtasPerSm CTAs per SM pack well (on the 1024^2, 11-level,
  // 80-column operand: 32 rows 0.69 ms, 64 rows 0.72 ms).
  const int ychunk = N < kBhRows ? N : kBhRows;
  const size_t smem = box_hist_smem(N, mode == kBhBf16);
  if (smem > 227 * 1024) return GSP_ERR_UNSUPPORTED;
  HistOut oo = o;
  if (col_prefix_bytes(N, B2) == 0 || (1 << (levels - 1)) < 2 * kBhRows) oo.colp = nullptr;
  dim3 grid(B2 / kBhG, N / ychunk, levels);
  prof_begin(PROF_DOUBLE, s);  // one interval: the prefix table and the histograms
  int rc = oo.colp ? launch_col_prefix(d_bins, N, B2, o.groups, oo.colp, s) : GSP_OK;
  if (rc == GSP_OK) {
    if (N >= 1024)
      rc = launch_box_hist_cpl<4>(d_bins, N, B2, ychunk, grid, smem, oo, mode, tm, s);
    else if (N >= 512)
      rc = launch_box_hist_cpl<2>(d_bins, N, B2, ychunk, grid, smem, oo, mode, tm, s);
    else
      rc = launch_box_hist_cpl<1>(d_bins, N, B2, ychunk, grid, smem, oo, mode, tm, s);
  }
  prof_end(PROF_DOUBLE, s);
  return rc;
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
  if (!d_normal_xy || !valid_map(N, levels, bins)) return GSP_ERR_INVALID_ARG;
  if (!d_ws || ws_bytes < gsp_build_workspace_bytes(N, levels, bins)) return GSP_ERR_WORKSPACE;
  cudaStream_t s = to_stream(stream);
  uint16_t* bins_map = static_cast<uint16_t*>(d_ws);
  uint32_t* groups = reinterpret_cast<uint32_t*>(
      static_cast<char*>(d_ws) + align_up(static_cast<size_t>(N) * N * sizeof(uint16_t), 256));
  GSP_TRY(launch_bins(d_normal_xy, N, bins, bins_map, d_status, groups, s));
  if (!d_hist) return GSP_OK;  // implicit form: the bin map, every footprint a box count of it
  HistOut o{};
  o.h = d_hist;
  o.groups = groups;
  for (int l = 0; l < levels; ++l) o.scale[l] = 1.0f;
  return launch_box_hist(bins_map, N, levels, bins * bins, o, s);
}
