// tcgen05 tensor-core MTTKRP passes of a CP-ALS sweep (BF16 or TF32 operand,
// FP32 accumulation in tensor memory).
//
// Both passes stream the operand tensor T [l][xy][st] (C order, st = s*B + t
// contiguous) once, in 128-byte-wide tiles loaded by TMA with 128-byte
// swizzling straight into the layout the tensor cores read.
//
//  Y' pass  D[xy][r] = sum_{l, st} T[l][xy][st] * KRt[r][l*B2 + st]
//           one 128-row xy tile per accumulator, K = L * B2; T is the K-major A
//           operand, KRt (fl*fs*ft, built per sweep) the K-major B operand.
//  Z' pass  D[st][r] = sum_y fy[y][r] sum_x T[l][y][x][st] * fx[x][r]
//           per (level, map row, st group); the same T tiles are now the
//           MN-major A operand and FXt (fx, built per sweep) the K-major B
//           operand; fy scales each map row's sums in the epilogue.  For the
//           BF16 hi + lo pair at rank 64 (k_lst_tc_rows) the roles are
//           exchanged, D[r2][st]: FXt's 128 hi and lo rows are the A operand
//           and the stored st columns the MN-major B operand, so no
//           accumulator row is padding.
//
// Accumulation is chunked: the tensor core's FP32 accumulation does not round
// to nearest, and over a chain of thousands of MMAs into one accumulator the
// sums drift low by a few parts in 10^5 (measured: ~5e-8 relative per
// accumulating MMA).  So every chunk (kChunk K steps for Y', one map row for
// Z') starts a fresh TMEM accumulator and the epilogue adds the chunk sums
// with round-to-nearest FP32 operations in a fixed order: for Y' into
// registers, from double-buffered chunk accumulators; for Z' into a
// running-sum region of tensor memory beside the chunk accumulator.
//
// CTA = 6 warps: warps 0-3 epilogue (TMEM lanes 0-127); warp 4 issues TMA;
// warp 5 owns TMEM and issues MMAs (one thread).  Every mbarrier wait is
// bounded by a clock budget: on expiry the CTA raises GSP_DEV_TIMEOUT, waits
// for its own copies and MMAs in flight (again bounded), frees its tensor
// memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "mttkrp.cuh"

namespace gsp {
namespace {

constexpr int kMaxStages = 8;
constexpr int kMaxRankTc = 64;  // CP ranks served by the tensor-core passes
constexpr int kThreads = 192;
constexpr long long kTimeoutCycles = 4000000000LL;  // about 2 s at GB300 clocks
constexpr int kTileBytes = 128 * 128;                // 128 rows x 128 bytes
constexpr int kChunk = 16;  // Y' K steps (4 MMAs each) per tensor-memory accumulator chunk

// ------------------------------------------------------------- PTX glue --
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase of parity `parity` to complete.  Returns false when the
// CTA's abort flag is (or becomes) set or the clock budget runs out.  The
// first test is inlined: the single TMA / MMA issuing threads are on the
// critical path and most of their waits are already satisfied.
__device__ __noinline__ bool mbar_wait_slow(uint32_t a, uint32_t parity, volatile int* abort) {
  const long long t0 = clock64();
  for (;;) {
    if (mbar_test(a, parity)) return true;
    if (*abort) return false;
    if (clock64() - t0 > kTimeoutCycles) {
      *abort = 1;
      return false;
    }
  }
}

__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, volatile int* abort) {
  return mbar_test(a, parity) || mbar_wait_slow(a, parity, abort);
}

// Bounded wait that ignores the abort flag (used to drain work in flight).
__device__ __noinline__ bool mbar_drain(uint32_t a, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_test(a, parity))
    if (clock64() - t0 > kTimeoutCycles) return false;
  return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(mbar)
      : "memory");
}

// tcgen05 shared-memory matrix descriptor, base offset 0.  layout: 2 = 128-byte
// swizzle of 16-byte chunks; 1 = 128-byte swizzle of 32-byte chunks (the form
// MN-major 32-bit operands take).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo,
                                          uint64_t layout = 2) {
  return static_cast<uint64_t>((addr & 0x3FFFFu) >> 4) |
         (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
         (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | (layout << 61);
}

// Instruction descriptor: FP32 accumulator, A/B format (1 = BF16, 2 = TF32),
// A and B major-ness (0 = K-major, 1 = MN-major), M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc(uint32_t fmt, uint32_t a_mn, uint32_t n,
                                             uint32_t b_mn = 0) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | (a_mn << 15) | (b_mn << 16) | ((n >> 3) << 17) |
         ((128u >> 4) << 24);
}

template <int ELEM>
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id,
                                     uint32_t accumulate) {
  if constexpr (ELEM == 2) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(id), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(id), "r"(accumulate)
        : "memory");
  }
}

__device__ __forceinline__ void umma_commit(uint32_t mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t slot_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot_smem),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes, one lane per thread.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// The same load without the wait, so that several can be in flight.
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes from registers.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
      "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15]))
      : "memory");
}

__device__ __forceinline__ void tmem_st_wait() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__host__ __device__ constexpr uint32_t tmem_cols_for(int cols) {
  uint32_t c = 32;
  while (c < static_cast<uint32_t>(cols)) c <<= 1;
  return c;
}

struct Barriers {
  uint64_t full[kMaxStages];
  uint64_t empty[kMaxStages];
  uint64_t acc_full[2];
  uint64_t acc_empty[2];
  uint64_t b_full[kMaxStages];
  uint64_t b_empty[kMaxStages];
  uint64_t drain;
  uint64_t xchg[2];  // rank-row Z' pass: hi sums stored, per segment
  uint32_t tmem_base;
  int abort;
};

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

// ------------------------------------------------------------ Y' pass --
// ELEM: 2 (BF16) or 4 (TF32/FP32 storage).  E128 = elements per 128 bytes.
// SPLIT: the B operand holds 2R rows, a hi part and its remainder (BF16 or
// TF32); each K slice then issues one MMA of N = 2R over both, into an
// accumulator whose columns R .. 2R-1 hold the remainder's sums (one N = 128
// MMA instead of two of N = 64 at rank 64: the tensor pipe was 66 % busy).
template <int ELEM, bool SPLIT>
__global__ void __launch_bounds__(kThreads, 1)
    k_xy_tc(const __grid_constant__ CUtensorMap mapT, const __grid_constant__ CUtensorMap mapKR,
            float* __restrict__ Yp, int n_tiles, long long N2, int L, int B2, int R, int kStages,
            uint32_t* err) {
  constexpr int E128 = 128 / ELEM;
  constexpr uint32_t FMT = ELEM == 2 ? 1u : 2u;
  extern __shared__ uint8_t smem_raw[];
  __shared__ Barriers bar;
  uint8_t* smem = align1024(smem_raw);
  const int b_bytes = R * 128 * (SPLIT ? 2 : 1);
  const int stage_bytes = kTileBytes + b_bytes;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kpl = B2 / E128;  // 128-byte K chunks per level
  const int kiters = L * kpl;
  // SPLIT: one MMA of N = 2R per K slice covers the hi and lo rows of the B
  // tile (they are contiguous), into an accumulator of 2R columns (hi sums,
  // then lo sums) that the epilogue adds; two such chunk accumulators.
  constexpr int AW = SPLIT ? 2 : 1;  // accumulator columns per rank
  const uint32_t ncols = tmem_cols_for(2 * AW * R);
  volatile int* abort = &bar.abort;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(smem_u32(&bar.full[s]), 1);
      mbar_init(smem_u32(&bar.empty[s]), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(smem_u32(&bar.acc_full[a]), 1);
      mbar_init(smem_u32(&bar.acc_empty[a]), 128);
    }
    mbar_init(smem_u32(&bar.drain), 1);
    bar.abort = 0;
    fence_barrier_init();
  }
  if (warp == 5) tmem_alloc(smem_u32(&bar.tmem_base), ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bar.tmem_base;

  if (warp == 4) {
    if (lane == 0) {  // ---- TMA producer
      int s = 0;
      uint32_t ph = 0;
      uint32_t issued_parity[kMaxStages];
      bool issued[kMaxStages];
      for (int i = 0; i < kMaxStages; ++i) issued[i] = false;
      for (int tile = blockIdx.x; tile < n_tiles && !*abort; tile += gridDim.x) {
        // T row of level l: l * N^2 + tile * 128; K column of the KR operand: l * B2 + kc * E128
        int trow = tile * 128, kcol = 0, kc = 0;
        for (int it = 0; it < kiters; ++it) {
          if (!mbar_wait(smem_u32(&bar.empty[s]), ph ^ 1u, abort)) goto producer_done;
          const uint32_t sa = smem_u32(smem + s * stage_bytes);
          const uint32_t fb = smem_u32(&bar.full[s]);
          mbar_expect_tx(fb, stage_bytes);
          tma_load_2d(sa, &mapT, kc * E128, trow, fb);
          tma_load_2d(sa + kTileBytes, &mapKR, kcol, 0, fb);
          kcol += E128;
          if (++kc == kpl) {
            kc = 0;
            trow += static_cast<int>(N2);
          }
          issued[s] = true;
          issued_parity[s] = ph;
          if (++s == kStages) {
            s = 0;
            ph ^= 1u;
          }
        }
      }
    producer_done:
      if (*abort)  // wait for this CTA's own copies still in flight
        for (int i = 0; i < kStages; ++i)
          if (issued[i]) mbar_drain(smem_u32(&bar.full[i]), issued_parity[i]);
    }
  } else if (warp == 5) {
    if (lane == 0) {  // ---- MMA issuer
      const uint32_t id = idesc(FMT, 0, static_cast<uint32_t>(AW * R));
      int s = 0, acc = 0;
      uint32_t ph = 0, aph = 0;
      bool any = false;
      for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        for (int it0 = 0; it0 < kiters; it0 += kChunk) {  // a fresh accumulator per chunk
          if (!mbar_wait(smem_u32(&bar.acc_empty[acc]), aph ^ 1u, abort)) goto mma_done;
          tc_fence_after();
          const uint32_t d = tmem + static_cast<uint32_t>(acc * AW * R);
          const int it1 = it0 + kChunk < kiters ? it0 + kChunk : kiters;
          for (int it = it0; it < it1; ++it) {
            if (!mbar_wait(smem_u32(&bar.full[s]), ph, abort)) goto mma_done;
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + s * stage_bytes);
            // descriptor address fields are in 16-byte units: slice j adds 2 j
            const uint64_t a0 = sdesc(sa, 16, 1024), b0 = sdesc(sa + kTileBytes, 16, 1024);
#pragma unroll
            for (int j = 0; j < 4; ++j)  // four K slices of 32 bytes per 128-byte row
              umma<ELEM>(d, a0 + 2 * j, b0 + 2 * j, id, (it > it0 || j > 0) ? 1u : 0u);
            any = true;
            umma_commit(smem_u32(&bar.empty[s]));
            if (++s == kStages) {
              s = 0;
              ph ^= 1u;
            }
          }
          umma_commit(smem_u32(&bar.acc_full[acc]));
          if (++acc == 2) {
            acc = 0;
            aph ^= 1u;
          }
        }
      }
    mma_done:
      if (*abort && any) {  // wait for the MMAs already issued
        umma_commit(smem_u32(&bar.drain));
        mbar_drain(smem_u32(&bar.drain), 0);
      }
    }
  } else {  // ---- epilogue warps 0-3: chunk sums -> registers -> Y'
    int acc = 0;
    uint32_t aph = 0;
    const int nch = (kiters + kChunk - 1) / kChunk;
    const uint32_t lane_base = tmem + (static_cast<uint32_t>(warp * 32) << 16);
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
      float sum[kMaxRankTc];
#pragma unroll
      for (int i = 0; i < kMaxRankTc; ++i) sum[i] = 0.0f;
      for (int ch = 0; ch < nch; ++ch) {
        if (!mbar_wait(smem_u32(&bar.acc_full[acc]), aph, abort)) goto epi_done;
        tc_fence_after();
#pragma unroll
        for (int c = 0; c < kMaxRankTc / 16; ++c) {
          if (c * 16 < R) {
            const uint32_t col = static_cast<uint32_t>(acc * AW * R + c * 16);
            if constexpr (SPLIT) {  // hi sums + lo sums
              uint32_t h[16], lo[16];
              tmem_ld16_nowait(lane_base + col, h);
              tmem_ld16_nowait(lane_base + col + R, lo);
              tmem_ld_wait();
#pragma unroll
              for (int i = 0; i < 16; ++i)
                sum[c * 16 + i] += __uint_as_float(h[i]) + __uint_as_float(lo[i]);
            } else {
              float v[16];
              tmem_ld16(lane_base + col, v);
#pragma unroll
              for (int i = 0; i < 16; ++i) sum[c * 16 + i] += v[i];
            }
          }
        }
        tc_fence_before();
        mbar_arrive(smem_u32(&bar.acc_empty[acc]));
        if (++acc == 2) {
          acc = 0;
          aph ^= 1u;
        }
      }
      float* row = Yp + (static_cast<size_t>(tile) * 128 + warp * 32 + lane) * R;
#pragma unroll
      for (int c = 0; c < kMaxRankTc / 4; ++c)
        if (c * 4 < R)
          reinterpret_cast<float4*>(row)[c] =
              make_float4(sum[4 * c], sum[4 * c + 1], sum[4 * c + 2], sum[4 * c + 3]);
    }
  epi_done:;
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && bar.abort && err) atomicOr(err, GSP_DEV_TIMEOUT);
  if (warp == 5) {
    tc_fence_after();
    tmem_dealloc(tmem, ncols);
  }
}

// ------------------------------------------------------------ Z' pass --
// Z'[l][st][r] = sum_y fy[y][r] U_{l,y}[st][r],  U_{l,y}[st][r] = sum_x T[l][y][x][st] fx[x][r].
//
// The K steps (E128 x values of one map row each; N >= E128) of all levels
// form one sequence of L N (N / E128) steps; CTA p of st group g takes the
// contiguous range [p K / P, (p+1) K / P).  With P >= L a range holds at most
// two segments (the part in its first level and the part in the next); each
// segment's sums go to partial slice 2p + seg of the group's st rows and a
// fixed-order reduce adds the slices of each level.
//
// Per step the producer loads the B tile (the step's E128 rows of fx as the
// K-major operand FXt, a BF16 hi + lo pair for the split precision) and, for
// every st block m of the group, the [E128 x rows x 128 st] T tile as 128/E128
// MN-major TMA boxes (LBO = box bytes).  The accumulators collect U of one map
// row (a chunk of N / E128 steps); at the row's end the epilogue warps add
// fy[y][r] times the chunk to the running sums in TMEM columns
// [nAcc MB R, (nAcc + 1) MB R) with FP32 round-to-nearest FMAs, or, for the
// segment's last row, write the result to the partial slice.  With nAcc = 2
// (when 3 MB R <= 512 columns) consecutive rows alternate between two chunk
// accumulators, so the MMAs of a row run while the epilogue drains the last.  fy is applied in FP32 and never rounded to the
// operand type.
struct LstRange {
  long long k0, k1;     // this CTA's steps
  long long mid;        // end of the first segment
  int level0;
};

__device__ __forceinline__ LstRange lst_range(int p, int P, long long K, long long spl) {
  LstRange r;
  r.k0 = K * p / P;
  r.k1 = K * (p + 1) / P;
  r.level0 = static_cast<int>(r.k0 / spl);
  const long long lend = (r.level0 + 1) * spl;
  r.mid = r.k1 < lend ? r.k1 : lend;
  return r;
}

template <int ELEM, bool SPLIT>
__global__ void __launch_bounds__(kThreads, 1)
    k_lst_tc(const __grid_constant__ CUtensorMap mapT, const __grid_constant__ CUtensorMap mapFX,
             const float* __restrict__ fy, float* __restrict__ Zpart, int P, int logN, int L,
             int B2, int R, int MB, int G, int kStages, int nB, int nAcc, uint32_t* err) {
  constexpr int E128 = 128 / ELEM;
  constexpr uint32_t FMT = ELEM == 2 ? 1u : 2u;
  constexpr int BOXES = 128 / E128;                 // TMA boxes per 128-wide st block
  constexpr int BOX_BYTES = E128 * 128;             // E128 rows x 128 bytes
  constexpr int MMA_K_ROWS = 32 / ELEM;             // K rows per MMA (32 bytes of K)
  constexpr uint64_t A_LAYOUT = ELEM == 2 ? 2 : 1;  // MN-major TF32 uses 32-byte atoms
  constexpr uint32_t A_SBO = ELEM == 2 ? 1024 : 512;  // K-row group stride of that layout
  extern __shared__ uint8_t smem_raw[];
  __shared__ Barriers bar;
  uint8_t* smem = align1024(smem_raw);
  uint8_t* bslots = smem + kStages * kTileBytes;
  const int b_rows = R * (SPLIT ? 2 : 1);
  const int b_bytes = b_rows * 128;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int N = 1 << logN;
  const long long N2 = static_cast<long long>(N) * N;
  const int spr = N / E128;               // steps per map row (one chunk)
  const long long spl = N2 / E128;        // steps per level
  const long long K = spl * L;
  const int g = blockIdx.x % G, p = blockIdx.x / G;
  const LstRange rg = lst_range(p, P, K, spl);
  // nAcc chunk accumulators (two: the MMAs of a map row run while the epilogue
  // drains the previous row) and the running sums
  const uint32_t ncols = tmem_cols_for((nAcc + 1) * MB * R);
  volatile int* abort = &bar.abort;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(smem_u32(&bar.full[s]), 1);
      mbar_init(smem_u32(&bar.empty[s]), 1);
    }
    for (int b = 0; b < nAcc; ++b) {
      mbar_init(smem_u32(&bar.acc_full[b]), 1);
      mbar_init(smem_u32(&bar.acc_empty[b]), 128);
    }
    for (int b = 0; b < nB; ++b) {
      mbar_init(smem_u32(&bar.b_full[b]), 1);
      mbar_init(smem_u32(&bar.b_empty[b]), 1);
    }
    mbar_init(smem_u32(&bar.drain), 1);
    bar.abort = 0;
    fence_barrier_init();
  }
  if (warp == 5) tmem_alloc(smem_u32(&bar.tmem_base), ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bar.tmem_base;

  if (warp == 4) {
    if (lane == 0) {  // ---- TMA producer: per step the B tile, then MB T tiles
      int s = 0, bs = 0;
      uint32_t ph = 0, bph = 0;
      uint32_t issued_parity[kMaxStages], b_parity[kMaxStages];
      bool issued[kMaxStages], b_issued[kMaxStages];
      for (int i = 0; i < kMaxStages; ++i) issued[i] = b_issued[i] = false;
      int xb = static_cast<int>(rg.k0 % spr);  // x block of step k
      for (long long k = rg.k0; k < rg.k1 && !*abort; ++k, xb = xb + 1 == spr ? 0 : xb + 1) {
        if (!mbar_wait(smem_u32(&bar.b_empty[bs]), bph ^ 1u, abort)) goto producer_done;
        {
          const uint32_t bb = smem_u32(&bar.b_full[bs]);
          mbar_expect_tx(bb, static_cast<uint32_t>(b_bytes));
          tma_load_2d(smem_u32(bslots + bs * b_bytes), &mapFX, xb * E128, 0, bb);
          b_issued[bs] = true;
          b_parity[bs] = bph;
          if (++bs == nB) {
            bs = 0;
            bph ^= 1u;
          }
        }
        for (int m = 0; m < MB; ++m) {
          if (!mbar_wait(smem_u32(&bar.empty[s]), ph ^ 1u, abort)) goto producer_done;
          const uint32_t sa = smem_u32(smem + s * kTileBytes);
          const uint32_t fb = smem_u32(&bar.full[s]);
          mbar_expect_tx(fb, kTileBytes);
          const int st0 = (g * MB + m) * 128;
          const int trow = static_cast<int>(k * E128);
#pragma unroll
          for (int b = 0; b < BOXES; ++b)
            tma_load_2d(sa + b * BOX_BYTES, &mapT, st0 + b * E128, trow, fb);
          issued[s] = true;
          issued_parity[s] = ph;
          if (++s == kStages) {
            s = 0;
            ph ^= 1u;
          }
        }
      }
    producer_done:
      if (*abort) {  // wait for this CTA's own copies still in flight
        for (int i = 0; i < kStages; ++i)
          if (issued[i]) mbar_drain(smem_u32(&bar.full[i]), issued_parity[i]);
        for (int i = 0; i < nB; ++i)
          if (b_issued[i]) mbar_drain(smem_u32(&bar.b_full[i]), b_parity[i]);
      }
    }
  } else if (warp == 5) {
    if (lane == 0) {  // ---- MMA issuer
      const uint32_t id = idesc(FMT, 1, static_cast<uint32_t>(R));
      int s = 0, bs = 0;
      uint32_t ph = 0, bph = 0, uph = 0;
      int ab = 0;  // chunk accumulator of the current map row
      bool any = false;
      for (int seg = 0; seg < 2; ++seg) {
        const long long kb = seg == 0 ? rg.k0 : rg.mid, ke = seg == 0 ? rg.mid : rg.k1;
        for (long long c0 = kb; c0 < ke;) {  // one chunk (accumulator) per map row
          const long long row_end = (c0 / spr + 1) * spr;
          const long long c1 = row_end < ke ? row_end : ke;
          if (!mbar_wait(smem_u32(&bar.acc_empty[ab]), uph ^ 1u, abort)) goto mma_done;
          tc_fence_after();
          for (long long k = c0; k < c1; ++k) {
            if (!mbar_wait(smem_u32(&bar.b_full[bs]), bph, abort)) goto mma_done;
            tc_fence_after();
            const uint64_t b0 = sdesc(smem_u32(bslots + bs * b_bytes), 16, 1024);
            const uint64_t blo = static_cast<uint64_t>(R * 128 / 16);
            for (int m = 0; m < MB; ++m) {
              if (!mbar_wait(smem_u32(&bar.full[s]), ph, abort)) goto mma_done;
              tc_fence_after();
              const uint32_t sa = smem_u32(smem + s * kTileBytes);
              const uint32_t d = tmem + static_cast<uint32_t>((ab * MB + m) * R);
              // descriptor address fields are in 16-byte units
              const uint64_t a0 = sdesc(sa, BOX_BYTES, A_SBO, A_LAYOUT);
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const uint64_t a = a0 + static_cast<uint64_t>(j * MMA_K_ROWS * 128 / 16);
                umma<ELEM>(d, a, b0 + 2 * j, id, (k > c0 || j > 0) ? 1u : 0u);
                if constexpr (SPLIT) umma<ELEM>(d, a, b0 + blo + 2 * j, id, 1u);
              }
              any = true;
              umma_commit(smem_u32(&bar.empty[s]));
              if (++s == kStages) {
                s = 0;
                ph ^= 1u;
              }
            }
            umma_commit(smem_u32(&bar.b_empty[bs]));
            if (++bs == nB) {
              bs = 0;
              bph ^= 1u;
            }
          }
          umma_commit(smem_u32(&bar.acc_full[ab]));
          if (++ab == nAcc) {
            ab = 0;
            uph ^= 1u;
          }
          c0 = c1;
        }
      }
    mma_done:
      if (*abort && any) {
        umma_commit(smem_u32(&bar.drain));
        mbar_drain(smem_u32(&bar.drain), 0);
      }
    }
  } else {  // ---- warps 0-3: per map row, running sums += fy[y] * chunk
    uint32_t uph = 0;
    int ab = 0;
    const uint32_t lane_base = tmem + (static_cast<uint32_t>(warp * 32) << 16);
    const uint32_t sum_col = static_cast<uint32_t>(nAcc * MB * R);
    for (int seg = 0; seg < 2; ++seg) {
      const long long kb = seg == 0 ? rg.k0 : rg.mid, ke = seg == 0 ? rg.mid : rg.k1;
      if (kb >= ke) continue;
      const long long row0 = kb / spr, row1 = (ke - 1) / spr;  // map rows (l N + y)
      float* part = Zpart + (static_cast<size_t>(p) * 2 + seg) * B2 * R;
      for (long long row = row0; row <= row1; ++row) {
        const bool first = row == row0, last = row == row1;
        // the row's fy values, loaded while the MMAs still run
        const float4* fyr = reinterpret_cast<const float4*>(fy + static_cast<size_t>(row & (N - 1)) * R);
        float f[kMaxRankTc];
#pragma unroll
        for (int i = 0; i < kMaxRankTc / 4; ++i) {
          if (4 * i < R) {
            const float4 q = __ldg(fyr + i);
            f[4 * i] = q.x; f[4 * i + 1] = q.y; f[4 * i + 2] = q.z; f[4 * i + 3] = q.w;
          }
        }
        if (!mbar_wait(smem_u32(&bar.acc_full[ab]), uph, abort)) goto epi_done;
        tc_fence_after();
        for (int m = 0; m < MB; ++m) {
          float* out = part + (static_cast<size_t>((g * MB + m) * 128) + warp * 32 + lane) * R;
#pragma unroll
          for (int cb = 0; cb < kMaxRankTc / 16; ++cb) {
            if (cb * 16 < R) {
              const uint32_t col = static_cast<uint32_t>(m * R + cb * 16);
              uint32_t a[16], b[16];
              tmem_ld16_nowait(lane_base + static_cast<uint32_t>(ab * MB * R) + col, a);
              if (!first) tmem_ld16_nowait(lane_base + sum_col + col, b);
              tmem_ld_wait();
              float v[16];
#pragma unroll
              for (int i = 0; i < 16; ++i)
                v[i] = first ? f[cb * 16 + i] * __uint_as_float(a[i])
                             : fmaf(f[cb * 16 + i], __uint_as_float(a[i]), __uint_as_float(b[i]));
              if (last) {
                float4* dst = reinterpret_cast<float4*>(out + cb * 16);
                dst[0] = make_float4(v[0], v[1], v[2], v[3]);
                dst[1] = make_float4(v[4], v[5], v[6], v[7]);
                dst[2] = make_float4(v[8], v[9], v[10], v[11]);
                dst[3] = make_float4(v[12], v[13], v[14], v[15]);
              } else {
                tmem_st16(lane_base + sum_col + col, v);
              }
            }
          }
        }
        if (!last) tmem_st_wait();
        tc_fence_before();
        mbar_arrive(smem_u32(&bar.acc_empty[ab]));
        if (++ab == nAcc) {
          ab = 0;
          uph ^= 1u;
        }
      }
    }
  epi_done:;
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && bar.abort && err) atomicOr(err, GSP_DEV_TIMEOUT);
  if (warp == 5) {
    tc_fence_after();
    tmem_dealloc(tmem, ncols);
  }
}

// ------------------------------------------------- Z' pass, rank rows --
// The same contraction with the operands' roles exchanged, for the BF16 hi + lo
// pair at rank 64: the FXt tile (hi rows 0..63, lo rows 64..127) is the K-major
// A operand (M = 128) and the W st columns of the CTA's group the MN-major B
// operand, loaded as boxes of 16 columns x E128 rows with 32-byte swizzling.
// One MMA of N = W per K slice then covers the hi and lo parts, and no
// accumulator row is padding (with st as M, 48 of the 128 rows were padding at
// 80 stored columns, and hi and lo took an MMA each).  TMEM lane
// r2 = 32 warp + lane holds rank r2 mod 64 of the hi (r2 < 64) or lo part, so
// fy[y][r] is one scalar per thread.  At a segment's last row the hi threads
// store their sums to the partial slice; the lo threads keep theirs in the
// running sums and, once the hi threads have arrived at the segment's exchange
// barrier, add them to the slice.  Columns at or past Bt (the stored columns)
// are not written.
constexpr int kSwRank = 64;          // M = 2R = 128
constexpr int kSwMaxCols = 80;       // 3 W <= 256 TMEM columns: two CTAs per SM
constexpr int kSwBox = 64 * 16 * 2;  // one box: E128 = 64 rows x 16 BF16 columns

__global__ void __launch_bounds__(kThreads, 1)
    k_lst_tc_rows(const __grid_constant__ CUtensorMap mapT, const __grid_constant__ CUtensorMap mapFX,
                  const float* __restrict__ fy, float* __restrict__ Zpart, int P, int logN, int L,
                  int B2, int Bt, int W, int G, int kStages, int nB, int nAcc, uint32_t* err) {
  constexpr int E128 = 64;
  constexpr int R = kSwRank;
  constexpr int b_bytes = 2 * R * 128;
  extern __shared__ uint8_t smem_raw[];
  __shared__ Barriers bar;
  uint8_t* smem = align1024(smem_raw);
  const int t_bytes = W * 128;  // W / 16 boxes; a multiple of 2048 bytes
  uint8_t* bslots = smem + kStages * t_bytes;
  const int nbox = W / 16;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int N = 1 << logN;
  const long long N2 = static_cast<long long>(N) * N;
  const int spr = N / E128;
  const long long spl = N2 / E128;
  const long long K = spl * L;
  const int g = blockIdx.x % G, p = blockIdx.x / G;
  const int st0 = g * W;
  const LstRange rg = lst_range(p, P, K, spl);
  const uint32_t ncols = tmem_cols_for((nAcc + 1) * W);
  volatile int* abort = &bar.abort;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(smem_u32(&bar.full[s]), 1);
      mbar_init(smem_u32(&bar.empty[s]), 1);
    }
    for (int b = 0; b < nAcc; ++b) {
      mbar_init(smem_u32(&bar.acc_full[b]), 1);
      mbar_init(smem_u32(&bar.acc_empty[b]), 128);
    }
    for (int b = 0; b < nB; ++b) {
      mbar_init(smem_u32(&bar.b_full[b]), 1);
      mbar_init(smem_u32(&bar.b_empty[b]), 1);
    }
    mbar_init(smem_u32(&bar.drain), 1);
    mbar_init(smem_u32(&bar.xchg[0]), 64);
    mbar_init(smem_u32(&bar.xchg[1]), 64);
    bar.abort = 0;
    fence_barrier_init();
  }
  if (warp == 5) tmem_alloc(smem_u32(&bar.tmem_base), ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bar.tmem_base;

  if (warp == 4) {
    if (lane == 0) {  // ---- TMA producer: per step the FXt tile, then the T tile
      int s = 0, bs = 0;
      uint32_t ph = 0, bph = 0;
      uint32_t issued_parity[kMaxStages], b_parity[kMaxStages];
      bool issued[kMaxStages], b_issued[kMaxStages];
      for (int i = 0; i < kMaxStages; ++i) issued[i] = b_issued[i] = false;
      int xb = static_cast<int>(rg.k0 % spr);
      for (long long k = rg.k0; k < rg.k1 && !*abort; ++k, xb = xb + 1 == spr ? 0 : xb + 1) {
        if (!mbar_wait(smem_u32(&bar.b_empty[bs]), bph ^ 1u, abort)) goto producer_done;
        {
          const uint32_t bb = smem_u32(&bar.b_full[bs]);
          mbar_expect_tx(bb, static_cast<uint32_t>(b_bytes));
          tma_load_2d(smem_u32(bslots + bs * b_bytes), &mapFX, xb * E128, 0, bb);
          b_issued[bs] = true;
          b_parity[bs] = bph;
          if (++bs == nB) {
            bs = 0;
            bph ^= 1u;
          }
        }
        if (!mbar_wait(smem_u32(&bar.empty[s]), ph ^ 1u, abort)) goto producer_done;
        {
          const uint32_t sa = smem_u32(smem + s * t_bytes);
          const uint32_t fb = smem_u32(&bar.full[s]);
          mbar_expect_tx(fb, static_cast<uint32_t>(t_bytes));
          const int trow = static_cast<int>(k * E128);
          for (int b = 0; b < nbox; ++b) tma_load_2d(sa + b * kSwBox, &mapT, st0 + 16 * b, trow, fb);
          issued[s] = true;
          issued_parity[s] = ph;
          if (++s == kStages) {
            s = 0;
            ph ^= 1u;
          }
        }
      }
    producer_done:
      if (*abort) {  // wait for this CTA's own copies still in flight
        for (int i = 0; i < kStages; ++i)
          if (issued[i]) mbar_drain(smem_u32(&bar.full[i]), issued_parity[i]);
        for (int i = 0; i < nB; ++i)
          if (b_issued[i]) mbar_drain(smem_u32(&bar.b_full[i]), b_parity[i]);
      }
    }
  } else if (warp == 5) {
    if (lane == 0) {  // ---- MMA issuer
      const uint32_t id = idesc(1u, 0u, static_cast<uint32_t>(W), 1u);
      int s = 0, bs = 0;
      uint32_t ph = 0, bph = 0, uph = 0;
      int ab = 0;
      bool any = false;
      for (int seg = 0; seg < 2; ++seg) {
        const long long kb = seg == 0 ? rg.k0 : rg.mid, ke = seg == 0 ? rg.mid : rg.k1;
        for (long long c0 = kb; c0 < ke;) {  // one chunk (accumulator) per map row
          const long long row_end = (c0 / spr + 1) * spr;
          const long long c1 = row_end < ke ? row_end : ke;
          if (!mbar_wait(smem_u32(&bar.acc_empty[ab]), uph ^ 1u, abort)) goto mma_done;
          tc_fence_after();
          const uint32_t d = tmem + static_cast<uint32_t>(ab * W);
          for (long long k = c0; k < c1; ++k) {
            if (!mbar_wait(smem_u32(&bar.b_full[bs]), bph, abort)) goto mma_done;
            if (!mbar_wait(smem_u32(&bar.full[s]), ph, abort)) goto mma_done;
            tc_fence_after();
            // A: 128 FXt rows of 128 bytes, 8-row groups 1024 bytes apart.
            // B: 16-column boxes kSwBox apart (LBO), 8-row groups of 32-byte rows
            // 256 bytes apart (SBO); a K slice of 16 rows is 512 bytes.
            const uint64_t a0 = sdesc(smem_u32(bslots + bs * b_bytes), 16, 1024);
            const uint64_t b0 = sdesc(smem_u32(smem + s * t_bytes), kSwBox, 256, 6);
#pragma unroll
            for (int j = 0; j < 4; ++j)
              umma<2>(d, a0 + 2 * j, b0 + 32 * j, id, (k > c0 || j > 0) ? 1u : 0u);
            any = true;
            umma_commit(smem_u32(&bar.empty[s]));
            umma_commit(smem_u32(&bar.b_empty[bs]));
            if (++s == kStages) {
              s = 0;
              ph ^= 1u;
            }
            if (++bs == nB) {
              bs = 0;
              bph ^= 1u;
            }
          }
          umma_commit(smem_u32(&bar.acc_full[ab]));
          if (++ab == nAcc) {
            ab = 0;
            uph ^= 1u;
          }
          c0 = c1;
        }
      }
    mma_done:
      if (*abort && any) {
        umma_commit(smem_u32(&bar.drain));
        mbar_drain(smem_u32(&bar.drain), 0);
      }
    }
  } else {  // ---- warps 0-3: per map row, running sums += fy[y][r] * chunk
    uint32_t uph = 0;
    int ab = 0;
    const int r2 = warp * 32 + lane, r = r2 & (R - 1);
    const bool hi = r2 < R;
    const uint32_t lane_base = tmem + (static_cast<uint32_t>(warp * 32) << 16);
    const uint32_t sum_col = static_cast<uint32_t>(nAcc * W);
    for (int seg = 0; seg < 2; ++seg) {
      const long long kb = seg == 0 ? rg.k0 : rg.mid, ke = seg == 0 ? rg.mid : rg.k1;
      if (kb >= ke) continue;
      const long long row0 = kb / spr, row1 = (ke - 1) / spr;  // map rows (l N + y)
      float* out = Zpart + (static_cast<size_t>(p) * 2 + seg) * B2 * R + static_cast<size_t>(st0) * R + r;
      for (long long row = row0; row <= row1; ++row) {
        const bool first = row == row0, last = row == row1;
        const bool to_slice = last && hi;
        const float f = __ldg(fy + static_cast<size_t>(row & (N - 1)) * R + r);
        if (!mbar_wait(smem_u32(&bar.acc_full[ab]), uph, abort)) goto epi_done;
        tc_fence_after();
        for (int cb = 0; cb < nbox; ++cb) {
          const uint32_t col = static_cast<uint32_t>(cb * 16);
          uint32_t a[16], b[16];
          tmem_ld16_nowait(lane_base + static_cast<uint32_t>(ab * W) + col, a);
          if (!first) tmem_ld16_nowait(lane_base + sum_col + col, b);
          tmem_ld_wait();
          float v[16];
#pragma unroll
          for (int i = 0; i < 16; ++i)
            v[i] = first ? f * __uint_as_float(a[i]) : fmaf(f, __uint_as_float(a[i]), __uint_as_float(b[i]));
          if (to_slice) {
            if (st0 + 16 * cb < Bt) {
#pragma unroll
              for (int i = 0; i < 16; ++i) out[static_cast<size_t>(16 * cb + i) * R] = v[i];
            }
          } else {
            tmem_st16(lane_base + sum_col + col, v);
          }
        }
        if (!to_slice) tmem_st_wait();
        tc_fence_before();
        mbar_arrive(smem_u32(&bar.acc_empty[ab]));
        if (++ab == nAcc) {
          ab = 0;
          uph ^= 1u;
        }
        if (last) {  // hi + lo into the partial slice
          if (hi) {
            mbar_arrive(smem_u32(&bar.xchg[seg]));
          } else {
            if (!mbar_wait(smem_u32(&bar.xchg[seg]), 0u, abort)) goto epi_done;
            tc_fence_after();
            for (int cb = 0; cb < nbox; ++cb) {
              uint32_t b[16];
              tmem_ld16_nowait(lane_base + sum_col + static_cast<uint32_t>(cb * 16), b);
              tmem_ld_wait();
              if (st0 + 16 * cb < Bt) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                  float* o = out + static_cast<size_t>(16 * cb + i) * R;
                  *o = *o + __uint_as_float(b[i]);
                }
              }
            }
          }
        }
      }
    }
  epi_done:;
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && bar.abort && err) atomicOr(err, GSP_DEV_TIMEOUT);
  if (warp == 5) {
    tc_fence_after();
    tmem_dealloc(tmem, ncols);
  }
}

// One CTA waits for a phase of an mbarrier that nothing arrives at: the
// bounded wait gives up after kTimeoutCycles and the status path runs.
__global__ void k_selftest_timeout(uint32_t* err) {
  __shared__ uint64_t mb;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&mb), 1);
    abort_flag = 0;
    fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(smem_u32(&mb), 0u, &abort_flag)) atomicOr(err, GSP_DEV_TIMEOUT);
}

// FXt[r][x] = fx[x][r] in the operand type (K-major B operand of the Z' pass):
// BF16, or FP32 rounded to the nearest TF32; with `split` rows R..2R-1 hold
// the remainder fx - hi rounded the same way.
template <typename OutT>
__global__ void k_fx_cols(const float* __restrict__ fx, int N, int R, int split,
                          OutT* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N * R) return;
  const int r = i / N, x = i - r * N;
  const float v = fx[static_cast<size_t>(x) * R + r];
  if constexpr (sizeof(OutT) == 2) {
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    out[i] = hi;
    if (split) out[static_cast<size_t>(R) * N + i] = __float2bfloat16_rn(v - __bfloat162float(hi));
  } else {
    const float hi = round_tf32(v);
    out[i] = hi;
    if (split) out[static_cast<size_t>(R) * N + i] = round_tf32(v - hi);
  }
}

// Level of each CTA's two partial slices (-1: slice not written).
struct LstSegments {
  int8_t level[kLstMaxRanges][2];
};

// Z'[l][st][r] = sum over CTAs p (in order) of the partial slices whose segment
// lies in level l; zero for st rows at or past `rows` (not written by the pass).
__global__ void k_lst_reduce(const float* __restrict__ Zpart, float* __restrict__ Zp, int P,
                             int L, long long per_level, long long rows_elems,
                             const __grid_constant__ LstSegments sg) {
  const long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (e >= per_level * L) return;
  const int l = static_cast<int>(e / per_level);
  const long long rem = e - l * per_level;
  float acc = 0.0f;
  if (rem >= rows_elems) {
    Zp[e] = 0.0f;
    return;
  }
  for (int p = 0; p < P; ++p) {
    if (sg.level[p][0] == l) acc += Zpart[(static_cast<long long>(p) * 2) * per_level + rem];
    if (sg.level[p][1] == l) acc += Zpart[(static_cast<long long>(p) * 2 + 1) * per_level + rem];
  }
  Zp[e] = acc;
}

// ----------------------------------------------------------- host side --

}  // namespace

// The driver's cuTensorMapEncodeTiled (null without a driver); shared with the
// histogram build.
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

namespace {

// 2D map over a row-major [rows][cols] matrix, box = [box_rows][box_cols]
// (default: 128 bytes of columns), 128B swizzle by default.
int make_map(CUtensorMap* map, const void* base, int elem, long long rows, long long cols,
             int box_rows, CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_128B, int box_cols = 0) {
  auto fn = encode_fn();
  if (!fn) return GSP_ERR_UNSUPPORTED;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(cols) * elem};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(box_cols ? box_cols : 128 / elem),
                       static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, elem == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                  2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? GSP_OK : GSP_ERR_CUDA;
}

// Ring depth: as many stages as fit in ~200 KB, between 3 and 8.
int stages_for(size_t stage_bytes, size_t fixed) {
  size_t avail = 200 * 1024 - fixed;
  int st = static_cast<int>(avail / stage_bytes);
  return st > kMaxStages ? kMaxStages : (st < 3 ? 3 : st);
}

size_t xy_stage_bytes(int R, bool split) { return kTileBytes + static_cast<size_t>(R) * 128 * (split ? 2 : 1); }
// Two Y' CTAs per SM, each with a ring of ~110 KB (at least 3 stages): two
// independent TMA / MMA / epilogue pipelines per SM.  Their tensor memory
// (two chunk accumulators of R columns each) fits twice in the 512 columns.
constexpr int kXyCtasPerSm = 2;
int xy_stages(int R, bool split) {
  const int st = static_cast<int>((110 * 1024 - 1024) / xy_stage_bytes(R, split));
  return st > kMaxStages ? kMaxStages : (st < 3 ? 3 : st);
}
size_t xy_smem(int R, bool split) { return 1024 + xy_stages(R, split) * xy_stage_bytes(R, split); }

size_t lst_b_bytes(int R, bool split) { return static_cast<size_t>(R) * 128 * (split ? 2 : 1); }

// Z' ring shapes: T stages of one tile and B slots of one FXt tile.  A step
// takes one B slot and streams its MB T tiles through the T ring, so the
// producer runs min(B slots * MB, stages) T tiles ahead of the tensor core;
// the split of ~200 KB that maximises that lead is taken (the first one on
// ties, so a large MB keeps two B slots and the deepest T ring).
struct LstCfg {
  int stages, bslots;
  size_t smem;
};
// Chunk accumulators of the Z' pass (two when three accumulators' columns fit).
int lst_accs(int R, int MB) { return 3 * MB * R <= 512 ? 2 : 1; }
// Z' CTAs per SM: two when two CTAs' tensor memory fits in the 512 columns.
int lst_ctas_per_sm(int R, int MB) {
  return 2 * static_cast<int>(tmem_cols_for((lst_accs(R, MB) + 1) * MB * R)) <= 512 ? 2 : 1;
}
LstCfg lst_cfg(int R, bool split, int MB) {
  const int per_sm = lst_ctas_per_sm(R, MB);
  const size_t b = lst_b_bytes(R, split), budget = (per_sm == 2 ? 110 : 200) * 1024 - 1024;
  LstCfg best{3, 2, 0};
  int lead = -1;
  for (int nb = 2; nb <= kMaxStages && nb * b + 3 * kTileBytes <= budget; ++nb) {
    int st = static_cast<int>((budget - nb * b) / kTileBytes);
    if (st > kMaxStages) st = kMaxStages;
    if (st < 3) continue;
    const int ahead = nb * MB < st ? nb * MB : st;
    if (ahead > lead) {
      lead = ahead;
      best = LstCfg{st, nb, 0};
    }
  }
  // With one CTA per SM the Z' pass may allocate up to all 512 TMEM columns,
  // so it then asks for enough shared memory that no second CTA fits.
  const size_t need = 1024 + best.stages * static_cast<size_t>(kTileBytes) + best.bslots * b;
  best.smem = per_sm == 1 && need < 120 * 1024 ? 120 * 1024 : need;
  return best;
}

// The rank-row Z' pass (k_lst_tc_rows) serves the BF16 hi + lo pair at rank 64.
// Its st groups: G groups of W <= kSwMaxCols stored columns (a multiple of 16).
bool lst_rows(const MttkrpDims& d, int elem, bool split) {
  return elem == 2 && split && d.R == kSwRank;
}
int lst_rows_groups(const MttkrpDims& d, int* W) {
  const int bt = d.B2t();
  const int G = (bt + kSwMaxCols - 1) / kSwMaxCols;
  *W = ((bt + G - 1) / G + 15) / 16 * 16;
  return G;
}
// Its ring: T stages of W x 128 bytes and FXt slots of 2R x 128 bytes in ~110 KB
// (two CTAs per SM), the split that lets the producer run furthest ahead.
LstCfg lst_rows_cfg(int W) {
  const size_t t = static_cast<size_t>(W) * 128, b = 2 * kSwRank * 128, budget = 110 * 1024 - 1024;
  LstCfg best{3, 2, 0};
  int lead = -1;
  for (int nb = 2; nb <= kMaxStages && nb * b + 3 * t <= budget; ++nb) {
    int st = static_cast<int>((budget - nb * b) / t);
    if (st > kMaxStages) st = kMaxStages;
    const int ahead = nb < st ? nb : st;
    if (ahead > lead) {
      lead = ahead;
      best = LstCfg{st, nb, 0};
    }
  }
  best.smem = 1024 + best.stages * t + best.bslots * b;
  return best;
}

// SMs the persistent passes occupy: all but one, which stays free for the
// FP64 Gram solve that gsp_cp_sweeps runs on its side stream under each pass
// (a single-CTA kernel: with every SM held by the pass it waited for the
// pass to end, 0.2 ms per sweep at rank 64).
int pass_sms() {
  const int n = sm_count();
  return n > 1 ? n - 1 : 1;
}

template <typename K>
int set_smem(K kernel, size_t bytes) {
  GSP_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(bytes)));
  return GSP_OK;
}

// st blocks per CTA (MB) and st groups (G): the chunk accumulators and the
// running sums take 2 MB R <= 512 tensor-memory columns.
int lst_groups(const MttkrpDims& d, int* MB) {
  int blocks = d.B2() / 128;
  int mb = 256 / d.R;
  if (mb > blocks) mb = blocks;
  *MB = mb;
  return blocks / mb;
}

}  // namespace

bool tc_supported(const MttkrpDims& d, int precision) {
  if (precision != GSP_PREC_BF16 && precision != GSP_PREC_BF16_1X && precision != GSP_PREC_TF32)
    return false;
  if (!(d.R == 16 || d.R == 32 || d.R == 64)) return false;
  if (d.B < 16 || d.N < 128 / (precision == GSP_PREC_TF32 ? 4 : 2)) return false;  // Z' steps stay in one map row
  if (d.L * d.N2() >= (1LL << 31)) return false;  // TMA row coordinate is int32
  const bool split = precision != GSP_PREC_BF16_1X;  // BF16 and TF32 use hi + lo pairs
  int MB = 0;
  lst_groups(d, &MB);
  return xy_smem(d.R, split) <= 227 * 1024 && lst_cfg(d.R, split, MB).smem <= 227 * 1024 &&
         encode_fn() != nullptr;
}

int tc_mttkrp_xy(const void* T, const void* KRt, float* Yp, const MttkrpDims& d, int precision,
                 uint32_t* err, cudaStream_t s) {
  if (!tc_supported(d, precision)) return GSP_ERR_UNSUPPORTED;
  const int elem = precision == GSP_PREC_TF32 ? 4 : 2;
  const bool split = precision != GSP_PREC_BF16_1X;  // BF16 and TF32 use hi + lo pairs
  const int brows = d.R * (split ? 2 : 1);
  CUtensorMap mT, mK;
  // T rows hold B2t() stored columns; the K chunks past them read zeros
  GSP_TRY(make_map(&mT, T, elem, d.L * d.N2(), d.B2t(), 128));
  GSP_TRY(make_map(&mK, KRt, elem, brows, static_cast<long long>(d.L) * d.B2(), brows));
  const int n_tiles = static_cast<int>(d.N2() / 128);
  int grid = pass_sms() * kXyCtasPerSm;
  if (grid > n_tiles) grid = n_tiles;
  const size_t smem = xy_smem(d.R, split);
  const int stages = xy_stages(d.R, split);
  prof_begin(PROF_MTTKRP_XY, s);
  if (elem == 4) {
    GSP_TRY(set_smem(k_xy_tc<4, true>, smem));
    k_xy_tc<4, true><<<grid, kThreads, smem, s>>>(mT, mK, Yp, n_tiles, d.N2(), d.L, d.B2(), d.R,
                                                  stages, err);
  } else if (split) {
    GSP_TRY(set_smem(k_xy_tc<2, true>, smem));
    k_xy_tc<2, true><<<grid, kThreads, smem, s>>>(mT, mK, Yp, n_tiles, d.N2(), d.L, d.B2(), d.R,
                                                  stages, err);
  } else {
    GSP_TRY(set_smem(k_xy_tc<2, false>, smem));
    k_xy_tc<2, false><<<grid, kThreads, smem, s>>>(mT, mK, Yp, n_tiles, d.N2(), d.L, d.B2(), d.R,
                                                   stages, err);
  }
  prof_end(PROF_MTTKRP_XY, s);
  GSP_CHECK_LAUNCH();
  return GSP_OK;
}

int tc_lst_ctas(const MttkrpDims& d, bool rows) {
  int MB = 0, W = 0;
  const int G = rows ? lst_rows_groups(d, &W) : lst_groups(d, &MB);
  int P = (rows ? 2 : lst_ctas_per_sm(d.R, MB)) * pass_sms() / G;
  if (P < d.L) P = d.L;  // a range is then at most one level long: <= 2 segments
  if (P > kLstMaxRanges) P = kLstMaxRanges;
  return P;
}

int tc_mttkrp_lst(const void* T, const float* fx, const float* fy, void* FXt, float* Zpart,
                  float* Zp, const MttkrpDims& d, int precision, uint32_t* err, cudaStream_t s) {
  if (!tc_supported(d, precision)) return GSP_ERR_UNSUPPORTED;
  const int elem = precision == GSP_PREC_TF32 ? 4 : 2;
  const bool split = precision != GSP_PREC_BF16_1X;  // BF16 and TF32 use hi + lo pairs
  const int E128 = 128 / elem;
  const int brows = d.R * (split ? 2 : 1);
  const int nr = d.N * d.R;
  if (elem == 2)
    k_fx_cols<__nv_bfloat16><<<grid_for(nr, 256), 256, 0, s>>>(
        fx, d.N, d.R, split ? 1 : 0, static_cast<__nv_bfloat16*>(FXt));
  else
    k_fx_cols<float><<<grid_for(nr, 256), 256, 0, s>>>(fx, d.N, d.R, 1, static_cast<float*>(FXt));
  GSP_CHECK_LAUNCH();
  CUtensorMap mT, mF;
  GSP_TRY(make_map(&mF, FXt, elem, brows, d.N, brows));
  const bool rows = lst_rows(d, elem, split);
  const int P = tc_lst_ctas(d, rows);
  const int logN = ilog2(d.N);
  long long rows_elems = static_cast<long long>(d.B2()) * d.R;
  prof_begin(PROF_MTTKRP_LST, s);
  if (rows) {  // T as 16-column boxes, 32-byte swizzle: the MN-major B operand
    GSP_TRY(make_map(&mT, T, elem, d.L * d.N2(), d.B2t(), E128, CU_TENSOR_MAP_SWIZZLE_32B, 16));
    int W = 0;
    const int G = lst_rows_groups(d, &W);
    const LstCfg cfg = lst_rows_cfg(W);
    GSP_TRY(set_smem(k_lst_tc_rows, cfg.smem));
    k_lst_tc_rows<<<P * G, kThreads, cfg.smem, s>>>(mT, mF, fy, Zpart, P, logN, d.L, d.B2(), d.B2t(),
                                                     W, G, cfg.stages, cfg.bslots, 2, err);
    rows_elems = static_cast<long long>(d.B2t()) * d.R;
  } else {
    GSP_TRY(make_map(&mT, T, elem, d.L * d.N2(), d.B2t(), E128,
                     elem == 2 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_128B_ATOM_32B));
    int MB = 0;
    const int G = lst_groups(d, &MB);
    const int grid = P * G;
    const LstCfg cfg = lst_cfg(d.R, split, MB);
    const size_t smem = cfg.smem;
    const int stages = cfg.stages, nB = cfg.bslots;
    const int nAcc = lst_accs(d.R, MB);  // double-buffered chunk accumulator when it fits
    if (elem == 4) {
      GSP_TRY(set_smem(k_lst_tc<4, true>, smem));
      k_lst_tc<4, true><<<grid, kThreads, smem, s>>>(mT, mF, fy, Zpart, P, logN, d.L, d.B2(), d.R,
                                                     MB, G, stages, nB, nAcc, err);
    } else if (split) {
      GSP_TRY(set_smem(k_lst_tc<2, true>, smem));
      k_lst_tc<2, true><<<grid, kThreads, smem, s>>>(mT, mF, fy, Zpart, P, logN, d.L, d.B2(), d.R,
                                                     MB, G, stages, nB, nAcc, err);
    } else {
      GSP_TRY(set_smem(k_lst_tc<2, false>, smem));
      k_lst_tc<2, false><<<grid, kThreads, smem, s>>>(mT, mF, fy, Zpart, P, logN, d.L, d.B2(), d.R,
                                                      MB, G, stages, nB, nAcc, err);
    }
  }
  prof_end(PROF_MTTKRP_LST, s);
  GSP_CHECK_LAUNCH();
  const long long per_level = static_cast<long long>(d.B2()) * d.R;
  LstSegments sg;
  const long long spl = d.N2() / E128, K = spl * d.L;
  for (int p = 0; p < kLstMaxRanges; ++p) sg.level[p][0] = sg.level[p][1] = -1;
  for (int p = 0; p < P; ++p) {  // the same split as lst_range() in the kernel
    const long long k0 = K * p / P, k1 = K * (p + 1) / P;
    if (k0 >= k1) continue;
    const int l0 = static_cast<int>(k0 / spl);
    sg.level[p][0] = static_cast<int8_t>(l0);
    if (k1 > (l0 + 1) * spl) sg.level[p][1] = static_cast<int8_t>(l0 + 1);
  }
  k_lst_reduce<<<grid_for(per_level * d.L, 256), 256, 0, s>>>(Zpart, Zp, P, d.L, per_level,
                                                              rows_elems, sg);
  GSP_CHECK_LAUNCH();
  return GSP_OK;
}



}  // namespace gsp

extern "C" int gsp_selftest_wait_timeout(uint32_t* d_err, gsp_stream stream) {
  if (!d_err) return GSP_ERR_INVALID_ARG;
  gsp::k_selftest_timeout<<<1, 32, 0, gsp::to_stream(stream)>>>(d_err);
  GSP_CHECK_LAUNCH();
  return GSP_OK;
}

