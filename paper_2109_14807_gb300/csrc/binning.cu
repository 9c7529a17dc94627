// Rows a1-a3: binning of the normal map and exhaustive multi-level footprint
// histograms (Sec. 4.1), written straight into int32 counts and/or the
// scaled MTTKRP operand.
//
// Every level is computed from the 2-byte bin map alone (it stays in L2) by
// box sums of per-bin indicators staged in shared memory, so the only HBM
// traffic is the output itself; all arithmetic is integer, hence bit-exact.
#include "ndf_build.cuh"

namespace gsp {

namespace {

__global__ void k_bin_normals(const float2* __restrict__ nxy, int n, int bins,
                              uint16_t* __restrict__ out, uint32_t* status) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float2 v = nxy[i];
  uint16_t code = 0;
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

__device__ __forceinline__ void sink_store(const LevelSink& o, long long i, int4 v) {
  if (o.h) reinterpret_cast<int4*>(o.h)[i] = v;
  if (o.f32) {
    float4 f = make_float4(static_cast<float>(v.x) * o.scale, static_cast<float>(v.y) * o.scale,
                           static_cast<float>(v.z) * o.scale, static_cast<float>(v.w) * o.scale);
    reinterpret_cast<float4*>(o.f32)[i] = f;
  }
  if (o.bf16) {
    __nv_bfloat162 a = __floats2bfloat162_rn(static_cast<float>(v.x) * o.scale,
                                             static_cast<float>(v.y) * o.scale);
    __nv_bfloat162 b = __floats2bfloat162_rn(static_cast<float>(v.z) * o.scale,
                                             static_cast<float>(v.w) * o.scale);
    uint2 p;
    p.x = *reinterpret_cast<uint32_t*>(&a);
    p.y = *reinterpret_cast<uint32_t*>(&b);
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
// all N footprints are window sums of V along x, read from an exclusive
// prefix sum S over x: two look-ups per count, three across the wrap.
//  - updates: thread t owns the columns x = t, t + 256, ... (no atomics);
//  - prefix: thread t scans the contiguous columns [t*sl, (t+1)*sl) for all 16
//    bins with 16-byte shared-memory accesses, the segment totals are combined
//    by a warp shuffle scan plus one pass over the 8 warp totals;
//  - outputs: four bins per thread-item, 16-byte reads of S.
constexpr int kHistG = 16;
constexpr int kHistThreads = 256;

__global__ void __launch_bounds__(kHistThreads, 2)
    k_box_hist(const uint16_t* __restrict__ bins_map, int logN, int B2, int ychunk,
               const __grid_constant__ HistOut o) {
  constexpr int G = kHistG;
  extern __shared__ __align__(16) uint8_t smem_b[];
  __shared__ int wtot[kHistThreads / 32][G];
  const int N = 1 << logN, m = N - 1;
  uint16_t* V = reinterpret_cast<uint16_t*>(smem_b);          // [N][16], 32 B per column
  int* S = reinterpret_cast<int*>(smem_b + N * G * sizeof(uint16_t));  // [N + 1][16]
  const int g0 = blockIdx.x * G;
  const int y0 = blockIdx.y * ychunk;
  const int l = blockIdx.z;
  const int w = 1 << l, a = w >> 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (int i = tid; i < N * G / 8; i += kHistThreads)
    reinterpret_cast<uint4*>(V)[i] = make_uint4(0, 0, 0, 0);
  __syncthreads();
  for (int x = tid; x < N; x += kHistThreads)
    for (int j = 0; j < w; ++j) {
      const int b = static_cast<int>(bins_map[(((y0 - a + j) & m) << logN) + x]) - g0;
      if (static_cast<unsigned>(b) < static_cast<unsigned>(G)) V[x * G + b] += 1;
    }

  // contiguous scan segments: sl columns per thread, `active` threads
  const int sl = N >= kHistThreads ? N / kHistThreads : 1;
  const int active = N / sl;
  const float sc = o.scale[l];
  unsigned long long sumsq = 0;

  for (int y = y0; y < y0 + ychunk; ++y) {
    if (y > y0) {
      const int ro = (y - 1 - a) & m, ri = (y - 1 - a + w) & m;
      for (int x = tid; x < N; x += kHistThreads) {
        const int bo = static_cast<int>(bins_map[(ro << logN) + x]) - g0;
        const int bi = static_cast<int>(bins_map[(ri << logN) + x]) - g0;
        if (static_cast<unsigned>(bo) < static_cast<unsigned>(G)) V[x * G + bo] -= 1;
        if (static_cast<unsigned>(bi) < static_cast<unsigned>(G)) V[x * G + bi] += 1;
      }
    }
    __syncthreads();
    // 1) running sums inside this thread's segment (S[x+1] = sum up to x)
    int acc[G];
#pragma unroll
    for (int b = 0; b < G; ++b) acc[b] = 0;
    if (tid < active) {
      for (int i = 0; i < sl; ++i) {
        const int x = tid * sl + i;
        const uint4 p0 = reinterpret_cast<const uint4*>(V)[x * 2];
        const uint4 p1 = reinterpret_cast<const uint4*>(V)[x * 2 + 1];
        const uint32_t wds[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          acc[2 * k] += static_cast<int>(wds[k] & 0xFFFFu);
          acc[2 * k + 1] += static_cast<int>(wds[k] >> 16);
        }
        int4* dst = reinterpret_cast<int4*>(S + (x + 1) * G);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          dst[q] = make_int4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
      }
    }
    // 2) exclusive prefix of the segment totals: warp shuffle scan, then warps
    int incl[G];
#pragma unroll
    for (int b = 0; b < G; ++b) incl[b] = acc[b];
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
      for (int b = 0; b < G; ++b) {
        const int v = __shfl_up_sync(0xffffffffu, incl[b], off);
        if (lane >= off) incl[b] += v;
      }
    }
    if (lane == 31) {
#pragma unroll
      for (int b = 0; b < G; ++b) wtot[warp][b] = incl[b];
    }
    __syncthreads();
    if (tid < active) {
      int off[G];
#pragma unroll
      for (int b = 0; b < G; ++b) off[b] = incl[b] - acc[b];
      for (int k = 0; k < warp; ++k)
#pragma unroll
        for (int b = 0; b < G; ++b) off[b] += wtot[k][b];
      for (int i = 0; i < sl; ++i) {
        int4* dst = reinterpret_cast<int4*>(S + (tid * sl + i + 1) * G);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          int4 v = dst[q];
          v.x += off[4 * q];
          v.y += off[4 * q + 1];
          v.z += off[4 * q + 2];
          v.w += off[4 * q + 3];
          dst[q] = v;
        }
      }
      if (tid == 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) reinterpret_cast<int4*>(S)[q] = make_int4(0, 0, 0, 0);
      }
    }
    __syncthreads();
    // 3) counts of every footprint of row y, four bins per item
    const long long row4 = ((static_cast<long long>(l) * N + y) * N * B2) >> 2;
    for (int e = tid; e < N * (G / 4); e += kHistThreads) {
      const int x = e >> 2, q = e & 3;
      const int st = (x - a) & m, en = st + w;
      const int4 lo = reinterpret_cast<const int4*>(S + st * G)[q];
      int4 c;
      if (en <= N) {
        const int4 hi = reinterpret_cast<const int4*>(S + en * G)[q];
        c = make_int4(hi.x - lo.x, hi.y - lo.y, hi.z - lo.z, hi.w - lo.w);
      } else {
        const int4 hi = reinterpret_cast<const int4*>(S + N * G)[q];
        const int4 wr = reinterpret_cast<const int4*>(S + (en - N) * G)[q];
        c = make_int4(hi.x - lo.x + wr.x, hi.y - lo.y + wr.y, hi.z - lo.z + wr.z,
                      hi.w - lo.w + wr.w);
      }
      const long long i4 = row4 + ((static_cast<long long>(x) * B2 + g0) >> 2) + q;
      if (o.h) reinterpret_cast<int4*>(o.h)[i4] = c;
      if (o.f32)
        reinterpret_cast<float4*>(o.f32)[i4] = make_float4(c.x * sc, c.y * sc, c.z * sc, c.w * sc);
      if (o.bf16) {
        __nv_bfloat162 p0 = __floats2bfloat162_rn(c.x * sc, c.y * sc);
        __nv_bfloat162 p1 = __floats2bfloat162_rn(c.z * sc, c.w * sc);
        uint2 p;
        p.x = *reinterpret_cast<uint32_t*>(&p0);
        p.y = *reinterpret_cast<uint32_t*>(&p1);
        reinterpret_cast<uint2*>(o.bf16)[i4] = p;
      }
      if (o.sumsq)
        sumsq += static_cast<unsigned long long>(c.x) * c.x + static_cast<unsigned long long>(c.y) * c.y +
                 static_cast<unsigned long long>(c.z) * c.z + static_cast<unsigned long long>(c.w) * c.w;
    }
    // the next row's updates touch V only; S is rewritten after the barrier
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
                cudaStream_t s) {
  int n = N * N;
  prof_begin(PROF_BINS, s);
  k_bin_normals<<<grid_for(n, kThreads), kThreads, 0, s>>>(
      reinterpret_cast<const float2*>(d_normal_xy), n, bins, d_bins, d_status);
  prof_end(PROF_BINS, s);
  GSP_CHECK_LAUNCH();
  return GSP_OK;
}

size_t box_hist_smem(int N) {
  return static_cast<size_t>(N) * kHistG * sizeof(uint16_t) +
         static_cast<size_t>(N + 1) * kHistG * sizeof(int);
}

int launch_box_hist(const uint16_t* d_bins, int N, int levels, int bins, const HistOut& o,
                    cudaStream_t s) {
  const int B2 = bins * bins;
  if (B2 % kHistG) return GSP_ERR_UNSUPPORTED;
  const int ychunk = N >= 128 ? 128 : N;
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
  if (!d_normal_xy || !d_bins || !is_pow2(N) || N < 2 || N > 4096 || !is_pow2(bins) ||
      bins < 4 || bins > 128)
    return GSP_ERR_INVALID_ARG;
  return launch_bins(d_normal_xy, N, bins, d_bins, d_status, to_stream(stream));
}

extern "C" size_t gsp_build_workspace_bytes(int N, int levels, int bins) {
  if (!valid_map(N, levels, bins)) return 0;
  return align_up(static_cast<size_t>(N) * N * sizeof(uint16_t), 256);
}

extern "C" int gsp_build_footprint_ndfs(const float* d_normal_xy, int N, int levels, int bins,
                                        int32_t* d_hist, void* d_ws, size_t ws_bytes,
                                        uint32_t* d_status, gsp_stream stream) {
  if (!d_normal_xy || !d_hist || !valid_map(N, levels, bins)) return GSP_ERR_INVALID_ARG;
  if (!d_ws || ws_bytes < gsp_build_workspace_bytes(N, levels, bins)) return GSP_ERR_WORKSPACE;
  cudaStream_t s = to_stream(stream);
  uint16_t* bins_map = static_cast<uint16_t*>(d_ws);
  GSP_TRY(launch_bins(d_normal_xy, N, bins, bins_map, d_status, s));
  HistOut o{};
  o.h = d_hist;
  for (int l = 0; l < levels; ++l) o.scale[l] = 1.0f;
  return launch_box_hist(bins_map, N, levels, bins, o, s);
}
