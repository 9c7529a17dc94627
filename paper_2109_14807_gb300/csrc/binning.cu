// Rows a1-a3: binning of the normal map and exhaustive multi-level footprint
// histograms (Sec. 4.1), written straight into int32 counts and/or the
// scaled MTTKRP operand.
//
// Level 0 is the one-hot count of every texel's bin.  Level l+1 follows from
// level l because a 2^(l+1) box window centred as in Sec. 4.1 splits into two
// 2^l windows shifted by -/+ 2^(l-1) along each axis, so every count of the
// next level is the sum of four counts of the current one.  All arithmetic is
// integer, hence bit-exact.  The kernels are bound by HBM traffic: each level
// reads one int32 slice and writes one (plus the optional operand copy).
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

// one thread per 4 consecutive bins of one texel
__global__ void k_level0(const uint16_t* __restrict__ bins_map, long long total, int vpt_log,
                         LevelSink o) {
  long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  bool active = i < total;
  int4 v = make_int4(0, 0, 0, 0);
  if (active) {
    long long texel = i >> vpt_log;
    int b0 = static_cast<int>(i & ((1LL << vpt_log) - 1)) * 4;
    int code = bins_map[texel];
    v = make_int4(code == b0, code == b0 + 1, code == b0 + 2, code == b0 + 3);
    sink_store(o, i, v);
  }
  sink_sumsq(o, v, active);
}

// Level l+1 from level l.  Output rows are visited in the order
// y = j + i * 2d (j < 2d, i < N / 2d) so that consecutive rows share one of
// their two input rows (y + d of one is y' - d of the next) while it is in L2.
__global__ void k_double(const int4* __restrict__ in, long long total, int logN, int vpt_log,
                         int lo, int hi, int d2, LevelSink o) {
  long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  bool active = i < total;
  int4 s = make_int4(0, 0, 0, 0);
  if (active) {
    const int N = 1 << logN;
    const int row_log = logN + vpt_log;
    int k = static_cast<int>(i >> row_log);
    long long rem = i & ((1LL << row_log) - 1);
    int x = static_cast<int>(rem >> vpt_log);
    int b = static_cast<int>(rem & ((1LL << vpt_log) - 1));
    int y = k;
    if (d2 > 0) {
      int G = N / d2;
      y = (k / G) + (k % G) * d2;
    }
    const int m = N - 1;
    int ya = (y + lo) & m, yb = (y + hi) & m, xa = (x + lo) & m, xb = (x + hi) & m;
    int4 a = in[(((static_cast<long long>(ya) << logN) + xa) << vpt_log) + b];
    int4 c = in[(((static_cast<long long>(ya) << logN) + xb) << vpt_log) + b];
    int4 e = in[(((static_cast<long long>(yb) << logN) + xa) << vpt_log) + b];
    int4 g = in[(((static_cast<long long>(yb) << logN) + xb) << vpt_log) + b];
    s = make_int4(a.x + c.x + e.x + g.x, a.y + c.y + e.y + g.y, a.z + c.z + e.z + g.z,
                  a.w + c.w + e.w + g.w);
    long long oi = (((static_cast<long long>(y) << logN) + x) << vpt_log) + b;
    sink_store(o, oi, s);
  }
  sink_sumsq(o, s, active);
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

int launch_level0(const uint16_t* d_bins, int N, int bins, LevelSink o, cudaStream_t s) {
  int vpt_log = ilog2(static_cast<long long>(bins) * bins / 4);
  long long total = static_cast<long long>(N) * N << vpt_log;
  prof_begin(PROF_LEVEL0, s);
  k_level0<<<grid_for(total, kThreads), kThreads, 0, s>>>(d_bins, total, vpt_log, o);
  prof_end(PROF_LEVEL0, s);
  GSP_CHECK_LAUNCH();
  return GSP_OK;
}

int launch_double(const int32_t* d_in, int N, int bins, int level_in, LevelSink o, cudaStream_t s) {
  int vpt_log = ilog2(static_cast<long long>(bins) * bins / 4);
  int logN = ilog2(N);
  long long total = static_cast<long long>(N) * N << vpt_log;
  int lo, hi, d2;
  if (level_in == 0) {
    lo = -1, hi = 0, d2 = 0;
  } else {
    int d = 1 << (level_in - 1);
    lo = -d, hi = d, d2 = 2 * d <= N ? 2 * d : 0;
  }
  prof_begin(PROF_DOUBLE, s);
  k_double<<<grid_for(total, kThreads), kThreads, 0, s>>>(reinterpret_cast<const int4*>(d_in),
                                                          total, logN, vpt_log, lo, hi, d2, o);
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
  const long long slice = static_cast<long long>(N) * N * bins * bins;
  LevelSink o{d_hist, nullptr, nullptr, 1.0f, nullptr};
  GSP_TRY(launch_level0(bins_map, N, bins, o, s));
  for (int l = 1; l < levels; ++l) {
    o.h = d_hist + slice * l;
    GSP_TRY(launch_double(d_hist + slice * (l - 1), N, bins, l - 1, o, s));
  }
  return GSP_OK;
}
