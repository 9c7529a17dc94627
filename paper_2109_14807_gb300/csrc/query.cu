// Rows a5-a7: query tables (1D summed-area tables, Sec. 4.4), the batched
// spatio-angular range query (Eq. 5 over five modes, Sec. 4.3-4.4), its adjoint
// and the Adam refinement step.
//
// Query mapping: a group of LANES consecutive lanes serves one query; lane j
// owns runs of V consecutive ranks (V = 4, 2 or 1, as the ranks and the
// alignment of the factor rows allow), j*V, j*V + V*LANES, ... of every
// 32-rank block, and reads each run of a table row as one vector load per
// plane.  The rank sum is a butterfly over the group (results do not depend
// on LANES or V).  Every table row a query touches is read by the group as one
// contiguous run (coalesced), and the small per-material tables stay resident
// in L1/L2.  Warps claim `chunk` batches of 32 queries at a time from a global
// counter (persistent CTAs, dynamic balance over uneven materials); the
// per-query terms of a batch are formed once, one query per lane, and shared
// with the lane groups through shared memory.
#include <math.h>

#include <mutex>

#include "common.cuh"

namespace gsp {
namespace {

struct MatParams {
  gsp_material m[GSP_MAX_MATERIALS];
  int n;
};

// The SAT region starts after flw, padded to a multiple of 4 floats so that
// it is 16-byte aligned.
__host__ __device__ __forceinline__ size_t flw_floats(int L, int R) {
  return (static_cast<size_t>(L) * R + 3) / 4 * 4;
}

// Summed-area table of one angular side: rows i = 0..B of three planes of R
// floats: hi, lo (hi + lo = sum_{k<i} f[k], an FP64 sum split into two FP32)
// and the bin value f[i] (0 at i = B).
constexpr int kSatPlanes = 3;
__device__ __forceinline__ const float* sat_plane(const float* sat, int R, int i, int c) {
  return sat + (static_cast<size_t>(i) * kSatPlanes + c) * R;
}

// V consecutive floats (p aligned to min(V, 4) floats).
template <int V>
__device__ __forceinline__ void ldg_n(const float* __restrict__ p, float (&v)[V]) {
  if constexpr (V % 4 == 0) {
#pragma unroll
    for (int i = 0; i < V; i += 4) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(p + i));
      v[i] = a.x; v[i + 1] = a.y; v[i + 2] = a.z; v[i + 3] = a.w;
    }
  } else if constexpr (V == 2) {
    const float2 a = __ldg(reinterpret_cast<const float2*>(p));
    v[0] = a.x; v[1] = a.y;
  } else {
    v[0] = __ldg(p);
  }
}

struct GradParams {
  gsp_material_grad g[GSP_MAX_MATERIALS];
  float* dps[GSP_MAX_MATERIALS];  // [B+1][R] gradient w.r.t. the s-table prefix sums
  float* dpt[GSP_MAX_MATERIALS];
  // When use_smem: each CTA accumulates the small per-material tables
  // (dflw, dps, dpt, dfs, dft, in that order from soff[m]) in shared memory and
  // adds them to global memory once at the end.
  int soff[GSP_MAX_MATERIALS + 1];
  int use_smem;
  // Packed-query kernel (k_range_query_bwd_q): kBwdCopies private copies of
  // the small tables in the workspace, priv_floats floats each; material m's
  // tables (dflw [L][R], dP_s [B+1][R], dP_t [B+1][R]) at poff[m] in a copy.
  float* priv;
  int poff[GSP_MAX_MATERIALS + 1];
  int priv_floats;
};

struct SmallGrad {
  float *dflw, *dps, *dpt, *dfs, *dft;
};

__device__ __forceinline__ SmallGrad small_tables(float* base, const gsp_material& M) {
  const int R = M.rank, L = M.levels, B = M.bins;
  SmallGrad t;
  t.dflw = base;
  t.dps = t.dflw + L * R;
  t.dpt = t.dps + (B + 1) * R;
  t.dfs = t.dpt + (B + 1) * R;
  t.dft = t.dfs + B * R;
  return t;
}

// ---------------------------------------------------------------- tables --
__global__ void k_tables(const float* __restrict__ fl, const float* __restrict__ lambda,
                         const float* __restrict__ fs, const float* __restrict__ ft, int L,
                         int B, int R, float* __restrict__ tables) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  const float lam = lambda[r];
  for (int l = 0; l < L; ++l) tables[l * R + r] = fl[l * R + r] * lam;
  float* sat = tables + flw_floats(L, R);
  for (int side = 0; side < 2; ++side) {
    const float* f = side == 0 ? fs : ft;
    float* t = sat + static_cast<size_t>(side) * (B + 1) * kSatPlanes * R;
    double P = 0.0;  // running prefix sum, FP64
    for (int i = 0; i <= B; ++i) {
      float hi = static_cast<float>(P);
      float lo = static_cast<float>(P - static_cast<double>(hi));
      float fi = i < B ? f[i * R + r] : 0.0f;
      float* row = t + static_cast<size_t>(i) * kSatPlanes * R;
      row[r] = hi;
      row[R + r] = lo;
      row[2 * R + r] = fi;
      if (i < B) P += static_cast<double>(fi);
    }
  }
}

// ----------------------------------------------------------- query terms --
// Everything a query needs besides per-rank table reads.
struct QTerms {
  int x, y, l0, l1;
  float f;          // level blend weight of l1
  int is0, is1, it0, it1;
  float fs0, fs1, ft0, ft1;  // fractional parts of the range ends
  float inv_ws, inv_wt;      // 1 / width, 0 for a zero-width side
  int isz, itz;              // bin of a zero-width side
  bool ok;
};

__device__ __forceinline__ void load_query(const gsp_query* __restrict__ q, long long i,
                                           gsp_query& d) {
  const int4* p = reinterpret_cast<const int4*>(q + i);
  int4 a = __ldg(p), b = __ldg(p + 1);
  d.x = a.x;
  d.y = a.y;
  d.level = __int_as_float(a.z);
  d.s0 = __int_as_float(a.w);
  d.s1 = __int_as_float(b.x);
  d.t0 = __int_as_float(b.y);
  d.t1 = __int_as_float(b.z);
  d.material = static_cast<uint32_t>(b.w);
}

__device__ __forceinline__ void range_side(float a, float b, int B, int& i0, int& i1, float& f0,
                                           float& f1, float& inv_w, int& iz) {
  a = fminf(fmaxf(a, 0.0f), static_cast<float>(B));
  b = fminf(fmaxf(b, 0.0f), static_cast<float>(B));
  if (b < a) {
    float t = a;
    a = b;
    b = t;
  }
  float fa = floorf(a), fb = floorf(b);
  i0 = static_cast<int>(fa);
  i1 = static_cast<int>(fb);
  f0 = a - fa;
  f1 = b - fb;
  float w = b - a;
  inv_w = w > 0.0f ? 1.0f / w : 0.0f;
  iz = min(i0, B - 1);
}

__device__ __forceinline__ QTerms query_terms(const gsp_query& d, const gsp_material& M) {
  QTerms t;
  const int N = M.N, L = M.levels, B = M.bins;
  t.ok = isfinite(d.level) && isfinite(d.s0) && isfinite(d.s1) && isfinite(d.t0) &&
         isfinite(d.t1);
  t.x = d.x & (N - 1);  // N is a power of two: two's complement wrap
  t.y = d.y & (N - 1);
  float lev = t.ok ? fminf(fmaxf(d.level, 0.0f), static_cast<float>(L - 1)) : 0.0f;
  float fl0 = floorf(lev);
  t.l0 = static_cast<int>(fl0);
  t.f = lev - fl0;
  t.l1 = min(t.l0 + 1, L - 1);
  range_side(t.ok ? d.s0 : 0.f, t.ok ? d.s1 : 0.f, B, t.is0, t.is1, t.fs0, t.fs1, t.inv_ws, t.isz);
  range_side(t.ok ? d.t0 : 0.f, t.ok ? d.t1 : 0.f, B, t.it0, t.it1, t.ft0, t.ft1, t.inv_wt, t.itz);
  return t;
}

// Range averages of the V consecutive ranks rb .. rb + V - 1 from the SAT of
// one side: prefix(i0 + 1), f[i0], prefix(i1) and f[i1].  The partial end bins
// are weighted directly and only the whole bins between them come from the
// prefix difference, so each part is rounded relative to its own size: a
// range that starts just before the end of a large bin followed by zeros
// keeps its small integral instead of cancelling two large prefix values.  A
// range inside one bin is that bin's value; a zero-width range the value of
// bin iz.  (i0 + 1 <= B whenever the width is positive.)
template <int V>
__device__ __forceinline__ void sat_mean(const float* __restrict__ sat, int R, int rb, int i0,
                                         int i1, float f0, float f1, float inv_w, int iz,
                                         float (&out)[V]) {
  if (inv_w > 0.0f) {
    float ah[V], al[V], af[V], bh[V], bl[V], bf[V];
    ldg_n<V>(sat_plane(sat, R, i0 + 1, 0) + rb, ah);
    ldg_n<V>(sat_plane(sat, R, i0 + 1, 1) + rb, al);
    ldg_n<V>(sat_plane(sat, R, i0, 2) + rb, af);
    ldg_n<V>(sat_plane(sat, R, i1, 0) + rb, bh);
    ldg_n<V>(sat_plane(sat, R, i1, 1) + rb, bl);
    ldg_n<V>(sat_plane(sat, R, i1, 2) + rb, bf);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const float mid = (bh[v] - ah[v]) + (bl[v] - al[v]);
      const float m = fmaf(f1, bf[v], fmaf(1.0f - f0, af[v], mid)) * inv_w;
      out[v] = i0 == i1 ? af[v] : m;  // inside one bin: the bin's value
    }
  } else {
    ldg_n<V>(sat_plane(sat, R, iz, 2) + rb, out);
  }
}

// Rank sum, identical for every launch shape: rank r belongs to "conceptual
// lane" c = r mod 32, accumulated in increasing r; the 32 conceptual lanes are
// then combined in the order of a 32-lane xor butterfly (offsets 16, 8, 4, 2,
// 1).  Lane j of a group of LANES holds NC = 32 / LANES conceptual lanes in
// registers, c = V*j + v + k*V*LANES (v < V, k < NC / V): runs of V
// consecutive ranks, read as one vector load per table row and plane.  The
// butterfly offsets >= V*LANES (bits of k) are register adds, those from V to
// V*LANES shuffles, those below V register adds again.
template <int LANES, bool FXY, int V>
__global__ void __launch_bounds__(256) k_range_query(const __grid_constant__ MatParams mp,
                                                     const gsp_query* __restrict__ q,
                                                     long long n, float* __restrict__ out,
                                                     uint32_t* status,
                                                     unsigned long long* counter, int chunk) {
  constexpr int QPW = 32 / LANES;  // queries per warp step
  constexpr int NC = 32 / LANES;   // conceptual lanes per lane
  // per warp: the terms of its current batch of 32 queries (blockDim.x <= 256),
  // packed into 3 float4 (4 with fractional x, y): small integers share words
  // and the zero-width bins are derived from the material by the reader
  constexpr int NS = FXY ? 4 : 3;
  __shared__ float4 tslots[8][32][NS];
  const int lane = threadIdx.x & 31;
  const int sub = lane / LANES;
  const int j = lane % LANES;
  float4 (*slots)[NS] = tslots[threadIdx.x >> 5];
  // a grab is `chunk` batches of 32 queries; lane k of the warp loads and
  // evaluates query k of a batch (one batch ahead: the HBM latency of the
  // descriptors overlaps the previous batch) and stores its terms in the
  // warp's slots, which the lane group processing that query reads
  const long long per_grab = static_cast<long long>(chunk) * 32;
  const long long warp_id = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) >> 5;
  const long long n_warps = (static_cast<long long>(gridDim.x) * blockDim.x) >> 5;
  long long grab = 0;
  auto next_grab = [&]() -> long long {
    if (counter) {
      unsigned long long b = 0;
      if (lane == 0) b = atomicAdd(counter, static_cast<unsigned long long>(per_grab));
      return static_cast<long long>(__shfl_sync(0xffffffffu, b, 0));
    }
    return (warp_id + (grab++) * n_warps) * per_grab;
  };
  long long base = next_grab();
  gsp_query dn{};
  if (base + lane < n) load_query(q, base + lane, dn);
  while (base < n) {
    const long long following = next_grab();  // the grab after this one, claimed early
    for (int bt = 0; bt < chunk; ++bt) {
      const long long bbase = base + static_cast<long long>(bt) * 32;
      {
        const long long qk = bbase + lane;
        const gsp_query dk = dn;
        const long long nb = bt + 1 < chunk ? bbase + 32 : following;
        if (nb < n && nb + lane < n) load_query(q, nb + lane, dn);
        QTerms tk{};
        int mk = 0, flags = 0, ixk = 0, iyk = 0;
        float wxk = 0.f, wyk = 0.f;
        if (qk < n) {
          flags = 1;
          if (dk.material >= static_cast<uint32_t>(mp.n)) {
            flags |= 2;
          } else {
            mk = static_cast<int>(dk.material);
            tk = query_terms(dk, mp.m[mk]);
            bool bad = !tk.ok;
            ixk = tk.x;
            iyk = tk.y;
            if constexpr (FXY) {
              const float xf = __int_as_float(dk.x), yf = __int_as_float(dk.y);
              if (!(fabsf(xf) < 1073741824.0f) || !(fabsf(yf) < 1073741824.0f)) bad = true;
              const float x0 = bad ? 0.f : floorf(xf), y0 = bad ? 0.f : floorf(yf);
              wxk = bad ? 0.f : xf - x0;
              wyk = bad ? 0.f : yf - y0;
              ixk = static_cast<int>(x0);
              iyk = static_cast<int>(y0);
            }
            if (bad) flags |= 2;
          }
          if (flags & 2) set_status(status, GSP_DEV_BAD_QUERY);
        }
        __syncwarp();  // every lane is done with the previous batch's slots
        // l0, l1 < 64 levels, material < 256, flags < 4; bins <= 4096 < 2^16
        const int small = tk.l0 | (tk.l1 << 8) | (mk << 16) | (flags << 24);
        slots[lane][0] = make_float4(__int_as_float(ixk), __int_as_float(iyk), __int_as_float(small),
                                     __int_as_float(tk.is0 | (tk.is1 << 16)));
        slots[lane][1] = make_float4(__int_as_float(tk.it0 | (tk.it1 << 16)), tk.f, tk.fs0, tk.fs1);
        slots[lane][2] = make_float4(tk.ft0, tk.ft1, tk.inv_ws, tk.inv_wt);
        if constexpr (FXY) slots[lane][3] = make_float4(wxk, wyk, 0.f, 0.f);
        __syncwarp();
      }
      for (int it = 0; it < LANES; ++it) {
        const int slot = it * QPW + sub;
        const long long qi = bbase + slot;
        const float4 s0 = slots[slot][0];
        const int small = __float_as_int(s0.z);
        const int flags = small >> 24;
        float4 s1 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (flags == 1) s1 = slots[slot][1];
        // the second level row only when a query of this warp step blends two
        // levels (with weight 0 the blend is the first row exactly)
        const bool blend = __any_sync(0xffffffffu, flags == 1 && s1.y != 0.0f);
        float acc[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) acc[k] = 0.0f;
        {
          if (flags == 1) {  // in range and well formed
            const float4 s2 = slots[slot][2];
            const int mi = (small >> 16) & 0xFF;
            const gsp_material& M = mp.m[mi];
            QTerms t;
            t.x = __float_as_int(s0.x); t.y = __float_as_int(s0.y);
            t.l0 = small & 0xFF; t.l1 = (small >> 8) & 0xFF;
            const int ps = __float_as_int(s0.w), pt = __float_as_int(s1.x);
            t.is0 = ps & 0xFFFF; t.is1 = ps >> 16; t.it0 = pt & 0xFFFF; t.it1 = pt >> 16;
            t.f = s1.y; t.fs0 = s1.z; t.fs1 = s1.w;
            t.ft0 = s2.x; t.ft1 = s2.y; t.inv_ws = s2.z; t.inv_wt = s2.w;
            t.isz = min(t.is0, M.bins - 1);
            t.itz = min(t.it0, M.bins - 1);
            t.ok = true;
            const int R = M.rank;
            const float* __restrict__ flw = M.tables;
            const float* sats = M.tables + flw_floats(M.levels, R);
            const float* satt = sats + static_cast<size_t>(M.bins + 1) * kSatPlanes * R;
            const float* __restrict__ fxr = M.fx + static_cast<size_t>(t.x) * R;
            const float* __restrict__ fyr = M.fy + static_cast<size_t>(t.y) * R;
            const float* __restrict__ fxr1 = fxr;
            const float* __restrict__ fyr1 = fyr;
            float wx = 0.f, wy = 0.f;
            if constexpr (FXY) {  // x, y hold floor of the float position; wx, wy the blend
              const float4 s3 = slots[slot][3];
              wx = s3.x;
              wy = s3.y;
              const int N = M.N, ix = t.x, iy = t.y;
              fxr = M.fx + static_cast<size_t>(ix & (N - 1)) * R;
              fxr1 = M.fx + static_cast<size_t>((ix + 1) & (N - 1)) * R;
              fyr = M.fy + static_cast<size_t>(iy & (N - 1)) * R;
              fyr1 = M.fy + static_cast<size_t>((iy + 1) & (N - 1)) * R;
            }
            const float* __restrict__ fl0 = flw + static_cast<size_t>(t.l0) * R;
            const float* __restrict__ fl1 = flw + static_cast<size_t>(t.l1) * R;
            const float g0 = 1.0f - t.f;
            for (int r0 = 0; r0 < R; r0 += 32) {
#pragma unroll
              for (int k = 0; k < NC / V; ++k) {
                const int rb = r0 + k * V * LANES + V * j;  // R % V == 0: the run is whole
                if (rb < R) {
                  float a0[V], a1[V], xv[V], yv[V], S[V], T[V];
                  ldg_n<V>(fl0 + rb, a0);
                  if (blend) {
                    ldg_n<V>(fl1 + rb, a1);
                  } else {
#pragma unroll
                    for (int v = 0; v < V; ++v) a1[v] = 0.0f;
                  }
                  ldg_n<V>(fxr + rb, xv);
                  ldg_n<V>(fyr + rb, yv);
                  sat_mean<V>(sats, R, rb, t.is0, t.is1, t.fs0, t.fs1, t.inv_ws, t.isz, S);
                  sat_mean<V>(satt, R, rb, t.it0, t.it1, t.ft0, t.ft1, t.inv_wt, t.itz, T);
                  if constexpr (FXY) {
                    float x1[V], y1[V];
                    ldg_n<V>(fxr1 + rb, x1);
                    ldg_n<V>(fyr1 + rb, y1);
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                      xv[v] = fmaf(wx, x1[v] - xv[v], xv[v]);
                      yv[v] = fmaf(wy, y1[v] - yv[v], yv[v]);
                    }
                  }
#pragma unroll
                  for (int v = 0; v < V; ++v) {
                    const float lv = fmaf(t.f, a1[v], g0 * a0[v]);
                    acc[k * V + v] = fmaf(xv[v] * yv[v], lv * S[v] * T[v], acc[k * V + v]);
                  }
                }
              }
            }
          }
        }
        // butterfly: bits of k (registers), of j (shuffles), of v (registers)
#pragma unroll
        for (int o = 16; o >= V * LANES; o >>= 1) {
          const int h = o / (V * LANES);
#pragma unroll
          for (int k = 0; k < NC / V; ++k)
            if (!(k & h)) {
#pragma unroll
              for (int v = 0; v < V; ++v) acc[k * V + v] = acc[k * V + v] + acc[(k | h) * V + v];
            }
        }
#pragma unroll
        for (int o = V * LANES / 2; o >= V; o >>= 1) {
#pragma unroll
          for (int v = 0; v < V; ++v) acc[v] = acc[v] + __shfl_xor_sync(0xffffffffu, acc[v], o / V);
        }
#pragma unroll
        for (int o = V / 2; o > 0; o >>= 1) {
#pragma unroll
          for (int v = 0; v < V; ++v)
            if (!(v & o)) acc[v] = acc[v] + acc[v | o];
        }
        const float v = acc[0];
        if ((flags & 1) && j == 0) out[qi] = (flags & 2) ? __int_as_float(0x7fc00000) : v;
      }
    }
    base = following;
  }
}

// ----------------------------------------------------------- adjoint --
// Atomic add of VEC consecutive floats as one vector reduction.
template <int VEC>
__device__ __forceinline__ void red_add(float* p, const float* v) {
  if constexpr (VEC == 4) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v[0]), "f"(v[1]),
                 "f"(v[2]), "f"(v[3])
                 : "memory");
  } else if constexpr (VEC == 2) {
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(v[0]), "f"(v[1]) : "memory");
  } else {
    atomicAdd(p, v[0]);
  }
}

constexpr int kBwdThreads = 256;
constexpr int kBwdWarps = kBwdThreads / 32;

// One small gradient table: in shared memory (SMEM, a 32-bit shared address;
// additions are shared-memory reductions) or in global memory (atomics).  The
// address space is explicit: a generic atomic whose pointer may be either runs
// at less than half the rate on shared memory.
template <bool SMEM>
struct GTab;
template <>
struct GTab<true> {
  uint32_t a;
  __device__ __forceinline__ void add(int i, float v) const {
    asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(a + 4u * static_cast<uint32_t>(i)), "f"(v)
                 : "memory");
  }
};
template <>
struct GTab<false> {
  float* p;
  __device__ __forceinline__ void add(int i, float v) const { atomicAdd(p + i, v); }
};

template <bool SMEM>
struct GTabs {
  GTab<SMEM> dflw, dps, dpt, dfs, dft;
};

// Gradient of one side's range average S with respect to its table (Sec. 4.4,
// the form the forward evaluates):
//   S = f[i0]                                             (i0 == i1)
//   S = ((1 - f0) f[i0] + P[i1] - P[i0+1] + f1 f[i1]) / w  (i0 < i1)
//   S = f[iz]                                             (zero width)
// scaled by c: df[i0], df[i1] get the end-bin weights and dP[i1], dP[i0+1]
// +-c / w, the prefix rows only when whole bins lie between the ends (for
// i1 = i0 + 1 they cancel exactly).  Every weight is at most 1 in magnitude.
template <bool SMEM>
__device__ __forceinline__ void side_grad(const GTab<SMEM>& dp, const GTab<SMEM>& df, int R, int r,
                                          float c, int i0, int i1, float f0, float f1, float inv_w,
                                          int iz) {
  if (inv_w > 0.0f) {
    if (i0 == i1) {
      df.add(i0 * R + r, c);
    } else {
      const float a = c * inv_w;
      df.add(i0 * R + r, a * (1.0f - f0));
      if (f1 != 0.0f) df.add(i1 * R + r, a * f1);
      if (i1 > i0 + 1) {
        dp.add(i1 * R + r, a);
        dp.add((i0 + 1) * R + r, -a);
      }
    }
  } else {
    df.add(iz * R + r, c);
  }
}

// LANES lanes per query; lane j handles the VEC consecutive ranks
// j*VEC + k*LANES*VEC .. + VEC-1, so that its fx / fy gradient updates are
// vector reductions.  The per-CTA shared-memory tables store rank r of a row
// at column (r mod VEC) * R/VEC + r / VEC, so that the lanes' atomics for one
// v = r mod VEC hit consecutive words (no bank conflicts); the flush undoes it.
template <int LANES, int VEC, bool SMEM>
__global__ void __launch_bounds__(kBwdThreads, 2) k_range_query_bwd(const __grid_constant__ MatParams mp,
                                                         const __grid_constant__ GradParams gp,
                                                         const gsp_query* __restrict__ q,
                                                         long long n,
                                                         const float* __restrict__ gout,
                                                         uint32_t* status) {
  extern __shared__ float sacc[];
  __shared__ float4 tslots[kBwdWarps][32][5];  // per warp: the terms of its batch of 32 queries
  constexpr int QPW = 32 / LANES;
  const int lane = threadIdx.x & 31;
  const int sub = lane / LANES;
  const int j = lane % LANES;
  const long long warp_id = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) >> 5;
  const long long n_warps = (static_cast<long long>(gridDim.x) * blockDim.x) >> 5;
  if (SMEM) {
    for (int e = threadIdx.x; e < gp.soff[mp.n]; e += blockDim.x) sacc[e] = 0.0f;
    __syncthreads();
  }
  // Query terms are formed once per query: a warp takes batches of 32
  // queries, lane k loads query k of the batch (one batch ahead, so the HBM
  // latency overlaps the current batch) and stores its terms in the warp's
  // shared slots; each lane group then reads the slot of the query it
  // processes (five broadcast 16-byte loads).
  float4 (*slots)[5] = tslots[threadIdx.x >> 5];
  const long long n_batches = (n + 31) / 32;
  gsp_query dn{};
  float gn = 0.0f;
  if (warp_id < n_batches && warp_id * 32 + lane < n) {
    load_query(q, warp_id * 32 + lane, dn);
    gn = __ldg(gout + warp_id * 32 + lane);
  }
  for (long long bt = warp_id; bt < n_batches; bt += n_warps) {
    {
      const long long qk = bt * 32 + lane;
      const gsp_query dk = dn;
      const float gk = gn;
      const long long qn = (bt + n_warps) * 32 + lane;
      if (bt + n_warps < n_batches && qn < n) {
        load_query(q, qn, dn);
        gn = __ldg(gout + qn);
      }
      int live = 0, mk = 0;
      QTerms tk{};
      if (qk < n) {
        if (dk.material >= static_cast<uint32_t>(mp.n)) {
          set_status(status, GSP_DEV_BAD_QUERY);
        } else {
          mk = static_cast<int>(dk.material);
          tk = query_terms(dk, mp.m[mk]);
          if (!tk.ok) set_status(status, GSP_DEV_BAD_QUERY);
          live = tk.ok && gk != 0.0f;
        }
      }
      __syncwarp();  // every lane is done with the previous batch's slots
      slots[lane][0] = make_float4(__int_as_float(tk.x), __int_as_float(tk.y), __int_as_float(tk.l0),
                                   __int_as_float(tk.l1));
      slots[lane][1] = make_float4(tk.f, __int_as_float(tk.is0), __int_as_float(tk.is1), __int_as_float(tk.it0));
      slots[lane][2] = make_float4(__int_as_float(tk.it1), tk.fs0, tk.fs1, tk.ft0);
      slots[lane][3] = make_float4(tk.ft1, tk.inv_ws, tk.inv_wt, __int_as_float(tk.isz));
      slots[lane][4] = make_float4(__int_as_float(tk.itz), __int_as_float(mk), gk, __int_as_float(live));
      __syncwarp();
    }
    for (int it = 0; it < LANES; ++it) {
      const int slot = it * QPW + sub;
      const float4 w4 = slots[slot][4];
      if (!__float_as_int(w4.w)) continue;  // past the end, malformed or a zero gradient
      const float4 w0 = slots[slot][0], w1 = slots[slot][1], w2 = slots[slot][2], w3 = slots[slot][3];
      QTerms t;
      t.x = __float_as_int(w0.x); t.y = __float_as_int(w0.y);
      t.l0 = __float_as_int(w0.z); t.l1 = __float_as_int(w0.w);
      t.f = w1.x; t.is0 = __float_as_int(w1.y); t.is1 = __float_as_int(w1.z); t.it0 = __float_as_int(w1.w);
      t.it1 = __float_as_int(w2.x); t.fs0 = w2.y; t.fs1 = w2.z; t.ft0 = w2.w;
      t.ft1 = w3.x; t.inv_ws = w3.y; t.inv_wt = w3.z; t.isz = __float_as_int(w3.w);
      t.itz = __float_as_int(w4.x);
      t.ok = true;
      const int m = __float_as_int(w4.y);
      const float g = w4.z;
      const gsp_material& M = mp.m[m];
      const int R = M.rank;
      const float* flw = M.tables;
      const float* sats = M.tables + flw_floats(M.levels, R);
      const float* satt = sats + static_cast<size_t>(M.bins + 1) * kSatPlanes * R;
      const gsp_material_grad& G = gp.g[m];
      GTabs<SMEM> sg;
      if constexpr (SMEM) {
        const SmallGrad st = small_tables(sacc + gp.soff[m], M);
        auto sa = [](const float* q) { return static_cast<uint32_t>(__cvta_generic_to_shared(q)); };
        sg.dflw.a = sa(st.dflw);
        sg.dps.a = sa(st.dps);
        sg.dpt.a = sa(st.dpt);
        sg.dfs.a = sa(st.dfs);
        sg.dft.a = sa(st.dft);
      } else {
        sg.dflw.p = G.dflw;
        sg.dps.p = gp.dps[m];
        sg.dpt.p = gp.dpt[m];
        sg.dfs.p = G.dfs;
        sg.dft.p = G.dft;
      }
      const float g0 = 1.0f - t.f;
      for (int rv = j * VEC; rv < R; rv += LANES * VEC) {
        float a0v[VEC], a1v[VEC], xvv[VEC], yvv[VEC], dx[VEC], dy[VEC], Sv[VEC], Tv[VEC];
        ldg_n<VEC>(flw + t.l0 * R + rv, a0v);
        ldg_n<VEC>(flw + t.l1 * R + rv, a1v);
        ldg_n<VEC>(M.fx + t.x * R + rv, xvv);
        ldg_n<VEC>(M.fy + t.y * R + rv, yvv);
        sat_mean<VEC>(sats, R, rv, t.is0, t.is1, t.fs0, t.fs1, t.inv_ws, t.isz, Sv);
        sat_mean<VEC>(satt, R, rv, t.it0, t.it1, t.ft0, t.ft1, t.inv_wt, t.itz, Tv);
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
          const int r0 = rv + v;
          // column of rank r0 in this CTA's shared-memory tables (global: r0)
          const int r = SMEM ? v * (R / VEC) + rv / VEC : r0;
          float lv = fmaf(t.f, a1v[v], g0 * a0v[v]);
          float S = Sv[v];
          float T = Tv[v];
          float xv = xvv[v], yv = yvv[v];
          float xy = xv * yv;
          float st = S * T;
          dx[v] = g * yv * lv * st;
          dy[v] = g * xv * lv * st;
          sg.dflw.add(t.l0 * R + r, g * g0 * xy * st);
          if (t.f != 0.0f) sg.dflw.add(t.l1 * R + r, g * t.f * xy * st);
          side_grad<SMEM>(sg.dps, sg.dfs, R, r, g * xy * lv * T, t.is0, t.is1, t.fs0, t.fs1,
                          t.inv_ws, t.isz);
          side_grad<SMEM>(sg.dpt, sg.dft, R, r, g * xy * lv * S, t.it0, t.it1, t.ft0, t.ft1,
                          t.inv_wt, t.itz);
        }
        red_add<VEC>(G.dfx + t.x * R + rv, dx);
        red_add<VEC>(G.dfy + t.y * R + rv, dy);
      }
    }
  }
  if (SMEM) {
    __syncthreads();
    for (int m = 0; m < mp.n; ++m) {
      const gsp_material& M = mp.m[m];
      const int R = M.rank, L = M.levels, B = M.bins;
      const SmallGrad sg = small_tables(sacc + gp.soff[m], M);
      const gsp_material_grad& G = gp.g[m];
      const int RV = R / VEC;
      // shared column c holds rank (c mod R/VEC) * VEC + c / (R/VEC)
      auto gidx = [&](int e) { const int c = e % R; return e - c + (c % RV) * VEC + c / RV; };
      for (int e = threadIdx.x; e < L * R; e += blockDim.x)
        if (sg.dflw[e] != 0.0f) atomicAdd(G.dflw + gidx(e), sg.dflw[e]);
      for (int e = threadIdx.x; e < (B + 1) * R; e += blockDim.x) {
        if (sg.dps[e] != 0.0f) atomicAdd(gp.dps[m] + gidx(e), sg.dps[e]);
        if (sg.dpt[e] != 0.0f) atomicAdd(gp.dpt[m] + gidx(e), sg.dpt[e]);
      }
      for (int e = threadIdx.x; e < B * R; e += blockDim.x) {
        if (sg.dfs[e] != 0.0f) atomicAdd(G.dfs + gidx(e), sg.dfs[e]);
        if (sg.dft[e] != 0.0f) atomicAdd(G.dft + gidx(e), sg.dft[e]);
      }
    }
  }
}

// ------------------------------------------------- packed-query adjoint --
// The adjoint with the forward's lane mapping: LANES lanes per query (W =
// LANES * 4 <= 32 ranks per block, runs of 4 consecutive ranks per lane,
// float4 gathers), 32 / LANES queries per warp step.  The per-query work (terms,
// addresses, branches) is then shared by a quarter of a warp instead of all of
// it.  The small gradient tables (level rows, and the angular gradients in the
// prefix rows only, below) are accumulated in kBwdCopies private copies in
// global memory, CTA b adding to copy b mod kBwdCopies: a lane adds its run of
// 4 ranks to a row with one 16-byte reduction, which the L2's atomic units
// take (shared-memory float reductions, 10 per query and rank, were the
// kernel's bound: 2.24 ms against 1.5 ms per 10^7 bench queries).  k_bwd_flush
// sums the copies afterwards.  With E[j] = dP[j + 1] and dS/df[k] =
// sum_{j >= k} E[j], a side's update is
//   zero width / one bin i0:  dP[i0 + 1] += c, dP[i0] -= c
//   i0 < i1, a = c / w:       dP[i1 + 1] += a f1, dP[i1] += a (1 - f1) (i1 > i0 + 1),
//                             dP[i0 + 1] += a (1 - f0) - a_{i0+1}, dP[i0] -= a (1 - f0)
// with a_{i0+1} = a (i1 > i0 + 1) or a f1 (i1 = i0 + 1); k_suffix turns the
// prefix rows into the bin gradients (dP[0] is never read).  A batch's live
// queries (well formed, non-zero upstream gradient) are packed to the front of
// the warp's slots, so no lane group waits on a skipped query.
constexpr int kBwdCopies = 128;

// Add v to p (4 consecutive floats) at the L2, without a memory clobber: the
// private copies are read only by the next kernel.
__device__ __forceinline__ void red_add4_nc(float* p, const float (&v)[4]) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v[0]), "f"(v[1]),
               "f"(v[2]), "f"(v[3]));
}

// The prefix-row updates of one side for 4 ranks (values c[v]): rows and
// values as above; a row whose value is zero for this query is not added.
__device__ __forceinline__ void side_grad4(float* dp, int R, int rb, const float (&c)[4], int i0,
                                           int i1, float f0, float f1, float inv_w, int iz, int B) {
  const bool span = inv_w > 0.0f && i0 != i1;  // the range crosses a bin border
  const bool wide = i1 > i0 + 1;               // whole bins between the ends
  const int i = inv_w > 0.0f ? i0 : iz;
  float v1[4], v2[4], v3[4], v4[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const float a = c[v] * inv_w;
    const float e0 = a * (1.0f - f0);
    v1[v] = span ? a * f1 : c[v];
    v2[v] = a - a * f1;
    v3[v] = wide ? e0 - a : e0 - a * f1;
    v4[v] = span ? -e0 : -c[v];
  }
  red_add4_nc(dp + (span ? min(i1 + 1, B) : i + 1) * R + rb, v1);  // f1 = 0 when i1 = B
  if (span && wide) red_add4_nc(dp + i1 * R + rb, v2);
  if (span) red_add4_nc(dp + (i0 + 1) * R + rb, v3);
  red_add4_nc(dp + i * R + rb, v4);
}

// One CTA of 16 warps per SM.
constexpr int kBwdQThreads = 512;
constexpr int kBwdQWarps = kBwdQThreads / 32;

template <int LANES>
__global__ void __launch_bounds__(kBwdQThreads, 1) k_range_query_bwd_q(
    const __grid_constant__ MatParams mp, const __grid_constant__ GradParams gp,
    const gsp_query* __restrict__ q, long long n, const float* __restrict__ gout, uint32_t* status) {
  constexpr int V = 4;
  constexpr int W = V * LANES;  // ranks per block
  constexpr int QPW = 32 / LANES;
  __shared__ float4 tslots[kBwdQWarps][32][5];
  const int lane = threadIdx.x & 31;
  const int sub = lane / LANES;
  const int j = lane % LANES;
  const long long warp_id = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) >> 5;
  const long long n_warps = (static_cast<long long>(gridDim.x) * blockDim.x) >> 5;
  float* const copy = gp.priv + static_cast<size_t>(blockIdx.x % kBwdCopies) * gp.priv_floats;
  float4 (*slots)[5] = tslots[threadIdx.x >> 5];
  const long long n_batches = (n + 31) / 32;
  gsp_query dn{};
  float gn = 0.0f;
  if (warp_id < n_batches && warp_id * 32 + lane < n) {
    load_query(q, warp_id * 32 + lane, dn);
    gn = __ldg(gout + warp_id * 32 + lane);
  }
  for (long long bt = warp_id; bt < n_batches; bt += n_warps) {
    int n_live;
    {
      const long long qk = bt * 32 + lane;
      const gsp_query dk = dn;
      const float gk = gn;
      const long long qn = (bt + n_warps) * 32 + lane;
      if (bt + n_warps < n_batches && qn < n) {
        load_query(q, qn, dn);
        gn = __ldg(gout + qn);
      }
      bool live = false;
      int mk = 0;
      QTerms tk{};
      if (qk < n) {
        if (dk.material >= static_cast<uint32_t>(mp.n)) {
          set_status(status, GSP_DEV_BAD_QUERY);
        } else {
          mk = static_cast<int>(dk.material);
          tk = query_terms(dk, mp.m[mk]);
          if (!tk.ok) set_status(status, GSP_DEV_BAD_QUERY);
          live = tk.ok && gk != 0.0f;
        }
      }
      const unsigned ball = __ballot_sync(0xffffffffu, live);
      n_live = __popc(ball);
      const int pos = __popc(ball & ((1u << lane) - 1u));
      __syncwarp();  // every lane is done with the previous batch's slots
      if (live) {
        slots[pos][0] = make_float4(__int_as_float(tk.x), __int_as_float(tk.y), __int_as_float(tk.l0),
                                    __int_as_float(tk.l1));
        slots[pos][1] = make_float4(tk.f, __int_as_float(tk.is0), __int_as_float(tk.is1),
                                    __int_as_float(tk.it0));
        slots[pos][2] = make_float4(__int_as_float(tk.it1), tk.fs0, tk.fs1, tk.ft0);
        slots[pos][3] = make_float4(tk.ft1, tk.inv_ws, tk.inv_wt, __int_as_float(tk.isz));
        slots[pos][4] = make_float4(__int_as_float(tk.itz), __int_as_float(mk), gk, 0.0f);
      }
      __syncwarp();
    }
    for (int s0 = 0; s0 < n_live; s0 += QPW) {
      const int slot = s0 + sub;
      if (slot >= n_live) continue;
      const float4 w0 = slots[slot][0], w1 = slots[slot][1], w2 = slots[slot][2],
                   w3 = slots[slot][3], w4 = slots[slot][4];
      const int x = __float_as_int(w0.x), y = __float_as_int(w0.y);
      const int l0 = __float_as_int(w0.z), l1 = __float_as_int(w0.w);
      const float f = w1.x;
      const int is0 = __float_as_int(w1.y), is1 = __float_as_int(w1.z), it0 = __float_as_int(w1.w);
      const int it1 = __float_as_int(w2.x);
      const float fs0 = w2.y, fs1 = w2.z, ft0 = w2.w, ft1 = w3.x, inv_ws = w3.y, inv_wt = w3.z;
      const int isz = __float_as_int(w3.w), itz = __float_as_int(w4.x);
      const int m = __float_as_int(w4.y);
      const float g = w4.z;
      const gsp_material& M = mp.m[m];
      const int R = M.rank, L = M.levels, B = M.bins;
      const float* flw = M.tables;
      const float* sats = M.tables + flw_floats(L, R);
      const float* satt = sats + static_cast<size_t>(B + 1) * kSatPlanes * R;
      const gsp_material_grad& G = gp.g[m];
      float* const tflw = copy + gp.poff[m];   // [L][R]
      float* const tps = tflw + L * R;         // [B + 1][R]
      float* const tpt = tps + (B + 1) * R;    // [B + 1][R]
      const float g0 = 1.0f - f;
      // the second level row only when a query of this step blends two levels
      // (warp-uniform over the active lane groups, so no divergence)
      const bool blend = __any_sync(__activemask(), f != 0.0f);
      for (int r0 = 0; r0 < R; r0 += W) {
        const int rb = r0 + V * j;
        float a0[V], a1[V], xv[V], yv[V], S[V], T[V], dx[V], dy[V];
        ldg_n<V>(flw + l0 * R + rb, a0);
        ldg_n<V>(flw + l1 * R + rb, a1);
        ldg_n<V>(M.fx + static_cast<size_t>(x) * R + rb, xv);
        ldg_n<V>(M.fy + static_cast<size_t>(y) * R + rb, yv);
        sat_mean<V>(sats, R, rb, is0, is1, fs0, fs1, inv_ws, isz, S);
        sat_mean<V>(satt, R, rb, it0, it1, ft0, ft1, inv_wt, itz, T);
        // each group of reductions goes out as soon as its values exist
        float lv[V], gxl[V], t4[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
          lv[v] = fmaf(f, a1[v], g0 * a0[v]);
          t4[v] = g * xv[v] * yv[v] * S[v] * T[v] * g0;  // level row l0
        }
        red_add4_nc(tflw + l0 * R + rb, t4);
        if (blend) {
#pragma unroll
          for (int v = 0; v < V; ++v) t4[v] = g * xv[v] * yv[v] * S[v] * T[v] * f;
          red_add4_nc(tflw + l1 * R + rb, t4);
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
          gxl[v] = g * xv[v] * yv[v] * lv[v];
          t4[v] = gxl[v] * T[v];
        }
        side_grad4(tps, R, rb, t4, is0, is1, fs0, fs1, inv_ws, isz, B);
#pragma unroll
        for (int v = 0; v < V; ++v) t4[v] = gxl[v] * S[v];
        side_grad4(tpt, R, rb, t4, it0, it1, ft0, ft1, inv_wt, itz, B);
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const float st = S[v] * T[v];
          dx[v] = g * yv[v] * lv[v] * st;
          dy[v] = g * xv[v] * lv[v] * st;
        }
        red_add<V>(G.dfx + static_cast<size_t>(x) * R + rb, dx);
        red_add<V>(G.dfy + static_cast<size_t>(y) * R + rb, dy);
      }
    }
  }
}

// The private copies of k_range_query_bwd_q summed into the level-row
// gradients (the caller's dflw, added to) and the prefix-row gradients (the
// workspace's dps, dpt); thread: one entry of one material's tables.
__global__ void k_bwd_flush(const __grid_constant__ MatParams mp, const __grid_constant__ GradParams gp,
                            int copies) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  const gsp_material& M = mp.m[m];
  const int R = M.rank, L = M.levels, B = M.bins;
  if (e >= (L + 2 * (B + 1)) * R) return;
  const float* src = gp.priv + gp.poff[m] + e;
  float sum = 0.0f;
#pragma unroll 8
  for (int c = 0; c < copies; ++c) sum += __ldcg(src + static_cast<size_t>(c) * gp.priv_floats);
  if (sum == 0.0f) return;
  if (e < L * R)
    atomicAdd(gp.g[m].dflw + e, sum);  // materials may share their gradient arrays
  else if (e < (L + B + 1) * R)
    gp.dps[m][e - L * R] += sum;
  else
    gp.dpt[m][e - (L + B + 1) * R] += sum;
}

// dP[i] is the gradient w.r.t. P[i] = sum_{k<i} f[k]; so df[k] += sum_{i>k} dP[i].
__global__ void k_suffix(const float* __restrict__ dp, float* __restrict__ df, int B, int R) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  float acc = 0.0f;
  for (int i = B; i >= 1; --i) {
    acc += dp[i * R + r];
    df[(i - 1) * R + r] += acc;
  }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  float gi = g[i];
  float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
  float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
  m[i] = mi;
  v[i] = vi;
  float mh = mi / c1, vh = vi / c2;
  p[i] -= lr * mh / (sqrtf(vh) + eps);
}

bool valid_material(const gsp_material& m) {
  return is_pow2(m.N) && m.N >= 1 && m.N <= (1 << 20) && m.levels >= 1 && m.levels <= 64 &&
         m.bins >= 1 && m.bins <= 4096 && m.rank >= 1 && m.rank <= 256 && m.fx && m.fy &&
         m.tables && (reinterpret_cast<uintptr_t>(m.tables) & 15) == 0;
}

// -------------------------------------------------------------- sampling --
// Hierarchical NDF importance sampling (Sec. 5.2).  LANES lanes per sample;
// lane j holds ranks j and j + LANES (LANES >= R / 2) with their
// constant factor c_r = fx[x,r] fy[y,r] flw(level)[r] and the summed-area-table
// prefix sums at the current square's edges.  A step loads the prefix sums at
// the two midpoints, forms the four quad averages per rank, sums them over
// the lanes by an xor butterfly and takes the same choice on every lane.  The
// step count is the maximum over the warp's samples, so the shuffles of a
// warp stay in step whatever the materials.
constexpr int kSampleMaxRank = 64;

// V = 2: lane j holds the rank pair 2j, 2j + 1 and reads it as one float2 per
// table row and plane; V = 1: ranks j and j + LANES.
template <int LANES, int V>
__global__ void __launch_bounds__(256) k_sample_ndf(const __grid_constant__ MatParams mp,
                                                    const gsp_sample_query* __restrict__ q,
                                                    long long n, const float* __restrict__ u,
                                                    float* __restrict__ out, uint32_t* status) {
  constexpr int QPW = 32 / LANES;
  constexpr int NC = 2;  // rank slots per lane
  static_assert(V == 1 || V == NC, "runs of 1 or 2 ranks");
  const int lane = threadIdx.x & 31, sub = lane / LANES, j = lane % LANES;
  // rank of slot k
  auto slot_rank = [&](int k) { return V == 2 ? 2 * j + k : j + k * LANES; };
  // the slots' values of one table row (V consecutive floats per load; 0 for
  // a slot past the rank, which is never read: with V = 2 the rank is even)
  auto row2 = [&](const float* p, int R, float (&v)[NC]) {
#pragma unroll
    for (int k = 0; k < NC; k += V) {
      float w[V];
#pragma unroll
      for (int i = 0; i < V; ++i) w[i] = 0.f;
      if (slot_rank(k) < R) ldg_n<V>(p + slot_rank(k), w);
#pragma unroll
      for (int i = 0; i < V; ++i) v[k + i] = w[i];
    }
  };
  const long long warp_id = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) >> 5;
  const long long n_warps = (static_cast<long long>(gridDim.x) * blockDim.x) >> 5;
  for (long long base = warp_id * QPW; base < n; base += n_warps * QPW) {  // warp-uniform
    const long long qi = base + sub;
    const bool active = qi < n;
    int4 dq = make_int4(0, 0, 0, 0);
    if (active) dq = __ldg(reinterpret_cast<const int4*>(q) + qi);
    const float level = __int_as_float(dq.z);
    const uint32_t mi = static_cast<uint32_t>(dq.w);
    const bool bad = active && (mi >= static_cast<uint32_t>(mp.n) || !isfinite(level));
    const bool live = active && !bad;
    const gsp_material& M = mp.m[live ? mi : 0];
    const int R = M.rank, B = M.bins, N = M.N, L = M.levels;
    const int x = dq.x & (N - 1), y = dq.y & (N - 1);
    const float lev = live ? fminf(fmaxf(level, 0.0f), static_cast<float>(L - 1)) : 0.0f;
    const int l0 = static_cast<int>(floorf(lev)), l1 = min(l0 + 1, L - 1);
    const float f = lev - static_cast<float>(l0), g0 = 1.0f - f;
    const float* flw = M.tables;
    const float* sats = M.tables + flw_floats(L, R);
    const float* satt = sats + static_cast<size_t>(B + 1) * kSatPlanes * R;
    // per rank slot: c_r and the prefix sums (hi, lo) at the square's edges
    float c[NC], s0h[NC], s0l[NC], s1h[NC], s1l[NC], t0h[NC], t0l[NC], t1h[NC], t1l[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      c[k] = 0.f;
      s0h[k] = s0l[k] = s1h[k] = s1l[k] = t0h[k] = t0l[k] = t1h[k] = t1l[k] = 0.f;
    }
    // R is even for V = 2, so a pair is whole or absent
    const bool have = live && slot_rank(0) < R;
    if (have) {
      float xv[NC], yv[NC], a1[NC], a0[NC];
      row2(M.fx + static_cast<size_t>(x) * R, R, xv);
      row2(M.fy + static_cast<size_t>(y) * R, R, yv);
      row2(flw + l1 * R, R, a1);
      row2(flw + l0 * R, R, a0);
      row2(sat_plane(sats, R, 0, 0), R, s0h);
      row2(sat_plane(sats, R, 0, 1), R, s0l);
      row2(sat_plane(sats, R, B, 0), R, s1h);
      row2(sat_plane(sats, R, B, 1), R, s1l);
      row2(sat_plane(satt, R, 0, 0), R, t0h);
      row2(sat_plane(satt, R, 0, 1), R, t0l);
      row2(sat_plane(satt, R, B, 0), R, t1h);
      row2(sat_plane(satt, R, B, 1), R, t1l);
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        if (slot_rank(k) < R) {
          c[k] = xv[k] * yv[k] * fmaf(f, a1[k], g0 * a0[k]);
        } else {
          s0h[k] = s0l[k] = s1h[k] = s1l[k] = t0h[k] = t0l[k] = t1h[k] = t1l[k] = 0.f;
        }
      }
    }
    const float* uq = u + (live ? qi : 0) * GSP_SAMPLE_UNIFORMS;  // this sample's uniforms
    const int my_steps = live ? 31 - __clz(B) : 0;  // B is a power of two
    int steps = my_steps;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) steps = max(steps, __shfl_xor_sync(0xffffffffu, steps, o));
    int s0 = 0, t0 = 0, sz = B;
    float pmf = 1.0f, value = 0.0f;
    for (int st = 0; st < steps; ++st) {
      const bool go = st < my_steps;
      const int half = sz >> 1, sm = s0 + half, tm = t0 + half;
      const float inv = go ? 1.0f / static_cast<float>(half) : 0.0f;
      float q4[4] = {0.f, 0.f, 0.f, 0.f};
      float smh[NC], sml[NC], tmh[NC], tml[NC];
#pragma unroll
      for (int k = 0; k < NC; ++k) smh[k] = sml[k] = tmh[k] = tml[k] = 0.f;
      if (go && have) {
        row2(sat_plane(sats, R, sm, 0), R, smh);
        row2(sat_plane(sats, R, sm, 1), R, sml);
        row2(sat_plane(satt, R, tm, 0), R, tmh);
        row2(sat_plane(satt, R, tm, 1), R, tml);
#pragma unroll
        for (int k = 0; k < NC; ++k) {
          if (slot_rank(k) < R) {
            const float sa = ((smh[k] - s0h[k]) + (sml[k] - s0l[k])) * inv;
            const float sb = ((s1h[k] - smh[k]) + (s1l[k] - sml[k])) * inv;
            const float ta = ((tmh[k] - t0h[k]) + (tml[k] - t0l[k])) * inv;
            const float tb = ((t1h[k] - tmh[k]) + (t1l[k] - tml[k])) * inv;
            const float ca = c[k] * sa, cb = c[k] * sb;
            q4[0] = fmaf(ca, ta, q4[0]);
            q4[1] = fmaf(ca, tb, q4[1]);
            q4[2] = fmaf(cb, ta, q4[2]);
            q4[3] = fmaf(cb, tb, q4[3]);
          } else {
            smh[k] = sml[k] = tmh[k] = tml[k] = 0.f;
          }
        }
      }
#pragma unroll
      for (int o = LANES / 2; o > 0; o >>= 1) {
#pragma unroll
        for (int i = 0; i < 4; ++i) q4[i] += __shfl_xor_sync(0xffffffffu, q4[i], o);
      }
      if (go) {
        float p[4], tot = 0.f;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          p[i] = fmaxf(q4[i], 0.0f);
          tot += p[i];
        }
        int ch;
        const float ust = __ldg(uq + st);
        if (tot > 0.0f) {
          const float target = ust * tot;
          float cum = p[0];
          ch = 0;
          if (!(target < cum)) { cum += p[1]; ch = 1; }
          if (ch == 1 && !(target < cum)) { cum += p[2]; ch = 2; }
          if (ch == 2 && !(target < cum)) ch = 3;
          if (p[ch] <= 0.0f) {  // rounding put the target past a zero quad: last positive one
            ch = p[3] > 0.f ? 3 : p[2] > 0.f ? 2 : p[1] > 0.f ? 1 : 0;
          }
          pmf *= p[ch] / tot;
        } else {
          ch = min(3, static_cast<int>(ust * 4.0f));
          pmf *= 0.25f;
        }
        value = q4[ch];
        const bool s_hi = ch >= 2, t_hi = ch & 1;
#pragma unroll
        for (int k = 0; k < NC; ++k) {
          if (s_hi) { s0h[k] = smh[k]; s0l[k] = sml[k]; } else { s1h[k] = smh[k]; s1l[k] = sml[k]; }
          if (t_hi) { t0h[k] = tmh[k]; t0l[k] = tml[k]; } else { t1h[k] = tmh[k]; t1l[k] = tml[k]; }
        }
        if (s_hi) s0 = sm;
        if (t_hi) t0 = tm;
        sz = half;
      }
    }
    if (active && j == 0) {
      float4 o;
      if (bad) {
        o = make_float4(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000),
                        __int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
        set_status(status, GSP_DEV_BAD_QUERY);
      } else {
        // rounded down, so that bin + u stays inside the bin for u < 1
        o = make_float4(__fadd_rd(static_cast<float>(s0), __ldg(uq + 6)),
                        __fadd_rd(static_cast<float>(t0), __ldg(uq + 7)), pmf, value);
      }
      reinterpret_cast<float4*>(out)[qi] = o;
    }
  }
}

// Default lanes per query (the autotuner's choice replaces it): 8 from rank 64
// up, else 4, so that each lane reads runs of up to 4 ranks.
int pick_lanes(const gsp_material* mats, int n_mats, const gsp_query_tuning* tn) {
  if (tn && tn->lanes_per_query) return tn->lanes_per_query;
  int rmax = 1;
  for (int i = 0; i < n_mats; ++i) rmax = rmax > mats[i].rank ? rmax : mats[i].rank;
  return rmax >= 64 ? 8 : 4;
}

template <int LANES, int VEC, bool SMEM>
int launch_bwd_k(long long blocks, int threads, size_t dyn, cudaStream_t s, const MatParams& mp,
                 const GradParams& gp, const gsp_query* d_q, long long n, const float* d_gout,
                 uint32_t* d_status) {
  GSP_CUDA(cudaFuncSetAttribute(k_range_query_bwd<LANES, VEC, SMEM>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
  // one wave of resident CTAs (registers, shared memory): the grid-stride
  // loop then spreads the batches evenly, with no partial second wave
  int per_sm = 0;
  GSP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, k_range_query_bwd<LANES, VEC, SMEM>, threads, dyn));
  const long long cap = static_cast<long long>(sm_count()) * (per_sm > 0 ? per_sm : 1);
  if (blocks > cap) blocks = cap;
  k_range_query_bwd<LANES, VEC, SMEM><<<blocks, threads, dyn, s>>>(mp, gp, d_q, n, d_gout, d_status);
  return GSP_OK;
}

template <int LANES, int VEC>
int launch_bwd_t(long long blocks, int threads, size_t dyn, cudaStream_t s, const MatParams& mp,
                 const GradParams& gp, const gsp_query* d_q, long long n, const float* d_gout,
                 uint32_t* d_status) {
  if (gp.use_smem)
    return launch_bwd_k<LANES, VEC, true>(blocks, threads, dyn, s, mp, gp, d_q, n, d_gout, d_status);
  return launch_bwd_k<LANES, VEC, false>(blocks, threads, dyn, s, mp, gp, d_q, n, d_gout, d_status);
}

template <int LANES>
int launch_bwd_q(long long blocks, size_t dyn, cudaStream_t s, const MatParams& mp,
                 const GradParams& gp, const gsp_query* d_q, long long n, const float* d_gout,
                 uint32_t* d_status) {
  GSP_CUDA(cudaFuncSetAttribute(k_range_query_bwd_q<LANES>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(dyn)));
  int per_sm = 0;
  GSP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_range_query_bwd_q<LANES>,
                                                         kBwdQThreads, dyn));
  const long long cap = static_cast<long long>(sm_count()) * (per_sm > 0 ? per_sm : 1);
  if (blocks > cap) blocks = cap;
  k_range_query_bwd_q<LANES><<<blocks, kBwdQThreads, dyn, s>>>(mp, gp, d_q, n, d_gout, d_status);
  return GSP_OK;
}

template <int VEC>
int launch_bwd_v(int lanes, long long blocks, int threads, size_t dyn, cudaStream_t s,
                 const MatParams& mp, const GradParams& gp, const gsp_query* d_q, long long n,
                 const float* d_gout, uint32_t* d_status) {
  switch (lanes) {
    case 4: return launch_bwd_t<4, VEC>(blocks, threads, dyn, s, mp, gp, d_q, n, d_gout, d_status);
    case 8: return launch_bwd_t<8, VEC>(blocks, threads, dyn, s, mp, gp, d_q, n, d_gout, d_status);
    case 16: return launch_bwd_t<16, VEC>(blocks, threads, dyn, s, mp, gp, d_q, n, d_gout, d_status);
    default: return launch_bwd_t<32, VEC>(blocks, threads, dyn, s, mp, gp, d_q, n, d_gout, d_status);
  }
}

int launch_bwd(int lanes, int vec, long long blocks, int threads, size_t dyn, cudaStream_t s,
               const MatParams& mp, const GradParams& gp, const gsp_query* d_q, long long n,
               const float* d_gout, uint32_t* d_status) {
  if (vec == 4) return launch_bwd_v<4>(lanes, blocks, threads, dyn, s, mp, gp, d_q, n, d_gout, d_status);
  if (vec == 2) return launch_bwd_v<2>(lanes, blocks, threads, dyn, s, mp, gp, d_q, n, d_gout, d_status);
  return launch_bwd_v<1>(lanes, blocks, threads, dyn, s, mp, gp, d_q, n, d_gout, d_status);
}

}  // namespace
}  // namespace gsp

using namespace gsp;

extern "C" size_t gsp_query_table_floats(int levels, int bins, int rank) {
  if (levels < 1 || bins < 1 || rank < 1) return 0;
  return flw_floats(levels, rank) + 2 * kSatPlanes * static_cast<size_t>(bins + 1) * rank;
}

extern "C" int gsp_build_query_tables(const gsp_material* h_mat, gsp_stream stream) {
  if (!h_mat) return GSP_ERR_INVALID_ARG;
  const gsp_material& m = *h_mat;
  if (!valid_material(m) || !m.fl || !m.fs || !m.ft || !m.lambda) return GSP_ERR_INVALID_ARG;
  int threads = 64;
  prof_begin(PROF_TABLES, to_stream(stream));
  k_tables<<<grid_for(m.rank, threads), threads, 0, to_stream(stream)>>>(
      m.fl, m.lambda, m.fs, m.ft, m.levels, m.bins, m.rank, m.tables);
  prof_end(PROF_TABLES, to_stream(stream));
  GSP_CHECK_LAUNCH();
  return GSP_OK;
}

namespace gsp {
namespace {
template <bool FXY, int LANES, int V>
void launch_query_lv(long long blocks, int threads, cudaStream_t s, const MatParams& mp,
                     const gsp_query* d_q, long long n, float* d_out, uint32_t* d_status,
                     unsigned long long* counter, int chunk) {
  k_range_query<LANES, FXY, V><<<blocks, threads, 0, s>>>(mp, d_q, n, d_out, d_status, counter, chunk);
}

template <bool FXY, int LANES>
void launch_query_l(int vec, long long blocks, int threads, cudaStream_t s, const MatParams& mp,
                    const gsp_query* d_q, long long n, float* d_out, uint32_t* d_status,
                    unsigned long long* counter, int chunk) {
  constexpr int NC = 32 / LANES;
  if (vec >= 4 && NC >= 4)
    launch_query_lv<FXY, LANES, (NC >= 4 ? 4 : 1)>(blocks, threads, s, mp, d_q, n, d_out, d_status, counter, chunk);
  else if (vec >= 2 && NC >= 2)
    launch_query_lv<FXY, LANES, (NC >= 2 ? 2 : 1)>(blocks, threads, s, mp, d_q, n, d_out, d_status, counter, chunk);
  else
    launch_query_lv<FXY, LANES, 1>(blocks, threads, s, mp, d_q, n, d_out, d_status, counter, chunk);
}

template <bool FXY>
void launch_query_t(int lanes, int vec, long long blocks, int threads, cudaStream_t s,
                    const MatParams& mp, const gsp_query* d_q, long long n, float* d_out,
                    uint32_t* d_status, unsigned long long* counter, int chunk) {
  switch (lanes) {
    case 4: launch_query_l<FXY, 4>(vec, blocks, threads, s, mp, d_q, n, d_out, d_status, counter, chunk); break;
    case 8: launch_query_l<FXY, 8>(vec, blocks, threads, s, mp, d_q, n, d_out, d_status, counter, chunk); break;
    case 16: launch_query_l<FXY, 16>(vec, blocks, threads, s, mp, d_q, n, d_out, d_status, counter, chunk); break;
    default: launch_query_l<FXY, 32>(vec, blocks, threads, s, mp, d_q, n, d_out, d_status, counter, chunk); break;
  }
}

// Ranks per vector run: the largest of 4, 2 (at most 32 / lanes) that divides
// every rank, leaves no lane of the group without a run (V * lanes <= rank)
// and keeps the fx, fy rows aligned; else 1.
int pick_query_vec(const gsp_material* mats, int n_mats, int lanes) {
  for (int v = 32 / lanes < 4 ? 32 / lanes : 4; v > 1; v >>= 1) {
    bool ok = true;
    for (int i = 0; i < n_mats; ++i) {
      const gsp_material& m = mats[i];
      const uintptr_t mask = static_cast<uintptr_t>(4 * v - 1);
      ok = ok && m.rank % v == 0 && v * lanes <= m.rank &&
           ((reinterpret_cast<uintptr_t>(m.fx) | reinterpret_cast<uintptr_t>(m.fy)) & mask) == 0;
    }
    if (ok) return v;
  }
  return 1;
}

template <bool FXY>
int range_query_launch(const gsp_material* h_mats, int n_mats, const gsp_query* d_q, int64_t n,
                       float* d_out, uint32_t* d_status, const gsp_query_tuning* tuning,
                       void* d_ws, size_t ws_bytes, gsp_stream stream) {
  if (!h_mats || n_mats < 1 || n_mats > GSP_MAX_MATERIALS || n < 0) return GSP_ERR_INVALID_ARG;
  if (n > 0 && (!d_q || !d_out || (reinterpret_cast<uintptr_t>(d_q) & 15))) return GSP_ERR_INVALID_ARG;
  MatParams mp;
  mp.n = n_mats;
  for (int i = 0; i < n_mats; ++i) {
    if (!valid_material(h_mats[i])) return GSP_ERR_INVALID_ARG;
    mp.m[i] = h_mats[i];
  }
  if (n == 0) return GSP_OK;
  int lanes = pick_lanes(h_mats, n_mats, tuning);
  int threads = tuning && tuning->threads ? tuning->threads : 256;
  int bpsm = tuning && tuning->blocks_per_sm ? tuning->blocks_per_sm : 8;
  int chunk = tuning && tuning->chunk ? tuning->chunk : 4;
  if (threads < 32 || threads > 256 || threads % 32 || bpsm < 1 || bpsm > 32 || chunk < 1 ||
      chunk > 64)
    return GSP_ERR_INVALID_ARG;
  cudaStream_t s = to_stream(stream);
  unsigned long long* counter = nullptr;
  if (d_ws) {
    if (ws_bytes < 16) return GSP_ERR_WORKSPACE;
    counter = static_cast<unsigned long long*>(d_ws);
    GSP_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s));
  }
  long long warps_needed = (n + 32LL * chunk - 1) / (32LL * chunk);  // a grab: chunk batches of 32
  long long blocks = static_cast<long long>(sm_count()) * bpsm;
  long long need = (warps_needed * 32 + threads - 1) / threads;
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  if (lanes != 4 && lanes != 8 && lanes != 16 && lanes != 32) return GSP_ERR_INVALID_ARG;
  const int vec = pick_query_vec(h_mats, n_mats, lanes);
  prof_begin(PROF_QUERY, s);
  launch_query_t<FXY>(lanes, vec, blocks, threads, s, mp, d_q, n, d_out, d_status, counter, chunk);
  prof_end(PROF_QUERY, s);
  GSP_CHECK_LAUNCH();
  return GSP_OK;
}
}  // namespace
}  // namespace gsp

extern "C" int gsp_range_query(const gsp_material* h_mats, int n_mats, const gsp_query* d_q,
                               int64_t n, float* d_out, uint32_t* d_status,
                               const gsp_query_tuning* tuning, void* d_ws, size_t ws_bytes,
                               gsp_stream stream) {
  return range_query_launch<false>(h_mats, n_mats, d_q, n, d_out, d_status, tuning, d_ws,
                                   ws_bytes, stream);
}

extern "C" int gsp_range_query_interp(const gsp_material* h_mats, int n_mats,
                                      const gsp_query_f* d_q, int64_t n, float* d_out,
                                      uint32_t* d_status, const gsp_query_tuning* tuning,
                                      void* d_ws, size_t ws_bytes, gsp_stream stream) {
  // same 32-byte layout; the kernel reads words 0 and 1 as floats
  return range_query_launch<true>(h_mats, n_mats, reinterpret_cast<const gsp_query*>(d_q), n,
                                  d_out, d_status, tuning, d_ws, ws_bytes, stream);
}

// The prefix-row gradients dP_s, dP_t of every material, then kBwdCopies
// private copies of the small tables (level rows and both prefix-row sets).
extern "C" size_t gsp_backward_workspace_bytes(const gsp_material* h_mats, int n_mats) {
  if (!h_mats || n_mats < 1 || n_mats > GSP_MAX_MATERIALS) return 0;
  size_t total = 0, copy = 0;
  for (int i = 0; i < n_mats; ++i) {
    const gsp_material& m = h_mats[i];
    total += 2 * align_up(static_cast<size_t>(m.bins + 1) * m.rank * sizeof(float), 256);
    copy += static_cast<size_t>(m.levels + 2 * (m.bins + 1)) * m.rank;
  }
  return total + align_up(kBwdCopies * copy * sizeof(float), 256);
}

extern "C" int gsp_range_query_backward(const gsp_material* h_mats, int n_mats,
                                        const gsp_query* d_q, int64_t n, const float* d_gout,
                                        const gsp_material_grad* h_grads, void* d_ws,
                                        size_t ws_bytes, uint32_t* d_status, gsp_stream stream) {
  if (!h_mats || !h_grads || n_mats < 1 || n_mats > GSP_MAX_MATERIALS || n < 0)
    return GSP_ERR_INVALID_ARG;
  if (n > 0 && (!d_q || !d_gout || (reinterpret_cast<uintptr_t>(d_q) & 15))) return GSP_ERR_INVALID_ARG;
  size_t need = gsp_backward_workspace_bytes(h_mats, n_mats);
  if (!d_ws || ws_bytes < need) return GSP_ERR_WORKSPACE;
  MatParams mp;
  GradParams gp;
  mp.n = n_mats;
  char* w = static_cast<char*>(d_ws);
  for (int i = 0; i < n_mats; ++i) {
    const gsp_material& m = h_mats[i];
    const gsp_material_grad& g = h_grads[i];
    if (!valid_material(m) || !g.dfx || !g.dfy || !g.dflw || !g.dfs || !g.dft)
      return GSP_ERR_INVALID_ARG;
    mp.m[i] = m;
    gp.g[i] = g;
    size_t b = align_up(static_cast<size_t>(m.bins + 1) * m.rank * sizeof(float), 256);
    gp.dps[i] = reinterpret_cast<float*>(w);
    gp.dpt[i] = reinterpret_cast<float*>(w + b);
    w += 2 * b;
  }
  gp.priv = reinterpret_cast<float*>(w);  // 256-aligned
  int po = 0;
  for (int i = 0; i < n_mats; ++i) {
    gp.poff[i] = po;
    po += h_mats[i].rank * (h_mats[i].levels + 2 * (h_mats[i].bins + 1));
  }
  gp.poff[n_mats] = po;
  gp.priv_floats = po;
  // small tables of all materials in shared memory when they fit in 96 KB
  int off = 0;
  for (int i = 0; i < n_mats; ++i) {
    gp.soff[i] = off;
    const gsp_material& m = h_mats[i];
    off += m.rank * (m.levels + 2 * (m.bins + 1) + 2 * m.bins);
  }
  gp.soff[n_mats] = off;
  const size_t smem = static_cast<size_t>(off) * sizeof(float);
  gp.use_smem = smem <= 96 * 1024 ? 1 : 0;
  cudaStream_t s = to_stream(stream);
  GSP_CUDA(cudaMemsetAsync(d_ws, 0, need, s));
  // Packed-query kernel: every rank a multiple of W = min(32, R) >= 8 (the
  // same W for all materials), factor and gradient rows 16-byte aligned.
  int pw = 0;
  bool packed = true;
  for (int i = 0; i < n_mats && packed; ++i) {
    const gsp_material& m = h_mats[i];
    const gsp_material_grad& g = h_grads[i];
    const int wm = m.rank < 32 ? m.rank : 32;
    if (pw == 0) pw = wm;
    const uintptr_t al = reinterpret_cast<uintptr_t>(m.fx) | reinterpret_cast<uintptr_t>(m.fy) |
                         reinterpret_cast<uintptr_t>(g.dfx) | reinterpret_cast<uintptr_t>(g.dfy);
    packed = wm == pw && wm >= 8 && (wm & (wm - 1)) == 0 && m.rank % wm == 0 && (al & 15) == 0;
  }
  const int plan = pw / 4;  // lanes per query
  if (n > 0 && packed) {
    const long long blocks = ((n + 31) / 32 * 32 + kBwdQThreads - 1) / kBwdQThreads;
    int lmax = 0;
    for (int i = 0; i < n_mats; ++i)
      lmax = std::max(lmax, h_mats[i].rank * (h_mats[i].levels + 2 * (h_mats[i].bins + 1)));
    prof_begin(PROF_QUERY_BWD, s);
    int rc = GSP_OK;
    if (plan == 8)
      rc = launch_bwd_q<8>(blocks, 0, s, mp, gp, d_q, n, d_gout, d_status);
    else if (plan == 4)
      rc = launch_bwd_q<4>(blocks, 0, s, mp, gp, d_q, n, d_gout, d_status);
    else
      rc = launch_bwd_q<2>(blocks, 0, s, mp, gp, d_q, n, d_gout, d_status);
    if (rc == GSP_OK) {
      k_bwd_flush<<<dim3((lmax + 255) / 256, n_mats), 256, 0, s>>>(mp, gp, kBwdCopies);
      rc = cudaGetLastError() == cudaSuccess ? GSP_OK : GSP_ERR_CUDA;
    }
    prof_end(PROF_QUERY_BWD, s);
    GSP_TRY(rc);
  } else if (n > 0) {
    // VEC: 2 when it divides every rank (with at least four vectors per rank
    // row) and keeps the factor rows and gradients aligned, else 1; LANES x
    // VEC covers the largest rank.  (Runs of 4 ranks, or several queries per
    // warp, were slower at rank 64: 4.0 - 5.8 ms instead of 2.6 ms per 10^7
    // queries, the lane groups' shared-memory reductions to one column of
    // different rows falling on one bank.)
    int vec = 2;
    for (int i = 0; i < n_mats; ++i) {
      const gsp_material& m = h_mats[i];
      const gsp_material_grad& g = h_grads[i];
      auto aligned = [&](int v) {
        const uintptr_t mask = static_cast<uintptr_t>(4 * v - 1);
        return ((reinterpret_cast<uintptr_t>(m.fx) | reinterpret_cast<uintptr_t>(m.fy) |
                 reinterpret_cast<uintptr_t>(g.dfx) | reinterpret_cast<uintptr_t>(g.dfy)) & mask) == 0;
      };
      while (vec > 1 && (m.rank % vec != 0 || m.rank / vec < 4 || !aligned(vec))) vec >>= 1;
    }
    int rmax = 1;
    for (int i = 0; i < n_mats; ++i) rmax = rmax > h_mats[i].rank ? rmax : h_mats[i].rank;
    int lanes = 4;
    while (lanes * vec < rmax && lanes < 32) lanes *= 2;
    const int threads = kBwdThreads;
    const size_t dyn = gp.use_smem ? smem : 0;
    long long warps = (n + 31) / 32;  // one batch of 32 queries per warp and step
    long long blocks = (warps * 32 + threads - 1) / threads;
    // CTAs per SM: as many as the shared memory (tables + query-term slots) allows, up to 8
    const size_t slot_bytes = static_cast<size_t>(kBwdWarps) * 32 * 5 * sizeof(float4);
    long long per_sm = static_cast<long long>((228 * 1024) / (dyn + slot_bytes + 1024));
    if (per_sm > 8) per_sm = 8;
    if (per_sm < 1) per_sm = 1;
    long long cap = static_cast<long long>(sm_count()) * per_sm;
    if (blocks > cap) blocks = cap;
    prof_begin(PROF_QUERY_BWD, s);
    GSP_TRY(launch_bwd(lanes, vec, blocks, threads, dyn, s, mp, gp, d_q, n, d_gout, d_status));
    prof_end(PROF_QUERY_BWD, s);
    GSP_CHECK_LAUNCH();
  }
  for (int i = 0; i < n_mats; ++i) {
    int R = h_mats[i].rank;
    k_suffix<<<grid_for(R, 64), 64, 0, s>>>(gp.dps[i], h_grads[i].dfs, h_mats[i].bins, R);
    GSP_CHECK_LAUNCH();
    k_suffix<<<grid_for(R, 64), 64, 0, s>>>(gp.dpt[i], h_grads[i].dft, h_mats[i].bins, R);
    GSP_CHECK_LAUNCH();
  }
  return GSP_OK;
}

extern "C" int gsp_sample_ndf(const gsp_material* h_mats, int n_mats, const gsp_sample_query* d_q,
                              int64_t n, const float* d_u, float* d_out, uint32_t* d_status,
                              gsp_stream stream) {
  if (!h_mats || n_mats < 1 || n_mats > GSP_MAX_MATERIALS || n < 0) return GSP_ERR_INVALID_ARG;
  if (n > 0 && (!d_q || !d_u || !d_out || (reinterpret_cast<uintptr_t>(d_q) & 15) ||
                (reinterpret_cast<uintptr_t>(d_u) & 15) || (reinterpret_cast<uintptr_t>(d_out) & 15)))
    return GSP_ERR_INVALID_ARG;
  MatParams mp;
  mp.n = n_mats;
  int rmax = 1;
  for (int i = 0; i < n_mats; ++i) {
    const gsp_material& m = h_mats[i];
    if (!valid_material(m)) return GSP_ERR_INVALID_ARG;
    if (!is_pow2(m.bins) || m.bins < 2 || m.bins > 64 || m.rank > kSampleMaxRank)
      return GSP_ERR_UNSUPPORTED;
    mp.m[i] = m;
    rmax = rmax > m.rank ? rmax : m.rank;
  }
  if (n == 0) return GSP_OK;
  int lanes = 4;
  while (lanes * 2 < rmax) lanes *= 2;  // two rank slots per lane (rmax <= 64)
  bool pairs = true;  // every rank even and the fx, fy rows 8-byte aligned
  for (int i = 0; i < n_mats; ++i)
    pairs = pairs && h_mats[i].rank % 2 == 0 &&
            ((reinterpret_cast<uintptr_t>(h_mats[i].fx) | reinterpret_cast<uintptr_t>(h_mats[i].fy)) & 7) == 0;
  const int threads = 256;
  const long long per_cta = threads / 32 * (32 / lanes);
  long long blocks = (n + per_cta - 1) / per_cta;
  const long long cap = static_cast<long long>(sm_count()) * 8;
  if (blocks > cap) blocks = cap;
  cudaStream_t s = to_stream(stream);
  if (pairs) {
    switch (lanes) {
      case 4: k_sample_ndf<4, 2><<<blocks, threads, 0, s>>>(mp, d_q, n, d_u, d_out, d_status); break;
      case 8: k_sample_ndf<8, 2><<<blocks, threads, 0, s>>>(mp, d_q, n, d_u, d_out, d_status); break;
      case 16: k_sample_ndf<16, 2><<<blocks, threads, 0, s>>>(mp, d_q, n, d_u, d_out, d_status); break;
      default: k_sample_ndf<32, 2><<<blocks, threads, 0, s>>>(mp, d_q, n, d_u, d_out, d_status); break;
    }
  } else {
    switch (lanes) {
      case 4: k_sample_ndf<4, 1><<<blocks, threads, 0, s>>>(mp, d_q, n, d_u, d_out, d_status); break;
      case 8: k_sample_ndf<8, 1><<<blocks, threads, 0, s>>>(mp, d_q, n, d_u, d_out, d_status); break;
      case 16: k_sample_ndf<16, 1><<<blocks, threads, 0, s>>>(mp, d_q, n, d_u, d_out, d_status); break;
      default: k_sample_ndf<32, 1><<<blocks, threads, 0, s>>>(mp, d_q, n, d_u, d_out, d_status); break;
    }
  }
  GSP_CHECK_LAUNCH();
  return GSP_OK;
}

// ------------------------------------------------------- env queries --
// Sec. 5.4: the compact-eps support angle of the chosen SG lobe gives the
// side of a square angular range centred on the half vector's bin.
struct EnvParams {
  int bins[GSP_MAX_MATERIALS];
  int n_mats;
};

__global__ void k_env_queries(const EnvParams ep, const gsp_sg* __restrict__ sgs, int n_sgs,
                              const gsp_env_record* __restrict__ rec, long long n, float eps,
                              gsp_query* __restrict__ q) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const gsp_env_record r = rec[i];
  gsp_query d;
  d.x = r.x;
  d.y = r.y;
  d.level = r.level;
  d.material = r.material;
  const bool ok_idx = r.sg < static_cast<uint32_t>(n_sgs) && r.material < static_cast<uint32_t>(ep.n_mats);
  const gsp_sg g = sgs[ok_idx ? r.sg : 0];
  const float B = static_cast<float>(ep.bins[ok_idx ? r.material : 0]);
  const float hx = r.wo[0] + g.axis[0], hy = r.wo[1] + g.axis[1], hz = r.wo[2] + g.axis[2];
  const float hn = sqrtf(hx * hx + hy * hy + hz * hz);
  float theta;
  if (!(g.amplitude > eps)) {
    theta = 0.0f;  // the lobe never exceeds eps: a point query
  } else {
    const float c = (logf(eps) - logf(g.amplitude)) / g.sharpness + 1.0f;
    theta = c <= -1.0f ? 3.14159265358979f : acosf(fminf(c, 1.0f));
  }
  const float side = B * theta / 3.14159265358979f;
  const float sc = (hx / hn + 1.0f) * 0.5f * B, tc = (hy / hn + 1.0f) * 0.5f * B;
  d.s0 = sc - 0.5f * side;
  d.s1 = sc + 0.5f * side;
  d.t0 = tc - 0.5f * side;
  d.t1 = tc + 0.5f * side;
  if (!ok_idx || !(hn > 0.0f)) d.level = __int_as_float(0x7fc00000);
  q[i] = d;
}

extern "C" int gsp_env_queries(const gsp_material* h_mats, int n_mats, const gsp_sg* d_sgs,
                               int n_sgs, const gsp_env_record* d_rec, int64_t n, float eps,
                               gsp_query* d_q, gsp_stream stream) {
  if (!h_mats || n_mats < 1 || n_mats > GSP_MAX_MATERIALS || n < 0 || n_sgs < 1 || !(eps > 0.0f))
    return GSP_ERR_INVALID_ARG;
  if (n > 0 && (!d_sgs || !d_rec || !d_q)) return GSP_ERR_INVALID_ARG;
  EnvParams ep;
  ep.n_mats = n_mats;
  for (int i = 0; i < n_mats; ++i) {
    if (h_mats[i].bins < 1) return GSP_ERR_INVALID_ARG;
    ep.bins[i] = h_mats[i].bins;
  }
  if (n == 0) return GSP_OK;
  k_env_queries<<<grid_for(n, 256), 256, 0, to_stream(stream)>>>(ep, d_sgs, n_sgs, d_rec, n, eps, d_q);
  GSP_CHECK_LAUNCH();
  return GSP_OK;
}

// ------------------------------------------------ no-allocation backward --
// Fixed device scratch for gsp_range_query_backward_noalloc: the prefix-sum
// gradient tables of the adjoint, for callers that cannot allocate.  Every
// device that loads the library holds this array until the process exits.
namespace gsp {
namespace {
constexpr size_t kNoAllocFloats = GSP_BACKWARD_NOALLOC_MAX_BYTES / sizeof(float);
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocFloats];

// Device address of the array, looked up once per device with that device
// current (host code cannot use the symbol's host-side name as a pointer).
int noalloc_scratch(void** out) {
  static std::mutex mu;
  static void* addr[64] = {};
  int dev = 0;
  GSP_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return GSP_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    GSP_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    addr[dev] = p;
  }
  *out = addr[dev];
  return GSP_OK;
}
}  // namespace
}  // namespace gsp

extern "C" int gsp_range_query_backward_noalloc(const gsp_material* h_mats, int n_mats,
                                                const gsp_query* d_q, int64_t n,
                                                const float* d_gout,
                                                const gsp_material_grad* h_grads,
                                                uint32_t* d_status, gsp_stream stream) {
  if (!h_mats || !h_grads || n_mats < 1 || n_mats > GSP_MAX_MATERIALS || n < 0)
    return GSP_ERR_INVALID_ARG;
  // malformed materials are argument errors, whatever scratch they would need
  for (int i = 0; i < n_mats; ++i) {
    const gsp_material_grad& g = h_grads[i];
    if (!valid_material(h_mats[i]) || !g.dfx || !g.dfy || !g.dflw || !g.dfs || !g.dft)
      return GSP_ERR_INVALID_ARG;
  }
  const size_t need = gsp_backward_workspace_bytes(h_mats, n_mats);
  if (need == 0) return GSP_ERR_INVALID_ARG;
  if (need > GSP_BACKWARD_NOALLOC_MAX_BYTES) return GSP_ERR_WORKSPACE;
  void* scratch = nullptr;
  GSP_TRY(noalloc_scratch(&scratch));
  // the workspace version clears the part it uses on `stream` before its kernels
  return gsp_range_query_backward(h_mats, n_mats, d_q, n, d_gout, h_grads, scratch,
                                  GSP_BACKWARD_NOALLOC_MAX_BYTES, d_status, stream);
}

extern "C" int gsp_adam_step(float* d_param, const float* d_grad, float* d_m, float* d_v,
                             int64_t n, int step, float lr, float beta1, float beta2, float eps,
                             gsp_stream stream) {
  if (n < 0 || step < 1 || (n > 0 && (!d_param || !d_grad || !d_m || !d_v)))
    return GSP_ERR_INVALID_ARG;
  if (n == 0) return GSP_OK;
  float c1 = static_cast<float>(1.0 - pow(static_cast<double>(beta1), step));
  float c2 = static_cast<float>(1.0 - pow(static_cast<double>(beta2), step));
  prof_begin(PROF_ADAM, to_stream(stream));
  k_adam<<<grid_for(n, 256), 256, 0, to_stream(stream)>>>(d_param, d_grad, d_m, d_v, n, lr, beta1,
                                                          beta2, eps, c1, c2);
  prof_end(PROF_ADAM, to_stream(stream));
  GSP_CHECK_LAUNCH();
  return GSP_OK;
}
