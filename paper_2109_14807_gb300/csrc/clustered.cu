// Row f2: the clustered compression layout of Sec. 4.2 on the GPU.
//
// Every NDF image (footprint histogram, B x B bins) is split into t x t angular
// blocks (t = 16); the blocks of the footprints centred in the same 8 x 8-texel
// region and lying at the same block position form one group; a group stacks
// its non-blank blocks (level, then y, then x) into a t x t x M tensor D_j and
// is decomposed by its own CP-ALS (Eq. 3: weights C_r and three vectors per
// rank).  A range query (Eq. 5 with the 1D SATs of Sec. 4.4) is split at the
// block borders it crosses.
//
// Kernels:
//   k_block_flags   one warp per (footprint, block): is any count non-zero
//   k_group_count   members per group;  k_group_scan: offsets (one CTA)
//   k_group_fill    member list (packed level, y, x) and the z index map
//   k_cluster_als<R> one CTA per group, persistent over its sweeps: the three
//                   3-mode MTTKRPs from z-slices staged in shared memory (FP32
//                   products, compensated FP32 sums), the FP64 Gram / Cholesky
//                   / inverse / apply / normalisation of each mode, the fit,
//                   and the |delta fit| < tol stop of Sec. 4.2
//   k_cluster_tables 1D SATs of X and Y per group (FP64 sums split hi + lo) and
//                   Z rows with the weights folded in
//   k_cluster_query R lanes per query, the sub-range of every block the bin
//                   rectangle touches, area-weighted, blended across levels
#include "solve.cuh"

namespace gsp {
namespace {

constexpr int kBlk = 16;        // t
constexpr int kRegion = 8;      // region side in texels
constexpr int kCThreads = 256;  // per-group CTA (the Cholesky's 16 x 16 grid)
constexpr int kZChunk = 8;      // z-slices staged per step
constexpr double kRankCut = 1e-12;  // relative eigenvalue cutoff of the group Gram solves

struct CDims {
  int N, L, B, nb, nr, G;
};
CDims cdims(int N, int L, int B) {
  CDims d;
  d.N = N;
  d.L = L;
  d.B = B;
  d.nb = B / kBlk;
  d.nr = N / kRegion;
  d.G = d.nr * d.nr * d.nb * d.nb;
  return d;
}

__host__ __device__ inline int32_t pack_member(int l, int y, int x) { return (l << 20) | (y << 10) | x; }
__device__ inline int member_l(int32_t m) { return m >> 20; }
__device__ inline int member_y(int32_t m) { return (m >> 10) & 1023; }
__device__ inline int member_x(int32_t m) { return m & 1023; }

// offset of row s' of block (bs, bt) of footprint (l, y, x) in H [l][y][x][s][t]
__device__ inline size_t block_row(int l, int y, int x, int bs, int bt, int s, int N, int B) {
  return ((static_cast<size_t>(l) * N + y) * N + x) * static_cast<size_t>(B) * B +
         static_cast<size_t>(bs * kBlk + s) * B + bt * kBlk;
}

__global__ void k_block_flags(const int32_t* __restrict__ H, int N, int L, int B, int nb,
                              uint8_t* __restrict__ flags) {
  const long long w = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const long long total = static_cast<long long>(L) * N * N * nb * nb;
  if (w >= total) return;
  const int blk = static_cast<int>(w % (nb * nb));
  const long long f = w / (nb * nb);
  const int x = static_cast<int>(f % N), y = static_cast<int>((f / N) % N), l = static_cast<int>(f / (static_cast<long long>(N) * N));
  const int bs = blk / nb, bt = blk % nb;
  const int4* p = reinterpret_cast<const int4*>(H + block_row(l, y, x, bs, bt, lane >> 1, N, B) + (lane & 1) * 8);
  const int4 a = __ldg(p), b = __ldg(p + 1);
  const bool nz = (a.x | a.y | a.z | a.w | b.x | b.y | b.z | b.w) != 0;
  const bool any = __any_sync(0xffffffffu, nz);
  if (lane == 0) flags[w] = any ? 1 : 0;
}

// candidates of group j in z order: level, then y, then x of its region
template <typename F>
__device__ inline void for_candidates(int j, const CDims& d, F&& f) {
  const int bt = j % d.nb, bs = (j / d.nb) % d.nb;
  const int reg = j / (d.nb * d.nb);
  const int cx = reg % d.nr, cy = reg / d.nr;
  for (int l = 0; l < d.L; ++l)
    for (int yy = 0; yy < kRegion; ++yy)
      for (int xx = 0; xx < kRegion; ++xx) f(l, cy * kRegion + yy, cx * kRegion + xx, bs, bt);
}

__global__ void k_group_count(const uint8_t* __restrict__ flags, CDims d, int32_t* __restrict__ count) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= d.G) return;
  int c = 0;
  for_candidates(j, d, [&](int l, int y, int x, int bs, int bt) {
    c += flags[((static_cast<size_t>(l) * d.N + y) * d.N + x) * d.nb * d.nb + bs * d.nb + bt];
  });
  count[j] = c;
}

// offsets[j] = sum_{i < j} count[i], offsets[G] = total; stats[0] = total,
// stats[1] = max count.  One CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_group_scan(const int32_t* __restrict__ count, int G,
                                                     int32_t* __restrict__ offsets,
                                                     long long* __restrict__ stats) {
  __shared__ long long wsum[32];
  __shared__ int wmax[32];
  const int per = (G + blockDim.x - 1) / blockDim.x;
  const int i0 = threadIdx.x * per, i1 = min(G, i0 + per);
  long long s = 0;
  int mx = 0;
  for (int i = i0; i < i1; ++i) {
    s += count[i];
    mx = max(mx, count[i]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long incl = s;
  for (int o = 1; o < 32; o <<= 1) {
    const long long v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  int m = mx;
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 31) wsum[warp] = incl;
  if (lane == 0) wmax[warp] = m;
  __syncthreads();
  long long base = 0;
  for (int w = 0; w < warp; ++w) base += wsum[w];
  long long run = base + incl - s;
  for (int i = i0; i < i1; ++i) {
    offsets[i] = static_cast<int32_t>(run);
    run += count[i];
  }
  if (threadIdx.x == blockDim.x - 1) {
    offsets[G] = static_cast<int32_t>(base + incl);
    stats[0] = base + incl;
    int mm = 0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) mm = max(mm, wmax[w]);
    stats[1] = mm;
  }
}

__global__ void k_group_fill(const uint8_t* __restrict__ flags, CDims d,
                             const int32_t* __restrict__ offsets, int32_t* __restrict__ members,
                             int32_t* __restrict__ zmap) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= d.G) return;
  int z = 0;
  const int base = offsets[j];
  for_candidates(j, d, [&](int l, int y, int x, int bs, int bt) {
    const size_t f = ((static_cast<size_t>(l) * d.N + y) * d.N + x) * d.nb * d.nb + bs * d.nb + bt;
    if (flags[f]) {
      members[base + z] = pack_member(l, y, x);
      zmap[f] = z;
      ++z;
    }
  });
}

__device__ __forceinline__ void sum2(float& hi, float& lo, float x) {
  const float t = __fadd_rn(hi, x);
  const float bp = __fsub_rn(t, hi);
  lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(x, bp)));
  hi = t;
}

// hi + lo += a * b, compensated: the product's rounding error from an FMA and
// the sum's from TwoSum both go to lo (Ogita, Rump & Oishi 2005, "Accurate sum
// and dot product", Dot2).  Explicit _rn operations keep the compiler from
// fusing the product into the sum.
__device__ __forceinline__ void dot2(float& hi, float& lo, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float pe = fmaf(a, b, -p);
  const float t = __fadd_rn(hi, p);
  const float bp = __fsub_rn(t, hi);
  lo = __fadd_rn(lo, __fadd_rn(__fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(p, bp)), pe));
  hi = t;
}

// Shared-memory layout of k_cluster_als<R> for a group of at most Mmax members.
// The factors and the MTTKRP results are kept as FP32 pairs (hi, lo) whose sum
// carries about twice FP32 precision: a group whose tensor is exactly of low
// rank drives ALS into nearly singular Gram systems, where factors rounded to
// FP32 between updates would be amplified into garbage.
struct AlsSmem {
  size_t f_X, f_Xl, f_Y, f_Yl, f_MXh, f_MXl, f_MYh, f_MYl, f_Z, f_Zl, f_cl, f_D, i_mem, d_G, d_V,
      d_L, d_Zt, d_invd, d_lam, d_red, bytes;
};
__host__ __device__ inline AlsSmem als_smem(int R, int Mmax) {
  AlsSmem o;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = (off + bytes + 15) & ~static_cast<size_t>(15);
    return at;
  };
  const size_t f = sizeof(float), dd = sizeof(double);
  o.f_X = take(kBlk * R * f);
  o.f_Xl = take(kBlk * R * f);
  o.f_Y = take(kBlk * R * f);
  o.f_Yl = take(kBlk * R * f);
  o.f_MXh = take(kBlk * R * f);
  o.f_MXl = take(kBlk * R * f);
  o.f_MYh = take(kBlk * R * f);
  o.f_MYl = take(kBlk * R * f);
  o.f_Z = take(static_cast<size_t>(Mmax) * R * f);
  o.f_Zl = take(static_cast<size_t>(Mmax) * R * f);
  o.f_cl = take(static_cast<size_t>(Mmax) * f);
  o.f_D = take(kZChunk * kBlk * kBlk * f);
  o.i_mem = take(static_cast<size_t>(Mmax) * sizeof(int32_t));
  o.d_G = take(3 * R * R * dd);
  o.d_V = take(R * (R + 1) * dd);
  o.d_L = take(R * R * dd);
  o.d_Zt = take(R * R * dd);
  o.d_invd = take(R * dd);
  o.d_lam = take(R * dd);
  o.d_red = take(kCThreads * dd);
  o.bytes = off;
  return o;
}

// Fixed-order block sum of one double per thread.
__device__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int w = kCThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const double s = red[0];
  __syncthreads();
  return s;
}

// G = A^T A for A = Ah + Al [I][R], compensated FP32 dot products (Dot2, with
// the cross terms of the low parts), FP64 result.
template <int R>
__device__ void gram_rows(const float* Ah, const float* Al, int I, double* G) {
  for (int e = threadIdx.x; e < R * R; e += kCThreads) {
    const int a = e / R, b = e % R;
    float hi = 0.0f, lo = 0.0f;
    for (int i = 0; i < I; ++i) {
      const float xa = Ah[i * R + a], xb = Ah[i * R + b];
      dot2(hi, lo, xa, xb);
      lo = fmaf(xa, Al[i * R + b], fmaf(Al[i * R + a], xb, lo));
    }
    G[e] = static_cast<double>(hi) + static_cast<double>(lo);
  }
  __syncthreads();
}

// Stage z-slices [z0, z0 + n) of the group (block bs, bt) as floats (counts
// are exact in FP32).
__device__ void stage_slices(const int32_t* __restrict__ H, const int32_t* mem, int z0, int n, int bs,
                             int bt, int N, int B, float* D) {
  for (int i = threadIdx.x; i < n * kBlk * (kBlk / 4); i += kCThreads) {
    const int zz = i / (kBlk * 4), rem = i % (kBlk * 4);
    const int s = rem >> 2, q = rem & 3;
    const int32_t m = mem[z0 + zz];
    const int4 v = __ldg(reinterpret_cast<const int4*>(
                             H + block_row(member_l(m), member_y(m), member_x(m), bs, bt, s, N, B)) + q);
    float* o = D + zz * kBlk * kBlk + s * kBlk + q * 4;
    o[0] = static_cast<float>(v.x);
    o[1] = static_cast<float>(v.y);
    o[2] = static_cast<float>(v.z);
    o[3] = static_cast<float>(v.w);
  }
}

// The least-squares update of one mode: V = G1 .* G2 (FP64); Cholesky, or,
// when a pivot falls below kRankCut of the largest diagonal, the
// pseudo-inverse from a Jacobi eigendecomposition with cutoff kRankCut
// lambda_max (GSP_DEV_NUMERIC);
// W = V^-1 (V^+); A = M W in FP64 per row with M = Mh + Ml, stored as
// Ah + Al; column norms into lam; A /= lam; G_out = A^T A.  (Mh, Ml) and
// (Ah, Al) may alias (a row is read into registers before it is written).
template <int R>
__device__ void mode_update(const double* G1, const double* G2, const float* Mh, const float* Ml,
                            float* Ah, float* Al, int I, double* Gout, const AlsSmem& o, char* sm,
                            uint32_t* flags) {
  double* V = reinterpret_cast<double*>(sm + o.d_V);
  double* Lf = reinterpret_cast<double*>(sm + o.d_L);
  double* Zt = reinterpret_cast<double*>(sm + o.d_Zt);
  double* W = reinterpret_cast<double*>(sm + o.d_V);  // V is not read once L is extracted
  double* invd = reinterpret_cast<double*>(sm + o.d_invd);
  double* lam = reinterpret_cast<double*>(sm + o.d_lam);
  double* red = reinterpret_cast<double*>(sm + o.d_red);
  const int ld = R + 1;
  double mx = 0.0;
  for (int k = 0; k < R; ++k) mx = fmax(mx, fabs(G1[k * R + k] * G2[k * R + k]));
  for (int e = threadIdx.x; e < R * R; e += kCThreads) V[(e / R) * ld + e % R] = G1[e] * G2[e];
  __syncthreads();
  // numerical rank: the MTTKRPs and Grams carry about 1e-14 relative accuracy
  // (compensated FP32), so directions of V below kRankCut of its largest are
  // noise; a pivot under that goes to the pseudo-inverse, which drops them
  const bool ok = cholesky_inplace(V, R, ld, kRankCut * mx, invd);
  __syncthreads();
  if (ok) {
    for (int e = threadIdx.x; e < R * R; e += kCThreads) {
      const int i = e / R, k = e % R;
      Lf[e] = k <= i ? V[i * ld + k] : 0.0;
    }
    __syncthreads();
    if (threadIdx.x < R) {  // column c of L^-1 by forward substitution
      const int c = threadIdx.x;
      for (int k = 0; k < R; ++k) {
        double zk = 0.0;
        if (k == c) {
          zk = invd[c];
        } else if (k > c) {
          double acc = 0.0;
          for (int j2 = c; j2 < k; ++j2) acc += Lf[k * R + j2] * Zt[c * R + j2];
          zk = -acc * invd[k];
        }
        Zt[c * R + k] = zk;
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < R * R; e += kCThreads) {
      const int a = e / R, b = e % R;
      double acc = 0.0;
      for (int k = a > b ? a : b; k < R; ++k) acc += Zt[a * R + k] * Zt[b * R + k];
      W[e] = acc;
    }
  } else {
    if (threadIdx.x == 0 && flags) atomicOr(flags, GSP_DEV_NUMERIC);
    for (int e = threadIdx.x; e < R * R; e += kCThreads) V[e] = G1[e] * G2[e];  // ld = R
    __syncthreads();
    jacobi_eigen(V, Lf, R);
    // the eigenvalues leave V before W (which shares V's storage) is written
    for (int k = threadIdx.x; k < R; k += kCThreads) invd[k] = V[k * R + k];
    __syncthreads();
    double lmax = 0.0;
    for (int k = 0; k < R; ++k) lmax = fmax(lmax, fabs(invd[k]));
    const double cut = kRankCut * lmax;
    for (int e = threadIdx.x; e < R * R; e += kCThreads) {
      const int a = e / R, b = e % R;
      double acc = 0.0;
      for (int k = 0; k < R; ++k) {
        const double l = invd[k];
        if (l > cut) acc += Lf[a * R + k] * Lf[b * R + k] / l;
      }
      W[e] = acc;
    }
  }
  __syncthreads();
  // A = M W in FP64 per row (M = Mh + Ml), stored as hi + lo
  for (int i = threadIdx.x; i < I; i += kCThreads) {
    double m[R];
#pragma unroll
    for (int k = 0; k < R; ++k)
      m[k] = static_cast<double>(Mh[i * R + k]) + (Ml ? static_cast<double>(Ml[i * R + k]) : 0.0);
    for (int c = 0; c < R; ++c) {
      double acc = 0.0;
#pragma unroll
      for (int k = 0; k < R; ++k) acc += m[k] * W[k * R + c];
      const float h = static_cast<float>(acc);
      Ah[i * R + c] = h;
      Al[i * R + c] = static_cast<float>(acc - static_cast<double>(h));
    }
  }
  __syncthreads();
  for (int c = 0; c < R; ++c) {
    double part = 0.0;
    for (int i = threadIdx.x; i < I; i += kCThreads) {
      const double v = static_cast<double>(Ah[i * R + c]) + static_cast<double>(Al[i * R + c]);
      part += v * v;
    }
    const double sum = block_sum(part, red);
    if (threadIdx.x == 0) lam[c] = sqrt(sum);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < I * R; e += kCThreads) {
    const double l = lam[e % R];
    if (l > 0.0) {
      const double v = (static_cast<double>(Ah[e]) + static_cast<double>(Al[e])) / l;
      const float h = static_cast<float>(v);
      Ah[e] = h;
      Al[e] = static_cast<float>(v - static_cast<double>(h));
    }
  }
  __syncthreads();
  gram_rows<R>(Ah, Al, I, Gout);
}

template <int R>
__global__ void __launch_bounds__(kCThreads) k_cluster_als(
    const int32_t* __restrict__ H, CDims d, const int32_t* __restrict__ offsets,
    const int32_t* __restrict__ members, const double* __restrict__ lscale, int Mmax,
    float* __restrict__ Xg, float* __restrict__ Yg, float* __restrict__ Zg, float* __restrict__ lamg,
    int max_sweeps, double tol, int32_t* __restrict__ sweeps_out, double* __restrict__ fit_out,
    uint32_t* flags) {
  extern __shared__ __align__(16) char sm[];
  const int j = blockIdx.x;
  const int off = offsets[j], M = offsets[j + 1] - off;
  if (M == 0) {
    if (threadIdx.x == 0) {
      sweeps_out[j] = 0;
      fit_out[j] = 0.0;
    }
    return;
  }
  const AlsSmem o = als_smem(R, Mmax);
  float* Xs = reinterpret_cast<float*>(sm + o.f_X);
  float* Xl = reinterpret_cast<float*>(sm + o.f_Xl);
  float* Ys = reinterpret_cast<float*>(sm + o.f_Y);
  float* Yl = reinterpret_cast<float*>(sm + o.f_Yl);
  float* Zs = reinterpret_cast<float*>(sm + o.f_Z);
  float* Zl = reinterpret_cast<float*>(sm + o.f_Zl);
  float* cl = reinterpret_cast<float*>(sm + o.f_cl);
  float* Ds = reinterpret_cast<float*>(sm + o.f_D);
  int32_t* mem = reinterpret_cast<int32_t*>(sm + o.i_mem);
  double* GX = reinterpret_cast<double*>(sm + o.d_G);
  double* GY = GX + R * R;
  double* GZ = GY + R * R;
  double* lam = reinterpret_cast<double*>(sm + o.d_lam);
  double* dred = reinterpret_cast<double*>(sm + o.d_red);
  const int bt = j % d.nb, bs = (j / d.nb) % d.nb;

  for (int e = threadIdx.x; e < kBlk * R; e += kCThreads) {
    Xs[e] = Xg[static_cast<size_t>(j) * kBlk * R + e];
    Ys[e] = Yg[static_cast<size_t>(j) * kBlk * R + e];
    Xl[e] = Yl[e] = 0.0f;
  }
  for (int e = threadIdx.x; e < M * R; e += kCThreads) {
    Zs[e] = Zg[static_cast<size_t>(off) * R + e];
    Zl[e] = 0.0f;
  }
  for (int z = threadIdx.x; z < M; z += kCThreads) {
    mem[z] = members[off + z];
    cl[z] = static_cast<float>(lscale[member_l(mem[z])]);  // a power of two: exact
  }
  __syncthreads();
  // ||D||^2: counts squared (exact in FP64) times c_l^2
  double nd = 0.0;
  for (int z0 = 0; z0 < M; z0 += kZChunk) {
    const int n = min(kZChunk, M - z0);
    stage_slices(H, mem, z0, n, bs, bt, d.N, d.B, Ds);
    __syncthreads();
    for (int i = threadIdx.x; i < n * kBlk * kBlk; i += kCThreads) {
      const double v = Ds[i];
      const double c = cl[z0 + i / (kBlk * kBlk)];
      nd += c * c * v * v;
    }
    __syncthreads();
  }
  const double normD2 = block_sum(nd, dred);
  gram_rows<R>(Xs, Xl, kBlk, GX);
  gram_rows<R>(Ys, Yl, kBlk, GY);
  gram_rows<R>(Zs, Zl, M, GZ);

  constexpr int kPairs = (kBlk * R + kCThreads - 1) / kCThreads;
  double prev = 0.0, fit = 0.0;
  int done = 0;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    // modes X and Y: M[a][r] = sum_z c_z Z[z][r] sum_b D_z(a, b) F[b][r] with
    // D_z(a, b) = D_z[a][b], F = Y (mode X) or D_z[b][a], F = X (mode Y)
    for (int mode = 0; mode < 2; ++mode) {
      const float* F = mode == 0 ? Ys : Xs;
      const float* Fl = mode == 0 ? Yl : Xl;
      float* Mh = reinterpret_cast<float*>(sm + (mode == 0 ? o.f_MXh : o.f_MYh));
      float* Ml = reinterpret_cast<float*>(sm + (mode == 0 ? o.f_MXl : o.f_MYl));
      float ah[kPairs], al[kPairs];
#pragma unroll
      for (int q = 0; q < kPairs; ++q) ah[q] = al[q] = 0.0f;
      for (int z0 = 0; z0 < M; z0 += kZChunk) {
        const int n = min(kZChunk, M - z0);
        stage_slices(H, mem, z0, n, bs, bt, d.N, d.B, Ds);
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kPairs; ++q) {
          const int p = threadIdx.x + q * kCThreads;
          if (p < kBlk * R) {
            const int a = p / R, r = p % R;
            for (int zz = 0; zz < n; ++zz) {
              const float* Dz = Ds + zz * kBlk * kBlk;
              float vh = 0.0f, vl = 0.0f;
#pragma unroll
              for (int b = 0; b < kBlk; ++b) {
                const float dv = mode == 0 ? Dz[a * kBlk + b] : Dz[b * kBlk + a];
                dot2(vh, vl, dv, F[b * R + r]);
                vl = fmaf(dv, Fl[b * R + r], vl);
              }
              const float c = cl[z0 + zz];  // a power of two: exact products
              const float czh = c * Zs[(z0 + zz) * R + r], czl = c * Zl[(z0 + zz) * R + r];
              dot2(ah[q], al[q], czh, vh);
              al[q] = fmaf(czh, vl, fmaf(czl, vh, al[q]));
            }
          }
        }
        __syncthreads();
      }
#pragma unroll
      for (int q = 0; q < kPairs; ++q) {
        const int p = threadIdx.x + q * kCThreads;
        if (p < kBlk * R) {
          Mh[p] = ah[q];
          Ml[p] = al[q];
        }
      }
      __syncthreads();
      if (mode == 0)
        mode_update<R>(GY, GZ, Mh, Ml, Xs, Xl, kBlk, GX, o, sm, flags);
      else
        mode_update<R>(GX, GZ, Mh, Ml, Ys, Yl, kBlk, GY, o, sm, flags);
    }
    // mode Z: M[z][r] = c_z sum_s X[s][r] sum_t D_z[s][t] Y[t][r], as (Zs, Zl);
    // one thread per (slice, rank) pair, the whole 16 x 16 contraction
    for (int z0 = 0; z0 < M; z0 += kZChunk) {
      const int n = min(kZChunk, M - z0);
      stage_slices(H, mem, z0, n, bs, bt, d.N, d.B, Ds);
      __syncthreads();
      for (int p = threadIdx.x; p < n * R; p += kCThreads) {
        const int zz = p / R, r = p % R;
        const float* Dz = Ds + zz * kBlk * kBlk;
        float hi = 0.0f, lo = 0.0f;
        for (int s2 = 0; s2 < kBlk; ++s2) {
          float vh = 0.0f, vl = 0.0f;
#pragma unroll
          for (int b = 0; b < kBlk; ++b) {
            dot2(vh, vl, Dz[s2 * kBlk + b], Ys[b * R + r]);
            vl = fmaf(Dz[s2 * kBlk + b], Yl[b * R + r], vl);
          }
          const float xh = Xs[s2 * R + r], xl = Xl[s2 * R + r];
          dot2(hi, lo, xh, vh);
          lo = fmaf(xh, vl, fmaf(xl, vh, lo));
        }
        const float c = cl[z0 + zz];  // a power of two: exact
        Zs[(z0 + zz) * R + r] = c * hi;
        Zl[(z0 + zz) * R + r] = c * lo;
      }
      __syncthreads();
    }
    mode_update<R>(GX, GY, Zs, Zl, Zs, Zl, M, GZ, o, sm, flags);
    // fit = 1 - ||D - D_hat|| / ||D|| from the explicit residual (the Gram
    // form is a difference of nearly equal terms near fit = 1).  Thread e owns
    // element (s, t) = (e / 16, e % 16) of every slice.
    float w[R], wl[R];
    {
      const int s = threadIdx.x / kBlk, t = threadIdx.x % kBlk;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const double v = lam[r] * (static_cast<double>(Xs[s * R + r]) + Xl[s * R + r]) *
                         (static_cast<double>(Ys[t * R + r]) + Yl[t * R + r]);
        w[r] = static_cast<float>(v);
        wl[r] = static_cast<float>(v - static_cast<double>(w[r]));
      }
    }
    float eh = 0.0f, el = 0.0f;
    for (int z0 = 0; z0 < M; z0 += kZChunk) {
      const int n = min(kZChunk, M - z0);
      stage_slices(H, mem, z0, n, bs, bt, d.N, d.B, Ds);
      __syncthreads();
      for (int zz = 0; zz < n; ++zz) {
        const float* zr = Zs + (z0 + zz) * R;
        const float* zrl = Zl + (z0 + zz) * R;
        float dh = 0.0f, dl = 0.0f;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          dot2(dh, dl, w[r], zr[r]);
          dl = fmaf(w[r], zrl[r], fmaf(wl[r], zr[r], dl));
        }
        // residual e = c D - (dh + dl), then e^2 added compensated
        const float x = cl[z0 + zz] * Ds[zz * kBlk * kBlk + threadIdx.x];
        const float e = __fadd_rn(__fsub_rn(x, dh), -dl);
        dot2(eh, el, e, e);
      }
      __syncthreads();
    }
    const double res = block_sum(static_cast<double>(eh) + static_cast<double>(el), dred);
    fit = normD2 > 0.0 ? 1.0 - sqrt(res) / sqrt(normD2) : 0.0;
    done = sweep + 1;
    if (tol > 0.0 && sweep > 0 && fabs(fit - prev) < tol) break;
    prev = fit;
  }
  for (int e = threadIdx.x; e < kBlk * R; e += kCThreads) {
    Xg[static_cast<size_t>(j) * kBlk * R + e] = Xs[e];
    Yg[static_cast<size_t>(j) * kBlk * R + e] = Ys[e];
  }
  for (int e = threadIdx.x; e < M * R; e += kCThreads) Zg[static_cast<size_t>(off) * R + e] = Zs[e];
  for (int r = threadIdx.x; r < R; r += kCThreads) lamg[static_cast<size_t>(j) * R + r] = static_cast<float>(lam[r]);
  if (threadIdx.x == 0) {
    sweeps_out[j] = done;
    fit_out[j] = fit;
  }
}

// SAT of one in-block factor: sat[i][r] = {hi, lo, f[i][r], 0} with hi + lo =
// sum_{k < i} f[k][r] (FP64 sum split into two FP32), i = 0 .. t.
__global__ void k_cluster_tables(const float* __restrict__ Xg, const float* __restrict__ Yg,
                                 const float* __restrict__ Zg, const float* __restrict__ lamg,
                                 const int32_t* __restrict__ offsets, int G, int R,
                                 float4* __restrict__ xsat, float4* __restrict__ ysat,
                                 float* __restrict__ zw) {
  const long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (e >= static_cast<long long>(G) * R) return;
  const int j = static_cast<int>(e / R), r = static_cast<int>(e % R);
  for (int which = 0; which < 2; ++which) {
    const float* F = (which ? Yg : Xg) + static_cast<size_t>(j) * kBlk * R;
    float4* S = (which ? ysat : xsat) + static_cast<size_t>(j) * (kBlk + 1) * R;
    double acc = 0.0;
    for (int i = 0; i <= kBlk; ++i) {
      const float hi = static_cast<float>(acc);
      const float lo = static_cast<float>(acc - static_cast<double>(hi));
      S[static_cast<size_t>(i) * R + r] =
          make_float4(hi, lo, i < kBlk ? F[i * R + r] : 0.0f, i > 0 ? F[(i - 1) * R + r] : 0.0f);
      if (i < kBlk) acc += static_cast<double>(F[i * R + r]);
    }
  }
  const float l = lamg[static_cast<size_t>(j) * R + r];
  for (int z = offsets[j]; z < offsets[j + 1]; ++z)
    zw[static_cast<size_t>(z) * R + r] = l * Zg[static_cast<size_t>(z) * R + r];
}

// One axis of a range against the blocks: ends clamped to [0, B] and ordered;
// for block k the local sub-range [a0, a1] of [0, t], its weight (length
// fraction; 1 for a zero-width range on its block) and whether it is touched.
struct Axis {
  float a, b, inv_w;
  int kz;  // the block of a zero-width range
};
__device__ inline Axis make_axis(float a, float b, int B) {
  a = fminf(fmaxf(a, 0.0f), static_cast<float>(B));
  b = fminf(fmaxf(b, 0.0f), static_cast<float>(B));
  if (b < a) {
    const float t = a;
    a = b;
    b = t;
  }
  Axis x;
  x.a = a;
  x.b = b;
  x.inv_w = b > a ? 1.0f / (b - a) : 0.0f;
  x.kz = min(static_cast<int>(floorf(a)), B - 1) / kBlk;
  return x;
}

// Range mean of one rank inside block k over [lo, hi] (global bin units, a
// zero-width range reads the value of its bin).  Sat rows are {hi, lo, f[i],
// f[i-1]} with hi + lo = sum_{k < i} f[k].  The two partial end bins are
// weighted directly and only the whole bins between them come from the SAT
// difference, so every part is rounded relative to its own size: a range that
// starts just before the end of a large bin followed by zeros keeps its small
// integral instead of cancelling two O(1) prefix values.
__device__ inline float block_mean(const float4* __restrict__ sat, int R, int r, float lo, float hi,
                                   int k) {
  const float base = static_cast<float>(k * kBlk);
  if (hi > lo) {
    const float u0 = lo - base, u1 = hi - base;
    const float f0 = floorf(u0), f1 = floorf(u1);
    const int i0 = static_cast<int>(f0), i1 = static_cast<int>(f1);
    if (i0 == i1) return __ldg(reinterpret_cast<const float*>(sat + static_cast<size_t>(i0) * R + r) + 2);
    const float4 a = __ldg(sat + static_cast<size_t>(i0 + 1) * R + r);  // prefix(i0 + 1), f[i0]
    const float4 b = __ldg(sat + static_cast<size_t>(i1) * R + r);      // prefix(i1), f[i1]
    const float mid = (b.x - a.x) + (b.y - a.y);
    const float head = ((f0 + 1.0f) - u0) * a.w;
    const float tail = (u1 - f1) * b.z;
    return ((head + mid) + tail) / (hi - lo);
  }
  const int i = min(static_cast<int>(floorf(lo - base)), kBlk - 1);
  return __ldg(reinterpret_cast<const float*>(sat + static_cast<size_t>(i) * R + r) + 2);
}

// out[q] for queries gsp_query (material ignored): R lanes per query.
template <int R>
__global__ void k_cluster_query(const gsp_query* __restrict__ qs, long long n, CDims d,
                                const int32_t* __restrict__ offsets, const int32_t* __restrict__ zmap,
                                const float4* __restrict__ xsat, const float4* __restrict__ ysat,
                                const float* __restrict__ zw, float* __restrict__ out,
                                uint32_t* status) {
  constexpr int QPW = 32 / R;
  const int lane = threadIdx.x & 31;
  const int r = lane % R;
  const long long qi = ((blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) >> 5) * QPW + lane / R;
  // every lane stays to the rank-sum shuffle: out-of-range and malformed
  // queries only skip the gathers
  const bool in = qi < n;
  gsp_query q{};
  if (in) q = qs[qi];
  const bool ok = in && isfinite(q.level) && isfinite(q.s0) && isfinite(q.s1) && isfinite(q.t0) &&
                  isfinite(q.t1);
  if (!ok) {
    q.level = q.s0 = q.s1 = q.t0 = q.t1 = 0.0f;
    q.x = q.y = 0;
  }
  const int x = q.x & (d.N - 1), y = q.y & (d.N - 1);
  const float lev = fminf(fmaxf(q.level, 0.0f), static_cast<float>(d.L - 1));
  const int l0 = static_cast<int>(floorf(lev));
  const float fr = lev - floorf(lev);
  const int l1 = min(l0 + 1, d.L - 1);
  const Axis as = make_axis(q.s0, q.s1, d.B), at = make_axis(q.t0, q.t1, d.B);
  const int bs0 = as.inv_w > 0.0f ? min(static_cast<int>(as.a) / kBlk, d.nb - 1) : as.kz;
  const int bs1 = as.inv_w > 0.0f ? min(static_cast<int>(ceilf(as.b)) - 1, d.B - 1) / kBlk : as.kz;
  const int bt0 = at.inv_w > 0.0f ? min(static_cast<int>(at.a) / kBlk, d.nb - 1) : at.kz;
  const int bt1 = at.inv_w > 0.0f ? min(static_cast<int>(ceilf(at.b)) - 1, d.B - 1) / kBlk : at.kz;
  const int reg = (y / kRegion) * d.nr + x / kRegion;
  float acc = 0.0f;
  for (int li = 0; li < 2 && ok; ++li) {
    const int l = li ? l1 : l0;
    const float wl = li ? fr : 1.0f - fr;
    if (wl == 0.0f) continue;
    const size_t fb = ((static_cast<size_t>(l) * d.N + y) * d.N + x) * d.nb * d.nb;
    for (int bs = bs0; bs <= bs1; ++bs) {
      const float slo = fmaxf(as.a, static_cast<float>(bs * kBlk)), shi = fminf(as.b, static_cast<float>((bs + 1) * kBlk));
      if (as.inv_w > 0.0f && !(shi > slo)) continue;
      const float ws = as.inv_w > 0.0f ? (shi - slo) * as.inv_w : 1.0f;
      for (int bt = bt0; bt <= bt1; ++bt) {
        const float tlo = fmaxf(at.a, static_cast<float>(bt * kBlk)), thi = fminf(at.b, static_cast<float>((bt + 1) * kBlk));
        if (at.inv_w > 0.0f && !(thi > tlo)) continue;
        const int z = __ldg(zmap + fb + bs * d.nb + bt);
        if (z < 0) continue;
        const float wt = at.inv_w > 0.0f ? (thi - tlo) * at.inv_w : 1.0f;
        const int j = (reg * d.nb + bs) * d.nb + bt;
        const float mx = block_mean(xsat + static_cast<size_t>(j) * (kBlk + 1) * R, R, r,
                                    as.inv_w > 0.0f ? slo : as.a, as.inv_w > 0.0f ? shi : as.a, bs);
        const float my = block_mean(ysat + static_cast<size_t>(j) * (kBlk + 1) * R, R, r,
                                    at.inv_w > 0.0f ? tlo : at.a, at.inv_w > 0.0f ? thi : at.a, bt);
        const float zv = __ldg(zw + (static_cast<size_t>(offsets[j]) + z) * R + r);
        acc = fmaf(wl * ws * wt, mx * my * zv, acc);
      }
    }
  }
#pragma unroll
  for (int o2 = R / 2; o2 > 0; o2 >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o2);
  if (in && r == 0) {
    out[qi] = ok ? acc : __int_as_float(0x7fc00000);
    if (!ok) set_status(status, GSP_DEV_BAD_QUERY);
  }
}

// lscale[l] = B^2 / (4 * 4^l) (counts -> density), or 1 with raw counts
__global__ void k_cluster_scales(int L, int B, int raw, double* __restrict__ lscale) {
  const int l = threadIdx.x;
  if (l < L) lscale[l] = raw ? 1.0 : static_cast<double>(B) * B / (4.0 * ldexp(1.0, 2 * l));
}

bool cluster_valid(int N, int L, int B, int R) {
  return valid_map(N, L, B) && N >= kRegion && B >= kBlk && (R == 8 || R == 16 || R == 32);
}

}  // namespace
}  // namespace gsp

using namespace gsp;

extern "C" size_t gsp_cluster_layout_bytes(int N, int levels, int bins) {
  if (!valid_map(N, levels, bins) || N < kRegion || bins < kBlk) return 0;
  const CDims d = cdims(N, levels, bins);
  const size_t blocks = static_cast<size_t>(levels) * N * N * d.nb * d.nb;
  return align_up(blocks, 256) + align_up(static_cast<size_t>(d.G) * sizeof(int32_t), 256) +
         align_up(2 * sizeof(long long), 256);
}

extern "C" int gsp_cluster_groups(int N, int levels, int bins) {
  if (!valid_map(N, levels, bins) || N < kRegion || bins < kBlk) return 0;
  return cdims(N, levels, bins).G;
}

extern "C" int gsp_cluster_layout(const int32_t* d_hist, int N, int levels, int bins,
                                  int32_t* d_offsets, int32_t* d_members, int32_t* d_zmap,
                                  int64_t* h_stats, void* d_ws, size_t ws_bytes, gsp_stream stream) {
  if (!d_hist || !d_offsets || !d_members || !d_zmap || !h_stats) return GSP_ERR_INVALID_ARG;
  if (!valid_map(N, levels, bins) || N < kRegion || bins < kBlk) return GSP_ERR_INVALID_ARG;
  if (!d_ws || ws_bytes < gsp_cluster_layout_bytes(N, levels, bins)) return GSP_ERR_WORKSPACE;
  const CDims d = cdims(N, levels, bins);
  cudaStream_t s = to_stream(stream);
  const size_t blocks = static_cast<size_t>(levels) * N * N * d.nb * d.nb;
  uint8_t* flags = static_cast<uint8_t*>(d_ws);
  int32_t* count = reinterpret_cast<int32_t*>(static_cast<char*>(d_ws) + align_up(blocks, 256));
  long long* stats = reinterpret_cast<long long*>(reinterpret_cast<char*>(count) +
                                                  align_up(static_cast<size_t>(d.G) * sizeof(int32_t), 256));
  k_block_flags<<<grid_for(static_cast<long long>(blocks) * 32, 256), 256, 0, s>>>(d_hist, N, levels, bins,
                                                                                  d.nb, flags);
  GSP_CHECK_LAUNCH();
  k_group_count<<<grid_for(d.G, 128), 128, 0, s>>>(flags, d, count);
  GSP_CHECK_LAUNCH();
  k_group_scan<<<1, 1024, 0, s>>>(count, d.G, d_offsets, stats);
  GSP_CHECK_LAUNCH();
  GSP_CUDA(cudaMemsetAsync(d_zmap, 0xff, blocks * sizeof(int32_t), s));
  k_group_fill<<<grid_for(d.G, 128), 128, 0, s>>>(flags, d, d_offsets, d_members, d_zmap);
  GSP_CHECK_LAUNCH();
  long long hs[2];
  GSP_CUDA(cudaMemcpyAsync(hs, stats, sizeof(hs), cudaMemcpyDeviceToHost, s));
  GSP_CUDA(cudaStreamSynchronize(s));
  h_stats[0] = hs[0];
  h_stats[1] = hs[1];
  return GSP_OK;
}

extern "C" size_t gsp_cluster_als_smem(int rank, int max_members) {
  if (!(rank == 8 || rank == 16 || rank == 32) || max_members < 0) return 0;
  return als_smem(rank, max_members).bytes;
}

extern "C" int gsp_cluster_als(const int32_t* d_hist, int N, int levels, int bins, int rank,
                               const int32_t* d_offsets, const int32_t* d_members, int max_members,
                               float* d_X, float* d_Y, float* d_Z, float* d_lambda, int max_sweeps,
                               double tol, int raw_counts, int32_t* d_sweeps, double* d_fit,
                               uint32_t* d_status, void* d_ws, size_t ws_bytes, gsp_stream stream) {
  if (!cluster_valid(N, levels, bins, rank) || !d_hist || !d_offsets || !d_members || !d_X || !d_Y ||
      !d_Z || !d_lambda || !d_sweeps || !d_fit || max_sweeps < 1 || max_sweeps > GSP_MAX_SWEEPS ||
      !(tol >= 0.0) || max_members < 0 || max_members > 64 * levels)
    return GSP_ERR_INVALID_ARG;
  if (!d_ws || ws_bytes < static_cast<size_t>(levels) * sizeof(double)) return GSP_ERR_WORKSPACE;
  const CDims d = cdims(N, levels, bins);
  const AlsSmem o = als_smem(rank, max_members);
  if (o.bytes > 227 * 1024) return GSP_ERR_UNSUPPORTED;
  cudaStream_t s = to_stream(stream);
  double* lscale = static_cast<double*>(d_ws);
  k_cluster_scales<<<1, 32, 0, s>>>(levels, bins, raw_counts, lscale);
  GSP_CHECK_LAUNCH();
  switch (rank) {
#define GSP_CALS(RR)                                                                               \
  case RR:                                                                                         \
    GSP_CUDA(cudaFuncSetAttribute(k_cluster_als<RR>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                  static_cast<int>(o.bytes)));                                     \
    k_cluster_als<RR><<<d.G, kCThreads, o.bytes, s>>>(d_hist, d, d_offsets, d_members, lscale,      \
                                                     max_members, d_X, d_Y, d_Z, d_lambda,         \
                                                     max_sweeps, tol, d_sweeps, d_fit, d_status);   \
    break;
    GSP_CALS(8)
    GSP_CALS(16)
    GSP_CALS(32)
#undef GSP_CALS
    default:
      return GSP_ERR_INVALID_ARG;
  }
  GSP_CHECK_LAUNCH();
  return GSP_OK;
}

extern "C" int gsp_cluster_tables(int N, int levels, int bins, int rank, const int32_t* d_offsets,
                                  const float* d_X, const float* d_Y, const float* d_Z,
                                  const float* d_lambda, float* d_xsat, float* d_ysat, float* d_zw,
                                  gsp_stream stream) {
  if (!cluster_valid(N, levels, bins, rank) || !d_offsets || !d_X || !d_Y || !d_Z || !d_lambda ||
      !d_xsat || !d_ysat || !d_zw)
    return GSP_ERR_INVALID_ARG;
  const CDims d = cdims(N, levels, bins);
  k_cluster_tables<<<grid_for(static_cast<long long>(d.G) * rank, 128), 128, 0, to_stream(stream)>>>(
      d_X, d_Y, d_Z, d_lambda, d_offsets, d.G, rank, reinterpret_cast<float4*>(d_xsat),
      reinterpret_cast<float4*>(d_ysat), d_zw);
  GSP_CHECK_LAUNCH();
  return GSP_OK;
}

extern "C" int gsp_cluster_range_query(int N, int levels, int bins, int rank,
                                       const int32_t* d_offsets, const int32_t* d_zmap,
                                       const float* d_xsat, const float* d_ysat, const float* d_zw,
                                       const gsp_query* d_q, int64_t n, float* d_out,
                                       uint32_t* d_status, gsp_stream stream) {
  if (!cluster_valid(N, levels, bins, rank) || n < 0 || (n > 0 && (!d_q || !d_out)) || !d_offsets ||
      !d_zmap || !d_xsat || !d_ysat || !d_zw)
    return GSP_ERR_INVALID_ARG;
  if (n == 0) return GSP_OK;
  const CDims d = cdims(N, levels, bins);
  const long long warps = (n * rank + 31) / 32;
  cudaStream_t s = to_stream(stream);
  switch (rank) {
#define GSP_CQ(RR)                                                                                 \
  case RR:                                                                                         \
    k_cluster_query<RR><<<grid_for(warps * 32, 256), 256, 0, s>>>(                                 \
        d_q, n, d, d_offsets, d_zmap, reinterpret_cast<const float4*>(d_xsat),                     \
        reinterpret_cast<const float4*>(d_ysat), d_zw, d_out, d_status);                           \
    break;
    GSP_CQ(8)
    GSP_CQ(16)
    GSP_CQ(32)
#undef GSP_CQ
    default:
      return GSP_ERR_INVALID_ARG;
  }
  GSP_CHECK_LAUNCH();
  return GSP_OK;
}
