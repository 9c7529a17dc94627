// FP64 building blocks of the small Gram solves (CP-ALS of the global tensor
// and the per-group CP-ALS of the clustered layout).  Device code only.
#pragma once

#include "common.cuh"

namespace gsp {

constexpr int kMaxSolveRank = 64;

// 1/d for d > 0 by the Newton-Raphson iteration x <- x + x (1 - d x), whose
// relative error squares every step: from the FP32 reciprocal (error below
// 2^-23) two steps reach FP64 precision.  Four dependent FMAs instead of a full
// FP64 division on the Cholesky's sequential pivot chain.  Outside the FP32
// range of d it falls back to the division.
__device__ __forceinline__ double recip_newton(double d) {
  if (!(d > 1e-30 && d < 1e30)) return 1.0 / d;
  double x = static_cast<double>(__frcp_rn(static_cast<float>(d)));
  double e = fma(-d, x, 1.0);
  x = fma(x, e, x);
  e = fma(-d, x, 1.0);
  return fma(x, e, x);
}

__device__ inline bool cholesky_inplace(double* V, int R, int ld, double thresh, double* invd) {
  // Right-looking, columns left unscaled until the end: step j subtracts
  // A_ij A_kj / A_jj from the trailing lower triangle, which only reads column
  // j and the pivot, so one barrier per column suffices; L_ij = A_ij / sqrt(A_jj)
  // is formed for all columns at the end.  Thread 0 owns element (j+1, j+1)
  // of step j's update, so it forms the next pivot's reciprocal right after
  // updating it, before the barrier (double-buffered: step j reads slot j & 1
  // while thread 0 fills slot (j + 1) & 1).  The reciprocal square roots of
  // the pivots are taken at the end, in parallel.
  __shared__ double piv_inv[2];
  __shared__ double piv[kMaxSolveRank];
  const int ti = threadIdx.x >> 4, tk = threadIdx.x & 15;  // 16 x 16 grid (blockDim.x == 256)
  if (threadIdx.x == 0 && V[0] > thresh) piv_inv[0] = recip_newton(V[0]);
  __syncthreads();
  for (int j = 0; j < R; ++j) {
    const double d = V[j * ld + j];  // final: written by step j - 1 before its barrier
    if (!(d > thresh)) return false;  // every thread reads the same pivot
    const double inv = piv_inv[j & 1];
    for (int i = j + 1 + ti; i < R; i += 16) {
      const double aij = V[i * ld + j] * inv;
      for (int k = j + 1 + tk; k <= i; k += 16) V[i * ld + k] -= aij * V[k * ld + j];
    }
    if (threadIdx.x == 0) {
      piv[j] = d;
      if (j + 1 < R) {
        const double dn = V[(j + 1) * ld + j + 1];
        if (dn > thresh) piv_inv[(j + 1) & 1] = recip_newton(dn);
      }
    }
    __syncthreads();
  }
  for (int j = threadIdx.x; j < R; j += blockDim.x) invd[j] = 1.0 / sqrt(piv[j]);
  __syncthreads();
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
    const int i = e / R, j = e % R;
    if (j <= i) V[i * ld + j] *= invd[j];
  }
  __syncthreads();
  return true;
}

// The same factorisation with the work of every step packed densely over the
// CTA's threads.  FP64 runs at about two FMAs per clock per SM on this GPU, so
// a warp instruction with idle lanes costs as much as a full one; a fixed
// thread grid over the shrinking trailing triangle left most lanes idle.  Step
// j: threads j < i < R form s_i = A_ij / A_jj; after a barrier the
// (R-1-j)(R-j)/2 trailing elements A_ik (j < k <= i) are dealt out to the
// threads in turn (row of element e from a table), A_ik -= s_i A_kj; a second
// barrier ends the step.  Columns are scaled at the end as in
// cholesky_inplace, with the same result: L in the lower triangle of V and
// invd = 1 / diag(L).
__device__ inline bool cholesky_packed(double* V, int R, int ld, double thresh, double* invd) {
  __shared__ double srow[kMaxSolveRank];
  __shared__ double piv[kMaxSolveRank];
  __shared__ unsigned char tri_row[kMaxSolveRank * (kMaxSolveRank - 1) / 2];
  // row r of element e = r (r + 1) / 2 + c (c <= r) of a triangle enumerated by rows
  for (int r = threadIdx.x; r < R - 1; r += blockDim.x)
    for (int c = 0; c <= r; ++c) tri_row[r * (r + 1) / 2 + c] = static_cast<unsigned char>(r);
  __syncthreads();
  for (int j = 0; j < R; ++j) {
    const double d = V[j * ld + j];  // final since step j - 1
    if (!(d > thresh)) return false;  // every thread reads the same pivot
    const int i = j + 1 + static_cast<int>(threadIdx.x);
    if (threadIdx.x == 0) piv[j] = d;
    if (i < R) srow[i] = V[i * ld + j] * recip_newton(d);
    __syncthreads();
    const int n = R - 1 - j;
    const int ne = n * (n + 1) / 2;
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
      const int r = tri_row[e];
      const int ii = j + 1 + r, kk = j + 1 + (e - r * (r + 1) / 2);
      V[ii * ld + kk] = fma(-srow[ii], V[kk * ld + j], V[ii * ld + kk]);
    }
    __syncthreads();
  }
  for (int j = threadIdx.x; j < R; j += blockDim.x) invd[j] = 1.0 / sqrt(piv[j]);
  __syncthreads();
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
    const int i = e / R, j = e % R;
    if (j <= i) V[i * ld + j] *= invd[j];
  }
  __syncthreads();
  return true;
}

// Largest |V_aa| (one warp; a maximum does not depend on the order).
__device__ inline double max_diag(const double* V, int R, int ld) {
  __shared__ double mx;
  if (threadIdx.x < 32) {
    double m = 0.0;
    for (int a = threadIdx.x; a < R; a += 32) m = fmax(m, fabs(V[a * ld + a]));
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
    if (threadIdx.x == 0) mx = m;
  }
  __syncthreads();
  return mx;
}

// Symmetric eigendecomposition by parallel cyclic Jacobi (Golub & Van Loan,
// Alg. 8.4.2/8.4.3 with round-robin ordering).  V is overwritten by a
// near-diagonal matrix, Q by the eigenvectors (columns).
__device__ inline void jacobi_eigen(double* V, double* Q, int R) {
  __shared__ double cs_c[kMaxSolveRank / 2], cs_s[kMaxSolveRank / 2];
  __shared__ int cs_p[kMaxSolveRank / 2], cs_q[kMaxSolveRank / 2];
  __shared__ int done;
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) Q[e] = (e / R == e % R) ? 1.0 : 0.0;
  __syncthreads();
  const int H = R / 2;
  for (int sweep = 0; sweep < 40; ++sweep) {
    if (threadIdx.x == 0) {
      double off = 0.0, tot = 0.0;
      for (int a = 0; a < R; ++a)
        for (int b = 0; b < R; ++b) {
          double v = V[a * R + b] * V[a * R + b];
          tot += v;
          if (a != b) off += v;
        }
      done = off <= 1e-30 * tot;
    }
    __syncthreads();
    if (done) break;
    for (int k = 0; k < R - 1; ++k) {
      for (int p = threadIdx.x; p < H; p += blockDim.x) {
        int a = (k + p) % (R - 1), b = (k - p + R - 1) % (R - 1);
        if (p == 0) b = R - 1;
        int P = a < b ? a : b, Qi = a < b ? b : a;
        double app = V[P * R + P], aqq = V[Qi * R + Qi], apq = V[P * R + Qi];
        double c = 1.0, s = 0.0;
        if (fabs(apq) > 1e-300) {
          double tau = (aqq - app) / (2.0 * apq);
          double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          c = 1.0 / sqrt(1.0 + t * t);
          s = t * c;
        }
        cs_c[p] = c;
        cs_s[p] = s;
        cs_p[p] = P;
        cs_q[p] = Qi;
      }
      __syncthreads();
      for (int w = threadIdx.x; w < H * R; w += blockDim.x) {  // rows: V <- J^T V
        int p = w / R, col = w % R;
        int P = cs_p[p], Qi = cs_q[p];
        double c = cs_c[p], s = cs_s[p];
        double vp = V[P * R + col], vq = V[Qi * R + col];
        V[P * R + col] = c * vp - s * vq;
        V[Qi * R + col] = s * vp + c * vq;
      }
      __syncthreads();
      for (int w = threadIdx.x; w < H * R; w += blockDim.x) {  // columns: V <- V J, Q <- Q J
        int p = w / R, row = w % R;
        int P = cs_p[p], Qi = cs_q[p];
        double c = cs_c[p], s = cs_s[p];
        double vp = V[row * R + P], vq = V[row * R + Qi];
        V[row * R + P] = c * vp - s * vq;
        V[row * R + Qi] = s * vp + c * vq;
        double qp = Q[row * R + P], qq = Q[row * R + Qi];
        Q[row * R + P] = c * qp - s * qq;
        Q[row * R + Qi] = s * qp + c * qq;
      }
      __syncthreads();
    }
  }
}

}  // namespace gsp
