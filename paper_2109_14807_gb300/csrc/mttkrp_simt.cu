// The plain FP32 path of the two MTTKRP contractions: shared-memory tiled FFMA
// on CUDA cores (64 x 64 output tile per CTA, 4 x 4 per thread, 32-deep K
// slices).  Compute-bound at 2 * |X| * R flops per pass; it is the comparator
// the tensor-core path is measured against, and the path for small shapes.
#include "mttkrp.cuh"

namespace gsp {
namespace {

constexpr int BM = 64, BN = 64, BK = 32;

// Y'[xy][r] = sum_l sum_st T[l][xy][st] * KR[l*B2 + st][r]
__global__ void __launch_bounds__(256) k_xy_simt(const float* __restrict__ T,
                                                 const float* __restrict__ KR,
                                                 float* __restrict__ Yp, long long N2, int L,
                                                 int B2, int R) {
  __shared__ float As[BK][BM + 1];
  __shared__ float Bs[BK][BN];
  const int tid = threadIdx.x;
  const long long row0 = blockIdx.x * static_cast<long long>(BM);
  const int col0 = blockIdx.y * BN;
  const int tx = tid & 15, ty = tid >> 4;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
  for (int l = 0; l < L; ++l) {
    const float* Tl = T + (static_cast<long long>(l) * N2 + row0) * B2;
    const float* KRl = KR + static_cast<long long>(l) * B2 * R;
    for (int k0 = 0; k0 < B2; k0 += BK) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        int m = (tid >> 5) + 8 * i;
        As[tid & 31][m] = __ldg(Tl + static_cast<long long>(m) * B2 + k0 + (tid & 31));
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        int k = (tid >> 6) + 4 * i;
        int n = col0 + (tid & 63);
        Bs[k][tid & 63] = n < R ? __ldg(KRl + static_cast<long long>(k0 + k) * R + n) : 0.0f;
      }
      __syncthreads();
#pragma unroll 8
      for (int k = 0; k < BK; ++k) {
        float a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[k][ty * 4 + i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx * 4 + j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int n = col0 + tx * 4 + j;
      if (n < R) Yp[(row0 + ty * 4 + i) * R + n] = acc[i][j];
    }
}

// Zpart[l*C + c][st][r] = sum_{xy in chunk c} T[l][xy][st] * fx[x][r] * fy[y][r]
__global__ void __launch_bounds__(256) k_lst_simt(const float* __restrict__ T,
                                                  const float* __restrict__ fx,
                                                  const float* __restrict__ fy,
                                                  float* __restrict__ Zpart, int logN, int L,
                                                  int B2, int R, int C) {
  __shared__ float As[BK][BM];
  __shared__ float Bs[BK][BN];
  const int tid = threadIdx.x;
  const int st0 = blockIdx.x * BM;
  const int r0 = blockIdx.y * BN;
  const int unit = blockIdx.z;
  const int l = unit / C, c = unit % C;
  const int N = 1 << logN;
  const long long N2 = static_cast<long long>(N) * N;
  const long long rows = N2 / C;
  const long long xy0 = c * rows;
  const float* Tl = T + static_cast<long long>(l) * N2 * B2;
  const int tx = tid & 15, ty = tid >> 4;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
  for (long long k0 = 0; k0 < rows; k0 += BK) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      int k = (tid >> 6) + 4 * i;
      As[k][tid & 63] = __ldg(Tl + (xy0 + k0 + k) * B2 + st0 + (tid & 63));
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      int k = (tid >> 6) + 4 * i;
      long long xy = xy0 + k0 + k;
      int x = static_cast<int>(xy & (N - 1));
      int y = static_cast<int>(xy >> logN);
      int r = r0 + (tid & 63);
      Bs[k][tid & 63] = r < R ? __ldg(fx + x * R + r) * __ldg(fy + y * R + r) : 0.0f;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < BK; ++k) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int r = r0 + tx * 4 + j;
      if (r < R)
        Zpart[(static_cast<long long>(unit) * B2 + st0 + ty * 4 + i) * R + r] = acc[i][j];
    }
}

}  // namespace

int lst_chunks(const MttkrpDims& d, int precision) {
  long long per_chunk_blocks;
  (void)precision;
  per_chunk_blocks = static_cast<long long>(d.B2() / BM) * ((d.R + BN - 1) / BN) * d.L;
  long long target = 4LL * 148;
  long long C = 1;
  while (C * per_chunk_blocks < target && C * 2 * 256 <= d.N2()) C *= 2;
  return static_cast<int>(C);
}

int simt_mttkrp_xy(const float* T, const float* KR, float* Yp, const MttkrpDims& d,
                   cudaStream_t s) {
  if (d.N2() % BM || d.B2() % BK) return GSP_ERR_UNSUPPORTED;
  dim3 grid(static_cast<unsigned>(d.N2() / BM), (d.R + BN - 1) / BN);
  prof_begin(PROF_MTTKRP_XY, s);
  k_xy_simt<<<grid, 256, 0, s>>>(T, KR, Yp, d.N2(), d.L, d.B2(), d.R);
  prof_end(PROF_MTTKRP_XY, s);
  GSP_CHECK_LAUNCH();
  return GSP_OK;
}

int simt_mttkrp_lst(const float* T, const float* fx, const float* fy, float* Zpart,
                    const MttkrpDims& d, int chunks, cudaStream_t s) {
  if (d.B2() % BM || (d.N2() / chunks) % BK) return GSP_ERR_UNSUPPORTED;
  dim3 grid(d.B2() / BM, (d.R + BN - 1) / BN, d.L * chunks);
  prof_begin(PROF_MTTKRP_LST, s);
  k_lst_simt<<<grid, 256, 0, s>>>(T, fx, fy, Zpart, ilog2(d.N), d.L, d.B2(), d.R, chunks);
  prof_end(PROF_MTTKRP_LST, s);
  GSP_CHECK_LAUNCH();
  return GSP_OK;
}

}  // namespace gsp
