// Tiled SIMT GEMM on strided operands: C(i, j) = sum_kk A(i, kk) B(kk, j).
//   A(i, kk) = A[i * a_rs + kk * a_cs],  B(kk, j) = B[kk * b_rs + j * b_cs],
//   C(i, j)  = C[z * c_zs + i * c_rs + j * c_cs]   (z = split-K slice).
// 64 x 64 output tile per CTA, 16-deep K slices through shared memory, 256
// threads with a 4 x 4 register micro-tile each.  Used for the FP64 products
// of the pseudo-inverse (these run at the FP64 pipe rate whatever the tiling)
// and for the small FP32 products.
#pragma once
#include "common.cuh"

namespace rlu {

template <typename TA, typename TB, typename TC, typename TACC>
__global__ void __launch_bounds__(256) k_gemm_simt(int64_t M, int64_t N, int64_t K, const TA* __restrict__ A,
                                                   int64_t a_rs, int64_t a_cs, const TB* __restrict__ B,
                                                   int64_t b_rs, int64_t b_cs, TC* __restrict__ C, int64_t c_rs,
                                                   int64_t c_cs, int64_t c_zs, int64_t k_per_split) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ TACC sA[BK][BM + 1];
  __shared__ TACC sB[BK][BN + 1];
  const int tid = threadIdx.x;
  const int64_t i0 = (int64_t)blockIdx.y * BM, j0 = (int64_t)blockIdx.x * BN;
  const int64_t kbeg = (int64_t)blockIdx.z * k_per_split;
  const int64_t kend = min(K, kbeg + k_per_split);
  const int ti = tid / 16, tj = tid % 16;
  TACC acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = zero_<TACC>();
  const bool a_kfast = (a_cs == 1);
  const bool b_jfast = (b_cs == 1);
  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
    // A tile: BM x BK
    for (int e = tid; e < BM * BK; e += 256) {
      int ii, kk;
      if (a_kfast) { kk = e % BK; ii = e / BK; } else { ii = e % BM; kk = e / BM; }
      const int64_t gi = i0 + ii, gk = k0 + kk;
      TACC v = zero_<TACC>();
      if (gi < M && gk < kend) v = cvt<TACC>(A[gi * a_rs + gk * a_cs]);
      sA[kk][ii] = v;
    }
    // B tile: BK x BN
    for (int e = tid; e < BK * BN; e += 256) {
      int kk, jj;
      if (b_jfast) { jj = e % BN; kk = e / BN; } else { kk = e % BK; jj = e / BK; }
      const int64_t gj = j0 + jj, gk = k0 + kk;
      TACC v = zero_<TACC>();
      if (gj < N && gk < kend) v = cvt<TACC>(B[gk * b_rs + gj * b_cs]);
      sB[kk][jj] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      TACC a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { a[q] = sA[kk][ti + 16 * q]; b[q] = sB[kk][tj + 16 * q]; }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = mad(a[x], b[y], acc[x][y]);
    }
    __syncthreads();
  }
  TC* Cz = C + (int64_t)blockIdx.z * c_zs;
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int64_t gi = i0 + ti + 16 * x, gj = j0 + tj + 16 * y;
      if (gi < M && gj < N) Cz[gi * c_rs + gj * c_cs] = cvt<TC>(acc[x][y]);
    }
}

// C = A B with FP32 products and FP32 accumulation inside K chunks of
// kFlushK, and float-float accumulation across chunks: the rounding error of
// a K-long FP32 sum grows with K, so the long contraction is cut into short
// FP32 pieces whose partial sums are added exactly enough.  C is float-float.
template <typename TA, typename TB>
__global__ void __launch_bounds__(256) k_gemm_chunked(int64_t M, int64_t N, int64_t K, const TA* __restrict__ A,
                                                      int64_t lda, const TB* __restrict__ B, int64_t ldb,
                                                      df32* __restrict__ C, int64_t ldc) {
  constexpr int BM = 64, BN = 64, BK = 16, kFlushK = 256;
  __shared__ float sA[BK][BM + 1];
  __shared__ float sB[BK][BN + 1];
  const int tid = threadIdx.x;
  const int64_t i0 = (int64_t)blockIdx.y * BM, j0 = (int64_t)blockIdx.x * BN;
  const int ti = tid / 16, tj = tid % 16;
  float acc[4][4];
  df32 tot[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) { acc[a][b] = 0.f; tot[a][b] = df_make(0.f, 0.f); }
  for (int64_t k0 = 0; k0 < K; k0 += BK) {
    for (int e = tid; e < BM * BK; e += 256) {
      const int kk = e % BK, ii = e / BK;
      const int64_t gi = i0 + ii, gk = k0 + kk;
      sA[kk][ii] = (gi < M && gk < K) ? to_float(A[gi * lda + gk]) : 0.f;
    }
    for (int e = tid; e < BK * BN; e += 256) {
      const int jj = e % BN, kk = e / BN;
      const int64_t gj = j0 + jj, gk = k0 + kk;
      sB[kk][jj] = (gj < N && gk < K) ? to_float(B[gk * ldb + gj]) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { a[q] = sA[kk][ti + 16 * q]; b[q] = sB[kk][tj + 16 * q]; }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(a[x], b[y], acc[x][y]);
    }
    __syncthreads();
    if (((k0 + BK) % kFlushK) == 0 || k0 + BK >= K) {
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) { tot[x][y] = tot[x][y] + df_make(acc[x][y], 0.f); acc[x][y] = 0.f; }
    }
  }
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int64_t gi = i0 + ti + 16 * x, gj = j0 + tj + 16 * y;
      if (gi < M && gj < N) C[gi * ldc + gj] = tot[x][y];
    }
}

template <typename TA, typename TB>
inline int gemm_chunked(cudaStream_t st, int64_t M, int64_t N, int64_t K, const TA* A, int64_t lda, const TB* B,
                        int64_t ldb, df32* C, int64_t ldc) {
  if (M <= 0 || N <= 0) return RLU_OK;
  dim3 grid((unsigned)cdiv(N, 64), (unsigned)cdiv(M, 64), 1);
  k_gemm_chunked<TA, TB><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  return RLU_OK;
}

// Sum S split-K slices of an M x N row-major partial buffer (fixed order).
template <typename TC>
__global__ void k_sum_slices(int64_t MN, int S, const double* __restrict__ part, TC* __restrict__ out) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= MN) return;
  double s = 0.0;
  for (int z = 0; z < S; ++z) s += part[(int64_t)z * MN + e];
  out[e] = (TC)s;
}

template <typename TA, typename TB, typename TC, typename TACC>
inline int gemm_simt(cudaStream_t st, int64_t M, int64_t N, int64_t K, const TA* A, int64_t a_rs, int64_t a_cs,
                     const TB* B, int64_t b_rs, int64_t b_cs, TC* C, int64_t c_rs, int64_t c_cs, int splits = 1,
                     int64_t c_zs = 0) {
  if (M <= 0 || N <= 0) return RLU_OK;
  int64_t kps = cdiv(K, splits);
  kps = cdiv(kps, 16) * 16;
  dim3 grid((unsigned)cdiv(N, 64), (unsigned)cdiv(M, 64), (unsigned)splits);
  k_gemm_simt<TA, TB, TC, TACC><<<grid, 256, 0, st>>>(M, N, K, A, a_rs, a_cs, B, b_rs, b_cs, C, c_rs, c_cs, c_zs,
                                                       kps);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  return RLU_OK;
}

}  // namespace rlu
