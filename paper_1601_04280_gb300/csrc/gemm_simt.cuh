// Tiled SIMT GEMM on strided operands: C(i, j) = sum_kk A(i, kk) B(kk, j).
//   A(i, kk) = A[i * a_rs + kk * a_cs],  B(kk, j) = B[kk * b_rs + j * b_cs],
//   C(i, j)  = C[z * c_zs + i * c_rs + j * c_cs]   (z = split-K slice).
// 64 x 64 output tile per CTA, 16-deep K slices through shared memory, 256
// threads with a 4 x 4 register micro-tile each.  Used for the FP64 products
// of the pseudo-inverse (these run at the FP64 pipe rate whatever the tiling)
// and for the small FP32 products.
#pragma once
#include <type_traits>

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

// Sum S split-K slices of a symmetric n x n product whose partials hold only
// the 64 x 64 tiles on and above the diagonal (fixed order).
static __global__ void k_sum_slices_sym(int64_t nn, int S, const double* __restrict__ part, double* __restrict__ out) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)nn * nn) return;
  const int64_t i = e / nn, j = e - i * nn;
  const int64_t src = (i / 64 > j / 64) ? j * nn + i : e;
  double s = 0.0;
  for (int z = 0; z < S; ++z) s += part[(int64_t)z * nn * nn + src];
  out[e] = s;
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

// The same product accumulated in float-float on the FP32 pipes, with the
// cheaper accumulation of Ogita, Rump and Oishi ("Accurate sum and dot
// product", SISC 2005, Algorithm Dot2-style): each term a*b is split exactly
// into p + e (TwoProd by FMA, plus the hi*lo cross terms), p enters the running
// sum s through TwoSum, and the rounding errors of both go into a plain FP32
// correction c; (s, c) is renormalised once per K slice.  12 FP32 operations
// per term instead of the 18 of a full float-float multiply-add; error of order
// K * 2^-48 relative to the sum of |a*b|.  Operands are held in shared memory
// as separate hi / lo planes, each thread's 4 x 4 outputs contiguous so that
// one 16-byte load feeds 4 terms; the next K slice is fetched into registers
// while the current one is consumed (two shared-memory buffers).
template <typename T> __device__ __forceinline__ df32 to_df(T x) { return cvt<df32>(x); }

template <typename TC> __device__ __forceinline__ TC from_df(float s, float c);
template <> __device__ __forceinline__ double from_df<double>(float s, float c) { return (double)s + (double)c; }
template <> __device__ __forceinline__ float from_df<float>(float s, float c) { return s + c; }
template <> __device__ __forceinline__ df32 from_df<df32>(float s, float c) { return quick_two_sum(s, c); }

template <typename TA, typename TB, typename TC>
__global__ void __launch_bounds__(256) k_gemm_df32(int64_t M, int64_t N, int64_t K, const TA* __restrict__ A,
                                                   int64_t a_rs, int64_t a_cs, const TB* __restrict__ B,
                                                   int64_t b_rs, int64_t b_cs, TC* __restrict__ C, int64_t c_rs,
                                                   int64_t c_cs, int64_t c_zs, int64_t k_per_split,
                                                   int upper_only) {
  constexpr int BM = 64, BN = 64, BK = 16;
  // symmetric products (C = A A^T): the tiles below the diagonal are skipped
  // and read transposed by the consumer
  if (upper_only && blockIdx.y > blockIdx.x) return;
  __shared__ __align__(16) float sAh[2][BK][BM], sAl[2][BK][BM];
  __shared__ __align__(16) float sBh[2][BK][BN], sBl[2][BK][BN];
  const int tid = threadIdx.x;
  const int64_t i0 = (int64_t)blockIdx.y * BM, j0 = (int64_t)blockIdx.x * BN;
  const int64_t kbeg = (int64_t)blockIdx.z * k_per_split;
  const int64_t kend = min(K, kbeg + k_per_split);
  const int ti = tid / 16, tj = tid % 16;  // rows ti*4.., columns tj*4..
  const bool a_kfast = (a_cs == 1);
  const bool b_jfast = (b_cs == 1);
  float s[4][4], c[4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) { s[x][y] = 0.f; c[x][y] = 0.f; }

  df32 ra[4], rb[4];  // the next slice, in registers
  auto fetch = [&](int64_t k0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + 256 * q;
      int ii, kk;
      if (a_kfast) { kk = e % BK; ii = e / BK; } else { ii = e % BM; kk = e / BM; }
      const int64_t gi = i0 + ii, gk = k0 + kk;
      ra[q] = (gi < M && gk < kend) ? to_df(A[gi * a_rs + gk * a_cs]) : df_make(0.f, 0.f);
      int jj, kb;
      if (b_jfast) { jj = e % BN; kb = e / BN; } else { kb = e % BK; jj = e / BK; }
      const int64_t gj = j0 + jj, gkb = k0 + kb;
      rb[q] = (gj < N && gkb < kend) ? to_df(B[gkb * b_rs + gj * b_cs]) : df_make(0.f, 0.f);
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + 256 * q;
      int ii, kk;
      if (a_kfast) { kk = e % BK; ii = e / BK; } else { ii = e % BM; kk = e / BM; }
      sAh[buf][kk][ii] = ra[q].hi;
      sAl[buf][kk][ii] = ra[q].lo;
      int jj, kb;
      if (b_jfast) { jj = e % BN; kb = e / BN; } else { kb = e % BK; jj = e / BK; }
      sBh[buf][kb][jj] = rb[q].hi;
      sBl[buf][kb][jj] = rb[q].lo;
    }
  };

  int buf = 0;
  if (kbeg < kend) {
    fetch(kbeg);
    stash(0);
  }
  __syncthreads();
  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
    const bool next = k0 + BK < kend;
    if (next) fetch(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 ah = *reinterpret_cast<const float4*>(&sAh[buf][kk][ti * 4]);
      const float4 al = *reinterpret_cast<const float4*>(&sAl[buf][kk][ti * 4]);
      const float4 bh = *reinterpret_cast<const float4*>(&sBh[buf][kk][tj * 4]);
      const float4 bl = *reinterpret_cast<const float4*>(&sBl[buf][kk][tj * 4]);
      const float a_h[4] = {ah.x, ah.y, ah.z, ah.w}, a_l[4] = {al.x, al.y, al.z, al.w};
      const float b_h[4] = {bh.x, bh.y, bh.z, bh.w}, b_l[4] = {bl.x, bl.y, bl.z, bl.w};
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          const float p = __fmul_rn(a_h[x], b_h[y]);
          float e = __fmaf_rn(a_h[x], b_h[y], -p);
          e = __fmaf_rn(a_h[x], b_l[y], e);
          e = __fmaf_rn(a_l[x], b_h[y], e);
          const float t = __fadd_rn(s[x][y], p);
          const float bb = __fsub_rn(t, s[x][y]);
          const float err = __fadd_rn(__fsub_rn(s[x][y], __fsub_rn(t, bb)), __fsub_rn(p, bb));
          s[x][y] = t;
          c[x][y] = __fadd_rn(c[x][y], __fadd_rn(err, e));
        }
    }
    // renormalise once per slice: s + c stays exact, |c| stays below ulp(s)
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        const df32 r = two_sum(s[x][y], c[x][y]);
        s[x][y] = r.hi;
        c[x][y] = r.lo;
      }
    if (next) stash(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
  TC* Cz = C + (int64_t)blockIdx.z * c_zs;
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int64_t gi = i0 + ti * 4 + x, gj = j0 + tj * 4 + y;
      if (gi < M && gj < N) Cz[gi * c_rs + gj * c_cs] = from_df<TC>(s[x][y], c[x][y]);
    }
}

// The same sum stored as float-float.
static __global__ void k_sum_slices_df(int64_t MN, int S, const double* __restrict__ part, df32* __restrict__ out) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= MN) return;
  double s = 0.0;
  for (int z = 0; z < S; ++z) s += part[(int64_t)z * MN + e];
  out[e] = df_from_double(s);
}

template <typename TA, typename TB, typename TC, typename TACC>
inline int gemm_simt(cudaStream_t st, int64_t M, int64_t N, int64_t K, const TA* A, int64_t a_rs, int64_t a_cs,
                     const TB* B, int64_t b_rs, int64_t b_cs, TC* C, int64_t c_rs, int64_t c_cs, int splits = 1,
                     int64_t c_zs = 0, int upper_only = 0) {
  if (M <= 0 || N <= 0) return RLU_OK;
  int64_t kps = cdiv(K, splits);
  kps = cdiv(kps, 16) * 16;
  dim3 grid((unsigned)cdiv(N, 64), (unsigned)cdiv(M, 64), (unsigned)splits);
  if constexpr (std::is_same<TACC, df32>::value)
    k_gemm_df32<TA, TB, TC><<<grid, 256, 0, st>>>(M, N, K, A, a_rs, a_cs, B, b_rs, b_cs, C, c_rs, c_cs, c_zs, kps,
                                                  upper_only);
  else
    k_gemm_simt<TA, TB, TC, TACC><<<grid, 256, 0, st>>>(M, N, K, A, a_rs, a_cs, B, b_rs, b_cs, C, c_rs, c_cs, c_zs,
                                                         kps);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  return RLU_OK;
}

}  // namespace rlu
