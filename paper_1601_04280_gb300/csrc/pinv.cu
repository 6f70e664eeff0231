// B = L_y^+ (P A) (Corollary 3.3, col:A_LLA, replacing steps 4-5 of
// Algorithm 1) and the assembly of L = L_y L_b, U = U_b (step 7).
//
// L_y^+ P = G^{-1} Lk^T with Lk the m x k unit lower trapezoidal factor in
// ORIGINAL row order (so no row gather of A is ever needed: W = L_y^+ P acts
// on A directly) and G = Lk^T Lk.  G = R^T R by a blocked Cholesky, R^{-1}
// by column back-substitution, G^{-1} = R^{-1} R^{-T}; all FP64.
#include "common.cuh"
#include "gemm_simt.cuh"
#include "pinv.cuh"

namespace rlu {

// Lk[i, c] (c < k) from the packed panel LU of Y: row i pivoted at step s
// holds L in columns < s and U from s on; unpivoted rows hold L everywhere.
__global__ void k_extract_Lk(int64_t m, int l, int k, const double* __restrict__ Y, const int32_t* __restrict__ pstep,
                             double* __restrict__ Lk) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m * k) return;
  int64_t i = e / k;
  int c = (int)(e - i * k);
  int s = pstep[i];
  double v;
  if (s < 0 || c < s) v = Y[i * l + c];
  else v = (c == s) ? 1.0 : 0.0;
  Lk[e] = v;
}

// Blocked right-looking Cholesky G = R^T R (R upper, overwriting the upper
// triangle of S), then R^{-1} column by column; one cooperative kernel with
// three grid barriers per 32-wide panel.
constexpr int kNb = 32;

__global__ void __launch_bounds__(256) k_chol_inv(int k, double* __restrict__ S, double* __restrict__ Rinv,
                                                  unsigned int* bar, unsigned int* status) {
  extern __shared__ __align__(16) double xs[];  // 8 warps x k
  __shared__ double blk[kNb][kNb + 1];
  const int tid = threadIdx.x;
  const int nt = (k + kNb - 1) / kNb;
  const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + tid;
  unsigned int epoch = 0;
  for (int J = 0; J < nt; ++J) {
    const int c0 = J * kNb;
    const int jb = min(kNb, k - c0);
    if (blockIdx.x == 0) {
      for (int e = tid; e < jb * jb; e += blockDim.x) {
        int r = e / jb, c = e % jb;
        blk[r][c] = S[(int64_t)(c0 + r) * k + c0 + c];
      }
      __syncthreads();
      for (int c = 0; c < jb; ++c) {
        if (tid == 0) {
          double d = blk[c][c];
          if (!(d > 0.0)) {
            set_flag(status, FLAG_ZERO_PIVOT);
            d = 1.0;
          }
          blk[c][c] = sqrt(d);
        }
        __syncthreads();
        const double dc = blk[c][c];
        for (int t = c + 1 + tid; t < jb; t += blockDim.x) blk[c][t] /= dc;
        __syncthreads();
        for (int e = tid; e < jb * jb; e += blockDim.x) {
          int r = e / jb, t = e % jb;
          if (r > c && t >= r) blk[r][t] -= blk[c][r] * blk[c][t];
        }
        __syncthreads();
      }
      for (int e = tid; e < jb * jb; e += blockDim.x) {
        int r = e / jb, c = e % jb;
        S[(int64_t)(c0 + r) * k + c0 + c] = (c >= r) ? blk[r][c] : 0.0;
      }
    }
    if (!grid_barrier(bar, ++epoch, status)) return;
    // panel row: S[J, K] <- R_JJ^{-T} S[J, K] for all columns right of the block
    const int rest = k - (c0 + jb);
    for (int64_t col = gtid; col < rest; col += gthreads) {
      const int gc = c0 + jb + (int)col;
      double x[kNb];
      for (int r = 0; r < jb; ++r) {
        double v = S[(int64_t)(c0 + r) * k + gc];
        for (int t = 0; t < r; ++t) v -= S[(int64_t)(c0 + t) * k + c0 + r] * x[t];
        x[r] = v / S[(int64_t)(c0 + r) * k + c0 + r];
      }
      for (int r = 0; r < jb; ++r) S[(int64_t)(c0 + r) * k + gc] = x[r];
    }
    if (!grid_barrier(bar, ++epoch, status)) return;
    // trailing update of the upper triangle: S[r, c] -= sum_t S[t, r] S[t, c]
    const int64_t tot = (int64_t)rest * rest;
    for (int64_t e = gtid; e < tot; e += gthreads) {
      const int r = c0 + jb + (int)(e / rest), c = c0 + jb + (int)(e % rest);
      if (c < r) continue;
      double s = 0.0;
      for (int t = 0; t < jb; ++t) s += S[(int64_t)(c0 + t) * k + r] * S[(int64_t)(c0 + t) * k + c];
      S[(int64_t)r * k + c] -= s;
    }
    if (!grid_barrier(bar, ++epoch, status)) return;
  }
  // R^{-1}: column c by back-substitution, one warp per column
  const int warp = tid >> 5, lane = tid & 31;
  double* x = xs + (int64_t)warp * k;
  const int64_t gwarp = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t c = gwarp; c < k; c += nwarps) {
    if (lane == 0) x[c] = 1.0 / S[c * k + c];
    __syncwarp();
    for (int64_t i = c - 1; i >= 0; --i) {
      double s = 0.0;
      for (int64_t t = i + 1 + lane; t <= c; t += 32) s += S[i * k + t] * x[t];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) x[i] = -s / S[i * k + i];
      __syncwarp();
    }
    for (int64_t i = lane; i < k; i += 32) Rinv[i * k + c] = (i <= c) ? x[i] : 0.0;
    __syncwarp();
  }
}

// Lk and the Gram matrix G = Lk^T Lk (split over row ranges, summed in fixed order).
int launch_gram(const PinvArgs& a, cudaStream_t st) {
  const int64_t m = a.m;
  const int k = a.k, l = a.l;
  k_extract_Lk<<<(unsigned)cdiv(m * k, 256), 256, 0, st>>>(m, l, k, a.Y, a.pstep, a.Lk);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  const int64_t tiles = cdiv(k, 64) * cdiv(k, 64);
  int S = (int)min64(a.max_gram_splits, max64(1, cdiv(2 * a.num_sms, tiles)));
  S = (int)min64(S, max64(1, cdiv(m, 64)));
  int rc = gemm_simt<double, double, double, double>(st, k, k, m, a.Lk, 1, k, a.Lk, k, 1, a.gram_part, k, 1, S,
                                                     (int64_t)k * k);
  if (rc) return rc;
  k_sum_slices<double><<<(unsigned)cdiv((int64_t)k * k, 256), 256, 0, st>>>((int64_t)k * k, S, a.gram_part, a.G);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  return RLU_OK;
}

// Cholesky G = R^T R and R^{-1}.
int launch_chol(const PinvArgs& a, cudaStream_t st) {
  const int k = a.k;
  RLU_CUDA_TRY(cudaMemsetAsync(a.bar, 0, sizeof(unsigned int), st));
  int G = a.num_sms;
  size_t smem = (size_t)8 * k * sizeof(double);
  RLU_CUDA_TRY(cudaFuncSetAttribute(k_chol_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  RLU_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_chol_inv, 256, smem));
  if (per_sm < 1) return RLU_EINVAL;
  double* Sm = a.G;
  double* Ri = a.Rinv;
  int kk = k;
  unsigned int* bar = a.bar;
  unsigned int* status = a.status;
  void* args[] = {&kk, &Sm, &Ri, &bar, &status};
  RLU_CUDA_TRY(cudaLaunchCooperativeKernel((void*)k_chol_inv, G, 256, args, smem, st));
  note_launch();
  return RLU_OK;
}

// G^{-1} = R^{-1} R^{-T}, then W = G^{-1} Lk^T (k x m), FP64 accumulate,
// stored in the B-product's type.
int launch_wform(const PinvArgs& a, cudaStream_t st) {
  const int64_t m = a.m;
  const int k = a.k;
  int rc = gemm_simt<double, double, double, double>(st, k, k, k, a.Rinv, k, 1, a.Rinv, 1, k, a.Ginv, k, 1);
  if (rc) return rc;
  if (a.w64)
    rc = gemm_simt<double, double, double, double>(st, k, m, k, a.Ginv, k, 1, a.Lk, 1, k,
                                                   reinterpret_cast<double*>(a.W), m, 1);
  else
    rc = gemm_simt<double, double, float, double>(st, k, m, k, a.Ginv, k, 1, a.Lk, 1, k,
                                                  reinterpret_cast<float*>(a.W), m, 1);
  return rc;
}

// ---------------------------------------------------------------------------
// Assembly of the outputs (step 7)
// ---------------------------------------------------------------------------
// L_y in P order: LyP[t, c] = Lk[perm[t], c]
template <typename T>
__global__ void k_build_LyP(int64_t m, int k, const double* __restrict__ Lk, const int64_t* __restrict__ perm,
                            T* __restrict__ LyP) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m * k) return;
  int64_t t = e / k;
  int c = (int)(e - t * k);
  LyP[e] = (T)Lk[perm[t] * k + c];
}

// From the packed column-pivoted LU of B (k x n, row-major, columns never
// moved): L_b[c, j] = B[c, q[j]] for c >= j; U[c, t] = B[c, q[t]] for t > c,
// 1 on the diagonal, 0 below.
template <typename T>
__global__ void k_build_Lb(int k, int64_t n, const T* __restrict__ Bp, const int64_t* __restrict__ q,
                           T* __restrict__ Lb) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * k) return;
  int c = e / k, j = e % k;
  Lb[e] = (c >= j) ? Bp[(int64_t)c * n + q[j]] : T(0);
}

template <typename T>
__global__ void k_build_U(int k, int64_t n, const T* __restrict__ Bp, const int64_t* __restrict__ q,
                          T* __restrict__ U) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)k * n) return;
  int64_t c = e / n, t = e - c * n;
  T v;
  if (t > c) v = Bp[c * n + q[t]];
  else v = (t == c) ? T(1) : T(0);
  U[e] = v;
}

template <typename T>
int launch_assemble(const AssembleArgs& a, cudaStream_t st) {
  const int64_t m = a.m, n = a.n;
  const int k = a.k;
  T* LyP = reinterpret_cast<T*>(a.LyP);
  T* Lb = reinterpret_cast<T*>(a.Lb);
  const T* Bp = reinterpret_cast<const T*>(a.Bp);
  k_build_LyP<T><<<(unsigned)cdiv(m * k, 256), 256, 0, st>>>(m, k, a.Lk, a.perm_y, LyP);
  k_build_Lb<T><<<(unsigned)cdiv((int64_t)k * k, 256), 256, 0, st>>>(k, n, Bp, a.perm_b, Lb);
  k_build_U<T><<<(unsigned)cdiv((int64_t)k * n, 256), 256, 0, st>>>(k, n, Bp, a.perm_b, reinterpret_cast<T*>(a.U));
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch(3);
  int rc = gemm_simt<T, T, T, T>(st, m, k, k, LyP, k, 1, Lb, k, 1, reinterpret_cast<T*>(a.L), k, 1);
  if (rc) return rc;
  RLU_CUDA_TRY(cudaMemcpyAsync(a.p, a.perm_y, sizeof(int64_t) * m, cudaMemcpyDeviceToDevice, st));
  RLU_CUDA_TRY(cudaMemcpyAsync(a.q, a.perm_b, sizeof(int64_t) * n, cudaMemcpyDeviceToDevice, st));
  return RLU_OK;
}

template int launch_assemble<double>(const AssembleArgs&, cudaStream_t);
template int launch_assemble<float>(const AssembleArgs&, cudaStream_t);

// ---------------------------------------------------------------------------
// B = W A (first version: SIMT, FP32 or FP64 accumulate)
// ---------------------------------------------------------------------------
int launch_bgemm_simt(const void* W, int w64, const void* A, int64_t lda, int dtype, int64_t m, int64_t n, int k,
                      void* B, cudaStream_t st) {
  if (w64) {
    if (dtype != RLU_F64) return RLU_EINVAL;
    return gemm_simt<double, double, double, double>(st, k, n, m, (const double*)W, m, 1, (const double*)A, lda, 1,
                                                     (double*)B, n, 1);
  }
  if (dtype == RLU_F32)
    return gemm_simt<float, float, float, float>(st, k, n, m, (const float*)W, m, 1, (const float*)A, lda, 1,
                                                 (float*)B, n, 1);
  if (dtype == RLU_BF16)
    return gemm_simt<float, __nv_bfloat16, float, float>(st, k, n, m, (const float*)W, m, 1,
                                                         (const __nv_bfloat16*)A, lda, 1, (float*)B, n, 1);
  return RLU_EINVAL;
}

}  // namespace rlu
