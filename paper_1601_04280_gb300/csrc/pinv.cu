// B = L_y^+ (P A) (Corollary 3.3, col:A_LLA, replacing steps 4-5 of
// Algorithm 1) and the assembly of L = L_y L_b, U = U_b (step 7).
//
// L_y^+ P = G^{-1} Lk^T with Lk the m x k unit lower trapezoidal factor in
// ORIGINAL row order (so no row gather of A is ever needed: W = L_y^+ P acts
// on A directly) and G = Lk^T Lk.  G = R^T R by a blocked Cholesky, R^{-1}
// by column back-substitution, G^{-1} = R^{-1} R^{-T}; all FP64.
#include <type_traits>

#include "common.cuh"
#include "gemm_simt.cuh"
#include "pinv.cuh"

namespace rlu {

// Lk[i, c] (c < k) from the packed panel LU of Y: row i pivoted at step s
// holds L in columns < s and U from s on; unpivoted rows hold L everywhere.
template <typename TL>
__global__ void k_extract_Lk(int64_t m, int l, int k, const double* __restrict__ Y, const int32_t* __restrict__ pstep,
                             TL* __restrict__ Lk) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m * k) return;
  int64_t i = e / k;
  int c = (int)(e - i * k);
  int s = pstep[i];
  double v;
  if (s < 0 || c < s) v = Y[i * l + c];
  else v = (c == s) ? 1.0 : 0.0;
  Lk[e] = cvt<TL>(v);
}

// Blocked right-looking Cholesky G = R^T R (R upper, overwriting the upper
// triangle of S), then R^{-1}; one cooperative kernel, FP64, with three grid
// barriers per 32-wide panel and two more before the column solves of R^{-1}.
constexpr int kNb = 32;

__global__ void __launch_bounds__(256) k_chol_inv(int k, double* __restrict__ S, double* __restrict__ Rinv,
                                                  unsigned int* bar, unsigned int* status, int tri_smem) {
  // FP64 on this part has long latency as well as low throughput, so every
  // sequential chain below is spread over threads: one thread per element in
  // the diagonal factor, one warp per column (lanes = rows) in the triangular
  // solves, with reciprocals of the diagonal computed once per block.
  __shared__ double blk[kNb][kNb + 1];
  __shared__ double rdiag[kNb];
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  constexpr int NW = 8;
  const int nt = (k + kNb - 1) / kNb;
  const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + tid;
  const int64_t gwarp = (int64_t)blockIdx.x * NW + warp;
  const int64_t nwarps = (int64_t)gridDim.x * NW;
  unsigned int epoch = 0;
  for (int J = 0; J < nt; ++J) {
    const int c0 = J * kNb;
    const int jb = min(kNb, k - c0);
    // (a) diagonal block by CTA 0, right-looking, all threads, in the form
    // G = U^T D^{-1} U (U = D R): column c only needs 1 / g_cc (every thread
    // takes it from the pivot in shared memory, no serial step), the update
    // g_rt -= g_cr g_ct / g_cc runs on unscaled rows, and the square roots and
    // the row scaling R[c][t] = g_ct / sqrt(g_cc) wait until the block is done.
    if (blockIdx.x == 0) {
      for (int e = tid; e < kNb * kNb; e += blockDim.x) {
        int r = e / kNb, c = e % kNb;
        blk[r][c] = (r < jb && c < jb) ? S[(int64_t)(c0 + r) * k + c0 + c] : (r == c ? 1.0 : 0.0);
      }
      __syncthreads();
      // FP64 issues at a small fraction of the FP32 rate whatever the active
      // lanes, so each FP64 instruction is issued once: warp 0 forms the
      // scaled row u_t = g_ct / g_cc, then warp w updates rows r = w, w+8, ...
      // (lane t, one FMA per row), skipping the rows already eliminated.
      for (int c = 0; c < jb; ++c) {
        if (warp == 0) {
          const double piv = blk[c][c];
          const double inv = (piv > 0.0) ? rcp_newton(piv) : 0.0;
          if (lane > c && lane < jb) rdiag[lane] = blk[c][lane] * inv;
        }
        __syncthreads();
        for (int r = c + 1 + ((warp - (c + 1)) % NW + NW) % NW; r < jb; r += NW)
          if (lane >= r && lane < jb) blk[r][lane] = fma(-blk[c][r], rdiag[lane], blk[r][lane]);
        __syncthreads();
      }
      if (tid < jb) {
        double d = blk[tid][tid];
        if (!(d > 0.0)) {
          set_flag(status, FLAG_ZERO_PIVOT);
          d = 1.0;
        }
        rdiag[tid] = 1.0 / sqrt(d);
      }
      __syncthreads();
      for (int e = tid; e < jb * jb; e += blockDim.x) {
        int r = e / jb, c = e % jb;
        S[(int64_t)(c0 + r) * k + c0 + c] = (c >= r) ? blk[r][c] * rdiag[r] : 0.0;
      }
    }
    if (!grid_barrier(bar, ++epoch, status)) return;
    const int rest = k - (c0 + jb);
    if (rest > 0) {
      // (b) panel row S[J, K] <- R_JJ^{-T} S[J, K]; warp per column, lane = row r:
      // after lane t finalizes x_t, lanes r > t remove R[t][r] x_t.
      double rcol[kNb];  // rcol[t] = R_JJ[t][lane]
#pragma unroll
      for (int t = 0; t < kNb; ++t) rcol[t] = (t < jb && lane < jb) ? S[(int64_t)(c0 + t) * k + c0 + lane] : 0.0;
      const double rinv_l = (lane < jb) ? rcp_newton(S[(int64_t)(c0 + lane) * k + c0 + lane]) : 1.0;
      for (int64_t col = gwarp; col < rest; col += nwarps) {
        const int gc = c0 + jb + (int)col;
        double b = (lane < jb) ? S[(int64_t)(c0 + lane) * k + gc] : 0.0;
        double xl = 0.0;
#pragma unroll
        for (int t = 0; t < kNb; ++t) {
          const double xt_local = (lane == t) ? b * rinv_l : 0.0;
          const double xt = __shfl_sync(0xffffffffu, xt_local, t);
          if (lane == t) xl = xt;
          if (lane > t) b -= rcol[t] * xt;
        }
        if (lane < jb) S[(int64_t)(c0 + lane) * k + gc] = xl;
      }
      if (!grid_barrier(bar, ++epoch, status)) return;
      // (c) trailing update of the upper triangle: S[r, c] -= sum_t S[t, r] S[t, c]
      const int64_t tot = (int64_t)rest * rest;
      for (int64_t e = gtid; e < tot; e += gthreads) {
        const int rr = (int)(e / rest), cc = (int)(e - (int64_t)rr * rest);
        if (cc < rr) continue;
        const int r = c0 + jb + rr, c = c0 + jb + cc;
        double acc0 = 0.0, acc1 = 0.0;
#pragma unroll
        for (int t = 0; t < kNb; t += 2) {
          if (t < jb) acc0 += S[(int64_t)(c0 + t) * k + r] * S[(int64_t)(c0 + t) * k + c];
          if (t + 1 < jb) acc1 += S[(int64_t)(c0 + t + 1) * k + r] * S[(int64_t)(c0 + t + 1) * k + c];
        }
        S[(int64_t)r * k + c] -= acc0 + acc1;
      }
      if (!grid_barrier(bar, ++epoch, status)) return;
    }
  }
  // R^{-1} column by column, FP64: column j solves R x = e_j from the bottom
  // up, one warp per column, the working vector w in this warp's part of
  // shared memory.  R's columns, each scaled by 1 / R[t][t], are first written
  // into the free strictly lower triangle of S (S[t][i] = R[i][t] / R[t][t],
  // i < t), so that a step of the solve is one FMA per entry on the dependent
  // chain, w_i -= S[t][i] w_t, and x_t = w_t / R[t][t] is taken at the end.
  // A CTA that owns columns first copies the rows it reads into shared memory
  // (packed: row t at t (t - 1) / 2) when tri_smem is set.
  if (!grid_barrier(bar, ++epoch, status)) return;
  for (int64_t e = gtid; e < (int64_t)k * k; e += gthreads) {
    const int t = (int)(e / k), i = (int)(e - (int64_t)t * k);
    if (i < t) S[(int64_t)t * k + i] = S[(int64_t)i * k + t] * (1.0 / S[(int64_t)t * k + t]);
  }
  if (!grid_barrier(bar, ++epoch, status)) return;
  extern __shared__ __align__(16) unsigned char chol_smem[];
  double* rdg = reinterpret_cast<double*>(chol_smem);                     // k: 1 / R[i][i]
  double* xw = rdg + k + (size_t)warp * k;                                 // k per warp
  double* tri = rdg + (size_t)(NW + 1) * k;                                // packed scaled rows
  for (int i = tid; i < k; i += blockDim.x) rdg[i] = 1.0 / S[(int64_t)i * k + i];
  int T = 0;  // rows this CTA reads: up to its last column
  for (int64_t j = (int64_t)blockIdx.x * NW; j < k; j += nwarps) T = (int)min((int64_t)k, j + NW);
  if (tri_smem)
    for (int t = warp; t < T; t += NW)
      for (int i = lane; i < t; i += 32) tri[(size_t)t * (t - 1) / 2 + i] = S[(int64_t)t * k + i];
  __syncthreads();
  for (int64_t j = gwarp; j < k; j += nwarps) {
    for (int i = lane; i <= j; i += 32) xw[i] = (i == j) ? 1.0 : 0.0;
    __syncwarp();
    // two loops so that the row loads of the global-memory one are known not
    // to alias w (and can be issued ahead of the chain)
    if (tri_smem) {
      for (int t = (int)j; t > 0; --t) {
        const double wt = xw[t];  // final: every step above t has been applied
        const double* rt = tri + (size_t)t * (t - 1) / 2;
        for (int i = lane; i < t; i += 32) xw[i] = fma(-wt, rt[i], xw[i]);
        __syncwarp();
      }
    } else {
      for (int t = (int)j; t > 0; --t) {
        const double wt = xw[t];
        const double* __restrict__ rt = S + (int64_t)t * k;
        for (int i = lane; i < t; i += 32) xw[i] = fma(-wt, __ldcg(rt + i), xw[i]);
        __syncwarp();
      }
    }
    for (int i = lane; i < k; i += 32) Rinv[(int64_t)i * k + j] = (i <= j) ? xw[i] * rdg[i] : 0.0;
    __syncwarp();
  }
}

// Lk and the Gram matrix G = Lk^T Lk (split over row ranges, summed in fixed
// order).  FP64 in the FP64 mode; float-float (about 48 bits) otherwise.
int launch_extract_Lk(const PinvArgs& a, cudaStream_t st) {
  const int64_t m = a.m;
  const int k = a.k, l = a.l;
  if (a.w64)
    k_extract_Lk<double><<<(unsigned)cdiv(m * k, 256), 256, 0, st>>>(m, l, k, a.Y, a.pstep,
                                                                      reinterpret_cast<double*>(a.Lk));
  else
    k_extract_Lk<df32><<<(unsigned)cdiv(m * k, 256), 256, 0, st>>>(m, l, k, a.Y, a.pstep,
                                                                    reinterpret_cast<df32*>(a.Lk));
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  return RLU_OK;
}

// out (cols x rows) = in (rows x cols, leading dimension ld_in) transposed,
// through 32 x 32 shared-memory tiles; TO(x) converts (FP64 from float-float).
template <typename TI, typename TO> __device__ __forceinline__ TO tr_cvt(TI x) { return (TO)x; }
template <> __device__ __forceinline__ double tr_cvt<df32, double>(df32 x) { return to_double(x); }

template <typename TI, typename TO>
__global__ void k_transpose_cvt(int64_t rows, int64_t cols, const TI* __restrict__ in, int64_t ld_in,
                                TO* __restrict__ out) {
  __shared__ TO t[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t r = r0 + y, c = c0 + threadIdx.x;
    if (r < rows && c < cols) t[y][threadIdx.x] = tr_cvt<TI, TO>(in[r * ld_in + c]);
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t c = c0 + y, r = r0 + threadIdx.x;
    if (r < rows && c < cols) out[c * rows + r] = t[threadIdx.x][y];
  }
}

template <typename TI, typename TO>
static int transpose_cvt(int64_t rows, int64_t cols, const TI* in, int64_t ld_in, TO* out, cudaStream_t st) {
  dim3 grid((unsigned)cdiv(cols, 32), (unsigned)cdiv(rows, 32));
  k_transpose_cvt<TI, TO><<<grid, dim3(32, 8), 0, st>>>(rows, cols, in, ld_in, out);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  return RLU_OK;
}

int launch_second_projection(const SecondArgs& s, const PinvArgs& a, SketchWs& ws2, cudaStream_t st) {
  const int64_t m = s.m, n = s.n;
  const int k = s.k, k2 = s.k2, l2 = s.l2;
  const bool w64 = a.w64 != 0;
  int rc;
  // step 4: Omega_2 over the m rows (hash, signs, frequencies, bucket lists)
  ws2.chunk = 1024;
  ws2.nchunks = cdiv(m, ws2.chunk);
  if ((rc = launch_sketch_params(ws2, m, l2, k2, s.seed2, st))) return rc;
  // step 5: Omega_2' A (through A^T: the first sketch applied to the n columns)
  if (s.dtype == RLU_F64)
    rc = transpose_cvt<double, double>(m, n, (const double*)s.A, s.lda, (double*)s.AT, st);
  else if (s.dtype == RLU_F32)
    rc = transpose_cvt<float, float>(m, n, (const float*)s.A, s.lda, (float*)s.AT, st);
  else
    rc = transpose_cvt<__nv_bfloat16, __nv_bfloat16>(m, n, (const __nv_bfloat16*)s.A, s.lda, (__nv_bfloat16*)s.AT,
                                                      st);
  if (rc) return rc;
  if ((rc = launch_sketch_dense(s.AT, m, s.dtype, s.dtype == RLU_F64, n, m, l2, k2, ws2, s.Y2T, a.status,
                                a.num_sms, st)))
    return rc;
  // ... and Omega_2' Lk, in FP64 (Lk is the L_1 of step 3 in A's row order)
  if ((rc = launch_extract_Lk(a, st))) return rc;
  if (w64)
    rc = transpose_cvt<double, double>(m, k, (const double*)a.Lk, k, s.LkT, st);
  else
    rc = transpose_cvt<df32, double>(m, k, (const df32*)a.Lk, k, s.LkT, st);
  if (rc) return rc;
  if ((rc = launch_sketch_dense(s.LkT, m, RLU_F64, true, k, m, l2, k2, ws2, s.ZT, a.status, a.num_sms, st)))
    return rc;
  // Z^+ = (Z^T Z)^{-1} Z^T with Z = ZT^T (k2 x k): Gram, Cholesky, inverse, as for L_y^+
  const int64_t tk = cdiv(k, 64);
  const int64_t tiles = w64 ? tk * tk : tk * (tk + 1) / 2;
  int S = (int)min64(a.max_gram_splits, max64(1, cdiv(2 * a.num_sms, tiles)));
  S = (int)min64(S, max64(1, cdiv(k2, 64)));
  const int64_t kps = cdiv(cdiv(k2, S), 16) * 16;
  S = (int)cdiv(k2, kps);
  if (w64) {
    rc = gemm_simt<double, double, double, double>(st, k, k, k2, s.ZT, k2, 1, s.ZT, 1, k2, a.gram_part, k, 1, S,
                                                   (int64_t)k * k);
    if (rc) return rc;
    k_sum_slices<double><<<(unsigned)cdiv((int64_t)k * k, 256), 256, 0, st>>>((int64_t)k * k, S, a.gram_part, a.G);
  } else {
    rc = gemm_simt<double, double, double, df32>(st, k, k, k2, s.ZT, k2, 1, s.ZT, 1, k2, a.gram_part, k, 1, S,
                                                 (int64_t)k * k, 1);
    if (rc) return rc;
    k_sum_slices_sym<<<(unsigned)cdiv((int64_t)k * k, 256), 256, 0, st>>>(k, S, a.gram_part, a.G);
  }
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  if ((rc = launch_chol(a, st))) return rc;
  // G^{-1} = R^{-1} R^{-T} (as in the W form), then W2 = G^{-1} Z^T and B = W2 Y2
  if (w64) {
    rc = gemm_simt<double, double, double, double>(st, k, k, k, a.Rinv, k, 1, a.Rinv, 1, k, a.Ginv, k, 1);
    if (rc) return rc;
    rc = gemm_simt<double, double, double, double>(st, k, k2, k, a.Ginv, k, 1, s.ZT, k2, 1, (double*)s.W2, k2, 1);
    if (rc) return rc;
    return gemm_simt<double, double, double, double>(st, k, n, k2, (const double*)s.W2, k2, 1, s.Y2T, 1, k2,
                                                     (double*)s.B, n, 1);
  }
  int Sg = (int)min64(a.max_gram_splits, max64(1, cdiv(2 * a.num_sms, tk * tk)));
  Sg = (int)min64(Sg, max64(1, cdiv(k, 16)));
  const int64_t kpsg = cdiv(cdiv(k, Sg), 16) * 16;
  Sg = (int)cdiv(k, kpsg);
  rc = gemm_simt<double, double, double, df32>(st, k, k, k, a.Rinv, k, 1, a.Rinv, 1, k, a.gram_part, k, 1, Sg,
                                               (int64_t)k * k);
  if (rc) return rc;
  df32* Ginv = reinterpret_cast<df32*>(a.Ginv);
  k_sum_slices_df<<<(unsigned)cdiv((int64_t)k * k, 256), 256, 0, st>>>((int64_t)k * k, Sg, a.gram_part, Ginv);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  rc = gemm_simt<df32, double, df32, df32>(st, k, k2, k, Ginv, k, 1, s.ZT, k2, 1, (df32*)s.W2, k2, 1);
  if (rc) return rc;
  return gemm_simt<df32, double, df32, df32>(st, k, n, k2, (const df32*)s.W2, k2, 1, s.Y2T, 1, k2, (df32*)s.B, n,
                                             1);
}

int launch_gram(const PinvArgs& a, cudaStream_t st) {
  const int64_t m = a.m;
  const int k = a.k, l = a.l;
  const int64_t tk = cdiv(k, 64);
  const int64_t tiles = a.w64 ? tk * tk : tk * (tk + 1) / 2;  // the float-float product skips the lower tiles
  int S = (int)min64(a.max_gram_splits, max64(1, cdiv(2 * a.num_sms, tiles)));
  S = (int)min64(S, max64(1, cdiv(m, 64)));
  int rc;
  if (a.w64) {
    double* Lk = reinterpret_cast<double*>(a.Lk);
    k_extract_Lk<double><<<(unsigned)cdiv(m * k, 256), 256, 0, st>>>(m, l, k, a.Y, a.pstep, Lk);
    RLU_CUDA_TRY(cudaGetLastError());
    note_launch();
    rc = gemm_simt<double, double, double, double>(st, k, k, m, Lk, 1, k, Lk, k, 1, a.gram_part, k, 1, S,
                                                   (int64_t)k * k);
  } else {
    df32* Lk = reinterpret_cast<df32*>(a.Lk);
    k_extract_Lk<df32><<<(unsigned)cdiv(m * k, 256), 256, 0, st>>>(m, l, k, a.Y, a.pstep, Lk);
    RLU_CUDA_TRY(cudaGetLastError());
    note_launch();
    if (a.ltc && a.ltc->ready) {
      // six-digit products on the tensor cores, FP64 partials per split of the rows
      return launch_gram_tc(*a.ltc, Lk, a.gram_part, a.max_gram_splits, a.G, a.status, st);
    }
    // G is symmetric: only the tiles on and above the diagonal are computed
    rc = gemm_simt<df32, df32, double, df32>(st, k, k, m, Lk, 1, k, Lk, k, 1, a.gram_part, k, 1, S,
                                             (int64_t)k * k, 1);
    if (rc) return rc;
    k_sum_slices_sym<<<(unsigned)cdiv((int64_t)k * k, 256), 256, 0, st>>>(k, S, a.gram_part, a.G);
    RLU_CUDA_TRY(cudaGetLastError());
    note_launch();
    return RLU_OK;
  }
  if (rc) return rc;
  k_sum_slices<double><<<(unsigned)cdiv((int64_t)k * k, 256), 256, 0, st>>>((int64_t)k * k, S, a.gram_part, a.G);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  return RLU_OK;
}

// Cholesky G = R^T R and R^{-1} (FP64).
int launch_chol(const PinvArgs& a, cudaStream_t st) {
  const int k = a.k;
  RLU_CUDA_TRY(cudaMemsetAsync(a.bar, 0, sizeof(unsigned int), st));
  // 1/diag(R) and one k-vector per warp (R^{-1} columns), and the scaled
  // triangle of R when it fits
  const size_t base = (size_t)9 * k * sizeof(double);
  const size_t trib = (size_t)k * (k - 1) / 2 * sizeof(double);
  int tri_smem = base + trib <= 200 * 1024 ? 1 : 0;
  const size_t smem = base + (tri_smem ? trib : 0);
  if (int rc_ = allow_dynamic_smem((const void*)k_chol_inv, smem)) return rc_;
  int per_sm = 0;
  RLU_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_chol_inv, 256, smem));
  if (per_sm < 1) return RLU_EINVAL;
  int G = a.coop_ctas > 0 ? min(a.coop_ctas, a.num_sms) : a.num_sms;
  double* Sm = a.G;
  double* Ri = a.Rinv;
  int kk = k;
  unsigned int* bar = a.bar;
  unsigned int* status = a.status;
  void* args[] = {&kk, &Sm, &Ri, &bar, &status, &tri_smem};
  RLU_CUDA_TRY(launch_cooperative((void*)k_chol_inv, G, 256, args, smem, st));
  note_launch();
  return RLU_OK;
}

// G^{-1} = R^{-1} R^{-T}, then W = G^{-1} Lk^T (k x m).  FP64 in the FP64
// mode; float-float products otherwise, W stored as FP32.
int launch_wform(const PinvArgs& a, cudaStream_t st) {
  const int64_t m = a.m;
  const int k = a.k;
  int rc;
  if (a.w64) {
    rc = gemm_simt<double, double, double, double>(st, k, k, k, a.Rinv, k, 1, a.Rinv, 1, k, a.Ginv, k, 1);
    if (rc) return rc;
    return gemm_simt<double, double, double, double>(st, k, m, k, a.Ginv, k, 1,
                                                     reinterpret_cast<const double*>(a.Lk), 1, k,
                                                     reinterpret_cast<double*>(a.W), m, 1);
  }
  // G^{-1} = R^{-1} R^{-T}: a small product (k x k x k), split over K so that it
  // fills the GPU; partials in the Gram scratch (free again after the
  // Cholesky), summed in FP64 and stored as float-float for the W product.
  const int64_t tiles = cdiv(k, 64) * cdiv(k, 64);
  int S = (int)min64(a.max_gram_splits, max64(1, cdiv(2 * a.num_sms, tiles)));
  S = (int)min64(S, max64(1, cdiv(k, 16)));
  const int64_t kps = cdiv(cdiv(k, S), 16) * 16;
  S = (int)cdiv(k, kps);
  rc = gemm_simt<double, double, double, df32>(st, k, k, k, a.Rinv, k, 1, a.Rinv, 1, k, a.gram_part, k, 1, S,
                                               (int64_t)k * k);
  if (rc) return rc;
  df32* Ginv = reinterpret_cast<df32*>(a.Ginv);
  k_sum_slices_df<<<(unsigned)cdiv((int64_t)k * k, 256), 256, 0, st>>>((int64_t)k * k, S, a.gram_part, Ginv);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  // W = G^{-1} Lk^T: an exact five-digit product on the tensor cores (which
  // also writes W's BF16 planes for the tensor-core B when given them), else
  // float-float on the SIMT pipes
  if (a.ltc && a.ltc->ready)
    return launch_w_tc(*a.ltc, Ginv, reinterpret_cast<const df32*>(a.Lk), reinterpret_cast<float*>(a.W), a.wplanes,
                       a.ldw, a.status, st);
  return gemm_simt<df32, df32, float, df32>(st, k, m, k, Ginv, k, 1, reinterpret_cast<const df32*>(a.Lk), 1, k,
                                            reinterpret_cast<float*>(a.W), m, 1);
}

// ---------------------------------------------------------------------------
// Assembly of the outputs (step 7)
// ---------------------------------------------------------------------------
// L_y in P order: LyP[t, c] = Lk[perm[t], c]
template <typename T>
__global__ void k_build_LyP(int64_t m, int k, const T* __restrict__ Lk, const int64_t* __restrict__ perm,
                            T* __restrict__ LyP) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m * k) return;
  int64_t t = e / k;
  int c = (int)(e - t * k);
  LyP[e] = Lk[perm[t] * k + c];
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
  Lb[e] = (c >= j) ? Bp[(int64_t)c * n + q[j]] : zero_<T>();
}

// L = (P L_y) L_b with FP32 products and FP32 accumulation, L_b (k x k,
// lower triangular) resident in shared memory as FP32 and the rows of P L_y
// gathered from Lk on the fly (row i of P L_y = row perm[i] of Lk).  A warp
// takes four rows at a time: lane owns columns j = lane + 32 q of them, and
// each L_b entry read from shared memory serves four rows.  The k-term sums
// run in ascending order of the summation index.
constexpr int kAsmRows = 4;
constexpr int kAsmMaxQ = 8;  // k <= 256
template <typename T, typename TO, int Q>
__global__ void __launch_bounds__(512, 1) k_assemble_rows(int64_t m, int k, const T* __restrict__ Lk,
                                                       const int64_t* __restrict__ perm, const T* __restrict__ Lb,
                                                       TO* __restrict__ L) {
  extern __shared__ __align__(16) float lbs[];  // k x k
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) lbs[e] = to_float(Lb[e]);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t tasks = cdiv(m, kAsmRows);
  for (int64_t task = wid; task < tasks; task += nw) {
    const int64_t i0 = task * kAsmRows;
    const T* src[kAsmRows];
#pragma unroll
    for (int r = 0; r < kAsmRows; ++r) src[r] = i0 + r < m ? Lk + perm[i0 + r] * k : nullptr;
    float acc[kAsmRows][Q];
#pragma unroll
    for (int r = 0; r < kAsmRows; ++r)
#pragma unroll
      for (int q = 0; q < Q; ++q) acc[r][q] = 0.f;
    // the next 32 entries of the four rows are loaded while these are used
    float an[kAsmRows];
#pragma unroll
    for (int r = 0; r < kAsmRows; ++r) an[r] = (src[r] && lane < k) ? to_float(src[r][lane]) : 0.f;
    for (int t0 = 0; t0 < k; t0 += 32) {
      float a[kAsmRows];
#pragma unroll
      for (int r = 0; r < kAsmRows; ++r) {
        a[r] = an[r];
        an[r] = (src[r] && t0 + 32 + lane < k) ? to_float(src[r][t0 + 32 + lane]) : 0.f;
      }
      const int tn = min(32, k - t0);
      for (int tt = 0; tt < tn; ++tt) {
        const float* brow = lbs + (size_t)(t0 + tt) * k;
        float b[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) b[q] = lane + 32 * q < k ? brow[lane + 32 * q] : 0.f;
#pragma unroll
        for (int r = 0; r < kAsmRows; ++r) {
          const float av = __shfl_sync(0xffffffffu, a[r], tt);
#pragma unroll
          for (int q = 0; q < Q; ++q) acc[r][q] = fmaf(av, b[q], acc[r][q]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < kAsmRows; ++r)
      if (i0 + r < m)
#pragma unroll
        for (int q = 0; q < Q; ++q)
          if (lane + 32 * q < k) L[(i0 + r) * k + lane + 32 * q] = (TO)acc[r][q];
  }
}

template <typename T, typename TO>
__global__ void k_build_U(int k, int64_t n, const T* __restrict__ Bp, const int64_t* __restrict__ q,
                          TO* __restrict__ U) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)k * n) return;
  int64_t c = e / n, t = e - c * n;
  TO v;
  if (t > c) v = cvt<TO>(Bp[c * n + q[t]]);
  else v = (t == c) ? TO(1) : TO(0);
  U[e] = v;
}

template <typename T, typename TO>
int launch_assemble(const AssembleArgs& a, cudaStream_t st) {
  const int64_t m = a.m, n = a.n;
  const int k = a.k;
  T* LyP = reinterpret_cast<T*>(a.LyP);
  T* Lb = reinterpret_cast<T*>(a.Lb);
  const T* Bp = reinterpret_cast<const T*>(a.Bp);
  // FP32 outputs: L = L_y L_b as an exact digit product on the tensor cores
  // (k <= 512), else as an FP32 product with L_b resident in shared memory
  // (no P L_y copy), else the SIMT GEMM
  const bool tc_digits = a.fp32_product && std::is_same<T, df32>::value && a.ltc && a.ltc->ready;
  const bool rows_kernel = !tc_digits && a.fp32_product && !std::is_same<T, double>::value && k <= 32 * kAsmMaxQ &&
                           (size_t)k * k * sizeof(float) <= 200 * 1024 && a.num_sms > 0;
  if (!rows_kernel && !tc_digits) {
    k_build_LyP<T><<<(unsigned)cdiv(m * k, 256), 256, 0, st>>>(m, k, reinterpret_cast<const T*>(a.Lk), a.perm_y,
                                                                LyP);
    note_launch();
  }
  if (!tc_digits) {
    k_build_Lb<T><<<(unsigned)cdiv((int64_t)k * k, 256), 256, 0, st>>>(k, n, Bp, a.perm_b, Lb);
    note_launch();
  }
  k_build_U<T, TO><<<(unsigned)cdiv((int64_t)k * n, 256), 256, 0, st>>>(k, n, Bp, a.perm_b,
                                                                          reinterpret_cast<TO*>(a.U));
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  // L = L_y L_b: FP64 in the FP64 mode; FP32 accumulation over the k terms in
  // the others, whose L is FP32: that rounding (about sqrt(k) units of 2^-24
  // per entry) keeps ||L U - P A Q|| / ||A|| within the FP32 bar (dense FP32
  // 8192^2: 4.5e-6 against 3.3e-6 with a float-float product)
  int rc;
  if constexpr (std::is_same<T, df32>::value && std::is_same<TO, float>::value) {
    if (tc_digits) {
      rc = launch_l_tc(*a.ltc, reinterpret_cast<const df32*>(a.Lk), a.perm_y, Bp, a.perm_b, n,
                       reinterpret_cast<float*>(a.L), a.status, st);
      if (rc) return rc;
      RLU_CUDA_TRY(cudaMemcpyAsync(a.p, a.perm_y, sizeof(int64_t) * m, cudaMemcpyDeviceToDevice, st));
      RLU_CUDA_TRY(cudaMemcpyAsync(a.q, a.perm_b, sizeof(int64_t) * n, cudaMemcpyDeviceToDevice, st));
      return RLU_OK;
    }
  }
  if (rows_kernel) {
    const size_t smem = (size_t)k * k * sizeof(float);
    auto kern = k <= 64 ? k_assemble_rows<T, TO, 2> : (k <= 128 ? k_assemble_rows<T, TO, 4> : k_assemble_rows<T, TO, 8>);
    if (int rc_ = allow_dynamic_smem((const void*)kern, smem)) return rc_;
    kern<<<(unsigned)a.num_sms, 512, smem, st>>>(m, k, reinterpret_cast<const T*>(a.Lk), a.perm_y, Lb,
                                                 reinterpret_cast<TO*>(a.L));
    RLU_CUDA_TRY(cudaGetLastError());
    note_launch();
    rc = RLU_OK;
  } else if (a.fp32_product && !std::is_same<T, double>::value)
    rc = gemm_simt<T, T, TO, float>(st, m, k, k, LyP, k, 1, Lb, k, 1, reinterpret_cast<TO*>(a.L), k, 1);
  else
    rc = gemm_simt<T, T, TO, T>(st, m, k, k, LyP, k, 1, Lb, k, 1, reinterpret_cast<TO*>(a.L), k, 1);
  if (rc) return rc;
  RLU_CUDA_TRY(cudaMemcpyAsync(a.p, a.perm_y, sizeof(int64_t) * m, cudaMemcpyDeviceToDevice, st));
  RLU_CUDA_TRY(cudaMemcpyAsync(a.q, a.perm_b, sizeof(int64_t) * n, cudaMemcpyDeviceToDevice, st));
  return RLU_OK;
}

template int launch_assemble<double, double>(const AssembleArgs&, cudaStream_t);
template int launch_assemble<df32, float>(const AssembleArgs&, cudaStream_t);

// ---------------------------------------------------------------------------
// B = W A (first version: SIMT, FP32 or FP64 accumulate)
// ---------------------------------------------------------------------------
int bgemm_simt_splits(int64_t m, int64_t n, int k, int num_sms) {
  // enough slices of the m-long contraction for two CTAs per SM, each at least
  // 64 rows deep
  const int64_t tiles = cdiv(k, 64) * cdiv(n, 64);
  int64_t S = cdiv(2 * (int64_t)num_sms, tiles);
  S = min64(S, max64(1, m / 64));
  return (int)max64(1, S);
}

int launch_bgemm_simt(const void* W, int w64, const void* A, int64_t lda, int dtype, int64_t m, int64_t n, int k,
                      void* B, double* part, int num_sms, cudaStream_t st) {
  if (w64) {
    if (dtype != RLU_F64) return RLU_EINVAL;
    // small k x n: split the m-long contraction (partials summed in fixed order)
    const int S = part ? bgemm_simt_splits(m, n, k, num_sms) : 1;
    if (S > 1) {
      int rc = gemm_simt<double, double, double, double>(st, k, n, m, (const double*)W, m, 1, (const double*)A, lda,
                                                         1, part, n, 1, S, (int64_t)k * n);
      if (rc) return rc;
      k_sum_slices<double><<<(unsigned)cdiv((int64_t)k * n, 256), 256, 0, st>>>((int64_t)k * n, S, part,
                                                                                (double*)B);
      RLU_CUDA_TRY(cudaGetLastError());
      note_launch();
      return RLU_OK;
    }
    return gemm_simt<double, double, double, double>(st, k, n, m, (const double*)W, m, 1, (const double*)A, lda, 1,
                                                     (double*)B, n, 1);
  }
  if (dtype == RLU_F32)
    return gemm_chunked<float, float>(st, k, n, m, (const float*)W, m, (const float*)A, lda, (df32*)B, n);
  if (dtype == RLU_BF16)
    return gemm_chunked<float, __nv_bfloat16>(st, k, n, m, (const float*)W, m, (const __nv_bfloat16*)A, lda,
                                              (df32*)B, n);
  return RLU_EINVAL;
}

}  // namespace rlu
