// Rank-revealing column order of the sketch (an option beyond Algorithm 1,
// whose panel LU takes Y's columns as they come): QR with column pivoting
// (Businger and Golub), computed as the greedy pivoted Cholesky of the Gram
// matrix Y^T Y, which makes the same choices in exact arithmetic: the
// diagonal of the Schur complement holds the squared norms of the columns'
// residuals after the columns already chosen.  Then Y := Y[:, order] and the
// panel LU of step 3 runs unchanged, so L_y spans the k most independent of
// the l sketch columns and the oversampling l - k enters the projection.
//
//   * G = Y^T Y: float-float accumulation of the FP64 sketch (SIMT), split
//     over the m rows, FP64 partials summed in FP64;
//   * the greedy elimination on G: one CTA, float-float Schur updates (about
//     48 bits: the choices match FP64 except on near-ties), rows and columns
//     of G swapped as in the textbook algorithm, ties to the first position;
//   * the column gather of Y through a scratch copy.
#include "colpiv.cuh"
#include "gemm_simt.cuh"

namespace rlu {

// One CTA of 1024 threads.  S (l x l, float-float, row-major) holds G on entry
// and is destroyed; order[0..l) receives the column order.
__global__ void __launch_bounds__(1024) k_greedy_order(int l, df32* __restrict__ S, int32_t* __restrict__ order) {
  __shared__ unsigned long long s_key[32];
  __shared__ int s_pos[32];
  __shared__ int s_win;
  __shared__ float s_rinv_hi, s_rinv_lo;
  __shared__ int s_stop;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int c = tid; c < l; c += blockDim.x) order[c] = c;
  if (tid == 0) s_stop = 0;
  __syncthreads();
  for (int j = 0; j < l; ++j) {
    // the largest remaining diagonal entry (first position on ties)
    unsigned long long bk = 0ull;
    int bp = 0x7fffffff;
    for (int c = j + tid; c < l; c += blockDim.x) {
      const df32 d = S[(int64_t)c * l + c];
      // order-preserving key of d as a non-negative value (negatives, from
      // rounding below zero, count as zero)
      const float h = d.hi > 0.f ? d.hi : 0.f;
      const float lo = d.hi > 0.f ? d.lo : 0.f;
      unsigned int lb = __float_as_uint(lo);
      lb = (lb & 0x80000000u) ? ~lb : (lb | 0x80000000u);
      const unsigned long long key = ((unsigned long long)__float_as_uint(h) << 32) | lb;
      if (key > bk || (key == bk && c < bp)) { bk = key; bp = c; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
      const int op = __shfl_xor_sync(0xffffffffu, bp, o);
      if (ok > bk || (ok == bk && op < bp)) { bk = ok; bp = op; }
    }
    if (lane == 0) { s_key[warp] = bk; s_pos[warp] = bp; }
    __syncthreads();
    if (tid == 0) {
      unsigned long long k0 = s_key[0];
      int p0 = s_pos[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        if (s_key[w] > k0 || (s_key[w] == k0 && s_pos[w] < p0)) { k0 = s_key[w]; p0 = s_pos[w]; }
      s_win = p0;
    }
    __syncthreads();
    const int c = s_win;
    // swap rows and columns j and c of S, and the order
    if (c != j && c < l) {
      for (int t = tid; t < l; t += blockDim.x) {
        const df32 a = S[(int64_t)j * l + t], b = S[(int64_t)c * l + t];
        S[(int64_t)j * l + t] = b;
        S[(int64_t)c * l + t] = a;
      }
      __syncthreads();
      for (int t = tid; t < l; t += blockDim.x) {
        const df32 a = S[(int64_t)t * l + j], b = S[(int64_t)t * l + c];
        S[(int64_t)t * l + j] = b;
        S[(int64_t)t * l + c] = a;
      }
      if (tid == 0) {
        const int o = order[j];
        order[j] = order[c];
        order[c] = o;
      }
      __syncthreads();
    }
    if (tid == 0) {
      const df32 piv = S[(int64_t)j * l + j];
      const double pv = (double)piv.hi + (double)piv.lo;
      if (!(pv > 0.0)) {
        s_stop = 1;  // the remaining columns lie in the span of the chosen ones
      } else {
        const df32 r = df_from_double(1.0 / sqrt(pv));
        s_rinv_hi = r.hi;
        s_rinv_lo = r.lo;
      }
    }
    __syncthreads();
    if (s_stop) break;
    const df32 rinv = df_make(s_rinv_hi, s_rinv_lo);
    // row j of the factor: r_t = S[j][t] / sqrt(S[j][j]), kept in row j
    for (int t = j + 1 + tid; t < l; t += blockDim.x) S[(int64_t)j * l + t] = S[(int64_t)j * l + t] * rinv;
    __syncthreads();
    // trailing update S[a][b] -= r_a r_b (a, b > j)
    const int w = l - j - 1;
    for (int64_t e = tid; e < (int64_t)w * w; e += blockDim.x) {
      const int a = j + 1 + (int)(e / w), b = j + 1 + (int)(e % w);
      S[(int64_t)a * l + b] = S[(int64_t)a * l + b] - S[(int64_t)j * l + a] * S[(int64_t)j * l + b];
    }
    __syncthreads();
  }
}

// Y (m x l, row-major) -> Yp[i][t] = Y[i][order[t]].
__global__ void k_gather_cols_f64(int64_t m, int l, const double* __restrict__ Y, const int32_t* __restrict__ order,
                                  double* __restrict__ Yp) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m * l) return;
  const int64_t i = e / l;
  const int t = (int)(e - i * l);
  Yp[e] = Y[i * l + order[t]];
}

__global__ void k_df_from_f64(int64_t count, const double* __restrict__ x, df32* __restrict__ y) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < count) y[e] = df_from_double(x[e]);
}

size_t colpiv_buffer_bytes(int64_t m, int l, int max_splits) {
  return sizeof(double) * ((size_t)max_splits * l * l + (size_t)l * l + (size_t)m * l) + sizeof(df32) * l * l +
         sizeof(int32_t) * l + 1024;
}

int launch_column_pivoting(double* Y, int64_t m, int l, void* buf, int max_splits, int num_sms, cudaStream_t st) {
  char* b = (char*)buf;
  double* part = (double*)b;
  b += sizeof(double) * (size_t)max_splits * l * l;
  double* G = (double*)b;
  b += sizeof(double) * (size_t)l * l;
  double* Ytmp = (double*)b;
  b += sizeof(double) * (size_t)m * l;
  df32* S = (df32*)b;
  b += sizeof(df32) * (size_t)l * l;
  int32_t* order = (int32_t*)b;
  // G = Y^T Y, split over the rows so that about two CTAs per SM run
  const int64_t tiles = cdiv(l, 64) * cdiv(l, 64);
  int S_ = (int)min64(max_splits, max64(1, cdiv(2 * (int64_t)num_sms, tiles)));
  S_ = (int)min64(S_, max64(1, cdiv(m, 64)));
  const int64_t kps = cdiv(cdiv(m, S_), 16) * 16;
  S_ = (int)cdiv(m, kps);
  int rc = gemm_simt<double, double, double, df32>(st, l, l, m, Y, 1, l, Y, l, 1, part, l, 1, S_, (int64_t)l * l);
  if (rc) return rc;
  k_sum_slices<double><<<(unsigned)cdiv((int64_t)l * l, 256), 256, 0, st>>>((int64_t)l * l, S_, part, G);
  k_df_from_f64<<<(unsigned)cdiv((int64_t)l * l, 256), 256, 0, st>>>((int64_t)l * l, G, S);
  k_greedy_order<<<1, 1024, 0, st>>>(l, S, order);
  RLU_CUDA_TRY(cudaMemcpyAsync(Ytmp, Y, sizeof(double) * (size_t)m * l, cudaMemcpyDeviceToDevice, st));
  k_gather_cols_f64<<<(unsigned)cdiv(m * l, 256), 256, 0, st>>>(m, l, Ytmp, order, Y);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch(4);
  return RLU_OK;
}

}  // namespace rlu
