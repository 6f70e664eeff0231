// CSR input: row classification, and B = W A for sparse A (step 6 of
// Algorithm 1; the sketch of CSR rows is in sketch.cu).
//
// Rows with at least n/4 entries ("heavy") are densified by the sketch and
// multiply W through the dense tensor-core path; the remaining ("light")
// entries are transposed to CSC with each column's entries sorted by row, so
// that every B[:, j] is a fixed-order sum  sum_(i, v) v * W[:, i]  read from
// W^T rows.  All orders are fixed: results repeat bit for bit.
#include <type_traits>

#include "bgemm.cuh"
#include "common.cuh"
#include "csr.cuh"
#include "pinv.cuh"
#include "sketch.cuh"

namespace rlu {

// Row classes: heavy (>= n/4 entries: densified, dense kernels), light (the
// rest: the sparse product for B), and among the light rows the "mid" ones
// with more than direct_max entries, whose sketch goes through the FFT kernel
// (the others are evaluated directly; direct_max < 0: every light row is mid).
__global__ void k_csr_classify(int64_t m, int64_t n, int64_t nnz, int64_t direct_max,
                               const int64_t* __restrict__ rowptr, int32_t* __restrict__ hflag,
                               int32_t* __restrict__ lflag, int32_t* __restrict__ mflag, unsigned int* status) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int64_t s = rowptr[i], e = rowptr[i + 1];
  bool bad = s < 0 || e < s || e > nnz;
  if (i == 0 && s != 0) bad = true;
  if (i == m - 1 && e != nnz) bad = true;
  if (bad) set_flag(status, FLAG_BAD_CSR);
  const bool heavy = !bad && (e - s) > 0 && 4 * (e - s) >= n;
  const bool light = !bad && !heavy;  // rows with a bad range are skipped (their Y rows stay zero)
  hflag[i] = heavy ? 1 : 0;
  lflag[i] = light ? 1 : 0;
  mflag[i] = (light && (e - s) > direct_max) ? 1 : 0;
}

__global__ void k_csr_lists(int64_t m, const int32_t* __restrict__ hflag, const int32_t* __restrict__ lflag,
                            const int32_t* __restrict__ mflag, const int32_t* __restrict__ hpos,
                            const int32_t* __restrict__ lpos, const int32_t* __restrict__ mpos,
                            const int32_t* __restrict__ loff, int32_t* __restrict__ heavy,
                            int32_t* __restrict__ light, int32_t* __restrict__ mid, int32_t* count) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < m) {
    if (hflag[i]) heavy[hpos[i]] = (int32_t)i;
    if (lflag[i]) light[lpos[i]] = (int32_t)i;
    if (mflag[i]) mid[mpos[i]] = (int32_t)i;
  }
  if (i == 0) {
    count[0] = lpos[m];
    count[1] = hpos[m];
    count[2] = mpos[m];
    count[3] = loff[m];  // light entries
  }
}

// ---- CSC of the light entries ------------------------------------------------
__global__ void k_csc_count(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colind, int64_t n,
                            const int32_t* __restrict__ light, int64_t nlight, int32_t* __restrict__ ccnt) {
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  for (int64_t r = gw; r < nlight; r += nw) {
    const int row = light[r];
    for (int64_t e = rowptr[row] + lane; e < rowptr[row + 1]; e += 32) {
      const int c = colind[e];
      if (c >= 0 && (int64_t)c < n) atomicAdd(&ccnt[c], 1);
    }
  }
}

// ---- light entries sorted by column (stable): CSC with rows ascending ----------
// The light entries are laid out flat in row order (rows ascending, each row's
// entries in CSR order), then sorted by column with a stable least-significant-
// digit radix sort (8-bit digits): per chunk of entries a histogram of the
// digit, an exclusive scan over (digit, chunk), and a scatter in which every
// entry lands after all earlier entries of its digit.  Stability keeps each
// column's entries in row order, so the column sums of the sparse product run
// in a fixed order without a sort by row.

// lens[i] = number of entries of row i if it is light, else 0
__global__ void k_light_lens(int64_t m, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ lflag,
                             int32_t* __restrict__ lens) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < m) lens[i] = lflag[i] ? (int32_t)(rowptr[i + 1] - rowptr[i]) : 0;
}

// Flat arrays of the light entries: a warp per light row, at offset loff[row].
// A column index outside [0, n) becomes n (sorted past every column, never read).
template <typename TV>
__global__ void k_light_expand(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                               const TV* __restrict__ val, int64_t n, const int32_t* __restrict__ light,
                               const int32_t* __restrict__ count, const int32_t* __restrict__ loff,
                               int32_t* __restrict__ key, int32_t* __restrict__ row, TV* __restrict__ v) {
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t nlight = count[0];
  for (int64_t r = gw; r < nlight; r += nw) {
    const int rw = light[r];
    const int64_t s = rowptr[rw], len = rowptr[rw + 1] - s, o = loff[rw];
    for (int64_t t = lane; t < len; t += 32) {
      const int c = colind[s + t];
      key[o + t] = (c >= 0 && (int64_t)c < n) ? c : (int32_t)n;
      row[o + t] = rw;
      v[o + t] = val[s + t];
    }
  }
}

constexpr int kRadixThreads = 256;
// chunk b holds entries [b * 256 * it, (b + 1) * 256 * it); hist[d * nchunks + b]
__global__ void __launch_bounds__(kRadixThreads) k_radix_hist(int64_t N, int it, int shift, int64_t nchunks,
                                                               const int32_t* __restrict__ key,
                                                               int32_t* __restrict__ hist) {
  __shared__ int cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRadixThreads * it;
  for (int r = 0; r < it; ++r) {
    const int64_t e = base + (int64_t)r * kRadixThreads + threadIdx.x;
    if (e < N) atomicAdd(&cnt[(key[e] >> shift) & 255], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nchunks + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: in each round of 256 entries, an entry's place is the
// running count of its digit (earlier rounds), plus the counts of its digit in
// the earlier warps of the round, plus its rank among the earlier lanes of its
// warp with the same digit.
template <typename TV>
__global__ void __launch_bounds__(kRadixThreads) k_radix_scatter(
    int64_t N, int it, int shift, int64_t nchunks, const int32_t* __restrict__ offs, const int32_t* __restrict__ kin,
    const int32_t* __restrict__ rin, const TV* __restrict__ vin, int32_t* __restrict__ kout, int32_t* __restrict__ rout,
    TV* __restrict__ vout) {
  constexpr int NW = kRadixThreads / 32;
  __shared__ int run[256];
  __shared__ int wc[NW][256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  run[tid] = offs[(int64_t)tid * nchunks + blockIdx.x];
  for (int w = 0; w < NW; ++w) wc[w][tid] = 0;
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
  const int64_t base = (int64_t)blockIdx.x * kRadixThreads * it;
  // the keys of the first kPre rounds are loaded before the rounds start (the
  // rounds are separated by block barriers, so a load issued inside a round
  // waits out its full latency)
  constexpr int kPre = 8;
  int kpre[kPre], rpre[kPre];
  TV vpre[kPre];
#pragma unroll
  for (int r = 0; r < kPre; ++r) {
    const int64_t e = base + (int64_t)r * kRadixThreads + tid;
    const bool ok = r < it && e < N;
    kpre[r] = ok ? kin[e] : 0;
    rpre[r] = ok ? rin[e] : 0;
    vpre[r] = ok ? vin[e] : TV(0);
  }
  for (int r = 0; r < it; ++r) {
    const int64_t e = base + (int64_t)r * kRadixThreads + tid;
    const bool valid = e < N;
    int kv = 0, rv = 0;
    TV vv = TV(0);
#pragma unroll
    for (int q = 0; q < kPre; ++q)
      if (q == r) {
        kv = kpre[q];
        rv = rpre[q];
        vv = vpre[q];
      }
    if (r >= kPre && valid) {
      kv = kin[e];
      rv = rin[e];
      vv = vin[e];
    }
    const int d = valid ? ((kv >> shift) & 255) : 256 + lane;  // lanes without an entry never match
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & lt);
    if (valid && rank == 0) wc[warp][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      int dest = run[d] + rank;
      for (int w = 0; w < warp; ++w) dest += wc[w][d];
      kout[dest] = kv;
      rout[dest] = rv;
      vout[dest] = vv;
    }
    __syncthreads();
    int tot = 0;
    for (int w = 0; w < NW; ++w) {
      tot += wc[w][tid];
      wc[w][tid] = 0;
    }
    run[tid] += tot;
    __syncthreads();
  }
}

// W^T (m x k) from W (k x m), 32 x 32 tiles through shared memory.
template <typename TW>
__global__ void k_transpose(int64_t k, int64_t m, const TW* __restrict__ W, TW* __restrict__ Wt) {
  __shared__ TW t[32][33];
  const int64_t c0 = (int64_t)blockIdx.y * 32, i0 = (int64_t)blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t c = c0 + r, i = i0 + threadIdx.x;
    if (c < k && i < m) t[r][threadIdx.x] = W[c * m + i];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t i = i0 + r, c = c0 + threadIdx.x;
    if (c < k && i < m) Wt[i * k + c] = t[threadIdx.x][r];
  }
}

// W_h[c][r] = W[c][heavy[r]]
template <typename TW>
__global__ void k_gather_cols(int64_t k, int64_t m, int64_t nh, const TW* __restrict__ W,
                              const int32_t* __restrict__ heavy, TW* __restrict__ Wh) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= k * nh) return;
  const int64_t c = e / nh, r = e - c * nh;
  Wh[e] = W[c * m + heavy[r]];
}

// B[:, j] += sum over the light entries (i, v) of column j of v * W^T[i, :]
// (warp per column; lane handles rows c = lane + 32 t of B).
template <typename TV, typename TW, typename TB, int KPL>
__global__ void __launch_bounds__(256) k_spmm_csc(int64_t n, int k, const int32_t* __restrict__ cstart,
                                                  const int32_t* __restrict__ crow, const TV* __restrict__ cval,
                                                  const TW* __restrict__ Wt, TB* __restrict__ B) {
  using TACC = typename std::conditional<sizeof(TV) == 8, double, float>::type;
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = gw; j < n; j += nw) {
    TACC acc[KPL];
#pragma unroll
    for (int t = 0; t < KPL; ++t) acc[t] = TACC(0);
    const int a = cstart[j], b = cstart[j + 1];
    for (int e = a; e < b; ++e) {
      const int64_t i = crow[e];
      const TACC v = (TACC)cval[e];
      const TW* w = Wt + i * k;
#pragma unroll
      for (int t = 0; t < KPL; ++t) {
        const int c = lane + 32 * t;
        if (c < k) acc[t] += v * (TACC)w[c];
      }
    }
#pragma unroll
    for (int t = 0; t < KPL; ++t) {
      const int c = lane + 32 * t;
      if (c < k) {
        TB& o = B[(int64_t)c * n + j];
        if constexpr (std::is_same<TB, double>::value) o = o + (double)acc[t];
        else o = o + df_make((float)acc[t], 0.f);
      }
    }
  }
}

// ---- host side -----------------------------------------------------------------
int csr_classify(CsrWs& w, const int64_t* rowptr, int64_t m, int64_t n, int64_t nnz, int64_t direct_max,
                 unsigned int* status, CsrRows& cr, int32_t* cnt, cudaStream_t st) {
  const unsigned g = (unsigned)cdiv(m, 256);
  k_csr_classify<<<g, 256, 0, st>>>(m, n, nnz, direct_max, rowptr, w.hflag, w.lflag, w.mflag, status);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  int rc;
  if ((rc = launch_scan_i32(m, w.hflag, w.hpos, w.scan_tmp, st))) return rc;
  if ((rc = launch_scan_i32(m, w.lflag, w.lpos, w.scan_tmp, st))) return rc;
  if ((rc = launch_scan_i32(m, w.mflag, w.mpos, w.scan_tmp, st))) return rc;
  k_light_lens<<<g, 256, 0, st>>>(m, rowptr, w.lflag, w.llen);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  if ((rc = launch_scan_i32(m, w.llen, w.loff, w.scan_tmp, st))) return rc;
  k_csr_lists<<<g, 256, 0, st>>>(m, w.hflag, w.lflag, w.mflag, w.hpos, w.lpos, w.mpos, w.loff, w.heavy, w.light,
                                 w.mid, w.count);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  RLU_CUDA_TRY(cudaMemcpyAsync(cnt, w.count, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  RLU_CUDA_TRY(cudaStreamSynchronize(st));
  cr.light = w.light;
  cr.heavy = w.heavy;
  cr.mid = w.mid;
  cr.d_count = w.count;
  cr.n_light = cnt[0];
  cr.n_heavy = cnt[1];
  cr.n_mid = cnt[2];
  cr.n_light_nnz = cnt[3];
  cr.direct_max = direct_max;
  return RLU_OK;
}

template <typename TV, typename TW, typename TB>
static int spmm_light_cfg(const CsrWs& w, const int32_t* crow, const void* cval_, int64_t n, int k, const TW* Wt,
                          TB* B, int num_sms, cudaStream_t st) {
  const unsigned grid = (unsigned)min64(cdiv(n * 32, 256), (int64_t)num_sms * 8);
  const TV* cval = reinterpret_cast<const TV*>(cval_);
#define RLU_SPMM(K)                                                                                     \
  k_spmm_csc<TV, TW, TB, K><<<grid, 256, 0, st>>>(n, k, w.cstart, crow, cval, Wt, B);
  if (k <= 32) RLU_SPMM(1)
  else if (k <= 64) RLU_SPMM(2)
  else if (k <= 128) RLU_SPMM(4)
  else if (k <= 256) RLU_SPMM(8)
  else if (k <= 512) RLU_SPMM(16)
  else RLU_SPMM(32)
#undef RLU_SPMM
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  return RLU_OK;
}

template <typename TV>
static int light_part(const CsrWs& w, const int64_t* rowptr, const int32_t* colind, const TV* val, int64_t m,
                      int64_t n, int k, const CsrRows& cr, const void* W, void* Wt, void* B, bool f64, int num_sms,
                      cudaStream_t st) {
  if (cr.n_light == 0) return RLU_OK;
  const unsigned gr = (unsigned)min64(cdiv(cr.n_light * 32, 256), (int64_t)num_sms * 8);
  RLU_CUDA_TRY(cudaMemsetAsync(w.ccnt, 0, sizeof(int32_t) * (n + 1), st));
  k_csc_count<<<gr, 256, 0, st>>>(rowptr, colind, n, cr.light, cr.n_light, w.ccnt);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  int rc;
  if ((rc = launch_scan_i32(n, w.ccnt, w.cstart, w.scan_tmp, st))) return rc;
  // the light entries, flat in row order, then sorted by column (stable)
  const int64_t N = cr.n_light_nnz;
  int32_t* key[2] = {w.ekey[0], w.ekey[1]};
  int32_t* row[2] = {w.erow[0], w.erow[1]};
  TV* vv[2] = {reinterpret_cast<TV*>(w.eval[0]), reinterpret_cast<TV*>(w.eval[1])};
  k_light_expand<TV><<<gr, 256, 0, st>>>(rowptr, colind, val, n, cr.light, cr.d_count, w.loff, key[0], row[0],
                                         vv[0]);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  int cur = 0;
  if (N > 0) {
    const int it = (int)max64(8, cdiv(cdiv(N, kRadixThreads), kRadixMaxChunks));
    const int64_t nchunks = cdiv(N, (int64_t)kRadixThreads * it);
    int bits = 1;
    while (((int64_t)1 << bits) <= n) ++bits;  // keys run up to n
    for (int shift = 0; shift < bits; shift += 8) {
      k_radix_hist<<<(unsigned)nchunks, kRadixThreads, 0, st>>>(N, it, shift, nchunks, key[cur], w.rhist);
      RLU_CUDA_TRY(cudaGetLastError());
      note_launch();
      if ((rc = launch_scan_i32(256 * nchunks, w.rhist, w.roffs, w.scan_tmp, st))) return rc;
      k_radix_scatter<TV><<<(unsigned)nchunks, kRadixThreads, 0, st>>>(N, it, shift, nchunks, w.roffs, key[cur],
                                                                       row[cur], vv[cur], key[cur ^ 1],
                                                                       row[cur ^ 1], vv[cur ^ 1]);
      RLU_CUDA_TRY(cudaGetLastError());
      note_launch();
      cur ^= 1;
    }
  }
  const int32_t* crow = row[cur];
  const void* cval = vv[cur];
  dim3 tg((unsigned)cdiv(m, 32), (unsigned)cdiv(k, 32));
  if (f64) {
    k_transpose<double><<<tg, dim3(32, 8), 0, st>>>(k, m, (const double*)W, (double*)Wt);
    RLU_CUDA_TRY(cudaGetLastError());
    note_launch();
    return spmm_light_cfg<TV, double, double>(w, crow, cval, n, k, (const double*)Wt, (double*)B, num_sms, st);
  }
  k_transpose<float><<<tg, dim3(32, 8), 0, st>>>(k, m, (const float*)W, (float*)Wt);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  return spmm_light_cfg<TV, float, df32>(w, crow, cval, n, k, (const float*)Wt, (df32*)B, num_sms, st);
}

int csr_bgemm(CsrWs& w, const int64_t* rowptr, const int32_t* colind, const void* val, int dtype, int prec,
              int64_t m, int64_t n, int k, const CsrRows& cr, const void* W, void* B, unsigned int* status,
              int num_sms, cudaStream_t st) {
  const bool f64 = (dtype == RLU_F64);
  const size_t bsz = (size_t)k * n * 8;  // double or float-float
  int rc;
  // heavy rows: dense product W_h D
  if (cr.n_heavy > 0) {
    const int64_t nh = cr.n_heavy;
    const unsigned g = (unsigned)cdiv((int64_t)k * nh, 256);
    if (f64) {
      k_gather_cols<double><<<g, 256, 0, st>>>(k, m, nh, (const double*)W, cr.heavy, (double*)w.Wh);
      RLU_CUDA_TRY(cudaGetLastError());
      note_launch();
      rc = launch_bgemm_simt(w.Wh, 1, w.D, n, RLU_F64, nh, n, k, B, nullptr, num_sms, st);
    } else {
      k_gather_cols<float><<<g, 256, 0, st>>>(k, m, nh, (const float*)W, cr.heavy, (float*)w.Wh);
      RLU_CUDA_TRY(cudaGetLastError());
      note_launch();
      if (w.tc.ready)
        rc = launch_bgemm_tc(w.tc, (const float*)w.Wh, w.D, n, RLU_F32, prec, nh, n, k, (df32*)B, status, st);
      else
        rc = launch_bgemm_simt(w.Wh, 0, w.D, n, RLU_F32, nh, n, k, B, nullptr, num_sms, st);
    }
    if (rc) return rc;
  } else {
    RLU_CUDA_TRY(cudaMemsetAsync(B, 0, bsz, st));
  }
  // light entries
  if (f64)
    return light_part<double>(w, rowptr, colind, (const double*)val, m, n, k, cr, W, w.Wt, B, true, num_sms, st);
  return light_part<float>(w, rowptr, colind, (const float*)val, m, n, k, cr, W, w.Wt, B, false, num_sms, st);
}

}  // namespace rlu
