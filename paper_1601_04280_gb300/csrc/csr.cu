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
                            int32_t* __restrict__ heavy, int32_t* __restrict__ light, int32_t* __restrict__ mid,
                            int32_t* count) {
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

template <typename TV>
__global__ void k_csc_fill(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                           const TV* __restrict__ val, int64_t n, const int32_t* __restrict__ light, int64_t nlight,
                           const int32_t* __restrict__ cstart, int32_t* __restrict__ ccur, int32_t* __restrict__ crow,
                           TV* __restrict__ cval) {
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  for (int64_t r = gw; r < nlight; r += nw) {
    const int row = light[r];
    for (int64_t e = rowptr[row] + lane; e < rowptr[row + 1]; e += 32) {
      const int c = colind[e];
      if (c >= 0 && (int64_t)c < n) {
        const int p = cstart[c] + atomicAdd(&ccur[c], 1);
        crow[p] = row;
        cval[p] = val[e];
      }
    }
  }
}

// Sort each column's (row, value) entries by row (then by value bits, so that
// duplicate coordinates also come out in a fixed order): a warp per column,
// bitonic sort through shared memory for up to kSortMax entries, insertion
// sort by one lane beyond that.
constexpr int kSortMax = 256;
template <typename TV>
__global__ void __launch_bounds__(256) k_csc_sort(int64_t n, const int32_t* __restrict__ cstart,
                                                  int32_t* __restrict__ crow, TV* __restrict__ cval) {
  __shared__ unsigned long long keys[8][kSortMax];
  __shared__ TV vals[8][kSortMax];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t gw = (int64_t)blockIdx.x * 8 + warp;
  const int64_t nw = (int64_t)gridDim.x * 8;
  auto key_of = [](int32_t r, TV v) -> unsigned long long {
    unsigned int vb;
    if constexpr (sizeof(TV) == 8) vb = (unsigned int)(__double_as_longlong((double)v) >> 32);
    else vb = __float_as_uint((float)v);
    return ((unsigned long long)(uint32_t)r << 32) | vb;
  };
  for (int64_t j = gw; j < n; j += nw) {
    const int a = cstart[j], b = cstart[j + 1], len = b - a;
    if (len <= 1) continue;
    if (len <= kSortMax) {
      int P = 1;
      while (P < len) P <<= 1;
      for (int t = lane; t < P; t += 32) {
        keys[warp][t] = t < len ? key_of(crow[a + t], cval[a + t]) : ~0ull;
        vals[warp][t] = t < len ? cval[a + t] : TV(0);
      }
      __syncwarp();
      for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
          for (int t = lane; t < P; t += 32) {
            const int partner = t ^ stride;
            if (partner > t) {
              const bool up = (t & size) == 0;
              const unsigned long long kt = keys[warp][t], kp = keys[warp][partner];
              if ((kt > kp) == up) {
                keys[warp][t] = kp;
                keys[warp][partner] = kt;
                const TV vt = vals[warp][t];
                vals[warp][t] = vals[warp][partner];
                vals[warp][partner] = vt;
              }
            }
          }
          __syncwarp();
        }
      }
      for (int t = lane; t < len; t += 32) {
        crow[a + t] = (int32_t)(keys[warp][t] >> 32);
        cval[a + t] = vals[warp][t];
      }
      __syncwarp();
    } else if (lane == 0) {
      for (int i = a + 1; i < b; ++i) {
        const int32_t r = crow[i];
        const TV v = cval[i];
        const unsigned long long kv = key_of(r, v);
        int t = i - 1;
        while (t >= a && key_of(crow[t], cval[t]) > kv) {
          crow[t + 1] = crow[t];
          cval[t + 1] = cval[t];
          --t;
        }
        crow[t + 1] = r;
        cval[t + 1] = v;
      }
    }
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
  k_csr_lists<<<g, 256, 0, st>>>(m, w.hflag, w.lflag, w.mflag, w.hpos, w.lpos, w.mpos, w.heavy, w.light, w.mid,
                                 w.count);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  RLU_CUDA_TRY(cudaMemcpyAsync(cnt, w.count, 3 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  RLU_CUDA_TRY(cudaStreamSynchronize(st));
  cr.light = w.light;
  cr.heavy = w.heavy;
  cr.mid = w.mid;
  cr.d_count = w.count;
  cr.n_light = cnt[0];
  cr.n_heavy = cnt[1];
  cr.n_mid = cnt[2];
  cr.direct_max = direct_max;
  return RLU_OK;
}

template <typename TV, typename TW, typename TB>
static int spmm_light_cfg(const CsrWs& w, int64_t n, int k, const TW* Wt, TB* B, int num_sms, cudaStream_t st) {
  const unsigned grid = (unsigned)min64(cdiv(n * 32, 256), (int64_t)num_sms * 8);
  const TV* cval = reinterpret_cast<const TV*>(w.cval);
#define RLU_SPMM(K)                                                                                     \
  k_spmm_csc<TV, TW, TB, K><<<grid, 256, 0, st>>>(n, k, w.cstart, w.crow, cval, Wt, B);
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
  RLU_CUDA_TRY(cudaMemsetAsync(w.ccnt, 0, sizeof(int32_t) * (n + 1), st));
  k_csc_fill<TV><<<gr, 256, 0, st>>>(rowptr, colind, val, n, cr.light, cr.n_light, w.cstart, w.ccnt, w.crow,
                                     reinterpret_cast<TV*>(w.cval));
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  k_csc_sort<TV><<<(unsigned)min64(cdiv(n, 8), (int64_t)num_sms * 4), 256, 0, st>>>(n, w.cstart, w.crow,
                                                                                   reinterpret_cast<TV*>(w.cval));
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  dim3 tg((unsigned)cdiv(m, 32), (unsigned)cdiv(k, 32));
  if (f64) {
    k_transpose<double><<<tg, dim3(32, 8), 0, st>>>(k, m, (const double*)W, (double*)Wt);
    RLU_CUDA_TRY(cudaGetLastError());
    note_launch();
    return spmm_light_cfg<TV, double, double>(w, n, k, (const double*)Wt, (double*)B, num_sms, st);
  }
  k_transpose<float><<<tg, dim3(32, 8), 0, st>>>(k, m, (const float*)W, (float*)Wt);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  return spmm_light_cfg<TV, float, df32>(w, n, k, (const float*)Wt, (df32*)B, num_sms, st);
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
