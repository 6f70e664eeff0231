// Partial-pivoted LU of a tall matrix X (rows >= cols), `steps` elimination
// steps, in one persistent cooperative kernel.  Used twice:
//   * step 3 of Algorithm 1: P Y = L_Y U_Y on the m x l sketch (FP64), and
//   * step 6: the LU of B with right (column) pivoting, run as partial
//     pivoting on B^T (rows = columns of B) through strides.
//
// Semantics follow LAPACK getf2: at step j the pivot is the row with the
// largest |X[., j]| among the rows not yet pivoted, ties going to the row
// with the smallest current position (positions change by the getf2 swap
// of position j with the pivot's position); a nonzero pivot scales the
// column below it by its reciprocal; the rank-1 update runs on the trailing
// block.  An exactly zero pivot skips the scaling and raises FLAG_ZERO_PIVOT.
//
// Rows are never moved.  Each CTA owns a contiguous slab of rows (kept in
// shared memory when it fits) and tracks their current positions; every CTA
// keeps an identical copy of the occupants of positions 0..steps-1, so the
// whole permutation follows from one broadcast pivot per step.  One grid
// barrier per step: before it each CTA publishes its best candidate and that
// row's trailing values; after it every CTA picks the same winner.
#include "common.cuh"
#include "pivlu.cuh"

namespace rlu {

struct __align__(16) Cand {
  unsigned long long key;  // order-preserving bits of |pivot candidate|; 0 if the CTA has no candidate
  int pos;                 // current position of the candidate row
  int row;                 // original row index, -1 if none
};

// |x| as an unsigned key whose integer order is the numeric order of |x|
// (IEEE bit patterns of non-negative numbers sort as integers), so the pivot
// search needs no floating-point compares.  Any finite |x| maps above the
// "no candidate" key 0 except +0, which maps to 1.
__device__ __forceinline__ unsigned long long mag_key(double x) {
  return (unsigned long long)(__double_as_longlong(x) & 0x7fffffffffffffffll) + 1ull;
}
__device__ __forceinline__ unsigned long long mag_key(float x) {
  return ((unsigned long long)(__float_as_uint(x) & 0x7fffffffu) << 32) + 1ull;
}
__device__ __forceinline__ unsigned long long mag_key(df32 x) {
  // |x| = |hi| + lo * sign(hi): order by |hi|, then by the signed low part
  const unsigned int h = __float_as_uint(x.hi) & 0x7fffffffu;
  const float l = (x.hi < 0.f) ? -x.lo : x.lo;
  unsigned int lb = __float_as_uint(l);
  lb = (lb & 0x80000000u) ? ~lb : (lb | 0x80000000u);  // order-preserving map of a signed float
  return (((unsigned long long)h << 32) | lb) + 1ull;
}

__device__ __forceinline__ bool cand_better(unsigned long long ka, int pa, unsigned long long kb, int pb) {
  return ka > kb || (ka == kb && pa < pb);
}

template <typename T> __device__ __forceinline__ T recip(T x) { return one_<T>() / x; }

template <typename T>
__device__ __forceinline__ T& xref(T* X, int64_t rs, int64_t cs, int64_t i, int c) {
  return X[i * rs + (int64_t)c * cs];
}

template <typename T, bool SMEM, int NT>
__global__ void __launch_bounds__(NT) k_pivoted_lu(T* __restrict__ X, int64_t rows, int cols, int64_t rs,
                                                   int64_t cs, int steps, int64_t rpc, int32_t* __restrict__ pos_out,
                                                   int32_t* __restrict__ pstep_out, int64_t* __restrict__ perm_out,
                                                   Cand* __restrict__ cand, T* __restrict__ candrow,
                                                   unsigned int* bar, unsigned int* status) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int NW = NT / 32;
  const int G = gridDim.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * rpc;
  const int nr = (int)max((int64_t)0, min(rpc, rows - r0));
  const int rp = (int)rpc;
  // shared layout
  T* slab = reinterpret_cast<T*>(smem);                               // nr x cols (SMEM variant)
  T* urow = slab + (SMEM ? (size_t)rp * cols : 0);                    // cols
  T* lval = urow + cols;                                              // rpc
  int32_t* lpos = reinterpret_cast<int32_t*>(lval + rp);              // rpc
  int32_t* lstep = lpos + rp;                                         // rpc
  int32_t* pwin = lstep + rp;                                         // steps
  __shared__ unsigned long long red_v[NW];
  __shared__ int red_p[NW];
  __shared__ int red_r[NW];
  __shared__ int s_zero, s_cand;
  __shared__ int s_wrow, s_wpos, s_wcta;

  const bool row_fast = (cs == 1) ? false : true;  // B^T: consecutive rows are contiguous in memory
  auto at = [&](int r, int c) -> T& {
    if (SMEM) return slab[(size_t)r * cols + c];
    return xref(X, rs, cs, r0 + r, c);
  };

  // load slab, init bookkeeping
  if (SMEM) {
    if (row_fast) {
      for (int c = warp; c < cols; c += NW)
        for (int r = lane; r < nr; r += 32) slab[(size_t)r * cols + c] = xref(X, rs, cs, r0 + r, c);
    } else {
      for (int r = warp; r < nr; r += NW)
        for (int c = lane; c < cols; c += 32) slab[(size_t)r * cols + c] = xref(X, rs, cs, r0 + r, c);
    }
  }
  for (int r = tid; r < rp; r += NT) {
    lpos[r] = (int32_t)(r0 + r);
    lstep[r] = -1;
  }
  for (int t = tid; t < steps; t += NT) pwin[t] = t;
  __syncthreads();

  // Publish this CTA's best candidate for column jc (rows not yet pivoted):
  // its |value|, current position and row, and the row's values jc..cols-1.
  auto publish = [&](int jc) {
    unsigned long long bv = 0ull;
    int bp = 0x7fffffff, br = -1;
    for (int r = tid; r < nr; r += NT) {
      if (lstep[r] < 0) {
        const unsigned long long v = mag_key(at(r, jc));
        const int p = lpos[r];
        if (cand_better(v, p, bv, bp)) { bv = v; bp = p; br = r; }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long ov = __shfl_down_sync(0xffffffffu, bv, o);
      int op = __shfl_down_sync(0xffffffffu, bp, o);
      int orr = __shfl_down_sync(0xffffffffu, br, o);
      if (cand_better(ov, op, bv, bp)) { bv = ov; bp = op; br = orr; }
    }
    if (lane == 0) { red_v[warp] = bv; red_p[warp] = bp; red_r[warp] = br; }
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < NW; ++w)
        if (cand_better(red_v[w], red_p[w], bv, bp)) { bv = red_v[w]; bp = red_p[w]; br = red_r[w]; }
      s_cand = br;
    }
    __syncthreads();
    return s_cand;  // local row, or -1
  };
  auto write_cand = [&](int jc, int lr) {
    if (tid == 0) {
      Cand cd;
      cd.key = lr >= 0 ? mag_key(at(lr, jc)) : 0ull;
      cd.pos = lr >= 0 ? lpos[lr] : 0x7fffffff;
      cd.row = lr < 0 ? -1 : (int)(r0 + lr);
      cand[(jc & 1) * G + blockIdx.x] = cd;
    }
    T* dst = candrow + ((size_t)(jc & 1) * G + blockIdx.x) * cols;
    if (lr >= 0)
      for (int c = jc + tid; c < cols; c += NT) dst[c - jc] = at(lr, c);
  };

  // step 0 candidate
  {
    const int lr = publish(0);
    write_cand(0, lr);
    grid_arrive(bar);
  }
  for (int j = 0; j < steps; ++j) {
    // 1. wait for every CTA's candidate of step j
    if (!grid_wait(bar, (unsigned)(j + 1), status)) return;
    // 2. every CTA picks the same winner (warp 0 scans the G candidates)
    if (warp == 0) {
      unsigned long long bv = 0ull;
      int bp = 0x7fffffff, bc = -1, bw = -1;
      for (int g = lane; g < G; g += 32) {
        const Cand cd = cand[(j & 1) * G + g];
        if (cd.row >= 0 && cand_better(cd.key, cd.pos, bv, bp)) { bv = cd.key; bp = cd.pos; bc = g; bw = cd.row; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        unsigned long long ov = __shfl_down_sync(0xffffffffu, bv, o);
        int op = __shfl_down_sync(0xffffffffu, bp, o);
        int oc = __shfl_down_sync(0xffffffffu, bc, o);
        int ow = __shfl_down_sync(0xffffffffu, bw, o);
        if (cand_better(ov, op, bv, bp)) { bv = ov; bp = op; bc = oc; bw = ow; }
      }
      if (lane == 0) {
        s_wcta = bc;
        s_wpos = bp;
        s_wrow = bw;
      }
    }
    __syncthreads();
    const int wcta = s_wcta;
    if (wcta < 0) {  // no row left (cannot happen with steps <= rows)
      if (tid == 0) set_flag(status, FLAG_ZERO_PIVOT);
      break;
    }
    {
      const T* src = candrow + ((size_t)(j & 1) * G + wcta) * cols;
      for (int c = j + tid; c < cols; c += NT) urow[c - j] = src[c - j];
    }
    __syncthreads();
    if (tid == 0) {
      const int w = s_wrow, wpos = s_wpos;
      s_zero = (urow[0] == zero_<T>()) ? 1 : 0;
      if (s_zero && blockIdx.x == 0) set_flag(status, FLAG_ZERO_PIVOT);
      // getf2 swap of positions j and wpos
      const int occ = pwin[j];
      pwin[j] = w;
      if (wpos < steps) pwin[wpos] = occ;
      if (occ != w && occ >= r0 && occ < r0 + nr) lpos[occ - r0] = wpos;
      if (w >= r0 && w < r0 + nr) {
        lpos[w - r0] = j;
        lstep[w - r0] = j;
      }
    }
    __syncthreads();
    const bool zero = s_zero != 0;
    // 3. column j below the pivot: l = x / pivot; then column j+1 (look-ahead)
    if (!zero) {
      const T rpiv = recip(urow[0]);
      const T u1 = (j + 1 < cols) ? urow[1] : zero_<T>();
      for (int r = tid; r < nr; r += NT) {
        if (lstep[r] < 0) {
          T lv = at(r, j) * rpiv;
          at(r, j) = lv;
          lval[r] = lv;
          if (j + 1 < cols) {
            T& x = at(r, j + 1);
            x = mad(-lv, u1, x);
          }
        }
      }
    }
    __syncthreads();
    int rstar = -1;
    if (j + 1 < steps) {
      // 4. next candidate: its row is brought fully up to date before publishing
      rstar = publish(j + 1);
      if (!zero && rstar >= 0)
        for (int c = j + 2 + tid; c < cols; c += NT) {
          T& x = at(rstar, c);
          x = mad(-lval[rstar], urow[c - j], x);
        }
      __syncthreads();
      write_cand(j + 1, rstar);
      grid_arrive(bar);
    }
    // 5. the rest of the rank-1 update (columns j+2.., rows other than rstar)
    const int c0 = j + 2;
    if (!zero && c0 < cols) {
      if (SMEM) {
        for (int r = warp; r < nr; r += NW) {
          if (lstep[r] < 0 && r != rstar) {
            const T lv = -lval[r];
            for (int c = c0 + lane; c < cols; c += 32) {
              T& x = at(r, c);
              x = mad(lv, urow[c - j], x);
            }
          }
        }
      } else {
        // global memory: a flat loop over (row, column) with several independent
        // elements per thread in flight; the fast index follows the memory layout
        const int width = cols - c0;
        const int tot = nr * width;
        constexpr int U = 4;
        for (int base = tid; base < tot; base += NT * U) {
          T xv[U];
          int rr[U], cc[U];
          bool act[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int idx = base + u * NT;
            int r, c;
            if (row_fast) { r = idx % nr; c = idx / nr; } else { c = idx % width; r = idx / width; }
            rr[u] = r;
            cc[u] = c0 + c;
            act[u] = idx < tot && lstep[r < nr ? r : 0] < 0 && r != rstar;
            if (act[u]) xv[u] = at(r, c0 + c);
          }
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (act[u]) at(rr[u], cc[u]) = mad(-lval[rr[u]], urow[cc[u] - j], xv[u]);
        }
      }
    }
    __syncthreads();
  }

  // write back
  if (SMEM) {
    if (row_fast) {
      for (int c = warp; c < cols; c += NW)
        for (int r = lane; r < nr; r += 32) xref(X, rs, cs, r0 + r, c) = slab[(size_t)r * cols + c];
    } else {
      for (int r = warp; r < nr; r += NW)
        for (int c = lane; c < cols; c += 32) xref(X, rs, cs, r0 + r, c) = slab[(size_t)r * cols + c];
    }
  }
  for (int r = tid; r < nr; r += NT) {
    pos_out[r0 + r] = lpos[r];
    pstep_out[r0 + r] = lstep[r];
    perm_out[lpos[r]] = r0 + r;
  }
}

template <typename T, bool SMEM>
static size_t pivlu_smem(int64_t rpc, int cols, int steps) {
  size_t b = (SMEM ? (size_t)rpc * cols * sizeof(T) : 0) + (size_t)cols * sizeof(T) + (size_t)rpc * sizeof(T) +
             (size_t)rpc * 8 + (size_t)steps * 4;
  return (b + 15) & ~(size_t)15;
}

template <typename T, bool SMEM>
static int launch_cfg(T* X, int64_t rows, int cols, int64_t rs, int64_t cs, int steps, int G, PivLuWs& ws,
                      unsigned int* status, cudaStream_t st) {
  constexpr int NT = SMEM ? 256 : 1024;
  const int64_t rpc = cdiv(rows, G);
  size_t smem = pivlu_smem<T, SMEM>(rpc, cols, steps);
  auto kern = k_pivoted_lu<T, SMEM, NT>;
  if (int rc_ = allow_dynamic_smem((const void*)kern, smem)) return rc_;
  int per_sm = 0;
  RLU_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
  if (per_sm < 1) return RLU_EINVAL;
  RLU_CUDA_TRY(cudaMemsetAsync(ws.bar, 0, sizeof(unsigned int), st));
  Cand* cand = reinterpret_cast<Cand*>(ws.cand);
  T* candrow = reinterpret_cast<T*>(ws.candrow);
  void* args[] = {&X, &rows, &cols, &rs, &cs, &steps, (void*)&rpc, &ws.pos, &ws.pstep, &ws.perm,
                  &cand, &candrow, &ws.bar, &status};
  RLU_CUDA_TRY(launch_cooperative((void*)kern, G, NT, args, smem, st));
  note_launch();
  return RLU_OK;
}

size_t pivlu_cand_bytes(int max_ctas) { return (size_t)2 * max_ctas * sizeof(Cand); }

template <typename T>
int launch_pivoted_lu(T* X, int64_t rows, int cols, int64_t rs, int64_t cs, int steps, PivLuWs& ws,
                      unsigned int* status, int num_sms, cudaStream_t st) {
  if (steps > cols || steps > rows || cols > ws.max_cols) return RLU_EINVAL;
  // one CTA per SM, or fewer for small inputs (at least 8 rows per CTA)
  int G = (int)min64(num_sms, cdiv(rows, 8));
  if (G > ws.max_ctas) G = ws.max_ctas;
  const int64_t rpc = cdiv(rows, G);
  size_t smem = pivlu_smem<T, true>(rpc, cols, steps);
  if (smem <= 200 * 1024) return launch_cfg<T, true>(X, rows, cols, rs, cs, steps, G, ws, status, st);
  return launch_cfg<T, false>(X, rows, cols, rs, cs, steps, G, ws, status, st);
}

template int launch_pivoted_lu<double>(double*, int64_t, int, int64_t, int64_t, int, PivLuWs&, unsigned int*, int,
                                       cudaStream_t);
template int launch_pivoted_lu<float>(float*, int64_t, int, int64_t, int64_t, int, PivLuWs&, unsigned int*, int,
                                      cudaStream_t);
template int launch_pivoted_lu<df32>(df32*, int64_t, int, int64_t, int64_t, int, PivLuWs&, unsigned int*, int,
                                     cudaStream_t);

}  // namespace rlu
