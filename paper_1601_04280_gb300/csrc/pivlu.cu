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

// Lane holding the warp's best candidate (largest key, then smallest
// position) among the lanes with `valid`, or -1 if none: hardware max / min
// reductions on the two halves of the key and then on the position, in place
// of a shuffle tree (positions are distinct, so the winner is unique).
__device__ __forceinline__ int warp_best_lane(unsigned long long key, int pos, bool valid) {
  const unsigned int khi = valid ? (unsigned int)(key >> 32) : 0u;
  const unsigned int mhi = __reduce_max_sync(0xffffffffu, khi);
  const bool c1 = valid && khi == mhi;
  const unsigned int mlo = __reduce_max_sync(0xffffffffu, c1 ? (unsigned int)key : 0u);
  const bool c2 = c1 && (unsigned int)key == mlo;
  const unsigned int mp = __reduce_min_sync(0xffffffffu, c2 ? (unsigned int)pos : 0xffffffffu);
  const unsigned int ball = __ballot_sync(0xffffffffu, c2 && (unsigned int)pos == mp);
  return ball ? __ffs((int)ball) - 1 : -1;
}

template <typename T> __device__ __forceinline__ T recip(T x) { return one_<T>() / x; }
// FP64: Newton's reciprocal (a few dependent FMAs on the slow FP64 pipe instead
// of a full division), with the sign restored.
template <> __device__ __forceinline__ double recip<double>(double x) { return copysign(rcp_newton(fabs(x)), x); }

// Load through L2 only (values written by other CTAs in this launch).
template <typename T> __device__ __forceinline__ T ldcg_(const T* p) { return __ldcg(p); }
template <> __device__ __forceinline__ df32 ldcg_<df32>(const df32* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return df_make(v.x, v.y);
}

template <typename T>
__device__ __forceinline__ T& xref(T* X, int64_t rs, int64_t cs, int64_t i, int c) {
  return X[i * rs + (int64_t)c * cs];
}

template <typename T, bool SMEM, int NT>
__global__ void __launch_bounds__(NT) k_pivoted_lu(T* __restrict__ X, int64_t rows, int cols, int64_t rs,
                                                   int64_t cs, int steps, int64_t rpc, int32_t* __restrict__ pos_out,
                                                   int32_t* __restrict__ pstep_out, int64_t* __restrict__ perm_out,
                                                   Cand* __restrict__ cand, T* __restrict__ candrow,
                                                   unsigned int* bar, unsigned int* status, int defer, int j0,
                                                   int npos) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int NW = NT / 32;
  const int G = gridDim.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * rpc;
  const int nr = (int)max((int64_t)0, min(rpc, rows - r0));
  const int rp = (int)rpc;
  // shared layout
  // slab row stride: odd, so that lanes on different rows of one column
  // fall in different shared-memory banks
  const int sst = cols | 1;
  T* slab = reinterpret_cast<T*>(smem);                               // nr x sst (SMEM variant)
  // Pivot rows live in a ring of D + 1 slots (step t in slot t mod (D + 1)) and
  // the multipliers of the pending steps in D columns of lhist (step t in
  // column t mod D): the global-memory variant defers the trailing update and
  // applies D steps at once (D = 1 in shared memory: every step at once).
  const int D = SMEM ? 1 : defer;
  const int RU = D + 1;
  T* ring = slab + (SMEM ? (size_t)rp * sst : 0);                     // RU x cols
  T* lhist = ring + (size_t)RU * cols;                                // D x rpc
  int32_t* lpos = reinterpret_cast<int32_t*>(lhist + (size_t)D * rp); // rpc
  int32_t* lstep = lpos + rp;                                         // rpc
  int32_t* ldone = lstep + rp;                                        // rpc: last step applied to the whole row
  int32_t* pwin = ldone + rp;                                         // npos
  __shared__ unsigned long long red_v[NW];
  __shared__ int red_p[NW];
  __shared__ int red_r[NW];
  __shared__ int s_zero, s_stop, s_rstar;
  __shared__ unsigned long long s_ckey;
  __shared__ int s_cpos;
  __shared__ T s_rpiv;

  const bool row_fast = (cs == 1) ? false : true;  // B^T: consecutive rows are contiguous in memory
  auto at = [&](int r, int c) -> T& {
    if (SMEM) return slab[(size_t)r * sst + c];
    return xref(X, rs, cs, r0 + r, c);
  };

  // (row, column) of the e-th slab element in memory order (consecutive
  // lanes, consecutive addresses)
  auto slab_rc = [&](int e, int& r, int& c) {
    if (row_fast) {
      c = e / nr;
      r = e - c * nr;
    } else {
      r = e / cols;
      c = e - r * cols;
    }
  };
  // load slab (several loads in flight per thread), init bookkeeping
  if (SMEM) {
    const int tot = nr * cols;
    constexpr int U = 8;
    for (int base = tid; base < tot; base += NT * U) {
      T v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = base + u * NT;
        if (e < tot) {
          int r, c;
          slab_rc(e, r, c);
          v[u] = xref(X, rs, cs, r0 + r, c);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = base + u * NT;
        if (e < tot) {
          int r, c;
          slab_rc(e, r, c);
          slab[(size_t)r * sst + c] = v[u];
        }
      }
    }
  }
  // j0 > 0: a later panel of a blocked LU (steps j0 .. j0 + steps - 1 on the
  // columns passed here); positions, pivot steps and the occupants of
  // positions 0 .. npos - 1 come from the previous panel's launch
  for (int r = tid; r < rp; r += NT) {
    lpos[r] = (j0 > 0 && r < nr) ? pos_out[r0 + r] : (int32_t)(r0 + r);
    lstep[r] = (j0 > 0 && r < nr) ? pstep_out[r0 + r] : -1;
    ldone[r] = -1;
  }
  for (int t = tid; t < npos; t += NT) pwin[t] = j0 > 0 ? (int32_t)perm_out[t] : t;
  if (tid == 0) s_stop = 0;
  __syncthreads();

  // Warp 0 is the control warp: it waits for the grid's candidates of step j,
  // picks the winner, fetches the pivot row and keeps the permutation.  Warps
  // 1.. are the workers: they scale column j, bring column j+1 and the next
  // candidate row up to date, publish that candidate, and then apply the rest
  // of step j's rank-1 update while the control warp already waits for step
  // j+1.  Named barriers: 1 = pivot row of step j ready (control -> workers),
  // 2 = candidate of step j+1 ready (workers -> control), 3 = workers only.
  constexpr int NTW = NT - 32;
  constexpr int NWK = NW - 1;
  auto bar_sync = [](int id, int cnt) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(cnt) : "memory"); };
  auto bar_arrive = [](int id, int cnt) { asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(cnt) : "memory"); };

  if (warp == 0) {
    // ------------------------------------------------------------ control warp
    const Cand* cands = cand;
    for (int j = 0; j <= steps; ++j) {
      // publish the candidate for step j (prepared by the workers)
      if (j < steps) {
        bar_sync(2, NT);
        __syncwarp();
        if (lane == 0) {
          Cand cd;
          cd.key = s_ckey;
          cd.pos = s_cpos;
          cd.row = s_rstar < 0 ? -1 : (int)(r0 + s_rstar);
          if (s_rstar < 0) { cd.key = 0ull; cd.pos = 0x7fffffff; }
          cand[(j & 1) * G + blockIdx.x] = cd;
          // release (cumulative): this record and the workers' candidate row,
          // ordered before it by barrier 2, are visible to whoever acquires
          red_release_gpu_add(bar, 1u);
        }
      }
      if (j == steps) break;
      // wait for every CTA's candidate of step j (bounded)
      int ok = 1;
      if (lane == 0) {
        const unsigned int target = (unsigned)(j + 1) * (unsigned)G;
        const long long t0 = clock64();
        while (true) {
          const unsigned int v = ld_acquire_gpu(bar);
          if ((int)(v - target) >= 0) break;
          if (ld_acquire_gpu(status) & FLAG_TIMEOUT) { ok = 0; break; }
          if (clock64() - t0 > kSpinLimitCycles) { set_flag(status, FLAG_TIMEOUT); ok = 0; break; }
        }
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      __syncwarp();
      // the winner: every lane loads its share of the G records at once
      unsigned long long bv = 0ull;
      int bp = 0x7fffffff, bc = -1, bw = -1;
      if (ok) {
        for (int g0 = 0; g0 < G; g0 += 32 * 8) {
          int4 raw[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int g = g0 + lane + 32 * u;
            if (g < G) raw[u] = __ldcg(reinterpret_cast<const int4*>(cands + (j & 1) * G + g));
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int g = g0 + lane + 32 * u;
            if (g < G) {
              const Cand cd = *reinterpret_cast<const Cand*>(&raw[u]);
              if (cd.row >= 0 && cand_better(cd.key, cd.pos, bv, bp)) { bv = cd.key; bp = cd.pos; bc = g; bw = cd.row; }
            }
          }
        }
        const int best = warp_best_lane(bv, bp, bc >= 0);
        if (best >= 0) {
          bv = __shfl_sync(0xffffffffu, bv, best);
          bp = __shfl_sync(0xffffffffu, bp, best);
          bc = __shfl_sync(0xffffffffu, bc, best);
          bw = __shfl_sync(0xffffffffu, bw, best);
        } else {
          bc = -1;
        }
      }
      if (!ok || bc < 0) {  // timed out, or no row left (cannot happen with steps <= rows)
        if (lane == 0) {
          if (ok) set_flag(status, FLAG_ZERO_PIVOT);
          s_stop = 1;
        }
        __syncwarp();
        bar_arrive(1, NT);
        break;
      }
      // the pivot row (the winner's published values of columns j..cols-1)
      T* ub = ring + (size_t)(j % RU) * cols;
      {
        const T* src = candrow + ((size_t)(j & 1) * G + bc) * cols;
        for (int c = j + lane; c < cols; c += 32) ub[c - j] = ldcg_(src + (c - j));
      }
      __syncwarp();
      if (lane == 0) {
        const int w = bw, wpos = bp;
        const bool zero = (ub[0] == zero_<T>());
        s_zero = zero ? 1 : 0;
        if (zero && blockIdx.x == 0) set_flag(status, FLAG_ZERO_PIVOT);
        s_rpiv = zero ? zero_<T>() : recip(ub[0]);
        // getf2 swap of positions jg = j0 + j and wpos
        const int jg = j0 + j;
        const int occ = pwin[jg];
        pwin[jg] = w;
        if (wpos < npos) pwin[wpos] = occ;
        if (occ != w && occ >= r0 && occ < r0 + nr) lpos[occ - r0] = wpos;
        if (w >= r0 && w < r0 + nr) {
          lpos[w - r0] = jg;
          lstep[w - r0] = jg;
        }
      }
      __syncwarp();
      bar_arrive(1, NT);
    }
  } else {
    // ------------------------------------------------------------ workers
    const int tw = tid - 32, wk = warp - 1;
    // Candidate for column jc among the rows not yet pivoted: key and position
    // from each worker thread's rows, reduced over the workers; the result
    // (local row or -1) lands in s_rstar, s_ckey, s_cpos.
    auto reduce_cand = [&](unsigned long long bv, int bp, int br) {
      const int best = warp_best_lane(bv, bp, br >= 0);
      unsigned long long wv = 0ull;
      int wp = 0x7fffffff, wr = -1;
      if (best >= 0) {
        wv = __shfl_sync(0xffffffffu, bv, best);
        wp = __shfl_sync(0xffffffffu, bp, best);
        wr = __shfl_sync(0xffffffffu, br, best);
      }
      if (lane == 0) { red_v[wk] = wv; red_p[wk] = wp; red_r[wk] = wr; }
      bar_sync(3, NTW);
      if (tw == 0) {
        bv = red_v[0];
        bp = red_p[0];
        br = red_r[0];
        for (int w = 1; w < NWK; ++w)
          if (cand_better(red_v[w], red_p[w], bv, bp)) { bv = red_v[w]; bp = red_p[w]; br = red_r[w]; }
        s_rstar = br;
        s_ckey = bv;
        s_cpos = bp;
      }
      bar_sync(3, NTW);
    };
    auto write_candrow = [&](int jc) {
      const int lr = s_rstar;
      T* dst = candrow + ((size_t)(jc & 1) * G + blockIdx.x) * cols;
      if (lr >= 0)
        for (int c = jc + tw; c < cols; c += NTW) dst[c - jc] = at(lr, c);
    };

    // step 0 candidate
    if (steps > 0) {
      unsigned long long bv = 0ull;
      int bp = 0x7fffffff, br = -1;
      for (int r = tw; r < nr; r += NTW) {
        if (lstep[r] >= 0) continue;  // pivoted by an earlier panel
        const unsigned long long v = mag_key(at(r, 0));
        const int p = lpos[r];
        if (cand_better(v, p, bv, bp)) { bv = v; bp = p; br = r; }
      }
      reduce_cand(bv, bp, br);
      write_candrow(0);
      bar_arrive(2, NT);
    }
    int F = -1;  // last step whose update every row has received (columns >= its look-ahead)
    for (int j = 0; j < steps; ++j) {
      bar_sync(1, NT);  // pivot row and bookkeeping of step j are in place
      if (s_stop) break;
      const bool zero = s_zero != 0;
      const T rpiv = s_rpiv;
      const bool more = j + 1 < steps;
      T* lj = lhist + (size_t)(j % D) * rp;  // multipliers of step j
      // row r has every step up to max(F, ldone[r]) in its columns j+1..; the
      // pending ones, oldest first: t in (max(F, ldone[r]), j]
      auto pend_apply = [&](int r, int c, T x) -> T {
        if (SMEM) return mad(-lj[r], ring[(size_t)(j % RU) * cols + (c - j)], x);  // D = 1: step j only
        const int t0 = max(F, (int)ldone[r]) + 1;
        int sl = t0 % D, su = t0 % RU;  // ring slots of step t0, advanced without divisions
        for (int t = t0; t <= j; ++t) {
          x = mad(-lhist[(size_t)sl * rp + r], ring[(size_t)su * cols + (c - t)], x);
          if (++sl == D) sl = 0;
          if (++su == RU) su = 0;
        }
        return x;
      };
      // column j below the pivot (l = x / pivot), then column j+1 (look-ahead),
      // and the best candidate of column j+1 among this CTA's rows
      unsigned long long bv = 0ull;
      int bp = 0x7fffffff, br = -1;
      for (int r = tw; r < nr; r += NTW) {
        if (lstep[r] < 0) {
          T lv = zero_<T>();
          if (!zero) {
            lv = at(r, j) * rpiv;
            at(r, j) = lv;
          }
          lj[r] = lv;  // a zero pivot contributes no update
          if (j + 1 < cols) at(r, j + 1) = pend_apply(r, j + 1, at(r, j + 1));
          if (more) {
            const unsigned long long v = mag_key(at(r, j + 1));
            const int p = lpos[r];
            if (cand_better(v, p, bv, bp)) { bv = v; bp = p; br = r; }
          }
        }
      }
      int rstar = -1;
      if (more) {
        reduce_cand(bv, bp, br);  // ends with a worker barrier: lhist and column j+1 are complete
        rstar = s_rstar;
        // the candidate row is brought fully up to date before it is published
        if (rstar >= 0)
          for (int c = j + 2 + tw; c < cols; c += NTW) at(rstar, c) = pend_apply(rstar, c, at(rstar, c));
        bar_sync(3, NTW);
        if (tw == 0 && rstar >= 0) ldone[rstar] = j;
        write_candrow(j + 1);
        bar_arrive(2, NT);
      } else {
        bar_sync(3, NTW);
      }
      // the trailing update of the pending steps (columns j+2.., every row not
      // yet brought up to date): every step in shared memory, every D steps
      // (and at the last step) in global memory
      const bool flush = (j - F >= D) || !more;
      const int c0 = j + 2;
      if (flush && c0 < cols) {
        if (SMEM) {
          const T* ub = ring + (size_t)(j % RU) * cols;
          const int width = cols - c0;
          const int tot = nr * width;
          if (!zero && width >= 32) {
            // a warp per row, lanes along the row
            for (int r = wk; r < nr; r += NWK) {
              if (lstep[r] < 0 && r != rstar) {
                const T lv = -lj[r];
                for (int c = c0 + lane; c < cols; c += 32) {
                  T& x = at(r, c);
                  x = mad(lv, ub[c - j], x);
                }
              }
            }
          } else if (!zero && tot > 0) {
            // narrow blocks (panels of a blocked LU): a flat loop over (row,
            // column) keeps every lane busy (an FP64 instruction costs the
            // same issue time whatever its active lanes); (r, c) advance
            // without divisions
            const int dr = NTW / width, dc = NTW - dr * width;
            int r = tw / width, c = tw - r * width;
            for (int e = tw; e < tot; e += NTW) {
              if (lstep[r] < 0 && r != rstar) {
                T& x = at(r, c0 + c);
                x = mad(-lj[r], ub[c0 + c - j], x);
              }
              r += dr;
              c += dc;
              if (c >= width) {
                c -= width;
                ++r;
              }
            }
          }
        } else {
          // global memory: a flat loop over (row, column) with several independent
          // elements per thread in flight; the fast index follows the memory layout
          const int width = cols - c0;
          const int tot = nr * width;
          constexpr int U = 4;
          for (int base = tw; base < tot; base += NTW * U) {
            T xv[U];
            int rr[U], cc[U];
            bool act[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const int idx = base + u * NTW;
              int r, c;
              if (row_fast) { r = idx % nr; c = idx / nr; } else { c = idx % width; r = idx / width; }
              rr[u] = r;
              cc[u] = c0 + c;
              // rstar was brought up to date above (its watermark is set by one
              // thread and is not yet visible to all): excluded by index
              act[u] = idx < tot && r != rstar && lstep[r < nr ? r : 0] < 0 && ldone[r < nr ? r : 0] < j;
              if (act[u]) xv[u] = at(r, c0 + c);
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
              if (act[u]) at(rr[u], cc[u]) = pend_apply(rr[u], cc[u], xv[u]);
          }
        }
      }
      if (flush) F = j;
    }
  }
  __syncthreads();

  // write back
  if (SMEM) {
    for (int e = tid; e < nr * cols; e += NT) {
      int r, c;
      slab_rc(e, r, c);
      xref(X, rs, cs, r0 + r, c) = slab[(size_t)r * sst + c];
    }
  }
  for (int r = tid; r < nr; r += NT) {
    pos_out[r0 + r] = lpos[r];
    pstep_out[r0 + r] = lstep[r];
    perm_out[lpos[r]] = r0 + r;
  }
}

// Dynamic shared memory of the shared-memory variant (the per-block maximum is
// 227 KB, less the kernel's few hundred bytes of static shared memory).
constexpr size_t kSmemSlabBudget = 225 * 1024;

// Shared memory: the slab (shared-memory variant), D + 1 pivot rows, D columns
// of multipliers, and per-row position, pivot step and watermark.
template <typename T, bool SMEM>
static size_t pivlu_smem(int64_t rpc, int cols, int npos, int D) {
  size_t b = (SMEM ? (size_t)rpc * (cols | 1) * sizeof(T) : 0) + (size_t)(D + 1) * cols * sizeof(T) +
             (size_t)D * rpc * sizeof(T) + (size_t)rpc * 12 + (size_t)npos * 4;
  return (b + 15) & ~(size_t)15;
}

// Deferral depth of the global-memory variant: up to 16 steps per pass over
// the trailing block, as many as fit in the shared-memory budget.
template <typename T>
static int pivlu_defer(int64_t rpc, int cols, int npos, size_t budget) {
  int D = 16;
  while (D > 1 && pivlu_smem<T, false>(rpc, cols, npos, D) > budget) --D;
  return D;
}

template <typename T, bool SMEM>
static int launch_cfg(T* X, int64_t rows, int cols, int64_t rs, int64_t cs, int steps, int j0, int npos, int G,
                      PivLuWs& ws, unsigned int* status, cudaStream_t st) {
  constexpr int NT = SMEM ? 256 : 1024;
  const int64_t rpc = cdiv(rows, G);
  int defer = SMEM ? 1 : pivlu_defer<T>(rpc, cols, npos, 200 * 1024);
  size_t smem = pivlu_smem<T, SMEM>(rpc, cols, npos, defer);
  auto kern = k_pivoted_lu<T, SMEM, NT>;
  if (int rc_ = allow_dynamic_smem((const void*)kern, smem)) return rc_;
  int per_sm = 0;
  RLU_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
  if (per_sm < 1) return RLU_EINVAL;
  RLU_CUDA_TRY(cudaMemsetAsync(ws.bar, 0, sizeof(unsigned int), st));
  Cand* cand = reinterpret_cast<Cand*>(ws.cand);
  T* candrow = reinterpret_cast<T*>(ws.candrow);
  void* args[] = {&X, &rows, &cols, &rs, &cs, &steps, (void*)&rpc, &ws.pos, &ws.pstep, &ws.perm,
                  &cand, &candrow, &ws.bar, &status, &defer, &j0, &npos};
  RLU_CUDA_TRY(launch_cooperative((void*)kern, G, NT, args, smem, st));
  note_launch();
  return RLU_OK;
}

size_t pivlu_cand_bytes(int max_ctas) { return (size_t)2 * max_ctas * sizeof(Cand); }

// One CTA per SM, or fewer for small inputs (at least 8 rows per CTA).
static int pivlu_grid(int64_t rows, const PivLuWs& ws, int num_sms) {
  int G = (int)min64(num_sms, cdiv(rows, 8));
  return G > ws.max_ctas ? ws.max_ctas : G;
}

template <typename T>
int launch_pivoted_lu(T* X, int64_t rows, int cols, int64_t rs, int64_t cs, int steps, PivLuWs& ws,
                      unsigned int* status, int num_sms, cudaStream_t st) {
  return launch_pivoted_lu_panel<T>(X, rows, cols, rs, cs, steps, 0, steps, ws, status, num_sms, st);
}

template <typename T>
int launch_pivoted_lu_panel(T* X, int64_t rows, int cols, int64_t rs, int64_t cs, int steps, int j0, int npos,
                            PivLuWs& ws, unsigned int* status, int num_sms, cudaStream_t st) {
  if (steps > cols || j0 < 0 || j0 + steps > npos || npos > rows || cols > ws.max_cols) return RLU_EINVAL;
  const int G = pivlu_grid(rows, ws, num_sms);
  const int64_t rpc = cdiv(rows, G);
  size_t smem = pivlu_smem<T, true>(rpc, cols, npos, 1);
  if (smem <= kSmemSlabBudget) return launch_cfg<T, true>(X, rows, cols, rs, cs, steps, j0, npos, G, ws, status, st);
  return launch_cfg<T, false>(X, rows, cols, rs, cs, steps, j0, npos, G, ws, status, st);
}

bool pivlu_panel_in_smem(int64_t rows, int cols, int npos, const PivLuWs& ws, int num_sms) {
  const int G = pivlu_grid(rows, ws, num_sms);
  return pivlu_smem<double, true>(cdiv(rows, G), cols, npos, 1) <= kSmemSlabBudget;
}

template int launch_pivoted_lu<double>(double*, int64_t, int, int64_t, int64_t, int, PivLuWs&, unsigned int*, int,
                                       cudaStream_t);
template int launch_pivoted_lu<float>(float*, int64_t, int, int64_t, int64_t, int, PivLuWs&, unsigned int*, int,
                                      cudaStream_t);
template int launch_pivoted_lu<df32>(df32*, int64_t, int, int64_t, int64_t, int, PivLuWs&, unsigned int*, int,
                                     cudaStream_t);
template int launch_pivoted_lu_panel<double>(double*, int64_t, int, int64_t, int64_t, int, int, int, PivLuWs&,
                                             unsigned int*, int, cudaStream_t);
template int launch_pivoted_lu_panel<df32>(df32*, int64_t, int, int64_t, int64_t, int, int, int, PivLuWs&,
                                           unsigned int*, int, cudaStream_t);

}  // namespace rlu
