// Step 1 and step 2 of Algorithm 1 (Sec. 3): the random structures and the
// sketch Y = A S D H R / sqrt(l1).
//
//  * k_sketch_params / k_select_R: the hash h, signs s of the sparse embedding
//    matrix (Sec. 2.2) and the signs d and subsample R of the real FFT-based
//    projection (Sec. 2.1), all from Philox4x64-10 with key (seed, "RANDLU").
//  * bucket lists: for each column chunk and bucket b, the columns j of the
//    chunk with h(j) = b in ascending order, so the CountSketch is a
//    deterministic gather-sum in ascending column order (one chunk = whole
//    rows when they fit the whole-row kernel).
//  * k_sketch_rows: one pass over dense row-major A whose rows fit in shared
//    memory, a bulk copy per row; each row's bucket sums go straight into the
//    FFT input of its row pair (two real rows packed as real and imaginary
//    parts), batches of row pairs go through a complex mixed-radix Stockham
//    FFT in shared memory, and the Hartley outputs Re X - Im X of the l
//    selected frequencies are scaled by 1/sqrt(l1) and written to Y.
//  * k_sketch_dense_tma / k_sketch_dense: the same over column chunks of R-row
//    groups (rows too long for shared memory; rows that cannot be bulk-copied),
//    each thread summing the buckets it owns in registers.
//  Y1 never reaches global memory.
#include <cstdio>

#include "common.cuh"
#include "sketch.cuh"

#include <type_traits>

namespace rlu {

// ---------------------------------------------------------------------------
// Random structures
// ---------------------------------------------------------------------------
__global__ void k_sketch_params(int64_t n, int l1, uint64_t seed, uint32_t* hs, float* dsign, uint64_t* keys) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
    Philox4 b = philox4x64_10((uint64_t)i, 0, 0, 0, seed, kKeyTag);
    uint32_t h = (uint32_t)__umul64hi(b.w[0], (uint64_t)l1);
    uint32_t neg = (uint32_t)(b.w[1] >> 63);
    hs[i] = h | (neg << 31);
  }
  if (i < l1) {
    Philox4 b1 = philox4x64_10((uint64_t)i, 1, 0, 0, seed, kKeyTag);
    dsign[i] = (b1.w[0] >> 63) ? -1.0f : 1.0f;
    Philox4 b2 = philox4x64_10((uint64_t)i, 2, 0, 0, seed, kKeyTag);
    keys[i] = b2.w[0];
  }
}

// R = the l indices b with the smallest (key[b], b), in increasing order:
// each b counts the keys below its own (one warp per b, the lanes splitting
// the l1 keys) and, if that rank is < l, lands at R[rank].
__global__ void k_select_R(int l1, int l, const uint64_t* keys, int32_t* R) {
  const int b = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (b >= l1) return;
  const uint64_t kb = keys[b];
  int rank = 0;
  for (int t = lane; t < l1; t += 32) {
    const uint64_t kt = __ldg(keys + t);
    rank += (kt < kb) || (kt == kb && t < b);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) rank += __shfl_xor_sync(0xffffffffu, rank, o);
  if (lane == 0 && rank < l) R[rank] = b;
}

// ---------------------------------------------------------------------------
// Bucket lists per column chunk: super-bucket sb = chunk * l1 + h(j)
// ---------------------------------------------------------------------------
__global__ void k_bucket_count(int64_t n, int l1, int chunk, const uint32_t* hs, int32_t* cnt) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j < n) {
    int64_t sb = (j / chunk) * l1 + (hs[j] & 0x7fffffffu);
    atomicAdd(&cnt[sb], 1);
  }
}

// Exclusive scan of cnt[0..count) into start[0..count], one CTA of 1024 threads.
__global__ void k_scan_counts(int64_t count, const int32_t* cnt, int32_t* start) {
  __shared__ int64_t part[1024];
  const int T = blockDim.x;
  int64_t per = cdiv(count, T);
  int64_t a = threadIdx.x * per, b = min(count, a + per);
  int64_t s = 0;
  for (int64_t i = a; i < b; ++i) s += cnt[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t run = 0;
    for (int t = 0; t < T; ++t) {
      int64_t v = part[t];
      part[t] = run;
      run += v;
    }
  }
  __syncthreads();
  int64_t run = part[threadIdx.x];
  for (int64_t i = a; i < b; ++i) {
    start[i] = (int32_t)run;
    run += cnt[i];
  }
  if (threadIdx.x == T - 1) start[count] = (int32_t)run;
}

// Exclusive scan over many CTAs: CTA b owns the elements [b per, (b+1) per)
// and reads them in rounds of blockDim.x consecutive values (coalesced).
// k_scan_part writes each CTA's total; k_scan_final adds the totals of the
// CTAs before it and scans its own rounds.  Fixed order: exact integer sums.
__device__ __forceinline__ int64_t block_sum_i64(int64_t v, int64_t* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  int64_t t = 0;
  for (int w = 0; w < nw; ++w) t += red[w];
  return t;
}

__global__ void __launch_bounds__(1024) k_scan_part(int64_t count, int64_t per, const int32_t* __restrict__ cnt,
                                                    int64_t* __restrict__ part) {
  __shared__ int64_t red[32];
  const int64_t a = (int64_t)blockIdx.x * per, b = min64(count, a + per);
  int64_t s = 0;
  for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x) s += cnt[i];
  s = block_sum_i64(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(1024) k_scan_final(int64_t count, int64_t per, const int32_t* __restrict__ cnt,
                                                     const int64_t* __restrict__ part, int32_t* __restrict__ start) {
  __shared__ int64_t red[32];
  __shared__ int64_t wsum[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int64_t off = 0;
  for (int b = threadIdx.x; b < (int)blockIdx.x; b += blockDim.x) off += part[b];
  off = block_sum_i64(off, red);
  const int64_t a = (int64_t)blockIdx.x * per, e = min64(count, a + per);
  for (int64_t r0 = a; r0 < e; r0 += blockDim.x) {
    const int64_t i = r0 + threadIdx.x;
    const int64_t v = i < e ? cnt[i] : 0;
    int64_t x = v;  // inclusive scan within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    int64_t before = 0, round = 0;
    for (int w = 0; w < nw; ++w) {
      const int64_t t = wsum[w];
      if (w < warp) before += t;
      round += t;
    }
    if (i < e) start[i] = (int32_t)(off + before + x - v);
    off += round;
  }
  if (e == count && a < e && threadIdx.x == 0) start[count] = (int32_t)off;
  if (count == 0 && blockIdx.x == 0 && threadIdx.x == 0) start[0] = 0;
}

__global__ void k_bucket_fill(int64_t n, int l1, int chunk, const uint32_t* hs, const int32_t* start,
                              int32_t* cursor, uint32_t* list) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j < n) {
    uint32_t e = hs[j];
    int64_t c = j / chunk;
    int64_t sb = c * l1 + (e & 0x7fffffffu);
    int pos = start[sb] + atomicAdd(&cursor[sb], 1);
    list[pos] = (uint32_t)(j - c * chunk) | (e & 0x80000000u);
  }
}

// All of the above in one CTA when the super-buckets fit in shared memory:
// counts, exclusive scan into start[0..count], fill, then each list sorted by
// column.  Same lists as the four kernels.
constexpr int kListsOneMax = 8192;
__global__ void __launch_bounds__(1024) k_bucket_lists_one(int64_t n, int l1, int chunk, int count,
                                                           const uint32_t* __restrict__ hs, int32_t* start,
                                                           uint32_t* list) {
  extern __shared__ int lsm[];  // cnt[count + 1], cursor[count]
  __shared__ int wsum[32];
  int* cnt = lsm;
  int* cur = lsm + count + 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i <= count; i += blockDim.x) cnt[i] = 0;
  __syncthreads();
  for (int64_t j = tid; j < n; j += blockDim.x) atomicAdd(&cnt[(j / chunk) * l1 + (hs[j] & 0x7fffffffu)], 1);
  __syncthreads();
  // exclusive scan: a contiguous segment per thread, then warp and block offsets
  const int per = (count + (int)blockDim.x - 1) / (int)blockDim.x;
  const int a = min(count, tid * per), e = min(count, a + per);
  int sum = 0;
  for (int i = a; i < e; ++i) sum += cnt[i];
  int inc = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const int nw = (int)blockDim.x >> 5;
    int v = lane < nw ? wsum[lane] : 0, w = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    if (lane < nw) wsum[lane] = w - v;
    if (lane == 31) cnt[count] = w;  // total (cnt[count] is not part of any segment)
  }
  __syncthreads();
  int run = wsum[warp] + inc - sum;
  for (int i = a; i < e; ++i) {
    const int v = cnt[i];
    cnt[i] = run;
    run += v;
  }
  __syncthreads();
  for (int i = tid; i <= count; i += blockDim.x) {
    start[i] = cnt[i];
    if (i < count) cur[i] = cnt[i];
  }
  __syncthreads();
  for (int64_t j = tid; j < n; j += blockDim.x) {
    const uint32_t v = hs[j];
    const int64_t c = j / chunk;
    const int pos = atomicAdd(&cur[c * l1 + (v & 0x7fffffffu)], 1);
    list[pos] = (uint32_t)(j - c * chunk) | (v & 0x80000000u);
  }
  __syncthreads();
  for (int sb = tid; sb < count; sb += blockDim.x) {
    const int lo = cnt[sb], hi = cnt[sb + 1];
    for (int i = lo + 1; i < hi; ++i) {
      const uint32_t v = list[i];
      const uint32_t kv = v & 0x7fffffffu;
      int t = i - 1;
      while (t >= lo && (list[t] & 0x7fffffffu) > kv) {
        list[t + 1] = list[t];
        --t;
      }
      list[t + 1] = v;
    }
  }
}

// Sort each super-bucket's entries by column (insertion sort; buckets are short).
__global__ void k_bucket_sort(int64_t count, const int32_t* start, uint32_t* list) {
  int64_t sb = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (sb >= count) return;
  int a = start[sb], b = start[sb + 1];
  for (int i = a + 1; i < b; ++i) {
    uint32_t v = list[i];
    uint32_t kv = v & 0x7fffffffu;
    int t = i - 1;
    while (t >= a && (list[t] & 0x7fffffffu) > kv) {
      list[t + 1] = list[t];
      --t;
    }
    list[t + 1] = v;
  }
}

// Twiddles tw[e] = exp(-2 pi i e / N), computed in FP64 with sincospi.
__global__ void k_twiddles(int N, double2* tw64, float2* tw32) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N) return;
  double s, c;
  sincospi(-2.0 * (double)e / (double)N, &s, &c);
  tw64[e] = make_double2(c, s);
  tw32[e] = make_float2((float)c, (float)s);
}

// ---------------------------------------------------------------------------
// Complex arithmetic on float2 / double2
// ---------------------------------------------------------------------------
template <typename T> struct C2;
template <> struct C2<float> { using t = float2; };
template <> struct C2<double> { using t = double2; };

template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return V{a.x + b.x, a.y + b.y}; }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return V{a.x - b.x, a.y - b.y}; }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  return V{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// multiply by -i
template <typename V> __device__ __forceinline__ V cmi(V a) { return V{a.y, -a.x}; }

// One Stockham stage of radix r over N points: p = product of the radices
// already applied.  Butterfly i < N/r reads in[i + t N/r] (t < r), applies
// the twiddles exp(-2 pi i t (i mod p) / (p r)) and a length-r DFT, and
// writes out[(i - i mod p) r + i mod p + u p] (u < r).  Output is in natural
// order after the last stage.
// The same stage applied to `nb` independent transforms at once: transform t
// reads in + t * stride and writes out + t * stride (one barrier per stage
// for the whole batch instead of one per transform).
// Division by a plan constant (see FftPlan): exact for x < 2^16.
__device__ __forceinline__ uint32_t fdiv(uint32_t x, uint32_t m, uint32_t d) { return m ? __umulhi(x, m) : x / d; }
__host__ __device__ __forceinline__ uint32_t div_magic(int d) {
  return d < 2 ? 0u : (uint32_t)(((1ull << 32) + (unsigned long long)d - 1) / (unsigned long long)d);
}

// Length-5 DFT in place: X_u = sum_q x_q w^(u q), w = exp(-2 pi i / 5), from
// the symmetric sums s = x1 + x4, x2 + x3 and differences d = x1 - x4, x2 - x3
// (cos and sin of 2 pi / 5 and 4 pi / 5).
template <typename V, typename S>
__device__ __forceinline__ void dft5(V& x0, V& x1, V& x2, V& x3, V& x4) {
  const S c1 = S(0.30901699437494742410), c2 = S(-0.80901699437494742410);
  const S s1 = S(0.95105651629515357212), s2 = S(0.58778525229247312917);
  const V a = cadd(x1, x4), b = csub(x1, x4), c = cadd(x2, x3), d = csub(x2, x3);
  const V y1 = V{x0.x + c1 * a.x + c2 * c.x, x0.y + c1 * a.y + c2 * c.y};
  const V y2 = V{x0.x + c2 * a.x + c1 * c.x, x0.y + c2 * a.y + c1 * c.y};
  const V z1 = V{s1 * b.x + s2 * d.x, s1 * b.y + s2 * d.y};  // X1 = y1 - i z1, X4 = y1 + i z1
  const V z2 = V{s2 * b.x - s1 * d.x, s2 * b.y - s1 * d.y};  // X2 = y2 - i z2, X3 = y2 + i z2
  x0 = V{x0.x + a.x + c.x, x0.y + a.y + c.y};
  x1 = V{y1.x + z1.y, y1.y - z1.x};
  x4 = V{y1.x - z1.y, y1.y + z1.x};
  x2 = V{y2.x + z2.y, y2.y - z2.x};
  x3 = V{y2.x - z2.y, y2.y + z2.x};
}

// One Stockham stage (stage `st` of `plan`) applied to `nb` independent
// transforms at once: transform t reads in + t * stride and writes out + t *
// stride (one barrier per stage for the whole batch instead of one per
// transform).  Butterfly i < T reads in[i + t T] (t < r), applies the twiddles
// exp(-2 pi i t (i mod p) / (p r)) and a length-r DFT, and writes
// out[(i - i mod p) r + i mod p + u p] (u < r).  Output is in natural order
// after the last stage.
template <typename V, typename S>
__device__ void stockham_stage_batch(const V* __restrict__ in, V* __restrict__ out, int stride, int nb, int N,
                                     const FftPlan& plan, int st, const V* tw, int t0, int nthr) {
  const int r = plan.radix[st], p = plan.p[st], T = plan.T[st], step = plan.step[st];
  const uint32_t mT = plan.mT[st], mp = plan.mp[st];
  const int total = nb * T;
  for (int idx = t0; idx < total; idx += nthr) {
    const int tb = (int)fdiv((uint32_t)idx, mT, (uint32_t)T), i = idx - tb * T;
    const V* src = in + (size_t)tb * stride;
    V* dst = out + (size_t)tb * stride;
    const int k = p == 1 ? 0 : i - (int)fdiv((uint32_t)i, mp, (uint32_t)p) * p;
    const int obase = (i - k) * r + k;
    if (r == 4) {
      V x0 = src[i], x1 = src[i + T], x2 = src[i + 2 * T], x3 = src[i + 3 * T];
      if (k) {
        x1 = cmul(x1, tw[k * step]);
        x2 = cmul(x2, tw[2 * k * step]);
        x3 = cmul(x3, tw[3 * k * step]);
      }
      V a0 = cadd(x0, x2), a1 = csub(x0, x2), b0 = cadd(x1, x3), b1 = cmi(csub(x1, x3));
      dst[obase] = cadd(a0, b0);
      dst[obase + p] = cadd(a1, b1);
      dst[obase + 2 * p] = csub(a0, b0);
      dst[obase + 3 * p] = csub(a1, b1);
    } else if (r == 2) {
      V x0 = src[i], x1 = src[i + T];
      if (k) x1 = cmul(x1, tw[k * step]);
      dst[obase] = cadd(x0, x1);
      dst[obase + p] = csub(x0, x1);
    } else if (r == 3) {
      V x0 = src[i], x1 = src[i + T], x2 = src[i + 2 * T];
      if (k) {
        x1 = cmul(x1, tw[k * step]);
        x2 = cmul(x2, tw[2 * k * step]);
      }
      const S h = S(0.86602540378443864676);
      V sm = cadd(x1, x2), d = csub(x1, x2);
      V t = V{x0.x - S(0.5) * sm.x, x0.y - S(0.5) * sm.y};
      V u = V{h * d.y, -h * d.x};
      dst[obase] = cadd(x0, sm);
      dst[obase + p] = cadd(t, u);
      dst[obase + 2 * p] = csub(t, u);
    } else if (r == 5) {
      V x0 = src[i], x1 = src[i + T], x2 = src[i + 2 * T], x3 = src[i + 3 * T], x4 = src[i + 4 * T];
      if (k) {
        x1 = cmul(x1, tw[k * step]);
        x2 = cmul(x2, tw[2 * k * step]);
        x3 = cmul(x3, tw[3 * k * step]);
        x4 = cmul(x4, tw[4 * k * step]);
      }
      dft5<V, S>(x0, x1, x2, x3, x4);
      dst[obase] = x0;
      dst[obase + p] = x1;
      dst[obase + 2 * p] = x2;
      dst[obase + 3 * p] = x3;
      dst[obase + 4 * p] = x4;
    } else {
      const int wstep = N / r;
      for (int u = 0; u < r; ++u) {
        V y = src[i];
        int e = 0;
        for (int q = 1; q < r; ++q) {
          e += u;
          if (e >= r) e -= r;
          V v = src[i + q * T];
          if (k) v = cmul(v, tw[q * k * step]);
          y = cadd(y, cmul(v, tw[e * wstep]));
        }
        dst[obase + u * p] = y;
      }
    }
  }
}

template <typename V, typename S>
__device__ void stockham_stage(const V* __restrict__ in, V* __restrict__ out, int N, int r, int p, const V* tw) {
  const int T = N / r;
  const int step = N / (p * r);
  for (int i = threadIdx.x; i < T; i += blockDim.x) {
    const int k = i % p;
    const int obase = (i - k) * r + k;
    if (r == 4) {
      V x0 = in[i], x1 = in[i + T], x2 = in[i + 2 * T], x3 = in[i + 3 * T];
      if (k) {
        x1 = cmul(x1, tw[k * step]);
        x2 = cmul(x2, tw[2 * k * step]);
        x3 = cmul(x3, tw[3 * k * step]);
      }
      V a0 = cadd(x0, x2), a1 = csub(x0, x2), b0 = cadd(x1, x3), b1 = cmi(csub(x1, x3));
      out[obase] = cadd(a0, b0);
      out[obase + p] = cadd(a1, b1);
      out[obase + 2 * p] = csub(a0, b0);
      out[obase + 3 * p] = csub(a1, b1);
    } else if (r == 2) {
      V x0 = in[i], x1 = in[i + T];
      if (k) x1 = cmul(x1, tw[k * step]);
      out[obase] = cadd(x0, x1);
      out[obase + p] = csub(x0, x1);
    } else if (r == 3) {
      V x0 = in[i], x1 = in[i + T], x2 = in[i + 2 * T];
      if (k) {
        x1 = cmul(x1, tw[k * step]);
        x2 = cmul(x2, tw[2 * k * step]);
      }
      // W3 = exp(-2 pi i / 3) = -1/2 - i sqrt(3)/2
      const S h = S(0.86602540378443864676);
      V s = cadd(x1, x2), d = csub(x1, x2);
      V t = V{x0.x - S(0.5) * s.x, x0.y - S(0.5) * s.y};
      V u = V{h * d.y, -h * d.x};  // -i * (sqrt(3)/2) * d
      out[obase] = cadd(x0, s);
      out[obase + p] = cadd(t, u);
      out[obase + 2 * p] = csub(t, u);
    } else if (r <= 16) {
      V x[16];
      for (int t = 0; t < r; ++t) {
        V v = in[i + t * T];
        x[t] = (k && t) ? cmul(v, tw[t * k * step]) : v;
      }
      const int wstep = N / r;
      for (int u = 0; u < r; ++u) {
        V y = x[0];
        int e = 0;
        for (int t = 1; t < r; ++t) {
          e += u;
          if (e >= r) e -= r;
          y = cadd(y, cmul(x[t], tw[e * wstep]));
        }
        out[obase + u * p] = y;
      }
    } else {
      // large prime radix: direct sums, operands re-read from shared memory
      const int wstep = N / r;
      for (int u = 0; u < r; ++u) {
        V y = in[i];
        int e = 0;
        for (int t = 1; t < r; ++t) {
          e += u;
          if (e >= r) e -= r;
          V v = in[i + t * T];
          if (k) v = cmul(v, tw[t * k * step]);
          y = cadd(y, cmul(v, tw[e * wstep]));
        }
        out[obase + u * p] = y;
      }
    }
  }
}

template <typename TA> __device__ __forceinline__ float load_acc(const TA* p, float) { return to_float(*p); }
template <typename TA> __device__ __forceinline__ double load_acc(const TA* p, double) { return to_double(*p); }

// ---------------------------------------------------------------------------
// Fused dense sketch: CountSketch + signs + Hartley FFT + subsample
// ---------------------------------------------------------------------------
template <typename TA, typename TACC, int NT, int NB, int R>
__global__ void __launch_bounds__(NT) k_sketch_dense(const TA* __restrict__ A, int64_t lda, int64_t m, int64_t n,
                                                     int l1, int l, int chunk, const int32_t* __restrict__ bstart,
                                                     const uint32_t* __restrict__ blist,
                                                     const float* __restrict__ dsign, const int32_t* __restrict__ Rsel,
                                                     const typename C2<TACC>::t* __restrict__ tw, FftPlan plan,
                                                     double* __restrict__ Y, const int32_t* __restrict__ rowmap,
                                                     unsigned int* status) {
  using V = typename C2<TACC>::t;
  extern __shared__ __align__(16) unsigned char smem[];
  TA* tile = reinterpret_cast<TA*>(smem);
  V* buf0 = reinterpret_cast<V*>(smem);
  V* buf1 = buf0 + l1;
  const int tid = threadIdx.x;
  const int64_t ngroups = cdiv(m, R);
  const int nchunks = (int)cdiv(n, chunk);
  const TACC scale = TACC(1) / sqrt(TACC(l1));
  bool bad = false;
  constexpr int VEC = 16 / sizeof(TA);
  const bool vec_ok = ((lda * (int64_t)sizeof(TA)) % 16 == 0) && ((reinterpret_cast<uintptr_t>(A) % 16) == 0);

  for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
    const int64_t row0 = g * R;
    TACC acc[NB][R];
#pragma unroll
    for (int t = 0; t < NB; ++t)
#pragma unroll
      for (int r = 0; r < R; ++r) acc[t][r] = TACC(0);

    for (int c = 0; c < nchunks; ++c) {
      const int64_t col0 = (int64_t)c * chunk;
      const int width = (int)min((int64_t)chunk, n - col0);
      __syncthreads();
      // stage R x width of A (rows past m read as zero; they are never written)
      if (vec_ok && (width % VEC) == 0) {
        const int nv = width / VEC;
        for (int idx = tid; idx < R * nv; idx += NT) {
          const int r = idx / nv, v = idx - r * nv;
          uint4 val = make_uint4(0, 0, 0, 0);
          if (row0 + r < m) val = __ldg(reinterpret_cast<const uint4*>(A + (row0 + r) * lda + col0) + v);
          *reinterpret_cast<uint4*>(tile + r * chunk + v * VEC) = val;
          const TA* e = reinterpret_cast<const TA*>(&val);
#pragma unroll
          for (int q = 0; q < VEC; ++q) bad |= !finite_(e[q]);
        }
      } else {
        for (int idx = tid; idx < R * width; idx += NT) {
          const int r = idx / width, cc = idx - r * width;
          TA val = TA(0);
          if (row0 + r < m) val = A[(row0 + r) * lda + col0 + cc];
          tile[r * chunk + cc] = val;
          bad |= !finite_(val);
        }
      }
      __syncthreads();
      const int32_t* bs = bstart + (int64_t)c * l1;
#pragma unroll
      for (int t = 0; t < NB; ++t) {
        const int b = tid + t * NT;
        if (b < l1) {
          const int s0 = bs[b], s1 = bs[b + 1];
          for (int e = s0; e < s1; ++e) {
            const uint32_t ent = __ldg(blist + e);
            const int off = (int)(ent & 0x7fffffffu);
            const bool neg = (ent >> 31) != 0;
#pragma unroll
            for (int r = 0; r < R; ++r) {
              const TACC v = load_acc(tile + r * chunk + off, TACC(0));
              acc[t][r] += neg ? -v : v;
            }
          }
        }
      }
    }

    // Hartley transform of each row pair: z = d (y1[2q] + i y1[2q+1])
#pragma unroll
    for (int q = 0; q < R / 2; ++q) {
      __syncthreads();
#pragma unroll
      for (int t = 0; t < NB; ++t) {
        const int b = tid + t * NT;
        if (b < l1) {
          const TACC ds = (TACC)dsign[b];
          buf0[b] = V{ds * acc[t][2 * q], ds * acc[t][2 * q + 1]};
        }
      }
      __syncthreads();
      V* src = buf0;
      V* dst = buf1;
      int p = 1;
      for (int s = 0; s < plan.nstages; ++s) {
        const int r = plan.radix[s];
        stockham_stage<V, TACC>(src, dst, l1, r, p, tw);
        p *= r;
        __syncthreads();
        V* tmp = src;
        src = dst;
        dst = tmp;
      }
      // src holds Z = FFT(z).  X1 = (Z[f] + conj Z[-f]) / 2, X2 = (Z[f] - conj Z[-f]) / 2i,
      // Hartley H = Re X - Im X.
      const int64_t ra = row0 + 2 * q, rb = ra + 1;
      for (int cidx = tid; cidx < l; cidx += NT) {
        const int f = Rsel[cidx];
        const int fm = f == 0 ? 0 : l1 - f;
        const V z = src[f], w = src[fm];
        const TACC h1 = TACC(0.5) * ((z.x + w.x) - (z.y - w.y));
        const TACC h2 = TACC(0.5) * ((z.x - w.x) + (z.y + w.y));
        if (ra < m) Y[(rowmap ? (int64_t)rowmap[ra] : ra) * l + cidx] = (double)(h1 * scale);
        if (rb < m) Y[(rowmap ? (int64_t)rowmap[rb] : rb) * l + cidx] = (double)(h2 * scale);
      }
    }
  }
  if (bad) set_flag(status, FLAG_NONFINITE);
}

// ---------------------------------------------------------------------------
// Fused dense sketch, TMA-fed: the (row group, column chunk) tiles of A stream
// through a two-stage shared-memory ring with 1D bulk copies (one per row
// segment, completion on an mbarrier), so the next tile is in flight while
// the current one is summed and while a finished group runs its FFTs (whose
// buffers are separate from the ring).  Same arithmetic and order as
// k_sketch_dense.  Needs 16-byte aligned rows (lda * sizeof(TA) and the base
// address multiples of 16, and the chunk widths multiples of 16 bytes).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void sk_mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void sk_mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                   smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool sk_mbar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > kSpinLimitCycles) return false;
  }
}
__device__ __forceinline__ void sk_mbar_arrive(uint64_t* bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

template <typename TA, typename TACC, int NT, int NB, int R>
__global__ void __launch_bounds__(NT, 1) k_sketch_dense_tma(const TA* __restrict__ A, int64_t lda, int64_t m, int64_t n,
                                                         int l1, int l, int chunk,
                                                         const int32_t* __restrict__ bstart,
                                                         const uint32_t* __restrict__ blist,
                                                         const float* __restrict__ dsign,
                                                         const int32_t* __restrict__ Rsel,
                                                         const typename C2<TACC>::t* __restrict__ tw, FftPlan plan,
                                                         int pb, int lists_in_smem, double* __restrict__ Y,
                                                         const int32_t* __restrict__ rowmap, unsigned int* status) {
  using V = typename C2<TACC>::t;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[2];
  __shared__ int s_fail;
  TA* ring = reinterpret_cast<TA*>(smem);                       // [2][R][chunk]
  V* twsm = reinterpret_cast<V*>(smem + (size_t)2 * R * chunk * sizeof(TA));  // l1 twiddles
  V* fbuf = twsm + l1;                                          // [pb][2][l1] FFT ping-pong buffers
  // optional copy of the bucket lists (start offsets, then entries) after the FFT buffers
  int32_t* bs_sm = reinterpret_cast<int32_t*>(fbuf + (size_t)pb * 2 * l1);
  const int tid = threadIdx.x;
  const int64_t ngroups = cdiv(m, R);
  const int nchunks = (int)cdiv(n, chunk);
  const TACC scale = TACC(1) / sqrt(TACC(l1));
  const uint32_t ml = div_magic(l);
  // tiles of this CTA: t -> group blockIdx.x + (t / nchunks) * gridDim.x, chunk t % nchunks
  const int64_t my_groups = blockIdx.x < ngroups ? cdiv(ngroups - blockIdx.x, gridDim.x) : 0;
  const int64_t ntiles = my_groups * nchunks;
  bool bad = false;

  auto issue = [&](int64_t t) {  // thread 0 only
    const int s = (int)(t & 1);
    const int64_t g = blockIdx.x + (t / nchunks) * (int64_t)gridDim.x;
    const int c = (int)(t % nchunks);
    const int64_t row0 = g * R, col0 = (int64_t)c * chunk;
    const int width = (int)min64(chunk, n - col0);
    const int rows = (int)min64(R, m - row0);
    const uint32_t bytes = (uint32_t)width * sizeof(TA);
    sk_mbar_expect_tx(&full[s], bytes * rows);
    for (int r = 0; r < rows; ++r)
      bulk_g2s(ring + ((size_t)s * R + r) * chunk, A + (row0 + r) * lda + col0, bytes, &full[s]);
  };

  if (tid == 0) {
    sk_mbar_init(&full[0], 1);
    sk_mbar_init(&full[1], 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int e = tid; e < l1; e += NT) twsm[e] = tw[e];
  const int64_t nstart = (int64_t)nchunks * l1 + 1;
  uint32_t* bl_sm = reinterpret_cast<uint32_t*>(bs_sm + nstart);
  if (lists_in_smem) {
    for (int64_t e = tid; e < nstart; e += NT) bs_sm[e] = bstart[e];
    for (int64_t e = tid; e < n; e += NT) bl_sm[e] = blist[e];
  }
  const int32_t* bsrc = lists_in_smem ? bs_sm : bstart;
  const uint32_t* lsrc = lists_in_smem ? bl_sm : blist;
  __syncthreads();
  if (tid == 0 && ntiles > 0) issue(0);

  TACC acc[NB][R];
#pragma unroll
  for (int t = 0; t < NB; ++t)
#pragma unroll
    for (int r = 0; r < R; ++r) acc[t][r] = TACC(0);

  for (int64_t t = 0; t < ntiles; ++t) {
    const int s = (int)(t & 1);
    const int64_t g = blockIdx.x + (t / nchunks) * (int64_t)gridDim.x;
    const int c = (int)(t % nchunks);
    const int64_t row0 = g * R;
    const int rows = (int)min64(R, m - row0);
    // the other stage was released by the __syncthreads that ended tile t-1
    if (tid == 0 && t + 1 < ntiles) issue(t + 1);
    if (!sk_mbar_wait(&full[s], (uint32_t)((t >> 1) & 1))) s_fail = 1;
    __syncthreads();
    if (s_fail) {
      // drain the copy issued for tile t+1 (bounded) before leaving
      if (tid == 0 && t + 1 < ntiles) sk_mbar_wait(&full[(t + 1) & 1], (uint32_t)(((t + 1) >> 1) & 1));
      break;
    }
    const TA* tile = ring + (size_t)s * R * chunk;
    const int32_t* bs = bsrc + (int64_t)c * l1;
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int b = tid + q * NT;
      if (b < l1) {
        const int s0 = bs[b], s1 = bs[b + 1];
        for (int e = s0; e < s1; ++e) {
          const uint32_t ent = lsrc[e];
          const int off = (int)(ent & 0x7fffffffu);
          const TACC sg = (ent >> 31) ? TACC(-1) : TACC(1);
          // a NaN or Inf entry makes its bucket sum non-finite: checked once per
          // bucket when the row group is complete, not per element
#pragma unroll
          for (int r = 0; r < R; ++r) acc[q][r] = fma(sg, load_acc(tile + r * chunk + off, TACC(0)), acc[q][r]);
        }
      }
    }
    if (c == nchunks - 1) {
#pragma unroll
      for (int q = 0; q < NB; ++q)
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (r < rows && tid + q * NT < l1) bad |= !isfinite(acc[q][r]);
      // Hartley transforms of the finished group's row pairs, pb pairs per batch
      for (int q0 = 0; q0 < R / 2; q0 += pb) {
        const int nbat = min(pb, R / 2 - q0);
        __syncthreads();
#pragma unroll
        for (int q2 = 0; q2 < R / 2; ++q2) {
          if (q2 >= q0 && q2 < q0 + nbat) {
            const bool va = 2 * q2 < rows, vb = 2 * q2 + 1 < rows;
            V* z = fbuf + (size_t)(q2 - q0) * 2 * l1;
#pragma unroll
            for (int q = 0; q < NB; ++q) {
              const int b = tid + q * NT;
              if (b < l1) {
                const TACC ds = (TACC)dsign[b];
                z[b] = V{va ? ds * acc[q][2 * q2] : TACC(0), vb ? ds * acc[q][2 * q2 + 1] : TACC(0)};
              }
            }
          }
        }
        __syncthreads();
        V* src = fbuf;
        V* dst = fbuf + l1;
        for (int st = 0; st < plan.nstages; ++st) {
          stockham_stage_batch<V, TACC>(src, dst, 2 * l1, nbat, l1, plan, st, twsm, threadIdx.x, blockDim.x);
          __syncthreads();
          V* tmp = src;
          src = dst;
          dst = tmp;
        }
        for (int idx = tid; idx < nbat * l; idx += NT) {
          const int qb = (int)fdiv((uint32_t)idx, ml, (uint32_t)l), cidx = idx - qb * l;
          const V* zz = src + (size_t)qb * 2 * l1;
          const int q2 = q0 + qb;
          const int64_t ra = row0 + 2 * q2, rb = ra + 1;
          const int f = Rsel[cidx];
          const int fm = f == 0 ? 0 : l1 - f;
          const V z = zz[f], w = zz[fm];
          const TACC h1 = TACC(0.5) * ((z.x + w.x) - (z.y - w.y));
          const TACC h2 = TACC(0.5) * ((z.x - w.x) + (z.y + w.y));
          if (2 * q2 < rows) Y[(rowmap ? (int64_t)rowmap[ra] : ra) * l + cidx] = (double)(h1 * scale);
          if (2 * q2 + 1 < rows) Y[(rowmap ? (int64_t)rowmap[rb] : rb) * l + cidx] = (double)(h2 * scale);
        }
      }
#pragma unroll
      for (int q = 0; q < NB; ++q)
#pragma unroll
        for (int r = 0; r < R; ++r) acc[q][r] = TACC(0);
    }
    __syncthreads();  // every thread is done with stage s before it is refilled
  }
  if (bad) set_flag(status, FLAG_NONFINITE);
  if (tid == 0 && s_fail) set_flag(status, FLAG_TIMEOUT);
}

// ---------------------------------------------------------------------------
// Fused dense sketch over whole rows (rows that fit in shared memory): warp 0
// streams rows of A into an S-slot ring with one bulk copy per row (full /
// empty mbarriers per slot); the other warps sum each row's buckets (bucket b
// owned by one thread: its columns in ascending order, the same order as the
// chunked kernels, with the bucket lists built for a single chunk = n) and
// write d_b times the sum straight into the FFT buffer of its row pair (real
// part for the even row, imaginary for the odd one).  After 2 pb rows the
// batch of pb complex FFTs runs on the summing warps (named barrier 1) while
// the ring keeps filling; the Hartley outputs of the selected frequencies go
// to Y.  Nothing is kept in registers across rows.
// For n < 32768 each CTA first lays the bucket lists out in shared memory as
// 16-bit entries (column | sign << 15): buckets sorted by length (longest
// first) in groups of 32, one group per warp pass, the t-th entries of a
// group's 32 buckets side by side (padded with 0xffff), so a warp reads 32
// entries in one access and its lanes run for about the same number of
// entries.  A bucket is still summed by one thread in ascending column order,
// so the sums are the same as with plain lists.  Lists that do not fit that
// layout (a bucket longer than 255 entries, or too much padding: not expected
// at the at most 32 entries per bucket on average that the host allows) are
// kept as plain 16-bit lists; for n >= 32768 they are read through L1.
// ---------------------------------------------------------------------------
constexpr int kRowSlotsMax = 4;

// OR of `v` over the `nthr` threads of named barrier 1 (also a barrier).
__device__ __forceinline__ bool bar1_any(bool v, int nthr) {
  unsigned int r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((unsigned int)v), "r"(nthr)
      : "memory");
  return r != 0;
}

template <typename TA, typename TACC, int NT>
__global__ void __launch_bounds__(NT, 1) k_sketch_rows(const TA* __restrict__ A, int64_t lda, int64_t m, int64_t n,
                                                    int l1, int l, const int32_t* __restrict__ bstart,
                                                    const uint32_t* __restrict__ blist,
                                                    const float* __restrict__ dsign, const int32_t* __restrict__ Rsel,
                                                    const typename C2<TACC>::t* __restrict__ tw, FftPlan plan, int pb,
                                                    int nslots, int lists16, double* __restrict__ Y,
                                                    const int32_t* __restrict__ rowmap, unsigned int* status) {
  using V = typename C2<TACC>::t;
  constexpr int NC = NT - 32;  // summing / FFT threads
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kRowSlotsMax], empty[kRowSlotsMax];
  __shared__ int s_fail;
  __shared__ long long s_used;  // rows the summing warps have taken from the ring
  const size_t rowb = (size_t)n * sizeof(TA);
  TA* ring = reinterpret_cast<TA*>(smem);                              // [nslots][n]
  V* twsm = reinterpret_cast<V*>(smem + (size_t)nslots * rowb);       // l1 twiddles
  V* fbuf = twsm + l1;                                                 // [pb][2][l1]
  TACC* zs = reinterpret_cast<TACC*>(fbuf);                            // scalar view
  // list area: transposed layout = group offsets (ngroups + 1, int) | slot ->
  // bucket (l1, u16) | entries (n + 1024, u16); plain layout = starts (l1 + 1,
  // u16) | entries (n, u16), over the same bytes
  const int ngroups = (l1 + 31) >> 5;
  int* goff = reinterpret_cast<int*>(fbuf + (size_t)pb * 2 * l1);
  uint16_t* ord16 = reinterpret_cast<uint16_t*>(goff + ngroups + 1);
  uint16_t* tl16 = ord16 + l1;
  const int tcap = (int)n + 1024;
  uint16_t* st16 = reinterpret_cast<uint16_t*>(goff);
  uint16_t* ls16 = st16 + l1 + 1;
  __shared__ int s_hist[256];
  __shared__ int s_plain;
  const int tid = threadIdx.x, lane = tid & 31;
  const int64_t rows_per_batch = 2 * (int64_t)pb;
  const int64_t nbatches = cdiv(m, rows_per_batch);
  const TACC scale = TACC(1) / sqrt(TACC(l1));
  const uint32_t ml = div_magic(l);
  if (tid == 0) {
    for (int s = 0; s < nslots; ++s) {
      sk_mbar_init(&full[s], 1);
      sk_mbar_init(&empty[s], 1);
    }
    s_fail = 0;
    s_used = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int e = tid; e < l1; e += NT) twsm[e] = tw[e];
  auto enc16 = [](uint32_t ent) -> uint16_t { return (uint16_t)((ent & 0x7fffu) | ((ent >> 31) << 15)); };
  if (lists16) {
    // counting sort of the buckets by length, longest first
    for (int i = tid; i < 256; i += NT) s_hist[i] = 0;
    if (tid == 0) s_plain = 0;
    __syncthreads();
    for (int b = tid; b < l1; b += NT) {
      const int len = bstart[b + 1] - bstart[b];
      if (len > 255) s_plain = 1;
      else atomicAdd(&s_hist[255 - len], 1);
    }
    __syncthreads();
    if (tid < 32) {  // exclusive scan of the 256 bins, 8 per lane
      int v[8], sum = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) { v[i] = s_hist[lane * 8 + i]; sum += v[i]; }
      int inc = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
      }
      int run = inc - sum;
#pragma unroll
      for (int i = 0; i < 8; ++i) { s_hist[lane * 8 + i] = run; run += v[i]; }
    }
    __syncthreads();
    if (!s_plain)
      for (int b = tid; b < l1; b += NT) {
        const int len = bstart[b + 1] - bstart[b];
        ord16[atomicAdd(&s_hist[255 - len], 1)] = (uint16_t)b;
      }
    __syncthreads();
    if (!s_plain && tid < 32) {  // group offsets: 32 x the length of each group's first (longest) bucket
      int run = 0;
      for (int g0 = 0; g0 < ngroups; g0 += 32) {
        const int g = g0 + lane;
        int w = 0;
        if (g < ngroups) {
          const int b = ord16[32 * g];
          w = 32 * (bstart[b + 1] - bstart[b]);
        }
        int inc = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int t = __shfl_up_sync(0xffffffffu, inc, o);
          if (lane >= o) inc += t;
        }
        if (g < ngroups) goff[g] = run + inc - w;
        run += __shfl_sync(0xffffffffu, inc, 31);
      }
      if (lane == 0) {
        goff[ngroups] = run;
        if (run > tcap) s_plain = 1;
      }
    }
    __syncthreads();
    if (!s_plain) {
      for (int k = tid; k < 32 * ngroups; k += NT) {
        const int g = k >> 5, ln = k & 31;
        const int L = (goff[g + 1] - goff[g]) >> 5;
        const int b = k < l1 ? (int)ord16[k] : -1;
        const int e0 = b >= 0 ? bstart[b] : 0, len = b >= 0 ? bstart[b + 1] - e0 : 0;
        for (int it = 0; it < L; ++it) tl16[goff[g] + it * 32 + ln] = it < len ? enc16(blist[e0 + it]) : (uint16_t)0xffffu;
      }
    } else {
      for (int b = tid; b <= l1; b += NT) st16[b] = (uint16_t)bstart[b];
      for (int64_t e = tid; e < n; e += NT) ls16[e] = enc16(blist[e]);
    }
  }
  __syncthreads();
  const bool transposed = lists16 && !s_plain;

  long long issued = 0;
  if (tid < 32) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      for (int64_t bt = blockIdx.x; bt < nbatches; bt += gridDim.x) {
        const int64_t row0 = bt * rows_per_batch;
        const int rows = (int)min64(rows_per_batch, m - row0);
        bool quit = false;
        for (int rr = 0; rr < rows; ++rr) {
          const int s = (int)(issued % nslots);
          // the slot's previous row has been summed (bounded; the summing
          // warps raise s_fail if they stop early)
          if (issued >= nslots && !sk_mbar_wait(&empty[s], (uint32_t)(((issued / nslots) - 1) & 1))) {
            quit = true;
            break;
          }
          if (*(volatile int*)&s_fail) { quit = true; break; }
          sk_mbar_expect_tx(&full[s], (uint32_t)rowb);
          bulk_g2s(ring + (size_t)s * n, A + (row0 + rr) * lda, (uint32_t)rowb, &full[s]);
          ++issued;
        }
        if (quit) break;
      }
    }
  } else {
    // ------------------------------------------------------------ summing and FFT warps
    const int ct = tid - 32;
    long long used = 0;
    int slot = 0;         // ring slot of row `used`
    uint32_t phase = 0;   // its fill parity
    bool bad = false, stop = false;
    for (int64_t bt = blockIdx.x; bt < nbatches && !stop; bt += gridDim.x) {
      const int64_t row0 = bt * rows_per_batch;
      const int rows = (int)min64(rows_per_batch, m - row0);
      for (int rr = 0; rr < (int)rows_per_batch; ++rr) {
        const int qb = rr >> 1, part = rr & 1;
        if (rr >= rows) {  // past the last row: that half of the pair is zero
          for (int b = ct; b < l1; b += NC) zs[2 * ((size_t)qb * 2 * l1 + b) + part] = TACC(0);
          continue;
        }
        const int s = slot;
        const bool ok = sk_mbar_wait(&full[s], phase);
        if (ok) {
          const TA* row = ring + (size_t)s * n;
          if (transposed) {
            // warp pass over group g: lane = bucket slot, entries 32 apart
            for (int g = ct >> 5; g < ngroups; g += NC / 32) {
              const int base = goff[g], L = (goff[g + 1] - base) >> 5;
              const uint16_t* pl = tl16 + base + (ct & 31);
              TACC acc = TACC(0);
              int it = 0;
              for (; it + 4 <= L; it += 4) {
                uint16_t x[4];
                TACC v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) x[u] = pl[(it + u) * 32];
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = x[u] != 0xffffu ? load_acc(row + (x[u] & 0x7fffu), TACC(0)) : TACC(0);
#pragma unroll
                for (int u = 0; u < 4; ++u)
                  if (x[u] != 0xffffu) acc = fma((x[u] >> 15) ? TACC(-1) : TACC(1), v[u], acc);
              }
              for (; it < L; ++it) {
                const uint16_t x = pl[it * 32];
                if (x != 0xffffu) acc = fma((x >> 15) ? TACC(-1) : TACC(1), load_acc(row + (x & 0x7fffu), TACC(0)), acc);
              }
              const int k = 32 * g + (ct & 31);
              if (k < l1) {
                const int b = ord16[k];
                bad |= !isfinite(acc);
                zs[2 * ((size_t)qb * 2 * l1 + b) + part] = (TACC)dsign[b] * acc;
              }
            }
          } else
          for (int b = ct; b < l1; b += NC) {
            // entries in ascending column order, four loads in flight at a time
            TACC acc = TACC(0);
            if (lists16) {
              const int e0 = st16[b], e1 = st16[b + 1];
              int e = e0;
              for (; e + 4 <= e1; e += 4) {
                uint16_t x[4];
                TACC v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) x[u] = ls16[e + u];
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = load_acc(row + (x[u] & 0x7fffu), TACC(0));
#pragma unroll
                for (int u = 0; u < 4; ++u) acc = fma((x[u] >> 15) ? TACC(-1) : TACC(1), v[u], acc);
              }
              for (; e < e1; ++e) {
                const uint16_t x = ls16[e];
                acc = fma((x >> 15) ? TACC(-1) : TACC(1), load_acc(row + (x & 0x7fffu), TACC(0)), acc);
              }
            } else {
              const int e0 = __ldg(bstart + b), e1 = __ldg(bstart + b + 1);
              int e = e0;
              for (; e + 4 <= e1; e += 4) {
                uint32_t x[4];
                TACC v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) x[u] = __ldg(blist + e + u);
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = load_acc(row + (x[u] & 0x7fffffffu), TACC(0));
#pragma unroll
                for (int u = 0; u < 4; ++u) acc = fma((x[u] >> 31) ? TACC(-1) : TACC(1), v[u], acc);
              }
              for (; e < e1; ++e) {
                const uint32_t x = __ldg(blist + e);
                acc = fma((x >> 31) ? TACC(-1) : TACC(1), load_acc(row + (x & 0x7fffffffu), TACC(0)), acc);
              }
            }
            bad |= !isfinite(acc);
            zs[2 * ((size_t)qb * 2 * l1 + b) + part] = (TACC)dsign[b] * acc;
          }
        }
        // every summing thread is done with slot s (or one of them timed out)
        if (bar1_any(!ok, NC)) {
          stop = true;
          break;
        }
        ++used;
        if (++slot == nslots) { slot = 0; phase ^= 1u; }
        if (ct == 0) sk_mbar_arrive(&empty[s]);
      }
      if (stop) break;
      // the batch's FFTs (pairs past the last row are not needed)
      const int nbat = (rows + 1) / 2;
      V* src = fbuf;
      V* dst = fbuf + l1;
      for (int st = 0; st < plan.nstages; ++st) {
        stockham_stage_batch<V, TACC>(src, dst, 2 * l1, nbat, l1, plan, st, twsm, ct, NC);
        asm volatile("bar.sync 1, %0;" ::"r"(NC) : "memory");
        V* tmp = src;
        src = dst;
        dst = tmp;
      }
      for (int idx = ct; idx < nbat * l; idx += NC) {
        const int q = (int)fdiv((uint32_t)idx, ml, (uint32_t)l), cidx = idx - q * l;
        const V* zz = src + (size_t)q * 2 * l1;
        const int64_t ra = row0 + 2 * q, rb = ra + 1;
        const int f = Rsel[cidx];
        const int fm = f == 0 ? 0 : l1 - f;
        const V z = zz[f], w = zz[fm];
        const TACC h1 = TACC(0.5) * ((z.x + w.x) - (z.y - w.y));
        const TACC h2 = TACC(0.5) * ((z.x - w.x) + (z.y + w.y));
        Y[(rowmap ? (int64_t)rowmap[ra] : ra) * l + cidx] = (double)(h1 * scale);
        if (rb < m) Y[(rowmap ? (int64_t)rowmap[rb] : rb) * l + cidx] = (double)(h2 * scale);
      }
      // the next batch writes the FFT inputs again
      asm volatile("bar.sync 1, %0;" ::"r"(NC) : "memory");
    }
    if (bad) set_flag(status, FLAG_NONFINITE);
    if (ct == 0) {
      if (stop) {
        *(volatile int*)&s_fail = 1;
        set_flag(status, FLAG_TIMEOUT);
      }
      s_used = used;
    }
  }
  __syncthreads();
  // copies still in flight (only after a failure): wait for them (bounded)
  // before the CTA's shared memory is released
  if (tid == 0) {
    for (long long u = s_used; u < issued; ++u) sk_mbar_wait(&full[u % nslots], (uint32_t)((u / nslots) & 1));
  }
}

// ---------------------------------------------------------------------------
// CSR sketch.  Rows are split by the host side into light rows (a warp per
// row) and heavy rows (at least n/4 entries).  A warp scatters 32 entries of
// a light row at a time into the row's buckets in shared memory; lanes whose
// bucket no other lane of the round hits add directly, colliding lanes add one
// after another in lane order, so every bucket sums its entries in a fixed
// order; then the Hartley transforms of row pairs run as in the dense sketch.
// Heavy rows are densified (they are needed densely for the tensor-core
// product anyway) and sketched by the dense kernels.
template <typename TV, typename TACC>
__device__ __forceinline__ void csr_scatter_warp(const int32_t* __restrict__ colind, const TV* __restrict__ val,
                                                 int64_t e0, int64_t e1, int64_t n, const uint32_t* __restrict__ hs,
                                                 TACC* __restrict__ y1, TV* __restrict__ drow, bool& bad_csr,
                                                 bool& bad_val, bool* increasing = nullptr) {
  const int lane = threadIdx.x & 31;
  int prev_last = -1;  // last column of the previous round (for the strict-increase check)
  bool inc = true;
  for (int64_t base = e0; base < e1; base += 32) {
    const int64_t e = base + lane;
    bool valid = e < e1;
    int col = 0;
    TACC x = TACC(0);
    int b = -1 - lane;  // unique key for lanes without an entry
    if (valid) {
      col = colind[e];
      const TV v = val[e];
      if (col < 0 || (int64_t)col >= n) {
        bad_csr = true;
        valid = false;
      } else {
        bad_val |= !finite_(v);
        const uint32_t h = hs[col];
        b = (int)(h & 0x7fffffffu);
        x = (h >> 31) ? -(TACC)v : (TACC)v;
        if (drow) drow[col] = v;
      }
    }
    if (increasing) {
      const int c_prev = __shfl_up_sync(0xffffffffu, col, 1);
      const int before = lane == 0 ? prev_last : c_prev;
      if (e < e1 && col <= before) inc = false;
      const int64_t last = min64(31, e1 - 1 - base);
      prev_last = __shfl_sync(0xffffffffu, col, (int)last);
    }
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const bool collide = valid && __popc(peers) > 1;
    if (valid && !collide) y1[b] += x;
    if (__any_sync(0xffffffffu, collide)) {
      for (int src = 0; src < 32; ++src) {
        if (lane == src && collide) y1[b] += x;
        __syncwarp();
      }
    }
    __syncwarp();
  }
  if (increasing) *increasing = __all_sync(0xffffffffu, inc);
}

// Hartley transforms of `np` row pairs stored in yrows[2*np][l1] (TACC), rows
// out of range zero; writes Y[row[q] * l + c].
template <typename TACC>
__device__ void csr_pairs_fft(const TACC* __restrict__ yrows, int np, const int32_t* rows, int l1, int l,
                              const float* __restrict__ dsign, const int32_t* __restrict__ Rsel,
                              const typename C2<TACC>::t* twsm, typename C2<TACC>::t* fbuf, int pb, FftPlan plan,
                              double* __restrict__ Y) {
  using V = typename C2<TACC>::t;
  const TACC scale = TACC(1) / sqrt(TACC(l1));
  const uint32_t ml = div_magic(l), ml1 = div_magic(l1);
  for (int q0 = 0; q0 < np; q0 += pb) {
    const int nbat = min(pb, np - q0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nbat * l1; idx += blockDim.x) {
      const int qb = (int)fdiv((uint32_t)idx, ml1, (uint32_t)l1), b = idx - qb * l1;
      const int q2 = q0 + qb;
      const TACC ds = (TACC)dsign[b];
      fbuf[(size_t)qb * 2 * l1 + b] = V{ds * yrows[(size_t)(2 * q2) * l1 + b], ds * yrows[(size_t)(2 * q2 + 1) * l1 + b]};
    }
    __syncthreads();
    V* src = fbuf;
    V* dst = fbuf + l1;
    for (int st = 0; st < plan.nstages; ++st) {
      stockham_stage_batch<V, TACC>(src, dst, 2 * l1, nbat, l1, plan, st, twsm, threadIdx.x, blockDim.x);
      __syncthreads();
      V* tmp = src;
      src = dst;
      dst = tmp;
    }
    for (int idx = threadIdx.x; idx < nbat * l; idx += blockDim.x) {
      const int qb = (int)fdiv((uint32_t)idx, ml, (uint32_t)l), cidx = idx - qb * l;
      const V* zz = src + (size_t)qb * 2 * l1;
      const int q2 = q0 + qb;
      const int f = Rsel[cidx];
      const int fm = f == 0 ? 0 : l1 - f;
      const V z = zz[f], w = zz[fm];
      const TACC h1 = TACC(0.5) * ((z.x + w.x) - (z.y - w.y));
      const TACC h2 = TACC(0.5) * ((z.x - w.x) + (z.y + w.y));
      const int ra = rows[2 * q2], rb = rows[2 * q2 + 1];
      if (ra >= 0) Y[(int64_t)ra * l + cidx] = (double)(h1 * scale);
      if (rb >= 0) Y[(int64_t)rb * l + cidx] = (double)(h2 * scale);
    }
  }
  __syncthreads();
}

constexpr int kCsrWarps = 16;

// Light rows: warp w of a group takes row list[g * kCsrWarps + w].
template <typename TV, typename TACC>
__global__ void __launch_bounds__(kCsrWarps * 32, 1)
    k_sketch_csr_light(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                       const TV* __restrict__ val, int64_t n, const int32_t* __restrict__ list, const int32_t* count,
                       int l1, int l, const uint32_t* __restrict__ hs, const float* __restrict__ dsign,
                       const int32_t* __restrict__ Rsel, const typename C2<TACC>::t* __restrict__ tw, FftPlan plan,
                       int pb, double* __restrict__ Y, unsigned int* status) {
  using V = typename C2<TACC>::t;
  extern __shared__ __align__(16) unsigned char smem[];
  V* twsm = reinterpret_cast<V*>(smem);
  V* fbuf = twsm + l1;
  TACC* y1 = reinterpret_cast<TACC*>(fbuf + (size_t)pb * 2 * l1);  // [kCsrWarps][l1]
  __shared__ int32_t rows[kCsrWarps];
  const int warp = threadIdx.x >> 5;
  const int nrows = *count;
  const int ngroups = (nrows + kCsrWarps - 1) / kCsrWarps;
  for (int e = threadIdx.x; e < l1; e += blockDim.x) twsm[e] = tw[e];
  bool bad_csr = false, bad_val = false;
  for (int g = blockIdx.x; g < ngroups; g += gridDim.x) {
    __syncthreads();
    const int li = g * kCsrWarps + warp;
    const int row = li < nrows ? list[li] : -1;
    if ((threadIdx.x & 31) == 0) rows[warp] = row;
    TACC* my = y1 + (size_t)warp * l1;
    for (int b = threadIdx.x & 31; b < l1; b += 32) my[b] = TACC(0);
    __syncwarp();
    if (row >= 0) {
      const int64_t e0 = rowptr[row], e1 = rowptr[row + 1];
      csr_scatter_warp<TV, TACC>(colind, val, e0, e1, n, hs, my, (TV*)nullptr, bad_csr, bad_val);
    }
    __syncthreads();
    csr_pairs_fft<TACC>(y1, kCsrWarps / 2, rows, l1, l, dsign, Rsel, twsm, fbuf, pb, plan, Y);
  }
  if (bad_csr) set_flag(status, FLAG_BAD_CSR);
  if (bad_val) set_flag(status, FLAG_NONFINITE);
}

// Sparse light rows by direct evaluation: with T[b][c] = d(b) cas(2 pi b R_c /
// l1) / sqrt(l1) (the l1 x l matrix D H R / sqrt(l1)), row i of the sketch is
// Y[i][c] = sum over the row's entries (j, v) of s(j) v T[h(j)][c], the same
// linear map as the bucket sums followed by the transform, at nnz x l
// multiply-adds per row instead of an l1-point FFT.  T is built from the FFT
// twiddles (cas(2 pi t / l1) = Re w^t - Im w^t with w = exp(-2 pi i / l1)).
__global__ void k_fjl_table(int l1, int l, const float* __restrict__ dsign, const int32_t* __restrict__ Rsel,
                            const float2* __restrict__ tw, float* __restrict__ T) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)l1 * l) return;
  const int b = (int)(e / l), c = (int)(e - (int64_t)b * l);
  const int t = (int)(((int64_t)b * Rsel[c]) % l1);
  const float2 w = tw[t];
  T[e] = dsign[b] * (w.x - w.y) * rsqrtf((float)l1);
}

// A CTA holds the columns [c0, c0 + lg) of T in shared memory (blockIdx.y
// picks the group); warp w of CTA x takes kDirRows light rows at a time
// (those with at most direct_max entries), so that the dependent loads of
// four rows (list, row pointers, entries, hash) are in flight together.
// Lanes own the columns; each round of 32 entries per row is staged as
// (bucket, signed value) pairs and read back by every lane in entry order, one
// accumulator per row (a fixed order: results repeat bit for bit).  Staged
// slots past a row's end hold (0, 0) and add nothing.
constexpr int kDirWarps = 32;
constexpr int kDirRows = 4;
template <typename TV>
__global__ void __launch_bounds__(kDirWarps * 32, 1)
    k_sketch_csr_direct(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                        const TV* __restrict__ val, int64_t n, const int32_t* __restrict__ list,
                        const int32_t* count, int64_t direct_max, int l1, int l, int lg,
                        const float* __restrict__ T, const uint32_t* __restrict__ hs, double* __restrict__ Y,
                        unsigned int* status) {
  // l1 x lg, then 32 zeros: lane t reads Ts[b lg + t] for every t < 32, which
  // for lg < 32 runs past row b (into row b + 1, or the zero pad after the
  // last row); those lanes' sums are never stored
  extern __shared__ __align__(16) float Ts[];
  __shared__ int2 stage[kDirWarps][kDirRows][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c0 = blockIdx.y * lg;
  const int ncols = min(lg, l - c0);
  for (int64_t e = threadIdx.x; e < (int64_t)l1 * lg + 32; e += blockDim.x) {
    const int b = (int)(e / lg), cc = (int)(e - (int64_t)b * lg);
    Ts[e] = (b < l1 && cc < ncols) ? T[(int64_t)b * l + c0 + cc] : 0.f;
  }
  __syncthreads();
  const int nrows = *count;
  bool bad_csr = false, bad_val = false;
  const int64_t step = (int64_t)gridDim.x * kDirWarps * kDirRows;
  for (int64_t li0 = ((int64_t)blockIdx.x * kDirWarps + warp) * kDirRows; li0 < nrows; li0 += step) {
    int row[kDirRows];
    int64_t e0[kDirRows], len[kDirRows];
    int64_t len_max = 0;
#pragma unroll
    for (int q = 0; q < kDirRows; ++q) {
      row[q] = li0 + q < nrows ? list[li0 + q] : -1;
      e0[q] = 0;
      len[q] = 0;
      if (row[q] >= 0) {
        const int64_t a = rowptr[row[q]], z = rowptr[row[q] + 1];
        if (z - a <= direct_max) {  // longer rows (mid) are the FFT kernel's
          e0[q] = a;
          len[q] = z - a;
        } else {
          row[q] = -1;
        }
      }
      len_max = max(len_max, len[q]);
    }
    float acc[kDirRows];
#pragma unroll
    for (int q = 0; q < kDirRows; ++q) acc[q] = 0.f;
    for (int64_t base = 0; base < len_max; base += 32) {
#pragma unroll
      for (int q = 0; q < kDirRows; ++q) {
        int b = 0;
        float x = 0.f;
        if (base + lane < len[q]) {
          const int64_t e = e0[q] + base + lane;
          const int col = colind[e];
          if (col < 0 || (int64_t)col >= n) {
            bad_csr = true;
          } else {
            const TV v = val[e];
            bad_val |= !finite_(v);
            const uint32_t h = hs[col];
            b = (int)(h & 0x7fffffffu);
            x = (h >> 31) ? -(float)v : (float)v;
          }
        }
        stage[warp][q][lane] = make_int2(b * lg, __float_as_int(x));
      }
      __syncwarp();
      const int cnt = (int)min64(32, len_max - base);
      for (int t = 0; t < cnt; ++t) {
#pragma unroll
        for (int q = 0; q < kDirRows; ++q) {
          const int2 p = stage[warp][q][t];
          acc[q] = fmaf(__int_as_float(p.y), Ts[p.x + lane], acc[q]);
        }
      }
      __syncwarp();
    }
#pragma unroll
    for (int q = 0; q < kDirRows; ++q)
      if (row[q] >= 0 && lane < ncols) Y[(int64_t)row[q] * l + c0 + lane] = (double)acc[q];
  }
  if (bad_csr) set_flag(status, FLAG_BAD_CSR);
  if (bad_val) set_flag(status, FLAG_NONFINITE);
}

// Heavy rows: densified, a CTA per row, into D (row i of D = heavy row
// list[i], n columns; repeated coordinates summed), then sketched by the dense
// kernels with the row map list.  A row with exactly n strictly increasing
// columns is a plain copy; otherwise zeros, then stores, and if the columns
// are not strictly increasing, zeros again and atomic adds.
template <typename TV>
__global__ void __launch_bounds__(512) k_csr_densify(const int64_t* __restrict__ rowptr,
                                                     const int32_t* __restrict__ colind, const TV* __restrict__ val,
                                                     int64_t n, const int32_t* __restrict__ list, const int32_t* count,
                                                     TV* __restrict__ D, unsigned int* status) {
  const int nrows = *count;
  bool bad_csr = false;
  for (int i = blockIdx.x; i < nrows; i += gridDim.x) {
    const int row = list[i];
    TV* drow = D + (int64_t)i * n;
    const int64_t e0 = rowptr[row], e1 = rowptr[row + 1];
    if (e1 - e0 != n)
      for (int64_t c = threadIdx.x; c < n; c += blockDim.x) drow[c] = TV(0);
    __syncthreads();
    int inc = 1;
    // eight independent entries per thread in flight: all loads, then the stores
    constexpr int U = 8;
    for (int64_t base = e0 + threadIdx.x; base < e1; base += (int64_t)blockDim.x * U) {
      int cu[U], cp[U];
      TV vu[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t e = base + (int64_t)u * blockDim.x;
        if (e < e1) {
          cu[u] = colind[e];
          cp[u] = e > e0 ? colind[e - 1] : -1;
          vu[u] = val[e];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t e = base + (int64_t)u * blockDim.x;
        if (e < e1) {
          const int c = cu[u];
          if (c < 0 || (int64_t)c >= n) {
            bad_csr = true;
            continue;
          }
          if (cp[u] >= c) inc = 0;
          drow[c] = vu[u];
        }
      }
    }
    if (!__syncthreads_and(inc)) {  // repeated or unordered columns: rebuild with sums
      for (int64_t c = threadIdx.x; c < n; c += blockDim.x) drow[c] = TV(0);
      __syncthreads();
      for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const int c = colind[e];
        if (c >= 0 && (int64_t)c < n) atomicAdd(drow + c, val[e]);
      }
    }
    __syncthreads();
  }
  if (bad_csr) set_flag(status, FLAG_BAD_CSR);
}

template <typename TV, typename TACC>
static int launch_csr_cfg(const int64_t* rowptr, const int32_t* colind, const TV* val, int64_t n, const CsrRows& cr,
                          int l1, int l, const SketchWs& ws, TV* D, double* Y, float* table, unsigned int* status,
                          int num_sms, cudaStream_t st) {
  using V = typename C2<TACC>::t;
  const typename C2<TACC>::t* tw;
  if constexpr (sizeof(TACC) == 8) tw = ws.tw64; else tw = ws.tw32;
  const size_t budget = 220 * 1024;
  if constexpr (sizeof(TACC) == 4) {
    if (cr.direct_max >= 0 && cr.n_light > cr.n_mid) {
      if (!table) return RLU_EINVAL;
      k_fjl_table<<<(unsigned)cdiv((int64_t)l1 * l, 256), 256, 0, st>>>(l1, l, ws.dsign, ws.R, ws.tw32, table);
      RLU_CUDA_TRY(cudaGetLastError());
      note_launch();
      // column groups of at most 32 (a lane each) whose slice of T fits in shared
      // memory beside the 32 KB of staged entries
      const int lg_max = (int)min64(32, ((int64_t)(190 * 1024) - 128) / (4 * (int64_t)l1));
      if (lg_max < 1) return RLU_EINVAL;
      const int G = (int)cdiv(l, lg_max);
      const int lg = (int)cdiv(l, G);
      const size_t smem = (size_t)4 * ((size_t)l1 * lg + 32);  // the table slice and its zero pad
      auto kern = k_sketch_csr_direct<TV>;
      if (int rc_ = allow_dynamic_smem((const void*)kern, smem)) return rc_;
      const int64_t per_group = min64(cdiv(cr.n_light, (int64_t)kDirWarps * kDirRows), max64(1, cdiv((int64_t)num_sms, G)));
      kern<<<dim3((unsigned)per_group, (unsigned)G), kDirWarps * 32, smem, st>>>(
          rowptr, colind, val, n, cr.light, cr.d_count, cr.direct_max, l1, l, lg, table, ws.hs, Y, status);
      RLU_CUDA_TRY(cudaGetLastError());
      note_launch();
    }
  }
  if (cr.n_mid > 0) {
    auto kern = k_sketch_csr_light<TV, TACC>;
    const size_t fixed = (size_t)l1 * sizeof(V) + (size_t)kCsrWarps * l1 * sizeof(TACC);
    const size_t per_pair = (size_t)2 * l1 * sizeof(V);
    if (fixed + per_pair > budget) return RLU_EINVAL;
    int pb = (int)((budget - fixed) / per_pair);
    if (pb > kCsrWarps / 2) pb = kCsrWarps / 2;
    const size_t smem = fixed + (size_t)pb * per_pair;
    if (int rc_ = allow_dynamic_smem((const void*)kern, smem)) return rc_;
    const int64_t groups = cdiv(cr.n_mid, kCsrWarps);
    const unsigned grid = (unsigned)min64(groups, (int64_t)num_sms);
    kern<<<grid, kCsrWarps * 32, smem, st>>>(rowptr, colind, val, n, cr.mid, cr.d_count + 2, l1, l, ws.hs, ws.dsign,
                                             ws.R, tw, ws.plan, pb, Y, status);
    RLU_CUDA_TRY(cudaGetLastError());
    note_launch();
  }
  if (cr.n_heavy > 0) {
    const unsigned grid = (unsigned)min64(cr.n_heavy, (int64_t)num_sms * 4);
    k_csr_densify<TV><<<grid, 512, 0, st>>>(rowptr, colind, val, n, cr.heavy, cr.d_count + 1, D, status);
    RLU_CUDA_TRY(cudaGetLastError());
    note_launch();
    const int dt = std::is_same<TV, double>::value ? RLU_F64 : RLU_F32;
    int rc = launch_sketch_dense(D, n, dt, dt == RLU_F64, cr.n_heavy, n, l1, l, ws, Y, status, num_sms, st,
                                 cr.heavy);
    if (rc) return rc;
  }
  return RLU_OK;
}

int launch_sketch_csr(const int64_t* rowptr, const int32_t* colind, const void* val, int dtype, int64_t n,
                      const CsrRows& cr, int l1, int l, const SketchWs& ws, void* D, double* Y, float* table,
                      unsigned int* status, int num_sms, cudaStream_t st) {
  if (dtype == RLU_F64)
    return launch_csr_cfg<double, double>(rowptr, colind, (const double*)val, n, cr, l1, l, ws, (double*)D, Y,
                                          table, status, num_sms, st);
  if (dtype == RLU_F32)
    return launch_csr_cfg<float, float>(rowptr, colind, (const float*)val, n, cr, l1, l, ws, (float*)D, Y, table,
                                        status, num_sms, st);
  return RLU_EINVAL;
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
FftPlan make_fft_plan(int N) {
  FftPlan pl{};
  int x = N;
  auto push = [&](int r) { pl.radix[pl.nstages++] = r; };
  while (x % 4 == 0) { push(4); x /= 4; }
  while (x % 2 == 0) { push(2); x /= 2; }
  for (int f = 3; x > 1; f += 2) {
    while (x % f == 0) { push(f); x /= f; }
  }
  int p = 1;
  for (int s = 0; s < pl.nstages; ++s) {
    const int r = pl.radix[s];
    pl.p[s] = p;
    pl.T[s] = N / r;
    pl.step[s] = N / (p * r);
    pl.mT[s] = div_magic(N / r);
    pl.mp[s] = div_magic(p);
    p *= r;
  }
  return pl;
}

int launch_sketch_params(const SketchWs& ws, int64_t n, int l1, int l, uint64_t seed, cudaStream_t st) {
  int64_t cnt = n > l1 ? n : l1;
  k_sketch_params<<<(unsigned)cdiv(cnt, 256), 256, 0, st>>>(n, l1, seed, ws.hs, ws.dsign, ws.keys);
  k_select_R<<<(unsigned)cdiv((int64_t)l1 * 32, 256), 256, 0, st>>>(l1, l, ws.keys, ws.R);
  // bucket lists for the dense path
  const int64_t nsb = ws.nchunks * (int64_t)l1;
  if (nsb <= kListsOneMax) {
    const size_t smem = sizeof(int) * (size_t)(2 * nsb + 1);
    if (int rc_ = allow_dynamic_smem((const void*)k_bucket_lists_one, smem)) return rc_;
    k_bucket_lists_one<<<1, 1024, smem, st>>>(n, l1, ws.chunk, (int)nsb, ws.hs, ws.bstart, ws.blist);
    RLU_CUDA_TRY(cudaGetLastError());
    note_launch(3);
    return RLU_OK;
  }
  RLU_CUDA_TRY(cudaMemsetAsync(ws.bcnt, 0, sizeof(int32_t) * (nsb + 1), st));
  k_bucket_count<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(n, l1, ws.chunk, ws.hs, ws.bcnt);
  note_launch();
  if (int rc_ = launch_scan_i32(nsb, ws.bcnt, ws.bstart, ws.scan_tmp, st)) return rc_;
  RLU_CUDA_TRY(cudaMemsetAsync(ws.bcnt, 0, sizeof(int32_t) * (nsb + 1), st));
  k_bucket_fill<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(n, l1, ws.chunk, ws.hs, ws.bstart, ws.bcnt, ws.blist);
  k_bucket_sort<<<(unsigned)cdiv(nsb, 256), 256, 0, st>>>(nsb, ws.bstart, ws.blist);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch(4);
  return RLU_OK;
}

int launch_scan_i32(int64_t count, const int32_t* cnt, int32_t* start, int64_t* tmp, cudaStream_t st) {
  if (!tmp) {  // no scratch (the allocation-free sketch): one CTA
    k_scan_counts<<<1, 1024, 0, st>>>(count, cnt, start);
    RLU_CUDA_TRY(cudaGetLastError());
    note_launch();
    return RLU_OK;
  }
  // rounds of 1024 values, as few per CTA as kScanMaxParts CTAs allow (the
  // rounds of one CTA run one after another)
  const int64_t per = max64(1024, cdiv(cdiv(max64(count, 1), kScanMaxParts), 1024) * 1024);
  const int64_t parts = max64(1, cdiv(count, per));
  k_scan_part<<<(unsigned)parts, 1024, 0, st>>>(count, per, cnt, tmp);
  k_scan_final<<<(unsigned)parts, 1024, 0, st>>>(count, per, cnt, tmp, start);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch(2);
  return RLU_OK;
}

int launch_twiddles(int N, double2* tw64, float2* tw32, cudaStream_t st) {
  k_twiddles<<<(unsigned)cdiv(N, 256), 256, 0, st>>>(N, tw64, tw32);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  return RLU_OK;
}

// Shape of the whole-row sketch (k_sketch_rows) for rows of n elements of
// `es` bytes: ring slots and row pairs per FFT batch, or {0, 0} when the rows
// do not fit (or cannot be bulk-copied: rows must start on 16-byte boundaries
// and span a multiple of 16 bytes).
struct RowsShape {
  int nslots, pb;
};
static size_t rows_lists16_bytes(int64_t n, int l1) {
  // transposed layout (the larger of the two): group offsets, slot map, padded entries
  if (n >= 32768) return 0;
  const size_t b = (size_t)4 * ((l1 + 31) / 32 + 1) + (size_t)2 * l1 + (size_t)2 * (n + 1024);
  return (b + 15) & ~(size_t)15;
}
static RowsShape rows_shape(int64_t m, int64_t n, int l1, size_t es, size_t sv, bool aligned, int num_sms) {
  const size_t budget = 225 * 1024 - rows_lists16_bytes(n, l1);
  const size_t rowb = (size_t)n * es;
  if (!aligned || rowb % 16 != 0 || n < 1 || rows_lists16_bytes(n, l1) >= 225 * 1024) return {0, 0};
  // whole-row bucket lists hold n / l1 entries per bucket on average; beyond
  // 32 the column chunks keep the lists (and their insertion sort) short
  if (n > 32 * (int64_t)l1) return {0, 0};
  int pb_cap = (int)(m / (2 * (int64_t)(num_sms > 0 ? num_sms : 1)));
  pb_cap = pb_cap < 1 ? 1 : (pb_cap > 8 ? 8 : pb_cap);
  const size_t pair = (size_t)2 * l1 * sv, fixed = (size_t)l1 * sv;
  auto pairs_with = [&](int ns) -> int {
    const size_t used = (size_t)ns * rowb + fixed;
    if (used + pair > budget) return 0;
    const int64_t p = (int64_t)((budget - used) / pair);
    return (int)(p < pb_cap ? p : pb_cap);
  };
  const int want = pb_cap < 2 ? pb_cap : 2;
  for (int ns = 3; ns >= 2; --ns) {
    const int pb = pairs_with(ns);
    if (pb >= want) return {ns, pb};
  }
  const int pb = pairs_with(2);
  if (pb >= 1) return {2, pb};
  return {0, 0};
}

int sketch_chunk_cols(int dtype, int64_t m, int64_t n, int l1, bool aligned, int num_sms) {
  const size_t es = dtype == RLU_F64 ? 8 : (dtype == RLU_F32 ? 4 : 2);
  const size_t sv = dtype == RLU_F64 ? 16 : 8;
  if (rows_shape(m, n, l1, es, sv, aligned, num_sms).nslots > 0) return (int)n;  // one chunk: whole rows
  // 32 KB of A per staged tile (a two-stage ring leaves room for batched FFT buffers)
  if (dtype == RLU_F64) return 1024;  // 4 rows x 1024 x 8 B
  if (dtype == RLU_F32) return 1024;  // 8 rows x 1024 x 4 B
  return 2048;                        // 8 rows x 2048 x 2 B
}

template <typename TA, typename TACC, int NT, int NB, int R>
static int launch_dense_tma_cfg(const void* A, int64_t lda, int64_t m, int64_t n, int l1, int l, const SketchWs& ws,
                                double* Y, const int32_t* rowmap, unsigned int* status, int num_sms,
                                cudaStream_t st) {
  auto kern = k_sketch_dense_tma<TA, TACC, NT, NB, R>;
  using V = typename C2<TACC>::t;
  const size_t ring = (size_t)2 * R * ws.chunk * sizeof(TA);
  const size_t budget = 220 * 1024;
  const size_t per_pair = (size_t)2 * l1 * sizeof(V);
  const size_t fixed = ring + (size_t)l1 * sizeof(V);
  const size_t lists = (size_t)4 * (ws.nchunks * l1 + 1) + (size_t)4 * n;
  if (fixed + per_pair > budget) return RLU_EINVAL;
  // prefer the bucket lists in shared memory with at least two FFT pairs per batch
  int lists_in_smem = 0;
  int pb;
  if (fixed + lists + 2 * per_pair <= budget || (R / 2 < 2 && fixed + lists + per_pair <= budget)) {
    lists_in_smem = 1;
    pb = (int)((budget - fixed - lists) / per_pair);
  } else {
    pb = (int)((budget - fixed) / per_pair);
  }
  if (pb > R / 2) pb = R / 2;
  const size_t smem = fixed + (size_t)pb * per_pair + (lists_in_smem ? lists : 0);
  if (int rc_ = allow_dynamic_smem((const void*)kern, smem)) return rc_;
  int per_sm = 0;
  RLU_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
  if (per_sm < 1) return RLU_EINVAL;
  const int64_t groups = cdiv(m, R);
  int64_t grid = (int64_t)per_sm * num_sms;
  if (grid > groups) grid = groups;
  const typename C2<TACC>::t* tw;
  if constexpr (sizeof(TACC) == 8) tw = ws.tw64; else tw = ws.tw32;
  kern<<<(unsigned)grid, NT, smem, st>>>(reinterpret_cast<const TA*>(A), lda, m, n, l1, l, ws.chunk, ws.bstart,
                                         ws.blist, ws.dsign, ws.R, tw, ws.plan, pb, lists_in_smem, Y, rowmap, status);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  return RLU_OK;
}

template <typename TA, typename TACC>
static int launch_rows_cfg(const void* A, int64_t lda, int64_t m, int64_t n, int l1, int l, const SketchWs& ws,
                           double* Y, const int32_t* rowmap, unsigned int* status, int num_sms, RowsShape sh,
                           cudaStream_t st) {
  constexpr int NT = 1024;
  auto kern = k_sketch_rows<TA, TACC, NT>;
  using V = typename C2<TACC>::t;
  const size_t lb = rows_lists16_bytes(n, l1);
  const int lists16 = lb > 0 ? 1 : 0;
  const size_t smem =
      (size_t)sh.nslots * n * sizeof(TA) + (size_t)l1 * sizeof(V) + (size_t)sh.pb * 2 * l1 * sizeof(V) + lb;
  if (int rc_ = allow_dynamic_smem((const void*)kern, smem)) return rc_;
  int per_sm = 0;
  RLU_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
  if (per_sm < 1) return RLU_EINVAL;
  const int64_t batches = cdiv(m, 2 * (int64_t)sh.pb);
  int64_t grid = (int64_t)per_sm * num_sms;
  if (grid > batches) grid = batches;
  const V* tw;
  if constexpr (sizeof(TACC) == 8) tw = ws.tw64; else tw = ws.tw32;
  kern<<<(unsigned)grid, NT, smem, st>>>(reinterpret_cast<const TA*>(A), lda, m, n, l1, l, ws.bstart, ws.blist,
                                         ws.dsign, ws.R, tw, ws.plan, sh.pb, sh.nslots, lists16, Y, rowmap,
                                         status);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  return RLU_OK;
}

template <typename TA, typename TACC, int NT, int NB, int R>
static int launch_dense_cfg(const void* A, int64_t lda, int64_t m, int64_t n, int l1, int l, const SketchWs& ws,
                            double* Y, const int32_t* rowmap, unsigned int* status, int num_sms, cudaStream_t st) {
  // whole rows when the bucket lists were built for one chunk and the rows fit
  if (ws.chunk == n) {
    const bool al = ((uintptr_t)A % 16 == 0) && ((lda * (int64_t)sizeof(TA)) % 16 == 0);
    const RowsShape sh = rows_shape(m, n, l1, sizeof(TA), sizeof(typename C2<TACC>::t), al, num_sms);
    if (sh.nslots > 0)
      return launch_rows_cfg<TA, TACC>(A, lda, m, n, l1, l, ws, Y, rowmap, status, num_sms, sh, st);
  }
  // TMA-fed kernel when every row segment is a 16-byte-aligned run of 16-byte multiples
  // and the ring plus FFT buffers fit in shared memory
  const bool aligned = ((uintptr_t)A % 16 == 0) && ((lda * (int64_t)sizeof(TA)) % 16 == 0) &&
                       ((n * (int64_t)sizeof(TA)) % 16 == 0) && ((ws.chunk * (int64_t)sizeof(TA)) % 16 == 0);
  const size_t tma_smem = (size_t)2 * R * ws.chunk * sizeof(TA) + (size_t)3 * l1 * sizeof(typename C2<TACC>::t);
  if (aligned && tma_smem <= 220 * 1024)
    return launch_dense_tma_cfg<TA, TACC, NT, NB, R>(A, lda, m, n, l1, l, ws, Y, rowmap, status, num_sms, st);
  auto kern = k_sketch_dense<TA, TACC, NT, NB, R>;
  size_t tile_bytes = (size_t)R * ws.chunk * sizeof(TA);
  size_t fft_bytes = (size_t)2 * l1 * sizeof(typename C2<TACC>::t);
  size_t smem = tile_bytes > fft_bytes ? tile_bytes : fft_bytes;
  if (int rc_ = allow_dynamic_smem((const void*)kern, smem)) return rc_;
  int per_sm = 0;
  RLU_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
  if (per_sm < 1) return RLU_EINVAL;
  int64_t groups = cdiv(m, R);
  int64_t grid = (int64_t)per_sm * num_sms;
  if (grid > groups) grid = groups;
  const typename C2<TACC>::t* tw;
  if constexpr (sizeof(TACC) == 8) tw = ws.tw64; else tw = ws.tw32;
  kern<<<(unsigned)grid, NT, smem, st>>>(reinterpret_cast<const TA*>(A), lda, m, n, l1, l, ws.chunk, ws.bstart,
                                         ws.blist, ws.dsign, ws.R, tw, ws.plan, Y, rowmap, status);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  return RLU_OK;
}

int launch_sketch_dense(const void* A, int64_t lda, int dtype, bool acc64, int64_t m, int64_t n, int l1, int l,
                        const SketchWs& ws, double* Y, unsigned int* status, int num_sms, cudaStream_t st,
                        const int32_t* rowmap) {
  // 1024 threads per CTA; each thread owns NB buckets of R rows in registers
  if (dtype == RLU_F64) {
    if (l1 <= 2048) return launch_dense_cfg<double, double, 1024, 2, 4>(A, lda, m, n, l1, l, ws, Y, rowmap, status, num_sms, st);
    if (l1 <= 4096) return launch_dense_cfg<double, double, 1024, 4, 4>(A, lda, m, n, l1, l, ws, Y, rowmap, status, num_sms, st);
    if (l1 <= 8192) return launch_dense_cfg<double, double, 1024, 8, 2>(A, lda, m, n, l1, l, ws, Y, rowmap, status, num_sms, st);
    return launch_dense_cfg<double, double, 1024, 16, 2>(A, lda, m, n, l1, l, ws, Y, rowmap, status, num_sms, st);
  }
  if (acc64) return RLU_EINVAL;
  // l1 <= 1024: one bucket of 16 rows per thread (each bucket-list read serves 16 rows)
  if (dtype == RLU_F32) {
    if (l1 <= 1024) return launch_dense_cfg<float, float, 1024, 1, 16>(A, lda, m, n, l1, l, ws, Y, rowmap, status, num_sms, st);
    if (l1 <= 2048) return launch_dense_cfg<float, float, 1024, 2, 8>(A, lda, m, n, l1, l, ws, Y, rowmap, status, num_sms, st);
    if (l1 <= 4096) return launch_dense_cfg<float, float, 1024, 4, 8>(A, lda, m, n, l1, l, ws, Y, rowmap, status, num_sms, st);
    if (l1 <= 8192) return launch_dense_cfg<float, float, 1024, 8, 4>(A, lda, m, n, l1, l, ws, Y, rowmap, status, num_sms, st);
    return launch_dense_cfg<float, float, 1024, 16, 2>(A, lda, m, n, l1, l, ws, Y, rowmap, status, num_sms, st);
  }
  if (dtype == RLU_BF16) {
    using B = __nv_bfloat16;
    if (l1 <= 1024) return launch_dense_cfg<B, float, 1024, 1, 16>(A, lda, m, n, l1, l, ws, Y, rowmap, status, num_sms, st);
    if (l1 <= 2048) return launch_dense_cfg<B, float, 1024, 2, 8>(A, lda, m, n, l1, l, ws, Y, rowmap, status, num_sms, st);
    if (l1 <= 4096) return launch_dense_cfg<B, float, 1024, 4, 8>(A, lda, m, n, l1, l, ws, Y, rowmap, status, num_sms, st);
    if (l1 <= 8192) return launch_dense_cfg<B, float, 1024, 8, 4>(A, lda, m, n, l1, l, ws, Y, rowmap, status, num_sms, st);
    return launch_dense_cfg<B, float, 1024, 16, 2>(A, lda, m, n, l1, l, ws, Y, rowmap, status, num_sms, st);
  }
  return RLU_EINVAL;
}

}  // namespace rlu
