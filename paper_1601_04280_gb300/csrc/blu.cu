// Blocked partial-pivoted LU of the sketch, P Y = L_Y U_Y (step 3 of
// Algorithm 1), with the trailing updates on the tensor cores.
//
// Right-looking blocked elimination in panels of b columns (b = 16, 32, 64):
//   1. the panel's b steps run in the persistent pivoted-LU kernel on the
//      panel columns only (every row; the panel in shared memory), with
//      LAPACK getf2 semantics: the pivot choices depend only on the panel;
//   2. U12 = L11^{-1} A12 for the panel's pivot rows (FP64 forward
//      substitution with the unit lower L11, a warp per trailing column);
//   3. A22 -= L21 U12 for every row not yet pivoted.  The product runs as an
//      exact digit product (the error-free splitting of Ozaki, Ogita, Oishi
//      and Rump, Numer. Algorithms 59, 2012): each row of L21 and each column
//      of U12 is scaled by a power of two and cut into eight signed 7-bit
//      digits (56 bits); level v = s + t of the digit products accumulates
//      exactly in FP32 in its own tensor-memory accumulator (every level sum
//      stays below 2^22 for b <= 64); the epilogue combines the eight levels
//      exactly in 64-bit integers, assembles the double from the integer's
//      bits with the two scales in its exponent (rounded to 53 bits) and
//      subtracts it from A22: one FP64 operation per element.
// The only approximations are the digits' rounding (2^-57 of the row and
// column scales) and the dropped levels beyond the eighth, so the update
// carries the accuracy of an FP64 product while the slow FP64 pipe does only
// the panels (b^2/2 multiply-adds per row and panel instead of l^2/2 per
// row) and one subtraction per updated element.
//
// The digit planes are packed per row as [chunk of 16/32 columns][digit]
// [column in chunk], so one pipeline stage brings all eight digits of a
// chunk in a few 128-byte-wide TMA boxes and the MMA for digit pair (s, t)
// addresses its K-slice inside those boxes.
#include <cuda.h>
#include <climits>

#include "bgemm.cuh"
#include "blu.cuh"
#include "common.cuh"
#include "gemm_tc.cuh"

namespace rlu {
namespace blu {

constexpr int kD = 8;            // digits of 7 bits
constexpr int kBM = 128;         // rows per tile (MMA M)
constexpr int kNT = 32;          // columns per tile: two sets of 8 levels x 32 columns fill tensor memory
constexpr int kEpiWarps = 16;    // four per tensor-memory lane quarter
constexpr int kEpiCols = kNT / (kEpiWarps / 4);  // columns of a tile per epilogue thread
constexpr int kThreads = 64 + 32 * kEpiWarps;    // warp 0 TMA, warp 1 MMA, warps 2.. epilogue
constexpr int kMaxStages = 4;
constexpr uint32_t kTmemCols = 512;
constexpr int32_t kSkip = INT_MIN;
constexpr int kNoExp = -100000;

__host__ __device__ constexpr int chunk_of(int b) { return b >= 32 ? 32 : 16; }
inline int width_index(int b) { return b == 64 ? 0 : (b == 32 ? 1 : 2); }

template <int KC>
__host__ __device__ constexpr uint32_t stage_bytes() {
  return (uint32_t)(kD * KC / 64) * (uint32_t)(kBM * 128 + kNT * 128);
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::
          "r"(tc::smem_u32(dst)),
      "l"(map), "r"(tc::smem_u32(bar)), "r"(x), "r"(y), "r"(0)
      : "memory");
}

// frexp exponent of a finite nonzero double from its bits (|x| in [2^(e-1), 2^e)),
// kNoExp for zero, subnormal or non-finite values.
__device__ __forceinline__ int exp_of(double x) {
  const int ex = (int)((__double_as_longlong(x) >> 52) & 0x7ff);
  return (ex == 0 || ex == 0x7ff) ? kNoExp : ex - 1022;
}

// Eight balanced digits of x 2^-e (|x| < 2^e): X = round(x 2^(56 - e)) as a
// 64-bit integer from the bits of x, then X = sum_s d_s 128^(7 - s) with
// d_1..d_7 in [-64, 63] and |d_0| <= 128.  Integer operations only.
__device__ __forceinline__ void digits8(double x, int e, int (&d)[kD]) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ff);
  long long X = 0;
  if (ex != 0 && ex != 0x7ff) {
    const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = ex - 1075 + 56 - e;  // X = mant 2^sh; sh <= 3 since |x| < 2^e
    unsigned long long u = 0;
    if (sh >= 0) u = mant << sh;
    else if (sh > -64) u = (mant + (1ull << (-sh - 1))) >> (-sh);
    X = (b >> 63) ? -(long long)u : (long long)u;
  }
#pragma unroll
  for (int s = kD - 1; s >= 1; --s) {
    int r = (int)(X & 127);
    r -= (r >= 64) ? 128 : 0;
    d[s] = r;
    X = (X - r) >> 7;
  }
  d[0] = (int)X;
}

// An integer-valued float with |f| < 2^22 as an int (exact).
__device__ __forceinline__ int level_int(float f) { return __float_as_int(f + 12582912.0f) - 0x4B400000; }

// t 2^E as a double, rounded to 53 bits (half away from zero), built from the
// integer's bits; values outside the normal range take the slow FP64 route.
__device__ __forceinline__ double i64_scaled(long long t, int E) {
  if (t == 0) return 0.0;
  const unsigned long long neg = t < 0 ? (1ull << 63) : 0ull;
  unsigned long long a = t < 0 ? (unsigned long long)(-t) : (unsigned long long)t;
  const int lz = __clzll((long long)a);
  a <<= lz;
  const int ex = 63 - lz + E + 1023;
  if (ex < 1 || ex > 2046) return ldexp((double)t, E);
  const unsigned long long bits = ((unsigned long long)(ex - 1) << 52) + (a >> 11) + ((a >> 10) & 1ull);
  return __longlong_as_double((long long)(bits | neg));
}

// The digits and scale of a float-float value: the same balanced form from
// the top (first digit rint(x 2^(7 - e)) in [-128, 128], the next ones in
// [-64, 64]), every step exact in FP32.
__device__ __forceinline__ void digits8(df32 x, int e, int (&d)[kD]) {
  float yh = ldexpf(x.hi, 7 - e), yl = ldexpf(x.lo, 7 - e);
#pragma unroll
  for (int s = 0; s < kD; ++s) {
    const float t = rintf(yh);
    d[s] = (int)t;
    const df32 r = two_sum(yh - t, yl);
    yh = r.hi * 128.f;
    yl = r.lo * 128.f;
  }
}
__device__ __forceinline__ int exp_of(df32 x) {
  const int ex = (int)((__float_as_uint(x.hi) >> 23) & 0xff);
  return (ex == 0 || ex == 0xff) ? kNoExp : ex - 126;
}

// t 2^E as a float-float: t in three 24-bit pieces (each exact in FP32),
// summed with TwoSum, scaled by 2^E.  FP32 and integer operations only.
__device__ __forceinline__ df32 i64_scaled_df(long long t, int E) {
  const float fa = (float)(int)(t >> 48) * 0x1p48f;
  const float fb = (float)(int)((t >> 24) & 0xFFFFFF) * 0x1p24f;
  const float fc = (float)(int)(t & 0xFFFFFF);
  const df32 s = two_sum(fa, fb) + df_make(fc, 0.f);
  return df_make(ldexpf(s.hi, E), ldexpf(s.lo, E));
}

__device__ __forceinline__ double scaled_product(long long t, int E, double) { return i64_scaled(t, E); }
__device__ __forceinline__ df32 scaled_product(long long t, int E, df32) { return i64_scaled_df(t, E); }
__device__ __forceinline__ double sub(double y, double c) { return y - c; }
__device__ __forceinline__ df32 sub(df32 y, df32 c) { return y - c; }
__device__ __forceinline__ double shfl(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ df32 shfl(df32 v, int src) {
  return df_make(__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src));
}
template <typename T> __device__ __forceinline__ T zero_v() { return T(0); }
template <> __device__ __forceinline__ df32 zero_v<df32>() { return df_make(0.f, 0.f); }

// U12 = L11^{-1} A12 for the panel's pivot rows (positions j0 .. j0 + B - 1)
// of X (element (i, c) at X[i rs + c cs]), written back into X, and the digit
// planes of U12^T (row c = trailing column j0 + B + c) with their scales.
// One warp per trailing column.
template <int B, typename T>
__global__ void __launch_bounds__(256) k_u12(T* __restrict__ X, int64_t rs, int64_t cs, int j0, int w,
                                             const int64_t* __restrict__ perm, __nv_bfloat16* __restrict__ bdig,
                                             int32_t* __restrict__ bexp) {
  constexpr int KC = chunk_of(B);
  constexpr int R = (B + 31) / 32;
  __shared__ T LT[B][B + 1];  // LT[i][t] = L11[t][i] (t > i), the multiplier of pivot row t at panel column i
  __shared__ int64_t prow[B];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int t = tid; t < B; t += blockDim.x) prow[t] = perm[j0 + t];
  __syncthreads();
  for (int e = tid; e < B * B; e += blockDim.x) {
    const int t = e / B, i = e - t * B;
    LT[i][t] = (i < t) ? X[prow[t] * rs + (int64_t)(j0 + i) * cs] : zero_v<T>();
  }
  __syncthreads();
  const int c = blockIdx.x * (blockDim.x >> 5) + warp;
  if (c >= w) return;
  const int64_t col = ((int64_t)j0 + B + c) * cs;
  T a[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int t = lane + 32 * r;
    a[r] = (t < B) ? X[prow[t < B ? t : 0] * rs + col] : zero_v<T>();
  }
#pragma unroll
  for (int i = 0; i < B; ++i) {
    const T ui = shfl(a[i / 32], i % 32);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int t = lane + 32 * r;
      if (t > i && t < B) a[r] = mad(-LT[i][t], ui, a[r]);
    }
  }
  int e = kNoExp;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int t = lane + 32 * r;
    if (t < B) {
      X[prow[t] * rs + col] = a[r];
      e = max(e, exp_of(a[r]));
    }
  }
  e = __reduce_max_sync(0xffffffffu, e);
  if (e == kNoExp) e = 0;
  if (lane == 0) bexp[c] = e;
  __nv_bfloat16* row = bdig + (int64_t)c * (kD * B);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int t = lane + 32 * r;
    if (t < B) {
      int d[kD];
      digits8(a[r], e, d);
      const int base = (t / KC) * kD * KC + (t % KC);
#pragma unroll
      for (int s = 0; s < kD; ++s) row[base + s * KC] = __int2bfloat16_rn(d[s]);
    }
  }
}

// Digit planes of the multipliers L21 (panel columns j0 .. j0 + B - 1) of
// every row of X with their scales; rows already pivoted get zero digits and
// the skip mark.  min(B, 32) lanes per row (two rows per warp for B = 16).
template <int B, typename T>
__global__ void __launch_bounds__(256) k_l21(const T* __restrict__ X, int64_t rs, int64_t cs, int64_t m, int j0,
                                             const int32_t* __restrict__ pstep, __nv_bfloat16* __restrict__ adig,
                                             int32_t* __restrict__ aexp) {
  constexpr int KC = chunk_of(B);
  constexpr int LPR = B < 32 ? B : 32;  // lanes per row
  constexpr int R = B / LPR;
  const int lane = threadIdx.x & 31, sub_ = lane % LPR;
  const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / LPR;
  const bool valid = r < m;  // every lane stays for the shuffles
  const bool skip = !valid || pstep[valid ? r : 0] >= 0;
  T x[R];
  int e = kNoExp;
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int i = sub_ + LPR * q;
    x[q] = !skip ? X[r * rs + (int64_t)(j0 + i) * cs] : zero_v<T>();
    e = max(e, exp_of(x[q]));
  }
#pragma unroll
  for (int o = LPR / 2; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  if (e == kNoExp) e = 0;
  if (!valid) return;
  if (sub_ == 0) aexp[r] = skip ? kSkip : e;
  __nv_bfloat16* row = adig + r * (kD * B);
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int i = sub_ + LPR * q;
    int d[kD];
    digits8(x[q], e, d);
    const int base = (i / KC) * kD * KC + (i % KC);
#pragma unroll
    for (int s = 0; s < kD; ++s) row[base + s * KC] = __int2bfloat16_rn(d[s]);
  }
}

// X(i, c) -= (L21 U12)(i, c) for the M x N trailing block whose element
// (i, c) sits at X[i rs + c cs] (FP64 or float-float), from the packed digit
// planes (nch chunks of KC columns).  Persistent: CTA b takes tiles b,
// b + gridDim.x, ... (128 rows x 32 columns, column tile fastest); a ring of
// nst stages runs across tiles; two accumulator sets let the epilogue of one
// tile overlap the MMAs of the next.  The epilogue (about a hundred integer
// and FP64 instructions per entry) is issue- and latency-bound: sixteen warps,
// each thread owning eight entries of one row.
template <int KC, typename T>
__global__ void __launch_bounds__(kThreads, 1)
    k_digit_update(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int64_t M,
                   int N, int nch, int nt, int64_t tiles, int nst, const int32_t* __restrict__ aexp,
                   const int32_t* __restrict__ bexp, T* __restrict__ X, int64_t rs, int64_t cs,
                   unsigned int* status) {
  constexpr int NBOX = kD * KC / 64;
  constexpr uint32_t ABOX = kBM * 128, BBOX = kNT * 128;
  constexpr uint32_t SB = stage_bytes<KC>();
  constexpr uint32_t SET = kD * kNT;  // tensor-memory columns of one accumulator set
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages], tfull[2], tempty[2];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto boxA = [&](int s, int j) { return smem + (uint32_t)s * SB + (uint32_t)j * ABOX; };
  auto boxB = [&](int s, int j) { return smem + (uint32_t)s * SB + NBOX * ABOX + (uint32_t)j * BBOX; };

  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&tfull[b], 1);
      tc::mbar_init(&tempty[b], kEpiWarps);
    }
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(&tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    // ---- TMA producer: all digits of one chunk of both operands per stage ----
    if (lane == 0) {
      int64_t it = 0;
      for (int64_t tile = blockIdx.x; tile < tiles && !s_fail; tile += gridDim.x) {
        const int row0 = (int)((tile / nt) * kBM), col0 = (int)(tile % nt) * kNT;
        for (int q = 0; q < nch; ++q, ++it) {
          const int s = (int)(it % nst);
          if (it >= nst && !tc::mbar_wait(&empty[s], (uint32_t)(((it / nst) - 1) & 1))) {
            s_fail = 1;
            break;
          }
          tc::mbar_arrive_expect_tx(&full[s], SB);
          for (int j = 0; j < NBOX; ++j) {
            tma_load_3d(boxA(s, j), &mapA, &full[s], q * kD * KC + j * 64, row0);
            tma_load_3d(boxB(s, j), &mapB, &full[s], q * kD * KC + j * 64, col0);
          }
        }
      }
      // every issued load has landed before the CTA may exit
      for (int64_t j = it - nst < 0 ? 0 : it - nst; j < it; ++j)
        if (!tc::mbar_wait(&full[j % nst], (uint32_t)((j / nst) & 1))) s_fail = 1;
    }
  } else if (warp == 1) {
    // ---- MMA issuer: level v of set b in columns b * SET + v * kNT ----
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16(kBM, kNT);
      int64_t it = 0, local = 0;
      bool ok = true;
      for (int64_t tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x, ++local) {
        const int b = (int)(local & 1);
        if (local >= 2 && !tc::mbar_wait(&tempty[b], (uint32_t)(((local >> 1) - 1) & 1))) { ok = false; break; }
        tc::tc_fence_after();
        for (int q = 0; q < nch; ++q, ++it) {
          const int s = (int)(it % nst);
          if (!tc::mbar_wait(&full[s], (uint32_t)((it / nst) & 1))) { ok = false; break; }
          tc::tc_fence_after();
#pragma unroll
          for (int kk = 0; kk < KC / 16; ++kk) {
#pragma unroll
            for (int v = 0; v < kD; ++v) {
              const uint32_t dcol = tmem + (uint32_t)b * SET + (uint32_t)(v * kNT);
#pragma unroll
              for (int da = 0; da <= v; ++da) {
                const int ka = da * KC + kk * 16, kb = (v - da) * KC + kk * 16;
                const uint64_t aD = tc::sw128_desc(tc::smem_u32(boxA(s, ka >> 6)) + (uint32_t)(ka & 63) * 2u);
                const uint64_t bD = tc::sw128_desc(tc::smem_u32(boxB(s, kb >> 6)) + (uint32_t)(kb & 63) * 2u);
                tc::mma_bf16(dcol, aD, bD, idesc, (q == 0 && kk == 0 && da == 0) ? 0u : 1u);
              }
            }
          }
          tc::mma_commit(&empty[s]);
        }
        if (ok) tc::mma_commit(&tfull[b]);
      }
      if (!ok) s_fail = 1;
    }
  } else {
    // ---- epilogue (warps 2..): lane quarter warp mod 4, column group (warp - 2) / 4 ----
    const int quarter = warp & 3, grp = (warp - 2) >> 2;
    // Row-major X (cs == 1): this warp's 32 x 8 block of A22 is read and
    // written row-contiguously (lane -> row 4 it + lane / 8, column lane % 8:
    // four 64-byte row pieces per instruction) and turned around through a
    // 32 x 9 staging block in shared memory, because a thread owns a row in
    // tensor memory and row-per-lane accesses cost a transaction per row.
    // Otherwise (B^T) the lanes' rows are adjacent in memory already.
    const bool rowmaj = (cs == 1);
    T* stg = reinterpret_cast<T*>(smem + (uint32_t)nst * SB) + (warp - 2) * 32 * 9;
    const int sr = lane >> 3, sc = lane & 7;
    // this warp's entries of A22 and its rows' scales for a tile: loaded one
    // tile ahead, so their latency overlaps the previous tile's work
    T yn[kEpiCols];
    int ean = kSkip;
    auto prefetch = [&](int64_t tile) {
      const int64_t rbase = (tile / nt) * kBM + quarter * 32;
      const int cb = (int)(tile % nt) * kNT + grp * kEpiCols;
      ean = (tile < tiles && rbase + lane < M) ? aexp[rbase + lane] : kSkip;
      if (rowmaj) {
#pragma unroll
        for (int it = 0; it < kEpiCols; ++it) {
          const int64_t r = rbase + it * 4 + sr;
          yn[it] = (tile < tiles && r < M && cb + sc < N) ? X[r * rs + cb + sc] : zero_v<T>();
        }
      } else {
        const T* xr = X + (rbase + lane) * rs;
#pragma unroll
        for (int i = 0; i < kEpiCols; ++i)
          yn[i] = (ean != kSkip && cb + i < N) ? xr[(int64_t)(cb + i) * cs] : zero_v<T>();
      }
    };
    prefetch(blockIdx.x);
    int64_t local = 0;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++local) {
      const int b = (int)(local & 1);
      const int64_t rbase = (tile / nt) * kBM + quarter * 32;
      const int cb = (int)(tile % nt) * kNT + grp * kEpiCols;
      const int ea = ean;
      T y[kEpiCols];
      if (rowmaj) {
#pragma unroll
        for (int it = 0; it < kEpiCols; ++it) stg[(it * 4 + sr) * 9 + sc] = yn[it];
        __syncwarp();
#pragma unroll
        for (int i = 0; i < kEpiCols; ++i) y[i] = stg[lane * 9 + i];
        __syncwarp();
      } else {
#pragma unroll
        for (int i = 0; i < kEpiCols; ++i) y[i] = yn[i];
      }
      prefetch(tile + gridDim.x);
      if (!tc::mbar_wait(&tfull[b], (uint32_t)((local >> 1) & 1))) { s_fail = 1; break; }
      tc::tc_fence_after();
      const uint32_t tq = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)b * SET + (uint32_t)(grp * kEpiCols);
      // P = sum_{v <= 6} L_v 128^(6 - v) + floor(L_7 / 128): the product in
      // units of 2^-56 of the two scales (|P| < 2^62.1 for b <= 64); the
      // levels come in two batches of four loads with one wait each
      long long P[kEpiCols];
      uint32_t v[4][kEpiCols];
#pragma unroll
      for (int g = 0; g < 2; ++g) {
#pragma unroll
        for (int q = 0; q < 4; ++q) tc::tmem_ld8_issue(tq + (uint32_t)((4 * g + q) * kNT), v[q]);
        tc::tmem_ld_wait();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int lv = 4 * g + q;
#pragma unroll
          for (int i = 0; i < kEpiCols; ++i) {
            const int L = level_int(__uint_as_float(v[q][i]));
            if (lv == 0) P[i] = L;
            else if (lv < kD - 1) P[i] = P[i] * 128 + L;
            else P[i] += (long long)(L >> 7);
          }
        }
      }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&tempty[b]);
      if (rowmaj) {
        // results by row into the staging block, then out row-contiguously
        // (rows already pivoted are not written)
#pragma unroll
        for (int i = 0; i < kEpiCols; ++i) {
          const int c = cb + i;
          stg[lane * 9 + i] = (ea != kSkip && c < N) ? sub(y[i], scaled_product(P[i], ea + bexp[c] - 56, y[i])) : y[i];
        }
        __syncwarp();
#pragma unroll
        for (int it = 0; it < kEpiCols; ++it) {
          const int rr = it * 4 + sr;
          const int64_t r = rbase + rr;
          const int ear = __shfl_sync(0xffffffffu, ea, rr);
          if (ear != kSkip && r < M && cb + sc < N) X[r * rs + cb + sc] = stg[rr * 9 + sc];
        }
        __syncwarp();
      } else if (ea != kSkip) {
        T* xr = X + (rbase + lane) * rs;
#pragma unroll
        for (int i = 0; i < kEpiCols; ++i) {
          const int c = cb + i;
          if (c < N) xr[(int64_t)c * cs] = sub(y[i], scaled_product(P[i], ea + bexp[c] - 56, y[i]));
        }
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
  if (threadIdx.x == 0 && s_fail) set_flag(status, FLAG_TIMEOUT);
}

template <int KC, typename T>
int launch_update(const BluWs& w, int wi, int64_t M, int N, int nch, T* Xt, int64_t rs, int64_t cs,
                  unsigned int* status, cudaStream_t st) {
  constexpr uint32_t SB = stage_bytes<KC>();
  const int nst = (int)min64(kMaxStages, (int64_t)(200 * 1024) / SB);
  const size_t smem = (size_t)nst * SB + (size_t)kEpiWarps * 32 * 9 * sizeof(T) + 1024;  // stages, staging blocks
  auto kern = k_digit_update<KC, T>;
  if (int rc = allow_dynamic_smem((const void*)kern, smem)) return rc;
  const int nt = (int)cdiv(N, kNT);
  const int64_t tiles = cdiv(M, kBM) * nt;
  const unsigned grid = (unsigned)min64(tiles, (int64_t)w.num_sms);
  kern<<<grid, kThreads, smem, st>>>(*reinterpret_cast<const CUtensorMap*>(w.mapA[wi]),
                                     *reinterpret_cast<const CUtensorMap*>(w.mapB[wi]), M, N, nch, nt, tiles, nst,
                                     w.aexp, w.bexp, Xt, rs, cs, status);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  return RLU_OK;
}

// The trailing update after the panel at column j0 (width B) of the rows x
// cols matrix X (element (i, c) at X[i rs + c cs]).
template <int B, typename T>
int trailing(T* X, int64_t rows, int cols, int64_t rs, int64_t cs, int j0, const PivLuWs& pw, const BluWs& w,
             unsigned int* status, cudaStream_t st) {
  const int wt = cols - j0 - B;
  k_u12<B, T><<<(unsigned)cdiv(wt, 8), 256, 0, st>>>(X, rs, cs, j0, wt, pw.perm, w.bdig, w.bexp);
  RLU_CUDA_TRY(cudaGetLastError());
  k_l21<B, T><<<(unsigned)cdiv(rows * (B < 32 ? B : 32), 256), 256, 0, st>>>(X, rs, cs, rows, j0, pw.pstep, w.adig,
                                                                             w.aexp);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch(2);
  constexpr int KC = chunk_of(B);
  return launch_update<KC, T>(w, width_index(B), rows, wt, B / KC, X + (int64_t)(j0 + B) * cs, rs, cs, status, st);
}

// Widest panel whose rows fit the panel kernel's shared memory with `ctas` CTAs.
int widest_fit(int64_t rows, int cols, int ctas, int cap) {
  PivLuWs probe{};
  probe.max_ctas = 1 << 20;
  probe.max_cols = cols;
  for (int b : kBluWidths)
    if (b <= cap && b < cols && pivlu_panel_in_smem(rows, b, cols, probe, ctas)) return b;
  return 0;
}

// Panel width for the rows x cols LU: `block` forced (> 0), unblocked (-1),
// or chosen (0).  The form and the width depend only on the sizes and the
// device's SM count, never on a bound on the grid (coop_sms): results stay
// bit-for-bit the same under rlu_set_max_ctas (a panel whose rows no longer
// fit in shared memory runs the kernel's global-memory form, which performs
// the same operations in the same order).  Returns -1 for an invalid block.
int choose_width(int64_t rows, int cols, const PivLuWs& pw, const BluWs& bw, int block, int coop_sms) {
  const int sms = bw.num_sms > 0 ? bw.num_sms : coop_sms;
  if (block > 0) {
    if ((block != 16 && block != 32 && block != 64) || !bw.ready || block > bw.bmax || block >= cols ||
        rows > bw.rows_a)
      return -1;
    return block;
  }
  if (block < 0 || !bw.ready || cols < 32 || rows > bw.rows_a || pivlu_panel_in_smem(rows, cols, cols, pw, sms))
    return 0;
  // blocked when the unblocked kernel could not keep the matrix in shared
  // memory (its global-memory form is bound by the trailing updates); a
  // matrix that fits is bound by the per-step exchange, which blocking does
  // not shorten
  int b = widest_fit(rows, cols, (int)min64(sms, pw.max_ctas), bw.bmax);
  while (b > 16 && 2 * b > cols) b /= 2;
  return b;
}

// One launch of the pivoted-LU kernel, between two timer events when timed.
template <typename T>
int timed_panel(T* X, int64_t rows, int wid, int64_t rs, int64_t cs, int j0, int cols, PivLuWs& pw,
                unsigned int* status, int coop_sms, cudaStream_t st, PanelTimer* timer) {
  const bool rec = timer && timer->n < kMaxPanels && timer->ev[2 * timer->n];
  if (rec) RLU_CUDA_TRY(cudaEventRecord(timer->ev[2 * timer->n], st));
  const int rc = launch_pivoted_lu_panel<T>(X, rows, wid, rs, cs, wid, j0, cols, pw, status, coop_sms, st);
  if (rc) return rc;
  if (rec) {
    RLU_CUDA_TRY(cudaEventRecord(timer->ev[2 * timer->n + 1], st));
    ++timer->n;
  }
  return RLU_OK;
}

template <typename T>
int blocked_lu(T* X, int64_t rows, int cols, int64_t rs, int64_t cs, int b, PivLuWs& pw, const BluWs& bw,
               unsigned int* status, int coop_sms, cudaStream_t st, PanelTimer* timer) {
  for (int j0 = 0; j0 < cols; j0 += b) {
    const int wid = cols - j0 < b ? cols - j0 : b;
    int rc = timed_panel<T>(X + (int64_t)j0 * cs, rows, wid, rs, cs, j0, cols, pw, status, coop_sms, st, timer);
    if (rc) return rc;
    if (cols - j0 - wid == 0) break;
    switch (b) {
      case 64: rc = trailing<64, T>(X, rows, cols, rs, cs, j0, pw, bw, status, st); break;
      case 32: rc = trailing<32, T>(X, rows, cols, rs, cs, j0, pw, bw, status, st); break;
      default: rc = trailing<16, T>(X, rows, cols, rs, cs, j0, pw, bw, status, st); break;
    }
    if (rc) return rc;
  }
  return RLU_OK;
}

}  // namespace blu

namespace {
constexpr size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }
struct BluDims {
  int64_t rows_a;
  int rows_b;
  int bmax;
};
BluDims blu_dims(int64_t m, int64_t n, int k, int l, int num_sms) {
  BluDims d;
  d.rows_a = m > n ? m : n;
  d.rows_b = l;
  const int by = blu::widest_fit(m, l, num_sms, 64), bb = blu::widest_fit(n, k, num_sms, 64);
  d.bmax = by > bb ? by : bb;
  return d;
}
}  // namespace

size_t blu_workspace_bytes(int64_t m, int64_t n, int k, int l, int num_sms) {
  const BluDims d = blu_dims(m, n, k, l, num_sms);
  if (d.bmax == 0) return 0;
  const size_t row = (size_t)blu::kD * d.bmax * 2;
  return a256(row * (size_t)d.rows_a) + a256(row * (size_t)d.rows_b) + a256(4 * (size_t)d.rows_a) +
         a256(4 * (size_t)d.rows_b);
}

int blu_setup(BluWs& w, void* base, int64_t m, int64_t n, int k, int l, int num_sms) {
  w.ready = false;
  w.num_sms = num_sms;
  const BluDims d = blu_dims(m, n, k, l, num_sms);
  w.rows_a = d.rows_a;
  w.rows_b = d.rows_b;
  w.bmax = d.bmax;
  if (w.bmax == 0) return RLU_OK;
  const size_t row = (size_t)blu::kD * w.bmax * 2;
  unsigned char* b = (unsigned char*)base;
  w.adig = (__nv_bfloat16*)b;
  b += a256(row * (size_t)w.rows_a);
  w.bdig = (__nv_bfloat16*)b;
  b += a256(row * (size_t)w.rows_b);
  w.aexp = (int32_t*)b;
  b += a256(4 * (size_t)w.rows_a);
  w.bexp = (int32_t*)b;
  for (int bw : kBluWidths) {
    if (bw > w.bmax) continue;
    const int wi = blu::width_index(bw);
    const uint64_t kp = (uint64_t)blu::kD * bw;  // packed row: 8 digits of bw columns
    if (tc_encode_bf16_3d(w.mapA[wi], w.adig, kp, (uint64_t)w.rows_a, 1, kp, 64, blu::kBM) != RLU_OK ||
        tc_encode_bf16_3d(w.mapB[wi], w.bdig, kp, (uint64_t)w.rows_b, 1, kp, 64, blu::kNT) != RLU_OK) {
      cudaGetLastError();
      return RLU_OK;  // no tensor maps: the unblocked LUs run
    }
  }
  w.ready = true;
  return RLU_OK;
}

// The rows x cols LU of X (element (i, c) at X[i rs + c cs]), blocked or not.
template <typename T>
static int run_lu(T* X, int64_t rows, int cols, int64_t rs, int64_t cs, PivLuWs& pw, const BluWs& bw, int block,
                  unsigned int* status, int coop_sms, cudaStream_t st, PanelTimer* timer) {
  const int b = blu::choose_width(rows, cols, pw, bw, block, coop_sms);
  if (b < 0) return RLU_EINVAL;
  if (timer) {
    timer->n = 0;
    timer->width = b;
  }
  if (b == 0) return blu::timed_panel<T>(X, rows, cols, rs, cs, 0, cols, pw, status, coop_sms, st, timer);
  return blu::blocked_lu<T>(X, rows, cols, rs, cs, b, pw, bw, status, coop_sms, st, timer);
}

int launch_lu_y(double* Y, int64_t m, int l, PivLuWs& pw, const BluWs& bw, int block, unsigned int* status,
                int coop_sms, cudaStream_t st, PanelTimer* timer) {
  return run_lu<double>(Y, m, l, l, 1, pw, bw, block, status, coop_sms, st, timer);
}

template <typename T>
int launch_lu_b(T* B, int64_t n, int k, PivLuWs& pw, const BluWs& bw, int block, unsigned int* status,
                int coop_sms, cudaStream_t st, PanelTimer* timer) {
  // B^T (n x k): element (i, c) at B[c n + i]
  return run_lu<T>(B, n, k, 1, n, pw, bw, block, status, coop_sms, st, timer);
}

template int launch_lu_b<double>(double*, int64_t, int, PivLuWs&, const BluWs&, int, unsigned int*, int,
                                 cudaStream_t, PanelTimer*);
template int launch_lu_b<df32>(df32*, int64_t, int, PivLuWs&, const BluWs&, int, unsigned int*, int, cudaStream_t,
                               PanelTimer*);

}  // namespace rlu
