// Exact digit products on the 5th-generation tensor cores:
//   L = (P L_y) L_b          (step 7 of Algorithm 1), and
//   W = G^{-1} L_y^T         (W = L_y^+ P of Corollary 3.3, with G = L_y^T L_y).
//
// An error-free splitting in the manner of Ozaki, Ogita, Oishi and Rump
// ("Error-free transformations of matrix multiplication by using fast
// routines of matrix multiplication and its applications", Numer. Algorithms
// 59, 2012), carried out with BF16 tensor-core products and FP32 accumulation:
//
//   * every row of each operand is scaled by a power of two (exact) into
//     [-1, 1], and every scaled value x is cut into D signed digits,
//     x = sum_s d_s 2^(-7 s) + r 2^(-7 D), |d_1| <= 128, |d_s| <= 64 for s > 1,
//     |r| <= 1/2.  Digits are integers, exact in BF16; a product of two
//     digits is an integer below 2^14.
//   * level v = s + t (2 .. D + 1) collects the products d_s^A d_t^B; its sum
//     over a contraction of at most kLtcMaxK terms stays below 2^24, so the
//     FP32 accumulation in tensor memory is exact.  One accumulator per level:
//     D (D + 1) / 2 MMAs per 16-deep step.
//   * the epilogue combines the levels, sum_v D_v 2^(-7 v), with TwoSum on
//     the FP32 pipe, scales by the two powers of two and rounds once to FP32.
// The errors are the digits' truncation (2^-(7 D + 1) of the row scales) and
// the dropped levels > D + 1: 2^-29 with four digits (L), 2^-36 with five
// (W, whose entries cancel by up to cond(L_y) against |G^{-1}| |L_y^T|).
//
// The kernel is persistent: CTA b takes the tiles b, b + gridDim.x, ... (128
// rows x ntile columns each, column tile fastest).  Warp 0 streams the digit
// planes of both operands by TMA (128-byte swizzle, K-major) through a ring
// that runs across tiles; warp 1 owns tensor memory and issues the MMAs into
// one of two accumulator sets, so that warps 2..5 read the previous tile's
// accumulators (their four TMEM lane quarters) while the next tile's MMAs
// run.  Every wait is bounded: on timeout the kernel raises FLAG_TIMEOUT,
// waits for its own copies in flight, frees its tensor memory and returns.
#include <cuda.h>

#include "bgemm.cuh"
#include "gemm_tc.cuh"
#include "lgemm.cuh"

namespace rlu {
namespace ltc {

constexpr int kBM = 128;                   // rows per tile (MMA M)
constexpr int kBK = 64;                    // contraction depth per stage (one swizzle atom of BF16)
constexpr int kStages = 2;
constexpr int kThreads = 192;
constexpr uint32_t kTmemCols = 512;        // two accumulator sets of levels x ntile
constexpr uint32_t kATile = kBM * kBK * 2;  // one digit plane of the A tile: 16 KB

__host__ __device__ inline uint32_t b_tile_bytes(int ntile) { return (uint32_t)ntile * kBK * 2; }
template <int D>
__host__ __device__ inline uint32_t stage_bytes(int ntile) {
  return (uint32_t)D * (kATile + b_tile_bytes(ntile));
}
template <int D>
inline size_t smem_bytes(int ntile) {
  return (size_t)kStages * stage_bytes<D>(ntile) + 1024;
}

enum { kEpiRows = 0, kEpiTransposed = 1 };

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::
          "r"(tc::smem_u32(dst)),
      "l"(map), "r"(tc::smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// D digits of the float-float value (hi + lo) * 2^-e, |value| <= 1 (up to
// rounding of the scale choice): each step takes the nearest integer of the
// leading part, keeps the exact remainder as a float-float pair, and moves up
// by 2^7.  Every operation is exact in FP32.
template <int D>
__device__ __forceinline__ void digits(float hi, float lo, int e, __nv_bfloat16 (&d)[D]) {
  float yh = ldexpf(hi, 7 - e), yl = ldexpf(lo, 7 - e);
#pragma unroll
  for (int s = 0; s < D; ++s) {
    const float t = rintf(yh);
    d[s] = __float2bfloat16_rn(t);  // an integer of magnitude <= 128: exact
    const df32 r = two_sum(yh - t, yl);
    yh = r.hi * 128.f;
    yl = r.lo * 128.f;
  }
}

__device__ __forceinline__ int scale_exp(float amax) {
  if (!(amax > 0.f)) return 0;
  int e;
  frexpf(amax, &e);  // amax = f 2^e, f in [0.5, 1)
  return e;
}

// Digit planes of the rows of a float-float matrix X (rows x k, row-major):
// row i of the planes is row perm[i] of X (row i when perm is null), scaled
// by 2^-exps[i].  One warp per row.
template <int D>
__global__ void k_digits_rows(int64_t rows, int k, int64_t ldk, const df32* __restrict__ X,
                              const int64_t* __restrict__ perm, __nv_bfloat16* __restrict__ dig,
                              int32_t* __restrict__ exps) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (i >= rows) return;
  const df32* src = X + (perm ? perm[i] : i) * k;
  float amax = 0.f;
  for (int t = lane; t < k; t += 32) amax = fmaxf(amax, fabsf(src[t].hi));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  const int e = scale_exp(amax);
  if (lane == 0) exps[i] = e;
  const int64_t plane = rows * ldk;
  for (int t = lane; t < ldk; t += 32) {
    __nv_bfloat16 d[D];
    if (t < k) {
      const df32 v = src[t];
      digits<D>(v.hi, v.lo, e, d);
    } else {
#pragma unroll
      for (int s = 0; s < D; ++s) d[s] = __float2bfloat16_rn(0.f);
    }
#pragma unroll
    for (int s = 0; s < D; ++s) dig[s * plane + i * ldk + t] = d[s];
  }
}

// Digit planes of L_b^T: one warp per column c of L_b, L_b[t][c] = Bp[t][q[c]]
// for t >= c, zero above the diagonal.
template <int D>
__global__ void k_digits_lb(int k, int64_t n, int64_t ldk, const df32* __restrict__ Bp,
                            const int64_t* __restrict__ q, __nv_bfloat16* __restrict__ dig,
                            int32_t* __restrict__ exps) {
  const int lane = threadIdx.x & 31;
  const int c = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (c >= k) return;
  const int64_t col = q[c];
  float amax = 0.f;
  for (int t = c + lane; t < k; t += 32) amax = fmaxf(amax, fabsf(Bp[(int64_t)t * n + col].hi));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  const int e = scale_exp(amax);
  if (lane == 0) exps[c] = e;
  const int64_t plane = (int64_t)k * ldk;
  for (int t = lane; t < ldk; t += 32) {
    __nv_bfloat16 d[D];
    if (t < k && t >= c) {
      const df32 v = Bp[(int64_t)t * n + col];
      digits<D>(v.hi, v.lo, e, d);
    } else {
#pragma unroll
      for (int s = 0; s < D; ++s) d[s] = __float2bfloat16_rn(0.f);
    }
#pragma unroll
    for (int s = 0; s < D; ++s) dig[s * plane + (int64_t)c * ldk + t] = d[s];
  }
}

struct EpiOut {
  float* out;            // rows: out[row * ldo + col]; transposed: out[col * ldo + row]
  int64_t ldo;
  __nv_bfloat16* pl[3];  // transposed only (optional): BF16 planes of out, [col * ldp + row] for row < ldp
  int64_t ldp;
};

// C (M x N) = A (M x K) B^T (N x K) from D digit planes of each operand.
template <int D, int EPI>
__global__ void __launch_bounds__(kThreads, 1)
    k_digit_gemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int64_t M,
                 int N, int K, int ntile, int nt, int64_t tiles, const int32_t* __restrict__ aexp,
                 const int32_t* __restrict__ bexp, EpiOut eo, unsigned int* status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], tfull[2], tempty[2];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkb = (K + kBK - 1) / kBK;
  const uint32_t sb = stage_bytes<D>(ntile), bt = b_tile_bytes(ntile);
  const uint32_t set_cols = (uint32_t)(D * ntile);  // one accumulator set: D levels of ntile columns
  auto tileA = [&](int s, int d) { return smem + s * sb + d * kATile; };
  auto tileB = [&](int s, int d) { return smem + s * sb + D * kATile + d * bt; };

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&tfull[b], 1);
      tc::mbar_init(&tempty[b], 4);  // one arrival per epilogue warp
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
    // ---- TMA producer: D digit planes of both operands per stage ----
    if (lane == 0) {
      int64_t it = 0;
      for (int64_t tile = blockIdx.x; tile < tiles && !s_fail; tile += gridDim.x) {
        const int row0 = (int)((tile / nt) * kBM), col0 = (int)(tile % nt) * ntile;
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = (int)(it % kStages);
          if (it >= kStages && !tc::mbar_wait(&empty[s], (uint32_t)(((it / kStages) - 1) & 1))) {
            s_fail = 1;
            break;
          }
          tc::mbar_arrive_expect_tx(&full[s], D * (kATile + bt));
          for (int d = 0; d < D; ++d) {
            tma_load_3d(tileA(s, d), &mapA, &full[s], kb * kBK, row0, d);
            tma_load_3d(tileB(s, d), &mapB, &full[s], kb * kBK, col0, d);
          }
        }
      }
      // every issued load has landed before the CTA may exit
      for (int64_t j = it - kStages < 0 ? 0 : it - kStages; j < it; ++j)
        if (!tc::mbar_wait(&full[j % kStages], (uint32_t)((j / kStages) & 1))) s_fail = 1;
    }
  } else if (warp == 1) {
    // ---- MMA issuer: level v (0-based) of set b in columns b * set_cols + v * ntile ----
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16(kBM, ntile);
      int64_t it = 0, local = 0;
      bool ok = true;
      for (int64_t tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x, ++local) {
        const int b = (int)(local & 1);
        if (local >= 2 && !tc::mbar_wait(&tempty[b], (uint32_t)(((local >> 1) - 1) & 1))) { ok = false; break; }
        tc::tc_fence_after();
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = (int)(it % kStages);
          if (!tc::mbar_wait(&full[s], (uint32_t)((it / kStages) & 1))) { ok = false; break; }
          tc::tc_fence_after();
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk) {
            const uint32_t koff = kk * 32;  // 16 BF16 = 32 bytes along K inside the swizzle atom
            const bool first = (kb == 0 && kk == 0);
#pragma unroll
            for (int v = 0; v < D; ++v) {
              const uint32_t dcol = tmem + (uint32_t)b * set_cols + (uint32_t)(v * ntile);
#pragma unroll
              for (int da = 0; da <= v; ++da) {
                const uint64_t aD = tc::sw128_desc(tc::smem_u32(tileA(s, da)) + koff);
                const uint64_t bD = tc::sw128_desc(tc::smem_u32(tileB(s, v - da)) + koff);
                tc::mma_bf16(dcol, aD, bD, idesc, (first && da == 0) ? 0u : 1u);
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
    // ---- epilogue (warps 2..5): TMEM lane quarter = warp mod 4 ----
    const int quarter = warp & 3;
    // rows layout: each 32 x 16 piece goes out through a staging block in
    // shared memory (a thread owns a row in tensor memory; lanes writing their
    // own rows would cost a transaction per row), two 64-byte row pieces per
    // store instruction
    float* stg = reinterpret_cast<float*>(smem + (uint32_t)kStages * sb) + (warp - 2) * 32 * 17;
    int64_t local = 0;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++local) {
      const int b = (int)(local & 1);
      if (!tc::mbar_wait(&tfull[b], (uint32_t)((local >> 1) & 1))) { s_fail = 1; break; }
      tc::tc_fence_after();
      const int64_t rbase = (tile / nt) * kBM + quarter * 32;
      const int64_t row = rbase + lane;
      const int col0 = (int)(tile % nt) * ntile;
      const int ea = row < M ? aexp[row] : 0;
      const uint32_t tq = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)b * set_cols;
      for (int c0 = 0; c0 < ntile; c0 += 16) {
        float v[D][16];
#pragma unroll
        for (int lv = 0; lv < D; ++lv) tc::tmem_ld16(tq + (uint32_t)(lv * ntile + c0), v[lv]);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int c = col0 + c0 + i;
          if (c >= N) continue;
          // level sums are integers below 2^24: scaled, they are exact; TwoSum
          // keeps the two leading levels exact, the others enter the correction
          const df32 sum = two_sum(v[0][i] * 0x1p-14f, v[1][i] * 0x1p-21f);
          float corr = 0.f;
#pragma unroll
          for (int lv = D - 1; lv >= 2; --lv) corr += v[lv][i] * ldexpf(1.f, -7 * (lv + 2));
          const float r = (row < M) ? ldexpf(sum.hi + (sum.lo + corr), ea + bexp[c]) : 0.f;
          if (EPI == kEpiRows) {
            stg[lane * 17 + i] = r;
          } else {
            if (row < M) eo.out[(int64_t)c * eo.ldo + row] = r;
            if (eo.pl[0] && row < eo.ldp) {
              const __nv_bfloat16 h1 = __float2bfloat16_rn(r);
              const float r1 = r - __bfloat162float(h1);
              const __nv_bfloat16 h2 = __float2bfloat16_rn(r1);
              const int64_t o = (int64_t)c * eo.ldp + row;
              eo.pl[0][o] = h1;
              eo.pl[1][o] = h2;
              eo.pl[2][o] = __float2bfloat16_rn(r1 - __bfloat162float(h2));
            }
          }
        }
        if (EPI == kEpiRows) {
          __syncwarp();
#pragma unroll
          for (int it = 0; it < 16; ++it) {
            const int rr = it * 2 + (lane >> 4), cc = lane & 15;
            const int c = col0 + c0 + cc;
            if (rbase + rr < M && c < N) eo.out[(rbase + rr) * eo.ldo + c] = stg[rr * 17 + cc];
          }
          __syncwarp();
        }
      }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&tempty[b]);
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

// Digit planes of Lk^T from Lk (m x k float-float, row-major), unscaled:
// every column of Lk holds a 1 (its pivot row) and no entry above 1 in
// magnitude (partial pivoting), so its power-of-two scale is 2^0.  Row c of
// the output is column c of Lk packed by 32-row chunk, then digit:
// dig[c][q D 32 + s 32 + r] = digit s of Lk[32 q + r][c] (ldm = m rounded up
// to 32 rows; rows m .. ldm-1 are zeros).  A 32 x 32 tile per CTA through
// shared memory.
template <int D>
__global__ void __launch_bounds__(256) k_digits_cols(int64_t m, int k, int64_t ldm, const df32* __restrict__ Lk,
                                                     __nv_bfloat16* __restrict__ dig) {
  __shared__ df32 t[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32;  // chunk q = blockIdx.x
  const int c0 = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t r = r0 + y;
    const int c = c0 + threadIdx.x;
    t[y][threadIdx.x] = (r < m && c < k) ? Lk[r * k + c] : df_make(0.f, 0.f);
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int c = c0 + y;
    if (c >= k) continue;
    const df32 v = t[threadIdx.x][y];
    __nv_bfloat16 d[D];
    digits<D>(v.hi, v.lo, 0, d);
    __nv_bfloat16* row = dig + (int64_t)c * D * ldm + (int64_t)blockIdx.x * D * 32 + threadIdx.x;
#pragma unroll
    for (int s = 0; s < D; ++s) row[s * 32] = d[s];
  }
}

// G = Lk^T Lk (k x k) from the packed digit planes of Lk^T: work item = (row
// tile of 128, column tile of 32, split of the m-long contraction); tiles
// wholly below the diagonal are skipped (G is symmetric).  A pipeline stage
// holds all D digits of a 32-row chunk of both operands (three 128-byte
// boxes each for D = 6).  A split runs over its rows in exact chunks of at
// most kGramExactQ x 32 rows (every level sum below 2^24): the MMAs of a
// chunk fill one of two TMEM accumulator sets while the epilogue combines the
// previous chunk's levels (TwoSum) and adds them to float-float running sums;
// after its last chunk an item writes its FP64 partial part[split][c][c'].
constexpr int kGramN = 32;       // columns per tile
constexpr int kGramQ = 32;       // rows of Lk per pipeline stage
constexpr int kGramExactQ = 14;  // 448 rows per exact chunk
constexpr int kGramStages = 3;

__host__ __device__ inline bool gram_tile_below(int im, int in) { return in * kGramN + kGramN - 1 < im * kBM; }

template <int D>
__host__ __device__ constexpr uint32_t gram_stage_bytes() {
  return (uint32_t)(D * kGramQ / 64) * (uint32_t)(kBM * 128 + kGramN * 128);
}

template <int D>
__global__ void __launch_bounds__(kThreads, 1)
    k_digit_gram(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int k, int tm,
                 int tn, int S, int64_t nq, int64_t q_per_split, double* __restrict__ part, unsigned int* status) {
  static_assert((D * kGramQ) % 64 == 0, "a stage is whole 128-byte boxes");
  constexpr int NBOX = D * kGramQ / 64;
  constexpr uint32_t ABOX = kBM * 128, BBOX = kGramN * 128;
  constexpr uint32_t SB = gram_stage_bytes<D>();
  constexpr uint32_t SET = D * kGramN;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[kGramStages], empty[kGramStages], tfull[2], tempty[2];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t items = (int64_t)tm * tn * S;
  auto boxA = [&](int s, int j) { return smem + (uint32_t)s * SB + (uint32_t)j * ABOX; };
  auto boxB = [&](int s, int j) { return smem + (uint32_t)s * SB + NBOX * ABOX + (uint32_t)j * BBOX; };
  // item -> (row tile, column tile, split) and its chunk range; false for a
  // tile below the diagonal (every role skips it alike)
  auto decode = [&](int64_t item, int& it_m, int& it_n, int64_t& q0, int64_t& q1) -> bool {
    const int sp = (int)(item / ((int64_t)tm * tn));
    const int rest = (int)(item - (int64_t)sp * tm * tn);
    it_m = rest / tn;
    it_n = rest - it_m * tn;
    q0 = (int64_t)sp * q_per_split;
    q1 = min64(nq, q0 + q_per_split);
    return !gram_tile_below(it_m, it_n) && q0 < q1;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < kGramStages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&tfull[b], 1);
      tc::mbar_init(&tempty[b], 4);
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
    if (lane == 0) {
      int64_t it = 0;
      for (int64_t item = blockIdx.x; item < items && !s_fail; item += gridDim.x) {
        int im, in_;
        int64_t q0, q1;
        if (!decode(item, im, in_, q0, q1)) continue;
        for (int64_t q = q0; q < q1; ++q, ++it) {
          const int s = (int)(it % kGramStages);
          if (it >= kGramStages && !tc::mbar_wait(&empty[s], (uint32_t)(((it / kGramStages) - 1) & 1))) {
            s_fail = 1;
            break;
          }
          tc::mbar_arrive_expect_tx(&full[s], SB);
          for (int j = 0; j < NBOX; ++j) {
            const int x = (int)(q * D * kGramQ) + j * 64;
            tma_load_3d(boxA(s, j), &mapA, &full[s], x, im * kBM, 0);
            tma_load_3d(boxB(s, j), &mapB, &full[s], x, in_ * kGramN, 0);
          }
        }
      }
      for (int64_t j = it - kGramStages < 0 ? 0 : it - kGramStages; j < it; ++j)
        if (!tc::mbar_wait(&full[j % kGramStages], (uint32_t)((j / kGramStages) & 1))) s_fail = 1;
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16(kBM, kGramN);
      int64_t it = 0, unit = 0;
      bool ok = true;
      for (int64_t item = blockIdx.x; item < items && ok; item += gridDim.x) {
        int im, in_;
        int64_t q0, q1;
        if (!decode(item, im, in_, q0, q1)) continue;
        for (int64_t c0 = q0; c0 < q1 && ok; c0 += kGramExactQ, ++unit) {
          const int b = (int)(unit & 1);
          if (unit >= 2 && !tc::mbar_wait(&tempty[b], (uint32_t)(((unit >> 1) - 1) & 1))) { ok = false; break; }
          tc::tc_fence_after();
          const int64_t c1 = min64(q1, c0 + kGramExactQ);
          for (int64_t q = c0; q < c1; ++q, ++it) {
            const int s = (int)(it % kGramStages);
            if (!tc::mbar_wait(&full[s], (uint32_t)((it / kGramStages) & 1))) { ok = false; break; }
            tc::tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < kGramQ / 16; ++kk) {
#pragma unroll
              for (int v = 0; v < D; ++v) {
                const uint32_t dcol = tmem + (uint32_t)b * SET + (uint32_t)(v * kGramN);
#pragma unroll
                for (int da = 0; da <= v; ++da) {
                  const int ka = da * kGramQ + kk * 16, kb = (v - da) * kGramQ + kk * 16;
                  const uint64_t aD = tc::sw128_desc(tc::smem_u32(boxA(s, ka >> 6)) + (uint32_t)(ka & 63) * 2u);
                  const uint64_t bD = tc::sw128_desc(tc::smem_u32(boxB(s, kb >> 6)) + (uint32_t)(kb & 63) * 2u);
                  tc::mma_bf16(dcol, aD, bD, idesc, (q == c0 && kk == 0 && da == 0) ? 0u : 1u);
                }
              }
            }
            tc::mma_commit(&empty[s]);
          }
          if (ok) tc::mma_commit(&tfull[b]);
        }
      }
      if (!ok) s_fail = 1;
    }
  } else {
    const int quarter = warp & 3;
    int64_t unit = 0;
    bool ok = true;
    for (int64_t item = blockIdx.x; item < items && ok; item += gridDim.x) {
      int im, in_;
      int64_t q0, q1;
      if (!decode(item, im, in_, q0, q1)) continue;
      const int sp = (int)(item / ((int64_t)tm * tn));
      float rh[kGramN], rl[kGramN];  // running float-float sums of this row's columns
#pragma unroll
      for (int i = 0; i < kGramN; ++i) rh[i] = rl[i] = 0.f;
      for (int64_t c0 = q0; c0 < q1; c0 += kGramExactQ, ++unit) {
        const int b = (int)(unit & 1);
        if (!tc::mbar_wait(&tfull[b], (uint32_t)((unit >> 1) & 1))) { s_fail = 1; ok = false; break; }
        tc::tc_fence_after();
        const uint32_t tq = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)b * SET;
#pragma unroll
        for (int h = 0; h < kGramN / 16; ++h) {
          float v[D][16];
#pragma unroll
          for (int lv = 0; lv < D; ++lv) tc::tmem_ld16(tq + (uint32_t)(lv * kGramN + h * 16), v[lv]);
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const df32 head = two_sum(v[0][i] * 0x1p-14f, v[1][i] * 0x1p-21f);
            float corr = 0.f;
#pragma unroll
            for (int lv = D - 1; lv >= 2; --lv) corr += v[lv][i] * ldexpf(1.f, -7 * (lv + 2));
            const df32 chunk = quick_two_sum(head.hi, head.lo + corr);
            const df32 acc = df_make(rh[h * 16 + i], rl[h * 16 + i]) + chunk;
            rh[h * 16 + i] = acc.hi;
            rl[h * 16 + i] = acc.lo;
          }
        }
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&tempty[b]);
      }
      if (!ok) break;
      const int c = im * kBM + quarter * 32 + lane;
      if (c < k) {
        double* out = part + (int64_t)sp * k * k + (int64_t)c * k;
#pragma unroll
        for (int i = 0; i < kGramN; ++i) {
          const int c2 = in_ * kGramN + i;
          if (c2 < k) out[c2] = (double)rh[i] + (double)rl[i];
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

// G[c][c'] = the sum over the S splits of the partials, in split order; an
// entry whose tile was skipped (below the diagonal) takes its transpose's.
__global__ void k_sum_gram(int k, int S, const double* __restrict__ part, double* __restrict__ G) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)k * k) return;
  const int r = (int)(e / k), c = (int)(e - (int64_t)r * k);
  const int64_t src = gram_tile_below(r / kBM, c / kGramN) ? (int64_t)c * k + r : e;
  double s = 0.0;
  for (int z = 0; z < S; ++z) s += part[(int64_t)z * k * k + src];
  G[e] = s;
}

// Columns per tile for N output columns: equal tiles, multiples of 16, at
// most 512 / (2 D) columns (two accumulator sets of D levels in TMEM).
inline int tile_cols(int N, int D) {
  const int maxn = (512 / (2 * D)) / 16 * 16;
  const int nt = (int)cdiv(N, maxn);
  return (int)cdiv(cdiv(N, nt), 16) * 16;
}

template <int D, int EPI>
int launch_gemm(const void* mapA, const void* mapB, int64_t M, int N, int K, int ntile, const int32_t* aexp,
                const int32_t* bexp, const EpiOut& eo, unsigned int* status, int num_sms, cudaStream_t st) {
  // the rows layout's staging blocks (four epilogue warps, 32 x 17 floats each) after the stages
  const size_t smem = smem_bytes<D>(ntile) + (EPI == kEpiRows ? (size_t)4 * 32 * 17 * sizeof(float) : 0);
  auto kern = k_digit_gemm<D, EPI>;
  if (int rc = allow_dynamic_smem((const void*)kern, smem)) return rc;
  const int nt = (int)cdiv(N, ntile);
  const int64_t tiles = cdiv(M, kBM) * nt;
  const unsigned grid = (unsigned)min64(tiles, (int64_t)num_sms);
  kern<<<grid, kThreads, smem, st>>>(*reinterpret_cast<const CUtensorMap*>(mapA),
                                     *reinterpret_cast<const CUtensorMap*>(mapB), M, N, K, ntile, nt, tiles, aexp,
                                     bexp, eo, status);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  return RLU_OK;
}

}  // namespace ltc

namespace {
constexpr size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }
int64_t ltc_ldk(int k) { return cdiv(k, 8) * 8; }
constexpr int kDigL = 4;  // digits of the L product
constexpr int kDigW = 5;  // digits of the W product
constexpr int kDigG = 6;  // digits of the Gram product
// the M-side planes: row layout (m x ldk) for L and W, transposed (k x ldm) for G
size_t adig_bytes(int64_t m, int k) {
  const size_t rows = (size_t)kDigW * m * ltc_ldk(k) * 2;
  const size_t cols = (size_t)kDigG * k * (size_t)(cdiv(m, 32) * 32) * 2;
  return a256(rows > cols ? rows : cols);
}
}  // namespace

size_t ltc_workspace_bytes(int64_t m, int k) {
  const int64_t ldk = ltc_ldk(k);
  return adig_bytes(m, k) + a256((size_t)kDigW * k * ldk * 2) + a256(4 * (size_t)m) + a256(4 * (size_t)k);
}

int ltc_setup(LtcWs& w, void* base, int64_t m, int k, int num_sms) {
  w.ready = false;
  w.m = m;
  w.k = k;
  w.num_sms = num_sms;
  w.ldk = ltc_ldk(k);
  w.ldm = cdiv(m, 32) * 32;
  unsigned char* b = (unsigned char*)base;
  w.adig = (__nv_bfloat16*)b;
  b += adig_bytes(m, k);
  w.bdig = (__nv_bfloat16*)b;
  b += a256((size_t)kDigW * k * w.ldk * 2);
  w.aexp = (int32_t*)b;
  b += a256(4 * (size_t)m);
  w.bexp = (int32_t*)b;
  w.ntileL = ltc::tile_cols(k, kDigL);
  w.ntileW = ltc::tile_cols(k, kDigW);
  if (k > kLtcMaxK) return RLU_OK;
  // the same planes serve both products: four of them for L, five for W
  const uint64_t ldk = (uint64_t)w.ldk;
  if (tc_encode_bf16_3d(w.mapAL, w.adig, ldk, (uint64_t)m, kDigL, ldk, ltc::kBK, ltc::kBM) != RLU_OK ||
      tc_encode_bf16_3d(w.mapBL, w.bdig, ldk, (uint64_t)k, kDigL, ldk, ltc::kBK, (uint32_t)w.ntileL) != RLU_OK ||
      tc_encode_bf16_3d(w.mapAW, w.adig, ldk, (uint64_t)m, kDigW, ldk, ltc::kBK, ltc::kBM) != RLU_OK ||
      tc_encode_bf16_3d(w.mapBW, w.bdig, ldk, (uint64_t)k, kDigW, ldk, ltc::kBK, (uint32_t)w.ntileW) != RLU_OK ||
      tc_encode_bf16_3d(w.mapAG, w.adig, (uint64_t)kDigG * w.ldm, (uint64_t)k, 1, (uint64_t)kDigG * w.ldm, 64,
                        ltc::kBM) != RLU_OK ||
      tc_encode_bf16_3d(w.mapBG, w.adig, (uint64_t)kDigG * w.ldm, (uint64_t)k, 1, (uint64_t)kDigG * w.ldm, 64,
                        ltc::kGramN) != RLU_OK) {
    cudaGetLastError();
    return RLU_OK;  // no tensor maps: the callers keep the SIMT products
  }
  w.ready = true;
  return RLU_OK;
}

int launch_l_tc(const LtcWs& w, const df32* Lk, const int64_t* perm_y, const df32* Bp, const int64_t* perm_b,
                int64_t n, float* L, unsigned int* status, cudaStream_t st) {
  if (!w.ready) return RLU_EINVAL;
  const int64_t m = w.m;
  const int k = w.k;
  ltc::k_digits_rows<kDigL><<<(unsigned)cdiv(m * 32, 256), 256, 0, st>>>(m, k, w.ldk, Lk, perm_y, w.adig, w.aexp);
  RLU_CUDA_TRY(cudaGetLastError());
  ltc::k_digits_lb<kDigL><<<(unsigned)cdiv((int64_t)k * 32, 256), 256, 0, st>>>(k, n, w.ldk, Bp, perm_b, w.bdig,
                                                                                 w.bexp);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch(2);
  ltc::EpiOut eo{};
  eo.out = L;
  eo.ldo = k;
  return ltc::launch_gemm<kDigL, ltc::kEpiRows>(w.mapAL, w.mapBL, m, k, k, w.ntileL, w.aexp, w.bexp, eo, status,
                                                w.num_sms, st);
}

int launch_w_tc(const LtcWs& w, const df32* Ginv, const df32* Lk, float* W, __nv_bfloat16* const* planes,
                int64_t ldp, unsigned int* status, cudaStream_t st) {
  if (!w.ready) return RLU_EINVAL;
  const int64_t m = w.m;
  const int k = w.k;
  // W^T (m x k) = Lk G^{-T} = Lk G^{-1} (G symmetric): rows of Lk against rows of G^{-1}
  ltc::k_digits_rows<kDigW><<<(unsigned)cdiv(m * 32, 256), 256, 0, st>>>(m, k, w.ldk, Lk, nullptr, w.adig, w.aexp);
  RLU_CUDA_TRY(cudaGetLastError());
  ltc::k_digits_rows<kDigW><<<(unsigned)cdiv((int64_t)k * 32, 256), 256, 0, st>>>(k, k, w.ldk, Ginv, nullptr,
                                                                                  w.bdig, w.bexp);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch(2);
  ltc::EpiOut eo{};
  eo.out = W;
  eo.ldo = m;
  if (planes) {
    for (int q = 0; q < 3; ++q) eo.pl[q] = planes[q];
    eo.ldp = ldp;
  }
  return ltc::launch_gemm<kDigW, ltc::kEpiTransposed>(w.mapAW, w.mapBW, m, k, k, w.ntileW, w.aexp, w.bexp, eo,
                                                      status, w.num_sms, st);
}

int launch_gram_tc(const LtcWs& w, const df32* Lk, double* part, int max_splits, double* G, unsigned int* status,
                   cudaStream_t st) {
  if (!w.ready) return RLU_EINVAL;
  const int64_t m = w.m;
  const int k = w.k;
  const dim3 gd((unsigned)(w.ldm / 32), (unsigned)cdiv(k, 32));
  ltc::k_digits_cols<kDigG><<<gd, dim3(32, 8), 0, st>>>(m, k, w.ldm, Lk, w.adig);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  const int tm = (int)cdiv(k, ltc::kBM), tn = (int)cdiv(k, ltc::kGramN);
  int64_t kept = 0;
  for (int im = 0; im < tm; ++im)
    for (int in = 0; in < tn; ++in) kept += ltc::gram_tile_below(im, in) ? 0 : 1;
  const int64_t nq = w.ldm / ltc::kGramQ;
  // splits: about two work items per SM, each at least one exact chunk deep
  int64_t S = cdiv(2 * (int64_t)w.num_sms, kept);
  S = min64(S, (int64_t)max_splits);
  S = min64(S, cdiv(nq, ltc::kGramExactQ));
  S = max64(S, 1);
  const int64_t qps = cdiv(nq, S);
  S = cdiv(nq, qps);
  const size_t smem = (size_t)ltc::kGramStages * ltc::gram_stage_bytes<kDigG>() + 1024;
  auto kern = ltc::k_digit_gram<kDigG>;
  if (int rc = allow_dynamic_smem((const void*)kern, smem)) return rc;
  const int64_t items = (int64_t)tm * tn * S;
  const unsigned grid = (unsigned)min64(items, (int64_t)w.num_sms);
  kern<<<grid, ltc::kThreads, smem, st>>>(*reinterpret_cast<const CUtensorMap*>(w.mapAG),
                                          *reinterpret_cast<const CUtensorMap*>(w.mapBG), k, tm, tn, (int)S, nq, qps,
                                          part, status);
  RLU_CUDA_TRY(cudaGetLastError());
  ltc::k_sum_gram<<<(unsigned)cdiv((int64_t)k * k, 256), 256, 0, st>>>(k, (int)S, part, G);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch(2);
  return RLU_OK;
}

}  // namespace rlu
