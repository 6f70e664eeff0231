// L = L_y L_b on the 5th-generation tensor cores (step 7 of Algorithm 1).
//
// An exact product of integer digits, in the manner of the error-free
// splitting of Ozaki, Ogita, Oishi and Rump ("Error-free transformations of
// matrix multiplication by using fast routines of matrix multiplication and
// its applications", Numer. Algorithms 59, 2012), carried out with BF16
// tensor-core products and FP32 accumulation:
//
//   * row i of P L_y is scaled by 2^-a_i and column c of L_b by 2^-b_c
//     (powers of two: exact) into [-1, 1], and every scaled value x is cut
//     into four signed digits, x = sum_s d_s 2^(-7 s) + r 2^-28 with
//     |d_1| <= 128, |d_s| <= 64 for s > 1, |r| <= 1/2.  Digits are integers,
//     exact in BF16, and a product of two digits is an integer below 2^14.
//   * level v = s + t (2..5) collects the digit products d_s^A d_t^B; its
//     sum over the k terms of the contraction stays below 2^24 for k <= 512,
//     so the FP32 accumulation in tensor memory is exact.  One accumulator
//     per level: 10 MMAs per 16-deep step.
//   * the epilogue combines the levels, sum_v D_v 2^(-7 v), with TwoSum on
//     the FP32 pipe, scales by 2^(a_i + b_c) and rounds once to FP32.
// The only errors are the digits' truncation (2^-29 of the row and column
// scales) and the dropped levels >= 6, both far below the FP32 rounding of L.
//
// Kernel roles (192 threads): warp 0 issues the TMA loads of both digit
// stacks (128-byte swizzle, K-major), warp 1 owns tensor memory and issues the
// MMAs, warps 2..5 read the four TMEM lane quarters in the epilogue.  Every
// mbarrier wait is bounded: on timeout the kernel raises FLAG_TIMEOUT, waits
// for its own copies in flight, frees its tensor memory and returns.
#include <cuda.h>

#include "bgemm.cuh"
#include "gemm_tc.cuh"
#include "lgemm.cuh"

namespace rlu {
namespace ltc {

constexpr int kDig = 4;                    // digits per operand
constexpr int kLev = 4;                    // levels 2..5
constexpr int kBM = 128;                   // rows of L per CTA (MMA M)
constexpr int kBK = 64;                    // contraction depth per stage (one swizzle atom of BF16)
constexpr int kMaxN = 64;                  // columns of L per CTA
constexpr int kStages = 2;
constexpr int kThreads = 192;
constexpr uint32_t kTmemCols = 256;        // kLev x kMaxN
constexpr uint32_t kATile = kBM * kBK * 2;  // one digit plane of the A tile: 16 KB

__host__ __device__ inline uint32_t b_tile_bytes(int ntile) { return (uint32_t)ntile * kBK * 2; }
__host__ __device__ inline uint32_t stage_bytes(int ntile) {
  return (uint32_t)kDig * kATile + (uint32_t)kDig * b_tile_bytes(ntile);
}
inline size_t smem_bytes(int ntile) { return (size_t)kStages * stage_bytes(ntile) + 1024; }

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::
          "r"(tc::smem_u32(dst)),
      "l"(map), "r"(tc::smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// Four digits of the float-float value (hi + lo) * 2^-e, |value| <= 1 (up to
// rounding of the scale choice): each step takes the nearest integer of the
// leading part, keeps the exact remainder as a float-float pair, and moves up
// by 2^7.  Every operation is exact in FP32.
__device__ __forceinline__ void digits4(float hi, float lo, int e, __nv_bfloat16 (&d)[kDig]) {
  float yh = ldexpf(hi, 7 - e), yl = ldexpf(lo, 7 - e);
#pragma unroll
  for (int s = 0; s < kDig; ++s) {
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

// Digit planes of P L_y: one warp per row i of L (row perm[i] of Lk).
__global__ void k_digits_rows(int64_t m, int k, int64_t ldk, const df32* __restrict__ Lk,
                              const int64_t* __restrict__ perm, __nv_bfloat16* __restrict__ adig,
                              int32_t* __restrict__ aexp) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (i >= m) return;
  const df32* src = Lk + perm[i] * k;
  float amax = 0.f;
  for (int t = lane; t < k; t += 32) amax = fmaxf(amax, fabsf(src[t].hi));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  const int e = scale_exp(amax);
  if (lane == 0) aexp[i] = e;
  const int64_t plane = m * ldk;
  for (int t = lane; t < ldk; t += 32) {
    __nv_bfloat16 d[kDig];
    if (t < k) {
      const df32 v = src[t];
      digits4(v.hi, v.lo, e, d);
    } else {
#pragma unroll
      for (int s = 0; s < kDig; ++s) d[s] = __float2bfloat16_rn(0.f);
    }
#pragma unroll
    for (int s = 0; s < kDig; ++s) adig[s * plane + i * ldk + t] = d[s];
  }
}

// Digit planes of L_b^T: one warp per column c of L_b, L_b[t][c] = Bp[t][q[c]]
// for t >= c, zero above the diagonal.
__global__ void k_digits_lb(int k, int64_t n, int64_t ldk, const df32* __restrict__ Bp,
                            const int64_t* __restrict__ q, __nv_bfloat16* __restrict__ bdig,
                            int32_t* __restrict__ bexp) {
  const int lane = threadIdx.x & 31;
  const int c = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (c >= k) return;
  const int64_t col = q[c];
  float amax = 0.f;
  for (int t = c + lane; t < k; t += 32) amax = fmaxf(amax, fabsf(Bp[(int64_t)t * n + col].hi));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  const int e = scale_exp(amax);
  if (lane == 0) bexp[c] = e;
  const int64_t plane = (int64_t)k * ldk;
  for (int t = lane; t < ldk; t += 32) {
    __nv_bfloat16 d[kDig];
    if (t < k && t >= c) {
      const df32 v = Bp[(int64_t)t * n + col];
      digits4(v.hi, v.lo, e, d);
    } else {
#pragma unroll
      for (int s = 0; s < kDig; ++s) d[s] = __float2bfloat16_rn(0.f);
    }
#pragma unroll
    for (int s = 0; s < kDig; ++s) bdig[s * plane + (int64_t)c * ldk + t] = d[s];
  }
}

// One CTA per (128-row, ntile-column) tile of L; tiles ordered column tile
// fastest, so the CTAs that share a row tile read it close together in time.
__global__ void __launch_bounds__(kThreads, 1)
    k_l_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int64_t m, int k,
           int ntile, int nt, const int32_t* __restrict__ aexp, const int32_t* __restrict__ bexp,
           float* __restrict__ L, unsigned int* status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], accum_full;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ni = (int)(blockIdx.x % nt);
  const int64_t row0 = (int64_t)(blockIdx.x / nt) * kBM;
  const int col0 = ni * ntile;
  const int nkb = (k + kBK - 1) / kBK;
  const uint32_t sb = stage_bytes(ntile), bt = b_tile_bytes(ntile);
  auto tileA = [&](int s, int d) { return smem + s * sb + d * kATile; };
  auto tileB = [&](int s, int d) { return smem + s * sb + kDig * kATile + d * bt; };

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(&accum_full, 1);
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
    // ---- TMA producer: the four digit planes of both operands per stage ----
    if (lane == 0) {
      int issued = 0;
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % kStages;
        if (kb >= kStages && !tc::mbar_wait(&empty[s], ((kb / kStages) - 1) & 1)) { s_fail = 1; break; }
        if (s_fail) break;
        tc::mbar_arrive_expect_tx(&full[s], kDig * (kATile + bt));
        for (int d = 0; d < kDig; ++d) {
          tma_load_3d(tileA(s, d), &mapA, &full[s], kb * kBK, (int)row0, d);
          tma_load_3d(tileB(s, d), &mapB, &full[s], kb * kBK, col0, d);
        }
        issued = kb + 1;
      }
      // every issued load has landed before the CTA may exit
      for (int kb = issued - kStages < 0 ? 0 : issued - kStages; kb < issued; ++kb)
        if (!tc::mbar_wait(&full[kb % kStages], (kb / kStages) & 1)) s_fail = 1;
    }
  } else if (warp == 1) {
    // ---- MMA issuer: level v = s + t accumulates in columns (v - 2) * ntile ----
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16(kBM, ntile);
      bool ok = true;
      for (int kb = 0; kb < nkb && ok; ++kb) {
        const int s = kb % kStages;
        if (!tc::mbar_wait(&full[s], (kb / kStages) & 1)) { ok = false; break; }
        tc::tc_fence_after();
#pragma unroll
        for (int kk = 0; kk < kBK / 16; ++kk) {
          const uint32_t koff = kk * 32;  // 16 BF16 = 32 bytes along K inside the swizzle atom
          const bool first = (kb == 0 && kk == 0);
#pragma unroll
          for (int v = 0; v < kLev; ++v) {
            const uint32_t dcol = tmem + (uint32_t)(v * ntile);
#pragma unroll
            for (int da = 0; da <= v; ++da) {
              const int db = v - da;  // digit indices (0-based) with da + db = v
              const uint64_t aD = tc::sw128_desc(tc::smem_u32(tileA(s, da)) + koff);
              const uint64_t bD = tc::sw128_desc(tc::smem_u32(tileB(s, db)) + koff);
              tc::mma_bf16(dcol, aD, bD, idesc, (first && da == 0) ? 0u : 1u);
            }
          }
        }
        tc::mma_commit(&empty[s]);
      }
      if (!ok) s_fail = 1;
      tc::mma_commit(&accum_full);
    }
  } else {
    // ---- epilogue (warps 2..5): TMEM lane quarter = warp mod 4 ----
    const bool ok = tc::mbar_wait(&accum_full, 0);
    tc::tc_fence_after();
    if (!ok) {
      s_fail = 1;
    } else if (!s_fail) {
      const int quarter = warp & 3;
      const int64_t row = row0 + quarter * 32 + lane;
      const int ea = row < m ? aexp[row] : 0;
      const uint32_t tq = tmem + ((uint32_t)(quarter * 32) << 16);
      for (int c0 = 0; c0 < ntile; c0 += 16) {
        float v0[16], v1[16], v2[16], v3[16];
        tc::tmem_ld16(tq + (uint32_t)(0 * ntile + c0), v0);
        tc::tmem_ld16(tq + (uint32_t)(1 * ntile + c0), v1);
        tc::tmem_ld16(tq + (uint32_t)(2 * ntile + c0), v2);
        tc::tmem_ld16(tq + (uint32_t)(3 * ntile + c0), v3);
        if (row < m) {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int c = col0 + c0 + i;
            if (c < k) {
              // D_v are integers below 2^24: their scaled values are exact,
              // TwoSum keeps the two leading levels exact, the two small ones
              // enter the correction
              const df32 sum = two_sum(v0[i] * 0x1p-14f, v1[i] * 0x1p-21f);
              const float corr = sum.lo + (v2[i] * 0x1p-28f + v3[i] * 0x1p-35f);
              L[row * k + c] = ldexpf(sum.hi + corr, ea + bexp[c]);
            }
          }
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

}  // namespace ltc

namespace {
constexpr size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }
int64_t ltc_ldk(int k) { return cdiv(k, 8) * 8; }
}  // namespace

size_t ltc_workspace_bytes(int64_t m, int k) {
  const int64_t ldk = ltc_ldk(k);
  return a256((size_t)ltc::kDig * m * ldk * 2) + a256((size_t)ltc::kDig * k * ldk * 2) + a256(4 * (size_t)m) +
         a256(4 * (size_t)k);
}

int ltc_setup(LtcWs& w, void* base, int64_t m, int k) {
  w.ready = false;
  w.m = m;
  w.k = k;
  w.ldk = ltc_ldk(k);
  unsigned char* b = (unsigned char*)base;
  w.adig = (__nv_bfloat16*)b;
  b += a256((size_t)ltc::kDig * m * w.ldk * 2);
  w.bdig = (__nv_bfloat16*)b;
  b += a256((size_t)ltc::kDig * k * w.ldk * 2);
  w.aexp = (int32_t*)b;
  b += a256(4 * (size_t)m);
  w.bexp = (int32_t*)b;
  // columns per CTA: k split into equal tiles of at most 64, each a multiple of 16
  const int nt = (int)cdiv(k, ltc::kMaxN);
  w.ntile = (int)cdiv(cdiv(k, nt), 16) * 16;
  if (k > kLtcMaxK) return RLU_OK;
  if (tc_encode_bf16_3d(w.mapA, w.adig, (uint64_t)w.ldk, (uint64_t)m, ltc::kDig, (uint64_t)w.ldk, ltc::kBK,
                        ltc::kBM) != RLU_OK ||
      tc_encode_bf16_3d(w.mapB, w.bdig, (uint64_t)w.ldk, (uint64_t)k, ltc::kDig, (uint64_t)w.ldk, ltc::kBK,
                        (uint32_t)w.ntile) != RLU_OK) {
    cudaGetLastError();
    return RLU_OK;  // no tensor maps: the caller keeps the SIMT product
  }
  w.ready = true;
  return RLU_OK;
}

template <>
int launch_l_tc<df32>(const LtcWs& w, const df32* Lk, const int64_t* perm_y, const df32* Bp, const int64_t* perm_b,
                      int64_t n, float* L, unsigned int* status, cudaStream_t st) {
  if (!w.ready) return RLU_EINVAL;
  const int64_t m = w.m;
  const int k = w.k;
  ltc::k_digits_rows<<<(unsigned)cdiv(m * 32, 256), 256, 0, st>>>(m, k, w.ldk, Lk, perm_y, w.adig, w.aexp);
  RLU_CUDA_TRY(cudaGetLastError());
  ltc::k_digits_lb<<<(unsigned)cdiv((int64_t)k * 32, 256), 256, 0, st>>>(k, n, w.ldk, Bp, perm_b, w.bdig, w.bexp);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch(2);
  const size_t smem = ltc::smem_bytes(w.ntile);
  if (int rc = allow_dynamic_smem((const void*)ltc::k_l_tc, smem)) return rc;
  const int nt = (int)cdiv(k, w.ntile);
  const int64_t tiles = cdiv(m, ltc::kBM) * nt;
  ltc::k_l_tc<<<(unsigned)tiles, ltc::kThreads, smem, st>>>(
      *reinterpret_cast<const CUtensorMap*>(w.mapA), *reinterpret_cast<const CUtensorMap*>(w.mapB), m, k, w.ntile,
      nt, w.aexp, w.bexp, L, status);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  return RLU_OK;
}

}  // namespace rlu
