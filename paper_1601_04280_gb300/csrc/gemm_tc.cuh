// B^T = A^T W^T on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Step 6 of Algorithm 1 forms B = L_y^+ (P A) = W A with W = L_y^+ P (k x m)
// and A (m x n, row-major).  The contraction runs over the m rows of A, so A
// is the M-side operand after a transpose: D = B^T tile (128 columns of A x
// N = k rounded up to 16) accumulates in tensor memory (FP32).
//
// Precision (BF16 inputs, FP32 accumulate):
//   W = W1 + W2 + W3, three BF16 planes (24 significant bits), prepared once
//     per factorization and fed by TMA (128-byte swizzle, K-major).
//   A = A1 + A2, two BF16 pieces (16 bits) formed on chip from FP32 A, or A1
//     alone when A is stored in BF16; BF16 A with 16-byte aligned rows is
//     fed by TMA as it lies in memory (MN-major: the 128 columns of a tile
//     are contiguous in each row of A).
//   D += W1 A1 + W2 A1 + W3 A1 + W1 A2 + W2 A2 (the products of order <= 2^-16).
// The rounding of A to 16 bits enters B as W dA, whose effect on L_y B is the
// projection of dA onto range(L_y); W's rounding is amplified by cond(L_y),
// so W keeps 24 bits.
//
// Warp roles (320 threads): warp 0 = TMA producer for the W planes (and for
// A when A is fed by TMA), warp 1 = TMEM owner and single-thread MMA issuer,
// warps 2..9 = two groups of four converters of A into the K-major swizzled
// BF16 layout (group g takes the k-blocks kb = g mod 2, so the global loads
// of two k-blocks are in flight at once; idle when TMA feeds A), then the
// epilogue (TMEM -> registers -> FP32 split-K partials in
// global memory, each group half of the columns).  A k-block is 64 rows of A;
// two to four pipeline stages.  Every mbarrier wait is bounded; on timeout the kernel
// raises FLAG_TIMEOUT, drains and frees its tensor memory, and returns.
#pragma once
#include <cuda.h>

#include "common.cuh"

namespace rlu {
namespace tc {

constexpr int kThreads = 320;
constexpr int kConvGroups = 2;
constexpr int kBM = 128;        // columns of A per CTA (MMA M)
constexpr int kBK = 64;         // rows of A per k-block (one 128-byte swizzle atom of BF16)
constexpr int kMaxStages = 4;  // shared-memory ring depth (the host picks 2..4 by tile size)
constexpr int kMaxN = 256;      // k rounded up to 16
constexpr uint32_t kTmemCols = 256;
constexpr long long kWaitLimit = 2000000000ll;  // cycles, about a second

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// ---- mbarrier ----------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: true on completion of the phase, false after kWaitLimit cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > kWaitLimit) return false;
  }
  return true;
}

// ---- TMA ----------------------------------------------------------------------
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// ---- tcgen05 ------------------------------------------------------------------
// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (start address and offsets in 16-byte units; version 1).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);       // start address
  d |= (uint64_t)1 << 16;                         // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;               // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                         // descriptor version
  d |= (uint64_t)2 << 61;                         // swizzle mode: 128 B
  return d;
}
// Shared-memory matrix descriptor: MN-major, 128-byte swizzle.  Each 128-byte
// row holds 64 consecutive MN elements of one K index, 8 K rows form a
// 1024-byte swizzle atom; `lbo` = bytes between 64-element MN blocks, `sbo` =
// bytes between 8-row K groups.
__device__ __forceinline__ uint64_t sw128_mn_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// Instruction descriptor, kind::f16: BF16 x BF16 -> FP32, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4)                    // D format: F32
         | (1u << 7)                  // A format: BF16
         | (1u << 10)                 // B format: BF16
         | ((uint32_t)(N >> 3) << 17) // N
         | ((uint32_t)(M >> 4) << 24);// M
}
// The same with A MN-major (the transpose-A bit).
__host__ __device__ constexpr uint32_t idesc_bf16_amn(int M, int N) { return idesc_bf16(M, N) | (1u << 15); }
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 lanes x 16 consecutive columns of FP32 from tensor memory (this warp's lane quarter).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// The same load without its wait: several loads in flight, then one
// tmem_ld_wait() before the registers are read.
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
// 32 lanes x 8 consecutive columns, without the wait.
__device__ __forceinline__ void tmem_ld8_issue(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Byte offset of element (row r, k) in a 128-byte-swizzled K-major tile of
// BF16 with 64 elements (128 B) per row: 16-byte chunk c of row r sits at
// chunk position c ^ (r mod 8).
__device__ __forceinline__ uint32_t sw128_off(int r, int k) {
  return (uint32_t)r * 128u + ((uint32_t)((k >> 3) ^ (r & 7)) << 4) + (uint32_t)(k & 7) * 2u;
}

// Shared memory of one CTA, all tiles 1024-byte aligned; per stage: the
// BF16 pieces of A (16 KB each), then the W planes (npad rows x 128 B each).
constexpr uint32_t kATile = kBM * kBK * 2;
__host__ __device__ inline uint32_t w_tile_bytes(int npad) { return (uint32_t)npad * kBK * 2; }
__host__ __device__ inline uint32_t stage_bytes(int pieces, int wplanes, int npad) {
  return (uint32_t)pieces * kATile + (uint32_t)wplanes * w_tile_bytes(npad);
}

template <typename TA>
struct ALoader;

// A in FP32: two BF16 pieces
template <>
struct ALoader<float> {
  static constexpr int kPieces = 2;
  __device__ static void split(float a, __nv_bfloat16& h, __nv_bfloat16& l) {
    h = __float2bfloat16_rn(a);
    l = __float2bfloat16_rn(a - __bfloat162float(h));
  }
};
// A in BF16: one piece, exact
template <>
struct ALoader<__nv_bfloat16> {
  static constexpr int kPieces = 1;
  __device__ static void split(__nv_bfloat16 a, __nv_bfloat16& h, __nv_bfloat16& l) {
    h = a;
    l = __float2bfloat16_rn(0.f);
  }
};

// Grid: x = (column tile of A (128 columns)) * nz + (block of npad rows of W,
// of B), so the nz CTAs that read one tile of A run side by side and share it
// through L2; y = split of the m rows (kps rows each, a multiple of 64).
// part[y][c][j] (c < k, j < n) receives the FP32 partial sum of that split.
// wplanes: BF16 planes of W used.  a_tma (BF16 A only): A fed by TMA through
// tmA (boxes of 64 columns x 64 rows, 128-byte swizzle, zeros outside A).
template <typename TA>
__global__ void __launch_bounds__(kThreads, 1)
    k_bgemm_tc(const __grid_constant__ CUtensorMap tmW1, const __grid_constant__ CUtensorMap tmW2,
               const __grid_constant__ CUtensorMap tmW3, const __grid_constant__ CUtensorMap tmA, int a_tma,
               int wplanes, const TA* __restrict__ A, int64_t lda, int64_t m, int64_t n, int k, int npad, int nz,
               int64_t kps, float* __restrict__ part, unsigned int* status, int nst) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_w[kMaxStages], full_a[kMaxStages], empty[kMaxStages], accum_full;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t j0 = (int64_t)(blockIdx.x / nz) * kBM;
  const int crow0 = (int)(blockIdx.x % nz) * npad;  // first row of W (of B) handled here
  const int64_t kbeg = (int64_t)blockIdx.y * kps;
  const int64_t kend = min64(m, kbeg + kps);
  const int nkb = (int)cdiv(kend - kbeg, kBK);
  constexpr int P = ALoader<TA>::kPieces;
  const bool atma = P == 1 && a_tma != 0;
  const uint32_t wbytes = w_tile_bytes(npad);

  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(&full_w[s], 1);
      mbar_init(&full_a[s], 128);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&accum_full, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  const uint32_t sbytes = stage_bytes(P, wplanes, npad);
  auto stageA = [&](int s, int piece) { return smem + s * sbytes + piece * kATile; };
  auto stageW = [&](int s, int plane) { return smem + s * sbytes + P * kATile + plane * w_tile_bytes(npad); };

  if (warp == 0) {
    // ---- TMA producer: W planes (and A: two boxes of 64 columns) ----
    if (lane == 0) {
      int issued = 0;
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % nst;
        if (kb >= nst && !mbar_wait(&empty[s], ((kb / nst) - 1) & 1)) { s_fail = 1; break; }
        if (s_fail) break;
        mbar_arrive_expect_tx(&full_w[s], wbytes * wplanes + (atma ? kATile : 0u));
        const int x = (int)(kbeg + (int64_t)kb * kBK);
        tma_load_2d(stageW(s, 0), &tmW1, &full_w[s], x, crow0);
        if (wplanes > 1) tma_load_2d(stageW(s, 1), &tmW2, &full_w[s], x, crow0);
        if (wplanes > 2) tma_load_2d(stageW(s, 2), &tmW3, &full_w[s], x, crow0);
        if (atma) {
          tma_load_2d(stageA(s, 0), &tmA, &full_w[s], (int)j0, x);
          tma_load_2d(stageA(s, 0) + kATile / 2, &tmA, &full_w[s], (int)j0 + kBM / 2, x);
        }
        issued = kb + 1;
      }
      // drain: every issued load has landed before the CTA may exit
      for (int kb = issued - nst < 0 ? 0 : issued - nst; kb < issued; ++kb)
        if (!mbar_wait(&full_w[kb % nst], (kb / nst) & 1)) s_fail = 1;
    }
  } else if (warp == 1) {
    // ---- MMA issuer ----
    if (lane == 0) {
      const uint32_t idesc = atma ? idesc_bf16_amn(kBM, npad) : idesc_bf16(kBM, npad);
      bool ok = true;
      for (int kb = 0; kb < nkb && ok; ++kb) {
        const int s = kb % nst;
        const uint32_t par = (kb / nst) & 1;
        if (!mbar_wait(&full_w[s], par) || (!atma && !mbar_wait(&full_a[s], par))) { ok = false; break; }
        tc_fence_after();
        const uint32_t a1 = smem_u32(stageA(s, 0)), a2 = smem_u32(stageA(s, P - 1));
#pragma unroll
        for (int kk = 0; kk < kBK / 16; ++kk) {
          const uint32_t koff = kk * 32;  // 16 BF16 = 32 bytes along K inside the swizzle atom
          // MN-major A: 16 K rows = two 1024-byte atoms; the two 64-column boxes kATile / 2 apart
          const uint64_t dA1 = atma ? sw128_mn_desc(a1 + kk * 2048u, kATile / 2, 1024u) : sw128_desc(a1 + koff);
          const uint64_t dA2 = sw128_desc(a2 + koff);
          uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
          for (int q = 0; q < wplanes; ++q) {
            const uint64_t dW = sw128_desc(smem_u32(stageW(s, q)) + koff);
            mma_bf16(tmem, dA1, dW, idesc, acc);
            acc = 1u;
          }
          if (P > 1) {
            const int q2 = wplanes < 2 ? wplanes : 2;
            for (int q = 0; q < q2; ++q) {
              const uint64_t dW = sw128_desc(smem_u32(stageW(s, q)) + koff);
              mma_bf16(tmem, dA2, dW, idesc, 1u);
            }
          }
        }
        mma_commit(&empty[s]);
      }
      if (!ok) s_fail = 1;
      mma_commit(&accum_full);
    }
  } else {
    // ---- converters (warps 2..9): A rows kb*64.. into K-major swizzled BF16 ----
    const int grp = (warp - 2) >> 2;       // 0 or 1: k-blocks kb = grp mod 2
    const int t = (threadIdx.x - 64) & 127;  // row of the tile = column j0 + t of A
    const int64_t j = j0 + t;
    // the 64 values of a k-block are loaded before waiting for its stage, so
    // the loads are in flight while the tensor cores finish the stage's
    // previous k-block
    TA vals[kBK];
    const int nkb_conv = atma ? 0 : nkb;  // nothing to convert when TMA feeds A
    auto load_kb = [&](int kb) {
      const int64_t k0 = kbeg + (int64_t)kb * kBK;
#pragma unroll
      for (int e = 0; e < kBK; ++e) {
        const int64_t row = k0 + e;
        vals[e] = (row < kend && j < n) ? A[row * lda + j] : (TA)0.f;
      }
    };
    if (grp < nkb_conv) load_kb(grp);
    for (int kb = grp; kb < nkb_conv; kb += kConvGroups) {
      const int s = kb % nst;
      if (kb >= nst && !mbar_wait(&empty[s], ((kb / nst) - 1) & 1)) { s_fail = 1; break; }
      if (s_fail) break;
      unsigned char* A1 = stageA(s, 0);
      unsigned char* A2 = stageA(s, P - 1);
#pragma unroll
      for (int c8 = 0; c8 < kBK / 8; ++c8) {
        __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) ALoader<TA>::split(vals[c8 * 8 + e], h[e], l[e]);
        const uint32_t off = sw128_off(t, c8 * 8);
        *reinterpret_cast<uint4*>(A1 + off) = *reinterpret_cast<const uint4*>(h);
        if (P > 1) *reinterpret_cast<uint4*>(A2 + off) = *reinterpret_cast<const uint4*>(l);
      }
      fence_proxy_async();
      mbar_arrive(&full_a[s]);
      if (kb + kConvGroups < nkb_conv) load_kb(kb + kConvGroups);
    }
    // ---- epilogue: TMEM -> FP32 partials part[y][c][j] ----
    const bool ok = mbar_wait(&accum_full, 0);
    tc_fence_after();
    if (!ok) {
      s_fail = 1;
    } else if (!s_fail) {
      const int quarter = warp & 3;  // TMEM lanes 32*quarter .. +31
      const int64_t jj = j0 + quarter * 32 + lane;
      float* out = part + (int64_t)blockIdx.y * k * n;
      const int nch = npad / 16, half = (nch + 1) / 2;  // 16-column chunks: group 0 the first half
      const int cb = grp == 0 ? 0 : half * 16, ce = grp == 0 ? half * 16 : npad;
      for (int c0 = cb; c0 < ce; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int c = crow0 + c0 + i;
          if (c < k && jj < n) out[(int64_t)c * n + jj] = v[i];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
  if (threadIdx.x == 0 && s_fail) set_flag(status, FLAG_TIMEOUT);
}

// W (k x m, FP64 accurate values in float-float or double) -> three BF16 planes.
template <typename TW>
__global__ void k_split_w(int64_t km, const TW* __restrict__ W, __nv_bfloat16* __restrict__ W1,
                          __nv_bfloat16* __restrict__ W2, __nv_bfloat16* __restrict__ W3) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= km) return;
  const float w = to_float(W[e]);
  const __nv_bfloat16 h1 = __float2bfloat16_rn(w);
  const float r1 = w - __bfloat162float(h1);
  const __nv_bfloat16 h2 = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(h2);
  W1[e] = h1;
  W2[e] = h2;
  W3[e] = __float2bfloat16_rn(r2);
}

// Ring depth for a tile size: as many stages (2..kMaxStages) as fit in the
// shared memory of one CTA.
inline int stages_for(int pieces, int wplanes, int npad, size_t optin) {
  int st = kMaxStages;
  while (st > 2 && (size_t)st * stage_bytes(pieces, wplanes, npad) + 1024 > optin) --st;
  return st;
}

inline size_t smem_bytes(int pieces, int wplanes, int npad, int nst) {
  return (size_t)nst * stage_bytes(pieces, wplanes, npad) + 1024;
}

}  // namespace tc
}  // namespace rlu
