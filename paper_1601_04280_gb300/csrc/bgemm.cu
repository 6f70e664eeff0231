// Host side of B = W A on the tensor cores (step 6 of Algorithm 1, first
// half): W split into BF16 planes, TMA descriptors of the planes, the split-K
// tcgen05 kernel and the float-float reduction of its FP32 partials.
#include <cuda.h>

#include <type_traits>

#include "bgemm.cuh"
#include "gemm_tc.cuh"

namespace rlu {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn resolve_encode_fn() {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    return (EncodeTiledFn)p;
  cudaGetLastError();
  return nullptr;
}

// Resolved once (a function-local static: initialised exactly once even when
// several threads build handles at the same time).
static EncodeTiledFn encode_fn() {
  static const EncodeTiledFn fn = resolve_encode_fn();
  return fn;
}

int tc_encode_bf16_3d(void* map, void* base, uint64_t inner, uint64_t rows, uint64_t planes, uint64_t ld_elems,
                      uint32_t box_inner, uint32_t box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return RLU_ECUDA;
  cuuint64_t dims[3] = {(cuuint64_t)inner, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)(ld_elems * 2), (cuuint64_t)(ld_elems * 2 * rows)};
  cuuint32_t box[3] = {box_inner, box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = enc(reinterpret_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box,
                   es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? RLU_OK : RLU_ECUDA;
}

// Split-K: FP32 accumulation in tensor memory runs over at most max_kps rows
// of A (its rounding error grows with that depth); the split partials are
// summed in float-float.  Enough splits to fill the GPU twice over.
static void tc_splits(int64_t m, int64_t n, int nz, int num_sms, int64_t max_kps, int64_t& kps, int& splits) {
  const int64_t xt = cdiv(n, tc::kBM);
  int64_t S = max64(cdiv(m, max_kps), cdiv(2 * (int64_t)num_sms, xt * nz));
  S = min64(S, max64(1, cdiv(m, tc::kBK)));
  kps = cdiv(cdiv(m, S), tc::kBK) * tc::kBK;
  splits = (int)cdiv(m, kps);
}

// Deepest split for each arithmetic: 512 rows keeps the FP32 product within
// FP32 parity; with W in two BF16 planes (16 bits) or one (8 bits) the W
// representation error dominates the accumulation error of much deeper splits
// (the typical relative rounding of a depth-d FP32 sum, sqrt(d) 2^-24, stays
// below 2^-17 and 2^-9 for d = 2048 and 8192).  Fewer splits, fewer partials.
static int64_t tc_max_kps(int prec) {
  if (prec == RLU_PREC_BF16) return 8192;
  if (prec == RLU_PREC_BF16_REFINE) return 2048;
  return 512;
}

void tc_plan(int64_t m, int64_t n, int k, int num_sms, TcPlan& p) {
  p.nz = (k + 207) / 208;                 // N blocks of at most 208 rows of W (fits two stages in shared memory)
  p.npad = (int)cdiv(cdiv(k, p.nz), 16) * 16;
  p.ldw = cdiv(m, 8) * 8;                 // TMA row stride: multiple of 16 bytes
  tc_splits(m, n, p.nz, num_sms, 512, p.kps, p.splits);  // the most splits any precision uses
}

size_t tc_workspace_bytes(int64_t m, int64_t n, int k, int num_sms) {
  TcPlan p;
  tc_plan(m, n, k, num_sms, p);
  return (size_t)3 * k * p.ldw * 2 + (size_t)p.splits * k * n * 4;
}

int tc_setup(TcWs& w, void* base, int64_t m, int64_t n, int k, int num_sms) {
  tc_plan(m, n, k, num_sms, w.plan);
  w.num_sms = num_sms;
  unsigned char* b = (unsigned char*)base;
  const size_t plane = (size_t)k * w.plan.ldw * 2;
  for (int q = 0; q < 3; ++q) w.wp[q] = (__nv_bfloat16*)(b + q * plane);
  w.part = (float*)(b + 3 * plane);
  w.ready = false;
  w.a_tma = true;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return RLU_OK;  // no tensor-map support: the caller uses the SIMT path
  for (int q = 0; q < 3; ++q) {
    cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)k};
    cuuint64_t strides[1] = {(cuuint64_t)(w.plan.ldw * 2)};
    cuuint32_t box[2] = {(cuuint32_t)tc::kBK, (cuuint32_t)w.plan.npad};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(reinterpret_cast<CUtensorMap*>(w.map[q]), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, w.wp[q], dims,
                     strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return RLU_OK;
  }
  w.ready = true;
  return RLU_OK;
}

// W (k x m, row-major f32) -> planes (k x ldw)
__global__ void k_split_w_rows(int64_t m, int k, int64_t ldw, const float* __restrict__ W,
                               __nv_bfloat16* __restrict__ W1, __nv_bfloat16* __restrict__ W2,
                               __nv_bfloat16* __restrict__ W3) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t c = e / ldw, i = e - c * ldw;
  if (c >= k) return;
  const float w = i < m ? W[c * m + i] : 0.f;
  const __nv_bfloat16 h1 = __float2bfloat16_rn(w);
  const float r1 = w - __bfloat162float(h1);
  const __nv_bfloat16 h2 = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(h2);
  W1[e] = h1;
  W2[e] = h2;
  W3[e] = __float2bfloat16_rn(r2);
}

// B[c][j] = sum over splits of part[s][c][j], float-float, fixed order.
__global__ void k_sum_parts(int64_t kn, int S, const float* __restrict__ part, df32* __restrict__ B) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= kn) return;
  df32 acc = df_make(0.f, 0.f);
  for (int s = 0; s < S; ++s) acc = acc + df_make(part[(int64_t)s * kn + e], 0.f);
  B[e] = acc;
}

namespace tc {

// The persistent form of the product for BF16 A fed by TMA (one or two W
// planes): one CTA per SM walks the tiles t = blockIdx.x, blockIdx.x +
// gridDim.x, ..., where tile t is W block z = t mod nz, column tile x =
// (t / nz) mod xt and split y = t / (nz xt) (the CTAs running at one time
// share their W rows and, across z, their A tiles in L2).  The stage ring runs
// on from tile to tile, and the tile's FP32 sums alternate between two
// accumulators in tensor memory (columns 0 and 256), so the epilogue of one
// tile overlaps the products of the next.  Products and their order within a
// tile are those of k_bgemm_tc.  Warps: 0 = TMA producer, 1 = TMEM owner and
// MMA issuer, 2..9 = epilogue (two groups of four, each half of the columns).
// Every wait is bounded; on timeout the kernel raises FLAG_TIMEOUT.
constexpr int kEpiWarpsP = 8;

__global__ void __launch_bounds__(kThreads, 1)
    k_bgemm_tc_persist(const __grid_constant__ CUtensorMap tmW1, const __grid_constant__ CUtensorMap tmW2,
                       const __grid_constant__ CUtensorMap tmA, int wplanes, int64_t m, int64_t n, int k, int npad,
                       int nz, int64_t xt, int64_t kps, int splits, float* __restrict__ part,
                       unsigned int* status, int nst) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages], tfull[2], tempty[2];
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntiles = (int64_t)nz * xt * splits;
  const uint32_t wbytes = w_tile_bytes(npad);
  const uint32_t sbytes = stage_bytes(1, wplanes, npad);
  auto stageA = [&](int s) { return smem + (size_t)s * sbytes; };
  auto stageW = [&](int s, int q) { return smem + (size_t)s * sbytes + kATile + (size_t)q * wbytes; };
  // tile t: W block z, first column j0 of A, split y with its rows kbeg.. and k-blocks
  auto tile = [&](int64_t t, int& z, int64_t& j0, int& y, int64_t& kbeg, int& nkb) {
    z = (int)(t % nz);
    const int64_t r = t / nz;
    j0 = (r % xt) * kBM;
    y = (int)(r / xt);
    kbeg = (int64_t)y * kps;
    nkb = (int)cdiv(min64(m, kbeg + kps) - kbeg, kBK);
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], kEpiWarpsP);
    }
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(2 * kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  volatile int* fail = &s_fail;

  if (warp == 0) {
    // ---- TMA producer ----
    if (lane == 0) {
      int64_t it = 0;  // k-blocks issued so far (all tiles)
      for (int64_t t = blockIdx.x; t < ntiles && !*fail; t += gridDim.x) {
        int z, y, nkb;
        int64_t j0, kbeg;
        tile(t, z, j0, y, kbeg, nkb);
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = (int)(it % nst);
          if (it >= nst && !mbar_wait(&empty[s], (uint32_t)((it / nst) - 1) & 1)) { *fail = 1; break; }
          if (*fail) break;
          mbar_arrive_expect_tx(&full[s], wbytes * wplanes + kATile);
          const int x = (int)(kbeg + (int64_t)kb * kBK);
          tma_load_2d(stageW(s, 0), &tmW1, &full[s], x, z * npad);
          if (wplanes > 1) tma_load_2d(stageW(s, 1), &tmW2, &full[s], x, z * npad);
          tma_load_2d(stageA(s), &tmA, &full[s], (int)j0, x);
          tma_load_2d(stageA(s) + kATile / 2, &tmA, &full[s], (int)j0 + kBM / 2, x);
        }
      }
      // drain: every issued load has landed before the CTA may exit
      for (int64_t q = it > nst ? it - nst : 0; q < it; ++q)
        if (!mbar_wait(&full[q % nst], (uint32_t)(q / nst) & 1)) *fail = 1;
    }
  } else if (warp == 1) {
    // ---- MMA issuer ----
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16_amn(kBM, npad);
      int64_t it = 0;
      int i = 0;  // tiles of this CTA so far
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++i) {
        int z, y, nkb;
        int64_t j0, kbeg;
        tile(t, z, j0, y, kbeg, nkb);
        const int b = i & 1;
        // accumulator b is free once the epilogue has read tile i - 2 out of it
        if (i >= 2 && !mbar_wait(&tempty[b], (uint32_t)((i >> 1) - 1) & 1)) { ok = false; break; }
        tc_fence_after();
        const uint32_t acc_t = tmem + (uint32_t)(b * kTmemCols);
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = (int)(it % nst);
          if (!mbar_wait(&full[s], (uint32_t)(it / nst) & 1)) { ok = false; break; }
          tc_fence_after();
          const uint32_t a1 = smem_u32(stageA(s));
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk) {
            const uint64_t dA = sw128_mn_desc(a1 + kk * 2048u, kATile / 2, 1024u);
            uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
            for (int q = 0; q < wplanes; ++q) {
              mma_bf16(acc_t, dA, sw128_desc(smem_u32(stageW(s, q)) + kk * 32u), idesc, acc);
              acc = 1u;
            }
          }
          mma_commit(&empty[s]);
        }
        if (!ok) break;
        mma_commit(&tfull[b]);
      }
      if (!ok) *fail = 1;
    }
  } else {
    // ---- epilogue: accumulator -> FP32 partials part[y][c][j] ----
    const int grp = (warp - 2) >> 2;  // column half
    const int quarter = warp & 3;     // TMEM lanes 32*quarter .. +31
    const int nch = npad / 16, half = (nch + 1) / 2;
    const int cb = grp == 0 ? 0 : half * 16, ce = grp == 0 ? half * 16 : npad;
    int i = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      int z, y, nkb;
      int64_t j0, kbeg;
      tile(t, z, j0, y, kbeg, nkb);
      const int b = i & 1;
      if (!mbar_wait(&tfull[b], (uint32_t)(i >> 1) & 1)) { *fail = 1; break; }
      tc_fence_after();
      if (*fail) break;
      const int64_t jj = j0 + quarter * 32 + lane;
      float* out = part + (int64_t)y * k * n;
      for (int c0 = cb; c0 < ce; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * kTmemCols + c0), v);
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int c = z * npad + c0 + e;
          if (c < k && jj < n) out[(int64_t)c * n + jj] = v[e];
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[b]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTmemCols) : "memory");
  }
  if (threadIdx.x == 0 && s_fail) set_flag(status, FLAG_TIMEOUT);
}

}  // namespace tc

// TMA descriptor of BF16 A (m rows x n columns, row stride lda) in boxes of 64
// columns x 64 rows with the 128-byte swizzle: the MN-major operand tiles of
// k_bgemm_tc.  False when A's base or row stride is not 16-byte aligned.
static bool encode_a_bf16(CUtensorMap* map, const __nv_bfloat16* A, int64_t lda, int64_t m, int64_t n) {
  EncodeTiledFn enc = encode_fn();
  if (!enc || ((uintptr_t)A & 15) || (lda & 7) || lda < n) return false;
  cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)m};
  cuuint64_t strides[1] = {(cuuint64_t)(lda * 2)};
  cuuint32_t box[2] = {(cuuint32_t)(tc::kBM / 2), (cuuint32_t)tc::kBK};
  cuuint32_t es[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(A), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename TA>
static int launch_cfg(const TcWs& w, int wplanes, const TA* A, int64_t lda, int64_t m, int64_t n, int k,
                      int64_t kps, int splits, unsigned int* status, cudaStream_t st) {
  constexpr int P = std::is_same<TA, float>::value ? 2 : 1;
  const TcPlan& p = w.plan;
  const CUtensorMap* maps = reinterpret_cast<const CUtensorMap*>(w.map);
  CUtensorMap tmA = maps[0];  // unused unless A is fed by TMA
  int a_tma = 0;
  if constexpr (P == 1) {
    if (w.a_tma && encode_a_bf16(&tmA, A, lda, m, n)) a_tma = 1;
    else tmA = maps[0];
  }
  int dev = 0, optin = 0;
  RLU_CUDA_TRY(cudaGetDevice(&dev));
  RLU_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const int nst = tc::stages_for(P, wplanes, p.npad, (size_t)optin - 2048);  // room for the static barriers
  const size_t smem = tc::smem_bytes(P, wplanes, p.npad, nst);
  auto kern = tc::k_bgemm_tc<TA>;
  if (a_tma && wplanes <= 2) {
    // persistent: one CTA per SM over every (W block, column tile, split)
    auto pk = tc::k_bgemm_tc_persist;
    if (int rc_ = allow_dynamic_smem((const void*)pk, smem)) return rc_;
    const int64_t xt = cdiv(n, tc::kBM);
    const int64_t ntiles = xt * p.nz * splits;
    const unsigned g = (unsigned)min64(ntiles, (int64_t)w.num_sms);
    pk<<<g, tc::kThreads, smem, st>>>(maps[0], maps[1], tmA, wplanes, m, n, k, p.npad, p.nz, xt, kps, splits,
                                      w.part, status, nst);
    RLU_CUDA_TRY(cudaGetLastError());
    note_launch();
    return RLU_OK;
  }
  if (int rc_ = allow_dynamic_smem((const void*)kern, smem)) return rc_;
  dim3 grid((unsigned)(cdiv(n, tc::kBM) * p.nz), (unsigned)splits, 1);
  kern<<<grid, tc::kThreads, smem, st>>>(maps[0], maps[1], maps[2], tmA, a_tma, wplanes, A, lda, m, n, k, p.npad,
                                         p.nz, kps, w.part, status, nst);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  return RLU_OK;
}

int launch_bgemm_tc(const TcWs& w, const float* W, const void* A, int64_t lda, int dtype, int prec, int64_t m,
                    int64_t n, int k, df32* B, unsigned int* status, cudaStream_t st, bool planes_ready) {
  if (!w.ready) return RLU_EINVAL;
  const TcPlan& p = w.plan;
  if (!planes_ready) {
    const int64_t tot = (int64_t)k * p.ldw;
    k_split_w_rows<<<(unsigned)cdiv(tot, 256), 256, 0, st>>>(m, k, p.ldw, W, w.wp[0], w.wp[1], w.wp[2]);
    RLU_CUDA_TRY(cudaGetLastError());
    note_launch();
  }
  int wplanes = 3;
  if (prec == RLU_PREC_BF16) wplanes = 1;
  if (prec == RLU_PREC_BF16_REFINE) wplanes = 2;
  int64_t kps = p.kps;
  int splits = p.splits;
  tc_splits(m, n, p.nz, w.num_sms, tc_max_kps(prec), kps, splits);
  if (splits > p.splits) return RLU_EINVAL;  // the partial buffer holds p.splits
  int rc;
  if (dtype == RLU_F32)
    rc = launch_cfg<float>(w, wplanes, (const float*)A, lda, m, n, k, kps, splits, status, st);
  else if (dtype == RLU_BF16)
    rc = launch_cfg<__nv_bfloat16>(w, wplanes, (const __nv_bfloat16*)A, lda, m, n, k, kps, splits, status, st);
  else
    return RLU_EINVAL;
  if (rc) return rc;
  k_sum_parts<<<(unsigned)cdiv((int64_t)k * n, 256), 256, 0, st>>>((int64_t)k * n, splits, w.part, B);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  return RLU_OK;
}

}  // namespace rlu
