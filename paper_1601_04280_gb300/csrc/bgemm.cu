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
