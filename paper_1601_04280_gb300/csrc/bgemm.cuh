// Declarations of B = W A on the tensor cores.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "common.cuh"

namespace rlu {

struct TcPlan {
  int nz;        // blocks of rows of W (each <= 208 rows)
  int npad;      // rows per block, a multiple of 16
  int64_t ldw;   // row stride of the BF16 planes of W
  int64_t kps;   // rows of A per split (multiple of 64)
  int splits;    // split-K factor
};

struct TcWs {
  TcPlan plan;
  __nv_bfloat16* wp[3];          // BF16 planes of W, k x ldw
  float* part;                    // splits x k x n FP32 partials
  alignas(64) unsigned char map[3][128];  // TMA descriptors of the planes
  int num_sms;
  bool ready;
  bool a_tma;  // BF16 A fed by TMA where its alignment allows (else by the converter warps)
};

void tc_plan(int64_t m, int64_t n, int k, int num_sms, TcPlan& p);
size_t tc_workspace_bytes(int64_t m, int64_t n, int k, int num_sms);
int tc_setup(TcWs& w, void* base, int64_t m, int64_t n, int k, int num_sms);
// TMA descriptor (128-byte swizzle) of `planes` BF16 matrices of rows x inner
// elements, row stride ld_elems (a multiple of 8), stacked one after another:
// boxes of box_inner x box_rows x 1.  RLU_ECUDA when tensor maps are
// unavailable or the encoding is refused.
int tc_encode_bf16_3d(void* map, void* base, uint64_t inner, uint64_t rows, uint64_t planes, uint64_t ld_elems,
                      uint32_t box_inner, uint32_t box_rows);
// planes_ready: W's BF16 planes are already in w.wp (written with W).
int launch_bgemm_tc(const TcWs& w, const float* W, const void* A, int64_t lda, int dtype, int prec, int64_t m,
                    int64_t n, int k, df32* B, unsigned int* status, cudaStream_t st, bool planes_ready = false);

}  // namespace rlu
