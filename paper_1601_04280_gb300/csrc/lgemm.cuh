// Declarations of L = L_y L_b on the tensor cores (step 7 of Algorithm 1).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "common.cuh"

namespace rlu {

// Workspace of the digit product: the digit planes of P L_y (4 x m x ldk) and
// of L_b^T (4 x k x ldk), their power-of-two scales, and the TMA descriptors
// of both plane stacks (encoded once, at handle creation).
struct LtcWs {
  __nv_bfloat16* adig;  // 4 planes, m x ldk: digits of row i of P L_y / 2^aexp[i]
  __nv_bfloat16* bdig;  // 4 planes, k x ldk: digits of column c of L_b / 2^bexp[c]
  int32_t* aexp;        // m
  int32_t* bexp;        // k
  int64_t m;
  int k;
  int64_t ldk;          // row stride of the planes (k rounded up to 8)
  int ntile;            // columns of L per CTA (a multiple of 16, at most 64)
  alignas(64) unsigned char mapA[128];
  alignas(64) unsigned char mapB[128];
  bool ready;
};

// Largest k the exact digit product covers (every level sum stays below 2^24).
constexpr int kLtcMaxK = 512;

size_t ltc_workspace_bytes(int64_t m, int k);
// Carve the workspace at `base` and encode the TMA descriptors; ready = false
// (the caller keeps the SIMT product) when k > kLtcMaxK or tensor maps are
// unavailable.
int ltc_setup(LtcWs& w, void* base, int64_t m, int k);

// L (m x k, row-major FP32, rows in P order) = (P L_y) L_b, with P L_y row i =
// Lk[perm_y[i]] and L_b[t][c] = Bp[t][perm_b[c]] for t >= c (packed LU of B).
template <typename T>
int launch_l_tc(const LtcWs& w, const T* Lk, const int64_t* perm_y, const T* Bp, const int64_t* perm_b, int64_t n,
                float* L, unsigned int* status, cudaStream_t st);

}  // namespace rlu
