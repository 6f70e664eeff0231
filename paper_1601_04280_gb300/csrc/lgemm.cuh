// Declarations of L = L_y L_b on the tensor cores (step 7 of Algorithm 1).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "common.cuh"

namespace rlu {

// Workspace of the digit products: the digit planes of the M-side operand
// (up to 5 x m x ldk: P L_y for L, L_y for W) and of the N-side operand (up to
// 5 x k x ldk: L_b^T for L, G^{-1} for W), their power-of-two scales, and the
// TMA descriptors of both plane stacks for each product (encoded once, at
// handle creation).
struct LtcWs {
  __nv_bfloat16* adig;  // digit planes, m x ldk each
  __nv_bfloat16* bdig;  // digit planes, k x ldk each
  int32_t* aexp;        // m
  int32_t* bexp;        // k
  int64_t m;
  int k;
  int64_t ldk;          // row stride of the planes (k rounded up to 8)
  int64_t ldm;          // rows of Lk in the Gram product's packed planes (m rounded up to 32)
  int ntileL, ntileW;   // columns per tile of the L and W products (multiples of 16)
  int num_sms;
  alignas(64) unsigned char mapAL[128];
  alignas(64) unsigned char mapBL[128];
  alignas(64) unsigned char mapAW[128];
  alignas(64) unsigned char mapBW[128];
  alignas(64) unsigned char mapAG[128];
  alignas(64) unsigned char mapBG[128];
  bool ready;
};

// Largest k the exact digit products cover (every level sum stays below 2^24).
constexpr int kLtcMaxK = 512;

size_t ltc_workspace_bytes(int64_t m, int k);
// Carve the workspace at `base` and encode the TMA descriptors; ready = false
// (the callers keep the SIMT products) when k > kLtcMaxK or tensor maps are
// unavailable.
int ltc_setup(LtcWs& w, void* base, int64_t m, int k, int num_sms);

// L (m x k, row-major FP32, rows in P order) = (P L_y) L_b, with P L_y row i =
// Lk[perm_y[i]] and L_b[t][c] = Bp[t][perm_b[c]] for t >= c (packed LU of B).
int launch_l_tc(const LtcWs& w, const df32* Lk, const int64_t* perm_y, const df32* Bp, const int64_t* perm_b,
                int64_t n, float* L, unsigned int* status, cudaStream_t st);

// G = Lk^T Lk (k x k, FP64) as six-digit products of Lk^T's digit planes,
// split over the m rows (partials in part, at most max_splits x k x k) and
// summed in split order; tiles below the diagonal come from their transposes.
int launch_gram_tc(const LtcWs& w, const df32* Lk, double* part, int max_splits, double* G, unsigned int* status,
                   cudaStream_t st);

// W (k x m, row-major FP32) = G^{-1} Lk^T with G^{-1} (k x k) and Lk (m x k)
// in float-float; with `planes` (three k x ldp BF16 arrays) also W's split
// W = W1 + W2 + W3 into BF16 planes for the tensor-core B = W A (columns
// m .. ldp-1 zero).
int launch_w_tc(const LtcWs& w, const df32* Ginv, const df32* Lk, float* W, __nv_bfloat16* const* planes,
                int64_t ldp, unsigned int* status, cudaStream_t st);

}  // namespace rlu
