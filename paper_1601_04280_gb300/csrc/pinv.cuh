// Declarations of B = L_y^+ P A and of the output assembly.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "lgemm.cuh"
#include "sketch.cuh"

namespace rlu {

struct PinvArgs {
  int64_t m;
  int k, l;
  const double* Y;       // m x l packed panel LU (original row order)
  const int32_t* pstep;  // m
  void* Lk;              // m x k, double if w64 else float-float
  double* gram_part;     // max_gram_splits x k x k
  int max_gram_splits;
  double* G;             // k x k (Cholesky overwrites its upper triangle)
  double* Rinv;          // k x k
  double* Ginv;          // k x k
  void* W;               // k x m, double if w64 else float
  int w64;
  unsigned int* bar;
  unsigned int* status;
  int num_sms;
  int coop_ctas;  // CTAs of the grid-synchronised Cholesky kernel (<= num_sms)
  const LtcWs* ltc;              // exact digit products on the tensor cores (or null)
  __nv_bfloat16* const* wplanes;  // with ltc: also write W's BF16 planes here (3 x k x ldw), or null
  int64_t ldw;
};

struct AssembleArgs {
  int64_t m, n;
  int k;
  const void* Lk;         // m x k, same element type as the assembly
  const int64_t* perm_y;  // m
  const int64_t* perm_b;  // n
  const void* Bp;         // k x n packed LU of B
  void* LyP;              // m x k scratch
  void* Lb;               // k x k scratch
  void* L;                // m x k output
  void* U;                // k x n output
  int64_t* p;
  int64_t* q;
  int fp32_product;  // L = L_y L_b with FP32 outputs (FP32 and BF16 forms) instead of float-float
  int num_sms;       // grid of the row-streaming FP32 product
  const LtcWs* ltc;  // the exact digit product on the tensor cores (FP32 outputs, k <= 512), or null
  unsigned int* status;
};

int launch_gram(const PinvArgs& a, cudaStream_t st);

// The paper's own second projection (Algorithm 1, steps 4-6):
// B = (Omega_2 L_1)^+ Omega_2 P A with Omega_2 = Pi_2 S_2 drawn over A's
// original rows (so Omega_2 P A = Omega_2' A and Omega_2 L_1 = Omega_2' Lk).
struct SecondArgs {
  int64_t m, n;
  int k, k2, l2;
  uint64_t seed2;
  const void* A;
  int64_t lda;
  int dtype;
  void* AT;        // n x m, A's element type: A transposed
  double* LkT;     // k x m: Lk transposed, FP64
  double* Y2T;     // n x k2: (Omega_2' A)^T
  double* ZT;      // k x k2: (Omega_2' Lk)^T
  void* W2;        // k x k2: (Z^T Z)^{-1} Z^T, double if w64 else float-float
  void* B;         // k x n output, double if w64 else float-float
};
int launch_extract_Lk(const PinvArgs& a, cudaStream_t st);
int launch_second_projection(const SecondArgs& s, const PinvArgs& a, SketchWs& ws2, cudaStream_t st);
int launch_chol(const PinvArgs& a, cudaStream_t st);
int launch_wform(const PinvArgs& a, cudaStream_t st);
template <typename T, typename TO>
int launch_assemble(const AssembleArgs& a, cudaStream_t st);
// B = W A on the SIMT pipes; `part` (bgemm_simt_splits * k * n doubles, or
// null) lets the FP64 product split its contraction when k x n is small.
int bgemm_simt_splits(int64_t m, int64_t n, int k, int num_sms);
int launch_bgemm_simt(const void* W, int w64, const void* A, int64_t lda, int dtype, int64_t m, int64_t n, int k,
                      void* B, double* part, int num_sms, cudaStream_t st);

}  // namespace rlu
