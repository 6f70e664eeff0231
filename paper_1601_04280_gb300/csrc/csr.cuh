// Declarations of the CSR path (row classification, sparse B = W A).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "bgemm.cuh"
#include "sketch.cuh"

namespace rlu {

struct CsrWs {
  int32_t *hflag, *lflag, *hpos, *lpos, *heavy, *light, *count;  // rows (m, m+1) and counts
  int32_t *ccnt, *cstart, *crow;                                  // CSC of the light entries
  void* cval;
  void* D;   // heavy rows, dense (n_heavy x n)
  void* Wt;  // W^T (m x k)
  void* Wh;  // W restricted to the heavy rows (k x n_heavy)
  TcWs tc;   // tensor-core product of W_h and D
};

// Row classification; reads the two row counts back through `cnt` (two
// int32 of page-locked host memory).
int csr_classify(CsrWs& w, const int64_t* rowptr, int64_t m, int64_t n, int64_t nnz, unsigned int* status,
                 CsrRows& cr, int32_t* cnt, cudaStream_t st);
int csr_bgemm(CsrWs& w, const int64_t* rowptr, const int32_t* colind, const void* val, int dtype, int prec,
              int64_t m, int64_t n, int k, const CsrRows& cr, const void* W, void* B, unsigned int* status,
              int num_sms, cudaStream_t st);

}  // namespace rlu
