// Declarations of the CSR path (row classification, sparse B = W A).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "bgemm.cuh"
#include "sketch.cuh"

namespace rlu {

struct CsrWs {
  int32_t *hflag, *lflag, *hpos, *lpos, *heavy, *light, *count;  // rows (m, m+1) and counts (3)
  int32_t *mflag, *mpos, *mid;                                    // light rows sketched through the FFT
  int32_t *ccnt, *cstart;                                         // column counts and starts of the light entries
  int32_t *llen, *loff;                                           // light entries per row and their flat offsets
  int32_t *rhist, *roffs;                                         // radix sort: digit counts per chunk, offsets
  int32_t* ekey[2];                                               // light entries, two slots (keys = columns)
  int32_t* erow[2];
  void* eval[2];
  void* D;   // heavy rows, dense (n_heavy x n)
  void* Wt;  // W^T (m x k)
  void* Wh;  // W restricted to the heavy rows (k x n_heavy)
  TcWs tc;   // tensor-core product of W_h and D
  int64_t* scan_tmp;  // scratch of the multi-CTA scans (the handle's)
};

// Row classification; light rows with at most direct_max entries are
// sketched by direct evaluation (direct_max < 0: none).  Reads the three row
// counts (light, heavy, mid) and the number of light entries back through
// `cnt` (four int32 of page-locked host memory).
// Radix sort of the light entries: at most this many chunks per pass.
constexpr int64_t kRadixMaxChunks = 4096;
// Device bytes per light entry: two slots of (column, row, value up to 8 bytes).
constexpr size_t kCsrEntryBytes = 2 * (4 + 4 + 8);

int csr_classify(CsrWs& w, const int64_t* rowptr, int64_t m, int64_t n, int64_t nnz, int64_t direct_max,
                 unsigned int* status, CsrRows& cr, int32_t* cnt, cudaStream_t st);
int csr_bgemm(CsrWs& w, const int64_t* rowptr, const int32_t* colind, const void* val, int dtype, int prec,
              int64_t m, int64_t n, int k, const CsrRows& cr, const void* W, void* B, unsigned int* status,
              int num_sms, cudaStream_t st);

}  // namespace rlu
