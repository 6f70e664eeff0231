// Declarations of the sketch step (step 1 and 2 of Algorithm 1).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace rlu {

constexpr int kMaxFftStages = 24;

// Radices of the mixed-radix FFT of length l1, applied in order.
// Mixed-radix plan of an N-point Stockham FFT.  Per stage: radix r, the
// product p of the radices already applied, T = N / r butterflies per
// transform, the twiddle stride N / (p r), and multipliers for division by T
// and by p without a divide instruction: for 0 <= x < 2^16 and 2 <= d < 2^16,
// floor(x / d) = umulhi(x, ceil(2^32 / d)) exactly (0 marks d = 1).
struct FftPlan {
  int nstages;
  int radix[kMaxFftStages];
  int p[kMaxFftStages];
  int T[kMaxFftStages];
  int step[kMaxFftStages];
  uint32_t mT[kMaxFftStages];
  uint32_t mp[kMaxFftStages];
};

// Device buffers of the sketch step (owned by the handle).
struct SketchWs {
  uint32_t* hs;     // n: bucket h(j) in bits 0..30, sign s(j) < 0 in bit 31
  float* dsign;     // l1: +-1
  uint64_t* keys;   // l1: subsample selection keys
  int32_t* R;       // l: selected frequencies
  int chunk;        // columns per staged tile of the dense sketch
  int64_t nchunks;  // ceil(n / chunk)
  int32_t* bcnt;    // nchunks*l1 + 1: scratch counters
  int32_t* bstart;  // nchunks*l1 + 1: start of each (chunk, bucket) list
  uint32_t* blist;  // n: column offset within its chunk | sign bit, sorted by (chunk, bucket, column)
  double2* tw64;    // l1 twiddles exp(-2 pi i e / l1)
  float2* tw32;
  FftPlan plan;
  int64_t* scan_tmp;  // kScanMaxParts partial sums of the multi-CTA scan (null: one-CTA scan)
};

constexpr int kScanMaxParts = 4096;

// Rows of a CSR matrix split into light rows and heavy rows (a CTA each,
// densified), as device lists with device counts.  Light rows with at most
// direct_max entries are sketched by direct evaluation against the table of
// the projection (a warp each); the other light rows ("mid") by the FFT.
struct CsrRows {
  int32_t* light;      // light row indices, ascending
  int32_t* heavy;      // heavy row indices, ascending
  int32_t* mid;        // light rows with more than direct_max entries, ascending
  int32_t* d_count;    // device: [n_light, n_heavy, n_mid]
  int64_t n_light, n_heavy, n_mid;  // host copies
  int64_t n_light_nnz;                // entries of the light rows
  int64_t direct_max;  // < 0: no direct evaluation
};

// Largest l1 for which the CSR sketch evaluates sparse rows directly (the
// l1 x l table of D H R / sqrt(l1) then takes at most kDirectMaxL1 x 1024 x 4 bytes).
constexpr int kDirectMaxL1 = 2560;
// Light rows evaluated directly: at most this many entries per row (about
// the work of one FFT of length l1 per row).
inline int64_t csr_direct_max(int l1, int l) {
  if (l1 > kDirectMaxL1) return -1;
  int lg = 0;
  for (int x = l1; x > 1; x >>= 1) ++lg;
  return ((int64_t)4 * l1 * (lg + 1)) / l;
}

FftPlan make_fft_plan(int N);
// Columns per staged tile of the dense sketch: all n (whole rows, one chunk)
// when the rows of A (`aligned`: 16-byte aligned base and row stride) fit the
// whole-row kernel, else a fixed width by element size.
int sketch_chunk_cols(int dtype, int64_t m, int64_t n, int l1, bool aligned, int num_sms);
int launch_sketch_params(const SketchWs& ws, int64_t n, int l1, int l, uint64_t seed, cudaStream_t st);
int launch_twiddles(int N, double2* tw64, float2* tw32, cudaStream_t st);
// Exclusive scan of count int32 values into count + 1 offsets: over many
// CTAs with kScanMaxParts int64 of scratch at `tmp`, in one CTA when tmp is null.
int launch_scan_i32(int64_t count, const int32_t* cnt, int32_t* start, int64_t* tmp, cudaStream_t st);
// Dense sketch of the m rows of A; row i of the result goes to Y row rowmap[i]
// (row i when rowmap is null).
int launch_sketch_dense(const void* A, int64_t lda, int dtype, bool acc64, int64_t m, int64_t n, int l1, int l,
                        const SketchWs& ws, double* Y, unsigned int* status, int num_sms, cudaStream_t st,
                        const int32_t* rowmap = nullptr);
// Sketch of CSR A; heavy rows also written densely to D (n_heavy x n, row i of D = heavy[i]).
// `table` (l1 x l FP32 scratch) serves the direct evaluation of sparse rows
// (FP32 values, cr.direct_max >= 0).
int launch_sketch_csr(const int64_t* rowptr, const int32_t* colind, const void* val, int dtype, int64_t n,
                      const CsrRows& cr, int l1, int l, const SketchWs& ws, void* D, double* Y, float* table,
                      unsigned int* status, int num_sms, cudaStream_t st);

}  // namespace rlu
