// The other FFT-based projections of step 2 (Algorithm 1) for dense A: the
// subsampled randomized Walsh-Hadamard transform (Sec. 4 used it for real
// data; l1 a power of two) and the complex SRFT of Sec. 2.1 (D of
// unit-modulus entries, the DFT) in real form.  The default real Hartley
// projection keeps its fused kernels (sketch.cu); these two run as
//   Y1 = A S            (bucket sums in ascending column order, k_countsketch_y1)
//   Y  = Y1 M           (M = the l1 x l matrix of the projection, k_xform_table,
//                        a SIMT GEMM)
// with Y1 in global memory: l1 / l times the Hartley path's writes, but the
// same arithmetic per entry for every transform.
#include "common.cuh"
#include "gemm_simt.cuh"
#include "xform.cuh"

namespace rlu {

// One thread per bucket b of kY1Rows rows: Y1[i][b] = sum over the columns j
// of bucket b, ascending, of s(j) A[i][j] (whole-row lists: offset = j).
constexpr int kY1Rows = 8;
template <typename TA, typename TACC>
__global__ void __launch_bounds__(128) k_countsketch_y1(const TA* __restrict__ A, int64_t lda, int64_t m, int l1,
                                                        const int32_t* __restrict__ bstart,
                                                        const uint32_t* __restrict__ blist, TACC* __restrict__ Y1,
                                                        unsigned int* status) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t row0 = (int64_t)blockIdx.y * kY1Rows;
  if (b >= l1) return;
  TACC acc[kY1Rows];
#pragma unroll
  for (int r = 0; r < kY1Rows; ++r) acc[r] = TACC(0);
  bool bad = false;
  for (int e = bstart[b]; e < bstart[b + 1]; ++e) {
    const uint32_t ent = blist[e];
    const int64_t j = ent & 0x7fffffffu;
    const bool neg = (ent >> 31) != 0;
#pragma unroll
    for (int r = 0; r < kY1Rows; ++r) {
      if (row0 + r < m) {
        const TA a = A[(row0 + r) * lda + j];
        bad |= !finite_(a);
        const TACC v = sizeof(TACC) == 8 ? (TACC)to_double(a) : (TACC)to_float(a);
        acc[r] += neg ? -v : v;
      }
    }
  }
#pragma unroll
  for (int r = 0; r < kY1Rows; ++r)
    if (row0 + r < m) Y1[(row0 + r) * l1 + b] = acc[r];
  if (bad) set_flag(status, FLAG_NONFINITE);
}

// M (l1 x l) of the selected projection, computed in FP64 and stored as TACC:
//   SRHT: M[b][c] = d(b) (-1)^popcount(b & R_c) / sqrt(l1);
//   SRFT: with phi = theta_b - 2 pi ((b R_c') mod l1) / l1 for c' = c / 2,
//         M[b][c] = sqrt(2 / l1) cos phi (c even), sqrt(2 / l1) sin phi (c odd),
//         theta_b = 2 pi u, u = (word 0 of Philox block (b, 3)) >> 11 over 2^53.
template <typename TACC>
__global__ void k_xform_table(int transform, int l1, int l, uint64_t seed, const float* __restrict__ dsign,
                              const int32_t* __restrict__ Rsel, TACC* __restrict__ M) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)l1 * l) return;
  const int b = (int)(e / l), c = (int)(e - (int64_t)b * l);
  double v;
  if (transform == RLU_XFORM_SRHT) {
    v = ((__popc((unsigned)(b & Rsel[c])) & 1) ? -1.0 : 1.0) * (double)dsign[b] * rsqrt((double)l1);
  } else {
    const Philox4 w = philox4x64_10((uint64_t)b, 3, 0, 0, seed, kKeyTag);
    const double u = (double)(w.w[0] >> 11) * 0x1p-53;
    const int64_t t = ((int64_t)b * Rsel[c >> 1]) % l1;
    // phi / pi = 2 u - 2 t / l1, reduced to (-2, 2]
    const double phi_over_pi = 2.0 * u - 2.0 * (double)t / (double)l1;
    double sn, cs;
    sincospi(phi_over_pi, &sn, &cs);
    v = ((c & 1) ? sn : cs) * sqrt(2.0 / (double)l1);
  }
  M[e] = (TACC)v;
}

int launch_sketch_xform(int transform, const void* A, int64_t lda, int dtype, bool acc64, int64_t m, int64_t n,
                        int l1, int l, uint64_t seed, const SketchWs& ws, void* y1_buf, double* Y,
                        unsigned int* status, cudaStream_t st) {
  if (transform != RLU_XFORM_SRHT && transform != RLU_XFORM_SRFT) return RLU_EINVAL;
  if (ws.chunk != n) return RLU_EINVAL;  // whole-row bucket lists
  const dim3 g1((unsigned)cdiv(l1, 128), (unsigned)cdiv(m, kY1Rows));
  const unsigned gt = (unsigned)cdiv((int64_t)l1 * l, 256);
  if (acc64) {
    if (dtype != RLU_F64) return RLU_EINVAL;
    double* Y1 = (double*)y1_buf;
    double* M = Y1 + (size_t)m * l1;
    k_countsketch_y1<double, double><<<g1, 128, 0, st>>>((const double*)A, lda, m, l1, ws.bstart, ws.blist, Y1, status);
    k_xform_table<double><<<gt, 256, 0, st>>>(transform, l1, l, seed, ws.dsign, ws.R, M);
    RLU_CUDA_TRY(cudaGetLastError());
    note_launch(2);
    return gemm_simt<double, double, double, double>(st, m, l, l1, Y1, l1, 1, M, l, 1, Y, l, 1);
  }
  float* Y1 = (float*)y1_buf;
  float* M = Y1 + (size_t)m * l1;
  if (dtype == RLU_F32)
    k_countsketch_y1<float, float><<<g1, 128, 0, st>>>((const float*)A, lda, m, l1, ws.bstart, ws.blist, Y1, status);
  else if (dtype == RLU_BF16)
    k_countsketch_y1<__nv_bfloat16, float><<<g1, 128, 0, st>>>((const __nv_bfloat16*)A, lda, m, l1, ws.bstart,
                                                               ws.blist, Y1, status);
  else
    return RLU_EINVAL;
  k_xform_table<float><<<gt, 256, 0, st>>>(transform, l1, l, seed, ws.dsign, ws.R, M);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch(2);
  return gemm_simt<float, float, double, float>(st, m, l, l1, Y1, l1, 1, M, l, 1, Y, l, 1);
}

size_t xform_buffer_bytes(int64_t m, int l1, int l, bool acc64) {
  return (acc64 ? 8 : 4) * ((size_t)m * l1 + (size_t)l1 * l);
}

}  // namespace rlu
