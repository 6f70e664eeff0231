// Declarations of the blocked partial-pivoted LUs (steps 3 and 6 of
// Algorithm 1) with their trailing updates on the tensor cores.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "pivlu.cuh"

namespace rlu {

// Panel widths the blocked LU uses (the contraction depth of a trailing update).
constexpr int kBluWidths[3] = {64, 32, 16};

// Workspace: packed digit planes of the multipliers of a panel (up to
// max(m, n) rows) and of the transposed pivot rows U12^T (up to l rows),
// their power-of-two scales, and the TMA descriptors of both for every panel
// width.  Shared by the LU of the sketch Y and the LU of B^T.
struct BluWs {
  __nv_bfloat16* adig;  // rows_a x (8 b) per row, packed by 16/32-deep chunk, then digit
  __nv_bfloat16* bdig;  // rows_b x (8 b)
  int32_t* aexp;        // rows_a: scale exponent of a row's multipliers, a skip mark for pivoted rows
  int32_t* bexp;        // rows_b: scale exponent of a column of U12
  int64_t rows_a;
  int rows_b;
  int bmax;             // widest panel the planes hold
  int num_sms;
  alignas(64) unsigned char mapA[3][128];
  alignas(64) unsigned char mapB[3][128];
  bool ready;
};

// Device times of the panel launches of one LU (measurement hook): events
// around each launch of the pivoted-LU kernel (one launch when unblocked).
constexpr int kMaxPanels = 64;  // l <= 1024 in panels of 16 or more
struct PanelTimer {
  cudaEvent_t ev[2 * kMaxPanels] = {};
  int n = 0;      // launches recorded
  int width = 0;  // panel width, 0 when unblocked
};

size_t blu_workspace_bytes(int64_t m, int64_t n, int k, int l, int num_sms);
// Carve the workspace; ready = false (the unblocked LUs run) when tensor maps
// are unavailable or no panel fits.
int blu_setup(BluWs& w, void* base, int64_t m, int64_t n, int k, int l, int num_sms);

// P Y = L_Y U_Y, l steps, on the m x l row-major FP64 Y in place (step 3 of
// Algorithm 1), with the results and the state in `pw` exactly as
// launch_pivoted_lu<double> leaves them.  block: 0 picks the panel width (or
// the unblocked kernel), -1 forces the unblocked kernel, 16/32/64 force that
// width.
int launch_lu_y(double* Y, int64_t m, int l, PivLuWs& pw, const BluWs& bw, int block, unsigned int* status,
                int coop_sms, cudaStream_t st, PanelTimer* timer = nullptr);

// B Q = L_b U_b by partial pivoting of B^T (n x k, element (i, c) at
// B[c n + i]), k steps (step 6 of Algorithm 1), in FP64 or float-float; the
// same choices of form and width as launch_lu_y.
template <typename T>
int launch_lu_b(T* B, int64_t n, int k, PivLuWs& pw, const BluWs& bw, int block, unsigned int* status,
                int coop_sms, cudaStream_t st, PanelTimer* timer = nullptr);

}  // namespace rlu
