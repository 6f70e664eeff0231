// Declarations of the blocked partial-pivoted LU of the sketch (step 3 of
// Algorithm 1) with its trailing updates on the tensor cores.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "pivlu.cuh"

namespace rlu {

// Panel widths the blocked LU uses (the contraction depth of a trailing update).
constexpr int kBluWidths[3] = {64, 32, 16};

// Workspace: packed digit planes of the multipliers of a panel (m rows) and
// of the transposed pivot rows U12^T (up to l rows), their power-of-two
// scales, and the TMA descriptors of both for every panel width.
struct BluWs {
  __nv_bfloat16* adig;  // m x (8 b) per row, packed by 16/32-deep chunk, then digit
  __nv_bfloat16* bdig;  // l x (8 b)
  int32_t* aexp;        // m: scale exponent of a row's multipliers, kBluSkip for pivoted rows
  int32_t* bexp;        // l: scale exponent of a column of U12
  int64_t m;
  int l;
  int bmax;             // widest panel the planes hold
  int num_sms;
  alignas(64) unsigned char mapA[3][128];
  alignas(64) unsigned char mapB[3][128];
  bool ready;
};

size_t blu_workspace_bytes(int64_t m, int l, int num_sms);
// Carve the workspace; ready = false (the unblocked LU runs) when tensor maps
// are unavailable.
int blu_setup(BluWs& w, void* base, int64_t m, int l, int num_sms);

// P Y = L_Y U_Y, l steps, on the m x l row-major FP64 Y in place, with the
// results and the state in `pw` exactly as launch_pivoted_lu<double> leaves
// them.  block: 0 picks the panel width (or the unblocked kernel), -1 forces
// the unblocked kernel, 16/32/64 force that width.
int launch_lu_y(double* Y, int64_t m, int l, PivLuWs& pw, const BluWs& bw, int block, unsigned int* status,
                int coop_sms, cudaStream_t st);

}  // namespace rlu
