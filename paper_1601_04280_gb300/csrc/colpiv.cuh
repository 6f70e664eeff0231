// Declarations of the rank-revealing column order of the sketch.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace rlu {

// Y (m x l, row-major FP64, device) := Y[:, order] with order the greedy
// column order of QR with column pivoting; `buf` of colpiv_buffer_bytes bytes.
int launch_column_pivoting(double* Y, int64_t m, int l, void* buf, int max_splits, int num_sms, cudaStream_t st);
size_t colpiv_buffer_bytes(int64_t m, int l, int max_splits);

}  // namespace rlu
