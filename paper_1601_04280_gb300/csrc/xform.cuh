// Declarations of the SRHT and SRFT projections of step 2 (dense A).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"
#include "sketch.cuh"

namespace rlu {

// Y (m x l, row-major f64) = (A S) M for the projection `transform`
// (RLU_XFORM_SRHT or RLU_XFORM_SRFT): needs the whole-row bucket lists
// (ws.chunk == n) and y1_buf of xform_buffer_bytes(m, l1, l, acc64) bytes.
int launch_sketch_xform(int transform, const void* A, int64_t lda, int dtype, bool acc64, int64_t m, int64_t n,
                        int l1, int l, uint64_t seed, const SketchWs& ws, void* y1_buf, double* Y,
                        unsigned int* status, cudaStream_t st);
size_t xform_buffer_bytes(int64_t m, int l1, int l, bool acc64);

}  // namespace rlu
