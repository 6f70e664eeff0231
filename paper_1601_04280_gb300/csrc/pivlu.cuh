// Declarations of the persistent partial-pivoted LU (steps 3 and 6 of Algorithm 1).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace rlu {

struct PivLuWs {
  int32_t* pos;     // rows: final position of each row
  int32_t* pstep;   // rows: step at which the row was the pivot, -1 if never
  int64_t* perm;    // rows: perm[t] = row at position t
  void* cand;       // 2 x max_ctas candidate records
  void* candrow;    // 2 x max_ctas x max_cols values (double-sized)
  unsigned int* bar;
  int max_ctas;
  int max_cols;
};

size_t pivlu_cand_bytes(int max_ctas);

// LU of the rows x cols matrix X(i, c) = X[i*rs + c*cs], `steps` steps, in place.
template <typename T>
int launch_pivoted_lu(T* X, int64_t rows, int cols, int64_t rs, int64_t cs, int steps, PivLuWs& ws,
                      unsigned int* status, int num_sms, cudaStream_t st);

// One panel of a blocked LU: elimination steps j0 .. j0 + steps - 1 on the
// `cols` columns at X (column j0 of the whole matrix), over every row; rows
// pivoted by earlier panels (ws.pstep >= 0) are neither candidates nor
// updated.  Positions 0 .. npos - 1 are tracked (npos = the whole LU's
// steps); for j0 > 0 ws.pos, ws.pstep and ws.perm hold the state the previous
// panel left, and on return the state after this panel.
template <typename T>
int launch_pivoted_lu_panel(T* X, int64_t rows, int cols, int64_t rs, int64_t cs, int steps, int j0, int npos,
                            PivLuWs& ws, unsigned int* status, int num_sms, cudaStream_t st);

// Whether the panel kernel keeps a rows x cols panel in shared memory.
bool pivlu_panel_in_smem(int64_t rows, int cols, int npos, const PivLuWs& ws, int num_sms);

}  // namespace rlu
