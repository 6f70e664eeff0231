/*
 * rlu.h — C ABI of the GB300 sparse randomized LU library (librlu.so).
 *
 * The library computes a rank-k LU factorization P A Q ~= L U of an m x n
 * matrix A (dense row-major, or CSR) with the method of Aizenbud, Shabat and
 * Averbuch, "Randomized LU decomposition using sparse projections"
 * (arXiv 1601.04280): the problem statement of Sec. 1 (Eq. (1): find L m x k
 * lower, U k x n upper and permutations P, Q with ||LU - PAQ||_F = O(Delta_r))
 * and Algorithm 1 (Sec. 3), with the second projection of step 5 replaced by
 * the exact pseudo-inverse of Corollary 3.3 (col:A_LLA):
 *
 *   1. draw the sparse embedding matrix S (Sec. 2.2: hash h, signs s) and the
 *      real FFT-based projection (Sec. 2.1: signs d, Hartley transform, a
 *      subsample R of l of the l1 outputs) from a counter-based generator;
 *   2. Y = A S D H R / sqrt(l1)                     (m x l sketch, step 2);
 *   3. P Y = L_Y U_Y, partial (row) pivoting;      L_y = L_Y[:, :k] (step 3);
 *   4. B = L_y^+ P A                                (k x n, Corollary 3.3);
 *   5. B Q = L_b U_b, right (column) pivoting       (step 6);
 *   6. L = L_y L_b, U = U_b                         (step 7).
 *
 * Every step runs in the library's own CUDA kernels for sm_103a on the
 * caller's stream.  There is no CPU fallback: without a usable GPU every
 * compute entry point returns RLU_ECUDA.
 *
 * Conventions for every entry point
 *   - Return value: an rlu_status code (0 = success).  No entry point aborts,
 *     traps or prints.  RLU_WRANK is a warning: the factors are valid.
 *   - Pointers named "device" must be device memory of the current CUDA
 *     device (for example from torch or cudaMalloc); the caller owns them and
 *     keeps them alive until the call returns.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *   - Matrices are row-major with 0-based indices.  (PA)[i,:] = A[p[i],:] and
 *     (AQ)[:,j] = A[:,q[j]].
 */
#ifndef RLU_H_
#define RLU_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rlu_ctx* rlu_t; /* opaque; owns every device workspace of a factorization */

typedef enum {
  RLU_OK = 0,
  RLU_EINVAL = 1,     /* invalid argument (sizes, dtype, null pointer); nothing was launched */
  RLU_ENOMEM = 2,     /* workspace allocation failed */
  RLU_ECUDA = 3,      /* a CUDA call failed, or no usable GPU */
  RLU_ETIMEOUT = 4,   /* a bounded device wait gave up (co-residency lost); outputs undefined */
  RLU_ENONFINITE = 5, /* A holds NaN or Inf (or a sum of the sketch overflows FP32); outputs undefined */
  RLU_EBADCSR = 6,    /* CSR structure invalid (found on the device); outputs undefined */
  RLU_ETOOLARGE = 7,  /* sizes exceed the fixed scratch of rlu_sketch_dense_noalloc; nothing was launched */
  RLU_WRANK = 100     /* warning: an exactly zero pivot was met (rank deficiency); outputs valid */
} rlu_status;

/* Storage type of A's values. */
typedef enum { RLU_F64 = 0, RLU_F32 = 1, RLU_BF16 = 2 } rlu_dtype;

/* Arithmetic of the path.  In every mode the pivoted LU of the sketch, the
 * Cholesky factor of the Gram matrix L_y^T L_y and its inverse run in FP64.
 *   RLU_PREC_F64:         every step in FP64; outputs f64.
 *   RLU_PREC_F32:         sketch in FP32; the Gram matrix, L_y^+ and the LU of B
 *                         in float-float (about 48 significant bits); B = L_y^+ P A
 *                         on the tensor cores with FP32 accuracy (L_y^+ as three
 *                         BF16 planes, FP32 A as two BF16 pieces, FP32
 *                         accumulation over at most 512 rows of A and float-float
 *                         across them); L = L_y L_b in FP32; outputs f32.
 *   RLU_PREC_BF16:        as RLU_PREC_F32, but B from one BF16 pass (L_y^+
 *                         rounded to BF16, FP32 accumulate over 8192-row slices).
 *   RLU_PREC_BF16_REFINE: B from L_y^+ split into BF16 hi + lo parts (two
 *                         passes, FP32 accumulate over 2048-row slices): the
 *                         one-step refinement of B. */
typedef enum { RLU_PREC_F64 = 0, RLU_PREC_F32 = 1, RLU_PREC_BF16 = 2, RLU_PREC_BF16_REFINE = 3 } rlu_prec;

/* The FFT-based projection of step 2 (rlu_set_transform).
 *   RLU_XFORM_HARTLEY: random signs D, the real Hartley transform
 *                      cas(2 pi b f / l1) (Re - Im of the DFT), l kept
 *                      outputs R, scaled by 1/sqrt(l1): the real reading of
 *                      the SRFT of Sec. 2.1 (the default; fused kernels).
 *   RLU_XFORM_SRHT:    random signs D, the Walsh-Hadamard transform
 *                      (-1)^popcount(b & f) in Sylvester order, l kept outputs,
 *                      scaled by 1/sqrt(l1): the subsampled randomized
 *                      Hadamard transform the experiments of Sec. 4 used for
 *                      real data.  Needs l1 a power of two.
 *   RLU_XFORM_SRFT:    the complex SRFT of Sec. 2.1, D = diag(exp(i theta_b))
 *                      with theta_b = 2 pi u_b (u_b from the Philox stream 3
 *                      of the seed), the DFT, the first l/2 kept frequencies
 *                      R, each giving two columns (real and imaginary part)
 *                      scaled by sqrt(2/l1).  Needs l even. */
typedef enum { RLU_XFORM_HARTLEY = 0, RLU_XFORM_SRHT = 1, RLU_XFORM_SRFT = 2 } rlu_transform;

/* Create a handle for m x n inputs, output rank k, FJL width l and CountSketch
 * width l1 (Algorithm 1, step 1: k plays the role of the output rank, l of k1,
 * l1 of l1).  Requires 1 <= k <= l <= l1, l <= m, k <= min(m, n), m and n
 * below 2^31, l <= 1024 and l1 <= 16384.  l1 > n is allowed (empty buckets
 * stay zero).  `seed` fixes S, D and R: two calls with the same seed draw the
 * same projection.  Allocates the device workspace (see rlu_workspace_bytes)
 * on the current device; the default precision is RLU_PREC_F32.
 * Errors: RLU_EINVAL for bad sizes or a null `out`, RLU_ENOMEM, RLU_ECUDA. */
int rlu_create(int64_t m, int64_t n, int32_t k, int32_t l, int32_t l1, uint64_t seed, rlu_t* out);

/* As rlu_create, but the handle's workspace is the caller's device memory
 * `workspace` (256-byte aligned, at least rlu_workspace_bytes(...) bytes, kept
 * alive and unused by others until rlu_destroy): nothing is allocated on the
 * device, nothing waits for the device, and the one set-up kernel (the FFT
 * twiddles) is enqueued on `stream`.  For callers that manage device memory
 * themselves (a serving loop that admits requests by HBM footprint from its
 * own pool).  The handle's host words for the status read-back come from one
 * process-wide page-locked slab (allocated on the first call, 4096 handles at
 * a time).  The CSR entry point allocates its scratch on first use unless
 * rlu_set_csr_workspace gave it caller memory.  Errors: RLU_EINVAL (sizes,
 * null, misaligned or too small workspace), RLU_ENOMEM (host, or more than
 * 4096 such handles alive), RLU_ECUDA. */
int rlu_create_in(int64_t m, int64_t n, int32_t k, int32_t l, int32_t l1, uint64_t seed, void* workspace,
                  size_t workspace_bytes, void* stream, rlu_t* out);

/* Device bytes of caller-owned CSR scratch for a handle of sizes m, n, k that
 * will factor CSR inputs of at most max_nnz entries (the per-row lists, the
 * column-major copy of the light entries, and the dense copy of at most
 * min(m, max_nnz / ceil(n/4)) heavy rows with its tensor-core workspace).
 * The library's own extension; the paper has no counterpart.
 * Errors: RLU_EINVAL. */
int rlu_csr_workspace_bytes(int64_t m, int64_t n, int32_t k, int64_t max_nnz, size_t* bytes);

/* Give handle h caller-owned CSR scratch (device, 256-byte aligned, at least
 * rlu_csr_workspace_bytes(h's m, n, k, max_nnz) bytes).  The handle then never
 * allocates for rlu_factor_csr, and a later call with more than max_nnz
 * entries returns RLU_EINVAL.  The memory stays the caller's: rlu_destroy does
 * not free it, and it must outlive the handle's last factorization.  Must come
 * before the handle's first CSR factorization.
 * The library's own extension; the paper has no counterpart.
 * Errors: RLU_EINVAL (null, misaligned, too small, or CSR scratch already
 * allocated). */
int rlu_set_csr_workspace(rlu_t h, int64_t max_nnz, void* workspace, size_t workspace_bytes);

/* Select the arithmetic (rlu_prec).  Valid at any time between calls. */
int rlu_set_precision(rlu_t h, int prec);

/* Select the FFT-based projection of step 2 (rlu_transform); valid at any time
 * between calls.  RLU_XFORM_SRHT and RLU_XFORM_SRFT form Y1 = A S (bucket sums
 * in ascending column order) in a handle buffer of m x l1 values (8 bytes
 * each, allocated by the first dense factorization that uses it) and
 * Y = Y1 M with M the l1 x l matrix of the projection; dense A only
 * (rlu_factor_csr returns RLU_EINVAL while one of them is selected).
 * Errors: RLU_EINVAL (null handle, unknown transform, l1 not a power of two
 * for the SRHT, odd l for the SRFT). */
int rlu_set_transform(rlu_t h, int transform);

/* Use the paper's own second projection for B (Algorithm 1, steps 4-6)
 * instead of the exact pseudo-inverse of Corollary 3.3: Omega_2 = Pi_2 S_2
 * (k2 x m: a CountSketch of the m rows into l2 buckets with random signs, the
 * real Hartley transform and k2 of its l2 outputs, drawn from seed2 exactly
 * as the first projection is drawn from seed, over A's ORIGINAL row order),
 * Z = Omega_2 L_1 (k2 x k) and B = Z^+ Omega_2 P A, Z^+ by the Cholesky factor
 * of Z^T Z.  The dense product W A is replaced by a second pass over A (A is
 * transposed into a handle buffer of m n elements allocated on first use) and
 * small k2-wide products.  Requires k <= k2 <= l2, k2 <= 1024, l2 <= 4096 (Z is
 * sketched in FP64);
 * k2 = 0 switches back to the exact pseudo-inverse.  Dense A only
 * (rlu_factor_csr returns RLU_EINVAL while it is on).  Allocates its
 * parameters and k2-wide buffers now and waits for the device.
 * Errors: RLU_EINVAL, RLU_ENOMEM, RLU_ECUDA. */
int rlu_set_second_sketch(rlu_t h, int32_t k2, int32_t l2, uint64_t seed2);

/* Order the sketch's columns before the panel LU (on = 1) by QR with column
 * pivoting: at each step the column with the largest norm after removing the
 * span of the columns already chosen (Businger and Golub; computed as the
 * greedy pivoted Cholesky of Y^T Y with float-float arithmetic), so that L_y
 * spans the k most independent of the l sketch columns.  A rank-revealing
 * choice beyond Algorithm 1, whose panel LU takes the columns as they come;
 * it lets the oversampling l - k lower the error.  Off by default.  The first
 * call that turns it on allocates the Gram matrix, its split partials and a
 * copy of Y (m x l) and waits for the device.  rlu_debug_Y then returns the
 * reordered sketch.  Errors: RLU_EINVAL, RLU_ENOMEM, RLU_ECUDA. */
int rlu_set_column_pivoting(rlu_t h, int on);

/* Bound the CTAs of the two grid-synchronised kernels of handle h (the
 * pivoted LUs of steps 3 and 6, the Cholesky factor of G) to max_ctas; 0 (the
 * default) gives one CTA per SM.  Results do not depend on it (each kernel's
 * arithmetic per element and its pivot choice are independent of the grid);
 * fewer CTAs make a lone factorization's elimination steps longer but leave
 * SMs to factorizations running beside it on other streams (serving).
 * The library's own extension; the paper has no counterpart.
 * Errors: RLU_EINVAL (null handle, negative bound). */
int rlu_set_max_ctas(rlu_t h, int32_t max_ctas);

/* Device bytes that rlu_create allocates for these sizes and precision
 * (for admission by HBM footprint).  Errors: RLU_EINVAL. */
int rlu_workspace_bytes(int64_t m, int64_t n, int32_t k, int32_t l, int32_t l1, int prec, size_t* bytes);

/* Factor dense A.
 *   A:  device, m x n row-major values of type `dtype`, leading dimension
 *       lda >= n (elements).  Not modified.
 *   L:  device, m x k row-major, rows in P order, lower trapezoidal; f64 for
 *       RLU_PREC_F64, else f32.
 *   U:  device, k x n row-major, columns in Q order, unit upper trapezoidal
 *       with |U| <= 1; same type as L.
 *   p:  device, m int64: the row permutation.   q: device, n int64.
 * Enqueues the whole path on `stream`, waits for it, and returns the status.
 * The precision must match the dtype: RLU_PREC_F64 needs RLU_F64; the BF16
 * precisions need RLU_BF16; RLU_PREC_F32 takes RLU_F32 or RLU_BF16.
 * Errors: RLU_EINVAL (before any launch), RLU_ENONFINITE, RLU_ETIMEOUT,
 * RLU_ECUDA; warning RLU_WRANK. */
int rlu_factor_dense(rlu_t h, const void* A, int64_t lda, int dtype, void* L, void* U, int64_t* p, int64_t* q,
                     void* stream);

/* As rlu_factor_dense, but returns right after enqueueing: the status bits
 * (0 = success, else an rlu_status code) are written to `status_dev`
 * (device, one int32) on `stream`.  Launch-only: usable under CUDA graph
 * capture once the handle has run one factorization of the same dtype. */
int rlu_factor_dense_async(rlu_t h, const void* A, int64_t lda, int dtype, void* L, void* U, int64_t* p,
                           int64_t* q, int32_t* status_dev, void* stream);

/* Copy `rows` rows of `width_bytes` bytes from src (row pitch src_pitch
 * bytes) to dst (row pitch dst_pitch bytes), asynchronously on `stream`;
 * either side may be host (page-locked for an asynchronous copy) or device
 * memory.  Used to bring a request's matrix, or a block of a larger one, into
 * a caller-owned workspace before rlu_factor_dense.
 * The library's own extension; the paper has no counterpart.
 * Errors: RLU_EINVAL (null pointer, pitch below the width, negative size),
 * RLU_ECUDA. */
int rlu_copy_block_async(void* dst, int64_t dst_pitch, const void* src, int64_t src_pitch, int64_t width_bytes,
                         int64_t rows, void* stream);

/* Captured launch graphs (CUDA graphs) of one dense factorization.
 * rlu_graph_capture_dense records, without running it, the whole path of
 * rlu_factor_dense_async for these exact pointers on `stream` (not the legacy
 * default stream) and instantiates it.  The handle must have run one
 * factorization of the same dtype before (setup that allocates or reads back
 * happens then), and timing and debug copies must be off.  Each
 * rlu_graph_launch replays it on `stream`: the same A, L, U, p, q and status
 * addresses, new contents.  The handle and every captured buffer must outlive
 * the graph; one graph runs at a time per handle.
 * The library's own extension; the paper has no counterpart.
 * Errors: RLU_EINVAL, RLU_ENOMEM, RLU_ECUDA. */
typedef struct rlu_graph* rlu_graph_t;
int rlu_graph_capture_dense(rlu_t h, const void* A, int64_t lda, int dtype, void* L, void* U, int64_t* p,
                            int64_t* q, int32_t* status_dev, void* stream, rlu_graph_t* out);
int rlu_graph_launch(rlu_graph_t g, void* stream);
int rlu_graph_destroy(rlu_graph_t g);

/* Factor CSR A (m x n, nnz entries, nnz < 2^31).
 *   rowptr: device, m+1 int64, rowptr[0] = 0, non-decreasing, rowptr[m] = nnz.
 *   colind: device, nnz int32 in [0, n).  Order within a row is free;
 *           repeated coordinates are summed.
 *   val:    device, nnz values: RLU_F32 with RLU_PREC_F32, RLU_F64 with RLU_PREC_F64.
 * Outputs as rlu_factor_dense.  Rows with at least n/4 entries are copied to a
 * dense block for the tensor-core product; the handle allocates that block and
 * the per-entry scratch on first use (and grows them), and reads the number of
 * such rows back to the host once per call.  The structure is validated on the
 * device (RLU_EBADCSR).  Errors as rlu_factor_dense. */
int rlu_factor_csr(rlu_t h, const int64_t* rowptr, const int32_t* colind, const void* val, int64_t nnz, int dtype,
                   void* L, void* U, int64_t* p, int64_t* q, void* stream);

/* End-to-end variant of rlu_factor_dense on HOST buffers: copies A (host,
 * m x n row-major, lda = n) to a device staging buffer owned by the handle
 * (allocated on first use), factors it, and copies L, U, p, q back to the
 * host buffers.  Host buffers should be page-locked for full copy speed. */
int rlu_factor_dense_host(rlu_t h, const void* A_host, int dtype, void* L_host, void* U_host, int64_t* p_host,
                          int64_t* q_host, void* stream);

/* Release the handle and its workspace.  Null is accepted. */
int rlu_destroy(rlu_t h);

/* Static message for a status code. */
const char* rlu_strerror(int code);

/* ---- test hooks: copies of intermediates of the last factorization ---- */

/* Sketch parameters (Sec. 2.2 and 2.1): hash h (n int32), signs s (n int8),
 * signs d (l1 int8), subsample R (l int32).  Host buffers; synchronizes. */
int rlu_debug_sketch_params(rlu_t h, int32_t* hash, int8_t* s, int8_t* d, int32_t* R);

/* The sketch Y (m x l row-major f64) as written by the sketch kernel, before
 * the panel LU overwrote it (kept only when debug capture is enabled with
 * rlu_debug_enable(h, 1) before the factorization).  Host buffer. */
int rlu_debug_Y(rlu_t h, double* Y_host);

/* B = L_y^+ P A (k x n row-major, f64 on the host) as formed before its LU
 * (also needs rlu_debug_enable). */
int rlu_debug_B(rlu_t h, double* B_host);

/* Keep copies of Y and B during factorizations (costs device memory and time). */
int rlu_debug_enable(rlu_t h, int on);

/* Record CUDA events on the factorization stream between the stages of the
 * path (on = 1) so that rlu_debug_stage_ms can report their device times. */
int rlu_debug_timing(rlu_t h, int on);

/* Device milliseconds of the stages of the last factorization, in order:
 * 0 sketch parameters and bucket lists, 1 sketch (CountSketch + FFT),
 * 2 panel LU of Y, 3 Lk and Gram matrix, 4 Cholesky and R^{-1},
 * 5 G^{-1} and W = L_y^+ P, 6 B = W A, 7 LU of B, 8 assembly of L, U, p, q.
 * Writes min(max_stages, 9) values and their number to *count; waits for the
 * last factorization to finish.  Errors: RLU_EINVAL if timing was off. */
int rlu_debug_stage_ms(rlu_t h, float* ms, int max_stages, int* count);

/* Number of CUDA kernels this library has launched in this process so far. */
int rlu_debug_launch_count(int64_t* out);

/* Test hook, needs no GPU: the status code that the library reports for a
 * set of device flag bits (bit 0 a timed-out wait, bit 1 a non-finite value,
 * bit 2 an exactly zero pivot, bit 3 a malformed CSR structure), the same
 * mapping that every entry point and the device-side status writers use.
 * Errors: RLU_EINVAL (null status). */
int rlu_debug_status_of_flags(uint32_t flags, int* status);

/* Test hook: run one of the library's bounded device waits on a condition
 * that never comes true and report the status it leaves.  which = 0: the grid
 * barrier of the cooperative kernels (two CTAs wait for an arrival no CTA
 * makes); which = 1: the mbarrier wait of the tensor-core pipeline (a barrier
 * nothing arrives at).  Each wait gives up after about a second, sets the
 * timeout flag and returns, so *status receives RLU_ETIMEOUT and the context
 * stays usable.  Synchronous; allocates 8 bytes of device memory.
 * Errors: RLU_EINVAL, RLU_ENOMEM, RLU_ECUDA. */
int rlu_debug_wait_timeout(int which, int* status);

/* Measurement hook: fused multiply-add throughput of the current GPU in
 * TFLOP/s (2 flop per FMA), which = 0 for FP64, 1 for FP32, from a kernel of
 * eight independent FMA chains per thread, 2048 threads per SM, best of three
 * timed launches of about 20 ms each.  Synchronous.
 * Errors: RLU_EINVAL, RLU_ENOMEM, RLU_ECUDA. */
int rlu_debug_alu_peak(int which, double* tflops);

/* Test and measurement hook: how the two pivoted LUs run — step 3
 * (P Y = L_Y U_Y, m x l) and step 6 (partial pivoting of B^T, n x k) of
 * Algorithm 1.  block = 0 (default): each is blocked in panels of 64, 32 or
 * 16 columns when the unblocked kernel cannot keep its matrix in shared
 * memory and it has at least 32 columns (the widest panel whose rows fit the
 * panel kernel's shared memory with one CTA per SM, at least two panels),
 * else one unblocked kernel; -1: always the unblocked kernel; 16, 32, 64:
 * that panel width for both.  The choice depends only on the sizes and the
 * SM count.  The blocked form makes the same pivot choices as the unblocked
 * one wherever rounding does not decide them: its trailing updates are exact
 * digit products on the tensor cores (56 bits), subtracted in the LU's own
 * arithmetic (FP64 for Y and in FP64 mode, float-float for B otherwise).
 * Errors: RLU_EINVAL (null handle, other values, a width above
 * rlu_debug_lu_block's maximum or >= k). */
int rlu_debug_set_lu_block(rlu_t h, int32_t block);

/* Test hook: the result of step 3 of the last factorization — Y (m x l,
 * row-major FP64, rows in their ORIGINAL order: the row at position t of the
 * pivoted order holds its multipliers in columns < t and row t of U_Y from
 * column t on; a row never pivoted holds multipliers in all l columns) and
 * the row permutation (perm[t] = original row at position t, m entries), to
 * host buffers.  Synchronous.  Errors: RLU_EINVAL, RLU_ECUDA. */
int rlu_debug_lu_Y(rlu_t h, double* Y_host, int64_t* perm_host);

/* Measurement hook: the launches of the pivoted-LU kernel in the last timed
 * factorization (rlu_debug_timing on) of LU `which` (0: step 3, the sketch
 * Y; 1: step 6, B^T): *width = the panel width (0 when unblocked: one launch
 * over all l or k columns), *launches = the kernel's launches, *ms = their
 * summed device time from CUDA events recorded around each launch on the
 * handle's stream.  The blocked form's other kernels (the U12 solve and the
 * tensor-core trailing updates) are not included.  Synchronous.
 * Errors: RLU_EINVAL (null argument, which not 0 or 1, timing off or no
 * timed factorization yet), RLU_ECUDA. */
int rlu_debug_lu_panels(rlu_t h, int which, int32_t* width, int32_t* launches, double* ms);

/* Test hook: how the tensor-core product B = W A (step 6 of Algorithm 1)
 * reads a BF16 A.  on = 1 (the default): by TMA, as it lies in memory (the
 * MMA's A operand MN-major), whenever A's base address and row stride are
 * multiples of 16 bytes; on = 0: by the converter warps (global loads into
 * the K-major swizzled layout), the form used for FP32 A and unaligned BF16
 * A.  Both forms issue the same products in the same order.
 * Errors: RLU_EINVAL (null handle, on not 0 or 1). */
int rlu_debug_set_tma_a(rlu_t h, int on);

/* The block setting of rlu_debug_set_lu_block (return value) and, in
 * *block_max (may be null), the widest panel this handle's workspace holds
 * (0: the blocked form is unavailable).  RLU_EINVAL for a null handle. */
int rlu_debug_lu_block(rlu_t h, int32_t* block_max);

/* Test hook: the device FP64 reciprocal used on the Cholesky's dependent chain
 * (Newton's iteration seeded by the FP32 reciprocal approximation), applied to
 * n host values x (x > 0), results to host out.  Synchronous.
 * Errors: RLU_EINVAL, RLU_ENOMEM, RLU_ECUDA. */
int rlu_debug_recip(const double* x, double* out, int64_t n);

/* ---- sketch without allocation ----
 * The paper has no counterpart to this entry point: it exists for callers
 * that cannot allocate device memory on their call path — a serving loop
 * that must not call cudaMalloc (it synchronizes the whole device and stalls
 * every other stream), a process whose device memory already belongs to
 * another framework's pool, or an embedded caller with a fixed memory map.
 *
 * rlu_sketch_dense_noalloc computes the m x l sketch
 *   Y = A S D H R / sqrt(l1)   (row-major f64, device, written by the call),
 * with S (hash and signs), D (signs) and R (the kept Hartley outputs) drawn
 * from `seed` exactly as rlu_create(m, n, k, l, l1, seed) draws them, so Y
 * equals the sketch that a handle computes for the same inputs.
 * A: device, m x n row-major of `dtype` (RLU_F64 sums in FP64, RLU_F32 and
 * RLU_BF16 in FP32), leading dimension lda >= n.
 * It allocates nothing: its scratch (hash and sign arrays, per-chunk bucket
 * lists, twiddles, a status word) is one fixed file-scope device array of
 * RLU_NOALLOC_SCRATCH_BYTES bytes, present on every device that loads the
 * library until the process exits.  Sizes are limited accordingly:
 * n <= RLU_NOALLOC_MAX_N, l1 <= RLU_NOALLOC_MAX_L1, l <= RLU_NOALLOC_MAX_L;
 * larger sizes return RLU_ETOOLARGE before anything is launched.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  All calls on one device share the array and it keeps the last
 * call's contents (each call re-initializes what it needs); calls on the same
 * device whose GPU work overlaps race on it and must be serialized.
 * Asynchronous on `stream`: when the work completes, `status_dev` (device,
 * one int32) receives RLU_OK, RLU_ETIMEOUT (a bounded wait of the sketch's
 * copy pipeline gave up: Y is incomplete) or RLU_ENONFINITE (A holds NaN or
 * Inf, or a bucket sum overflowed).
 * Errors at call time: RLU_EINVAL, RLU_ETOOLARGE, RLU_ECUDA. */
#define RLU_NOALLOC_MAX_N 65536
#define RLU_NOALLOC_MAX_L1 4096
#define RLU_NOALLOC_MAX_L 1024
#define RLU_NOALLOC_SCRATCH_BYTES 2773760
int rlu_sketch_dense_noalloc(const void* A, int64_t lda, int dtype, int64_t m, int64_t n, int32_t l, int32_t l1,
                             uint64_t seed, double* Y, int32_t* status_dev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RLU_H_ */
