// C ABI of the sparse randomized LU library: handle, workspace and the
// orchestration of Algorithm 1 (with the exact L_y^+ of Corollary 3.3) on
// one CUDA stream.  See include/rlu.h for the contract of each entry point.
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "bgemm.cuh"
#include "blu.cuh"
#include "colpiv.cuh"
#include "common.cuh"
#include "csr.cuh"
#include "pinv.cuh"
#include "pivlu.cuh"
#include "sketch.cuh"
#include "xform.cuh"

using namespace rlu;

#include <mutex>

namespace rlu {
static std::atomic<long long> g_launches{0};
static thread_local long long t_launches = 0;  // this thread's share (graph capture counts its own)
void note_launch(int count) {
  g_launches.fetch_add(count, std::memory_order_relaxed);
  t_launches += count;
}

// Page-locked host words (status and CSR counts, 8 per handle) for handles
// built on caller memory: one slab allocated on first use (never freed),
// handed out from a free list.
static std::mutex g_slab_mu;
static unsigned int* g_slab = nullptr;
static std::vector<unsigned int*> g_slab_free;
constexpr int kSlabWords = 1 << 15;  // 8 words per handle, 4096 handles

unsigned int* status_slab_take() {
  std::lock_guard<std::mutex> lock(g_slab_mu);
  if (!g_slab) {
    void* p = nullptr;
    if (cudaHostAlloc(&p, sizeof(unsigned int) * kSlabWords, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    g_slab = (unsigned int*)p;
    g_slab_free.reserve(kSlabWords);
    for (int i = kSlabWords / 8 - 1; i >= 0; --i) g_slab_free.push_back(g_slab + 8 * i);
  }
  if (g_slab_free.empty()) return nullptr;
  unsigned int* w = g_slab_free.back();
  g_slab_free.pop_back();
  for (int i = 0; i < 8; ++i) w[i] = 0;
  return w;
}

void status_slab_give(unsigned int* w) {
  std::lock_guard<std::mutex> lock(g_slab_mu);
  g_slab_free.push_back(w);
}

// Cooperative launch of a kernel with grid barriers.  Such kernels on different
// streams are not ordered against each other: the driver starts a cooperative
// grid only once every one of its CTAs can be resident, so two of them never
// hold part of the GPU each while waiting for the rest (the serving loop runs
// them side by side; the bounded grid barriers would report the opposite as
// RLU_ETIMEOUT).
cudaError_t launch_cooperative(const void* func, dim3 grid, dim3 block, void** args, size_t smem, cudaStream_t st) {
  return cudaLaunchCooperativeKernel(func, grid, block, args, smem, st);
}

int allow_dynamic_smem(const void* kern, size_t smem) {
  int dev = 0, optin = 0;
  RLU_CUDA_TRY(cudaGetDevice(&dev));
  RLU_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa;
  RLU_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
  const int64_t lim = (int64_t)optin - (int64_t)fa.sharedSizeBytes;
  if ((int64_t)smem > lim) return RLU_EINVAL;
  RLU_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim));
  return RLU_OK;
}

}  // namespace rlu

struct rlu_graph {
  cudaGraphExec_t exec = nullptr;
  long long kernels = 0;  // kernels one launch of the graph runs
};

// Stages whose device time the timing hook reports, in order.
static const int kNumStages = 9;

struct rlu_ctx {
  int64_t m = 0, n = 0;
  int k = 0, l = 0, l1 = 0;
  uint64_t seed = 0;
  int prec = RLU_PREC_F32;
  int device = 0;
  int num_sms = 0;
  int max_ctas = 0;  // bound on the CTAs of the grid-synchronised kernels (0: one per SM)
  SketchWs sk{};
  double* Y = nullptr;
  PivLuWs pw{};
  int64_t* perm_y = nullptr;
  int64_t* perm_b = nullptr;
  void* Lk = nullptr;
  double* gram_part = nullptr;
  int max_gram_splits = 0;
  double* G = nullptr;
  double* Rinv = nullptr;
  double* Ginv = nullptr;
  void* W = nullptr;
  void* B = nullptr;
  void* LyP = nullptr;
  void* Lb = nullptr;
  double* bpart = nullptr;  // split-K partials of the FP64 SIMT B = W A
  TcWs tcw{};
  LtcWs ltc{};  // digit planes of the tensor-core L = L_y L_b
  BluWs blu{};  // digit planes of the blocked LU's trailing updates
  int lu_block = 0;  // panel width of the LUs of Y and B^T: 0 automatic, -1 unblocked
  PanelTimer ptimer[2];  // panel launch times of the two LUs (timing on)
  float* fjl_table = nullptr;  // l1 x l table of the CSR sketch's direct evaluation
  int colpiv = 0;                 // rank-revealing column order of the sketch
  void* cp_buf = nullptr;
  int cp_splits = 0;
  int xform = RLU_XFORM_HARTLEY;  // projection of step 2
  void* xf_buf = nullptr;         // Y1 and the projection matrix (SRHT, SRFT), allocated on first use
  unsigned int* status_dev = nullptr;
  unsigned int* bar2 = nullptr;
  // 8 page-locked host words: status (0) and the CSR counts (4..7); own
  // allocation when status_pinned, else a piece of the shared slab
  unsigned int* status_host = nullptr;
  bool status_pinned = false;
  bool status_slab = false;
  int debug = 0;
  double* Ydbg = nullptr;
  void* Bdbg = nullptr;
  int last_prec = -1;
  // host-buffer entry point staging
  void* A_stage = nullptr;
  size_t A_stage_bytes = 0;
  void* L_stage = nullptr;
  void* U_stage = nullptr;
  int64_t* p_stage = nullptr;
  int64_t* q_stage = nullptr;
  // CSR path workspace, sized on first use (rows) and grown with nnz / heavy rows
  CsrWs csr{};
  bool csr_rows_ready = false;
  int64_t csr_cap_nnz = -1, csr_cap_heavy = -1;
  void* csr_nnz_buf = nullptr;
  void* csr_heavy_buf = nullptr;
  void* csr_rows_buf = nullptr;
  bool csr_external = false;  // CSR scratch owned by the caller (rlu_set_csr_workspace)
  // the paper's second projection (rlu_set_second_sketch): off when k2 == 0
  int k2 = 0, l2 = 0;
  uint64_t seed2 = 0;
  SketchWs sk2{};
  void* sk2_buf = nullptr;  // Omega_2 parameters and lists, Y2T, LkT, ZT, W2
  double *Y2T = nullptr, *LkT = nullptr, *ZT = nullptr;
  void* W2 = nullptr;
  void* at_buf = nullptr;   // A transposed, grown on use
  size_t at_bytes = 0;
  // per-stage device timing (test hook)
  int timing = 0;
  cudaEvent_t ev[kNumStages + 1] = {};
  int ev_recorded = 0;
  std::vector<void*> allocs;
};

namespace {

constexpr int kMaxL = 1024;
constexpr int kMaxL1 = 16384;
constexpr int kMaxPivCtas = 1024;

struct Sizes {
  size_t total = 0;
  std::vector<size_t> parts;
  void add(size_t b) {
    b = (b + 255) & ~(size_t)255;
    parts.push_back(b);
    total += b;
  }
};

int max_gram_splits_for(int k, int num_sms) {
  const int64_t tk = cdiv(k, 64);
  int64_t tiles = tk * (tk + 1) / 2;  // the symmetric Gram product computes the upper tiles only
  int64_t s = cdiv(2 * (int64_t)num_sms, tiles);
  return (int)(s < 1 ? 1 : s);
}

// The order of `add` calls is the allocation order in rlu_create.
Sizes plan_sizes(int64_t m, int64_t n, int k, int l, int l1, int num_sms) {
  Sizes s;
  const int64_t nch = cdiv(n, 1024);  // smallest chunk of the dense sketch
  s.add(sizeof(uint32_t) * n);                       // hs
  s.add(sizeof(float) * l1);                         // dsign
  s.add(sizeof(uint64_t) * l1);                      // keys
  s.add(sizeof(int32_t) * l);                        // R
  s.add(sizeof(int32_t) * (nch * l1 + 1));           // bcnt
  s.add(sizeof(int32_t) * (nch * l1 + 1));           // bstart
  s.add(sizeof(uint32_t) * n);                       // blist
  s.add(sizeof(double2) * l1);                       // tw64
  s.add(sizeof(float2) * l1);                        // tw32
  s.add(sizeof(double) * m * l);                     // Y
  const int64_t mx = m > n ? m : n;
  s.add(sizeof(int32_t) * mx);                       // pos
  s.add(sizeof(int32_t) * mx);                       // pstep
  s.add(sizeof(int64_t) * m);                        // perm_y
  s.add(sizeof(int64_t) * n);                        // perm_b
  s.add(pivlu_cand_bytes(kMaxPivCtas));              // cand
  s.add(sizeof(double) * 2 * kMaxPivCtas * (l > k ? l : k));  // candrow
  s.add(sizeof(unsigned int) * 2);                   // bar (pivlu)
  s.add(sizeof(double) * m * k);                     // Lk
  s.add(sizeof(double) * max_gram_splits_for(k, num_sms) * k * k);  // gram partials
  s.add(sizeof(double) * k * k);                     // G
  s.add(sizeof(double) * k * k);                     // Rinv
  s.add(sizeof(double) * k * k);                     // Ginv
  s.add(sizeof(double) * k * m);                     // W
  s.add(sizeof(double) * k * n);                     // B
  s.add(sizeof(double) * m * k);                     // LyP
  s.add(sizeof(double) * k * k);                     // Lb
  s.add(sizeof(unsigned int) * 4);                   // status, bar2
  s.add(tc_workspace_bytes(m, n, k, num_sms));       // tensor-core GEMM: W planes, partials
  s.add(sizeof(double) * bgemm_simt_splits(m, n, k, num_sms) * k * n);  // FP64 B = W A partials
  s.add(ltc_workspace_bytes(m, k));                  // tensor-core L = L_y L_b: digit planes
  s.add(sizeof(int64_t) * kScanMaxParts);            // multi-CTA scan partials
  s.add(l1 <= kDirectMaxL1 ? sizeof(float) * l1 * l : 0);  // CSR sketch: table of D H R / sqrt(l1)
  s.add(blu_workspace_bytes(m, n, k, l, num_sms));   // blocked LUs of Y and B^T: digit planes of the trailing updates
  return s;
}

bool sizes_ok(int64_t m, int64_t n, int k, int l, int l1) {
  if (m < 1 || n < 1 || m >= (1ll << 31) || n >= (1ll << 31)) return false;
  if (k < 1 || k > l || l > l1) return false;
  if (l > m || k > (m < n ? m : n)) return false;
  if (l > kMaxL || l1 > kMaxL1) return false;
  return true;
}

// CTAs for the grid-synchronised kernels of this handle.
int coop_sms(const rlu_ctx* h) { return h->max_ctas > 0 && h->max_ctas < h->num_sms ? h->max_ctas : h->num_sms; }

int map_flags(unsigned int f) { return status_of_flags(f); }

__global__ void k_debug_recip(int64_t n, const double* x, double* out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = rcp_newton(x[i]);
}

__global__ void k_status_code(const unsigned int* flags, int32_t* out) { *out = status_of_flags(*flags); }

bool prec_dtype_ok(int prec, int dtype) {
  switch (prec) {
    case RLU_PREC_F64: return dtype == RLU_F64;
    case RLU_PREC_F32: return dtype == RLU_F32 || dtype == RLU_BF16;
    case RLU_PREC_BF16:
    case RLU_PREC_BF16_REFINE: return dtype == RLU_BF16;
    default: return false;
  }
}

// CSR scratch: three blocks (per row, per entry, per heavy row).  Heavy rows
// hold at least ceil(n/4) entries each, so nnz bounds their number.
struct CsrLayout {
  size_t rows, entries, heavy;
  int64_t heavy_cap;
};

Sizes csr_rows_sizes(int64_t m, int64_t n, int k) {
  Sizes sz;
  for (int i = 0; i < 6; ++i) sz.add(sizeof(int32_t) * (m + 1));  // hflag, lflag, mflag, hpos, lpos, mpos
  sz.add(sizeof(int32_t) * m);                                     // heavy
  sz.add(sizeof(int32_t) * m);                                     // light
  sz.add(sizeof(int32_t) * m);                                     // mid
  sz.add(sizeof(int32_t) * 4);                                     // count
  sz.add(sizeof(int32_t) * (n + 1));                               // ccnt
  sz.add(sizeof(int32_t) * (n + 1));                               // cstart
  sz.add((size_t)8 * m * k);                                       // W^T
  sz.add(sizeof(int32_t) * (m + 1));                               // llen
  sz.add(sizeof(int32_t) * (m + 1));                               // loff
  sz.add(sizeof(int32_t) * (256 * kRadixMaxChunks + 1));           // rhist
  sz.add(sizeof(int32_t) * (256 * kRadixMaxChunks + 1));           // roffs
  return sz;
}

// two slots of (column int32, row int32, value up to 8 bytes) per light entry
size_t csr_entry_bytes(int64_t nnz) {
  const size_t e = (size_t)max64(nnz, 1);
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  return 2 * (up(4 * e) + up(4 * e) + up(8 * e));
}

size_t csr_heavy_bytes(int64_t nheavy, int64_t n, int k, int num_sms, size_t* dbytes, size_t* wbytes) {
  const int64_t nh = max64(nheavy, 1);
  const size_t d = (((size_t)8 * nh * n) + 1023) & ~(size_t)1023;
  const size_t w = (((size_t)8 * k * nh) + 1023) & ~(size_t)1023;
  if (dbytes) *dbytes = d;
  if (wbytes) *wbytes = w;
  return d + w + tc_workspace_bytes(nh, n, k, num_sms);
}

CsrLayout csr_layout(int64_t m, int64_t n, int k, int64_t nnz, int num_sms) {
  CsrLayout c;
  c.rows = (csr_rows_sizes(m, n, k).total + 255) & ~(size_t)255;
  c.entries = csr_entry_bytes(nnz);
  const int64_t per = (n + 3) / 4;
  c.heavy_cap = min64(m, max64(nnz, 0) / max64(per, 1));
  c.heavy = (csr_heavy_bytes(c.heavy_cap, n, k, num_sms, nullptr, nullptr) + 255) & ~(size_t)255;
  return c;
}

void csr_carve_rows(rlu_ctx* h, char* b) {
  Sizes sz = csr_rows_sizes(h->m, h->n, h->k);
  size_t off = 0;
  int idx = 0;
  auto next = [&]() -> void* { void* p = b + off; off += sz.parts[idx++]; return p; };
  CsrWs& w = h->csr;
  w.hflag = (int32_t*)next(); w.lflag = (int32_t*)next(); w.mflag = (int32_t*)next();
  w.hpos = (int32_t*)next(); w.lpos = (int32_t*)next(); w.mpos = (int32_t*)next();
  w.heavy = (int32_t*)next(); w.light = (int32_t*)next(); w.mid = (int32_t*)next(); w.count = (int32_t*)next();
  w.ccnt = (int32_t*)next(); w.cstart = (int32_t*)next(); w.Wt = next();
  w.llen = (int32_t*)next(); w.loff = (int32_t*)next(); w.rhist = (int32_t*)next(); w.roffs = (int32_t*)next();
}

void csr_carve_entries(rlu_ctx* h, char* b, int64_t nnz) {
  const size_t e = (size_t)max64(nnz, 1);
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  for (int s = 0; s < 2; ++s) {
    h->csr.ekey[s] = (int32_t*)b;
    b += up(4 * e);
    h->csr.erow[s] = (int32_t*)b;
    b += up(4 * e);
    h->csr.eval[s] = b;
    b += up(8 * e);
  }
}

int csr_rows_alloc(rlu_ctx* h) {
  if (h->csr_rows_ready) return RLU_OK;
  char* b = nullptr;
  if (cudaMalloc(&b, csr_rows_sizes(h->m, h->n, h->k).total) != cudaSuccess) {
    cudaGetLastError();
    return RLU_ENOMEM;
  }
  h->csr_rows_buf = b;
  csr_carve_rows(h, b);
  h->csr_rows_ready = true;
  return RLU_OK;
}

int csr_grow(rlu_ctx* h, int64_t nnz, int64_t nheavy) {
  if (h->csr_external) {  // caller-owned scratch, sized for csr_cap_nnz entries
    if (nnz > h->csr_cap_nnz || nheavy > h->csr_cap_heavy) return RLU_EINVAL;
  }
  if (nnz > h->csr_cap_nnz) {
    if (h->csr_nnz_buf) cudaFree(h->csr_nnz_buf);
    h->csr_nnz_buf = nullptr;
    h->csr_cap_nnz = -1;
    char* b = nullptr;
    if (cudaMalloc(&b, csr_entry_bytes(nnz)) != cudaSuccess) { cudaGetLastError(); return RLU_ENOMEM; }
    h->csr_nnz_buf = b;
    csr_carve_entries(h, b, nnz);
    h->csr_cap_nnz = nnz;
  }
  if (nheavy > h->csr_cap_heavy) {
    if (h->csr_heavy_buf) cudaFree(h->csr_heavy_buf);
    h->csr_heavy_buf = nullptr;
    h->csr_cap_heavy = -1;
    char* b = nullptr;
    if (cudaMalloc(&b, csr_heavy_bytes(nheavy, h->n, h->k, h->num_sms, nullptr, nullptr)) != cudaSuccess) {
      cudaGetLastError();
      return RLU_ENOMEM;
    }
    h->csr_heavy_buf = b;
    h->csr_cap_heavy = nheavy;
  }
  if (nheavy > 0) {
    size_t dbytes = 0, wbytes = 0;
    csr_heavy_bytes(h->csr_cap_heavy, h->n, h->k, h->num_sms, &dbytes, &wbytes);
    h->csr.D = h->csr_heavy_buf;
    h->csr.Wh = (char*)h->csr_heavy_buf + dbytes;
    int rc = tc_setup(h->csr.tc, (char*)h->csr_heavy_buf + dbytes + wbytes, nheavy, h->n, h->k, h->num_sms);
    if (rc) return rc;
  }
  return RLU_OK;
}

int mark(rlu_ctx* h, int i, cudaStream_t st) {
  if (!h->timing) return RLU_OK;
  RLU_CUDA_TRY(cudaEventRecord(h->ev[i], st));
  if (i == kNumStages) h->ev_recorded = 1;
  return RLU_OK;
}

// Enqueue the dense path; the device status word receives the flags.
int enqueue_dense(rlu_ctx* h, const void* A, int64_t lda, int dtype, void* L, void* U, int64_t* p, int64_t* q,
                  cudaStream_t st) {
  const int64_t m = h->m, n = h->n;
  const int k = h->k, l = h->l, l1 = h->l1;
  const bool f64 = (h->prec == RLU_PREC_F64);
  int rc;
  RLU_CUDA_TRY(cudaMemsetAsync(h->status_dev, 0, sizeof(unsigned int), st));
  h->ev_recorded = 0;
  if ((rc = mark(h, 0, st))) return rc;
  // step 1: S, D, R (whole-row bucket lists for the SRHT and SRFT products)
  if (h->xform != RLU_XFORM_HARTLEY) {
    h->sk.chunk = (int)n;
    if (!h->xf_buf) {
      if (cudaMalloc(&h->xf_buf, xform_buffer_bytes(m, l1, l, true)) != cudaSuccess) {
        cudaGetLastError();
        h->xf_buf = nullptr;
        return RLU_ENOMEM;
      }
    }
  } else {
    const size_t es = dtype == RLU_F64 ? 8 : (dtype == RLU_F32 ? 4 : 2);
    const bool al = ((uintptr_t)A % 16 == 0) && (((size_t)lda * es) % 16 == 0);
    h->sk.chunk = sketch_chunk_cols(dtype, m, n, l1, al, h->num_sms);
  }
  h->sk.nchunks = cdiv(n, h->sk.chunk);
  if ((rc = launch_sketch_params(h->sk, n, l1, l, h->seed, st))) return rc;
  if ((rc = mark(h, 1, st))) return rc;
  // step 2: Y = A S D H R / sqrt(l1) (or the SRHT / SRFT projection)
  if (h->xform != RLU_XFORM_HARTLEY)
    rc = launch_sketch_xform(h->xform, A, lda, dtype, f64, m, n, l1, l, h->seed, h->sk, h->xf_buf, h->Y,
                             h->status_dev, st);
  else
    rc = launch_sketch_dense(A, lda, dtype, f64, m, n, l1, l, h->sk, h->Y, h->status_dev, h->num_sms, st);
  if (rc) return rc;
  if (h->colpiv && (rc = launch_column_pivoting(h->Y, m, l, h->cp_buf, h->cp_splits, h->num_sms, st))) return rc;
  if ((rc = mark(h, 2, st))) return rc;
  if (h->debug && h->Ydbg)
    RLU_CUDA_TRY(cudaMemcpyAsync(h->Ydbg, h->Y, sizeof(double) * m * l, cudaMemcpyDeviceToDevice, st));
  // step 3: P Y = L_Y U_Y (FP64, l steps)
  h->pw.perm = h->perm_y;
  if ((rc = launch_lu_y(h->Y, m, l, h->pw, h->blu, h->lu_block, h->status_dev, coop_sms(h), st,
                        h->timing ? &h->ptimer[0] : nullptr)))
    return rc;
  if ((rc = mark(h, 3, st))) return rc;
  // W = L_y^+ P
  PinvArgs pa{};
  pa.m = m; pa.k = k; pa.l = l;
  pa.Y = h->Y; pa.pstep = h->pw.pstep; pa.Lk = h->Lk;
  pa.gram_part = h->gram_part; pa.max_gram_splits = h->max_gram_splits;
  pa.G = h->G; pa.Rinv = h->Rinv; pa.Ginv = h->Ginv;
  pa.W = h->W; pa.w64 = f64 ? 1 : 0;
  pa.bar = h->bar2; pa.status = h->status_dev; pa.num_sms = h->num_sms; pa.coop_ctas = coop_sms(h);
  // W and its BF16 planes from the tensor-core digit product (FP32 outputs)
  const bool w_tc = !f64 && h->ltc.ready && h->tcw.ready;
  pa.ltc = w_tc ? &h->ltc : nullptr;
  pa.wplanes = w_tc ? h->tcw.wp : nullptr;
  pa.ldw = h->tcw.plan.ldw;
  if (h->k2 > 0) {
    // steps 4-6 of Algorithm 1: B = (Omega_2 L_1)^+ Omega_2 P A (the timing stage
    // "gram" covers all of it; chol, wform and bgemm then read zero)
    const size_t esz = dtype == RLU_F64 ? 8 : (dtype == RLU_F32 ? 4 : 2);
    const size_t need = esz * (size_t)m * n;
    if (h->at_bytes < need) {
      if (h->at_buf) cudaFree(h->at_buf);
      h->at_buf = nullptr;
      h->at_bytes = 0;
      if (cudaMalloc(&h->at_buf, need) != cudaSuccess) { cudaGetLastError(); return RLU_ENOMEM; }
      h->at_bytes = need;
    }
    SecondArgs sa{};
    sa.m = m; sa.n = n; sa.k = k; sa.k2 = h->k2; sa.l2 = h->l2; sa.seed2 = h->seed2;
    sa.A = A; sa.lda = lda; sa.dtype = dtype; sa.AT = h->at_buf;
    sa.LkT = h->LkT; sa.Y2T = h->Y2T; sa.ZT = h->ZT; sa.W2 = h->W2; sa.B = h->B;
    if ((rc = launch_second_projection(sa, pa, h->sk2, st))) return rc;
    for (int sidx = 4; sidx <= 7; ++sidx)
      if ((rc = mark(h, sidx, st))) return rc;
  } else {
    if ((rc = launch_gram(pa, st))) return rc;
    if ((rc = mark(h, 4, st))) return rc;
    if ((rc = launch_chol(pa, st))) return rc;
    if ((rc = mark(h, 5, st))) return rc;
    if ((rc = launch_wform(pa, st))) return rc;
    if ((rc = mark(h, 6, st))) return rc;
    // B = W A: tensor cores (BF16 splits) when available, else SIMT
    if (!f64 && h->tcw.ready)
      rc = launch_bgemm_tc(h->tcw, reinterpret_cast<const float*>(h->W), A, lda, dtype, h->prec, m, n, k,
                           reinterpret_cast<df32*>(h->B), h->status_dev, st, w_tc);
    else
      rc = launch_bgemm_simt(h->W, f64 ? 1 : 0, A, lda, dtype, m, n, k, h->B, h->bpart, h->num_sms, st);
    if (rc) return rc;
    if ((rc = mark(h, 7, st))) return rc;
  }
  if (h->debug && h->Bdbg)
    RLU_CUDA_TRY(cudaMemcpyAsync(h->Bdbg, h->B, 8 * (size_t)k * n, cudaMemcpyDeviceToDevice, st));
  // step 6: B Q = L_b U_b as partial pivoting of B^T
  h->pw.perm = h->perm_b;
  if (f64)
    rc = launch_lu_b<double>(reinterpret_cast<double*>(h->B), n, k, h->pw, h->blu, h->lu_block, h->status_dev,
                             coop_sms(h), st, h->timing ? &h->ptimer[1] : nullptr);
  else
    rc = launch_lu_b<df32>(reinterpret_cast<df32*>(h->B), n, k, h->pw, h->blu, h->lu_block, h->status_dev,
                           coop_sms(h), st, h->timing ? &h->ptimer[1] : nullptr);
  if (rc) return rc;
  if ((rc = mark(h, 8, st))) return rc;
  // step 7: L = L_y L_b, U = U_b, p, q
  AssembleArgs aa{};
  aa.m = m; aa.n = n; aa.k = k;
  aa.Lk = h->Lk; aa.perm_y = h->perm_y; aa.perm_b = h->perm_b; aa.Bp = h->B;
  aa.LyP = h->LyP; aa.Lb = h->Lb; aa.L = L; aa.U = U; aa.p = p; aa.q = q;
  aa.fp32_product = h->prec != RLU_PREC_F64 ? 1 : 0;  // FP32 outputs
  aa.num_sms = coop_sms(h);
  aa.ltc = &h->ltc;
  aa.status = h->status_dev;
  rc = f64 ? launch_assemble<double, double>(aa, st) : launch_assemble<df32, float>(aa, st);
  if (rc) return rc;
  if ((rc = mark(h, 9, st))) return rc;
  h->last_prec = h->prec;
  return RLU_OK;
}

// The CSR path: the same stages as enqueue_dense with the CSR sketch and the
// sparse B = W A; one host read-back of the heavy-row count after the row
// classification (it sizes the dense copy of the heavy rows).
int enqueue_csr(rlu_ctx* h, const int64_t* rowptr, const int32_t* colind, const void* val, int64_t nnz, int dtype,
                void* L, void* U, int64_t* p, int64_t* q, cudaStream_t st) {
  const int64_t m = h->m, n = h->n;
  const int k = h->k, l = h->l, l1 = h->l1;
  const bool f64 = (h->prec == RLU_PREC_F64);
  int rc;
  if ((rc = csr_rows_alloc(h))) return rc;
  RLU_CUDA_TRY(cudaMemsetAsync(h->status_dev, 0, sizeof(unsigned int), st));
  h->ev_recorded = 0;
  if ((rc = mark(h, 0, st))) return rc;
  // heavy rows are sketched from an aligned dense copy with row stride n
  h->sk.chunk = sketch_chunk_cols(dtype, m, n, l1, true, h->num_sms);
  h->sk.nchunks = cdiv(n, h->sk.chunk);
  if ((rc = launch_sketch_params(h->sk, n, l1, l, h->seed, st))) return rc;
  CsrRows cr{};
  const int64_t direct_max = f64 ? -1 : csr_direct_max(l1, l);  // FP64 sums keep the FFT route
  if ((rc = csr_classify(h->csr, rowptr, m, n, nnz, direct_max, h->status_dev, cr,
                         reinterpret_cast<int32_t*>(h->status_host + 4), st)))
    return rc;
  if ((rc = csr_grow(h, cr.n_light_nnz, cr.n_heavy))) return rc;  // entry scratch for the light entries
  if ((rc = mark(h, 1, st))) return rc;
  RLU_CUDA_TRY(cudaMemsetAsync(h->Y, 0, sizeof(double) * m * l, st));
  if ((rc = launch_sketch_csr(rowptr, colind, val, dtype, n, cr, l1, l, h->sk, h->csr.D, h->Y, h->fjl_table,
                              h->status_dev, h->num_sms, st)))
    return rc;
  if (h->colpiv && (rc = launch_column_pivoting(h->Y, m, l, h->cp_buf, h->cp_splits, h->num_sms, st))) return rc;
  if ((rc = mark(h, 2, st))) return rc;
  if (h->debug && h->Ydbg)
    RLU_CUDA_TRY(cudaMemcpyAsync(h->Ydbg, h->Y, sizeof(double) * m * l, cudaMemcpyDeviceToDevice, st));
  h->pw.perm = h->perm_y;
  if ((rc = launch_lu_y(h->Y, m, l, h->pw, h->blu, h->lu_block, h->status_dev, coop_sms(h), st,
                        h->timing ? &h->ptimer[0] : nullptr)))
    return rc;
  if ((rc = mark(h, 3, st))) return rc;
  PinvArgs pa{};
  pa.m = m; pa.k = k; pa.l = l;
  pa.Y = h->Y; pa.pstep = h->pw.pstep; pa.Lk = h->Lk;
  pa.gram_part = h->gram_part; pa.max_gram_splits = h->max_gram_splits;
  pa.G = h->G; pa.Rinv = h->Rinv; pa.Ginv = h->Ginv;
  pa.W = h->W; pa.w64 = f64 ? 1 : 0;
  pa.bar = h->bar2; pa.status = h->status_dev; pa.num_sms = h->num_sms; pa.coop_ctas = coop_sms(h);
  pa.ltc = (!f64 && h->ltc.ready) ? &h->ltc : nullptr;  // W from the digit product; the CSR path splits its own planes
  pa.wplanes = nullptr;
  pa.ldw = 0;
  if ((rc = launch_gram(pa, st))) return rc;
  if ((rc = mark(h, 4, st))) return rc;
  if ((rc = launch_chol(pa, st))) return rc;
  if ((rc = mark(h, 5, st))) return rc;
  if ((rc = launch_wform(pa, st))) return rc;
  if ((rc = mark(h, 6, st))) return rc;
  if ((rc = csr_bgemm(h->csr, rowptr, colind, val, dtype, h->prec, m, n, k, cr, h->W, h->B, h->status_dev,
                      h->num_sms, st)))
    return rc;
  if ((rc = mark(h, 7, st))) return rc;
  if (h->debug && h->Bdbg)
    RLU_CUDA_TRY(cudaMemcpyAsync(h->Bdbg, h->B, 8 * (size_t)k * n, cudaMemcpyDeviceToDevice, st));
  h->pw.perm = h->perm_b;
  if (f64)
    rc = launch_lu_b<double>(reinterpret_cast<double*>(h->B), n, k, h->pw, h->blu, h->lu_block, h->status_dev,
                             coop_sms(h), st, h->timing ? &h->ptimer[1] : nullptr);
  else
    rc = launch_lu_b<df32>(reinterpret_cast<df32*>(h->B), n, k, h->pw, h->blu, h->lu_block, h->status_dev,
                           coop_sms(h), st, h->timing ? &h->ptimer[1] : nullptr);
  if (rc) return rc;
  if ((rc = mark(h, 8, st))) return rc;
  AssembleArgs aa{};
  aa.m = m; aa.n = n; aa.k = k;
  aa.Lk = h->Lk; aa.perm_y = h->perm_y; aa.perm_b = h->perm_b; aa.Bp = h->B;
  aa.LyP = h->LyP; aa.Lb = h->Lb; aa.L = L; aa.U = U; aa.p = p; aa.q = q;
  aa.fp32_product = h->prec != RLU_PREC_F64 ? 1 : 0;  // FP32 outputs
  aa.num_sms = coop_sms(h);
  aa.ltc = &h->ltc;
  aa.status = h->status_dev;
  rc = f64 ? launch_assemble<double, double>(aa, st) : launch_assemble<df32, float>(aa, st);
  if (rc) return rc;
  if ((rc = mark(h, 9, st))) return rc;
  h->last_prec = h->prec;
  return RLU_OK;
}

// After a failed enqueue: wait for whatever was already enqueued (not while
// capturing), so no work of the call outlives it, and return `rc`.
int drain_after(int rc, cudaStream_t st) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) == cudaSuccess && cap == cudaStreamCaptureStatusNone) cudaStreamSynchronize(st);
  cudaGetLastError();
  return rc;
}

int finish_sync(rlu_ctx* h, cudaStream_t st) {
  RLU_CUDA_TRY(cudaMemcpyAsync(h->status_host, h->status_dev, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
  RLU_CUDA_TRY(cudaStreamSynchronize(st));
  return map_flags(*h->status_host);
}

}  // namespace

extern "C" {

const char* rlu_strerror(int code) {
  switch (code) {
    case RLU_OK: return "success";
    case RLU_EINVAL: return "invalid argument";
    case RLU_ENOMEM: return "device workspace allocation failed";
    case RLU_ECUDA: return "CUDA error or no usable GPU";
    case RLU_ETIMEOUT: return "a bounded device wait timed out";
    case RLU_ENONFINITE: return "input holds NaN or Inf";
    case RLU_EBADCSR: return "invalid CSR structure";
    case RLU_ETOOLARGE: return "sizes exceed the fixed scratch of the allocation-free sketch";
    case RLU_WRANK: return "warning: exactly zero pivot met (rank deficient input)";
    default: return "unknown status";
  }
}

int rlu_workspace_bytes(int64_t m, int64_t n, int32_t k, int32_t l, int32_t l1, int prec, size_t* bytes) {
  if (!bytes || !sizes_ok(m, n, k, l, l1) || prec < 0 || prec > 3) return RLU_EINVAL;
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  *bytes = plan_sizes(m, n, k, l, l1, sms).total;
  return RLU_OK;
}

int rlu_csr_workspace_bytes(int64_t m, int64_t n, int32_t k, int64_t max_nnz, size_t* bytes) {
  if (!bytes || m < 1 || n < 1 || k < 1 || max_nnz < 0 || max_nnz >= (1ll << 31)) return RLU_EINVAL;
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const CsrLayout c = csr_layout(m, n, k, max_nnz, sms);
  *bytes = c.rows + c.entries + c.heavy;
  return RLU_OK;
}

int rlu_set_csr_workspace(rlu_t h, int64_t max_nnz, void* workspace, size_t workspace_bytes) {
  if (!h || !workspace || max_nnz < 0 || max_nnz >= (1ll << 31) || ((uintptr_t)workspace % 256) != 0)
    return RLU_EINVAL;
  if (h->csr_rows_buf || h->csr_nnz_buf || h->csr_heavy_buf) return RLU_EINVAL;  // already has its own
  const CsrLayout c = csr_layout(h->m, h->n, h->k, max_nnz, h->num_sms);
  if (workspace_bytes < c.rows + c.entries + c.heavy) return RLU_EINVAL;
  char* b = (char*)workspace;
  h->csr_external = true;
  h->csr_rows_buf = b;
  csr_carve_rows(h, b);
  h->csr_rows_ready = true;
  h->csr_nnz_buf = b + c.rows;
  csr_carve_entries(h, b + c.rows, max_nnz);
  h->csr_cap_nnz = max_nnz;
  h->csr_heavy_buf = b + c.rows + c.entries;
  h->csr_cap_heavy = c.heavy_cap;
  return RLU_OK;
}

// Build a handle on workspace `base` (plan_sizes(...).total bytes).  With
// own_base the handle frees it; the caller's stream receives the twiddle
// launch.  `pinned` gives the handle its own page-locked host words for the
// status read-back; otherwise it takes them from the shared slab.
static int create_common(int64_t m, int64_t n, int32_t k, int32_t l, int32_t l1, uint64_t seed, char* base,
                         bool own_base, bool pinned, cudaStream_t st, rlu_t* out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RLU_ECUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return RLU_ECUDA;
  rlu_ctx* h = new (std::nothrow) rlu_ctx();
  if (!h) return RLU_ENOMEM;
  h->m = m; h->n = n; h->k = k; h->l = l; h->l1 = l1; h->seed = seed;
  h->device = dev; h->num_sms = sms;
  Sizes sz = plan_sizes(m, n, k, l, l1, sms);
  if (own_base) h->allocs.push_back(base);
  size_t off = 0;
  int idx = 0;
  auto next = [&](void) -> void* { void* p = base + off; off += sz.parts[idx++]; return p; };
  h->sk.hs = (uint32_t*)next();
  h->sk.dsign = (float*)next();
  h->sk.keys = (uint64_t*)next();
  h->sk.R = (int32_t*)next();
  h->sk.bcnt = (int32_t*)next();
  h->sk.bstart = (int32_t*)next();
  h->sk.blist = (uint32_t*)next();
  h->sk.tw64 = (double2*)next();
  h->sk.tw32 = (float2*)next();
  h->sk.plan = make_fft_plan(l1);
  h->Y = (double*)next();
  h->pw.pos = (int32_t*)next();
  h->pw.pstep = (int32_t*)next();
  h->perm_y = (int64_t*)next();
  h->perm_b = (int64_t*)next();
  h->pw.cand = next();
  h->pw.candrow = next();
  h->pw.bar = (unsigned int*)next();
  h->pw.max_ctas = kMaxPivCtas;
  h->pw.max_cols = l > k ? l : k;
  h->Lk = next();
  h->gram_part = (double*)next();
  h->max_gram_splits = max_gram_splits_for(k, sms);
  h->G = (double*)next();
  h->Rinv = (double*)next();
  h->Ginv = (double*)next();
  h->W = next();
  h->B = next();
  h->LyP = next();
  h->Lb = next();
  h->status_dev = (unsigned int*)next();
  h->bar2 = h->status_dev + 1;
  void* tcbase = next();
  h->bpart = (double*)next();
  void* ltcbase = next();
  h->sk.scan_tmp = (int64_t*)next();
  h->csr.scan_tmp = h->sk.scan_tmp;
  h->fjl_table = (float*)next();
  void* blubase = next();
  if (tc_setup(h->tcw, tcbase, m, n, k, sms) != RLU_OK || ltc_setup(h->ltc, ltcbase, m, k, sms) != RLU_OK ||
      blu_setup(h->blu, blubase, m, n, k, l, sms) != RLU_OK) {
    rlu_destroy(h);
    return RLU_ECUDA;
  }
  if (pinned) {
    if (cudaMallocHost(&h->status_host, 8 * sizeof(unsigned int)) != cudaSuccess) {
      cudaGetLastError();
      rlu_destroy(h);
      return RLU_ENOMEM;
    }
    h->status_pinned = true;
  } else {
    // a word of a shared page-locked slab: the status read-back stays a plain
    // DMA (a copy to pageable memory needs the calling thread's participation)
    h->status_host = status_slab_take();
    if (!h->status_host) {
      rlu_destroy(h);
      return RLU_ENOMEM;
    }
    h->status_slab = true;
  }
  if (launch_twiddles(l1, h->sk.tw64, h->sk.tw32, st) != RLU_OK) {
    rlu_destroy(h);
    return RLU_ECUDA;
  }
  *out = h;
  return RLU_OK;
}

int rlu_create(int64_t m, int64_t n, int32_t k, int32_t l, int32_t l1, uint64_t seed, rlu_t* out) {
  if (!out) return RLU_EINVAL;
  *out = nullptr;
  if (!sizes_ok(m, n, k, l, l1)) return RLU_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return RLU_ECUDA;
  char* base = nullptr;
  if (cudaMalloc(&base, plan_sizes(m, n, k, l, l1, sms).total) != cudaSuccess) {
    cudaGetLastError();
    return RLU_ENOMEM;
  }
  int rc = create_common(m, n, k, l, l1, seed, base, true, true, 0, out);
  if (rc) {
    if (!*out) cudaFree(base);
    return rc;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    rlu_destroy(*out);
    *out = nullptr;
    return RLU_ECUDA;
  }
  return RLU_OK;
}

int rlu_create_in(int64_t m, int64_t n, int32_t k, int32_t l, int32_t l1, uint64_t seed, void* workspace,
                  size_t workspace_bytes, void* stream, rlu_t* out) {
  if (!out) return RLU_EINVAL;
  *out = nullptr;
  if (!sizes_ok(m, n, k, l, l1) || !workspace || ((uintptr_t)workspace % 256) != 0) return RLU_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return RLU_ECUDA;
  if (workspace_bytes < plan_sizes(m, n, k, l, l1, sms).total) return RLU_EINVAL;
  return create_common(m, n, k, l, l1, seed, (char*)workspace, false, false, (cudaStream_t)stream, out);
}

int rlu_set_second_sketch(rlu_t h, int32_t k2, int32_t l2, uint64_t seed2) {
  if (!h) return RLU_EINVAL;
  if (k2 == 0) {
    h->k2 = 0;
    return RLU_OK;
  }
  // Z = Omega_2 L_1 is sketched in FP64, whose FFT buffers bound l2 by 4096
  if (k2 < h->k || k2 > l2 || k2 > kMaxL || l2 > 4096) return RLU_EINVAL;
  if (h->sk2_buf) cudaFree(h->sk2_buf);
  h->sk2_buf = nullptr;
  h->k2 = 0;
  const int64_t m = h->m, n = h->n, k = h->k;
  const int64_t nch = cdiv(m, 1024);
  Sizes sz;
  sz.add(sizeof(uint32_t) * m);                 // hs
  sz.add(sizeof(float) * l2);                   // dsign
  sz.add(sizeof(uint64_t) * l2);                // keys
  sz.add(sizeof(int32_t) * k2);                 // R
  sz.add(sizeof(int32_t) * (nch * l2 + 1));     // bcnt
  sz.add(sizeof(int32_t) * (nch * l2 + 1));     // bstart
  sz.add(sizeof(uint32_t) * m);                 // blist
  sz.add(sizeof(double2) * l2);                 // tw64
  sz.add(sizeof(float2) * l2);                  // tw32
  sz.add(sizeof(double) * n * k2);              // Y2T
  sz.add(sizeof(double) * k * m);               // LkT
  sz.add(sizeof(double) * k * k2);              // ZT
  sz.add((size_t)8 * k * k2);                   // W2
  char* b = nullptr;
  if (cudaMalloc(&b, sz.total) != cudaSuccess) {
    cudaGetLastError();
    return RLU_ENOMEM;
  }
  size_t off = 0;
  int idx = 0;
  auto next = [&]() -> void* { void* p = b + off; off += sz.parts[idx++]; return p; };
  SketchWs& w = h->sk2;
  w.hs = (uint32_t*)next(); w.dsign = (float*)next(); w.keys = (uint64_t*)next(); w.R = (int32_t*)next();
  w.bcnt = (int32_t*)next(); w.bstart = (int32_t*)next(); w.blist = (uint32_t*)next();
  w.tw64 = (double2*)next(); w.tw32 = (float2*)next();
  w.plan = make_fft_plan(l2);
  w.chunk = 1024;
  w.nchunks = nch;
  h->Y2T = (double*)next(); h->LkT = (double*)next(); h->ZT = (double*)next(); h->W2 = next();
  h->sk2_buf = b;
  if (launch_twiddles(l2, w.tw64, w.tw32, 0) != RLU_OK || cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return RLU_ECUDA;
  }
  h->k2 = k2;
  h->l2 = l2;
  h->seed2 = seed2;
  return RLU_OK;
}

int rlu_set_max_ctas(rlu_t h, int32_t max_ctas) {
  if (!h || max_ctas < 0) return RLU_EINVAL;
  h->max_ctas = max_ctas;
  return RLU_OK;
}

int rlu_set_precision(rlu_t h, int prec) {
  if (!h || prec < 0 || prec > 3) return RLU_EINVAL;
  h->prec = prec;
  return RLU_OK;
}

int rlu_debug_set_lu_block(rlu_t h, int32_t block) {
  if (!h) return RLU_EINVAL;
  if (block != -1 && block != 0 && block != 16 && block != 32 && block != 64) return RLU_EINVAL;
  if (block > 0 && (!h->blu.ready || block > h->blu.bmax || block >= h->k)) return RLU_EINVAL;
  h->lu_block = block;
  return RLU_OK;
}

int rlu_debug_set_tma_a(rlu_t h, int on) {
  if (!h || (on != 0 && on != 1)) return RLU_EINVAL;
  h->tcw.a_tma = on != 0;
  return RLU_OK;
}

int rlu_debug_lu_block(rlu_t h, int32_t* block_max) {
  if (!h) return RLU_EINVAL;
  if (block_max) *block_max = h->blu.ready ? h->blu.bmax : 0;
  return h->lu_block;
}

int rlu_set_column_pivoting(rlu_t h, int on) {
  if (!h) return RLU_EINVAL;
  if (on && !h->cp_buf) {
    const int splits = 4 * h->num_sms;
    if (cudaMalloc(&h->cp_buf, colpiv_buffer_bytes(h->m, h->l, splits)) != cudaSuccess) {
      cudaGetLastError();
      h->cp_buf = nullptr;
      return RLU_ENOMEM;
    }
    h->cp_splits = splits;
    if (cudaDeviceSynchronize() != cudaSuccess) return RLU_ECUDA;
  }
  h->colpiv = on ? 1 : 0;
  return RLU_OK;
}

int rlu_set_transform(rlu_t h, int transform) {
  if (!h) return RLU_EINVAL;
  if (transform == RLU_XFORM_SRHT && (h->l1 & (h->l1 - 1))) return RLU_EINVAL;
  if (transform == RLU_XFORM_SRFT && (h->l & 1)) return RLU_EINVAL;
  if (transform < RLU_XFORM_HARTLEY || transform > RLU_XFORM_SRFT) return RLU_EINVAL;
  h->xform = transform;
  return RLU_OK;
}

int rlu_destroy(rlu_t h) {
  if (!h) return RLU_OK;
  for (void* p : h->allocs) cudaFree(p);
  if (h->status_host) {
    if (h->status_pinned) cudaFreeHost(h->status_host);
    else if (h->status_slab) status_slab_give(h->status_host);
  }
  if (h->Ydbg) cudaFree(h->Ydbg);
  if (h->Bdbg) cudaFree(h->Bdbg);
  if (h->A_stage) cudaFree(h->A_stage);
  if (h->L_stage) cudaFree(h->L_stage);
  if (h->U_stage) cudaFree(h->U_stage);
  if (h->p_stage) cudaFree(h->p_stage);
  if (h->q_stage) cudaFree(h->q_stage);
  if (h->sk2_buf) cudaFree(h->sk2_buf);
  if (h->at_buf) cudaFree(h->at_buf);
  if (h->xf_buf) cudaFree(h->xf_buf);
  if (h->cp_buf) cudaFree(h->cp_buf);
  if (!h->csr_external) {
    if (h->csr_rows_buf) cudaFree(h->csr_rows_buf);
    if (h->csr_nnz_buf) cudaFree(h->csr_nnz_buf);
    if (h->csr_heavy_buf) cudaFree(h->csr_heavy_buf);
  }
  for (int i = 0; i <= kNumStages; ++i)
    if (h->ev[i]) cudaEventDestroy(h->ev[i]);
  for (PanelTimer& t : h->ptimer)
    for (cudaEvent_t e : t.ev)
      if (e) cudaEventDestroy(e);
  delete h;
  return RLU_OK;
}

int rlu_factor_dense_async(rlu_t h, const void* A, int64_t lda, int dtype, void* L, void* U, int64_t* p, int64_t* q,
                           int32_t* status_dev, void* stream) {
  if (!h || !A || !L || !U || !p || !q || !status_dev) return RLU_EINVAL;
  if (lda < h->n || !prec_dtype_ok(h->prec, dtype)) return RLU_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = enqueue_dense(h, A, lda, dtype, L, U, p, q, st);
  if (rc) return drain_after(rc, st);
  k_status_code<<<1, 1, 0, st>>>(h->status_dev, status_dev);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  return RLU_OK;
}

int rlu_factor_dense(rlu_t h, const void* A, int64_t lda, int dtype, void* L, void* U, int64_t* p, int64_t* q,
                     void* stream) {
  if (!h || !A || !L || !U || !p || !q) return RLU_EINVAL;
  if (lda < h->n || !prec_dtype_ok(h->prec, dtype)) return RLU_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = enqueue_dense(h, A, lda, dtype, L, U, p, q, st);
  if (rc) return drain_after(rc, st);
  return finish_sync(h, st);
}

int rlu_graph_capture_dense(rlu_t h, const void* A, int64_t lda, int dtype, void* L, void* U, int64_t* p,
                            int64_t* q, int32_t* status_dev, void* stream, rlu_graph_t* out) {
  if (!out) return RLU_EINVAL;
  *out = nullptr;
  if (!h || !A || !L || !U || !p || !q || !status_dev || !stream) return RLU_EINVAL;
  if (lda < h->n || !prec_dtype_ok(h->prec, dtype) || h->timing || h->debug) return RLU_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  RLU_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  const long long before = rlu::t_launches;
  int rc = enqueue_dense(h, A, lda, dtype, L, U, p, q, st);
  if (!rc) {
    k_status_code<<<1, 1, 0, st>>>(h->status_dev, status_dev);
    if (cudaGetLastError() != cudaSuccess) rc = RLU_ECUDA;
    rlu::note_launch();
  }
  // captured launches do not run now; the count moves to each graph launch
  const long long captured = rlu::t_launches - before;
  rlu::g_launches.fetch_sub(captured);
  rlu::t_launches -= captured;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(st, &g);
  if (rc || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return rc ? rc : RLU_ECUDA;
  }
  cudaGraphExec_t ge = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) {
    cudaGetLastError();
    return RLU_ECUDA;
  }
  rlu_graph* gr = new (std::nothrow) rlu_graph();
  if (!gr) {
    cudaGraphExecDestroy(ge);
    return RLU_ENOMEM;
  }
  gr->exec = ge;
  gr->kernels = captured;
  *out = gr;
  return RLU_OK;
}

int rlu_copy_block_async(void* dst, int64_t dst_pitch, const void* src, int64_t src_pitch, int64_t width_bytes,
                         int64_t rows, void* stream) {
  if (rows < 0 || width_bytes < 0) return RLU_EINVAL;
  if (rows == 0 || width_bytes == 0) return RLU_OK;
  if (!dst || !src || dst_pitch < width_bytes || src_pitch < width_bytes) return RLU_EINVAL;
  RLU_CUDA_TRY(cudaMemcpy2DAsync(dst, (size_t)dst_pitch, src, (size_t)src_pitch, (size_t)width_bytes, (size_t)rows,
                                 cudaMemcpyDefault, (cudaStream_t)stream));
  return RLU_OK;
}

int rlu_graph_launch(rlu_graph_t g, void* stream) {
  if (!g || !g->exec) return RLU_EINVAL;
  RLU_CUDA_TRY(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
  note_launch((int)g->kernels);
  return RLU_OK;
}

int rlu_graph_destroy(rlu_graph_t g) {
  if (!g) return RLU_OK;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  delete g;
  return RLU_OK;
}

int rlu_factor_csr(rlu_t h, const int64_t* rowptr, const int32_t* colind, const void* val, int64_t nnz, int dtype,
                   void* L, void* U, int64_t* p, int64_t* q, void* stream) {
  if (!h || !rowptr || !L || !U || !p || !q || nnz < 0 || nnz >= (1ll << 31)) return RLU_EINVAL;
  if (nnz > 0 && (!colind || !val)) return RLU_EINVAL;
  if (!((dtype == RLU_F64 && h->prec == RLU_PREC_F64) || (dtype == RLU_F32 && h->prec == RLU_PREC_F32)))
    return RLU_EINVAL;
  if (h->csr_external && nnz > h->csr_cap_nnz) return RLU_EINVAL;
  if (h->k2 > 0) return RLU_EINVAL;  // the second projection is built for dense A
  if (h->xform != RLU_XFORM_HARTLEY) return RLU_EINVAL;  // so are the SRHT and SRFT products
  cudaStream_t st = (cudaStream_t)stream;
  int rc = enqueue_csr(h, rowptr, colind, val, nnz, dtype, L, U, p, q, st);
  if (rc) return drain_after(rc, st);
  return finish_sync(h, st);
}

int rlu_factor_dense_host(rlu_t h, const void* A_host, int dtype, void* L_host, void* U_host, int64_t* p_host,
                          int64_t* q_host, void* stream) {
  if (!h || !A_host || !L_host || !U_host || !p_host || !q_host) return RLU_EINVAL;
  if (!prec_dtype_ok(h->prec, dtype)) return RLU_EINVAL;
  const size_t es = dtype == RLU_F64 ? 8 : (dtype == RLU_F32 ? 4 : 2);
  const size_t abytes = es * (size_t)h->m * h->n;
  const size_t os = h->prec == RLU_PREC_F64 ? 8 : 4;
  if (h->A_stage_bytes < abytes) {
    if (h->A_stage) cudaFree(h->A_stage);
    h->A_stage = nullptr;
    h->A_stage_bytes = 0;
    if (cudaMalloc(&h->A_stage, abytes) != cudaSuccess) { cudaGetLastError(); return RLU_ENOMEM; }
    h->A_stage_bytes = abytes;
  }
  if (!h->L_stage) {
    if (cudaMalloc(&h->L_stage, 8 * (size_t)h->m * h->k) != cudaSuccess ||
        cudaMalloc(&h->U_stage, 8 * (size_t)h->k * h->n) != cudaSuccess ||
        cudaMalloc(&h->p_stage, 8 * (size_t)h->m) != cudaSuccess ||
        cudaMalloc(&h->q_stage, 8 * (size_t)h->n) != cudaSuccess) {
      cudaGetLastError();
      return RLU_ENOMEM;
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  RLU_CUDA_TRY(cudaMemcpyAsync(h->A_stage, A_host, abytes, cudaMemcpyHostToDevice, st));
  int rc = enqueue_dense(h, h->A_stage, h->n, dtype, h->L_stage, h->U_stage, h->p_stage, h->q_stage, st);
  if (rc) return drain_after(rc, st);
  RLU_CUDA_TRY(cudaMemcpyAsync(L_host, h->L_stage, os * h->m * h->k, cudaMemcpyDeviceToHost, st));
  RLU_CUDA_TRY(cudaMemcpyAsync(U_host, h->U_stage, os * h->k * h->n, cudaMemcpyDeviceToHost, st));
  RLU_CUDA_TRY(cudaMemcpyAsync(p_host, h->p_stage, 8 * h->m, cudaMemcpyDeviceToHost, st));
  RLU_CUDA_TRY(cudaMemcpyAsync(q_host, h->q_stage, 8 * h->n, cudaMemcpyDeviceToHost, st));
  return finish_sync(h, st);
}

int rlu_debug_timing(rlu_t h, int on) {
  if (!h) return RLU_EINVAL;
  if (on && !h->ev[0])
    for (int i = 0; i <= kNumStages; ++i) RLU_CUDA_TRY(cudaEventCreate(&h->ev[i]));
  if (on && !h->ptimer[0].ev[0])
    for (PanelTimer& t : h->ptimer)
      for (cudaEvent_t& e : t.ev) RLU_CUDA_TRY(cudaEventCreate(&e));
  h->timing = on ? 1 : 0;
  h->ev_recorded = 0;
  return RLU_OK;
}

int rlu_debug_stage_ms(rlu_t h, float* ms, int max_stages, int* count) {
  if (!h || !ms || !count) return RLU_EINVAL;
  *count = 0;
  if (!h->timing || !h->ev_recorded) return RLU_EINVAL;
  RLU_CUDA_TRY(cudaEventSynchronize(h->ev[kNumStages]));
  int cnt = max_stages < kNumStages ? max_stages : kNumStages;
  for (int i = 0; i < cnt; ++i) RLU_CUDA_TRY(cudaEventElapsedTime(&ms[i], h->ev[i], h->ev[i + 1]));
  *count = cnt;
  return RLU_OK;
}

int rlu_debug_lu_panels(rlu_t h, int which, int32_t* width, int32_t* launches, double* ms) {
  if (!h || which < 0 || which > 1 || !width || !launches || !ms) return RLU_EINVAL;
  if (!h->timing || !h->ev_recorded) return RLU_EINVAL;
  const PanelTimer& t = h->ptimer[which];
  RLU_CUDA_TRY(cudaEventSynchronize(h->ev[kNumStages]));
  double tot = 0.0;
  for (int i = 0; i < t.n; ++i) {
    float x = 0.f;
    RLU_CUDA_TRY(cudaEventElapsedTime(&x, t.ev[2 * i], t.ev[2 * i + 1]));
    tot += x;
  }
  *width = t.width;
  *launches = t.n;
  *ms = tot;
  return RLU_OK;
}

int rlu_debug_status_of_flags(uint32_t flags, int* status) {
  if (!status) return RLU_EINVAL;
  *status = status_of_flags(flags);
  return RLU_OK;
}

int rlu_debug_launch_count(int64_t* out) {
  if (!out) return RLU_EINVAL;
  *out = (int64_t)rlu::g_launches.load();
  return RLU_OK;
}

int rlu_debug_recip(const double* x, double* out, int64_t n) {
  if (!x || !out || n < 0) return RLU_EINVAL;
  if (n == 0) return RLU_OK;
  double* d = nullptr;
  if (cudaMalloc(&d, sizeof(double) * 2 * n) != cudaSuccess) {
    cudaGetLastError();
    return RLU_ENOMEM;
  }
  int rc = RLU_OK;
  if (cudaMemcpy(d, x, sizeof(double) * n, cudaMemcpyHostToDevice) != cudaSuccess) rc = RLU_ECUDA;
  if (!rc) {
    k_debug_recip<<<(unsigned)cdiv(n, 256), 256>>>(n, d, d + n);
    note_launch();
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpy(out, d + n, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = RLU_ECUDA;
  }
  cudaFree(d);
  cudaGetLastError();
  return rc;
}

int rlu_debug_enable(rlu_t h, int on) {
  if (!h) return RLU_EINVAL;
  h->debug = on ? 1 : 0;
  if (h->debug && !h->Ydbg) {
    if (cudaMalloc(&h->Ydbg, sizeof(double) * h->m * h->l) != cudaSuccess ||
        cudaMalloc(&h->Bdbg, sizeof(double) * h->k * h->n) != cudaSuccess) {
      cudaGetLastError();
      return RLU_ENOMEM;
    }
  }
  return RLU_OK;
}

int rlu_debug_sketch_params(rlu_t h, int32_t* hash, int8_t* s, int8_t* d, int32_t* R) {
  if (!h || !hash || !s || !d || !R) return RLU_EINVAL;
  std::vector<uint32_t> hs(h->n);
  std::vector<float> ds(h->l1);
  RLU_CUDA_TRY(cudaDeviceSynchronize());
  RLU_CUDA_TRY(cudaMemcpy(hs.data(), h->sk.hs, sizeof(uint32_t) * h->n, cudaMemcpyDeviceToHost));
  RLU_CUDA_TRY(cudaMemcpy(ds.data(), h->sk.dsign, sizeof(float) * h->l1, cudaMemcpyDeviceToHost));
  RLU_CUDA_TRY(cudaMemcpy(R, h->sk.R, sizeof(int32_t) * h->l, cudaMemcpyDeviceToHost));
  for (int64_t j = 0; j < h->n; ++j) {
    hash[j] = (int32_t)(hs[j] & 0x7fffffffu);
    s[j] = (hs[j] >> 31) ? -1 : 1;
  }
  for (int b = 0; b < h->l1; ++b) d[b] = ds[b] < 0 ? -1 : 1;
  return RLU_OK;
}

int rlu_debug_Y(rlu_t h, double* Y_host) {
  if (!h || !Y_host || !h->Ydbg) return RLU_EINVAL;
  RLU_CUDA_TRY(cudaDeviceSynchronize());
  RLU_CUDA_TRY(cudaMemcpy(Y_host, h->Ydbg, sizeof(double) * h->m * h->l, cudaMemcpyDeviceToHost));
  return RLU_OK;
}

int rlu_debug_lu_Y(rlu_t h, double* Y_host, int64_t* perm_host) {
  if (!h || !Y_host || !perm_host) return RLU_EINVAL;
  RLU_CUDA_TRY(cudaDeviceSynchronize());
  RLU_CUDA_TRY(cudaMemcpy(Y_host, h->Y, sizeof(double) * h->m * h->l, cudaMemcpyDeviceToHost));
  RLU_CUDA_TRY(cudaMemcpy(perm_host, h->perm_y, sizeof(int64_t) * h->m, cudaMemcpyDeviceToHost));
  return RLU_OK;
}

int rlu_debug_B(rlu_t h, double* B_host) {
  if (!h || !B_host || !h->Bdbg) return RLU_EINVAL;
  RLU_CUDA_TRY(cudaDeviceSynchronize());
  const size_t cnt = (size_t)h->k * h->n;
  if (h->last_prec == RLU_PREC_F64) {
    RLU_CUDA_TRY(cudaMemcpy(B_host, h->Bdbg, sizeof(double) * cnt, cudaMemcpyDeviceToHost));
  } else {
    std::vector<float> tmp(2 * cnt);  // float-float pairs
    RLU_CUDA_TRY(cudaMemcpy(tmp.data(), h->Bdbg, sizeof(float) * 2 * cnt, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < cnt; ++i) B_host[i] = (double)tmp[2 * i] + (double)tmp[2 * i + 1];
  }
  return RLU_OK;
}

}  // extern "C"
