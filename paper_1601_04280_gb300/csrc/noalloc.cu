// rlu_sketch_dense_noalloc: the sketch step (Y = A S D H R / sqrt(l1)) for
// callers that cannot allocate device memory.
//
// Who needs it: code that must not call cudaMalloc on its hot path — a
// serving loop (cudaMalloc synchronizes the device and stalls every stream),
// a host that runs inside another framework's memory pool that has already
// reserved the device memory, or an embedded caller with a fixed memory map.
// Such callers pass only their input A and their output Y; the scratch this
// step needs (hash and sign arrays, per-chunk bucket lists, twiddles, a
// status word) lives in one file-scope device array of fixed size that every
// GPU loading this library keeps until the process exits.
//
// Each device has its own copy of the array.  On one device it is shared by
// all calls and keeps the previous call's contents: every call clears what
// must start at zero (bucket counters, status) before use.  Calls on the same
// device whose work overlaps on the GPU (for example on two streams) race on
// the scratch; serialize them.
#include <mutex>

#include "common.cuh"
#include "sketch.cuh"

namespace rlu {
namespace {

constexpr int64_t kMaxN = RLU_NOALLOC_MAX_N;
constexpr int64_t kMaxL1 = RLU_NOALLOC_MAX_L1;
constexpr int64_t kMaxL = RLU_NOALLOC_MAX_L;
constexpr int64_t kMinChunk = 1024;  // smallest column chunk of the dense sketch
constexpr int64_t kMaxChunks = (kMaxN + kMinChunk - 1) / kMinChunk;

constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t kOffHs = 0;
constexpr size_t kOffList = kOffHs + align256(4 * kMaxN);
constexpr size_t kOffCnt = kOffList + align256(4 * kMaxN);
constexpr size_t kOffStart = kOffCnt + align256(4 * (kMaxChunks * kMaxL1 + 1));
constexpr size_t kOffD = kOffStart + align256(4 * (kMaxChunks * kMaxL1 + 1));
constexpr size_t kOffKeys = kOffD + align256(4 * kMaxL1);
constexpr size_t kOffR = kOffKeys + align256(8 * kMaxL1);
constexpr size_t kOffTw64 = kOffR + align256(4 * kMaxL);
constexpr size_t kOffTw32 = kOffTw64 + align256(16 * kMaxL1);
constexpr size_t kOffStatus = kOffTw32 + align256(8 * kMaxL1);
constexpr size_t kScratchBytes = kOffStatus + 256;
static_assert(kScratchBytes == RLU_NOALLOC_SCRATCH_BYTES, "scratch size in rlu.h is out of date");

// The scratch itself.  In host code this name is only a stand-in for the
// symbol, not a device address: its address on each device comes from
// cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_sketch_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch on the current device, resolved once per
// device (with that device current) and cached.
int scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return RLU_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_sketch_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return RLU_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return RLU_OK;
}

// The same flag-to-status mapping as every other entry point: a timed-out
// wait (Y partly unwritten) reports RLU_ETIMEOUT ahead of a non-finite input.
__global__ void k_noalloc_status(const unsigned int* flags, int32_t* out) { *out = status_of_flags(*flags); }

}  // namespace
}  // namespace rlu

extern "C" int rlu_sketch_dense_noalloc(const void* A, int64_t lda, int dtype, int64_t m, int64_t n, int32_t l,
                                        int32_t l1, uint64_t seed, double* Y, int32_t* status_dev, void* stream) {
  using namespace rlu;
  if (!A || !Y || !status_dev) return RLU_EINVAL;
  if (dtype != RLU_F64 && dtype != RLU_F32 && dtype != RLU_BF16) return RLU_EINVAL;
  if (m < 1 || n < 1 || l < 1 || l > l1 || l > m || lda < n || m >= (1ll << 31)) return RLU_EINVAL;
  if (n > kMaxN || l1 > kMaxL1 || l > kMaxL) return RLU_ETOOLARGE;
  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
    cudaGetLastError();
    return RLU_ECUDA;
  }
  unsigned char* b = static_cast<unsigned char*>(base);
  SketchWs ws{};
  ws.hs = reinterpret_cast<uint32_t*>(b + kOffHs);
  ws.blist = reinterpret_cast<uint32_t*>(b + kOffList);
  ws.bcnt = reinterpret_cast<int32_t*>(b + kOffCnt);
  ws.bstart = reinterpret_cast<int32_t*>(b + kOffStart);
  ws.dsign = reinterpret_cast<float*>(b + kOffD);
  ws.keys = reinterpret_cast<uint64_t*>(b + kOffKeys);
  ws.R = reinterpret_cast<int32_t*>(b + kOffR);
  ws.tw64 = reinterpret_cast<double2*>(b + kOffTw64);
  ws.tw32 = reinterpret_cast<float2*>(b + kOffTw32);
  ws.plan = make_fft_plan(l1);
  {
    const size_t es = dtype == RLU_F64 ? 8 : (dtype == RLU_F32 ? 4 : 2);
    ws.chunk = sketch_chunk_cols(dtype, m, n, l1, ((uintptr_t)A % 16 == 0) && (((size_t)lda * es) % 16 == 0), sms);
  }
  ws.nchunks = cdiv(n, ws.chunk);
  unsigned int* status = reinterpret_cast<unsigned int*>(b + kOffStatus);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  RLU_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(unsigned int), st));
  if ((rc = launch_twiddles(l1, ws.tw64, ws.tw32, st))) return rc;
  if ((rc = launch_sketch_params(ws, n, l1, l, seed, st))) return rc;
  if ((rc = launch_sketch_dense(A, lda, dtype, dtype == RLU_F64, m, n, l1, l, ws, Y, status, sms, st))) return rc;
  k_noalloc_status<<<1, 1, 0, st>>>(status, status_dev);
  RLU_CUDA_TRY(cudaGetLastError());
  note_launch();
  return RLU_OK;
}
