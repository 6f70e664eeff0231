// Two measurement and test hooks that run no step of the factorization.
//
// rlu_debug_alu_peak: the FP64 or FP32 fused multiply-add throughput of this
// GPU, measured by a kernel of independent FMA chains on every SM (the peak
// that the ALU-bound kernels of the path are reported against).
//
// rlu_debug_wait_timeout: run one of the library's bounded device waits on a
// condition that never comes true, so that a test can see the wait give up,
// raise FLAG_TIMEOUT, and leave the context usable.
//
//   which = 0: the grid barrier of the cooperative kernels (the pivoted LUs,
//              the Cholesky factor).  Two co-resident CTAs each arrive once,
//              then wait for a second arrival that no CTA makes.
//   which = 1: the mbarrier wait of the tensor-core pipeline.  One thread
//              waits for the first phase of a barrier that nothing arrives at.
//
// Both waits are the production helpers (grid_arrive/grid_wait from
// common.cuh, tc::mbar_wait from gemm_tc.cuh) with their production limit of
// about a second; nothing here faults, traps or waits without a bound.
#include "common.cuh"
#include "gemm_tc.cuh"

namespace rlu {
namespace {

__global__ void k_wait_grid_never(unsigned int* counter, unsigned int* status) {
  grid_arrive(counter);
  grid_wait(counter, 2u, status);  // only one arrival per CTA is ever made
}

__global__ void k_wait_mbar_never(unsigned int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !tc::mbar_wait(&bar, 0)) set_flag(status, FLAG_TIMEOUT);
}

// Eight independent FMA chains per thread, `iters` rounds: 8 * iters FMAs per
// thread.  The multiplier is just below one and the addend small, so values
// stay finite; the sum is stored so that no chain can be dropped.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, T x, T y, T* out) {
  T a[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) a[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = fma(a[c], x, y);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += a[c];
  out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

template <typename T>
int fma_peak(int iters, double* tflops) {
  int dev = 0, sms = 0;
  RLU_CUDA_TRY(cudaGetDevice(&dev));
  RLU_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256;  // 2048 threads per SM
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * blocks * threads) != cudaSuccess) {
    cudaGetLastError();
    return RLU_ENOMEM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = RLU_OK;
  float best = 1e30f;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = RLU_ECUDA;
  for (int rep = 0; rep < 4 && !rc; ++rep) {  // the first launch warms up; the best of the rest counts
    cudaEventRecord(e0, 0);
    k_fma_chains<T><<<blocks, threads>>>(iters, (T)0.999999, (T)1e-3, out);
    cudaEventRecord(e1, 0);
    note_launch();
    float ms = 0.f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      rc = RLU_ECUDA;
      break;
    }
    if (rep > 0 && ms < best) best = ms;
  }
  if (!rc) *tflops = 2.0 * 8.0 * (double)iters * blocks * threads / (best * 1e-3) / 1e12;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  cudaGetLastError();
  return rc;
}

}  // namespace
}  // namespace rlu

extern "C" int rlu_debug_alu_peak(int which, double* tflops) {
  using namespace rlu;
  if (!tflops || which < 0 || which > 1) return RLU_EINVAL;
  *tflops = 0.0;
  // about 20 ms per launch at the expected rates (FP64 ~1.2, FP32 ~80 TFLOP/s)
  return which == 0 ? fma_peak<double>(4096, tflops) : fma_peak<float>(262144, tflops);
}

extern "C" int rlu_debug_wait_timeout(int which, int* status) {
  using namespace rlu;
  if (!status || which < 0 || which > 1) return RLU_EINVAL;
  unsigned int* d = nullptr;
  if (cudaMalloc(&d, 2 * sizeof(unsigned int)) != cudaSuccess) {
    cudaGetLastError();
    return RLU_ENOMEM;
  }
  int rc = RLU_OK;
  if (cudaMemset(d, 0, 2 * sizeof(unsigned int)) != cudaSuccess) rc = RLU_ECUDA;
  if (!rc) {
    cudaError_t e;
    if (which == 0) {
      unsigned int* counter = d;
      unsigned int* st = d + 1;
      void* args[] = {&counter, &st};
      e = launch_cooperative((const void*)k_wait_grid_never, dim3(2), dim3(32), args, 0, 0);
    } else {
      k_wait_mbar_never<<<1, 32>>>(d + 1);
      e = cudaGetLastError();
    }
    note_launch();
    unsigned int flags = 0;
    if (e != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(&flags, d + 1, sizeof(unsigned int), cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = RLU_ECUDA;
    else
      *status = status_of_flags(flags);
  }
  cudaFree(d);
  cudaGetLastError();
  return rc;
}
