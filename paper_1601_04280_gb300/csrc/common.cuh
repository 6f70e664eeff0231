// Shared device helpers of the sparse randomized LU library (sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "../../include/rlu.h"

namespace rlu {

// ---------------------------------------------------------------------------
// Device status word: bits set by kernels, read once by the host at the end.
// ---------------------------------------------------------------------------
enum : unsigned int {
  FLAG_TIMEOUT = 1u << 0,    // a bounded device wait gave up
  FLAG_NONFINITE = 1u << 1,  // NaN or Inf met in the input
  FLAG_ZERO_PIVOT = 1u << 2, // an exactly zero pivot column / row was met
  FLAG_BAD_CSR = 1u << 3,    // CSR structure invalid (row pointers or column range)
};

// Status code of a set of flag bits, in order of severity: a timed-out wait
// leaves outputs unwritten, so it outranks everything; then a malformed CSR,
// a non-finite input, and last the rank warning.  The one mapping used by the
// host read-back and by every kernel that writes a status code to the device.
__host__ __device__ __forceinline__ int status_of_flags(unsigned int f) {
  if (f & FLAG_TIMEOUT) return RLU_ETIMEOUT;
  if (f & FLAG_BAD_CSR) return RLU_EBADCSR;
  if (f & FLAG_NONFINITE) return RLU_ENONFINITE;
  if (f & FLAG_ZERO_PIVOT) return RLU_WRANK;
  return RLU_OK;
}

// Spin limit for every device wait: about a second at GB300 clocks.
constexpr long long kSpinLimitCycles = 2000000000ll;
// A spinning grid barrier also reads the status word (to leave once another
// block has timed out) on one poll in 16 (mask 15), so its polls of the
// awaited counter are one L2 round trip apart rather than two.
constexpr unsigned int kStatusPollEvery = 15u;

__device__ __forceinline__ void set_flag(unsigned int* status, unsigned int bit) {
  atomicOr(status, bit);
}

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_gpu_add(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier for cooperative (co-resident) launches.  Arrival is a
// release reduction by one thread after a CTA barrier (release is cumulative:
// writes of the other threads, ordered before it by the CTA barrier, become
// visible to every thread that acquires the counter), so no separate full fence
// is needed.  `counter` starts
// at zero for the launch; barrier number e (1, 2, ...) waits until all
// gridDim.x blocks have arrived e times.  The wait is bounded: on timeout it
// sets FLAG_TIMEOUT and returns false, and the caller must leave the kernel.
// Once any block has timed out, every later barrier returns false within 16
// polls.
__device__ __forceinline__ bool grid_barrier(unsigned int* counter, unsigned int epoch,
                                             unsigned int* status) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    red_release_gpu_add(counter, 1u);  // release: the CTA's writes before the __syncthreads come with it
    const unsigned int target = epoch * gridDim.x;
    long long t0 = clock64();
    int ok = 1;
    for (unsigned int it = 0;; ++it) {
      unsigned int v = ld_acquire_gpu(counter);
      if ((int)(v - target) >= 0) break;
      if ((it & kStatusPollEvery) == kStatusPollEvery && (ld_acquire_gpu(status) & FLAG_TIMEOUT)) { ok = 0; break; }
      if (clock64() - t0 > kSpinLimitCycles) {
        set_flag(status, FLAG_TIMEOUT);
        ok = 0;
        break;
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Split form of the same barrier: grid_arrive publishes this block's arrival
// (after every thread's prior writes); grid_wait(e) returns once all blocks
// have arrived e times, or false after the bounded wait (FLAG_TIMEOUT).
__device__ __forceinline__ void grid_arrive(unsigned int* counter) {
  __syncthreads();
  if (threadIdx.x == 0) red_release_gpu_add(counter, 1u);
}

__device__ __forceinline__ bool grid_wait(unsigned int* counter, unsigned int epoch, unsigned int* status) {
  __shared__ int s_ok2;
  if (threadIdx.x == 0) {
    const unsigned int target = epoch * gridDim.x;
    long long t0 = clock64();
    int ok = 1;
    for (unsigned int it = 0;; ++it) {
      unsigned int v = ld_acquire_gpu(counter);
      if ((int)(v - target) >= 0) break;
      if ((it & kStatusPollEvery) == kStatusPollEvery && (ld_acquire_gpu(status) & FLAG_TIMEOUT)) { ok = 0; break; }
      if (clock64() - t0 > kSpinLimitCycles) {
        set_flag(status, FLAG_TIMEOUT);
        ok = 0;
        break;
      }
    }
    s_ok2 = ok;
  }
  __syncthreads();
  return s_ok2 != 0;
}

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from its
// published definition: per round, two 64x64->128 products of counter words
// 0 and 2 with the multipliers, xor-mixed with words 1 and 3 and the key;
// the key is bumped by two Weyl constants between rounds.
// ---------------------------------------------------------------------------
struct Philox4 {
  uint64_t w[4];
};

__host__ __device__ __forceinline__ void mul64_wide(uint64_t a, uint64_t b, uint64_t& hi, uint64_t& lo) {
#ifdef __CUDA_ARCH__
  lo = a * b;
  hi = __umul64hi(a, b);
#else
  unsigned __int128 p = (unsigned __int128)a * b;
  lo = (uint64_t)p;
  hi = (uint64_t)(p >> 64);
#endif
}

__host__ __device__ __forceinline__ Philox4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                                          uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t hi0, lo0, hi1, lo1;
    mul64_wide(M0, c0, hi0, lo0);
    mul64_wide(M1, c2, hi1, lo1);
    uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  Philox4 o;
  o.w[0] = c0; o.w[1] = c1; o.w[2] = c2; o.w[3] = c3;
  return o;
}

// Second key word of every stream of the method: "RANDLU" in ASCII.
constexpr uint64_t kKeyTag = 0x52414E444C5500ull;

// ---------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T abs_(T x) { return x < T(0) ? -x : x; }

template <typename T> __device__ __forceinline__ double to_double(T x) { return (double)x; }
template <> __device__ __forceinline__ double to_double<__nv_bfloat16>(__nv_bfloat16 x) {
  return (double)__bfloat162float(x);
}
template <typename T> __device__ __forceinline__ float to_float(T x) { return (float)x; }
template <> __device__ __forceinline__ float to_float<__nv_bfloat16>(__nv_bfloat16 x) {
  return __bfloat162float(x);
}

template <typename T> __device__ __forceinline__ bool finite_(T x) { return isfinite(to_float(x)); }
template <> __device__ __forceinline__ bool finite_<double>(double x) { return isfinite(x); }

// ---------------------------------------------------------------------------
// Float-float ("double-single") numbers: value = hi + lo with |lo| <= ulp(hi)/2,
// about 48 significant bits on the FP32 pipes.  Built from the error-free
// transformations of Knuth (TwoSum), Dekker/Fast2Sum and the FMA-based TwoProd
// (Dekker 1971; Hida, Li and Bailey, "Algorithms for quad-double precision
// floating point arithmetic", 2001).
// ---------------------------------------------------------------------------
struct __align__(8) df32 {
  float hi, lo;
};

__device__ __forceinline__ df32 df_make(float hi, float lo) { df32 r; r.hi = hi; r.lo = lo; return r; }

// s + e = a + b exactly (Knuth TwoSum)
__device__ __forceinline__ df32 two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df_make(s, e);
}
// s + e = a + b exactly when |a| >= |b| (Fast2Sum)
__device__ __forceinline__ df32 quick_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return df_make(s, e);
}
__device__ __forceinline__ df32 operator+(df32 a, df32 b) {
  df32 s = two_sum(a.hi, b.hi);
  float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return quick_two_sum(s.hi, e);
}
__device__ __forceinline__ df32 operator-(df32 a) { return df_make(-a.hi, -a.lo); }
__device__ __forceinline__ df32 operator-(df32 a, df32 b) { return a + (-b); }
__device__ __forceinline__ df32 operator*(df32 a, df32 b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return quick_two_sum(p, e);
}
__device__ __forceinline__ df32 operator/(df32 a, df32 b) {
  float q1 = __fdiv_rn(a.hi, b.hi);
  df32 r = a - b * df_make(q1, 0.f);
  float q2 = __fdiv_rn(r.hi, b.hi);
  return quick_two_sum(q1, q2);
}
// c + a * b, one name for every arithmetic type of the templated kernels
__device__ __forceinline__ df32 mad(df32 a, df32 b, df32 c) { return c + a * b; }
__device__ __forceinline__ float mad(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double mad(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ bool operator!=(df32 a, df32 b) { return a.hi != b.hi || a.lo != b.lo; }
__device__ __forceinline__ bool operator==(df32 a, df32 b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ df32 df_from_double(double x) {
  float hi = __double2float_rn(x);
  return df_make(hi, __double2float_rn(x - (double)hi));
}
__device__ __forceinline__ df32 abs_(df32 x) { return x.hi < 0.f ? -x : x; }
template <> __device__ __forceinline__ double to_double<df32>(df32 x) { return (double)x.hi + (double)x.lo; }
template <> __device__ __forceinline__ float to_float<df32>(df32 x) { return x.hi; }

// Conversions used by templated kernels: cvt<To>(from)
template <typename To> struct Cvt;
template <> struct Cvt<double> {
  template <typename F> __device__ static double f(F x) { return to_double(x); }
};
template <> struct Cvt<float> {
  template <typename F> __device__ static float f(F x) { return to_float(x); }
};
template <> struct Cvt<df32> {
  __device__ static df32 f(double x) { return df_from_double(x); }
  __device__ static df32 f(float x) { return df_make(x, 0.f); }
  __device__ static df32 f(__nv_bfloat16 x) { return df_make(__bfloat162float(x), 0.f); }
  __device__ static df32 f(df32 x) { return x; }
};
template <typename To, typename F> __device__ __forceinline__ To cvt(F x) { return Cvt<To>::f(x); }
template <typename T> __device__ __forceinline__ T zero_() { return cvt<T>(0.0); }
template <typename T> __device__ __forceinline__ T one_() { return cvt<T>(1.0); }

// Reciprocal of a positive FP64 value by Newton's iteration r <- r (2 - x r)
// (written as r + r (1 - x r)), seeded by the FP32 hardware reciprocal
// approximation: two steps take the seed's ~2^-22 relative error to below
// 2^-52, with four dependent FMAs instead of a full-precision division on a
// latency-bound chain.  Outside the FP32 exponent range it falls back to the
// division.
__device__ __forceinline__ double rcp_newton(double x) {
  if (!(x > 1e-30 && x < 1e30)) return 1.0 / x;
  float s;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"((float)x));
  double r = (double)s;
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

// Process-wide count of kernels this library has launched (a test hook).
void note_launch(int count = 1);

// Cooperative launch of a kernel with grid barriers (all CTAs co-resident).
cudaError_t launch_cooperative(const void* func, dim3 grid, dim3 block, void** args, size_t smem, cudaStream_t st);

// Lift a kernel's dynamic shared-memory limit to the most the device allows
// beside its static shared memory.  Every call sets the same value, so a
// launch on one thread never finds the limit lowered by another thread that
// launches the same kernel with less.  RLU_EINVAL when `smem` is above it.
int allow_dynamic_smem(const void* kern, size_t smem);

__host__ __device__ __forceinline__ int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

}  // namespace rlu

#define RLU_CUDA_TRY(expr)                         \
  do {                                             \
    cudaError_t _e = (expr);                       \
    if (_e != cudaSuccess) {                       \
      cudaGetLastError();                          \
      return RLU_ECUDA;                            \
    }                                              \
  } while (0)
