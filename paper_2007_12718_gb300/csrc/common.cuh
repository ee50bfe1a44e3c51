// Shared device/host helpers for the Lippmann-Schwinger HBS library:
// complex arithmetic templated on the real type, error codes, a bounded
// grid barrier for cooperative kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#include "../../include/ls.h"

namespace ls {

template <class R>
struct __align__(2 * sizeof(R)) cx {
  R re, im;
};

typedef cx<double> z64;  // complex128
typedef cx<float> c32;   // complex64

__host__ __device__ __forceinline__ float mad(float a, float b, float c) { return fmaf(a, b, c); }
__host__ __device__ __forceinline__ double mad(double a, double b, double c) { return ::fma(a, b, c); }

template <class R>
__host__ __device__ __forceinline__ cx<R> mk(R a, R b) {
  cx<R> z;
  z.re = a;
  z.im = b;
  return z;
}
template <class R>
__host__ __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return mk<R>(a.re + b.re, a.im + b.im); }
template <class R>
__host__ __device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return mk<R>(a.re - b.re, a.im - b.im); }
template <class R>
__host__ __device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
  return mk<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <class R>
__host__ __device__ __forceinline__ cx<R> scale(cx<R> a, R s) { return mk<R>(a.re * s, a.im * s); }
template <class R>
__host__ __device__ __forceinline__ cx<R> conjz(cx<R> a) { return mk<R>(a.re, -a.im); }
// acc += a * b
template <class R>
__host__ __device__ __forceinline__ void fma_(cx<R>& acc, cx<R> a, cx<R> b) {
  acc.re = mad(a.re, b.re, mad(-a.im, b.im, acc.re));
  acc.im = mad(a.re, b.im, mad(a.im, b.re, acc.im));
}
// acc += conj(a) * b
template <class R>
__host__ __device__ __forceinline__ void fmac_(cx<R>& acc, cx<R> a, cx<R> b) {
  acc.re = mad(a.re, b.re, mad(a.im, b.im, acc.re));
  acc.im = mad(a.re, b.im, mad(-a.im, b.re, acc.im));
}
template <class R>
__host__ __device__ __forceinline__ R abs2(cx<R> a) { return a.re * a.re + a.im * a.im; }
template <class R>
__host__ __device__ __forceinline__ cx<R> inv(cx<R> a) {
  R d = R(1) / abs2(a);
  return mk<R>(a.re * d, -a.im * d);
}
template <class Ro, class Ri>
__host__ __device__ __forceinline__ cx<Ro> cvt(cx<Ri> a) { return mk<Ro>((Ro)a.re, (Ro)a.im); }

template <class R>
__device__ __forceinline__ cx<R> shfl_xor(cx<R> v, int m) {
  return mk<R>(__shfl_xor_sync(0xffffffffu, v.re, m), __shfl_xor_sync(0xffffffffu, v.im, m));
}
template <class R>
__device__ __forceinline__ cx<R> warp_sum(cx<R> v) {
  for (int m = 16; m; m >>= 1) v = v + shfl_xor(v, m);
  return v;
}
template <class T>
__device__ __forceinline__ T warp_sum_r(T v) {
  for (int m = 16; m; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}

// Loads that bypass L1 (data written by other blocks of the same grid).
template <class R>
__device__ __forceinline__ cx<R> ldcg_cx(const cx<R>* p);
template <>
__device__ __forceinline__ cx<float> ldcg_cx(const cx<float>* p) {
  float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return mk<float>(v.x, v.y);
}
template <>
__device__ __forceinline__ cx<double> ldcg_cx(const cx<double>* p) {
  double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return mk<double>(v.x, v.y);
}

// Grid-wide barrier for kernels launched with cudaLaunchCooperativeKernel
// (all blocks co-resident).  The arrival counter only grows: barrier number
// e (counted per block from 1) completes when it reaches e * nblocks.  Every
// spin is bounded: after `limit` polls the block raises *abort and the
// barrier returns false; every later barrier returns false at once, so the
// kernel unwinds without hanging.  count and abort must be zero at launch.
struct GridSync {
  unsigned int* count;   // arrival counter
  unsigned int* gen;     // unused (kept for layout)
  int* abort;            // set to 1 by a block that timed out
  long long limit;       // polls before giving up (ls_opts.wait_limit, default kSpinLimit)
};

static constexpr long long kSpinLimit = 20000000LL;  // ~ a second of polling

// Host side: the poll limit of the device waits launched by the calling thread
// (set from ls_opts.wait_limit for the duration of an entry point).
long long spin_limit();
struct SpinLimitScope {
  long long prev;
  explicit SpinLimitScope(long long limit);
  ~SpinLimitScope();
};

__device__ __forceinline__ bool grid_sync(const GridSync& g, unsigned int nblocks, unsigned int& epoch) {
  __shared__ int ok;
  __syncthreads();
  ++epoch;
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned int* vc = g.count;
    volatile int* vab = g.abort;
    __threadfence();
    atomicAdd(g.count, 1u);
    const unsigned int target = epoch * nblocks;
    long long spins = 0;
    while ((int)(*vc - target) < 0) {
      if (*vab) { ok = 0; break; }
      if (++spins >= g.limit) { atomicExch(g.abort, 1); ok = 0; break; }
    }
    __threadfence();
    if (*vab) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

// Counter of kernel launches made by this library (reported by ls_kernel_launches).
// With the environment variable LS_DEBUG_SYNC=1 every counted launch site first
// synchronizes the device and reports (stderr) the first device error together
// with the previous launch site, which localises an asynchronous fault.
struct LaunchCount {
  long long n = 1;
  LaunchCount() {}
  LaunchCount(long long v) : n(v) {}
};
void count_launch_at(const char* file, int line, LaunchCount c);
#define count_launch(...) ::ls::count_launch_at(__FILE__, __LINE__, ::ls::LaunchCount{__VA_ARGS__})
// Suppresses the debug synchronisation while a stream is being captured.
struct CaptureScope {
  CaptureScope();
  ~CaptureScope();
};

}  // namespace ls

#define LS_CUDA_TRY(expr)                                   \
  do {                                                      \
    cudaError_t _e = (expr);                                \
    if (_e != cudaSuccess) {                                \
      ls_set_last_cuda_error(_e, #expr, __FILE__, __LINE__); \
      return LS_ECUDA;                                      \
    }                                                       \
  } while (0)

void ls_set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line);
