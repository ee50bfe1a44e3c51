// Arithmetic-rate probes for the roofline denominators (not part of the
// method): long chains of independent fused multiply-adds in FP64, FP32 and
// packed FP32 (fma.rn.f32x2, two lanes per instruction), timed with CUDA events
// on the caller's stream.  Every block runs the same chain; the result is
// written so that the compiler keeps the arithmetic.
#include "handle.h"

namespace ls {
namespace {

constexpr int kChains = 8;  // independent accumulators per thread

template <class T>
__global__ void __launch_bounds__(256) fma_loop_kernel(T* out, int iters, T a, T b) {
  T acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = (T)(threadIdx.x + c);
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = acc[c] * a + b;
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c];
  if (s == (T)-1.2345) out[blockIdx.x] = s;  // practically never taken; keeps the loop live
}

__global__ void __launch_bounds__(256) ffma2_loop_kernel(float* out, int iters, float a, float b) {
  unsigned long long acc[kChains];
  const unsigned long long pa = ((unsigned long long)__float_as_uint(a) << 32) | __float_as_uint(a);
  const unsigned long long pb = ((unsigned long long)__float_as_uint(b) << 32) | __float_as_uint(b);
#pragma unroll
  for (int c = 0; c < kChains; ++c)
    acc[c] = ((unsigned long long)__float_as_uint((float)(threadIdx.x + c)) << 32) |
             __float_as_uint((float)(threadIdx.x - c));
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int c = 0; c < kChains; ++c) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(acc[c]) : "l"(pa), "l"(pb));
  float s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += __uint_as_float((unsigned)acc[c]) + __uint_as_float((unsigned)(acc[c] >> 32));
  if (s == -1.2345f) out[blockIdx.x] = s;
}

}  // namespace
}  // namespace ls

extern "C" int ls_measure_peak(int kind, double* tflops, void* stream) {
  using namespace ls;
  if (!tflops || kind < 0 || kind > 2) return LS_EINVAL;
  *tflops = 0;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  LS_CUDA_TRY(cudaGetDevice(&dev));
  LS_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = nsm * 8, threads = 256;
  const int iters = kind == 0 ? 1 << 12 : 1 << 16;
  void* out = nullptr;
  StreamScope scope(st);
  int rc = dalloc(&out, sizeof(double) * blocks);
  if (rc) return rc;
  cudaEvent_t e0, e1;
  LS_CUDA_TRY(cudaEventCreate(&e0));
  LS_CUDA_TRY(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {  // the first launch warms up; the best of the rest counts
    LS_CUDA_TRY(cudaEventRecord(e0, st));
    count_launch();
    if (kind == 0)
      fma_loop_kernel<double><<<blocks, threads, 0, st>>>((double*)out, iters, 0.999999, 1e-7);
    else if (kind == 1)
      fma_loop_kernel<float><<<blocks, threads, 0, st>>>((float*)out, iters, 0.999999f, 1e-7f);
    else
      ffma2_loop_kernel<<<blocks, threads, 0, st>>>((float*)out, iters, 0.999999f, 1e-7f);
    LS_CUDA_TRY(cudaEventRecord(e1, st));
    LS_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0;
    LS_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    if (rep > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  dfree(out);
  const double fma = (double)blocks * threads * iters * kChains * (kind == 2 ? 2.0 : 1.0);
  *tflops = 2.0 * fma / (best * 1e-3) / 1e12;
  return LS_OK;
}
