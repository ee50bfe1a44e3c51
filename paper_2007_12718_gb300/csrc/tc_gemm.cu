// Complex FP32 GEMM on the Blackwell tensor cores (tcgen05.mma, kind::tf32,
// accumulators in tensor memory), for the merge products of the HBS build
// (Eqs. 26-27: S G, S G^T, Y2 Y1, the Schur-complement blocks, X diag(S) U,
// U^T (.), and the trailing updates of the blocked inverse).
//
// C = alpha op(A) op(B) + beta C with complex operands is computed from real
// products of the real and imaginary planes (the 4M form):
//   re(C) = Ar Br - Ai Bi,   im(C) = Ar Bi + Ai Br,
// accumulated in three FP32 accumulators in tensor memory (Ar Br, Ai Bi and
// the imaginary part), combined in the epilogue.  In tf32x3 mode every plane
// is split into a tf32 head and a tf32 tail, x = hi + lo (round to nearest),
// and each real product P Q is P_hi Q_hi + P_hi Q_lo + P_lo Q_hi (the lo lo
// term, ~2^-22 of |P||Q|, is dropped): twelve MMAs per k step instead of four.
//
// In f16x3 mode (the FP16 split product) the planes are FP16 instead, hi =
// fp16(s x), lo = fp16(s x - hi), with s = 2^e per operand chosen from the
// operand's largest magnitude (a pre-pass) so that s max|x| < 2^14: the
// exponent range of FP16 then costs nothing, and hi + lo carries 22 bits of x
// as tf32 hi + lo does; kind::f16 MMAs (k = 16 per instruction, twice the
// tf32 rate) accumulate in FP32 and the epilogue multiplies by 1 / (sA sB),
// exact powers of two.  A stage then holds 32 complex k in the same 64 KB.
//
// One CTA computes a 128 x 128 complex tile.  Eight converter warps read the
// FP32 operands straight from global memory (per thread one row of op(A) and
// one column of op(B), half of a stage's complex k: 16-byte loads where that
// run is contiguous, element loads coalesced across the warp where it is not;
// the next two stages' values (FP16: the next one) are loaded while the
// current ones are converted), split them and store the planes in the K-major no-swizzle layout
// of 8-row x 16-byte core matrices (a fence makes them visible to the tensor
// cores), then arrive on the stage's "full" mbarrier; one thread of the ninth
// warp issues the MMAs of a stage and commits them to its "empty" mbarrier.
// Three stages of 64 KB.  The converter warps then read the accumulators back
// with tcgen05.ld, combine them into a tile in shared memory and write C
// coalesced.  Every mbarrier wait is bounded: on timeout the
// block records LS_ETIMEOUT in *err, issues nothing more, frees its tensor
// memory and returns.
#include <string.h>

#include <algorithm>

#include <cuda_fp16.h>

#include "handle.h"

namespace ls {
namespace {

constexpr int TC_BM = 128;                     // rows of C per tile
constexpr int TC_BN = 128;                     // complex columns of C per tile
constexpr int TC_BK = 16;                      // complex k per stage (tf32; f16: twice as many)
constexpr int TC_PLANE = TC_BM * TC_BK;        // floats per real plane (8 KB)
constexpr int TC_STAGE = 8 * TC_PLANE;         // Ar hi/lo, Ai hi/lo, Br hi/lo, Bi hi/lo: 64 KB
constexpr int TC_NS = 3;                       // stages in flight
constexpr int TC_CONV = 256;                   // converter / epilogue threads (warps 0-7)
constexpr int TC_THREADS = TC_CONV + 32;       // + the MMA warp (warp 8)
template <bool F16>
struct TcK {
  static constexpr int BK = F16 ? 2 * TC_BK : TC_BK;  // complex k per stage
  static constexpr int KH = BK / 2;                   // complex k per converter thread and stage
};
constexpr int TC_KH_MAX = TcK<true>::KH;
constexpr uint32_t TC_TMEM_COLS = 512;         // three 128-column accumulators
constexpr long long kMbarSpin = 1LL << 26;

enum { P_AR_HI = 0, P_AR_LO, P_AI_HI, P_AI_LO, P_BR_HI, P_BR_LO, P_BI_HI, P_BI_LO };

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major no-swizzle layout of one 128 x 16 plane: core matrix = 8 rows x 16
// bytes (4 tf32); LBO = 128 B between K-adjacent core matrices, SBO = 512 B
// between row-adjacent groups of eight rows.
__device__ __forceinline__ int kmaj(int row, int k) { return (row >> 3) * (TC_BK * 8) + (k >> 2) * 32 + (row & 7) * 4 + (k & 3); }

__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // fixed 0b001 at bits 46-48; base offset 0; no swizzle
  return d;
}

// Instruction descriptor: D = F32, A = B = TF32, both K-major.
__host__ __device__ constexpr uint32_t make_idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// Instruction descriptor: D = F32, A = B = F16, both K-major.
__host__ __device__ constexpr uint32_t make_idesc_f16(int M, int N) {
  return (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// The same K-major no-swizzle layout for a 128 x 32 FP16 plane (in halves):
// core matrix = 8 rows x 16 bytes (8 halves); LBO 128 B, SBO 512 B as above.
__device__ __forceinline__ int kmaj16(int row, int k) {
  return (row >> 3) * (2 * TC_BK * 8) + (k >> 3) * 64 + (row & 7) * 8 + (k & 7);
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  long long spins = 0;
  while (!done) {
    asm volatile(
        "{\n.reg .pred P1;\nmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\nselp.b32 %0, 1, 0, P1;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (!done && ++spins > kMbarSpin) return false;
  }
  return true;
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
}

template <bool F16>
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t accum) {
  if constexpr (F16)
    mma_f16(tmem, ad, bd, idesc, accum);
  else
    mma_tf32(tmem, ad, bd, idesc, accum);
}

// The 16 complex values k = kb .. kb + 15 of one row, scaled by sc, as the four
// FP16 planes (re hi, re lo, im hi, im lo) starting at plane p0 (two 16-byte
// core-matrix rows per plane).
__device__ __forceinline__ void store_row16(float* stage, int p0, int row, int kb, const c32 (&v)[TC_KH_MAX], float sc) {
  __half* st = reinterpret_cast<__half*>(stage);
  constexpr int PH = 2 * TC_PLANE;  // halves per plane
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    __align__(16) __half rh[8], rl[8], ih[8], il[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const c32 x = v[8 * q + e];
      const float xr = x.re * sc, xi = x.im * sc;
      const __half hr = __float2half_rn(xr), hi = __float2half_rn(xi);
      rh[e] = hr;
      ih[e] = hi;
      rl[e] = __float2half_rn(xr - __half2float(hr));
      il[e] = __float2half_rn(xi - __half2float(hi));
    }
    const int o = kmaj16(row, kb + 8 * q);
    *reinterpret_cast<uint4*>(st + (p0 + 0) * PH + o) = *reinterpret_cast<const uint4*>(rh);
    *reinterpret_cast<uint4*>(st + (p0 + 1) * PH + o) = *reinterpret_cast<const uint4*>(rl);
    *reinterpret_cast<uint4*>(st + (p0 + 2) * PH + o) = *reinterpret_cast<const uint4*>(ih);
    *reinterpret_cast<uint4*>(st + (p0 + 3) * PH + o) = *reinterpret_cast<const uint4*>(il);
  }
}

// The FP16 operand scale 2^e with 2^e * mx < 2^14 (e = 0 for mx = 0 or not finite).
__device__ __forceinline__ int f16_scale_exp(unsigned bits) {
  const float mx = __uint_as_float(bits);
  if (!(mx > 0.f) || !(mx < 3.0e38f)) return 0;
  int e;
  frexpf(mx, &e);  // mx < 2^e
  return min(14 - e, 100);
}

// out[0] = max over the batch of max(|re|, |im|) of X (rows x cols, row stride
// ld, batch stride sX), as float bits (non-negative floats order as unsigned).
__global__ void absmax_kernel(const c32* __restrict__ X, int rows, int cols, int ld, long long sX, int batch,
                              unsigned* out) {
  const long long per = (long long)rows * cols, tot = per * batch;
  float m = 0.f;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const long long b = t / per, r = (t % per) / cols, c = t % cols;
    const c32 x = X[b * sX + r * ld + c];
    m = fmaxf(m, fmaxf(fabsf(x.re), fabsf(x.im)));
  }
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(out, __float_as_uint(m));
}

// Store the 8 complex values k = kb .. kb + 7 of one row as the four planes
// (re hi, re lo, im hi, im lo) starting at plane p0; without `split` only the
// heads are stored.
__device__ __forceinline__ void store_row(float* stage, int p0, int row, int kb, const c32 (&v)[TC_BK / 2], bool split) {
#pragma unroll
  for (int q = 0; q < TC_BK / 8; ++q) {
    float4 rh, rl, ih, il;
    float* prh = &rh.x;
    float* prl = &rl.x;
    float* pih = &ih.x;
    float* pil = &il.x;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const c32 x = v[4 * q + e];
      const float hr = to_tf32(x.re), hi = to_tf32(x.im);
      prh[e] = hr;
      pih[e] = hi;
      prl[e] = split ? to_tf32(x.re - hr) : 0.f;
      pil[e] = split ? to_tf32(x.im - hi) : 0.f;
    }
    const int o = kmaj(row, kb + 4 * q);
    *reinterpret_cast<float4*>(stage + (p0 + 0) * TC_PLANE + o) = rh;
    *reinterpret_cast<float4*>(stage + (p0 + 2) * TC_PLANE + o) = ih;
    if (split) {
      *reinterpret_cast<float4*>(stage + (p0 + 1) * TC_PLANE + o) = rl;
      *reinterpret_cast<float4*>(stage + (p0 + 3) * TC_PLANE + o) = il;
    }
  }
}

// C[b] (M x N complex) = alpha op(A[b]) op(B[b]) + beta C[b]; row-major
// complex64 operands, op = transpose (no conjugate) when TA / TB.  F16: the
// FP16 split product, amax = {max|A|, max|B|} (float bits) from absmax_kernel.
template <bool TA, bool TB, bool F16>
__global__ void __launch_bounds__(TC_THREADS) tc_gemm_kernel(int M, int N, int K, c32 alpha, const c32* __restrict__ A,
                                                             int lda, long long sA, const c32* __restrict__ B, int ldb,
                                                             long long sB, c32 beta, c32* __restrict__ C, int ldc,
                                                             long long sC, int split, int band_lo, int band_hi,
                                                             int* err, const unsigned* __restrict__ amax, int vec) {
  constexpr int BK = TcK<F16>::BK, KH = TcK<F16>::KH;
  extern __shared__ __align__(1024) unsigned char smraw[];
  float* stages = reinterpret_cast<float*>(smraw);  // TC_NS x TC_STAGE floats
  __shared__ __align__(8) uint64_t full_bar[TC_NS], empty_bar[TC_NS], done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n0 = blockIdx.x * TC_BN, m0 = blockIdx.y * TC_BM, bz = blockIdx.z;
  A += bz * sA;
  B += bz * sB;
  C += bz * sC;
  const int S = (K + BK - 1) / BK;
  const bool sp = F16 || split != 0;
  const int ea = F16 ? f16_scale_exp(amax[0]) : 0, eb = F16 ? f16_scale_exp(amax[1]) : 0;
  const float sa = ldexpf(1.f, ea), sb = ldexpf(1.f, eb);

  if (warp == 8) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < TC_NS; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full_bar[i])), "r"(TC_CONV));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty_bar[i])), "r"(1));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&done_bar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_fail = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;

  if (warp < 8) {  // converters: row r of op(A) and of op(B)^T, k-half kh of every stage
    const int r = tid & (TC_BM - 1), kh = (tid >> 7) * KH;
    const int ra = m0 + r, cb = n0 + r;
    // The KH complex k of stage s for row ra of op(A) and column cb of op(B).
    // Where that run is contiguous in memory (A not transposed, B transposed)
    // and 16-byte aligned (vec bit 0 / bit 1), it is read as KH / 2 16-byte
    // loads; otherwise element by element (coalesced across the warp).
    auto load = [&](int s, c32* xa, c32* xb) {
      const int k0 = s * BK + kh;
      const bool kfull = k0 + KH <= K;
      if (!TA && (vec & 1) && kfull) {
        const float4* p = reinterpret_cast<const float4*>(A + (long long)(ra < M ? ra : 0) * lda + k0);
#pragma unroll
        for (int j = 0; j < KH / 2; ++j) {
          const float4 t = ra < M ? __ldg(p + j) : make_float4(0.f, 0.f, 0.f, 0.f);
          xa[2 * j] = mk<float>(t.x, t.y);
          xa[2 * j + 1] = mk<float>(t.z, t.w);
        }
      } else {
#pragma unroll
        for (int j = 0; j < KH; ++j) {
          const int k = k0 + j;
          xa[j] = (ra < M && k < K) ? (TA ? A[(long long)k * lda + ra] : A[(long long)ra * lda + k]) : mk<float>(0.f, 0.f);
        }
      }
      if (TB && (vec & 2) && kfull) {
        const float4* p = reinterpret_cast<const float4*>(B + (long long)(cb < N ? cb : 0) * ldb + k0);
#pragma unroll
        for (int j = 0; j < KH / 2; ++j) {
          const float4 t = cb < N ? __ldg(p + j) : make_float4(0.f, 0.f, 0.f, 0.f);
          xb[2 * j] = mk<float>(t.x, t.y);
          xb[2 * j + 1] = mk<float>(t.z, t.w);
        }
      } else {
#pragma unroll
        for (int j = 0; j < KH; ++j) {
          const int k = k0 + j;
          xb[j] = (cb < N && k < K) ? (TB ? B[(long long)cb * ldb + k] : B[(long long)k * ldb + cb]) : mk<float>(0.f, 0.f);
        }
      }
    };
    // Stage s: wait until the MMAs have released its buffer, split and store
    // the operands, make them visible to the tensor cores and arrive.
    auto put = [&](int s, const c32* xa, const c32* xb) -> bool {
      const int bi = s % TC_NS;
      if (s >= TC_NS && !mbar_wait(smem_u32(&empty_bar[bi]), ((s / TC_NS) - 1) & 1)) {
        atomicExch(&s_fail, 1);
        return false;
      }
      if (*(volatile int*)&s_fail) return false;
      float* stage = stages + (size_t)bi * TC_STAGE;
      if constexpr (F16) {
        store_row16(stage, P_AR_HI, r, kh, *reinterpret_cast<const c32(*)[TC_KH_MAX]>(xa), sa);
        store_row16(stage, P_BR_HI, r, kh, *reinterpret_cast<const c32(*)[TC_KH_MAX]>(xb), sb);
      } else {
        store_row(stage, P_AR_HI, r, kh, *reinterpret_cast<const c32(*)[TC_BK / 2]>(xa), sp);
        store_row(stage, P_BR_HI, r, kh, *reinterpret_cast<const c32(*)[TC_BK / 2]>(xb), sp);
      }
      // generic-proxy stores -> visible to the tensor cores (async proxy)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full_bar[bi])) : "memory");
      return true;
    };
    if constexpr (F16) {  // one stage loaded ahead (KH = 16 complex per operand)
      c32 va[KH], vb[KH];
      load(0, va, vb);
      for (int s = 0; s < S; ++s) {
        if (!put(s, va, vb)) break;
        if (s + 1 < S) load(s + 1, va, vb);
      }
    } else {  // two stages loaded ahead, in two register sets
      c32 va0[KH], vb0[KH], va1[KH], vb1[KH];
      load(0, va0, vb0);
      if (S > 1) load(1, va1, vb1);
      for (int s = 0; s < S; s += 2) {
        if (!put(s, va0, vb0)) break;
        if (s + 2 < S) load(s + 2, va0, vb0);
        if (s + 1 >= S || !put(s + 1, va1, vb1)) break;
        if (s + 3 < S) load(s + 3, va1, vb1);
      }
    }
  } else if (lane == 0) {  // MMA issuer
    const uint32_t idesc = F16 ? make_idesc_f16(TC_BM, TC_BN) : make_idesc_tf32(TC_BM, TC_BN);
    const uint32_t acc_rr = tmem, acc_ii = tmem + 128, acc_im = tmem + 256;
    bool ok = true;
    for (int s = 0; s < S; ++s) {
      const int bi = s % TC_NS;
      if (!mbar_wait(smem_u32(&full_bar[bi]), (s / TC_NS) & 1) || *(volatile int*)&s_fail) {
        atomicExch(&s_fail, 1);
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t base = smem_u32(stages + (size_t)bi * TC_STAGE);
      // one MMA k step covers 32 bytes of each row (8 tf32 or 16 f16): two core matrices
      auto pd = [&](int plane, int kk) { return make_desc(base + plane * TC_PLANE * 4 + kk * 256, 128, TC_BK * 8 * 4); };
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        const uint32_t first = (s == 0 && kk == 0) ? 0u : 1u;
        // Ar Br
        mma<F16>(acc_rr, pd(P_AR_HI, kk), pd(P_BR_HI, kk), idesc, first);
        // Ai Bi
        mma<F16>(acc_ii, pd(P_AI_HI, kk), pd(P_BI_HI, kk), idesc, first);
        // Ar Bi + Ai Br
        mma<F16>(acc_im, pd(P_AR_HI, kk), pd(P_BI_HI, kk), idesc, first);
        mma<F16>(acc_im, pd(P_AI_HI, kk), pd(P_BR_HI, kk), idesc, 1u);
        if (sp) {
          mma<F16>(acc_rr, pd(P_AR_HI, kk), pd(P_BR_LO, kk), idesc, 1u);
          mma<F16>(acc_rr, pd(P_AR_LO, kk), pd(P_BR_HI, kk), idesc, 1u);
          mma<F16>(acc_ii, pd(P_AI_HI, kk), pd(P_BI_LO, kk), idesc, 1u);
          mma<F16>(acc_ii, pd(P_AI_LO, kk), pd(P_BI_HI, kk), idesc, 1u);
          mma<F16>(acc_im, pd(P_AR_HI, kk), pd(P_BI_LO, kk), idesc, 1u);
          mma<F16>(acc_im, pd(P_AR_LO, kk), pd(P_BI_HI, kk), idesc, 1u);
          mma<F16>(acc_im, pd(P_AI_HI, kk), pd(P_BR_LO, kk), idesc, 1u);
          mma<F16>(acc_im, pd(P_AI_LO, kk), pd(P_BR_HI, kk), idesc, 1u);
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&empty_bar[bi])));
    }
    if (ok)
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&done_bar)));
  }
  // the converter warps wait for the last MMA (or a failure), then the epilogue
  bool ok = true;
  if (warp < 8 && S > 0) {
    uint32_t done = 0;
    long long spins = 0;
    while (!done) {
      asm volatile(
          "{\n.reg .pred P1;\nmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\nselp.b32 %0, 1, 0, P1;\n}\n"
          : "=r"(done)
          : "r"(smem_u32(&done_bar)), "r"(0u)
          : "memory");
      if (done) break;
      if (*(volatile int*)&s_fail || ++spins > kMbarSpin) {
        ok = false;
        break;
      }
    }
  }
  if (!ok) atomicExch(&s_fail, 1);  // one decision for the whole block after the barrier
  asm volatile("tcgen05.fence::after_thread_sync;");
  __syncthreads();
  if (warp < 8) {
    // epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. (rows of the tile),
    // columns 64 (w / 4) .. of the three accumulators, and stores the combined
    // values in the stage buffers (free once the last MMA is done), rows padded
    // to 129 entries; then the 256 threads write C row by row, coalesced.
    if (*(volatile int*)&s_fail) {
      if (tid == 0) atomicExch(err, LS_ETIMEOUT);
    } else if (S > 0) {
      c32* tile = reinterpret_cast<c32*>(stages);  // 128 x 129 complex, 132 KB
      constexpr int TLD = TC_BN + 1;
      const int q = warp & 3, ch = warp >> 2;
      const int rl = q * 32 + lane;
#pragma unroll 1
      for (int c0 = ch * (TC_BN / 2); c0 < (ch + 1) * (TC_BN / 2); c0 += 16) {
        uint32_t vr[16], vi[16], vm[16];
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(vr[0]), "=r"(vr[1]), "=r"(vr[2]), "=r"(vr[3]), "=r"(vr[4]), "=r"(vr[5]), "=r"(vr[6]), "=r"(vr[7]),
              "=r"(vr[8]), "=r"(vr[9]), "=r"(vr[10]), "=r"(vr[11]), "=r"(vr[12]), "=r"(vr[13]), "=r"(vr[14]),
              "=r"(vr[15])
            : "r"(taddr));
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(vi[0]), "=r"(vi[1]), "=r"(vi[2]), "=r"(vi[3]), "=r"(vi[4]), "=r"(vi[5]), "=r"(vi[6]), "=r"(vi[7]),
              "=r"(vi[8]), "=r"(vi[9]), "=r"(vi[10]), "=r"(vi[11]), "=r"(vi[12]), "=r"(vi[13]), "=r"(vi[14]),
              "=r"(vi[15])
            : "r"(taddr + 128u));
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(vm[0]), "=r"(vm[1]), "=r"(vm[2]), "=r"(vm[3]), "=r"(vm[4]), "=r"(vm[5]), "=r"(vm[6]), "=r"(vm[7]),
              "=r"(vm[8]), "=r"(vm[9]), "=r"(vm[10]), "=r"(vm[11]), "=r"(vm[12]), "=r"(vm[13]), "=r"(vm[14]),
              "=r"(vm[15])
            : "r"(taddr + 256u));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
        for (int e = 0; e < 16; ++e)
          tile[rl * TLD + c0 + e] = mk<float>(__uint_as_float(vr[e]) - __uint_as_float(vi[e]), __uint_as_float(vm[e]));
      }
      asm volatile("bar.sync 1, %0;" ::"r"(TC_CONV) : "memory");  // the converter warps only
      const bool zb = (beta.re == 0.f && beta.im == 0.f);
      // the FP16 operand scales, undone exactly (powers of two)
      const c32 al = F16 ? mk<float>(ldexpf(alpha.re, -(ea + eb)), ldexpf(alpha.im, -(ea + eb))) : alpha;
      for (int e = tid; e < TC_BM * TC_BN; e += TC_CONV) {
        const int r = e / TC_BN, c = e % TC_BN, row = m0 + r, col = n0 + c;
        const bool band = (row >= band_lo && row < band_hi) || (col >= band_lo && col < band_hi);
        if (row < M && col < N && !band) {
          c32 out = al * tile[r * TLD + c];
          if (!zb) out = out + beta * C[(long long)row * ldc + col];
          C[(long long)row * ldc + col] = out;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 8) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
}

}  // namespace

template <bool TA, bool TB, bool F16>
int launch_tc(cudaStream_t st, int M, int N, int K, c32 alpha, const c32* A, int lda, long long sA, const c32* B,
              int ldb, long long sB, c32 beta, c32* C, int ldc, long long sC, int batch, int split, int* err,
              int band_lo, int band_hi, const unsigned* amax) {
  const size_t smem = sizeof(float) * (size_t)TC_NS * TC_STAGE;
  LS_CUDA_TRY(cudaFuncSetAttribute((const void*)tc_gemm_kernel<TA, TB, F16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
  dim3 grid((N + TC_BN - 1) / TC_BN, (M + TC_BM - 1) / TC_BM, batch);
  count_launch();
  // 16-byte row loads where a row of op(A) / column of op(B) is contiguous and
  // every such row of every batch entry starts on a 16-byte boundary
  auto al16 = [](const void* p) { return ((uintptr_t)p & 15u) == 0; };
  int vec = 0;
  if (!TA && al16(A) && lda % 2 == 0 && (sA % 2 == 0 || batch == 1)) vec |= 1;
  if (TB && al16(B) && ldb % 2 == 0 && (sB % 2 == 0 || batch == 1)) vec |= 2;
  tc_gemm_kernel<TA, TB, F16><<<grid, TC_THREADS, smem, st>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC,
                                                              split, band_lo, band_hi, err, amax, vec);
  return check_launch("tc_cgemm");
}

// Host entry: same contract as the SIMT gemm (batched, row-major, op N/T, a
// stride of 0 shares an operand across the batch).  split: 0 tf32, 1 tf32x3,
// 2 f16x3 (the FP16 split product: a max-abs pre-pass over A and B, on st).
// Entries in rows or columns [band_lo, band_hi) of C are left untouched.
int tc_cgemm(cudaStream_t st, bool ta, bool tb, int M, int N, int K, c32 alpha, const c32* A, int lda, long long sA,
             const c32* B, int ldb, long long sB, c32 beta, c32* C, int ldc, long long sC, int batch, int split,
             int* err, int band_lo, int band_hi) {
  if (M <= 0 || N <= 0 || batch <= 0 || K <= 0) return LS_OK;
  if (batch > 65535) {  // the batch is the grid's z dimension
    for (int b0 = 0; b0 < batch; b0 += 65535) {
      int rc = tc_cgemm(st, ta, tb, M, N, K, alpha, A + b0 * sA, lda, sA, B + b0 * sB, ldb, sB, beta, C + b0 * sC, ldc,
                        sC, std::min(65535, batch - b0), split, err, band_lo, band_hi);
      if (rc) return rc;
    }
    return LS_OK;
  }
  int rc;
  if (split == 2) {
    StreamScope scope(st);  // the two maxima live on st
    unsigned* amax = nullptr;
    if ((rc = dalloc((void**)&amax, 2 * sizeof(unsigned)))) return rc;
    LS_CUDA_TRY(cudaMemsetAsync(amax, 0, 2 * sizeof(unsigned), st));
    // stored shapes: op(A) is M x K (A stored K x M when transposed), op(B) K x N
    const int ar = ta ? K : M, ac = ta ? M : K, br = tb ? N : K, bc = tb ? K : N;
    const int nbA = (int)std::min<long long>(1024, ((long long)ar * ac * (sA ? batch : 1) + 255) / 256);
    const int nbB = (int)std::min<long long>(1024, ((long long)br * bc * (sB ? batch : 1) + 255) / 256);
    count_launch(2);
    absmax_kernel<<<nbA, 256, 0, st>>>(A, ar, ac, lda, sA, sA ? batch : 1, amax);
    absmax_kernel<<<nbB, 256, 0, st>>>(B, br, bc, ldb, sB, sB ? batch : 1, amax + 1);
    if (!ta && !tb)
      rc = launch_tc<false, false, true>(st, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch, split,
                                         err, band_lo, band_hi, amax);
    else if (ta && !tb)
      rc = launch_tc<true, false, true>(st, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch, split,
                                        err, band_lo, band_hi, amax);
    else if (!ta && tb)
      rc = launch_tc<false, true, true>(st, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch, split,
                                        err, band_lo, band_hi, amax);
    else
      rc = launch_tc<true, true, true>(st, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch, split, err,
                                       band_lo, band_hi, amax);
    dfree(amax);
    return rc;
  }
  if (!ta && !tb)
    return launch_tc<false, false, false>(st, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch, split,
                                          err, band_lo, band_hi, nullptr);
  if (ta && !tb)
    return launch_tc<true, false, false>(st, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch, split,
                                         err, band_lo, band_hi, nullptr);
  if (!ta && tb)
    return launch_tc<false, true, false>(st, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch, split,
                                         err, band_lo, band_hi, nullptr);
  return launch_tc<true, true, false>(st, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch, split, err,
                                      band_lo, band_hi, nullptr);
}

}  // namespace ls
