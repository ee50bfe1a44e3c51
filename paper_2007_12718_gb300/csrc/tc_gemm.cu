// Complex FP32 GEMM on the Blackwell tensor cores (tcgen05.mma, kind::tf32,
// accumulators in tensor memory), for the merge products of the HBS build
// (Eqs. 26-27: S G, S G^T, Y2 Y1, the Schur-complement blocks, X diag(S) U,
// U^T (.), and the trailing updates of the blocked inverse).
//
// A complex product is one real product of twice the size: with A stored
// interleaved (re, im), row i of A is the real row (a_r0, a_i0, a_r1, a_i1, ..)
// of length 2K, and every complex entry b = (br, bi) of B becomes the 2x2 real
// block [[br, bi], [-bi, br]] of a 2K x 2N real matrix B'.  Then A' B' is C
// interleaved.  In tf32x3 mode each operand is split into a tf32 head and a
// tf32 tail (x = hi + lo) and the K loop runs over [A_hi A_hi A_lo] x
// [B_hi; B_lo; B_hi], which restores ~FP32 accuracy (the lo*lo term is
// dropped).
//
// Tile: 128 (M) x 128 (real N = 64 complex columns) per block, K staged 32
// real (16 complex) at a time through shared memory in the K-major
// no-swizzle layout of 8-row x 16-byte core matrices; one elected thread
// issues four m128n128k8 MMAs per stage and commits them to an mbarrier; the
// accumulator (128 lanes x 128 columns of FP32) is read back with tcgen05.ld.
// Every mbarrier wait is bounded: on timeout the block sets *err, still frees
// its tensor memory and returns.
#include <string.h>

#include <algorithm>

#include "handle.h"

namespace ls {
namespace {

constexpr int TC_BM = 128;   // rows per tile
constexpr int TC_BN = 128;   // real columns per tile (64 complex)
constexpr int TC_BK = 32;    // real K per stage (16 complex)
constexpr int TC_THREADS = 128;
constexpr long long kMbarSpin = 1LL << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// K-major, no swizzle: core matrix = 8 rows x 16 bytes (4 tf32), contiguous.
// LBO = byte distance between core matrices adjacent in K, SBO = between
// core matrices adjacent in M/N.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // fixed 0b001 at bits 46-48
  // base offset 0, relative LBO, swizzle mode 0 (none)
  return d;
}

// Instruction descriptor: D = F32, A = B = TF32, both K-major, M = 128, N = 128.
__host__ __device__ constexpr uint32_t make_idesc_tf32(int M, int N) {
  return (1u << 4)                 // D format F32
         | (2u << 7)               // A format TF32
         | (2u << 10)              // B format TF32
         | ((uint32_t)(N >> 3) << 17)
         | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm volatile("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// offset (in floats) of element (row, k) in a K-major no-swizzle tile of BK columns
__device__ __forceinline__ int kmaj(int row, int k) {
  return (row >> 3) * (TC_BK * 8) + (k >> 2) * 32 + (row & 7) * 4 + (k & 3);
}

// C[b] = alpha op(A[b]) op(B[b]) + beta C[b] for complex FP32 (interleaved),
// row-major, op = N or T.  split: 0 = plain tf32, 1 = tf32x3.
template <bool TA, bool TB>
__global__ void __launch_bounds__(TC_THREADS) tc_cgemm_kernel(int M, int N, int K, c32 alpha, const c32* __restrict__ A,
                                                              int lda, long long sA, const c32* __restrict__ B,
                                                              int ldb, long long sB, c32 beta, c32* __restrict__ C,
                                                              int ldc, long long sC, int split, int* err) {
  __shared__ __align__(1024) float sa[TC_BM * TC_BK];  // 16 KB
  __shared__ __align__(1024) float sb[TC_BN * TC_BK];  // 16 KB
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int bz = blockIdx.z;
  A += bz * sA;
  B += bz * sB;
  C += bz * sC;
  const int m0 = blockIdx.y * TC_BM;   // complex rows
  const int n0 = blockIdx.x * (TC_BN / 2);  // complex columns

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(TC_BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_fail = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = make_idesc_tf32(TC_BM, TC_BN);

  // K stages: real K' = 2K (interleaved), times 3 in split mode
  const int Kr = 2 * K;
  const int nparts = split ? 3 : 1;
  const int stages_per_part = (Kr + TC_BK - 1) / TC_BK;
  const int nstages = stages_per_part * nparts;
  uint32_t phase = 0;
  bool ok = true;
  for (int s = 0; s < nstages && ok; ++s) {
    const int part = s / stages_per_part;        // 0: hi*hi, 1: hi*lo, 2: lo*hi
    const int kr0 = (s % stages_per_part) * TC_BK;  // real k offset
    const bool a_lo = split && part == 2, b_lo = split && part == 1;
    // A tile: 128 rows x 32 real k (16 complex)
    for (int t = tid; t < TC_BM * (TC_BK / 2); t += TC_THREADS) {
      int r, kc;
      if (TA) {  // A stored K x M: consecutive threads along M
        r = t % TC_BM;
        kc = t / TC_BM;
      } else {   // A stored M x K: consecutive threads along K
        kc = t % (TC_BK / 2);
        r = t / (TC_BK / 2);
      }
      const int gi = m0 + r, gk = kr0 / 2 + kc;
      c32 v = mk<float>(0.f, 0.f);
      if (gi < M && gk < K) v = TA ? A[(long long)gk * lda + gi] : A[(long long)gi * lda + gk];
      float hr = to_tf32(v.re), hi = to_tf32(v.im);
      if (a_lo) {
        hr = to_tf32(v.re - hr);
        hi = to_tf32(v.im - hi);
      }
      sa[kmaj(r, 2 * kc)] = hr;
      sa[kmaj(r, 2 * kc + 1)] = hi;
    }
    // B tile: 128 real columns (64 complex) x 32 real k: entry (k=2q+e, n=2j+f) from b_qj
    for (int t = tid; t < (TC_BN / 2) * (TC_BK / 2); t += TC_THREADS) {
      int j, q;
      if (TB) {  // B stored N x K: consecutive threads along K
        q = t % (TC_BK / 2);
        j = t / (TC_BK / 2);
      } else {   // B stored K x N: consecutive threads along N
        j = t % (TC_BN / 2);
        q = t / (TC_BN / 2);
      }
      const int gj = n0 + j, gq = kr0 / 2 + q;
      c32 v = mk<float>(0.f, 0.f);
      if (gj < N && gq < K) v = TB ? B[(long long)gj * ldb + gq] : B[(long long)gq * ldb + gj];
      float br = to_tf32(v.re), bi = to_tf32(v.im);
      if (b_lo) {
        br = to_tf32(v.re - br);
        bi = to_tf32(v.im - bi);
      }
      // real B' rows (k) 2q, 2q+1; columns (n) 2j, 2j+1:  [[br, bi], [-bi, br]]
      sb[kmaj(2 * j, 2 * q)] = br;
      sb[kmaj(2 * j, 2 * q + 1)] = -bi;
      sb[kmaj(2 * j + 1, 2 * q)] = bi;
      sb[kmaj(2 * j + 1, 2 * q + 1)] = br;
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a0 = smem_u32(sa), b0 = smem_u32(sb);
#pragma unroll
      for (int kk = 0; kk < TC_BK / 8; ++kk) {
        // each MMA consumes K = 8 tf32 = two 16-byte core-matrix columns
        const uint64_t ad = make_desc(a0 + kk * 2 * 128, 128, TC_BK * 8 * 4);
        const uint64_t bd = make_desc(b0 + kk * 2 * 128, 128, TC_BK * 8 * 4);
        const uint32_t accum = (s > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&mbar)));
    }
    // wait for the MMAs of this stage (bounded)
    {
      uint32_t done = 0;
      long long spins = 0;
      while (!done) {
        asm volatile(
            "{\n.reg .pred P1;\nmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\nselp.b32 %0, 1, 0, P1;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(&mbar)), "r"(phase));
        if (!done && ++spins > kMbarSpin) break;
      }
      if (!done) s_fail = 1;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    __syncthreads();
    if (s_fail) ok = false;
  }
  if (!ok) {
    if (tid == 0) atomicExch(err, LS_ETIMEOUT);
  } else if (nstages > 0) {
    // epilogue: warp w owns TMEM lanes (rows) 32w .. 32w+31; 16 columns at a time
    const int row = m0 + warp * 32 + lane;
    const bool zb = (beta.re == 0.f && beta.im == 0.f);
#pragma unroll 1
    for (int c0 = 0; c0 < TC_BN; c0 += 16) {
      uint32_t v[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (row < M) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int col = n0 + c0 / 2 + e;
          if (col < N) {
            c32 acc = mk<float>(__uint_as_float(v[2 * e]), __uint_as_float(v[2 * e + 1]));
            c32 out = alpha * acc;
            if (!zb) out = out + beta * C[(long long)row * ldc + col];
            C[(long long)row * ldc + col] = out;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_BN));
}

}  // namespace

// Host entry: same contract as the SIMT gemm (batched, row-major, op N/T).
int tc_cgemm(cudaStream_t st, bool ta, bool tb, int M, int N, int K, c32 alpha, const c32* A, int lda, long long sA,
             const c32* B, int ldb, long long sB, c32 beta, c32* C, int ldc, long long sC, int batch, int split,
             int* err) {
  if (M <= 0 || N <= 0 || batch <= 0 || K <= 0) return LS_OK;
  dim3 grid((N + TC_BN / 2 - 1) / (TC_BN / 2), (M + TC_BM - 1) / TC_BM, batch);
  count_launch();
  if (!ta && !tb)
    tc_cgemm_kernel<false, false><<<grid, TC_THREADS, 0, st>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc,
                                                               sC, split, err);
  else if (ta && !tb)
    tc_cgemm_kernel<true, false><<<grid, TC_THREADS, 0, st>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc,
                                                              sC, split, err);
  else if (!ta && tb)
    tc_cgemm_kernel<false, true><<<grid, TC_THREADS, 0, st>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc,
                                                              sC, split, err);
  else
    tc_cgemm_kernel<true, true><<<grid, TC_THREADS, 0, st>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc,
                                                             sC, split, err);
  return check_launch("tc_cgemm");
}

}  // namespace ls
