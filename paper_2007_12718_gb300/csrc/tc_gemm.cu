// Complex FP32 GEMM on the Blackwell tensor cores (tcgen05.mma, kind::tf32,
// accumulators in tensor memory), for the merge products of the HBS build
// (Eqs. 26-27: S G, S G^T, Y2 Y1, the Schur-complement blocks, X diag(S) U,
// U^T (.), and the trailing updates of the blocked inverse).
//
// A complex product is one real product of twice the size: with A stored
// interleaved (re, im), row i of A is the real row (a_r0, a_i0, a_r1, ...)
// of length 2K, and every complex entry b = (br, bi) of B becomes the 2x2 real
// block [[br, bi], [-bi, br]] of a 2K x 2N real matrix B'.  Then A' B' is C
// interleaved.  In tf32x3 mode each operand is split into a tf32 head and a
// tf32 tail (x = hi + lo) and the K loop runs over [A_hi A_hi A_lo] x
// [B_hi; B_lo; B_hi] (~FP32 accuracy; the lo*lo term is dropped).
//
// Data path: two packing kernels write op(A) and op(B) as "stage images",
// each stage (128 rows x 64 real k, 32 KB) already in the K-major no-swizzle
// shared-memory layout of 8-row x 16-byte core matrices.  The GEMM kernel
// (one 128 x 128-real tile per block) moves each stage with two 32 KB
// cp.async.bulk copies into a ring of three 64 KB buffers (full/empty
// mbarriers), one thread issues eight m128n128k8 MMAs per stage and commits
// them to the buffer's "empty" barrier, and the 128 x 128 FP32 accumulator is
// read back from tensor memory with tcgen05.ld.  Every mbarrier wait is
// bounded: on timeout the block sets *err, issues nothing more, frees its
// tensor memory and returns.
#include <string.h>

#include <algorithm>

#include "handle.h"

namespace ls {
namespace {

constexpr int TC_BM = 128;                      // rows per tile
constexpr int TC_BN = 128;                      // real columns per tile (64 complex)
constexpr int TC_BK = 64;                       // real k per stage (32 complex)
constexpr int TC_IMG = TC_BM * TC_BK;           // floats per stage image (32 KB)
constexpr int TC_NBUF = 3;                      // ring of stage buffers
constexpr int TC_THREADS = 128;
constexpr long long kMbarSpin = 1LL << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major no-swizzle layout: core matrix = 8 rows x 16 bytes; LBO = 128 B
// between K-adjacent core matrices, SBO = 2048 B between M/N-adjacent ones.
__device__ __forceinline__ int kmaj(int row, int k) {
  return (row >> 3) * (TC_BK * 8) + (k >> 2) * 32 + (row & 7) * 4 + (k & 3);
}

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

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void split2(float x, bool lo, float& out) {
  float h = to_tf32(x);
  out = lo ? to_tf32(x - h) : h;
}

// imgA[part][b][mt][ks]: op(A)(row, kc) -> real (row, 2kc + {0: re, 1: im}).
template <bool TA>
__global__ void pack_a_kernel(const c32* __restrict__ A, int lda, long long sA, int M, int K, int MT, int KS,
                              int nparts, float* __restrict__ img, long long s_img_b) {
  const int b = blockIdx.y;
  const long long per_part = s_img_b * gridDim.y;
  const long long total = (long long)MT * TC_BM * KS * (TC_BK / 2);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    // consecutive threads along k (row-major A) or along rows (transposed A)
    int row, kc;
    if (TA) {
      row = (int)(t % (MT * TC_BM));
      kc = (int)(t / (MT * TC_BM));
    } else {
      kc = (int)(t % (KS * (TC_BK / 2)));
      row = (int)(t / (KS * (TC_BK / 2)));
    }
    c32 v = mk<float>(0.f, 0.f);
    if (row < M && kc < K) v = TA ? A[b * sA + (long long)kc * lda + row] : A[b * sA + (long long)row * lda + kc];
    const int mt = row / TC_BM, r = row % TC_BM, ks = kc / (TC_BK / 2), k2 = 2 * (kc % (TC_BK / 2));
    const long long base = b * s_img_b + ((long long)mt * KS + ks) * TC_IMG;
    for (int part = 0; part < nparts; ++part) {
      float re, im;
      split2(v.re, part == 1, re);
      split2(v.im, part == 1, im);
      img[part * per_part + base + kmaj(r, k2)] = re;
      img[part * per_part + base + kmaj(r, k2 + 1)] = im;
    }
  }
}

// imgB[part][b][nt][ks]: op(B)(q, j) -> 2x2 real block of B'^T rows 2j, 2j+1, k 2q, 2q+1.
template <bool TB>
__global__ void pack_b_kernel(const c32* __restrict__ B, int ldb, long long sB, int K, int N, int NT, int KS,
                              int nparts, float* __restrict__ img, long long s_img_b) {
  const int b = blockIdx.y;
  const long long per_part = s_img_b * gridDim.y;
  const int NC = NT * (TC_BN / 2), KC = KS * (TC_BK / 2);
  const long long total = (long long)NC * KC;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    int j, q;
    if (TB) {  // B stored N x K: consecutive threads along K
      q = (int)(t % KC);
      j = (int)(t / KC);
    } else {   // B stored K x N: consecutive threads along N
      j = (int)(t % NC);
      q = (int)(t / NC);
    }
    c32 v = mk<float>(0.f, 0.f);
    if (j < N && q < K) v = TB ? B[b * sB + (long long)j * ldb + q] : B[b * sB + (long long)q * ldb + j];
    const int nt = j / (TC_BN / 2), jl = j % (TC_BN / 2), ks = q / (TC_BK / 2), ql = q % (TC_BK / 2);
    const long long base = b * s_img_b + ((long long)nt * KS + ks) * TC_IMG;
    for (int part = 0; part < nparts; ++part) {
      float br, bi;
      split2(v.re, part == 1, br);
      split2(v.im, part == 1, bi);
      float* o = img + part * per_part + base;
      o[kmaj(2 * jl, 2 * ql)] = br;
      o[kmaj(2 * jl, 2 * ql + 1)] = -bi;
      o[kmaj(2 * jl + 1, 2 * ql)] = bi;
      o[kmaj(2 * jl + 1, 2 * ql + 1)] = br;
    }
  }
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

// C[b] (M x N complex) = alpha A'B' + beta C[b], from the stage images.
__global__ void __launch_bounds__(TC_THREADS) tc_gemm_kernel(int M, int N, int KS, int nparts, const float* __restrict__ imgA,
                                                             long long sIA, long long partA, const float* __restrict__ imgB,
                                                             long long sIB, long long partB, int MT, int NT, c32 alpha,
                                                             c32 beta, c32* __restrict__ C, int ldc, long long sC,
                                                             int* err) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  float* buf = reinterpret_cast<float*>(smraw);  // TC_NBUF x (A image | B image)
  __shared__ __align__(8) uint64_t full_bar[TC_NBUF], empty_bar[TC_NBUF], done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nt = blockIdx.x, mt = blockIdx.y, bz = blockIdx.z;
  const float* gA = imgA + bz * sIA + (long long)mt * KS * TC_IMG;
  const float* gB = imgB + bz * sIB + (long long)nt * KS * TC_IMG;
  C += bz * sC;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(TC_BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < TC_NBUF; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full_bar[i])), "r"(1));
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
  const int S = KS * nparts;

  if (tid == 0) {  // producer: stage s into buffer s % NBUF
    for (int s = 0; s < S; ++s) {
      const int bi = s % TC_NBUF;
      if (s >= TC_NBUF && !mbar_wait(smem_u32(&empty_bar[bi]), ((s / TC_NBUF) - 1) & 1)) {
        atomicExch(&s_fail, 1);
        break;
      }
      if (*(volatile int*)&s_fail) break;
      const int part = s / KS, ks = s % KS;
      const int pa = (nparts == 3 && part == 2) ? 1 : 0;  // A: hi, hi, lo
      const int pb = (nparts == 3 && part == 1) ? 1 : 0;  // B: hi, lo, hi
      const float* srcA = gA + pa * partA + (long long)ks * TC_IMG;
      const float* srcB = gB + pb * partB + (long long)ks * TC_IMG;
      float* dA = buf + (long long)bi * 2 * TC_IMG;
      float* dB = dA + TC_IMG;
      const uint32_t fb = smem_u32(&full_bar[bi]);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(2 * TC_IMG * 4)
                   : "memory");
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       smem_u32(dA)),
                   "l"(srcA), "r"(TC_IMG * 4), "r"(fb)
                   : "memory");
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       smem_u32(dB)),
                   "l"(srcB), "r"(TC_IMG * 4), "r"(fb)
                   : "memory");
    }
  } else if (tid == 32) {  // MMA issuer
    const uint32_t idesc = make_idesc_tf32(TC_BM, TC_BN);
    bool ok = true;
    for (int s = 0; s < S; ++s) {
      const int bi = s % TC_NBUF;
      if (!mbar_wait(smem_u32(&full_bar[bi]), (s / TC_NBUF) & 1) || *(volatile int*)&s_fail) {
        atomicExch(&s_fail, 1);
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a0 = smem_u32(buf + (long long)bi * 2 * TC_IMG), b0 = a0 + TC_IMG * 4;
#pragma unroll
      for (int kk = 0; kk < TC_BK / 8; ++kk) {
        const uint64_t ad = make_desc(a0 + kk * 256, 128, TC_BK * 8 * 4);
        const uint64_t bd = make_desc(b0 + kk * 256, 128, TC_BK * 8 * 4);
        const uint32_t accum = (s > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&empty_bar[bi])));
    }
    if (ok) {
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&done_bar)));
    }
  }
  // everyone: wait for the last MMA (or a failure)
  bool ok = true;
  if (S > 0) {
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
  asm volatile("tcgen05.fence::after_thread_sync;");
  __syncthreads();
  if (!ok || s_fail) {
    if (tid == 0) atomicExch(err, LS_ETIMEOUT);
  } else if (S > 0) {
    const int row = mt * TC_BM + warp * 32 + lane;
    const int n0 = nt * (TC_BN / 2);
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
// Operands shared by the whole batch (stride 0) are packed once.
int tc_cgemm(cudaStream_t st, bool ta, bool tb, int M, int N, int K, c32 alpha, const c32* A, int lda, long long sA,
             const c32* B, int ldb, long long sB, c32 beta, c32* C, int ldc, long long sC, int batch, int split,
             int* err) {
  if (M <= 0 || N <= 0 || batch <= 0 || K <= 0) return LS_OK;
  const int MT = (M + TC_BM - 1) / TC_BM, NT = (N + TC_BN / 2 - 1) / (TC_BN / 2);
  const int KS = (2 * K + TC_BK - 1) / TC_BK;
  const int nparts = split ? 3 : 1, nimg = split ? 2 : 1;
  const int batchA = sA ? batch : 1, batchB = sB ? batch : 1;
  const long long sIA = (long long)MT * KS * TC_IMG, sIB = (long long)NT * KS * TC_IMG;
  float* img = nullptr;
  int rc = dalloc((void**)&img, sizeof(float) * (size_t)nimg * ((size_t)sIA * batchA + (size_t)sIB * batchB));
  if (rc) return rc;
  float* imgA = img;
  float* imgB = img + (size_t)nimg * sIA * batchA;
  {
    long long tot = (long long)MT * TC_BM * KS * (TC_BK / 2);
    dim3 g((unsigned)std::min<long long>(4096, (tot + 255) / 256), batchA);
    count_launch();
    if (ta)
      pack_a_kernel<true><<<g, 256, 0, st>>>(A, lda, sA, M, K, MT, KS, nimg, imgA, sIA);
    else
      pack_a_kernel<false><<<g, 256, 0, st>>>(A, lda, sA, M, K, MT, KS, nimg, imgA, sIA);
  }
  {
    long long tot = (long long)NT * (TC_BN / 2) * KS * (TC_BK / 2);
    dim3 g((unsigned)std::min<long long>(4096, (tot + 255) / 256), batchB);
    count_launch();
    if (tb)
      pack_b_kernel<true><<<g, 256, 0, st>>>(B, ldb, sB, K, N, NT, KS, nimg, imgB, sIB);
    else
      pack_b_kernel<false><<<g, 256, 0, st>>>(B, ldb, sB, K, N, NT, KS, nimg, imgB, sIB);
  }
  const size_t smem = sizeof(float) * (size_t)TC_NBUF * 2 * TC_IMG;
  LS_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid(NT, MT, batch);
  count_launch();
  tc_gemm_kernel<<<grid, TC_THREADS, smem, st>>>(M, N, KS, nparts, imgA, sA ? sIA : 0, sIA * batchA, imgB,
                                                  sB ? sIB : 0, sIB * batchB, MT, NT, alpha, beta, C, ldc, sC, err);
  rc = check_launch("tc_cgemm");
  dfree(img);
  return rc;
}

}  // namespace ls
