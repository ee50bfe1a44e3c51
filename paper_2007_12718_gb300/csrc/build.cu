// HBS inverse: Algorithm 1 (build) and Algorithm 2 (apply) of Sec. 4.1.
//
// Data layout (precision R = float or double, complex interleaved):
//   leaf level L : X_tau = (I + B_tau G_tau)^-1        [2^L][s^2][s^2]   (Eq. 20)
//                  XBU_tau = X_tau B_tau U_L           [2^L][s^2][k_L]
//                  S_tau = U_L^T XBU_tau               [2^L][k_L][k_L]   (Eq. 23)
//   level l < L  : X_tau = [[I, S_a G],[S_b G^T, I]]^-1 [2^l][2k][2k]     (Eq. 26)
//                  S_tau = U_l^T X_tau diag(S_a,S_b) U_l [2^l][k_l][k_l] (Eq. 27)
// with k = k_{l+1}, G = G_sib of level l+1 (shared by every parent of level
// l), U_l shared by every node of level l (translation invariance, Sec. 3.2),
// V^* read as U^T (G is complex symmetric).  Children of node t are 2t, 2t+1,
// so the pair [r_a; r_b] of a parent is contiguous in the child arrays.
//
// Kernels: a batched complex GEMM (operands may be shared across the batch),
// in-shared-memory Gauss-Jordan inversion with partial pivoting (one block
// per matrix; the leaf kernel fuses it with the X B U and S products), and a
// cooperative multi-block Gauss-Jordan for the large top-level matrices.
#include <cooperative_groups.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "handle.h"
#include "prof.h"

namespace ls {
namespace {

// ---------------------------------------------------------------- GEMM
constexpr int TM = 32, TN = 32, TK = 16;

// Outputs a GEMM leaves untouched: rows and columns in [lo, hi) (empty by default).
struct Band {
  int lo = 0, hi = 0;
  __host__ __device__ bool skip(int i, int j) const { return (i >= lo && i < hi) || (j >= lo && j < hi); }
};

// C[b] = alpha op(A[b]) op(B[b]) + beta C[b]   (row-major, op = N or T)
template <class R, bool TA, bool TB>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, cx<R> alpha, const cx<R>* __restrict__ A,
                                                   int lda, long long sA, const cx<R>* __restrict__ B, int ldb,
                                                   long long sB, cx<R> beta, cx<R>* __restrict__ C, int ldc,
                                                   long long sC, Band bd) {
  __shared__ cx<R> As[TK][TM + 1];
  __shared__ cx<R> Bs[TK][TN + 1];
  const int b = blockIdx.z;
  A += b * sA;
  B += b * sB;
  C += b * sC;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  cx<R> acc[2][2];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) acc[i][j] = mk<R>(0, 0);
  for (int k0 = 0; k0 < K; k0 += TK) {
    for (int t = threadIdx.x; t < TK * TM; t += 256) {
      int kk, i;
      if (TA) {  // A stored K x M: read along M
        i = t % TM;
        kk = t / TM;
      } else {   // A stored M x K: read along K
        kk = t % TK;
        i = t / TK;
      }
      int gi = m0 + i, gk = k0 + kk;
      cx<R> v = mk<R>(0, 0);
      if (gi < M && gk < K) v = TA ? A[(long long)gk * lda + gi] : A[(long long)gi * lda + gk];
      As[kk][i] = v;
    }
    for (int t = threadIdx.x; t < TK * TN; t += 256) {
      int kk, j;
      if (TB) {  // B stored N x K
        kk = t % TK;
        j = t / TK;
      } else {   // B stored K x N
        j = t % TN;
        kk = t / TN;
      }
      int gj = n0 + j, gk = k0 + kk;
      cx<R> v = mk<R>(0, 0);
      if (gj < N && gk < K) v = TB ? B[(long long)gj * ldb + gk] : B[(long long)gk * ldb + gj];
      Bs[kk][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      cx<R> a0 = As[kk][ty], a1 = As[kk][ty + 16];
      cx<R> b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
      fma_(acc[0][0], a0, b0);
      fma_(acc[0][1], a0, b1);
      fma_(acc[1][0], a1, b0);
      fma_(acc[1][1], a1, b1);
    }
    __syncthreads();
  }
  const bool zb = (beta.re == R(0) && beta.im == R(0));
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      int gi = m0 + ty + 16 * i, gj = n0 + tx + 16 * j;
      if (gi < M && gj < N && !bd.skip(gi, gj)) {
        cx<R> v = alpha * acc[i][j];
        if (!zb) v = v + beta * C[(long long)gi * ldc + gj];
        C[(long long)gi * ldc + gj] = v;
      }
    }
}

// 64 x 64 output tile per block, 4 x 4 outputs per thread (rows ty + 16 i,
// columns tx + 16 j), K staged 16 at a time through shared memory.
template <class R, bool TA, bool TB>
__global__ void __launch_bounds__(256) gemm64_kernel(int M, int N, int K, cx<R> alpha, const cx<R>* __restrict__ A,
                                                     int lda, long long sA, const cx<R>* __restrict__ B, int ldb,
                                                     long long sB, cx<R> beta, cx<R>* __restrict__ C, int ldc,
                                                     long long sC, Band bd) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ cx<R> As[BK][BM + 1];
  __shared__ cx<R> Bs[BK][BN + 1];
  const int b = blockIdx.z;
  A += b * sA;
  B += b * sB;
  C += b * sC;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  cx<R> acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = mk<R>(0, 0);
  for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int t = threadIdx.x + 256 * r;
      int kk, i;
      if (TA) {
        i = t % BM;
        kk = t / BM;
      } else {
        kk = t % BK;
        i = t / BK;
      }
      int gi = m0 + i, gk = k0 + kk;
      cx<R> v = mk<R>(0, 0);
      if (gi < M && gk < K) v = TA ? A[(long long)gk * lda + gi] : A[(long long)gi * lda + gk];
      As[kk][i] = v;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int t = threadIdx.x + 256 * r;
      int kk, j;
      if (TB) {
        kk = t % BK;
        j = t / BK;
      } else {
        j = t % BN;
        kk = t / BN;
      }
      int gj = n0 + j, gk = k0 + kk;
      cx<R> v = mk<R>(0, 0);
      if (gj < N && gk < K) v = TB ? B[(long long)gj * ldb + gk] : B[(long long)gk * ldb + gj];
      Bs[kk][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      cx<R> a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) fma_(acc[i][j], a[i], bb[j]);
    }
    __syncthreads();
  }
  const bool zb = (beta.re == R(0) && beta.im == R(0));
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gi = m0 + ty + 16 * i, gj = n0 + tx + 16 * j;
      if (gi < M && gj < N && !bd.skip(gi, gj)) {
        cx<R> v = alpha * acc[i][j];
        if (!zb) v = v + beta * C[(long long)gi * ldc + gj];
        C[(long long)gi * ldc + gj] = v;
      }
    }
}

// FP32 complex GEMM with packed two-lane FMAs (fma.rn.f32x2): the same 64 x 64
// tile, 4 x 4 outputs per thread and K loop as gemm64_kernel, with each complex
// multiply-add as two packed FMAs on (re, im) pairs instead of four scalar ones
// (in the same order as fma_, so the results are the same bits):
//   acc += (-a.im, a.im) * (b.im, b.re);  acc += (a.re, a.re) * (b.re, b.im).
// The operand tiles are staged in shared memory already in those forms.
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long pk2(float lo, float hi) {
  return ((unsigned long long)__float_as_uint(hi) << 32) | (unsigned long long)__float_as_uint(lo);
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(256) gemm64x2_kernel(int M, int N, int K, c32 alpha, const c32* __restrict__ A,
                                                       int lda, long long sA, const c32* __restrict__ B, int ldb,
                                                       long long sB, c32 beta, c32* __restrict__ C, int ldc,
                                                       long long sC, Band bd) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ ulonglong2 As[BK][BM + 1];  // x = (re, re), y = (-im, im)
  __shared__ ulonglong2 Bs[BK][BN + 1];  // x = (re, im), y = (im, re)
  const int b = blockIdx.z;
  A += b * sA;
  B += b * sB;
  C += b * sC;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  unsigned long long acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0ULL;
  // the next K tile is loaded into registers while the current one is used
  c32 pa[4], pb[4];
  auto load_tiles = [&](int k0) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int t = threadIdx.x + 256 * r;
      const int kk = TA ? t / BM : t % BK, i = TA ? t % BM : t / BK;
      const int gi = m0 + i, gk = k0 + kk;
      pa[r] = (gi < M && gk < K) ? (TA ? A[(long long)gk * lda + gi] : A[(long long)gi * lda + gk]) : mk<float>(0, 0);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int t = threadIdx.x + 256 * r;
      const int kk = TB ? t % BK : t / BN, j = TB ? t / BK : t % BN;
      const int gj = n0 + j, gk = k0 + kk;
      pb[r] = (gj < N && gk < K) ? (TB ? B[(long long)gj * ldb + gk] : B[(long long)gk * ldb + gj]) : mk<float>(0, 0);
    }
  };
  auto store_tiles = [&]() {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int t = threadIdx.x + 256 * r;
      const int kk = TA ? t / BM : t % BK, i = TA ? t % BM : t / BK;
      As[kk][i] = make_ulonglong2(pk2(pa[r].re, pa[r].re), pk2(-pa[r].im, pa[r].im));
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int t = threadIdx.x + 256 * r;
      const int kk = TB ? t % BK : t / BN, j = TB ? t / BK : t % BN;
      Bs[kk][j] = make_ulonglong2(pk2(pb[r].re, pb[r].im), pk2(pb[r].im, pb[r].re));
    }
  };
  load_tiles(0);
  for (int k0 = 0; k0 < K; k0 += BK) {
    store_tiles();
    __syncthreads();
    if (k0 + BK < K) load_tiles(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      ulonglong2 a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = ffma2(a[i].x, bb[j].x, ffma2(a[i].y, bb[j].y, acc[i][j]));
    }
    __syncthreads();
  }
  const bool zb = (beta.re == 0.0f && beta.im == 0.0f);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gi = m0 + ty + 16 * i, gj = n0 + tx + 16 * j;
      if (gi < M && gj < N && !bd.skip(gi, gj)) {
        const c32 av = mk<float>(__uint_as_float((unsigned)acc[i][j]), __uint_as_float((unsigned)(acc[i][j] >> 32)));
        c32 v = alpha * av;
        if (!zb) v = v + beta * C[(long long)gi * ldc + gj];
        C[(long long)gi * ldc + gj] = v;
      }
    }
}

// Engine of the FP32 merge GEMMs for the build in progress on this thread:
// 0 = SIMT FP32, 1 = tensor cores tf32, 2 = tensor cores tf32x3.
thread_local int g_tc_engine = 0;  // 0 SIMT, 1 tf32, 2 tf32x3, 3 f16x3 (tc_cgemm's split + 1)
thread_local int* g_tc_err = nullptr;

// The tensor-core engine of a handle's precision mode (0: the SIMT kernels).
int tc_engine_of(const ls_handle* H) {
  return H->prec == LS_TF32 ? 1 : H->prec == LS_TF32X3 ? 2 : H->prec == LS_FP16SPLIT ? 3 : 0;
}

// Batches beyond the grid's y / z limit are launched in chunks.
constexpr int kMaxGridYZ = 65535;

template <class R>
void gemm(cudaStream_t st, bool ta, bool tb, int M, int N, int K, cx<R> alpha, const cx<R>* A, int lda, long long sA,
          const cx<R>* B, int ldb, long long sB, cx<R> beta, cx<R>* C, int ldc, long long sC, int batch,
          Band bd = Band()) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  if (batch > kMaxGridYZ) {
    for (int b0 = 0; b0 < batch; b0 += kMaxGridYZ)
      gemm<R>(st, ta, tb, M, N, K, alpha, A + b0 * sA, lda, sA, B + b0 * sB, ldb, sB, beta, C + b0 * sC, ldc, sC,
              std::min(kMaxGridYZ, batch - b0), bd);
    return;
  }
  if (K <= 0) return;  // only reached with beta = 1 (nothing to add)
  // tensor cores for every product with at least one 128 x 128 tile and ~2^25
  // complex MACs: measured 2x (K = 64 updates) to 4x (K in the thousands) the
  // SIMT kernel's rate in tf32x3; smaller products stay on the SIMT kernels
  if (sizeof(R) == 4 && g_tc_engine > 0 && M >= 128 && N >= 128 && K >= 32 &&
      (double)M * N * K * batch >= 3.3e7) {
    tc_cgemm(st, ta, tb, M, N, K, *reinterpret_cast<const c32*>(&alpha), reinterpret_cast<const c32*>(A), lda, sA,
             reinterpret_cast<const c32*>(B), ldb, sB, *reinterpret_cast<const c32*>(&beta),
             reinterpret_cast<c32*>(C), ldc, sC, batch, g_tc_engine - 1, g_tc_err, bd.lo, bd.hi);
    return;
  }
  count_launch();
  // 64 x 64 tiles unless they leave most SMs idle (then 32 x 32 tiles: four times the blocks)
  if (M >= 48 && N >= 48 && (long long)((N + 63) / 64) * ((M + 63) / 64) * batch >= 128) {
    dim3 grid((N + 63) / 64, (M + 63) / 64, batch);
    if constexpr (sizeof(R) == 4) {
      const c32* A2 = reinterpret_cast<const c32*>(A);
      const c32* B2 = reinterpret_cast<const c32*>(B);
      c32* C2 = reinterpret_cast<c32*>(C);
      const c32 al = *reinterpret_cast<const c32*>(&alpha), be = *reinterpret_cast<const c32*>(&beta);
      if (!ta && !tb)
        gemm64x2_kernel<false, false><<<grid, 256, 0, st>>>(M, N, K, al, A2, lda, sA, B2, ldb, sB, be, C2, ldc, sC, bd);
      else if (ta && !tb)
        gemm64x2_kernel<true, false><<<grid, 256, 0, st>>>(M, N, K, al, A2, lda, sA, B2, ldb, sB, be, C2, ldc, sC, bd);
      else if (!ta && tb)
        gemm64x2_kernel<false, true><<<grid, 256, 0, st>>>(M, N, K, al, A2, lda, sA, B2, ldb, sB, be, C2, ldc, sC, bd);
      else
        gemm64x2_kernel<true, true><<<grid, 256, 0, st>>>(M, N, K, al, A2, lda, sA, B2, ldb, sB, be, C2, ldc, sC, bd);
      return;
    }
    if (!ta && !tb)
      gemm64_kernel<R, false, false><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, bd);
    else if (ta && !tb)
      gemm64_kernel<R, true, false><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, bd);
    else if (!ta && tb)
      gemm64_kernel<R, false, true><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, bd);
    else
      gemm64_kernel<R, true, true><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, bd);
    return;
  }
  dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM, batch);
  if (!ta && !tb)
    gemm_kernel<R, false, false><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, bd);
  else if (ta && !tb)
    gemm_kernel<R, true, false><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, bd);
  else if (!ta && tb)
    gemm_kernel<R, false, true><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, bd);
  else
    gemm_kernel<R, true, true><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, bd);
}

template <class R>
cx<R> one() { return mk<R>(R(1), R(0)); }
template <class R>
cx<R> zero() { return mk<R>(R(0), R(0)); }

// ------------------------------------------- Gauss-Jordan in shared memory
// In-place inverse of the n x n matrix a (row stride lda) with partial row
// pivoting; column interchanges undo the row pivoting at the end.  Returns
// false (in every thread) on an exactly zero pivot.
template <class R>
__device__ bool gj_inverse_smem(cx<R>* a, int n, int lda, int* piv, cx<R>* col) {
  if (n > 256) return false;  // the elimination keeps at most 8 x 32 pivot-row entries per lane
  __shared__ int s_p;
  __shared__ int s_bad;
  __shared__ cx<R> s_d;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int k = 0; k < n; ++k) {
    if (warp == 0) {  // pivot: largest |a(i,k)| over i >= k, lowest row on ties
      R best = R(-1);
      int bi = n;
      for (int i = k + lane; i < n; i += 32) {
        R v = abs2(a[i * lda + k]);
        if (v > best) {
          best = v;
          bi = i;
        }
      }
      for (int o = 16; o; o >>= 1) {
        R ob = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (lane == 0) {
        s_p = bi;
        piv[k] = bi;
        s_bad = !(best > R(0));
        if (!s_bad) s_d = inv(a[bi * lda + k]);
      }
    }
    __syncthreads();
    if (s_bad) return false;
    const int p = s_p;
    const cx<R> d = s_d;
    // multipliers of column k after the interchange; rows k and p exchanged
    // (and the new row k scaled by d) in every column except k
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      col[i] = (i == k) ? a[p * lda + k] : (i == p ? a[k * lda + k] : a[i * lda + k]);
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      if (j == k) continue;
      cx<R> tk = a[k * lda + j], tp = a[p * lda + j];
      if (p != k) a[p * lda + j] = tk;
      a[k * lda + j] = tp * d;
    }
    __syncthreads();
    // elimination: warp w takes rows w, w + nwarp, ...; lane takes columns lane + 32 q,
    // the scaled pivot row is held in registers for the whole step
    {
      cx<R> kr[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int j = lane + 32 * q;
        kr[q] = (j < n && j != k) ? a[k * lda + j] : mk<R>(0, 0);
      }
      const cx<R> nd = mk<R>(-d.re, -d.im);
      for (int i = warp; i < n; i += nwarp) {
        cx<R>* arow = a + i * lda;
        if (i == k) {
          if (lane == 0) arow[k] = d;
          continue;
        }
        const cx<R> f = col[i];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int j = lane + 32 * q;
          if (j < n) {
            if (j == k) {
              arow[j] = f * nd;
            } else {
              cx<R> v = arow[j];
              v.re -= f.re * kr[q].re - f.im * kr[q].im;
              v.im -= f.re * kr[q].im + f.im * kr[q].re;
              arow[j] = v;
            }
          }
        }
      }
    }
    __syncthreads();
  }
  for (int k = n - 1; k >= 0; --k) {
    int p = piv[k];
    if (p != k)
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        cx<R> t = a[i * lda + k];
        a[i * lda + k] = a[i * lda + p];
        a[i * lda + p] = t;
      }
    __syncthreads();
  }
  return true;
}

// A handle holds G >= 1 problems on the same grid (a forest of G trees of the
// same geometry, sharing the compression): the nodes of level l are indexed
// g 2^l + j (problem g, node j of its tree), so the children of node i are 2i
// and 2i + 1 across the whole forest, and the problems' grid vectors are stacked
// as one grid of G ny rows.
struct TreeGeom {
  int L, s, nx, ny, G;
  int cw[32], ch[32];  // child box dims for the cut l -> l+1
};

// Lower-left grid point of a leaf (leaf = g 2^L + j): rows of problem g start at g ny.
__device__ __forceinline__ void leaf_origin(const TreeGeom& g, int leaf, int& ox, int& oy) {
  ox = 0;
  oy = (leaf >> g.L) * g.ny;
  for (int l = 0; l < g.L; ++l) {
    int bit = (leaf >> (g.L - 1 - l)) & 1;
    if (l % 2 == 0) {
      if (bit) ox += g.cw[l];
    } else {
      if (!bit) oy += g.ch[l];  // alpha = upper half
    }
  }
}

// Leaf matrices for the batched leaf build: X[leaf] = I + B G_leaf (Eq. (20) before
// the inverse) and BU[leaf] = B U; one thread per entry of either.
template <class R>
__global__ void leaf_matrix_kernel(TreeGeom g, const double* __restrict__ b, double kap2, const cx<R>* __restrict__ Gleaf,
                                   const cx<R>* __restrict__ U, int k, cx<R>* __restrict__ X, cx<R>* __restrict__ BU,
                                   long long nleaf) {
  const int n = g.s * g.s;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= nleaf * n * n) return;
  const int leaf = (int)(t / ((long long)n * n)), i = (int)((t / n) % n), j = (int)(t % n);
  int ox, oy;
  leaf_origin(g, leaf, ox, oy);
  const R bi = (R)(kap2 * b[(long long)(oy + i / g.s) * g.nx + ox + i % g.s]);
  cx<R> v = scale(Gleaf[i * n + j], bi);
  if (i == j) v.re += R(1);
  X[t] = v;
  if (j < k) BU[((long long)leaf * n + i) * k + j] = scale(U[i * k + j], bi);
}

// Leaf build (Algorithm 1, leaf loop): one block per leaf.
template <class R>
__global__ void __launch_bounds__(256) leaf_build_kernel(TreeGeom g, const double* __restrict__ b, double kap2,
                                                         const cx<R>* __restrict__ Gleaf, const cx<R>* __restrict__ U,
                                                         int k, cx<R>* __restrict__ X, cx<R>* __restrict__ XBU,
                                                         cx<R>* __restrict__ S, int* __restrict__ err) {
  extern __shared__ unsigned char smraw[];
  const int n = g.s * g.s, ls = n + 1;         // odd row stride (no bank conflicts on columns)
  cx<R>* a = reinterpret_cast<cx<R>*>(smraw);  // n x n, stride ls
  cx<R>* xbu = a + n * ls;                     // n x k
  cx<R>* col = xbu + n * k;                    // n
  R* Bv = reinterpret_cast<R*>(col + n);       // n
  int* piv = reinterpret_cast<int*>(Bv + n);   // n
  const int leaf = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int ox, oy;
  leaf_origin(g, leaf, ox, oy);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int lx = i % g.s, ly = i / g.s;
    Bv[i] = (R)(kap2 * b[(long long)(oy + ly) * g.nx + ox + lx]);
  }
  __syncthreads();
  for (int i = warp; i < n; i += 8)
    for (int j = lane; j < n; j += 32) {
      cx<R> v = scale(Gleaf[i * n + j], Bv[i]);
      if (i == j) v.re += R(1);
      a[i * ls + j] = v;
    }
  __syncthreads();
  if (!gj_inverse_smem(a, n, ls, piv, col)) {
    if (threadIdx.x == 0) atomicExch(err, LS_ESINGULAR);
    return;
  }
  // XBU = X diag(B) U
  for (int t = threadIdx.x; t < n * k; t += blockDim.x) {
    int i = t / k, c = t % k;
    cx<R> acc = mk<R>(0, 0);
    for (int j = 0; j < n; ++j) fma_(acc, a[i * ls + j], scale(U[j * k + c], Bv[j]));
    xbu[t] = acc;
  }
  __syncthreads();
  cx<R>* Xo = X + (long long)leaf * n * n;
  for (int i = warp; i < n; i += 8)
    for (int j = lane; j < n; j += 32) Xo[i * n + j] = a[i * ls + j];
  cx<R>* XBUo = XBU + (long long)leaf * n * k;
  for (int t = threadIdx.x; t < n * k; t += blockDim.x) XBUo[t] = xbu[t];
  // S = U^T XBU
  cx<R>* So = S + (long long)leaf * k * k;
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
    int r = t / k, c = t % k;
    cx<R> acc = mk<R>(0, 0);
    for (int i = 0; i < n; ++i) fma_(acc, U[i * k + r], xbu[i * k + c]);
    So[t] = acc;
  }
}

// Batched in-smem inverse, one block per matrix (matrix b at X + b*sX, row stride lda).
template <class R>
__global__ void __launch_bounds__(512) inverse_smem_kernel(cx<R>* X, int n, int lda, long long sX, int* err) {
  extern __shared__ unsigned char smraw[];
  const int ls = n + 1;  // odd row stride: column reads without bank conflicts
  cx<R>* a = reinterpret_cast<cx<R>*>(smraw);
  cx<R>* col = a + n * ls;
  int* piv = reinterpret_cast<int*>(col + n);
  cx<R>* M = X + blockIdx.x * sX;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  for (int i = warp; i < n; i += nw)
    for (int j = lane; j < n; j += 32) a[i * ls + j] = M[(long long)i * lda + j];
  __syncthreads();
  if (!gj_inverse_smem(a, n, ls, piv, col)) {
    if (threadIdx.x == 0) atomicExch(err, LS_ESINGULAR);
    return;
  }
  for (int i = warp; i < n; i += nw)
    for (int j = lane; j < n; j += 32) M[(long long)i * lda + j] = a[i * ls + j];
}

// Gauss-Jordan inversion without interchanges, register resident: one block per
// matrix, eight threads per row, thread r of a row group holding columns
// r, r + 8, ..., r + 8 (CPT - 1) in registers.  Per elimination step the pivot
// row is staged in a double-buffered shared row (one block barrier per step)
// and the multiplier a(i, k) comes from a register of the row group by a
// shuffle.  n <= 8 CPT, blockDim = 8 n rounded up to a warp.  A zero or
// non-finite pivot sets *err = LS_ESINGULAR (the check is uniform over the
// block).  Accuracy is checked by the caller (probe vector), with the
// row-pivoted kernels as the fallback.
template <class R, int CPT>
__global__ void __launch_bounds__(1024) gj_reg_kernel(cx<R>* __restrict__ X, int n, int lda, long long sX,
                                                      int* __restrict__ err) {
  __shared__ cx<R> prow[2][8 * CPT];
  const int tid = threadIdx.x, row = tid >> 3, r = tid & 7;
  const bool live = row < n;
  cx<R>* M = X + blockIdx.x * sX;
  cx<R> a[CPT];
#pragma unroll
  for (int q = 0; q < CPT; ++q) {
    const int j = q * 8 + r;
    a[q] = (live && j < n) ? M[(long long)row * lda + j] : mk<R>(0, 0);
  }
  // the column block kq is a compile-time index, so the multiplier is read from
  // a fixed register of thread kr of the row group
#pragma unroll
  for (int kq = 0; kq < CPT; ++kq) {
    for (int kr = 0; kr < 8; ++kr) {
      const int k = kq * 8 + kr;
      if (k >= n) break;
      cx<R> f;
      f.re = __shfl_sync(0xffffffffu, a[kq].re, kr, 8);
      f.im = __shfl_sync(0xffffffffu, a[kq].im, kr, 8);
      cx<R>* pr = prow[k & 1];
      if (row == k) {
#pragma unroll
        for (int q = 0; q < CPT; ++q) pr[q * 8 + r] = a[q];
      }
      __syncthreads();
      const cx<R> pk = pr[k];
      const R den = abs2(pk);
      if (!(den > R(0)) || !(den < R(INFINITY))) {
        if (tid == 0) atomicExch(err, LS_ESINGULAR);
        return;
      }
      const cx<R> d = inv(pk);
      if (row == k) {
#pragma unroll
        for (int q = 0; q < CPT; ++q) a[q] = a[q] * d;
        if (r == kr) a[kq] = d;
      } else {
        const cx<R> fd = f * d;
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
          const cx<R> pj = pr[q * 8 + r];
          a[q].re -= fd.re * pj.re - fd.im * pj.im;
          a[q].im -= fd.re * pj.im + fd.im * pj.re;
        }
        if (r == kr) a[kq] = mk<R>(-fd.re, -fd.im);
      }
    }
  }
  if (live) {
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
      const int j = q * 8 + r;
      if (j < n) M[(long long)row * lda + j] = a[q];
    }
  }
}

// Register-blocked Gauss-Jordan inverse without interchanges (FP32), one
// block per matrix: a TR x TC thread grid, each thread an RM x RN block of the
// zero-padded matrix in registers.  At step k the owners of row k and of column
// k put them in shared memory (row k's entry k replaced by 1, column k's by -1)
// and the owner of entry (k, k) its reciprocal d; then every element becomes
//   a[i][j] = z[i][j] - c[i] (d r[j]),   z = a with row k and column k zeroed,
// which is the whole Gauss-Jordan step as one rank-1 formula: row k scaled by
// d, column k set to -a[i][k] d, a[k][k] = d, the Schur update elsewhere.  Per
// step a thread reads RN + RM values from shared memory for RM RN updates, each
// two packed FMAs on (re, im) pairs.  A zero or non-finite pivot sets
// *err = LS_ESINGULAR; the sweep runs on, and the caller's probe check rejects
// the result.
// The sweep of gj2d_kernel on the register blocks a (thread (tr, tc) of the
// TR x TC grid); shared by the plain kernel and the blocked sweep's panel kernel.
template <int TR, int TC, int RM, int RN>
__device__ __forceinline__ void gj2d_sweep(unsigned long long (&a)[RM][RN], int n, int tr, int tc, int* err) {
  constexpr int KU = RM > RN ? RM : RN;
  static_assert(KU % RM == 0 && KU % RN == 0 && KU % 2 == 0 && RN % 2 == 0 && RM % 2 == 0, "block shape");
  __shared__ __align__(16) c32 rowk[2][TC * RN];
  __shared__ __align__(16) c32 colk[2][TR * RM];
  __shared__ c32 dk[2];
  const int nk = (n + KU - 1) / KU;
  for (int kb = 0; kb < nk; ++kb) {
#pragma unroll
    for (int u = 0; u < KU; ++u) {
      if (kb * KU + u >= n) break;
      const int rg = kb * (KU / RM) + u / RM, ur = u % RM;  // owner row group and register row of k
      const int cg = kb * (KU / RN) + u / RN, uc = u % RN;
      const int buf = u & 1;
      const bool rown = tr == rg, cown = tc == cg;
      if (rown) {
#pragma unroll
        for (int v = 0; v < RN; ++v) {
          float lo, hi;
          asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a[ur][v]));
          rowk[buf][tc * RN + v] = (cown && v == uc) ? mk<float>(1.f, 0.f) : mk<float>(lo, hi);
        }
      }
      if (cown) {
#pragma unroll
        for (int v = 0; v < RM; ++v) {
          float lo, hi;
          asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a[v][uc]));
          colk[buf][tr * RM + v] = (rown && v == ur) ? mk<float>(-1.f, 0.f) : mk<float>(lo, hi);
        }
        if (rown) {
          float lo, hi;
          asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a[ur][uc]));
          const c32 p = mk<float>(lo, hi);
          const float den = abs2(p);
          if (!(den > 0.f) || !(den < INFINITY)) atomicExch(err, LS_ESINGULAR);
          dk[buf] = inv(p);
        }
      }
      __syncthreads();
      const c32 d = dk[buf];
      unsigned long long R1[RN], R2[RN];
      const float4* rp = reinterpret_cast<const float4*>(&rowk[buf][tc * RN]);
#pragma unroll
      for (int v = 0; v < RN / 2; ++v) {
        const float4 q = rp[v];
        const c32 s0 = d * mk<float>(q.x, q.y), s1 = d * mk<float>(q.z, q.w);
        R1[2 * v] = pk2(s0.re, s0.im);
        R2[2 * v] = pk2(s0.im, s0.re);
        R1[2 * v + 1] = pk2(s1.re, s1.im);
        R2[2 * v + 1] = pk2(s1.im, s1.re);
      }
      if (rown) {
#pragma unroll
        for (int v = 0; v < RN; ++v) a[ur][v] = 0ull;
      }
      if (cown) {
#pragma unroll
        for (int v = 0; v < RM; ++v) a[v][uc] = 0ull;
      }
      const float4* cp = reinterpret_cast<const float4*>(&colk[buf][tr * RM]);
#pragma unroll
      for (int i2 = 0; i2 < RM / 2; ++i2) {
        const float4 q = cp[i2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float cre = h ? q.z : q.x, cim = h ? q.w : q.y;
          const unsigned long long C1 = pk2(-cre, -cre), C2 = pk2(cim, -cim);
#pragma unroll
          for (int j = 0; j < RN; ++j) a[2 * i2 + h][j] = ffma2(C1, R1[j], ffma2(C2, R2[j], a[2 * i2 + h][j]));
        }
      }
    }
  }
}

template <int TR, int TC, int RM, int RN>
__global__ void __launch_bounds__(TR * TC) gj2d_kernel(c32* __restrict__ X, int n, int lda, long long sX,
                                                       int* __restrict__ err) {
  const int tid = threadIdx.x, tc = tid % TC, tr = tid / TC;
  c32* M = X + blockIdx.x * sX;
  unsigned long long a[RM][RN];
#pragma unroll
  for (int i = 0; i < RM; ++i) {
    const int row = tr * RM + i;
#pragma unroll
    for (int j = 0; j < RN; ++j) {
      const int col = tc * RN + j;
      const c32 v = (row < n && col < n) ? M[(long long)row * lda + col] : mk<float>(0.f, 0.f);
      a[i][j] = pk2(v.re, v.im);
    }
  }
  gj2d_sweep<TR, TC, RM, RN>(a, n, tr, tc, err);
#pragma unroll
  for (int i = 0; i < RM; ++i) {
    const int row = tr * RM + i;
#pragma unroll
    for (int j = 0; j < RN; ++j) {
      const int col = tc * RN + j;
      if (row < n && col < n) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a[i][j]));
        M[(long long)row * lda + col] = mk<float>(lo, hi);
      }
    }
  }
}

// Panel kernel of the FP32 blocked sweep (one block of 16 x 16 threads per
// matrix, 4 x 4 entries each).  From the pending panel's A^-1 (Aip, w x w), Mb
// (Mbp, w x n) and Cb (Cbp, n x w) it forms
//   t  = A^-1 Mb[:, J]             (the columns J of the pending panel's Rb)
//   Ab = X[J, J] - Cb[J, :] t
// as two 64^3 products from shared memory (operands stored in the two packed
// forms of gemm64x2_kernel), zeroes X[J, J] (the pending update skips it; this
// panel's update writes A^-1 there) and inverts Ab in registers into Aout
// (w1 x w1).  With w = 0 it is Ab = X[J, J].  Dynamic shared memory:
// kPanelSmem bytes.
// PA rows are padded to 65 entries (its transposed stores then fall in distinct
// banks); PB stores column j of a row at slot (j % 4) * 16 + j / 4, so that the
// four columns tc * 4 + jj a thread reads are 16 slots apart and the 16
// threads of a half-warp read consecutive slots.
constexpr int kPanelNB = 64, kPanelLdA = kPanelNB + 1;
constexpr size_t kPanelSmem = sizeof(ulonglong2) * (kPanelLdA + kPanelNB) * kPanelNB;
__device__ __forceinline__ int panel_bslot(int j) { return (j & 3) * 16 + (j >> 2); }

__device__ __forceinline__ void panel_mma(const ulonglong2* __restrict__ PA, const ulonglong2* __restrict__ PB, int K,
                                          int tr, int tc, unsigned long long (&acc)[4][4]) {
#pragma unroll 2
  for (int q = 0; q < K; ++q) {
    ulonglong2 av[4], bv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) av[i] = PA[q * kPanelLdA + tr * 4 + i];
#pragma unroll
    for (int j = 0; j < 4; ++j) bv[j] = PB[q * kPanelNB + j * 16 + tc];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = ffma2(av[i].x, bv[j].x, ffma2(av[i].y, bv[j].y, acc[i][j]));
  }
}

__global__ void __launch_bounds__(256) gjb_panel_kernel(c32* __restrict__ X, int n, int lda, long long sX, int w,
                                                        const c32* __restrict__ Aip, const c32* __restrict__ Mbp,
                                                        const c32* __restrict__ Cbp, int k1, int w1,
                                                        c32* __restrict__ Aout, int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char panel_sm[];
  ulonglong2* PA = reinterpret_cast<ulonglong2*>(panel_sm);  // PA[q][i]: A operand entry (i, q)
  ulonglong2* PB = PA + kPanelLdA * kPanelNB;                // PB[q][slot(j)]: B operand entry (q, j)
  const int b = blockIdx.x, tid = threadIdx.x, tc = tid % 16, tr = tid / 16;
  c32* M = X + b * sX;
  unsigned long long a[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = tr * 4 + i, c = tc * 4 + j;
      c32 v = mk<float>(0.f, 0.f);
      if (r < w1 && c < w1) {
        c32* e = M + (long long)(k1 + r) * lda + k1 + c;
        v = *e;
        *e = mk<float>(0.f, 0.f);
      }
      a[i][j] = pk2(v.re, v.im);
    }
  if (w > 0) {
    const c32* aip = Aip + (long long)b * w * w;
    const c32* mbp = Mbp + (long long)b * w * n;
    const c32* cbp = Cbp + (long long)b * n * w;
    for (int t = tid; t < kPanelNB * kPanelNB; t += blockDim.x) {
      const int r = t / kPanelNB, c = t % kPanelNB;
      const c32 x = (r < w && c < w) ? aip[r * w + c] : mk<float>(0.f, 0.f);
      PA[c * kPanelLdA + r] = make_ulonglong2(pk2(x.re, x.re), pk2(-x.im, x.im));
      const c32 y = (r < w && c < w1) ? mbp[(long long)r * n + k1 + c] : mk<float>(0.f, 0.f);
      PB[r * kPanelNB + panel_bslot(c)] = make_ulonglong2(pk2(y.re, y.im), pk2(y.im, y.re));
    }
    __syncthreads();
    unsigned long long acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0ull;
    panel_mma(PA, PB, w, tr, tc, acc);  // t = A^-1 Mb[:, J]
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float re, im;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(re), "=f"(im) : "l"(acc[i][j]));
        PB[(tr * 4 + i) * kPanelNB + j * 16 + tc] = make_ulonglong2(pk2(re, im), pk2(im, re));
        acc[i][j] = 0ull;
      }
    for (int t = tid; t < kPanelNB * kPanelNB; t += blockDim.x) {
      const int r = t / kPanelNB, c = t % kPanelNB;
      const c32 x = (r < w1 && c < w) ? cbp[(long long)(k1 + r) * w + c] : mk<float>(0.f, 0.f);
      PA[c * kPanelLdA + r] = make_ulonglong2(pk2(x.re, x.re), pk2(-x.im, x.im));
    }
    __syncthreads();
    panel_mma(PA, PB, w, tr, tc, acc);  // Cb[J, :] t
    const unsigned long long mone2 = pk2(-1.f, -1.f);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) a[i][j] = ffma2(mone2, acc[i][j], a[i][j]);
  }
  gj2d_sweep<16, 16, 4, 4>(a, w1, tr, tc, err);
  c32* out = Aout + (long long)b * w1 * w1;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = tr * 4 + i, c = tc * 4 + j;
      if (r < w1 && c < w1) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a[i][j]));
        out[r * w1 + c] = mk<float>(lo, hi);
      }
    }
}

// Largest order handled by gj_reg_kernel (registers per thread: 2 CPT reals).
template <class R>
constexpr int gj_reg_max() {
  return sizeof(R) == 4 ? 128 : 64;
}

template <class R>
int invert_reg_nopiv(cx<R>* X, int n, int lda, long long sX, int P, int* err, cudaStream_t st) {
  if (n <= 0 || P <= 0) return LS_OK;
  const unsigned thr = (unsigned)(((n * 8 + 31) / 32) * 32);
  count_launch();
  if constexpr (sizeof(R) == 4) {
    if (n <= 32)
      gj2d_kernel<8, 8, 4, 4><<<P, 64, 0, st>>>(X, n, lda, sX, err);
    else if (n <= 64)
      gj2d_kernel<16, 16, 4, 4><<<P, 256, 0, st>>>(X, n, lda, sX, err);
    else if (n <= 96)
      gj2d_kernel<12, 24, 8, 4><<<P, 288, 0, st>>>(X, n, lda, sX, err);
    else if (n <= 128)
      gj2d_kernel<16, 32, 8, 4><<<P, 512, 0, st>>>(X, n, lda, sX, err);
    else
      return LS_EINVAL;
    return check_launch("gj2d");
  }
  if (n <= 32)
    gj_reg_kernel<R, 4><<<P, thr, 0, st>>>(X, n, lda, sX, err);
  else if (n <= 64)
    gj_reg_kernel<R, 8><<<P, thr, 0, st>>>(X, n, lda, sX, err);
  else if (sizeof(R) == 4 && n <= 96)
    gj_reg_kernel<R, 12><<<P, thr, 0, st>>>(X, n, lda, sX, err);
  else if (sizeof(R) == 4 && n <= 128)
    gj_reg_kernel<R, 16><<<P, thr, 0, st>>>(X, n, lda, sX, err);
  else
    return LS_EINVAL;
  return check_launch("gj_reg");
}

// Blocked Gauss-Jordan inversion, panel step (one block per matrix).  The nb
// <= 32 panel columns [k0, k0+nb) of all n rows are loaded to shared memory
// and eliminated in place with partial row pivoting over the rows not yet used
// as pivots.  Warp w owns rows i = w (mod 8), lane c owns panel column c.  On
// exit the panel holds the columns J of the accumulated transform (rows J:
// the pivot block's inverse), piv the row interchanges, and perm (2*nb
// (destination, source) row pairs, -1 terminated) their net permutation for
// gj_swap_extract_kernel.
template <class R>
__global__ void __launch_bounds__(256) gj_panel_kernel(cx<R>* X, int n, int lda, long long sX, int k0, int nb,
                                                       int* piv, int* perm, int* err) {
  extern __shared__ unsigned char smraw[];
  cx<R>* pn = reinterpret_cast<cx<R>*>(smraw);  // n x nb, row stride nb + 1 (no bank conflicts)
  const int ldp = nb + 1;
  __shared__ cx<R> prow[32];
  __shared__ R s_v[8];
  __shared__ int s_i[8];
  __shared__ int s_pos[64], s_org[64];
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned lmask = nb >= 32 ? 0xffffffffu : ((1u << nb) - 1u);
  cx<R>* M = X + b * sX;
  if (tid == 0) {  // valid (identity) interchanges even if the panel stops at a zero pivot
    for (int jj = 0; jj < nb; ++jj) piv[(long long)b * n + k0 + jj] = k0 + jj;
    perm[(long long)b * 2 * 64] = -1;
  }
  for (int i = warp; i < n; i += 8)
    if (lane < nb) pn[i * ldp + lane] = M[(long long)i * lda + k0 + lane];
  __syncthreads();
  for (int jj = 0; jj < nb; ++jj) {
    const int j = k0 + jj;
    R best = R(-1);
    int bi = n;
    for (int i = j + tid; i < n; i += blockDim.x) {
      R v = abs2(pn[i * ldp + jj]);
      if (v > best) {
        best = v;
        bi = i;
      }
    }
    for (int o = 16; o; o >>= 1) {
      R ob = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    if (lane == 0) {
      s_v[warp] = best;
      s_i[warp] = bi;
    }
    __syncthreads();
    best = s_v[0];
    bi = s_i[0];
    for (int w = 1; w < 8; ++w)
      if (s_v[w] > best || (s_v[w] == best && s_i[w] < bi)) {
        best = s_v[w];
        bi = s_i[w];
      }
    if (!(best > R(0))) {
      if (tid == 0) atomicExch(err, LS_ESINGULAR);
      return;  // every thread takes this branch
    }
    const int p = bi;
    const cx<R> d = inv(pn[p * ldp + jj]);
    if (tid == 0) piv[(long long)b * n + j] = p;
    if (warp == 0 && lane < nb) {
      cx<R> a = pn[j * ldp + lane], bv = pn[p * ldp + lane];
      prow[lane] = (lane == jj) ? d : bv * d;
      if (p != j) pn[p * ldp + lane] = a;
    }
    __syncthreads();
    for (int i = warp; i < n; i += 8) {
      if (lane >= nb) continue;
      if (i == j) {
        pn[i * ldp + lane] = prow[lane];
        continue;
      }
      cx<R> f = pn[i * ldp + jj];
      __syncwarp(lmask);
      if (lane == jj) {
        pn[i * ldp + lane] = mk<R>(-(f.re * d.re - f.im * d.im), -(f.re * d.im + f.im * d.re));
      } else {
        cx<R> r = prow[lane], v = pn[i * ldp + lane];
        v.re -= f.re * r.re - f.im * r.im;
        v.im -= f.re * r.im + f.im * r.re;
        pn[i * ldp + lane] = v;
      }
    }
    __syncthreads();
  }
  for (int i = warp; i < n; i += 8)
    if (lane < nb) M[(long long)i * lda + k0 + lane] = pn[i * ldp + lane];
  if (tid == 0) {  // net permutation of the panel's interchanges
    int cnt = 0;
    for (int jj = 0; jj < nb; ++jj) {
      int j = k0 + jj, p = piv[(long long)b * n + j];
      if (p == j) continue;
      int ij = -1, ip = -1;
      for (int t = 0; t < cnt; ++t) {
        if (s_pos[t] == j) ij = t;
        if (s_pos[t] == p) ip = t;
      }
      if (ij < 0) {
        s_pos[cnt] = j;
        s_org[cnt] = j;
        ij = cnt++;
      }
      if (ip < 0) {
        s_pos[cnt] = p;
        s_org[cnt] = p;
        ip = cnt++;
      }
      int t = s_org[ij];
      s_org[ij] = s_org[ip];
      s_org[ip] = t;
    }
    int* pr = perm + (long long)b * 2 * 64;
    for (int t = 0; t < cnt; ++t) {
      pr[2 * t] = s_pos[t];
      pr[2 * t + 1] = s_org[t];
    }
    if (cnt < 64) pr[2 * cnt] = -1;
  }
}

// Panel step of the blocked Gauss-Jordan inverse across a thread-block
// cluster: the CL blocks of a cluster share one matrix, block r keeping rows
// [r*rows_per, (r+1)*rows_per) of the n x nb panel in shared memory.  Per pivot
// column: local argmax, cluster barrier, every block reads the CL candidates
// through distributed shared memory and takes the same winner (largest |.|,
// lowest row on ties); the owners of the pivot row p and of row j publish the
// scaled pivot row and old row j; cluster barrier; every block eliminates its
// own rows.  Same result, piv and perm as gj_panel_kernel.
template <class R>
__global__ void __launch_bounds__(256) gj_panel_cluster_kernel(cx<R>* X, int n, int lda, long long sX, int k0, int nb,
                                                               int* piv, int* perm, int* err) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ unsigned char smraw[];
  const int CL = (int)cluster.num_blocks();
  const int crank = (int)cluster.block_rank();
  const int mat = blockIdx.x / CL;
  const int rows_per = (n + CL - 1) / CL;
  const int r0 = min(n, crank * rows_per), r1 = min(n, r0 + rows_per);
  const int ldp = nb + 1;
  cx<R>* pn = reinterpret_cast<cx<R>*>(smraw);  // (r1 - r0) x nb, stride nb + 1
  __shared__ cx<R> s_prow[32], s_oldj[32], l_prow[32], l_oldj[32];
  __shared__ R s_v[8];
  __shared__ int s_i[8];
  __shared__ R s_best;
  __shared__ int s_bidx;
  __shared__ int s_pos[64], s_org[64];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned lmask = nb >= 32 ? 0xffffffffu : ((1u << nb) - 1u);
  cx<R>* M = X + mat * sX;
  if (crank == 0 && tid == 0) {  // valid (identity) interchanges even if the panel stops at a zero pivot
    for (int jj = 0; jj < nb; ++jj) piv[(long long)mat * n + k0 + jj] = k0 + jj;
    perm[(long long)mat * 2 * 64] = -1;
  }
  for (int i = r0 + warp; i < r1; i += 8)
    if (lane < nb) pn[(i - r0) * ldp + lane] = M[(long long)i * lda + k0 + lane];
  __syncthreads();
  for (int jj = 0; jj < nb; ++jj) {
    const int j = k0 + jj;
    R best = R(-1);
    int bi = n;
    for (int i = max(j, r0) + tid; i < r1; i += blockDim.x) {
      R v = abs2(pn[(i - r0) * ldp + jj]);
      if (v > best) {
        best = v;
        bi = i;
      }
    }
    for (int o = 16; o; o >>= 1) {
      R ob = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    if (lane == 0) {
      s_v[warp] = best;
      s_i[warp] = bi;
    }
    __syncthreads();
    if (tid == 0) {
      R bb = s_v[0];
      int ii = s_i[0];
      for (int w = 1; w < 8; ++w)
        if (s_v[w] > bb || (s_v[w] == bb && s_i[w] < ii)) {
          bb = s_v[w];
          ii = s_i[w];
        }
      s_best = bb;
      s_bidx = ii;
    }
    cluster.sync();
    best = R(-1);
    bi = n;
    for (int r = 0; r < CL; ++r) {
      R ob = *cluster.map_shared_rank(&s_best, r);
      int oi = *cluster.map_shared_rank(&s_bidx, r);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    if (!(best > R(0))) {
      if (tid == 0 && crank == 0) atomicExch(err, LS_ESINGULAR);
      return;  // every thread of every block of the cluster takes this branch
    }
    const int p = bi;
    const int own_p = p / rows_per, own_j = j / rows_per;
    if (crank == 0 && tid == 0) piv[(long long)mat * n + j] = p;
    if (crank == own_p && warp == 0 && lane < nb) {
      cx<R> dd = inv(pn[(p - r0) * ldp + jj]);
      s_prow[lane] = (lane == jj) ? dd : pn[(p - r0) * ldp + lane] * dd;
    }
    if (crank == own_j && warp == 1 && lane < nb) s_oldj[lane] = pn[(j - r0) * ldp + lane];
    cluster.sync();
    if (warp == 0 && lane < nb) l_prow[lane] = *cluster.map_shared_rank(&s_prow[lane], own_p);
    if (warp == 1 && lane < nb && p != j && p >= r0 && p < r1)
      l_oldj[lane] = *cluster.map_shared_rank(&s_oldj[lane], own_j);
    __syncthreads();
    const cx<R> d = l_prow[jj];
    for (int i = r0 + warp; i < r1; i += 8) {
      if (lane >= nb) continue;
      cx<R>* row = pn + (i - r0) * ldp;
      if (i == j) {
        row[lane] = l_prow[lane];
        continue;
      }
      const bool moved = (i == p);  // old row j lands at position p
      cx<R> f = moved ? l_oldj[jj] : row[jj];
      cx<R> v = moved ? l_oldj[lane] : row[lane];
      __syncwarp(lmask);
      if (lane == jj) {
        row[lane] = mk<R>(-(f.re * d.re - f.im * d.im), -(f.re * d.im + f.im * d.re));
      } else {
        cx<R> r = l_prow[lane];
        v.re -= f.re * r.re - f.im * r.im;
        v.im -= f.re * r.im + f.im * r.re;
        row[lane] = v;
      }
    }
    __syncthreads();
  }
  for (int i = r0 + warp; i < r1; i += 8)
    if (lane < nb) M[(long long)i * lda + k0 + lane] = pn[(i - r0) * ldp + lane];
  if (crank == 0 && tid == 0) {  // net permutation of the panel's interchanges
    int cnt = 0;
    for (int jj = 0; jj < nb; ++jj) {
      int j = k0 + jj, p = piv[(long long)mat * n + j];
      if (p == j) continue;
      int ij = -1, ip = -1;
      for (int t = 0; t < cnt; ++t) {
        if (s_pos[t] == j) ij = t;
        if (s_pos[t] == p) ip = t;
      }
      if (ij < 0) {
        s_pos[cnt] = j;
        s_org[cnt] = j;
        ij = cnt++;
      }
      if (ip < 0) {
        s_pos[cnt] = p;
        s_org[cnt] = p;
        ip = cnt++;
      }
      int t = s_org[ij];
      s_org[ij] = s_org[ip];
      s_org[ip] = t;
    }
    int* pr = perm + (long long)mat * 2 * 64;
    for (int t = 0; t < cnt; ++t) {
      pr[2 * t] = s_pos[t];
      pr[2 * t + 1] = s_org[t];
    }
    if (cnt < 64) pr[2 * cnt] = -1;
  }
  cluster.sync();  // no block leaves while others may still read its shared memory
}

// For every column c outside the panel: apply the panel's net row
// permutation, move rows J = [k0, k0+nb) to Mb (nb x n) and zero them in X, so
// that X[:, c] += Panel * Mb[:, c] completes the step.
template <class R>
__global__ void gj_swap_extract_kernel(cx<R>* X, int n, int lda, long long sX, int k0, int nb, const int* perm,
                                       cx<R>* Mb, long long sM) {
  const int b = blockIdx.y;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n || (c >= k0 && c < k0 + nb)) return;
  cx<R>* M = X + b * sX;
  cx<R>* out = Mb + b * sM;
  const int* pr = perm + (long long)b * 2 * 64;
  cx<R> vals[64];
  int cnt = 0;
  for (; cnt < 64 && pr[2 * cnt] >= 0 && pr[2 * cnt] < n && (unsigned)pr[2 * cnt + 1] < (unsigned)n; ++cnt)
    vals[cnt] = M[(long long)pr[2 * cnt + 1] * lda + c];
  for (int t = 0; t < cnt; ++t) M[(long long)pr[2 * t] * lda + c] = vals[t];
  for (int jj = 0; jj < nb; ++jj) {
    out[(long long)jj * n + c] = M[(long long)(k0 + jj) * lda + c];
    M[(long long)(k0 + jj) * lda + c] = mk<R>(0, 0);
  }
}

// Undo the row pivoting by column interchanges in reverse pivot order, in
// place, one block per (row chunk, matrix).
template <class R>
__global__ void unpivot_rows_kernel(cx<R>* X, int n, int lda, long long sX, const int* piv, int rows_per) {
  extern __shared__ unsigned char smraw[];
  int* idx = reinterpret_cast<int*>(smraw);
  cx<R>* row = reinterpret_cast<cx<R>*>(idx + ((n + 3) & ~3));
  const int b = blockIdx.y;
  for (int j = threadIdx.x; j < n; j += blockDim.x) idx[j] = j;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int k = n - 1; k >= 0; --k) {
      int p = piv[(long long)b * n + k];
      if ((unsigned)p >= (unsigned)n) p = k;
      int t = idx[k];
      idx[k] = idx[p];
      idx[p] = t;
    }
  __syncthreads();
  cx<R>* M = X + b * sX;
  const int r0 = blockIdx.x * rows_per, r1 = min(n, r0 + rows_per);
  for (int r = r0; r < r1; ++r) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) row[j] = M[(long long)r * lda + j];
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) M[(long long)r * lda + j] = row[idx[j]];
    __syncthreads();
  }
}

template <class R>
__global__ void set_identity_kernel(cx<R>* X, int n, int lda, long long sX, int P) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)P * n * n) return;
  long long b = t / ((long long)n * n);
  int i = (int)((t / n) % n), j = (int)(t % n);
  X[b * sX + (long long)i * lda + j] = mk<R>(i == j ? R(1) : R(0), R(0));
}

// In-place inverse of P matrices (n x n, row stride lda, batch stride sX).
// Small n: one block per matrix in shared memory.  Larger n: blocked
// Gauss-Jordan, nb columns per panel; each panel is one panel kernel, one
// interchange/extract kernel and one batched GEMM X += Panel * Mb, so the
// O(n^3) work is in the GEMM.
// Blocked Gauss-Jordan without interchanges (the merge matrices are I plus a
// perturbation, Sec. 4.3; a probe check decides whether the pivoted sweep is
// needed).  Per diagonal block J of width w: A = X[J,J], A^-1 in registers,
// then one rank-w update of all of X.
// Lookahead form of the blocked Gauss-Jordan sweep.  Panel J = [k0, k0 + w)
// leaves Cb (n x w: X[:, J] with rows J set to -I) and Rb = A^-1 Mb (w x n:
// the rows X[J, :] with columns J set to I, so Rb[:, J] = A^-1); with X[J, :]
// and X[:, J] zeroed when they were read, the single update X -= Cb Rb writes
// X[J, :] = Rb, X[:, J] = -Cb A^-1 and the Schur complement elsewhere.  That
// update skips the rows and columns of the next panel J' = [k1, k1 + w1),
// whose operands are formed with it applied on the fly:
//   Ab = X[J', J'] - Cb[J', :] Rb[:, J']                 (gjb_diag_kernel)
//   Mb = X[J', :] - Cb[J', :] Rb, columns J' set to I    (gjb_extract_kernel)
//   Cb' = X[:, J'] - Cb Rb[:, J'], rows J' set to -I
// With w = 0 (the first panel) there is no pending update.
template <class R>
__global__ void gjb_diag_kernel(const cx<R>* __restrict__ X, int n, int lda, long long sX, int w,
                                const cx<R>* __restrict__ Cbp, const cx<R>* __restrict__ Rbp, int k1, int w1,
                                cx<R>* __restrict__ Ab) {
  const int b = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= w1 * w1) return;
  const int r = t / w1, q = t % w1;
  const cx<R>* crow = Cbp + (long long)b * n * w + (long long)(k1 + r) * w;
  const cx<R>* rcol = Rbp + (long long)b * w * n + k1 + q;
  cx<R> acc = mk<R>(0, 0);
#pragma unroll 8
  for (int p = 0; p < w; ++p) fma_(acc, crow[p], rcol[(long long)p * n]);
  Ab[(long long)b * w1 * w1 + t] = X[b * sX + (long long)(k1 + r) * lda + k1 + q] - acc;
}

// Mb and Cb' of panel J' (above); X[J', :] and X[:, J'] are zeroed once read
// (X[J', J'] only with zero_diag: the FP32 panel kernel zeroes it itself).
// The pending update skips these rows and columns, and each element is read
// and zeroed by the same thread, so the kernel may run beside that update.
template <class R>
__global__ void gjb_extract_kernel(cx<R>* __restrict__ X, int n, int lda, long long sX, int w,
                                   const cx<R>* __restrict__ Cbp, const cx<R>* __restrict__ Rbp, int k1, int w1,
                                   cx<R>* __restrict__ Mb, cx<R>* __restrict__ Cb, int zero_diag) {
  const int b = blockIdx.y;
  cx<R>* M = X + b * sX;
  const cx<R>* cbp = Cbp + (long long)b * n * w;  // n x w
  const cx<R>* rbp = Rbp + (long long)b * w * n;  // w x n
  const long long t1 = (long long)w1 * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < 2 * t1;
       t += (long long)gridDim.x * blockDim.x) {
    if (t < t1) {  // Mb: row r of J', column c
      const int r = (int)(t / n), c = (int)(t % n);
      cx<R> v;
      const bool diag = c >= k1 && c < k1 + w1;
      if (diag) {
        v = mk<R>(c - k1 == r ? R(1) : R(0), R(0));
      } else {
        const cx<R>* crow = cbp + (long long)(k1 + r) * w;
        cx<R> acc = mk<R>(0, 0);
#pragma unroll 8
        for (int q = 0; q < w; ++q) fma_(acc, crow[q], rbp[(long long)q * n + c]);
        v = M[(long long)(k1 + r) * lda + c] - acc;
      }
      if (!diag || zero_diag) M[(long long)(k1 + r) * lda + c] = mk<R>(0, 0);
      Mb[b * t1 + t] = v;
    } else {  // Cb': row i, column q of J'
      const long long u = t - t1;
      const int i = (int)(u / w1), q = (int)(u % w1);
      cx<R> v;
      if (i >= k1 && i < k1 + w1) {
        v = mk<R>(i - k1 == q ? R(-1) : R(0), R(0));
      } else {
        const cx<R>* crow = cbp + (long long)i * w;
        cx<R> acc = mk<R>(0, 0);
#pragma unroll 8
        for (int p = 0; p < w; ++p) fma_(acc, crow[p], rbp[(long long)p * n + k1 + q]);
        v = M[(long long)i * lda + k1 + q] - acc;
        M[(long long)i * lda + k1 + q] = mk<R>(0, 0);
      }
      Cb[b * t1 + u] = v;
    }
  }
}

// Probe check of an inverse W of Z = I - Y2 Y1 with a fixed vector v of
// unit-modulus entries: r = Z (W v) - v, formed with the batched GEMV kernels;
// probe_max_kernel folds max_i |r_i| over all matrices into *worst (float bits,
// atomicMax on non-negative floats; NaN or overflow counts as 3e38).
template <class R>
__global__ void probe_vector_kernel(cx<R>* v, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float a = 0.7548776662f * (float)(i + 1);
  a -= floorf(a);
  v[i] = mk<R>((R)cospif(2.f * a), (R)sinpif(2.f * a));
}

template <class R>
__global__ void probe_max_kernel(const cx<R>* r, const cx<R>* v, int n, long long total, int* worst) {
  float mx = 0.f;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    cx<R> e = r[t] - v[t % n];
    float x = (float)sqrt(abs2(e));
    if (!(x <= 3e38f)) x = 3e38f;
    mx = fmaxf(mx, x);
  }
  for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0.f) atomicMax(worst, __float_as_int(mx));
}

// dst[b] (rows x cols, row stride ldd) = src[b] (row stride lds), one grid row per matrix b.
template <class R>
__global__ void copy_block_kernel(cx<R>* dst, int ldd, long long sD, const cx<R>* src, int lds, long long sS, int rows,
                                  int cols) {
  const int b = blockIdx.y;
  const long long tot = (long long)rows * cols;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t / cols), j = (int)(t % cols);
    dst[b * sD + (long long)i * ldd + j] = src[b * sS + (long long)i * lds + j];
  }
}

template <class R>
void gemv(cudaStream_t st, bool ta, int M, int K, cx<R> alpha, const cx<R>* A, int lda, long long sA, const cx<R>* x,
          long long sx, cx<R> beta, cx<R>* y, long long sy, int batch);

// FP32 form of the lookahead sweep: the chain (st) is one panel kernel per
// panel, which forms its diagonal block from the pending panel's A^-1, Mb and
// Cb itself; on se, each panel's Mb and Cb (beside its panel kernel) and then
// Rb = A^-1 Mb; on sb, its update X -= Cb Rb, which skips the next panel's rows
// and columns.  Buffers alternate by panel parity.
int invert_batch_nopiv_f32(ls_handle* H, c32* X, int n, int lda, long long sX, int P, void* scratch,
                           size_t scratch_bytes, cudaStream_t st) {
  const int nb = kPanelNB, np = (n + nb - 1) / nb;
  const size_t wm = nb;
  if (sizeof(c32) * (size_t)P * (2 * wm * wm + 6 * wm * (size_t)n) > scratch_bytes) return LS_ENOMEM;
  c32* p = reinterpret_cast<c32*>(scratch);
  c32 *Ab[2], *Cb[2], *Rb[2], *Mb[2];
  for (int q = 0; q < 2; ++q) {
    Ab[q] = p;
    p += (size_t)P * wm * wm;
    Cb[q] = p;
    p += (size_t)P * wm * n;
    Rb[q] = p;
    p += (size_t)P * wm * n;
    Mb[q] = p;
    p += (size_t)P * wm * n;
  }
  if (!H->inv_stream) LS_CUDA_TRY(cudaStreamCreateWithFlags(&H->inv_stream, cudaStreamNonBlocking));
  if (!H->ext_stream) LS_CUDA_TRY(cudaStreamCreateWithFlags(&H->ext_stream, cudaStreamNonBlocking));
  LS_CUDA_TRY(cudaFuncSetAttribute(gjb_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPanelSmem));
  cudaStream_t sb = H->inv_stream, se = H->ext_stream;
  std::vector<cudaEvent_t> evG(np), evE(np), evR(np), evU(np);
  cudaEvent_t ev0;
  LS_CUDA_TRY(cudaEventCreateWithFlags(&ev0, cudaEventDisableTiming));
  for (int i = 0; i < np; ++i) {
    LS_CUDA_TRY(cudaEventCreateWithFlags(&evG[i], cudaEventDisableTiming));
    LS_CUDA_TRY(cudaEventCreateWithFlags(&evE[i], cudaEventDisableTiming));
    LS_CUDA_TRY(cudaEventCreateWithFlags(&evR[i], cudaEventDisableTiming));
    LS_CUDA_TRY(cudaEventCreateWithFlags(&evU[i], cudaEventDisableTiming));
  }
  struct Events {
    std::vector<cudaEvent_t>* v[4];
    cudaEvent_t e;
    ~Events() {
      for (auto* a : v)
        for (auto x : *a) cudaEventDestroy(x);
      cudaEventDestroy(e);
    }
  } events{{&evG, &evE, &evR, &evU}, ev0};
  LS_CUDA_TRY(cudaEventRecord(ev0, st));
  LS_CUDA_TRY(cudaStreamWaitEvent(se, ev0, 0));
  LS_CUDA_TRY(cudaStreamWaitEvent(sb, ev0, 0));
  const c32 one1 = mk<float>(1.f, 0.f), zero1 = mk<float>(0.f, 0.f), mone = mk<float>(-1.f, 0.f);
  for (int i = 0; i < np; ++i) {
    const int k1 = i * nb, w1 = std::min(nb, n - k1), par = i & 1;
    const int w = i > 0 ? nb : 0;  // the pending panel (all but the last are full)
    const long long t1 = (long long)n * w1;
    // chain: X[J, J] after panel i-2's update; the pending panel's Mb and Cb
    if (i >= 2) LS_CUDA_TRY(cudaStreamWaitEvent(st, evU[i - 2], 0));
    if (i >= 1) LS_CUDA_TRY(cudaStreamWaitEvent(st, evE[i - 1], 0));
    count_launch();
    gjb_panel_kernel<<<P, 256, kPanelSmem, st>>>(X, n, lda, sX, w, Ab[par ^ 1], Mb[par ^ 1], Cb[par ^ 1], k1, w1,
                                                 Ab[par], H->d_err + 3);
    LS_CUDA_TRY(cudaEventRecord(evG[i], st));
    // operands: X[J, :] and X[:, J] after panel i-2's update
    if (i >= 2) LS_CUDA_TRY(cudaStreamWaitEvent(se, evU[i - 2], 0));
    dim3 g((unsigned)std::min<long long>(1024, (2 * t1 + 255) / 256), P);
    count_launch();
    gjb_extract_kernel<float><<<g, 256, 0, se>>>(X, n, lda, sX, w, Cb[par ^ 1], Rb[par ^ 1], k1, w1, Mb[par],
                                                 Cb[par], 0);
    LS_CUDA_TRY(cudaEventRecord(evE[i], se));
    LS_CUDA_TRY(cudaStreamWaitEvent(se, evG[i], 0));
    gemm<float>(se, false, false, w1, n, w1, one1, Ab[par], w1, (long long)w1 * w1, Mb[par], n, t1, zero1, Rb[par],
                n, t1, P);
    LS_CUDA_TRY(cudaEventRecord(evR[i], se));
    // update, leaving the next panel's rows and columns to its own kernels
    LS_CUDA_TRY(cudaStreamWaitEvent(sb, evR[i], 0));
    Band band;
    if (i + 1 < np) {
      band.lo = k1 + w1;
      band.hi = std::min(n, k1 + w1 + nb);
    }
    gemm<float>(sb, false, false, n, n, w1, mone, Cb[par], w1, t1, Rb[par], n, t1, one1, X, lda, sX, P, band);
    LS_CUDA_TRY(cudaEventRecord(evU[i], sb));
  }
  LS_CUDA_TRY(cudaStreamWaitEvent(st, evU[np - 1], 0));
  return check_launch("inverse_blocked_nopiv");
}

template <class R>
int invert_batch_nopiv(ls_handle* H, cx<R>* X, int n, int lda, long long sX, int P, void* scratch,
                       size_t scratch_bytes, cudaStream_t st) {
  if constexpr (sizeof(R) == 4)
    return invert_batch_nopiv_f32(H, reinterpret_cast<c32*>(X), n, lda, sX, P, scratch, scratch_bytes, st);
  // Blocked Gauss-Jordan sweep over 64-wide panels with one panel of lookahead
  // on three streams.  On st (the chain): panel i's diagonal block with panel
  // i-1's pending update applied, its inverse, and Rb = A^-1 Mb.  On se: panel
  // i's Mb and Cb (beside the inverse).  On sb: panel i's update X -= Cb Rb,
  // which skips panel i+1's rows and columns, so that panel i+1's chain runs
  // beside it.  Panel buffers alternate by parity.
  const int nb = 64;  // panel width: a 64-wide panel inverse takes ~1/4 the time of a 128-wide one
  const int np = (n + nb - 1) / nb;
  const size_t wm = nb;
  if (sizeof(cx<R>) * (size_t)P * (2 * wm * wm + 5 * wm * (size_t)n) > scratch_bytes) return LS_ENOMEM;
  cx<R>* p = reinterpret_cast<cx<R>*>(scratch);
  cx<R>* Ab[2];
  cx<R>* Cb[2];
  cx<R>* Rb[2];
  for (int q = 0; q < 2; ++q) {
    Ab[q] = p;
    p += (size_t)P * wm * wm;
    Cb[q] = p;
    p += (size_t)P * wm * n;
    Rb[q] = p;
    p += (size_t)P * wm * n;
  }
  cx<R>* Mb = p;
  if (!H->inv_stream) LS_CUDA_TRY(cudaStreamCreateWithFlags(&H->inv_stream, cudaStreamNonBlocking));
  if (!H->ext_stream) LS_CUDA_TRY(cudaStreamCreateWithFlags(&H->ext_stream, cudaStreamNonBlocking));
  cudaStream_t sb = H->inv_stream, se = H->ext_stream;
  std::vector<cudaEvent_t> evA(np), evE(np), evR(np), evU(np);
  cudaEvent_t ev0;
  LS_CUDA_TRY(cudaEventCreateWithFlags(&ev0, cudaEventDisableTiming));
  for (int i = 0; i < np; ++i) {
    LS_CUDA_TRY(cudaEventCreateWithFlags(&evA[i], cudaEventDisableTiming));
    LS_CUDA_TRY(cudaEventCreateWithFlags(&evE[i], cudaEventDisableTiming));
    LS_CUDA_TRY(cudaEventCreateWithFlags(&evR[i], cudaEventDisableTiming));
    LS_CUDA_TRY(cudaEventCreateWithFlags(&evU[i], cudaEventDisableTiming));
  }
  struct Events {
    std::vector<cudaEvent_t>* v[4];
    cudaEvent_t e;
    ~Events() {
      for (auto* a : v)
        for (auto x : *a) cudaEventDestroy(x);
      cudaEventDestroy(e);
    }
  } events{{&evA, &evE, &evR, &evU}, ev0};
  LS_CUDA_TRY(cudaEventRecord(ev0, st));
  LS_CUDA_TRY(cudaStreamWaitEvent(sb, ev0, 0));
  const cx<R> mone = mk<R>(R(-1), R(0));
  for (int i = 0; i < np; ++i) {
    const int k1 = i * nb, w1 = std::min(nb, n - k1), par = i & 1;
    const int w = i > 0 ? nb : 0;  // the pending panel (all but the last are full)
    const long long t1 = (long long)n * w1;
    if (i >= 2) LS_CUDA_TRY(cudaStreamWaitEvent(st, evU[i - 2], 0));  // X after panel i-2; its buffers free
    count_launch();
    gjb_diag_kernel<R><<<dim3((unsigned)((w1 * w1 + 255) / 256), P), 256, 0, st>>>(
        X, n, lda, sX, w, Cb[par ^ 1], Rb[par ^ 1], k1, w1, Ab[par]);
    LS_CUDA_TRY(cudaEventRecord(evA[i], st));
    LS_CUDA_TRY(cudaStreamWaitEvent(se, evA[i], 0));
    dim3 g((unsigned)std::min<long long>(1024, (2 * t1 + 255) / 256), P);
    count_launch();
    gjb_extract_kernel<R><<<g, 256, 0, se>>>(X, n, lda, sX, w, Cb[par ^ 1], Rb[par ^ 1], k1, w1, Mb, Cb[par], 1);
    LS_CUDA_TRY(cudaEventRecord(evE[i], se));
    int rc = invert_reg_nopiv<R>(Ab[par], w1, w1, (long long)w1 * w1, P, H->d_err + 3, st);
    if (rc) return rc;
    LS_CUDA_TRY(cudaStreamWaitEvent(st, evE[i], 0));
    gemm<R>(st, false, false, w1, n, w1, one<R>(), Ab[par], w1, (long long)w1 * w1, Mb, n, t1, zero<R>(), Rb[par], n,
            t1, P);
    LS_CUDA_TRY(cudaEventRecord(evR[i], st));
    LS_CUDA_TRY(cudaStreamWaitEvent(sb, evR[i], 0));
    Band band;  // the next panel's rows and columns: its operands carry this update
    if (i + 1 < np) {
      band.lo = k1 + w1;
      band.hi = std::min(n, k1 + w1 + nb);
    }
    gemm<R>(sb, false, false, n, n, w1, mone, Cb[par], w1, t1, Rb[par], n, t1, one<R>(), X, lda, sX, P, band);
    LS_CUDA_TRY(cudaEventRecord(evU[i], sb));
  }
  LS_CUDA_TRY(cudaStreamWaitEvent(st, evU[np - 1], 0));
  return check_launch("inverse_blocked_nopiv");
}

template <class R>
int invert_batch(ls_handle* H, cx<R>* X, int n, int lda, long long sX, int P, void* scratch, size_t scratch_bytes,
                 cudaStream_t st) {
  const size_t smem_small = sizeof(cx<R>) * ((size_t)n * (n + 1) + n) + sizeof(int) * n;
  if (smem_small <= 200 * 1024) {
    LS_CUDA_TRY(cudaFuncSetAttribute(inverse_smem_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem_small));
    count_launch();
    inverse_smem_kernel<R><<<P, 512, smem_small, st>>>(X, n, lda, sX, H->d_err);
    return check_launch("inverse_smem");
  }
  // clusters of CL blocks share one panel when the matrix is large enough; the
  // panel width nb (<= 32) is the largest whose rows fit the shared memory of the
  // kernel that will run (a block of the cluster holds n / CL rows)
  int CL = n >= 512 ? 16 : (n >= 256 ? 8 : 1);
  if (CL == 16 && cudaFuncSetAttribute(gj_panel_cluster_kernel<R>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                      cudaSuccess) {
    cudaGetLastError();
    CL = 8;
  }
  auto panel_smem = [&](int cl, int w) { return sizeof(cx<R>) * (size_t)((n + cl - 1) / cl) * (w + 1); };
  auto pick_nb = [&](int cl) {
    int w = 32;
    while (w > 4 && panel_smem(cl, w) > 200 * 1024) w >>= 1;
    return w;
  };
  int nb = pick_nb(CL);
  size_t smem_cl = panel_smem(CL, nb);
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  if (CL > 1) {
    LS_CUDA_TRY(cudaFuncSetAttribute(gj_panel_cluster_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem_cl));
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(P * CL);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem_cl;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, (void*)gj_panel_cluster_kernel<R>, &cfg) != cudaSuccess ||
        nclusters < 1) {
      cudaGetLastError();
      CL = 1;
    }
  }
  if (CL == 1) nb = pick_nb(1);
  const size_t smem_panel = panel_smem(1, nb);
  if (panel_smem(CL, nb) > 200 * 1024) {
    set_last_error_text("merge matrix too large for the panel kernel");
    return LS_EINVAL;
  }
  if (CL == 1)
    LS_CUDA_TRY(cudaFuncSetAttribute(gj_panel_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_panel));
  cx<R>* Mb = reinterpret_cast<cx<R>*>(scratch);
  int* piv = reinterpret_cast<int*>(Mb + (size_t)P * nb * n);
  int* perm = piv + (size_t)P * n;
  if (sizeof(cx<R>) * (size_t)P * nb * n + sizeof(int) * (size_t)P * (n + 128) > scratch_bytes) return LS_ENOMEM;
  for (int k0 = 0; k0 < n; k0 += nb) {
    const int w = std::min(nb, n - k0);
    count_launch();
    if (CL > 1) {
      LS_CUDA_TRY(cudaLaunchKernelEx(&cfg, gj_panel_cluster_kernel<R>, X, n, lda, sX, k0, w, piv, perm, H->d_err));
    } else {
      gj_panel_kernel<R><<<P, 256, smem_panel, st>>>(X, n, lda, sX, k0, w, piv, perm, H->d_err);
    }
    count_launch();
    gj_swap_extract_kernel<R><<<dim3((n + 127) / 128, P), 128, 0, st>>>(X, n, lda, sX, k0, w, perm, Mb,
                                                                       (long long)w * n);
    // X[:, c] += Panel (n x w, columns k0.. of X) * Mb[:, c] for the columns c outside the panel
    gemm<R>(st, false, false, n, k0, w, one<R>(), X + k0, lda, sX, Mb, n, (long long)w * n, one<R>(), X, lda, sX, P);
    gemm<R>(st, false, false, n, n - k0 - w, w, one<R>(), X + k0, lda, sX, Mb + k0 + w, n, (long long)w * n, one<R>(),
            X + k0 + w, lda, sX, P);
  }
  const int rows_per = 16;
  const size_t smem_u = sizeof(int) * ((n + 3) & ~3) + sizeof(cx<R>) * n;
  if (smem_u > 48 * 1024)
    LS_CUDA_TRY(cudaFuncSetAttribute(unpivot_rows_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_u));
  count_launch();
  unpivot_rows_kernel<R><<<dim3((n + rows_per - 1) / rows_per, P), 256, smem_u, st>>>(X, n, lda, sX, piv, rows_per);
  return check_launch("inverse_blocked");
}

TreeGeom make_geom(const ls_handle* H) {
  TreeGeom g;
  g.L = H->L;
  g.s = H->s;
  g.nx = H->grid.nx;
  g.ny = H->grid.ny;
  g.G = H->nprob;
  for (int l = 0; l < H->L; ++l) {
    g.cw[l] = H->lev[l + 1].w;
    g.ch[l] = H->lev[l + 1].h;
  }
  return g;
}

int apply_persistent_init(ls_handle* H, cudaStream_t st);
int level_transpose(ls_handle* H, int l, cudaStream_t st);
int lowrank_transpose(ls_handle* H, int l, cudaStream_t st);

// The apply's temporaries (one right-hand side: leaf blocks, per-level
// expansions) and the persistent apply's transposes and operation list, made at
// the end of the build rather than at the first apply.  Needs every level's
// ranks and factor pointers, not their contents; a second call does nothing.
template <class R>
int apply_prepare(ls_handle* H, cudaStream_t st) {
  if (H->work) return LS_OK;
  const int L = H->L, n = H->s * H->s;
  size_t vec = (size_t)2 * ((size_t)H->nprob << L) * n;
  for (int l = 1; l <= L; ++l) vec += (size_t)3 * ((size_t)H->nprob << l) * std::max(1, H->lev[l].k) * 2;
  for (int l = 0; l < L; ++l) vec += ((size_t)H->nprob << l) * 2 * std::max(0, H->lev[l].xr);  // Q_R x per node
  H->work_bytes = sizeof(cx<R>) * vec;
  int rc;
  if ((rc = dalloc(&H->work, H->work_bytes))) return rc;
  return apply_persistent_init(H, st);
}

// ------------------------------------------------- Woodbury form of the merge
// The sibling block of a level is close to low rank (its entries couple the
// skeletons of two adjacent boxes, mostly through their shared side; Sec. 4.1,
// the remark on Eq. (26)): G ~ L R^T with L, R of k x r, r ~ k/3, computed once
// per level by a row ID of G (rows as candidates, tolerance eps in the
// Frobenius norm): G ~ T G(J,:), L = T, R = G(J,:)^T.  Then G^T = R L^T, and
// with A1 = S_a L, A2 = S_b R, C1 = L^T A1, C2 = R^T A2 (r x r),
// M = (I - C2 C1)^-1, N = I + C1 M C2 = (I - C1 C2)^-1, the Woodbury identity
// turns the Schur form X = [[I + Y1 W Y2, -Y1 W], [-W Y2, W]] (Y1 = S_a G,
// Y2 = S_b G^T, W = (I - Y2 Y1)^-1) into
//   W = I + A2 (C1 M) R^T,  -Y1 W = -A1 M R^T,  -W Y2 = -A2 N L^T,
//   I + Y1 W Y2 = I + A1 (C2 N) L^T:
// one inverse of order r instead of k, and ~6 k^2 r + 6 k r^2 flops of
// products instead of ~6 k^3.  (The middle block of the paper's form carries
// the children's S matrices: I + QP = [[I, R^T S_b R], [L^T S_a L, I]] in this
// notation; C2 and C1 are its off-diagonal blocks.)

// R[i][j] = G[J[j]][i]: the rows J of G, transposed (k x r).
template <class R>
__global__ void gather_rows_t_kernel(const cx<R>* __restrict__ G, int k, const int* __restrict__ J, int r,
                                     cx<R>* __restrict__ Rt) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)k * r) return;
  const int i = (int)(t / r), j = (int)(t % r);
  Rt[t] = G[(long long)J[j] * k + i];
}

// Levels whose sibling block takes the Woodbury form: large enough that the
// products dominate, and a rank at most half the order (else the Schur form
// costs no more).
constexpr int kWoodburyMinRank = 48;
// Sibling blocks from this order on are factored from a random sketch (Sec. 2.1,
// the randomised ID): the row ID of Y = G Omega (k x s, Omega Gaussian) selects
// the same kind of skeleton rows J and interpolation matrix T as the ID of G
// itself (Y's rows are G's rows mixed by one fixed matrix), at s / k of the cost.
constexpr int kSketchMinRank = 1024;

// splitmix64 (Steele, Lea and Flood, 2014): a counter-based generator, one
// 64-bit output per index.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  unsigned long long z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Om[t] = complex Gaussian (Box-Muller on two 24-bit uniforms of splitmix64(seed + t)).
template <class R>
__global__ void gaussian_kernel(cx<R>* __restrict__ Om, long long n, unsigned long long seed) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const unsigned long long h = splitmix64(seed + (unsigned long long)t);
  const float u1 = ((float)(h >> 40) + 1.0f) * (1.0f / 16777216.0f);  // (0, 1]
  const float u2 = (float)(h & 0xFFFFFFull) * (1.0f / 16777216.0f);   // [0, 1)
  const float rad = sqrtf(-2.0f * logf(u1));
  float sn, cs;
  sincospif(2.0f * u2, &sn, &cs);
  Om[t] = mk<R>((R)(rad * cs), (R)(rad * sn));
}

// The sibling factorisations of even and odd levels may run on two threads.
std::mutex g_sibling_flops_mu;
void add_sibling_flops(ls_handle* H, double f) {
  std::lock_guard<std::mutex> lk(g_sibling_flops_mu);
  H->flops_sibling += f;
}

// L, R of level l's sibling block (once per level; lv.gr = -1 when the level
// keeps the Schur form).
template <class R>
int sibling_lowrank(ls_handle* H, int l, cudaStream_t st) {
  LevelData& lv = H->lev[l];
  if (lv.gr != 0) return LS_OK;
  const int k = lv.k;
  const int mode = H->opts.woodbury;  // 0 off, 1 where it pays, 2 every level with r < k
  if (mode == 0 || k == 0 || (mode == 1 && k < kWoodburyMinRank)) {
    lv.gr = -1;
    return LS_OK;
  }
  const size_t kk = (size_t)k * k;
  cx<R>* A = nullptr;
  cx<R>* T = nullptr;
  int* dJ = nullptr;
  int rc;
  struct Free {
    void** p[3];
    ~Free() {
      for (auto q : p)
        if (*q) dfree(*q);
    }
  } fr{{(void**)&A, (void**)&T, (void**)&dJ}};
  if ((rc = dalloc((void**)&T, sizeof(cx<R>) * kk))) return rc;
  int r = 0;
  std::vector<int> J;
  // sketch width: from the rank two levels below (the same cut direction; the
  // level between may still be in the making on another stream), scaled to
  // this order, with margin; no sketch where it would not be well below k
  int sw = 0;
  if (k >= kSketchMinRank) {
    double pred = 0;
    if (l + 2 <= H->L) {
      const LevelData& lo = H->lev[l + 2];
      if (lo.gr > 0 && lo.k > 0) pred = (double)lo.gr * k / lo.k;
    }
    if (pred > 0) sw = (int)std::min<double>(k, 1.2 * pred + 64);
    if (sw > 0.6 * k) sw = 0;
  }
  const int prev_engine = g_tc_engine;
  if (sw > 0) {
    cx<R>* Om = nullptr;
    cx<R>* Y = nullptr;
    const long long ks = (long long)k * sw;
    if ((rc = dalloc((void**)&Om, sizeof(cx<R>) * ks)) || (rc = dalloc((void**)&Y, sizeof(cx<R>) * ks))) {
      if (Om) dfree(Om);
      return rc;
    }
    count_launch();
    gaussian_kernel<R><<<(unsigned)((ks + 255) / 256), 256, 0, st>>>(Om, ks, 0x5EED0000ull + (unsigned long long)l);
    // the sketch on the handle's GEMM engine (its rounding is far below the tolerance);
    // the ID itself keeps the FP32 SIMT GEMMs (its residual decides the rank)
    g_tc_engine = tc_engine_of(H);
    gemm<R>(st, false, false, k, sw, k, one<R>(), reinterpret_cast<const cx<R>*>(lv.Gsib), k, 0, Om, sw, 0, zero<R>(),
            Y, sw, 0, 1);
    g_tc_engine = 0;
    rc = check_launch("sibling sketch");
    if (!rc) rc = blocked_row_id<R>(Y, k, sw, H->tol, st, nullptr, T, &r, &J);
    g_tc_engine = prev_engine;
    LS_CUDA_TRY(cudaStreamSynchronize(st));
    dfree(Om);
    dfree(Y);
    if (rc) return rc;
    add_sibling_flops(H, 8.0 * ks * k + 8.0 * ks * r);
    if (r > sw - 32) sw = 0;  // the sketch was too narrow for the rank: the ID of G itself
  }
  if (sw == 0) {
    if ((rc = dalloc((void**)&A, sizeof(cx<R>) * kk))) return rc;
    LS_CUDA_TRY(cudaMemcpyAsync(A, lv.Gsib, sizeof(cx<R>) * kk, cudaMemcpyDeviceToDevice, st));
    g_tc_engine = 0;
    rc = blocked_row_id<R>(A, k, k, H->tol, st, nullptr, T, &r, &J);
    g_tc_engine = prev_engine;
    if (rc) return rc;
    add_sibling_flops(H, 8.0 * kk * r);
  }
  if (r == 0 || (mode == 1 ? 2 * r > k : r >= k)) {
    lv.gr = -1;
    return LS_OK;
  }
  if ((rc = dalloc(&lv.GL, sizeof(cx<R>) * (size_t)k * r)) || (rc = dalloc(&lv.GR, sizeof(cx<R>) * (size_t)k * r)) ||
      (rc = dalloc((void**)&dJ, sizeof(int) * r)))
    return rc;
  int* pin = static_cast<int*>(pinned_scratch(sizeof(int) * r));
  if (!pin) return LS_ENOMEM;
  memcpy(pin, J.data(), sizeof(int) * r);
  LS_CUDA_TRY(cudaMemcpyAsync(dJ, pin, sizeof(int) * r, cudaMemcpyHostToDevice, st));
  LS_CUDA_TRY(cudaMemcpyAsync(lv.GL, T, sizeof(cx<R>) * (size_t)k * r, cudaMemcpyDeviceToDevice, st));
  count_launch();
  gather_rows_t_kernel<R><<<(unsigned)(((long long)k * r + 255) / 256), 256, 0, st>>>(
      reinterpret_cast<const cx<R>*>(lv.Gsib), k, dJ, r, reinterpret_cast<cx<R>*>(lv.GR));
  if ((rc = check_launch("sibling low-rank factors"))) return rc;
  LS_CUDA_TRY(cudaStreamSynchronize(st));  // pin and the temporaries are released on return
  lv.gr = r;
  if ((rc = lowrank_transpose(H, l, st))) return rc;
  return LS_OK;
}

// Batched inverse of P matrices Z (n x n, row stride lda, stride sZ) in place:
// without interchanges, probe-checked against a copy of Z, the row-pivoted
// inverse as fallback (and as the only path when merge_pivoting = 1).  The
// acceptance rule is the Schur form's: max_i |(Z W v - v)_i| <= max(tol, 10 u n).
template <class R>
int invert_checked(ls_handle* H, cx<R>* Z, int n, int lda, long long sZ, int P, void* scratch, size_t scratch_bytes,
                   cudaStream_t st) {
  if (H->opts.merge_pivoting == 1) return invert_batch<R>(H, Z, n, lda, sZ, P, scratch, scratch_bytes, st);
  const long long nn = (long long)n * n;
  cx<R>* Zc = reinterpret_cast<cx<R>*>(scratch);
  cx<R>* pv = Zc + (size_t)P * nn;  // v (n), then u, t (P n each)
  cx<R>* pu = pv + n;
  cx<R>* pt = pu + (size_t)P * n;
  void* scr2 = pt + (size_t)P * n;
  const size_t used = sizeof(cx<R>) * ((size_t)P * nn + n + 2 * (size_t)P * n);
  if (scratch_bytes < used + 256) {
    set_last_error_text("merge inverse scratch too small");
    return LS_EINVAL;
  }
  const size_t scr2_bytes = scratch_bytes - used;
  int rc;
  dim3 gc((unsigned)std::min<long long>(1024, (nn + 255) / 256), 1);
  for (int b0 = 0; b0 < P; b0 += kMaxGridYZ) {
    gc.y = std::min(kMaxGridYZ, P - b0);
    count_launch();
    copy_block_kernel<R><<<gc, 256, 0, st>>>(Zc + (size_t)b0 * nn, n, nn, Z + (size_t)b0 * sZ, lda, sZ, n, n);
  }
  LS_CUDA_TRY(cudaMemsetAsync(H->d_err + 2, 0, 2 * sizeof(int), st));
  if (n <= gj_reg_max<R>()) {
    if ((rc = invert_reg_nopiv<R>(Z, n, lda, sZ, P, H->d_err + 3, st))) return rc;
  } else {
    if ((rc = invert_batch_nopiv<R>(H, Z, n, lda, sZ, P, scr2, scr2_bytes, st))) return rc;
  }
  count_launch();
  probe_vector_kernel<R><<<(n + 255) / 256, 256, 0, st>>>(pv, n);
  gemv<R>(st, false, n, n, one<R>(), Z, lda, sZ, pv, 0, zero<R>(), pu, n, P);
  gemv<R>(st, false, n, n, one<R>(), Zc, n, nn, pu, n, zero<R>(), pt, n, P);
  count_launch();
  probe_max_kernel<R><<<64, 256, 0, st>>>(pt, pv, n, (long long)P * n, H->d_err + 2);
  int* flags = static_cast<int*>(pinned_scratch(2 * sizeof(int)));
  if (!flags) return LS_ENOMEM;
  LS_CUDA_TRY(cudaMemcpyAsync(flags, H->d_err + 2, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  LS_CUDA_TRY(cudaStreamSynchronize(st));
  float worst;
  memcpy(&worst, &flags[0], sizeof(float));
  H->probe_resid_max = std::max(H->probe_resid_max, (double)worst);
  const double unit = sizeof(R) == 4 ? 5.96e-8 : 1.11e-16;
  const double limit = std::max(H->tol, 10.0 * unit * n);
  if (flags[1] != 0 || !((double)worst <= limit)) {
    for (int b0 = 0; b0 < P; b0 += kMaxGridYZ) {
      gc.y = std::min(kMaxGridYZ, P - b0);
      count_launch();
      copy_block_kernel<R><<<gc, 256, 0, st>>>(Z + (size_t)b0 * sZ, lda, sZ, Zc + (size_t)b0 * nn, n, nn, n, n);
    }
    if ((rc = invert_batch<R>(H, Z, n, lda, sZ, P, scr2, scr2_bytes, st))) return rc;
    ++H->pivot_fallbacks;
  }
  return check_launch("merge inverse (checked)");
}

// X of the P parents of level l (children of rank kc, sibling factors of rank r)
// in the Woodbury form above, kept factored: X = I + P_L Q_R with
//   P_L = [[A1 (C2 N), -A1 M], [-A2 N, A2 (C1 M)]]   (2kc x 2r per node, in X)
//   Q_R = diag(L^T, R^T)                             (the level's shared L, R),
// since P_L Q_R = [[A1 C2 N L^T, -A1 M R^T], [-A2 N L^T, A2 C1 M R^T]] = X - I.
// The apply and the S products use the factors; no 2kc x 2kc block is formed
// (4 kc r entries per node instead of 4 kc^2).
template <class R>
int merge_woodbury(ls_handle* H, int l, cx<R>* X, const cx<R>* Sc, cudaStream_t st) {
  const LevelData& ch = H->lev[l + 1];
  const int P = H->nprob << l, kc = ch.k, n2 = 2 * kc, r = ch.gr, r2 = 2 * r;
  const long long sP = (long long)n2 * r2, kk = (long long)kc * kc, kr = (long long)kc * r, rr = (long long)r * r;
  const cx<R>* Lf = reinterpret_cast<const cx<R>*>(ch.GL);
  const cx<R>* Rf = reinterpret_cast<const cx<R>*>(ch.GR);
  // A1, A2 (kc x r each), C1, C2, M, N, T (r x r each), then the inverse's scratch
  const size_t inv_scr = sizeof(cx<R>) * (size_t)P * (2 * rr + 128 * 128 + 3 * 128 * (size_t)r + 4 * (size_t)r) +
                         sizeof(int) * (size_t)P * (4 * (size_t)r + 256) + (1 << 16);
  const size_t bytes = sizeof(cx<R>) * (size_t)P * (2 * kr + 5 * rr) + inv_scr;
  void* work = nullptr;
  int rc;
  if ((rc = dalloc(&work, bytes))) return rc;
  struct FreeOnExit {
    void* p;
    ~FreeOnExit() { dfree(p); }
  } free_work{work};
  cx<R>* A1 = reinterpret_cast<cx<R>*>(work);
  cx<R>* A2 = A1 + (size_t)P * kr;
  cx<R>* C1 = A2 + (size_t)P * kr;
  cx<R>* C2 = C1 + (size_t)P * rr;
  cx<R>* Mm = C2 + (size_t)P * rr;
  cx<R>* Nm = Mm + (size_t)P * rr;
  cx<R>* Tm = Nm + (size_t)P * rr;
  void* scratch = Tm + (size_t)P * rr;
  const cx<R> mone = mk<R>(R(-1), R(0)), on = one<R>(), ze = zero<R>();
  auto ident = [&](cx<R>* D, int n, int ld, long long sD) {
    const long long tot = (long long)P * n * n;
    count_launch();
    set_identity_kernel<R><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(D, n, ld, sD, P);
  };
  int tg = prof_begin(st);
  gemm<R>(st, false, false, kc, r, kc, on, Sc, kc, 2 * kk, Lf, r, 0, ze, A1, r, kr, P);       // A1 = S_a L
  gemm<R>(st, false, false, kc, r, kc, on, Sc + kk, kc, 2 * kk, Rf, r, 0, ze, A2, r, kr, P);  // A2 = S_b R
  gemm<R>(st, true, false, r, r, kc, on, Lf, r, 0, A1, r, kr, ze, C1, r, rr, P);              // C1 = L^T A1
  gemm<R>(st, true, false, r, r, kc, on, Rf, r, 0, A2, r, kr, ze, C2, r, rr, P);              // C2 = R^T A2
  ident(Mm, r, r, rr);
  gemm<R>(st, false, false, r, r, r, mone, C2, r, rr, C1, r, rr, on, Mm, r, rr, P);           // I - C2 C1
  if ((rc = check_launch("woodbury merge"))) return rc;
  prof_end(tg, PR_MERGE_GEMM, st, sizeof(cx<R>) * P * (2.0 * kk + 4.0 * kr + 3.0 * rr),
           P * 8.0 * (2.0 * kk * r + 2.0 * kr * r + (double)rr * r));
  int ti = prof_begin(st);
  if ((rc = invert_checked<R>(H, Mm, r, r, rr, P, scratch, inv_scr, st))) return rc;  // M
  prof_end(ti, PR_MERGE_INV, st, sizeof(cx<R>) * P * 2.0 * rr, P * 8.0 * (double)rr * r);
  if (l == 0) host_mark("root_inverse_checked");
  tg = prof_begin(st);
  cx<R>* PTL = X;                     // rows 0..kc, columns 0..r of P_L
  cx<R>* PTR = X + r;                 // rows 0..kc, columns r..2r
  cx<R>* PBL = X + (size_t)kc * r2;   // rows kc..2kc, columns 0..r
  cx<R>* PBR = PBL + r;               // rows kc..2kc, columns r..2r
  gemm<R>(st, false, false, r, r, r, on, Mm, r, rr, C2, r, rr, ze, Tm, r, rr, P);             // M C2
  ident(Nm, r, r, rr);
  gemm<R>(st, false, false, r, r, r, on, C1, r, rr, Tm, r, rr, on, Nm, r, rr, P);             // N = I + C1 M C2
  gemm<R>(st, false, false, r, r, r, on, C2, r, rr, Nm, r, rr, ze, Tm, r, rr, P);             // C2 N
  gemm<R>(st, false, false, kc, r, r, on, A1, r, kr, Tm, r, rr, ze, PTL, r2, sP, P);          // A1 C2 N
  gemm<R>(st, false, false, kc, r, r, mone, A1, r, kr, Mm, r, rr, ze, PTR, r2, sP, P);        // -A1 M
  gemm<R>(st, false, false, kc, r, r, mone, A2, r, kr, Nm, r, rr, ze, PBL, r2, sP, P);        // -A2 N
  gemm<R>(st, false, false, r, r, r, on, C1, r, rr, Mm, r, rr, ze, Tm, r, rr, P);             // C1 M
  gemm<R>(st, false, false, kc, r, r, on, A2, r, kr, Tm, r, rr, ze, PBR, r2, sP, P);          // A2 C1 M
  if ((rc = check_launch("woodbury merge factors"))) return rc;
  const double fl = 8.0 * (4.0 * rr * r + 4.0 * kr * r);
  prof_end(tg, PR_MERGE_GEMM, st, sizeof(cx<R>) * P * ((double)sP + 2.0 * kr), P * fl);
  H->flops_build += P * (fl + 8.0 * (2.0 * kk * r + 2.0 * kr * r + 2.0 * (double)rr * r));
  return LS_OK;
}

// out[b](i, :) = src[b](idx[i], :), i < nidx, rows of `cols` entries.
template <class R>
__global__ void gather_rows_kernel(const cx<R>* __restrict__ src, long long sS, int lds, const int* __restrict__ idx,
                                   int nidx, int cols, cx<R>* __restrict__ dst, long long sD, int ldd) {
  const int b = blockIdx.y;
  const long long tot = (long long)nidx * cols;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / cols), c = (int)(t % cols);
    dst[b * sD + (long long)i * ldd + c] = src[b * sS + (long long)idx[i] * lds + c];
  }
}

// out[b](i, c) = src[b](i, idx[c]), i < rows, c < nidx.
template <class R>
__global__ void gather_cols_kernel(const cx<R>* __restrict__ src, long long sS, int lds, const int* __restrict__ idx,
                                   int nidx, int rows, cx<R>* __restrict__ dst, long long sD, int ldd) {
  const int b = blockIdx.y;
  const long long tot = (long long)rows * nidx;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / nidx), c = (int)(t % nidx);
    dst[b * sD + (long long)i * ldd + c] = src[b * sS + (long long)i * lds + idx[c]];
  }
}

// The skeleton part of D[b] = diag(S_a, S_b) U (Sc[b] = S_a, S_b, kc x kc each;
// U(J, :) = I): D(i, c) = S_h(i - h kc, piv[c] - h kc) where row i and pivot
// piv[c] lie in the same half h, else 0.
template <class R>
__global__ void d_skeleton_kernel(const cx<R>* __restrict__ Sc, int kc, const int* __restrict__ piv, int kp,
                                  cx<R>* __restrict__ D) {
  const int b = blockIdx.y, n2 = 2 * kc;
  const long long tot = (long long)n2 * kp, kk = (long long)kc * kc;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / kp), c = (int)(t % kp);
    const int h = i >= kc, j = piv[c];
    D[b * tot + t] = (j >= kc) == (bool)h ? Sc[b * 2 * kk + h * kk + (long long)(i - h * kc) * kc + (j - h * kc)]
                                          : mk<R>(0, 0);
  }
}

// D[b] = diag(S_a, S_b) U (n2 x kp) for the ID's U of level l:
// D(:, c) picks column piv[c] of S_a or S_b, and the interpolation rows add
// S_h(:, J^c_h) U(J^c_h, :) -- products of order |J^c_h| instead of kc.
// Without the pivot list (a level kept uncompressed or restored without it)
// the two full products.
template <class R>
int su_product(ls_handle* H, int l, const cx<R>* Sc, int kc, int kp, cx<R>* D, int P, cudaStream_t st,
               double* flops) {
  const LevelData& lv = H->lev[l];
  const cx<R>* U = reinterpret_cast<const cx<R>*>(lv.U);
  const int n2 = 2 * kc;
  const long long kk = (long long)kc * kc;
  if ((int)lv.piv.size() != kp || lv.m != n2) {
    gemm<R>(st, false, false, kc, kp, kc, one<R>(), Sc, kc, 2 * kk, U, kp, 0, zero<R>(), D, kp, (long long)n2 * kp, P);
    gemm<R>(st, false, false, kc, kp, kc, one<R>(), Sc + kk, kc, 2 * kk, U + (size_t)kc * kp, kp, 0, zero<R>(),
            D + (size_t)kc * kp, kp, (long long)n2 * kp, P);
    *flops = P * 2.0 * 8 * (double)kc * kc * kp;
    return check_launch("S U");
  }
  // index list: piv (kp), then the top complement (columns of S_a), then the
  // bottom complement (columns of S_b)
  std::vector<int> idx(lv.piv);
  std::vector<char> in(n2, 0);
  for (int a : lv.piv) in[a] = 1;
  int nct = 0, ncb = 0;
  for (int i = 0; i < kc; ++i)
    if (!in[i]) {
      idx.push_back(i);
      ++nct;
    }
  for (int i = kc; i < n2; ++i)
    if (!in[i]) {
      idx.push_back(i - kc);
      ++ncb;
    }
  const int nc = nct + ncb;
  int* didx = nullptr;
  cx<R>* T = nullptr;  // U(J^c_top, :) then U(J^c_bot, :): nc x kp
  cx<R>* G = nullptr;  // S_a(:, J^c_top) then S_b(:, J^c_bot): P x kc x nc
  struct Free {
    void** p[3];
    ~Free() {
      for (auto q : p)
        if (*q) dfree(*q);
    }
  } fr{{(void**)&didx, (void**)&T, (void**)&G}};
  int rc;
  if ((rc = dalloc((void**)&didx, sizeof(int) * (kp + 2 * (size_t)nc + 1)))) return rc;
  if ((rc = dalloc((void**)&T, sizeof(cx<R>) * std::max<size_t>((size_t)nc * kp, 1)))) return rc;
  if ((rc = dalloc((void**)&G, sizeof(cx<R>) * std::max<size_t>((size_t)P * kc * nc, 1)))) return rc;
  // U's rows of the complement, as row indices of U (the bottom ones shifted back by kc)
  for (int i = 0; i < nc; ++i) idx.push_back(idx[kp + i] + (i >= nct ? kc : 0));
  // pageable source: the call returns once the indices are staged
  LS_CUDA_TRY(cudaMemcpyAsync(didx, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice, st));
  const int* dpiv = didx;
  const int* dct = didx + kp;
  const int* dcb = dct + nct;
  const int* drow = didx + kp + nc;
  for (int b0 = 0; b0 < P; b0 += kMaxGridYZ) {
    const int nb = std::min(kMaxGridYZ, P - b0);
    const dim3 g((unsigned)std::min<long long>(1024, ((long long)n2 * kp + 255) / 256), nb);
    count_launch();
    d_skeleton_kernel<R><<<g, 256, 0, st>>>(Sc + (size_t)b0 * 2 * kk, kc, dpiv, kp, D + (size_t)b0 * n2 * kp);
    if (nc > 0) {
      const dim3 gg((unsigned)std::min<long long>(1024, ((long long)kc * nc + 255) / 256), nb);
      if (nct > 0) {
        count_launch();
        gather_cols_kernel<R><<<gg, 256, 0, st>>>(Sc + (size_t)b0 * 2 * kk, 2 * kk, kc, dct, nct, kc,
                                                  G + (size_t)b0 * kc * nc, (long long)kc * nc, nc);
      }
      if (ncb > 0) {
        count_launch();
        gather_cols_kernel<R><<<gg, 256, 0, st>>>(Sc + (size_t)b0 * 2 * kk + kk, 2 * kk, kc, dcb, ncb, kc,
                                                  G + (size_t)b0 * kc * nc + nct, (long long)kc * nc, nc);
      }
    }
  }
  if (nc > 0) {
    const dim3 gt((unsigned)std::min<long long>(1024, ((long long)nc * kp + 255) / 256), 1);
    count_launch();
    gather_rows_kernel<R><<<gt, 256, 0, st>>>(U, 0, kp, drow, nc, kp, T, 0, kp);
    if (nct > 0)
      gemm<R>(st, false, false, kc, kp, nct, one<R>(), G, nc, (long long)kc * nc, T, kp, 0, one<R>(), D, kp,
              (long long)n2 * kp, P);
    if (ncb > 0)
      gemm<R>(st, false, false, kc, kp, ncb, one<R>(), G + nct, nc, (long long)kc * nc, T + (size_t)nct * kp, kp, 0,
              one<R>(), D + (size_t)kc * kp, kp, (long long)n2 * kp, P);
  }
  if ((rc = check_launch("S U (skeleton columns)"))) return rc;
  *flops = P * 8.0 * (double)kc * kp * nc;
  return LS_OK;
}

// S[b] = U^T E[b] (U: n2 x kp, E[b]: n2 x kp) for the ID's U, whose skeleton rows
// J are the identity: U^T E = E(J, :) + T^T E(J^c, :), T = U(J^c, :) -- a product of
// order (n2 - kp) instead of n2.  `scratch` holds P (n2 - kp) x kp entries.
template <class R>
int ut_product(ls_handle* H, int l, const cx<R>* E, int n2, int kp, cx<R>* S, int P, cx<R>* scratch,
               cudaStream_t st, double* flops) {
  const LevelData& lv = H->lev[l];
  const cx<R>* U = reinterpret_cast<const cx<R>*>(lv.U);
  if ((int)lv.piv.size() != kp || lv.m != n2) {
    gemm<R>(st, true, false, kp, kp, n2, one<R>(), U, kp, 0, E, kp, (long long)n2 * kp, zero<R>(), S, kp,
            (long long)kp * kp, P);
    *flops = P * 8.0 * (double)kp * n2 * kp;
    return check_launch("U^T E");
  }
  const int nc = n2 - kp;
  std::vector<int> sel(lv.piv);
  {
    std::vector<char> in(n2, 0);
    for (int a : sel) in[a] = 1;
    for (int i = 0; i < n2; ++i)
      if (!in[i]) sel.push_back(i);
  }
  int* dsel = nullptr;
  cx<R>* T = nullptr;
  int rc;
  if ((rc = dalloc((void**)&dsel, sizeof(int) * n2))) return rc;
  if ((rc = dalloc((void**)&T, sizeof(cx<R>) * std::max<size_t>((size_t)nc * kp, 1)))) {
    dfree(dsel);
    return rc;
  }
  // pageable source: the call returns once the indices are staged
  LS_CUDA_TRY(cudaMemcpyAsync(dsel, sel.data(), sizeof(int) * n2, cudaMemcpyHostToDevice, st));
  auto gather = [&](const cx<R>* src, long long sS, const int* idx, int nidx, cx<R>* dst, long long sD, int batch) {
    for (int b0 = 0; b0 < batch; b0 += kMaxGridYZ) {
      const dim3 g((unsigned)std::min<long long>(1024, ((long long)nidx * kp + 255) / 256), std::min(kMaxGridYZ, batch - b0));
      count_launch();
      gather_rows_kernel<R><<<g, 256, 0, st>>>(src + (size_t)b0 * sS, sS, kp, idx, nidx, kp, dst + (size_t)b0 * sD, sD,
                                               kp);
    }
  };
  gather(E, (long long)n2 * kp, dsel, kp, S, (long long)kp * kp, P);  // E(J, :)
  if (nc > 0) {
    gather(U, 0, dsel + kp, nc, T, 0, 1);                                       // T = U(J^c, :)
    gather(E, (long long)n2 * kp, dsel + kp, nc, scratch, (long long)nc * kp, P);  // E(J^c, :)
    gemm<R>(st, true, false, kp, kp, nc, one<R>(), T, kp, 0, scratch, kp, (long long)nc * kp, one<R>(), S, kp,
            (long long)kp * kp, P);
  }
  dfree(T);
  dfree(dsel);
  *flops = P * 8.0 * (double)kp * nc * kp;
  return check_launch("U^T E (skeleton rows)");
}

// Bytes of one apply (Algorithm 2): every factor once, the X of levels L-1..1
// a second time (the upward and the downward pass both apply it), the grid vectors.
template <class R>
void apply_bytes(ls_handle* H) {
  double fb = H->factor_bytes;
  for (int l = 1; l <= H->L - 1; ++l) {
    const double n2 = 2.0 * H->lev[l + 1].k, cols = H->lev[l].xr > 0 ? 2.0 * H->lev[l].xr : n2;
    fb += sizeof(cx<R>) * (double)(H->nprob << l) * n2 * cols;
  }
  H->bytes_apply = fb + (double)H->grid.nx * H->grid.ny * (16.0 * 2);
}

template <class R>
int build_t(ls_handle* H, cudaStream_t st, const LevelWait& wait_level, const LevelWait& wait_sibling) {
  const int L = H->L, n = H->s * H->s;
  int rc;
  struct EngineScope {
    explicit EngineScope(ls_handle* H) {
      g_tc_engine = tc_engine_of(H);
      g_tc_err = H->d_err;
    }
    ~EngineScope() {
      g_tc_engine = 0;
      g_tc_err = nullptr;
    }
  } engine_scope(H);
  // leaves (once level L is compressed)
  if ((rc = leaf_block(H, st))) return rc;
  if (wait_level && (rc = wait_level(L))) return rc;
  LevelData& lf = H->lev[L];
  const int kL = lf.k;
  const size_t nleaf = (size_t)H->nprob << L;
  if ((rc = dalloc(&lf.X, sizeof(cx<R>) * nleaf * n * n))) return rc;
  if ((rc = dalloc(&H->XBU, sizeof(cx<R>) * nleaf * n * std::max(kL, 1)))) return rc;
  if ((rc = dalloc(&lf.S, sizeof(cx<R>) * nleaf * std::max(kL * kL, 1)))) return rc;
  H->factor_bytes += sizeof(cx<R>) * nleaf * ((double)n * n + (double)n * kL + (double)kL * kL);
  TreeGeom g = make_geom(H);
  size_t smem = sizeof(cx<R>) * ((size_t)n * (n + 1) + (size_t)n * kL + n) + sizeof(R) * n + sizeof(int) * n + 64;
  int tk = prof_begin(st);
  // Batched by default where the leaf order fits the register Gauss-Jordan
  // (probe-checked, row-pivoted fallback) and where the fused kernel's shared
  // memory would not fit; LS_LEAF_FUSED=1 (diagnostic) keeps the fused kernel.
  static const bool force_fused = [] {
    const char* v = getenv("LS_LEAF_FUSED");
    return v && v[0] && v[0] != '0';
  }();
  const bool reg_inverse = n <= gj_reg_max<R>();
  if (smem <= 220 * 1024 && (force_fused || !reg_inverse)) {  // one block per leaf, everything in shared memory
    LS_CUDA_TRY(cudaFuncSetAttribute(leaf_build_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    count_launch();
    leaf_build_kernel<R><<<(unsigned)nleaf, 256, smem, st>>>(g, H->b, H->kappa * H->kappa,
                                                            reinterpret_cast<const cx<R>*>(H->Gleaf),
                                                            reinterpret_cast<const cx<R>*>(lf.U), kL,
                                                            reinterpret_cast<cx<R>*>(lf.X),
                                                            reinterpret_cast<cx<R>*>(H->XBU),
                                                            reinterpret_cast<cx<R>*>(lf.S), H->d_err);
  } else {  // batched leaf matrices, inverses and GEMMs
    cx<R>* Xl = reinterpret_cast<cx<R>*>(lf.X);
    cx<R>* BU = nullptr;
    // scratch of the checked inverse (a copy of the matrices, the probe vectors) or of
    // the row-pivoted blocked one
    const size_t ib = reg_inverse ? sizeof(cx<R>) * (nleaf * ((size_t)n * n + 2 * (size_t)n) + n) + (1 << 16)
                                  : sizeof(cx<R>) * nleaf * ((size_t)n * 32 + 128) + sizeof(int) * nleaf * (n + 128) +
                                        (1 << 16);
    void* scr = nullptr;
    if ((rc = dalloc((void**)&BU, sizeof(cx<R>) * nleaf * n * std::max(kL, 1))) || (rc = dalloc(&scr, ib))) return rc;
    struct FreeOnExit2 {
      void* a;
      void* b;
      ~FreeOnExit2() {
        dfree(a);
        dfree(b);
      }
    } fr{BU, scr};
    const long long tot = (long long)nleaf * n * n, totk = (long long)nleaf * n * kL;
    count_launch(2);
    leaf_matrix_kernel<R><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(g, H->b, H->kappa * H->kappa,
                                                                       reinterpret_cast<const cx<R>*>(H->Gleaf),
                                                                       reinterpret_cast<const cx<R>*>(lf.U), kL, Xl,
                                                                       BU, (long long)nleaf);
    if ((rc = reg_inverse ? invert_checked<R>(H, Xl, n, n, (long long)n * n, (int)nleaf, scr, ib, st)
                          : invert_batch<R>(H, Xl, n, n, (long long)n * n, (int)nleaf, scr, ib, st)))
      return rc;
    (void)totk;
    gemm<R>(st, false, false, n, kL, n, one<R>(), Xl, n, (long long)n * n, BU, kL, (long long)n * kL, zero<R>(),
            reinterpret_cast<cx<R>*>(H->XBU), kL, (long long)n * kL, (int)nleaf);  // X B U
    gemm<R>(st, true, false, kL, kL, n, one<R>(), reinterpret_cast<const cx<R>*>(lf.U), kL, 0,
            reinterpret_cast<const cx<R>*>(H->XBU), kL, (long long)n * kL, zero<R>(),
            reinterpret_cast<cx<R>*>(lf.S), kL, (long long)kL * kL, (int)nleaf);  // U^T X B U
  }
  if ((rc = check_launch("leaf_build"))) return rc;
  {
    double fl = nleaf * (8.0 * n * n * n + 8.0 * n * n * kL + 8.0 * kL * n * kL);
    prof_end(tk, PR_LEAF, st, sizeof(cx<R>) * nleaf * ((double)n * n + (double)n * kL + (double)kL * kL) + 8.0 * nleaf * n,
             fl);
    H->flops_build += fl;
  }

  // merges, level by level.  X of level l needs the children's S and sibling
  // block (compression of level l + 1, already waited for); only S of level l
  // needs this level's U, so the wait for compression level l sits before it
  // and X of level l is formed while level l is being compressed.
  for (int l = L - 1; l >= 0; --l) {
    // G of the two children (Eq. 15), U^T and G^T for the apply, G = L R^T where the
    // Woodbury form pays: made here, or by the pipeline's sibling worker
    if (wait_sibling) {
      if ((rc = wait_sibling(l + 1))) return rc;
    } else if ((rc = sibling_prepare(H, l + 1, st))) {
      return rc;
    }
    LevelData& lv = H->lev[l];
    const LevelData& ch = H->lev[l + 1];
    const int P = H->nprob << l, kc = ch.k, n2 = 2 * kc;
    const bool woodbury = kc > 0 && ch.gr > 0;
    // scratch of X in the Schur form: the larger of (pivoted-inverse panels +
    // pivots) and Y1, Y2, a copy of Z with the blocked-inverse panels (width <=
    // 128); the S products get their own once this level's rank is known
    size_t work_bytes = 0;
    if (!woodbury) {
      const size_t Pz = (size_t)P, kz = (size_t)kc, nz = (size_t)n2;
      work_bytes = sizeof(cx<R>) * Pz * nz * nz + sizeof(int) * Pz * nz;
      work_bytes = std::max(work_bytes, sizeof(cx<R>) * Pz * (3 * kz * kz + 128 * 128 + 3 * 128 * kz) +
                                            sizeof(int) * Pz * (nz + 256) + 4096);
    }
    void* work = nullptr;
    if (work_bytes && (rc = dalloc(&work, work_bytes))) return rc;
    struct FreeOnExit {
      void* p;
      ~FreeOnExit() {
        if (p) dfree(p);
      }
    } free_work{work};
    // X per node: 2kc x 2kc, or its factor P_L (2kc x 2r) in the Woodbury form
    lv.xr = woodbury ? ch.gr : 0;
    const long long xcols = woodbury ? 2LL * ch.gr : n2;
    if ((rc = dalloc(&lv.X, sizeof(cx<R>) * (size_t)P * std::max<long long>(n2 * xcols, 1)))) return rc;
    H->factor_bytes += sizeof(cx<R>) * (double)P * n2 * xcols;
    cx<R>* X = reinterpret_cast<cx<R>*>(lv.X);
    const cx<R>* Sc = reinterpret_cast<const cx<R>*>(ch.S);
    const cx<R>* Gs = reinterpret_cast<const cx<R>*>(ch.Gsib);
    if (woodbury) {
      if (l == 0 && (rc = apply_prepare<R>(H, st))) return rc;
      if ((rc = merge_woodbury<R>(H, l, X, Sc, st))) return rc;
    } else if (kc > 0) {
      // Schur complement form of Eq. (26):  with Y1 = S_a G, Y2 = S_b G^T and
      // W = (I - Y2 Y1)^-1,  X = [[I + Y1 W Y2, -Y1 W], [-W Y2, W]].
      const long long sX = (long long)n2 * n2, kk = (long long)kc * kc;
      cx<R>* Y1 = reinterpret_cast<cx<R>*>(work);
      cx<R>* Y2 = Y1 + (size_t)P * kk;
      void* scratch = Y2 + (size_t)P * kk;
      size_t scratch_bytes = work_bytes - sizeof(cx<R>) * 2 * (size_t)P * kk;
      cx<R>* X11 = X;
      cx<R>* X12 = X + kc;
      cx<R>* X21 = X + (size_t)kc * n2;
      cx<R>* X22 = X21 + kc;
      const cx<R> mone = mk<R>(R(-1), R(0));
      int tg = prof_begin(st);
      gemm<R>(st, false, false, kc, kc, kc, one<R>(), Sc, kc, 2 * kk, Gs, kc, 0, zero<R>(), Y1, kc, kk, P);
      gemm<R>(st, false, true, kc, kc, kc, one<R>(), Sc + kk, kc, 2 * kk, Gs, kc, 0, zero<R>(), Y2, kc, kk, P);
      long long tot = (long long)P * kk;
      count_launch();
      set_identity_kernel<R><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(X22, kc, n2, sX, P);
      gemm<R>(st, false, false, kc, kc, kc, mone, Y2, kc, kk, Y1, kc, kk, one<R>(), X22, n2, sX, P);  // Z
      if ((rc = check_launch("merge gemm"))) return rc;
      prof_end(tg, PR_MERGE_GEMM, st, sizeof(cx<R>) * P * (5.0 * kk), P * 3.0 * 8.0 * (double)kc * kc * kc);
      int ti = prof_begin(st);
      // W = Z^-1 without interchanges (register-resident Gauss-Jordan for small
      // orders, blocked otherwise), checked with a probe vector; the row-pivoted
      // kernels are the fallback, and the only path when merge_pivoting = 1
      if (H->opts.merge_pivoting == 1) {
        if ((rc = invert_batch<R>(H, X22, kc, n2, sX, P, scratch, scratch_bytes, st))) return rc;
      } else {
        cx<R>* Zc = reinterpret_cast<cx<R>*>(scratch);  // copy of Z for the fallback
        void* scr2 = Zc + (size_t)P * kk;
        size_t scr2_bytes = scratch_bytes - sizeof(cx<R>) * (size_t)P * kk;
        dim3 gc((unsigned)std::min<long long>(1024, (kk + 255) / 256), std::min(P, kMaxGridYZ));
        for (int b0 = 0; b0 < P; b0 += kMaxGridYZ) {
          gc.y = std::min(kMaxGridYZ, P - b0);
          count_launch();
          copy_block_kernel<R><<<gc, 256, 0, st>>>(Zc + (size_t)b0 * kk, kc, kk, X22 + (size_t)b0 * sX, n2, sX, kc, kc);
        }
        LS_CUDA_TRY(cudaMemsetAsync(H->d_err + 2, 0, 2 * sizeof(int), st));
        if (kc <= gj_reg_max<R>()) {
          if ((rc = invert_reg_nopiv<R>(X22, kc, n2, sX, P, H->d_err + 3, st))) return rc;
        } else {
          if ((rc = invert_batch_nopiv<R>(H, X22, kc, n2, sX, P, scr2, scr2_bytes, st))) return rc;
        }
        {
          cx<R>* pv = reinterpret_cast<cx<R>*>(scr2);  // v (kc), then u, t, r (P kc each)
          cx<R>* pu = pv + kc;
          cx<R>* pt = pu + (size_t)P * kc;
          cx<R>* pr = pt + (size_t)P * kc;
          count_launch();
          probe_vector_kernel<R><<<(kc + 255) / 256, 256, 0, st>>>(pv, kc);
          gemv<R>(st, false, kc, kc, one<R>(), X22, n2, sX, pv, 0, zero<R>(), pu, kc, P);
          gemv<R>(st, false, kc, kc, one<R>(), Y1, kc, kk, pu, kc, zero<R>(), pt, kc, P);
          LS_CUDA_TRY(cudaMemcpyAsync(pr, pu, sizeof(cx<R>) * (size_t)P * kc, cudaMemcpyDeviceToDevice, st));
          gemv<R>(st, false, kc, kc, mk<R>(R(-1), R(0)), Y2, kc, kk, pt, kc, one<R>(), pr, kc, P);
          count_launch();
          probe_max_kernel<R><<<64, 256, 0, st>>>(pr, pv, kc, (long long)P * kc, H->d_err + 2);
        }
        // the root: the persistent apply's operation list (pointers only) is made and
        // uploaded while the GPU still runs the inverse, before the host waits for it
        if (l == 0 && (rc = apply_prepare<R>(H, st))) return rc;
        int* flags = static_cast<int*>(pinned_scratch(2 * sizeof(int)));  // worst probe residual (float bits), zero-pivot flag
        if (!flags) return LS_ENOMEM;
        LS_CUDA_TRY(cudaMemcpyAsync(flags, H->d_err + 2, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
        LS_CUDA_TRY(cudaStreamSynchronize(st));
        if (l == 0) host_mark("root_inverse_checked");
        float worst;
        memcpy(&worst, &flags[0], sizeof(float));
        H->probe_resid_max = std::max(H->probe_resid_max, (double)worst);
        // W is accepted when max_i |(Z W v - v)_i| (|v_i| = 1) is within the HBS
        // tolerance, so that the inverse adds no more error than the compression,
        // or within 10 k_c units of the working precision, what a stable
        // elimination of order k_c attains (in FP32 that is above the tolerance
        // from k_c ~ 170 on; a row-pivoted inverse in the same precision would
        // not do better).  A larger residual means growth in the elimination
        // without interchanges: the row-pivoted inverse replaces it.
        const double unit = sizeof(R) == 4 ? 5.96e-8 : 1.11e-16;
        const double limit = std::max(H->tol, 10.0 * unit * kc);
        if (flags[1] != 0 || !((double)worst <= limit)) {
          // restore Z and invert with row interchanges
          for (int b0 = 0; b0 < P; b0 += kMaxGridYZ) {
            gc.y = std::min(kMaxGridYZ, P - b0);
            count_launch();
            copy_block_kernel<R><<<gc, 256, 0, st>>>(X22 + (size_t)b0 * sX, n2, sX, Zc + (size_t)b0 * kk, kc, kk, kc, kc);
          }
          if ((rc = invert_batch<R>(H, X22, kc, n2, sX, P, scr2, scr2_bytes, st))) return rc;
          ++H->pivot_fallbacks;
        }
      }
      prof_end(ti, PR_MERGE_INV, st, sizeof(cx<R>) * P * 2.0 * kk, P * 8.0 * (double)kc * kc * kc);
      tg = prof_begin(st);
      if (l == 0) {
        // the root's X is only ever applied: it is kept as W, Y1 (in the X12 block) and
        // Y2 (in the X21 block), and X [r_a; r_b] = [r_a - Y1 u; u], u = W (r_b - Y2 r_a)
        dim3 gc((unsigned)std::min<long long>(1024, (kk + 255) / 256), P);
        count_launch();
        copy_block_kernel<R><<<gc, 256, 0, st>>>(X21, n2, sX, Y2, kc, kk, kc, kc);
        count_launch();
        copy_block_kernel<R><<<gc, 256, 0, st>>>(X12, n2, sX, Y1, kc, kk, kc, kc);
        if ((rc = check_launch("root blocks"))) return rc;
        prof_end(tg, PR_MERGE_GEMM, st, sizeof(cx<R>) * P * 4.0 * kk, 0.0);
        H->factor_bytes -= sizeof(cx<R>) * (double)P * kk;  // the X11 blocks are not read
      } else {
        gemm<R>(st, false, false, kc, kc, kc, mone, X22, n2, sX, Y2, kc, kk, zero<R>(), X21, n2, sX, P);  // -W Y2
        gemm<R>(st, false, false, kc, kc, kc, mone, Y1, kc, kk, X22, n2, sX, zero<R>(), X12, n2, sX, P);  // -Y1 W
        count_launch();
        set_identity_kernel<R><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(X11, kc, n2, sX, P);
        gemm<R>(st, false, false, kc, kc, kc, mone, Y1, kc, kk, X21, n2, sX, one<R>(), X11, n2, sX, P);  // I + Y1 W Y2
        if ((rc = check_launch("merge blocks"))) return rc;
        prof_end(tg, PR_MERGE_GEMM, st, sizeof(cx<R>) * P * (4.0 * kk + (double)sX),
                 P * 3.0 * 8.0 * (double)kc * kc * kc);
      }
    }
    if (!woodbury) H->flops_build += P * (6.0 * 8 * (double)kc * kc * kc + 8.0 * (double)kc * kc * kc);
    {
      char mark[48];
      snprintf(mark, sizeof(mark), "merge_X_level_%d", l);
      host_mark(mark);
    }
    if (l == 0) break;
    if (wait_level && (rc = wait_level(l))) return rc;
    const int kp = lv.k;
    if ((rc = dalloc(&lv.S, sizeof(cx<R>) * (size_t)P * std::max(kp * kp, 1)))) return rc;
    H->factor_bytes += sizeof(cx<R>) * (double)P * kp * kp;
    if (kp == 0 || kc == 0) continue;
    void* work_s = nullptr;
    if ((rc = dalloc(&work_s, sizeof(cx<R>) * 2 * (size_t)P * n2 * kp))) return rc;
    FreeOnExit free_work_s{work_s};
    cx<R>* D = reinterpret_cast<cx<R>*>(work_s);  // P x n2 x kp
    cx<R>* E = D + (size_t)P * n2 * kp;
    int ts = prof_begin(st);
    if (woodbury) {
      // X = I + P_L Q_R, Q_R = diag(L^T, R^T) (the children's sibling factors)
      const int r = ch.gr, r2 = 2 * r;
      const long long sP = (long long)n2 * r2, kk = (long long)kc * kc;
      const cx<R>* Lf = reinterpret_cast<const cx<R>*>(ch.GL);
      const cx<R>* Rf = reinterpret_cast<const cx<R>*>(ch.GR);
      cx<R>* Sl = reinterpret_cast<cx<R>*>(lv.S);
      const cx<R> on = one<R>(), ze = zero<R>();
      double fl;
      if (l <= H->opts.top_uncompressed && kp == n2) {
        // S = X diag(S_a, S_b) = diag(S_a, S_b) + P_L diag(L^T S_a, R^T S_b)
        cx<R>* Z = D;  // L^T S_a and R^T S_b: P x r x kc each
        gemm<R>(st, true, false, r, kc, kc, on, Lf, r, 0, Sc, kc, 2 * kk, ze, Z, kc, (long long)r * kc, P);
        gemm<R>(st, true, false, r, kc, kc, on, Rf, r, 0, Sc + kk, kc, 2 * kk, ze, Z + (size_t)P * r * kc, kc,
                (long long)r * kc, P);
        LS_CUDA_TRY(cudaMemsetAsync(Sl, 0, sizeof(cx<R>) * (size_t)P * kp * kp, st));
        // diag(S_a, S_b) into each node's S
        for (int b0 = 0; b0 < P; b0 += kMaxGridYZ) {
          dim3 gc((unsigned)std::min<long long>(1024, (kk + 255) / 256), std::min(kMaxGridYZ, P - b0));
          count_launch(2);
          copy_block_kernel<R><<<gc, 256, 0, st>>>(Sl + (size_t)b0 * kp * kp, kp, (long long)kp * kp,
                                                   Sc + (size_t)b0 * 2 * kk, kc, 2 * kk, kc, kc);
          copy_block_kernel<R><<<gc, 256, 0, st>>>(Sl + (size_t)b0 * kp * kp + (size_t)kc * kp + kc, kp,
                                                   (long long)kp * kp, Sc + (size_t)b0 * 2 * kk + kk, kc, 2 * kk, kc,
                                                   kc);
        }
        gemm<R>(st, false, false, n2, kc, r, on, X, r2, sP, Z, kc, (long long)r * kc, on, Sl, kp, (long long)kp * kp, P);
        gemm<R>(st, false, false, n2, kc, r, on, X + r, r2, sP, Z + (size_t)P * r * kc, kc, (long long)r * kc, on,
                Sl + kc, kp, (long long)kp * kp, P);
        fl = P * (2.0 * 8 * (double)r * kc * kc + 2.0 * 8 * (double)n2 * r * kc);
      } else {
        // D = [S_a U_top ; S_b U_bot];  E = X D = D + P_L (Q_R D) (in D);  S = U^T E
        double fd = 0;
        if ((rc = su_product<R>(H, l, Sc, kc, kp, D, P, st, &fd))) return rc;
        cx<R>* F = E;  // Q_R D: P x 2r x kp
        gemm<R>(st, true, false, r, kp, kc, on, Lf, r, 0, D, kp, (long long)n2 * kp, ze, F, kp, (long long)r2 * kp, P);
        gemm<R>(st, true, false, r, kp, kc, on, Rf, r, 0, D + (size_t)kc * kp, kp, (long long)n2 * kp, ze,
                F + (size_t)r * kp, kp, (long long)r2 * kp, P);
        gemm<R>(st, false, false, n2, kp, r2, on, X, r2, sP, F, kp, (long long)r2 * kp, on, D, kp, (long long)n2 * kp,
                P);
        double fu = 0;
        if ((rc = ut_product<R>(H, l, D, n2, kp, Sl, P, E, st, &fu))) return rc;
        fl = P * (2.0 * 8 * (double)r * kc * kp + 8.0 * (double)n2 * r2 * kp) + fd + fu;
      }
      if ((rc = check_launch("merge S (Woodbury)"))) return rc;
      prof_end(ts, PR_MERGE_GEMM, st, sizeof(cx<R>) * P * ((double)sP + 2.0 * kc * kc + (double)kp * kp), fl);
      H->flops_build += fl;
      continue;
    }
    if (l <= H->opts.top_uncompressed && kp == n2) {
      // uncompressed level (U = I): S = X diag(S_a, S_b), two column blocks of X
      cx<R>* Sl = reinterpret_cast<cx<R>*>(lv.S);
      gemm<R>(st, false, false, n2, kc, kc, one<R>(), X, n2, (long long)n2 * n2, Sc, kc, 2LL * kc * kc, zero<R>(), Sl,
              kp, (long long)kp * kp, P);
      gemm<R>(st, false, false, n2, kc, kc, one<R>(), X + kc, n2, (long long)n2 * n2, Sc + (size_t)kc * kc, kc,
              2LL * kc * kc, zero<R>(), Sl + kc, kp, (long long)kp * kp, P);
      if ((rc = check_launch("merge S"))) return rc;
      const double fl = P * 2.0 * 8 * (double)n2 * kc * kc;
      prof_end(ts, PR_MERGE_GEMM, st, sizeof(cx<R>) * P * ((double)n2 * n2 + 2.0 * kc * kc + (double)kp * kp), fl);
      H->flops_build += fl;
      continue;
    }
    // D = [S_a U_top ; S_b U_bot]
    double fd = 0;
    if ((rc = su_product<R>(H, l, Sc, kc, kp, D, P, st, &fd))) return rc;
    // E = X D ; S = U^T E
    gemm<R>(st, false, false, n2, kp, n2, one<R>(), X, n2, (long long)n2 * n2, D, kp, (long long)n2 * kp, zero<R>(),
            E, kp, (long long)n2 * kp, P);
    double fu = 0;
    if ((rc = ut_product<R>(H, l, E, n2, kp, reinterpret_cast<cx<R>*>(lv.S), P, D, st, &fu))) return rc;
    if ((rc = check_launch("merge S"))) return rc;
    {
      double fl = P * (8.0 * (double)n2 * n2 * kp) + fd + fu;
      prof_end(ts, PR_MERGE_GEMM, st, sizeof(cx<R>) * P * ((double)n2 * n2 + 2.0 * kc * kc + (double)kp * kp), fl);
      H->flops_build += fl;
    }
  }
  if ((rc = apply_prepare<R>(H, st))) return rc;  // no-op when the root merge made it
  int* pin = static_cast<int*>(pinned_scratch(sizeof(int)));
  if (!pin) return LS_ENOMEM;
  LS_CUDA_TRY(cudaMemcpyAsync(pin, H->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  LS_CUDA_TRY(cudaStreamSynchronize(st));
  host_mark("build_checked");
  if (pin[0]) return pin[0];
  apply_bytes<R>(H);
  return LS_OK;
}

// ------------------------------------------------------------- apply
// y[b] = alpha A[b] x[b] + beta y[b], A[b] M x K row-major: one warp per row.
template <class R>
__global__ void __launch_bounds__(256) gemv_n_kernel(int M, int K, cx<R> alpha, const cx<R>* __restrict__ A, int lda,
                                                     long long sA, const cx<R>* __restrict__ x, long long sx,
                                                     cx<R> beta, cx<R>* __restrict__ y, long long sy) {
  const int b = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * 8 + warp;
  if (i >= M) return;
  const cx<R>* a = A + b * sA + (long long)i * lda;
  const cx<R>* xv = x + b * sx;
  cx<R> acc = mk<R>(0, 0);
  for (int j = lane; j < K; j += 32) fma_(acc, a[j], xv[j]);
  acc = warp_sum(acc);
  if (lane == 0) {
    cx<R> v = alpha * acc;
    if (beta.re != R(0) || beta.im != R(0)) v = v + beta * y[b * sy + i];
    y[b * sy + i] = v;
  }
}

// y[b] = alpha A[b]^T x[b] + beta y[b], A[b] K x M row-major (rows i < K, columns j < M):
// lanes over 32 adjacent columns, the 8 warps split the rows, reduced in shared memory.
template <class R>
__global__ void __launch_bounds__(256) gemv_t_kernel(int M, int K, cx<R> alpha, const cx<R>* __restrict__ A, int lda,
                                                     long long sA, const cx<R>* __restrict__ x, long long sx,
                                                     cx<R> beta, cx<R>* __restrict__ y, long long sy) {
  __shared__ cx<R> part[8][32];
  const int b = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * 32 + lane;
  const cx<R>* a = A + b * sA;
  const cx<R>* xv = x + b * sx;
  cx<R> acc = mk<R>(0, 0);
  if (j < M)
    for (int i = warp; i < K; i += 8) fma_(acc, a[(long long)i * lda + j], xv[i]);
  part[warp][lane] = acc;
  __syncthreads();
  if (warp == 0 && j < M) {
    cx<R> v = part[0][lane];
    for (int w = 1; w < 8; ++w) v = v + part[w][lane];
    v = alpha * v;
    if (beta.re != R(0) || beta.im != R(0)) v = v + beta * y[b * sy + j];
    y[b * sy + j] = v;
  }
}

// y = alpha op(A) x + beta y for a batch of vectors (op(A) is M x K).
template <class R>
void gemv(cudaStream_t st, bool ta, int M, int K, cx<R> alpha, const cx<R>* A, int lda, long long sA, const cx<R>* x,
          long long sx, cx<R> beta, cx<R>* y, long long sy, int batch) {
  if (M <= 0 || K <= 0 || batch <= 0) return;
  if (batch > kMaxGridYZ) {
    for (int b0 = 0; b0 < batch; b0 += kMaxGridYZ)
      gemv<R>(st, ta, M, K, alpha, A + b0 * sA, lda, sA, x + b0 * sx, sx, beta, y + b0 * sy, sy,
              std::min(kMaxGridYZ, batch - b0));
    return;
  }
  count_launch();
  if (!ta)
    gemv_n_kernel<R><<<dim3((M + 7) / 8, batch), 256, 0, st>>>(M, K, alpha, A, lda, sA, x, sx, beta, y, sy);
  else
    gemv_t_kernel<R><<<dim3((M + 31) / 32, batch), 256, 0, st>>>(M, K, alpha, A, lda, sA, x, sx, beta, y, sy);
}

template <class R>
__global__ void gather_leaves_kernel(TreeGeom g, const z64* const* __restrict__ fslot, cx<R>* __restrict__ F) {
  const int n = g.s * g.s;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long nl = (long long)g.G << g.L;
  if (t >= nl * n) return;
  const z64* f = *fslot;
  int leaf = (int)(t / n), i = (int)(t % n);
  int ox, oy;
  leaf_origin(g, leaf, ox, oy);
  int lx = i % g.s, ly = i / g.s;
  F[t] = cvt<R>(f[(long long)(oy + ly) * g.nx + ox + lx]);
}

template <class R>
__global__ void scatter_leaves_kernel(TreeGeom g, const cx<R>* __restrict__ Q, z64* const* __restrict__ qslot) {
  const int n = g.s * g.s;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long nl = (long long)g.G << g.L;
  if (t >= nl * n) return;
  z64* q = *qslot;
  int leaf = (int)(t / n), i = (int)(t % n);
  int ox, oy;
  leaf_origin(g, leaf, ox, oy);
  int lx = i % g.s, ly = i / g.s;
  q[(long long)(oy + ly) * g.nx + ox + lx] = cvt<double>(Q[t]);
}

// Block-level helpers for the per-node fused apply kernels (vectors in shared memory).
// y[i] = sum_j A[i*lda + j] x[j], i < rows: one warp per row.
template <class R, class F>
__device__ __forceinline__ void blk_rows(const cx<R>* __restrict__ A, int lda, const cx<R>* x, int rows, int cols, F out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = warp; i < rows; i += nw) {
    const cx<R>* a = A + (long long)i * lda;
    cx<R> acc0 = mk<R>(0, 0), acc1 = mk<R>(0, 0);
    int j = lane;
    for (; j + 32 < cols; j += 64) {
      fma_(acc0, a[j], x[j]);
      fma_(acc1, a[j + 32], x[j + 32]);
    }
    if (j < cols) fma_(acc0, a[j], x[j]);
    cx<R> acc = warp_sum(acc0 + acc1);
    if (lane == 0) out(i, acc);
  }
}
// y[j] = sum_i A[i*lda + j] x[i], j < cols (A^T x): lanes over 32 columns, warps over rows,
// partial sums reduced in shared memory. Called by all threads of a 256-thread block.
template <class R, class F>
__device__ __forceinline__ void blk_cols(const cx<R>* __restrict__ A, int lda, const cx<R>* x, int rows, int cols, F out) {
  __shared__ cx<R> part[8][33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j0 = 0; j0 < cols; j0 += 32) {
    const int j = j0 + lane;
    cx<R> acc = mk<R>(0, 0);
    if (j < cols)
      for (int i = warp; i < rows; i += 8) fma_(acc, A[(long long)i * lda + j], x[i]);
    part[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && j < cols) {
      cx<R> v = part[0][lane];
      for (int w = 1; w < 8; ++w) v = v + part[w][lane];
      out(j, v);
    }
    __syncthreads();
  }
}

// Leaves, up: r = X f (kept for the last step), r~ = U^T r (Eq. (24)); one block per leaf.
template <class R>
__global__ void __launch_bounds__(256) leaf_up_kernel(TreeGeom g, const z64* const* __restrict__ fslot,
                                                      const cx<R>* __restrict__ X, const cx<R>* __restrict__ U, int k,
                                                      cx<R>* __restrict__ Rl, cx<R>* __restrict__ rt) {
  __shared__ cx<R> f[256], r[256];
  const int n = g.s * g.s, leaf = blockIdx.x;
  int ox, oy;
  leaf_origin(g, leaf, ox, oy);
  const z64* fin = *fslot;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    f[i] = cvt<R>(fin[(long long)(oy + i / g.s) * g.nx + ox + i % g.s]);
  __syncthreads();
  cx<R>* rl = Rl + (long long)leaf * n;
  blk_rows<R>(X + (long long)leaf * n * n, n, f, n, n, [&](int i, cx<R> v) {
    r[i] = v;
    rl[i] = v;
  });
  __syncthreads();
  cx<R>* ro = rt + (long long)leaf * k;
  blk_cols<R>(U, k, r, n, k, [&](int j, cx<R> v) { ro[j] = v; });
}

// Up pass for one parent: r~_tau = U^T X [r~_a; r~_b] (Eq. (28)).
template <class R>
__global__ void __launch_bounds__(256) up_node_kernel(int n2, int kp, const cx<R>* __restrict__ X,
                                                      const cx<R>* __restrict__ U, const cx<R>* __restrict__ rin,
                                                      cx<R>* __restrict__ rout) {
  extern __shared__ unsigned char smraw[];
  cx<R>* x = reinterpret_cast<cx<R>*>(smraw);
  cx<R>* t = x + n2;
  const int node = blockIdx.x;
  for (int i = threadIdx.x; i < n2; i += blockDim.x) x[i] = rin[(long long)node * n2 + i];
  __syncthreads();
  blk_rows<R>(X + (long long)node * n2 * n2, n2, x, n2, n2, [&](int i, cx<R> v) { t[i] = v; });
  __syncthreads();
  cx<R>* ro = rout + (long long)node * kp;
  blk_cols<R>(U, kp, t, n2, kp, [&](int j, cx<R> v) { ro[j] = v; });
}

// Down pass for one parent (Lemma 4.1): Uw = U w~, q~ = X([r~_a; r~_b] - diag(S_a, S_b) Uw),
// w~_a = Uw_a + G q~_b, w~_b = Uw_b + G^T q~_a.
template <class R>
__global__ void __launch_bounds__(256) down_node_kernel(int kc, int kp, const cx<R>* __restrict__ U,
                                                        const cx<R>* __restrict__ S, const cx<R>* __restrict__ X,
                                                        const cx<R>* __restrict__ G, const cx<R>* __restrict__ win,
                                                        const cx<R>* __restrict__ rab, cx<R>* __restrict__ wout) {
  extern __shared__ unsigned char smraw[];
  const int n2 = 2 * kc, node = blockIdx.x;
  cx<R>* w = reinterpret_cast<cx<R>*>(smraw);  // kp
  cx<R>* uw = w + kp;                          // n2
  cx<R>* t = uw + n2;                          // n2
  cx<R>* q = t + n2;                           // n2
  for (int i = threadIdx.x; i < kp; i += blockDim.x) w[i] = win[(long long)node * kp + i];
  __syncthreads();
  blk_rows<R>(U, kp, w, n2, kp, [&](int i, cx<R> v) { uw[i] = v; });
  __syncthreads();
  const cx<R>* ra = rab + (long long)node * n2;
  const cx<R>* Sa = S + (long long)(2 * node) * kc * kc;
  blk_rows<R>(Sa, kc, uw, kc, kc, [&](int i, cx<R> v) { t[i] = ra[i] - v; });
  blk_rows<R>(Sa + (long long)kc * kc, kc, uw + kc, kc, kc, [&](int i, cx<R> v) { t[kc + i] = ra[kc + i] - v; });
  __syncthreads();
  blk_rows<R>(X + (long long)node * n2 * n2, n2, t, n2, n2, [&](int i, cx<R> v) { q[i] = v; });
  __syncthreads();
  cx<R>* wo = wout + (long long)node * n2;
  blk_rows<R>(G, kc, q + kc, kc, kc, [&](int i, cx<R> v) { wo[i] = uw[i] + v; });
  blk_cols<R>(G, kc, q, kc, kc, [&](int j, cx<R> v) { wo[kc + j] = uw[kc + j] + v; });
}

// Leaves, last step: q = r - X B U w~, scattered to the grid.
template <class R>
__global__ void __launch_bounds__(256) leaf_down_kernel(TreeGeom g, z64* const* __restrict__ qslot,
                                                        const cx<R>* __restrict__ XBU, int k,
                                                        const cx<R>* __restrict__ wt, const cx<R>* __restrict__ Rl) {
  __shared__ cx<R> w[256];
  const int n = g.s * g.s, leaf = blockIdx.x;
  int ox, oy;
  leaf_origin(g, leaf, ox, oy);
  for (int i = threadIdx.x; i < k; i += blockDim.x) w[i] = wt[(long long)leaf * k + i];
  __syncthreads();
  z64* qo = *qslot;
  const cx<R>* rl = Rl + (long long)leaf * n;
  blk_rows<R>(XBU + (long long)leaf * n * k, k, w, n, k, [&](int i, cx<R> v) {
    qo[(long long)(oy + i / g.s) * g.nx + ox + i % g.s] = cvt<double>(rl[i] - v);
  });
}

__global__ void set_slots_kernel(z64** slots, const z64* f, z64* q) {
  slots[0] = const_cast<z64*>(f);
  slots[1] = q;
}

// Algorithm 2 for one right-hand side read from *slots[0], written to *slots[1].
template <class R>
int apply_core(ls_handle* H, z64** slots, cudaStream_t st) {
  const int L = H->L, n = H->s * H->s;
  const long long nleaf = (long long)H->nprob << L;
  TreeGeom g = make_geom(H);
  cx<R>* F = reinterpret_cast<cx<R>*>(H->work);  // leaf blocks of f
  cx<R>* Rl = F + nleaf * n;                      // r = X f on the leaves
  cx<R>* p = Rl + nleaf * n;
  std::vector<cx<R>*> rt(L + 1), wt(L + 1), tmp(L + 1);
  for (int l = 1; l <= L; ++l) {
    size_t sz = ((size_t)H->nprob << l) * std::max(1, H->lev[l].k) * 2;
    rt[l] = p;
    p += sz;
    wt[l] = p;
    p += sz;
    tmp[l] = p;
    p += sz;
  }
  std::vector<cx<R>*> ub(L + 1, nullptr);  // Q_R x of the levels whose X is factored
  for (int l = 0; l < L; ++l)
    if (H->lev[l].xr > 0) {
      ub[l] = p;
      p += ((size_t)H->nprob << l) * 2 * H->lev[l].xr;
    }
  const cx<R> mone = mk<R>(R(-1), R(0));
  // y[b] = X_l x[b] (2k_{l+1} entries per node): X itself, or I + P_L Q_R
  auto xprod = [&](int l, const cx<R>* x, cx<R>* y) -> int {
    const int kc = H->lev[l + 1].k, n2 = 2 * kc, P = H->nprob << l, r = H->lev[l].xr;
    const cx<R>* X = reinterpret_cast<const cx<R>*>(H->lev[l].X);
    if (r <= 0) {
      gemv<R>(st, false, n2, n2, one<R>(), X, n2, (long long)n2 * n2, x, n2, zero<R>(), y, n2, P);
      return LS_OK;
    }
    gemv<R>(st, false, r, kc, one<R>(), reinterpret_cast<const cx<R>*>(H->lev[l + 1].GLT), kc, 0, x, n2, zero<R>(),
            ub[l], 2 * r, P);
    gemv<R>(st, false, r, kc, one<R>(), reinterpret_cast<const cx<R>*>(H->lev[l + 1].GRT), kc, 0, x + kc, n2,
            zero<R>(), ub[l] + r, 2 * r, P);
    LS_CUDA_TRY(cudaMemcpy2DAsync(y, sizeof(cx<R>) * n2, x, sizeof(cx<R>) * n2, sizeof(cx<R>) * n2, P,
                                  cudaMemcpyDeviceToDevice, st));
    gemv<R>(st, false, n2, 2 * r, one<R>(), X, 2 * r, (long long)n2 * 2 * r, ub[l], 2 * r, one<R>(), y, n2, P);
    return LS_OK;
  };
  int xrc;
  const LevelData& lf = H->lev[L];
  const int kL = lf.k;
  // nodes of a level with at least this many parents are applied by one block each
  const int kFusedMinNodes = 512;
  const bool leaf_fused = n <= 256 && kL <= 256;
  if (leaf_fused) {
    count_launch();
    leaf_up_kernel<R><<<(unsigned)nleaf, 256, 0, st>>>(g, slots, reinterpret_cast<const cx<R>*>(lf.X),
                                                       reinterpret_cast<const cx<R>*>(lf.U), kL, Rl, rt[L]);
  } else {
    count_launch();
    gather_leaves_kernel<R><<<(unsigned)((nleaf * n + 255) / 256), 256, 0, st>>>(g, slots, F);
    // leaves: r = X f, r~ = U^T r  (Eq. (24))
    gemv<R>(st, false, n, n, one<R>(), reinterpret_cast<const cx<R>*>(lf.X), n, (long long)n * n, F, n, zero<R>(),
            Rl, n, (int)nleaf);
    gemv<R>(st, true, kL, n, one<R>(), reinterpret_cast<const cx<R>*>(lf.U), kL, 0, Rl, n, zero<R>(), rt[L], kL,
            (int)nleaf);
  }
  // upward pass: r~_tau = U^T X [r~_a; r~_b]  (Eq. (28)); X [.;.] goes to the child-level scratch
  for (int l = L - 1; l >= 1; --l) {
    const int P = H->nprob << l, kc = H->lev[l + 1].k, n2 = 2 * kc, kp = H->lev[l].k;
    if (H->lev[l].xr > 0) {
      if ((xrc = xprod(l, rt[l + 1], tmp[l + 1]))) return xrc;
      gemv<R>(st, true, kp, n2, one<R>(), reinterpret_cast<const cx<R>*>(H->lev[l].U), kp, 0, tmp[l + 1], n2,
              zero<R>(), rt[l], kp, P);
      continue;
    }
    if (P >= kFusedMinNodes && sizeof(cx<R>) * 2 * n2 <= 48 * 1024) {
      count_launch();
      up_node_kernel<R><<<P, 256, sizeof(cx<R>) * 2 * n2, st>>>(n2, kp, reinterpret_cast<const cx<R>*>(H->lev[l].X),
                                                                reinterpret_cast<const cx<R>*>(H->lev[l].U),
                                                                rt[l + 1], rt[l]);
      continue;
    }
    gemv<R>(st, false, n2, n2, one<R>(), reinterpret_cast<const cx<R>*>(H->lev[l].X), n2, (long long)n2 * n2,
            rt[l + 1], n2, zero<R>(), tmp[l + 1], n2, P);
    gemv<R>(st, true, kp, n2, one<R>(), reinterpret_cast<const cx<R>*>(H->lev[l].U), kp, 0, tmp[l + 1], n2, zero<R>(),
            rt[l], kp, P);
  }
  // root: q = X_0 [r~_a; r~_b];  w~_a = G q_b, w~_b = G^T q_a  (Eq. (29), Lemma 4.1)
  {
    const int kc = H->lev[1].k, n2 = 2 * kc, G = H->nprob;  // one root per problem
    const long long sX = (long long)n2 * n2;
    const size_t pitch = sizeof(cx<R>) * n2, width = sizeof(cx<R>) * kc;
    cx<R>* qr = tmp[1];
    const cx<R>* G1 = reinterpret_cast<const cx<R>*>(H->lev[1].Gsib);
    const cx<R>* X0 = reinterpret_cast<const cx<R>*>(H->lev[0].X);  // [., Y1; Y2, W]
    cx<R>* tb = wt[1] + kc;
    if (H->lev[0].xr > 0) {
      if ((xrc = xprod(0, rt[1], qr))) return xrc;
    } else {
      LS_CUDA_TRY(cudaMemcpy2DAsync(tb, pitch, rt[1] + kc, pitch, width, G, cudaMemcpyDeviceToDevice, st));
      gemv<R>(st, false, kc, kc, mone, X0 + (size_t)kc * n2, n2, sX, rt[1], n2, one<R>(), tb, n2, G);  // r_b - Y2 r_a
      gemv<R>(st, false, kc, kc, one<R>(), X0 + (size_t)kc * n2 + kc, n2, sX, tb, n2, zero<R>(), qr + kc, n2, G);
      LS_CUDA_TRY(cudaMemcpy2DAsync(qr, pitch, rt[1], pitch, width, G, cudaMemcpyDeviceToDevice, st));
      gemv<R>(st, false, kc, kc, mone, X0 + kc, n2, sX, qr + kc, n2, one<R>(), qr, n2, G);  // q_a = r_a - Y1 q_b
    }
    gemv<R>(st, false, kc, kc, one<R>(), G1, kc, 0, qr + kc, n2, zero<R>(), wt[1], n2, G);
    gemv<R>(st, true, kc, kc, one<R>(), G1, kc, 0, qr, n2, zero<R>(), wt[1] + kc, n2, G);
  }
  // downward pass, l = 1 .. L-1:  q~ = X ([r~_a; r~_b] - diag(S_a,S_b) U w~),
  // then w~_children = offdiag(G) q~ + U w~ (Lemma 4.1)
  for (int l = 1; l <= L - 1; ++l) {
    const int P = H->nprob << l, kc = H->lev[l + 1].k, n2 = 2 * kc, kp = H->lev[l].k;
    const cx<R>* U = reinterpret_cast<const cx<R>*>(H->lev[l].U);
    const cx<R>* Sc = reinterpret_cast<const cx<R>*>(H->lev[l + 1].S);
    const cx<R>* X = reinterpret_cast<const cx<R>*>(H->lev[l].X);
    const cx<R>* Gs = reinterpret_cast<const cx<R>*>(H->lev[l + 1].Gsib);
    if (H->lev[l].xr <= 0 && P >= kFusedMinNodes && sizeof(cx<R>) * (kp + 3 * n2) <= 48 * 1024) {
      count_launch();
      down_node_kernel<R><<<P, 256, sizeof(cx<R>) * (kp + 3 * n2), st>>>(kc, kp, U, Sc, X, Gs, wt[l], rt[l + 1],
                                                                          wt[l + 1]);
      continue;
    }
    cx<R>* Uw = wt[l + 1];  // U w~_tau, laid out as the children's incoming expansions
    cx<R>* t = tmp[l + 1];
    gemv<R>(st, false, n2, kp, one<R>(), U, kp, 0, wt[l], kp, zero<R>(), Uw, n2, P);
    LS_CUDA_TRY(cudaMemcpyAsync(t, rt[l + 1], sizeof(cx<R>) * (size_t)P * n2, cudaMemcpyDeviceToDevice, st));
    gemv<R>(st, false, kc, kc, mone, Sc, kc, 2LL * kc * kc, Uw, n2, one<R>(), t, n2, P);
    gemv<R>(st, false, kc, kc, mone, Sc + (size_t)kc * kc, kc, 2LL * kc * kc, Uw + kc, n2, one<R>(), t + kc, n2, P);
    cx<R>* qbuf = rt[l + 1];  // q~ overwrites [r~_a; r~_b], which no later step reads
    if ((xrc = xprod(l, t, qbuf))) return xrc;
    gemv<R>(st, false, kc, kc, one<R>(), Gs, kc, 0, qbuf + kc, n2, one<R>(), Uw, n2, P);
    gemv<R>(st, true, kc, kc, one<R>(), Gs, kc, 0, qbuf, n2, one<R>(), Uw + kc, n2, P);
  }
  // leaves: q = r - X B U w~
  if (leaf_fused) {
    count_launch();
    leaf_down_kernel<R><<<(unsigned)nleaf, 256, 0, st>>>(g, slots + 1, reinterpret_cast<const cx<R>*>(H->XBU), kL,
                                                         wt[L], Rl);
  } else {
    gemv<R>(st, false, n, kL, mone, reinterpret_cast<const cx<R>*>(H->XBU), kL, (long long)n * kL, wt[L], kL,
            one<R>(), Rl, n, (int)nleaf);
    count_launch();
    scatter_leaves_kernel<R><<<(unsigned)((nleaf * n + 255) / 256), 256, 0, st>>>(g, Rl, slots + 1);
  }
  return check_launch("hbs_apply");
}

// ------------------------------------------------- apply as one persistent kernel
// Algorithm 2 is a fixed sequence of batched matrix-vector products between
// which every result must be complete.  As ~60 separate launches it is bound by
// launch and tail latency; here one cooperative kernel runs the whole sequence,
// a phase at a time, with a grid barrier (release add / acquire poll) between
// phases.  Within a phase every output row is one warp's dot product (lanes
// over the row), so results do not depend on the schedule.  Transposed
// products use the U^T and G^T copies made once per handle.
struct ApplyOp {
  int type;        // 0: y[b] = y0[b] + alpha A[b] x[b];  1: gather leaves (y <- f);  2: scatter leaves (q <- x)
                   // 3: leaves up (r = X f -> y0, r~ = U^T r -> y; A = X, x = U^T)
                   // 4: leaves down (q = y0 + alpha A x scattered to the grid; A = X B U, x = w~)
  int M, K, lda, batch;
  int phase_end;   // a grid barrier follows this operation
  int rb;          // lanes per row (8, 16 or 32): short rows share a warp
  long long sA, sx, sy, sy0;
  const void* A;
  const void* x;   // null for the gather (reads f)
  void* y;         // null for the scatter (writes q)
  const void* y0;  // may be null (y0 = 0)
  double ar, ai;   // alpha
};

__device__ __forceinline__ bool apply_barrier(unsigned* count, unsigned* abort, unsigned target, int* sflag,
                                              long long limit) {
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
    unsigned v;
    long long spins = 0;
    int ok = 1;
    while (true) {
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
      if ((int)(v - target) >= 0) break;
      if (++spins >= limit || ((spins & 1023) == 0 && *(volatile unsigned*)abort)) {
        atomicExch(abort, 1u);
        ok = 0;
        break;
      }
    }
    *sflag = ok;
  }
  __syncthreads();
  return *sflag != 0;
}

// One warp task: 32 / GS consecutive output rows of y = y0 + alpha A x, each
// row a dot product over a group of GS lanes (GS = 8 or 16 for short rows, so
// that lanes are not idle and the reduction takes log2(GS) shuffle rounds; 32
// for long rows), four chunks of the row in flight per lane.
template <class R, int GS>
__device__ __forceinline__ void apply_rows(const ApplyOp& op, long long gw, long long nwarps, int lane) {
  constexpr int RPW = 32 / GS;
  const cx<R>* A = reinterpret_cast<const cx<R>*>(op.A);
  const cx<R>* X = reinterpret_cast<const cx<R>*>(op.x);
  const cx<R>* Y0 = reinterpret_cast<const cx<R>*>(op.y0);
  cx<R>* Y = reinterpret_cast<cx<R>*>(op.y);
  const cx<R> alpha = mk<R>((R)op.ar, (R)op.ai);
  const int K = op.K, grp = lane / GS, li = lane % GS;
  const long long rows = (long long)op.batch * op.M, tasks = (rows + RPW - 1) / RPW;
  for (long long task = gw; task < tasks; task += nwarps) {
    const long long r = task * RPW + grp;
    const bool ok = r < rows;
    const long long rc = ok ? r : 0;
    const int b = (int)(rc / op.M), i = (int)(rc % op.M);
    const cx<R>* a = A + b * op.sA + (long long)i * op.lda;
    const cx<R>* xv = X + b * op.sx;
    // the addend is read before the dot product so that its latency overlaps it
    const cx<R> y0v = (Y0 && ok && li == 0) ? ldcg_cx(Y0 + b * op.sy0 + i) : mk<R>(0, 0);
    cx<R> acc0 = mk<R>(0, 0), acc1 = mk<R>(0, 0), acc2 = mk<R>(0, 0), acc3 = mk<R>(0, 0);
    int j = li;
    if (ok) {
      for (; j + 3 * GS < K; j += 4 * GS) {
        const cx<R> a0 = a[j], a1 = a[j + GS], a2 = a[j + 2 * GS], a3 = a[j + 3 * GS];
        const cx<R> x0 = ldcg_cx(xv + j), x1 = ldcg_cx(xv + j + GS), x2 = ldcg_cx(xv + j + 2 * GS),
                    x3 = ldcg_cx(xv + j + 3 * GS);
        fma_(acc0, a0, x0);
        fma_(acc1, a1, x1);
        fma_(acc2, a2, x2);
        fma_(acc3, a3, x3);
      }
      for (; j < K; j += GS) fma_(acc0, a[j], ldcg_cx(xv + j));
    }
    cx<R> v = (acc0 + acc1) + (acc2 + acc3);
#pragma unroll
    for (int o = GS / 2; o; o >>= 1) v = v + shfl_xor(v, o);
    if (li == 0 && ok) Y[b * op.sy + i] = alpha * v + y0v;
  }
}

// Rows of more than 160 entries when there are at least two rows per warp of
// the grid: one warp per row, eight chunks of 32 entries in flight per lane,
// no block barrier (the split-K form below serves operations with few rows).
template <class R>
__device__ __forceinline__ void apply_rows_long(const ApplyOp& op, long long gw, long long nwarps, int lane) {
  const cx<R>* A = reinterpret_cast<const cx<R>*>(op.A);
  const cx<R>* X = reinterpret_cast<const cx<R>*>(op.x);
  const cx<R>* Y0 = reinterpret_cast<const cx<R>*>(op.y0);
  cx<R>* Y = reinterpret_cast<cx<R>*>(op.y);
  const cx<R> alpha = mk<R>((R)op.ar, (R)op.ai);
  const int K = op.K, M = op.M;
  const long long rows = (long long)op.batch * M;
  for (long long r = gw; r < rows; r += nwarps) {
    const int b = (int)(r / M), i = (int)(r % M);
    const cx<R>* a = A + b * op.sA + (long long)i * op.lda;
    const cx<R>* xv = X + b * op.sx;
    const cx<R> y0v = (Y0 && lane == 0) ? ldcg_cx(Y0 + b * op.sy0 + i) : mk<R>(0, 0);
    cx<R> acc0 = mk<R>(0, 0), acc1 = mk<R>(0, 0);
    int j = lane;
    for (; j + 7 * 32 < K; j += 8 * 32) {
      cx<R> av[8], xw[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) av[u] = a[j + 32 * u];
#pragma unroll
      for (int u = 0; u < 8; ++u) xw[u] = ldcg_cx(xv + j + 32 * u);
#pragma unroll
      for (int u = 0; u < 8; u += 2) {
        fma_(acc0, av[u], xw[u]);
        fma_(acc1, av[u + 1], xw[u + 1]);
      }
    }
    for (; j < K; j += 32) fma_(acc0, a[j], ldcg_cx(xv + j));
    cx<R> v = acc0 + acc1;
#pragma unroll
    for (int o = 16; o; o >>= 1) v = v + shfl_xor(v, o);
    if (lane == 0) Y[b * op.sy + i] = alpha * v + y0v;
  }
}

// Rows of more than 160 entries (rb = 32): split-K form.  A block takes a tile
// of RT consecutive rows; each warp one (row, 256-entry chunk) pair with all
// eight of a lane's loads issued before the first multiply-add, so that one
// memory round trip serves a whole tile even when the rows are too few to give
// every warp a row; the chunk sums are added in chunk order through shared
// memory (part, kSplitParts entries), so the result does not depend on timing.
constexpr int kSplitParts = 1024;
template <class R>
__device__ __forceinline__ void apply_rows_split(const ApplyOp& op, cx<R>* part, int lane) {
  constexpr int U = sizeof(R) == 4 ? 8 : 4, CH = 32 * U;
  const cx<R>* A = reinterpret_cast<const cx<R>*>(op.A);
  const cx<R>* X = reinterpret_cast<const cx<R>*>(op.x);
  const cx<R>* Y0 = reinterpret_cast<const cx<R>*>(op.y0);
  cx<R>* Y = reinterpret_cast<cx<R>*>(op.y);
  const cx<R> alpha = mk<R>((R)op.ar, (R)op.ai);
  const int K = op.K, M = op.M, nch = (K + CH - 1) / CH;
  const long long rows = (long long)op.batch * M;
  const long long per_block = (rows + gridDim.x - 1) / gridDim.x;
  const int RT = (int)max(1LL, min((long long)(kSplitParts / nch), per_block));
  const long long ntiles = (rows + RT - 1) / RT;
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();  // part may still be read by the previous operation
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long r0 = tile * RT;
    const int nr = (int)min((long long)RT, rows - r0);
    for (int it = warp; it < nr * nch; it += nw) {
      const int rl = it / nch, c = it % nch;
      const long long r = r0 + rl;
      const int b = (int)(r / M), i = (int)(r % M);
      const cx<R>* a = A + b * op.sA + (long long)i * op.lda;
      const cx<R>* xv = X + b * op.sx;
      const int j0 = c * CH + lane;
      cx<R> av[U], xw[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int j = j0 + 32 * u;
        av[u] = j < K ? a[j] : mk<R>(0, 0);
        xw[u] = j < K ? ldcg_cx(xv + j) : mk<R>(0, 0);
      }
      cx<R> acc0 = mk<R>(0, 0), acc1 = mk<R>(0, 0);
#pragma unroll
      for (int u = 0; u < U; u += 2) {
        fma_(acc0, av[u], xw[u]);
        fma_(acc1, av[u + 1], xw[u + 1]);
      }
      cx<R> v = acc0 + acc1;
#pragma unroll
      for (int o = 16; o; o >>= 1) v = v + shfl_xor(v, o);
      if (lane == 0) part[rl * nch + c] = v;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nr; t += blockDim.x) {
      cx<R> v = part[t * nch];
      for (int c = 1; c < nch; ++c) v = v + part[t * nch + c];
      const long long r = r0 + t;
      const int b = (int)(r / M), i = (int)(r % M);
      const cx<R> y0v = Y0 ? ldcg_cx(Y0 + b * op.sy0 + i) : mk<R>(0, 0);
      Y[b * op.sy + i] = alpha * v + y0v;
    }
    __syncthreads();  // part is reused by the next tile
  }
}

// Leaf operations of the persistent apply: four warps (a 128-thread group,
// named barrier 1 + group) take one leaf at a time, the leaf's vectors in
// shared memory, so that Algorithm 2's three leaf steps of each pass need no
// grid barrier between them.  Rows of a product are dot products over groups
// of GS lanes (8 for rows of <= 64 entries, 16 up to 128, else 32).
template <class R, class F>
__device__ __forceinline__ void group_rows(const cx<R>* __restrict__ A, int lda, const cx<R>* xs, int rows, int cols,
                                           int gt, F out) {
  const int GS = cols <= 64 ? 8 : cols <= 128 ? 16 : 32;
  const int rpp = 128 / GS, li = gt % GS;
  for (int r0 = 0; r0 < rows; r0 += rpp) {
    const int r = r0 + gt / GS;
    cx<R> acc0 = mk<R>(0, 0), acc1 = mk<R>(0, 0);
    if (r < rows) {
      const cx<R>* a = A + (long long)r * lda;
      int j = li;
      for (; j + GS < cols; j += 2 * GS) {
        fma_(acc0, a[j], xs[j]);
        fma_(acc1, a[j + GS], xs[j + GS]);
      }
      if (j < cols) fma_(acc0, a[j], xs[j]);
    }
    cx<R> v = acc0 + acc1;
    for (int o = GS / 2; o; o >>= 1) v = v + shfl_xor(v, o);
    if (li == 0 && r < rows) out(r, v);
  }
}

// type 3: for each leaf, r = X f (kept in op.y0 for the last step), r~ = U^T r.
template <class R>
__device__ __forceinline__ void apply_leaf_up(const ApplyOp& op, const TreeGeom& g, const z64* __restrict__ f,
                                              cx<R>* gs_mem) {
  const int n = g.s * g.s, kL = op.M;
  const int grp = threadIdx.x >> 7, gt = threadIdx.x & 127, ngrp = blockDim.x >> 7;
  const unsigned bar = 1 + grp;
  cx<R>* fs = gs_mem + (size_t)grp * 2 * n;
  cx<R>* rs = fs + n;
  const cx<R>* X = reinterpret_cast<const cx<R>*>(op.A);
  const cx<R>* UT = reinterpret_cast<const cx<R>*>(op.x);
  cx<R>* Rl = reinterpret_cast<cx<R>*>(const_cast<void*>(op.y0));
  cx<R>* rt = reinterpret_cast<cx<R>*>(op.y);
  for (long long leaf = (long long)blockIdx.x * ngrp + grp; leaf < op.batch; leaf += (long long)gridDim.x * ngrp) {
    int ox, oy;
    leaf_origin(g, (int)leaf, ox, oy);
    for (int i = gt; i < n; i += 128) fs[i] = cvt<R>(f[(long long)(oy + i / g.s) * g.nx + ox + i % g.s]);
    asm volatile("bar.sync %0, 128;" ::"r"(bar) : "memory");
    cx<R>* rl = Rl + leaf * n;
    group_rows<R>(X + leaf * n * n, n, fs, n, n, gt, [&](int i, cx<R> v) {
      rs[i] = v;
      rl[i] = v;
    });
    asm volatile("bar.sync %0, 128;" ::"r"(bar) : "memory");
    cx<R>* ro = rt + leaf * kL;
    group_rows<R>(UT, n, rs, kL, n, gt, [&](int i, cx<R> v) { ro[i] = v; });
    asm volatile("bar.sync %0, 128;" ::"r"(bar) : "memory");  // fs, rs reused by the next leaf
  }
}

// type 4: for each leaf, q = r + alpha X B U w~ (r = op.y0) written to the grid.
template <class R>
__device__ __forceinline__ void apply_leaf_down(const ApplyOp& op, const TreeGeom& g, z64* __restrict__ q,
                                                cx<R>* gs_mem) {
  const int n = g.s * g.s, kL = op.K;
  const int grp = threadIdx.x >> 7, gt = threadIdx.x & 127, ngrp = blockDim.x >> 7;
  const unsigned bar = 1 + grp;
  cx<R>* ws = gs_mem + (size_t)grp * 2 * n;
  const cx<R>* XBU = reinterpret_cast<const cx<R>*>(op.A);
  const cx<R>* wt = reinterpret_cast<const cx<R>*>(op.x);
  const cx<R>* Rl = reinterpret_cast<const cx<R>*>(op.y0);
  const cx<R> alpha = mk<R>((R)op.ar, (R)op.ai);
  for (long long leaf = (long long)blockIdx.x * ngrp + grp; leaf < op.batch; leaf += (long long)gridDim.x * ngrp) {
    int ox, oy;
    leaf_origin(g, (int)leaf, ox, oy);
    for (int i = gt; i < kL; i += 128) ws[i] = ldcg_cx(wt + leaf * kL + i);
    asm volatile("bar.sync %0, 128;" ::"r"(bar) : "memory");
    const cx<R>* rl = Rl + leaf * n;
    group_rows<R>(XBU + leaf * n * kL, kL, ws, n, kL, gt, [&](int i, cx<R> v) {
      q[(long long)(oy + i / g.s) * g.nx + ox + i % g.s] = cvt<double>(ldcg_cx(rl + i) + alpha * v);
    });
    asm volatile("bar.sync %0, 128;" ::"r"(bar) : "memory");
  }
}

// The operation list is copied to shared memory once per launch (dynamic
// shared memory, nops entries), so that each operation's descriptor is a
// shared-memory read rather than a global load on the critical path.
template <class R>
__global__ void __launch_bounds__(1024) apply_persistent_kernel(const ApplyOp* __restrict__ ops_g, int nops,
                                                                TreeGeom g, const z64* __restrict__ f,
                                                                z64* __restrict__ q, unsigned* bar, unsigned epoch0,
                                                                int* err, long long spin_limit) {
  __shared__ int s_ok;
  extern __shared__ unsigned char smraw[];
  ApplyOp* ops = reinterpret_cast<ApplyOp*>(smraw);
  cx<R>* leaf_mem = reinterpret_cast<cx<R>*>(smraw + ((sizeof(ApplyOp) * (size_t)nops + 15) & ~(size_t)15));
  {
    const int words = nops * (int)(sizeof(ApplyOp) / sizeof(int));
    const int* src = reinterpret_cast<const int*>(ops_g);
    int* dst = reinterpret_cast<int*>(smraw);
    for (int t = threadIdx.x; t < words; t += blockDim.x) dst[t] = src[t];
  }
  __syncthreads();
  const int wpb = blockDim.x >> 5;
  const long long nwarps = (long long)gridDim.x * wpb, nthreads = (long long)gridDim.x * blockDim.x;
  const long long gw = (long long)blockIdx.x * wpb + (threadIdx.x >> 5);
  const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  unsigned target = epoch0;
  for (int o = 0; o < nops; ++o) {
    const ApplyOp& op = ops[o];  // fields read from shared memory where used
    const long long rows = (long long)op.batch * op.M;
    if (op.type == 3) {
      apply_leaf_up<R>(op, g, f, leaf_mem);
    } else if (op.type == 4) {
      apply_leaf_down<R>(op, g, q, leaf_mem);
    } else if (op.type == 1 || op.type == 2) {  // leaf gather / scatter, one entry per thread
      const int n = g.s * g.s;
      for (long long t = gt; t < rows; t += nthreads) {
        const int leaf = (int)(t / n), i = (int)(t % n);
        int ox, oy;
        leaf_origin(g, leaf, ox, oy);
        const long long gi = (long long)(oy + i / g.s) * g.nx + ox + i % g.s;
        if (op.type == 1)
          reinterpret_cast<cx<R>*>(op.y)[t] = cvt<R>(f[gi]);
        else
          q[gi] = cvt<double>(ldcg_cx(reinterpret_cast<const cx<R>*>(op.x) + t));
      }
    } else {
      if (op.rb == 8)
        apply_rows<R, 8>(op, gw, nwarps, lane);
      else if (op.rb == 16)
        apply_rows<R, 16>(op, gw, nwarps, lane);
      else if (rows >= 2 * nwarps)
        apply_rows_long<R>(op, gw, nwarps, lane);
      else
        apply_rows_split<R>(op, leaf_mem, lane);
    }
    if (op.phase_end && o + 1 < nops) {
      target += gridDim.x;
      if (!apply_barrier(bar, bar + 1, target, &s_ok, spin_limit)) {
        if (threadIdx.x == 0 && blockIdx.x == 0) atomicExch(err, LS_ETIMEOUT);
        return;
      }
    }
  }
}

// T[b] = A[b]^T for a batch of row-major M x N matrices (stride M N), 32 x 32
// tiles staged through shared memory so that reads and writes are coalesced.
template <class R>
__global__ void __launch_bounds__(256) transpose_batch_kernel(const cx<R>* __restrict__ A, int M, int N, int batch,
                                                              cx<R>* __restrict__ T) {
  __shared__ cx<R> tile[32][33];
  const long long stride = (long long)M * N;
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  for (int bi = blockIdx.z; bi < batch; bi += gridDim.z) {
    const cx<R>* a = A + bi * stride;
    cx<R>* t = T + bi * stride;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
      const int i = i0 + r, j = j0 + threadIdx.x;
      if (i < M && j < N) tile[r][threadIdx.x] = a[(long long)i * N + j];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
      const int j = j0 + r, i = i0 + threadIdx.x;
      if (i < M && j < N) t[(long long)j * M + i] = tile[threadIdx.x][r];
    }
    __syncthreads();
  }
}

// dst (es-byte complex entries) = batch of transposed M x N blocks of src.
int transpose_batch(bool fp64, const void* src, int M, int N, int batch, void* dst, cudaStream_t st) {
  if ((long long)M * N <= 0 || batch <= 0) return LS_OK;
  const dim3 grid((unsigned)((N + 31) / 32), (unsigned)((M + 31) / 32), (unsigned)std::min(batch, 65535));
  count_launch();
  if (fp64)
    transpose_batch_kernel<double><<<grid, dim3(32, 8), 0, st>>>((const z64*)src, M, N, batch, (z64*)dst);
  else
    transpose_batch_kernel<float><<<grid, dim3(32, 8), 0, st>>>((const c32*)src, M, N, batch, (c32*)dst);
  return check_launch("transpose_batch");
}

// Operation list of Algorithm 2 (the same products as apply_core).
template <class R>
std::vector<ApplyOp> apply_ops(ls_handle* H) {
  const int L = H->L, n = H->s * H->s;
  const long long nleaf = (long long)H->nprob << L;
  cx<R>* F = reinterpret_cast<cx<R>*>(H->work);
  cx<R>* Rl = F + nleaf * n;
  cx<R>* p = Rl + nleaf * n;
  std::vector<cx<R>*> rt(L + 1), wt(L + 1), tmp(L + 1);
  for (int l = 1; l <= L; ++l) {
    size_t sz = ((size_t)H->nprob << l) * std::max(1, H->lev[l].k) * 2;
    rt[l] = p;
    p += sz;
    wt[l] = p;
    p += sz;
    tmp[l] = p;
    p += sz;
  }
  std::vector<cx<R>*> ub(L + 1, nullptr);  // Q_R x of the levels whose X is factored
  for (int l = 0; l < L; ++l)
    if (H->lev[l].xr > 0) {
      ub[l] = p;
      p += ((size_t)H->nprob << l) * 2 * H->lev[l].xr;
    }
  std::vector<ApplyOp> ops;
  auto gemv = [&](int M, int K, const void* A, int lda, long long sA, const void* x, long long sx, void* y,
                  long long sy, int batch, bool end, double ar = 1.0, const void* y0 = nullptr, long long sy0 = 0) {
    ApplyOp o;
    memset(&o, 0, sizeof(o));
    o.type = 0;
    o.M = M;
    o.K = K;
    o.A = A;
    o.lda = lda;
    o.sA = sA;
    o.x = x;
    o.sx = sx;
    o.y = y;
    o.sy = sy;
    o.batch = batch;
    o.phase_end = end ? 1 : 0;
    o.ar = ar;
    o.ai = 0.0;
    o.y0 = y0;
    o.sy0 = sy0;
    ops.push_back(o);
  };
  auto leafop = [&](int type, void* y, const void* x, bool end) {
    ApplyOp o;
    memset(&o, 0, sizeof(o));
    o.type = type;
    o.M = n;
    o.batch = (int)nleaf;
    o.y = y;
    o.x = x;
    o.phase_end = end ? 1 : 0;
    ops.push_back(o);
  };
  // y[b] = X_l x[b] (vectors of 2k_{l+1} entries, stride n2): X itself, or I + P_L Q_R
  auto xprod = [&](int l, const cx<R>* x, cx<R>* y, bool end) {
    const int kc = H->lev[l + 1].k, n2 = 2 * kc, P = H->nprob << l, r = H->lev[l].xr;
    if (r <= 0) {
      gemv(n2, n2, H->lev[l].X, n2, (long long)n2 * n2, x, n2, y, n2, P, end);
      return;
    }
    gemv(r, kc, H->lev[l + 1].GLT, kc, 0, x, n2, ub[l], 2 * r, P, false);           // L^T x_a
    gemv(r, kc, H->lev[l + 1].GRT, kc, 0, x + kc, n2, ub[l] + r, 2 * r, P, true);   // R^T x_b
    gemv(n2, 2 * r, H->lev[l].X, 2 * r, (long long)n2 * 2 * r, ub[l], 2 * r, y, n2, P, end, 1.0, x, n2);
  };
  const LevelData& lf = H->lev[L];
  const int kL = lf.k;
  {                                                                                  // leaves (Eq. 24)
    ApplyOp o;                                                                       // r = X f, r~ = U^T r
    memset(&o, 0, sizeof(o));
    o.type = 3;
    o.M = kL;
    o.K = n;
    o.batch = (int)nleaf;
    o.A = lf.X;
    o.x = lf.UT;
    o.y = rt[L];
    o.y0 = Rl;
    o.phase_end = 1;
    ops.push_back(o);
  }
  // an uncompressed level (U = I) skips its U and U^T products
  auto identity_u = [&](int l) { return l <= H->opts.top_uncompressed && H->lev[l].k == 2 * H->lev[l + 1].k; };
  for (int l = L - 1; l >= 1; --l) {                                                 // up pass (Eq. 28)
    const int P = H->nprob << l, kc = H->lev[l + 1].k, n2 = 2 * kc, kp = H->lev[l].k;
    if (identity_u(l)) {
      xprod(l, rt[l + 1], rt[l], true);
      continue;
    }
    xprod(l, rt[l + 1], tmp[l + 1], true);
    gemv(kp, n2, H->lev[l].UT, n2, 0, tmp[l + 1], n2, rt[l], kp, P, true);
  }
  {                                                                                  // root (Eq. 29)
    const int kc = H->lev[1].k, n2 = 2 * kc, G = H->nprob;                           // one root per problem
    const long long sX = (long long)n2 * n2;
    const cx<R>* X0 = reinterpret_cast<const cx<R>*>(H->lev[0].X);
    if (H->lev[0].xr > 0) {  // q = X_0 [r_a; r_b] with X_0 = I + P_L Q_R
      xprod(0, rt[1], tmp[1], true);
    } else {                 // X_0 kept as [., Y1; Y2, W]
      gemv(kc, kc, X0 + (size_t)kc * n2, n2, sX, rt[1], n2, wt[1] + kc, n2, G, true, -1.0, rt[1] + kc, n2);  // r_b - Y2 r_a
      gemv(kc, kc, X0 + (size_t)kc * n2 + kc, n2, sX, wt[1] + kc, n2, tmp[1] + kc, n2, G, true);            // q_b = W (.)
      gemv(kc, kc, X0 + kc, n2, sX, tmp[1] + kc, n2, tmp[1], n2, G, true, -1.0, rt[1], n2);                  // q_a = r_a - Y1 q_b
    }
    gemv(kc, kc, H->lev[1].Gsib, kc, 0, tmp[1] + kc, n2, wt[1], n2, G, false);
    gemv(kc, kc, H->lev[1].GT, kc, 0, tmp[1], n2, wt[1] + kc, n2, G, true);
  }
  for (int l = 1; l <= L - 1; ++l) {                                                 // down pass (Lemma 4.1)
    const int P = H->nprob << l, kc = H->lev[l + 1].k, n2 = 2 * kc, kp = H->lev[l].k;
    const cx<R>* Sc = reinterpret_cast<const cx<R>*>(H->lev[l + 1].S);
    cx<R>* Uw = wt[l + 1];  // U w~ (w~ itself when U = I)
    if (identity_u(l))
      Uw = wt[l];
    else
      gemv(n2, kp, H->lev[l].U, kp, 0, wt[l], kp, wt[l + 1], n2, P, true);         // U w~
    gemv(kc, kc, Sc, kc, 2LL * kc * kc, Uw, n2, tmp[l + 1], n2, P, false, -1.0, rt[l + 1], n2);
    gemv(kc, kc, Sc + (size_t)kc * kc, kc, 2LL * kc * kc, Uw + kc, n2, tmp[l + 1] + kc, n2, P, true, -1.0,
         rt[l + 1] + kc, n2);                                                        // t = r~ - diag(S) U w~
    xprod(l, tmp[l + 1], rt[l + 1], true);                                          // q~ = X t
    gemv(kc, kc, H->lev[l + 1].Gsib, kc, 0, rt[l + 1] + kc, n2, wt[l + 1], n2, P, false, 1.0, Uw, n2);
    gemv(kc, kc, H->lev[l + 1].GT, kc, 0, rt[l + 1], n2, wt[l + 1] + kc, n2, P, true, 1.0, Uw + kc, n2);
  }
  {                                                                                  // q = r - XBU w~ -> grid
    ApplyOp o;
    memset(&o, 0, sizeof(o));
    o.type = 4;
    o.M = n;
    o.K = kL;
    o.batch = (int)nleaf;
    o.A = H->XBU;
    o.x = wt[L];
    o.y0 = Rl;
    o.ar = -1.0;
    o.phase_end = 1;
    ops.push_back(o);
  }
  return ops;
}

// Operation list of the transposed apply q = M^T g: the steps of Algorithm 2
// in reverse order, each factor transposed (plain transpose, no conjugate):
//   leaves      w~_L = -(X B U)^T g
//   l = L-1..1  t_l = X_l^T Gamma w~_{l+1}  (Gamma: the sibling map of Lemma 4.1,
//               [[0, G], [G^T, 0]], its own transpose; t_l kept for later),
//               w~_l = U_l^T (w~_{l+1} - diag(S_a, S_b)^T t_l)
//   root        r~_1 = X_0^T Gamma w~_1
//   l = 1..L-1  r~_{l+1} = t_l + X_l^T U_l r~_l
//   leaves      q = X_L^T (g + U_L r~_L)
// It reads the transposed copies XT, ST, XBUT, UT, GT and the plain U, G.
template <class R>
std::vector<ApplyOp> apply_ops_transpose(ls_handle* H) {
  const int L = H->L, n = H->s * H->s;
  const long long nleaf = (long long)H->nprob << L;
  cx<R>* F = reinterpret_cast<cx<R>*>(H->work);
  cx<R>* Rl = F + nleaf * n;
  cx<R>* p = Rl + nleaf * n;
  std::vector<cx<R>*> rt(L + 1), wt(L + 1), tmp(L + 1);
  for (int l = 1; l <= L; ++l) {
    size_t sz = ((size_t)H->nprob << l) * std::max(1, H->lev[l].k) * 2;
    rt[l] = p;
    p += sz;
    wt[l] = p;
    p += sz;
    tmp[l] = p;
    p += sz;
  }
  std::vector<cx<R>*> ub(L + 1, nullptr);  // P_L^T x of the levels whose X is factored
  for (int l = 0; l < L; ++l)
    if (H->lev[l].xr > 0) {
      ub[l] = p;
      p += ((size_t)H->nprob << l) * 2 * H->lev[l].xr;
    }
  std::vector<ApplyOp> ops;
  auto gemv = [&](int M, int K, const void* A, int lda, long long sA, const void* x, long long sx, void* y,
                  long long sy, int batch, bool end, double ar = 1.0, const void* y0 = nullptr, long long sy0 = 0) {
    ApplyOp o;
    memset(&o, 0, sizeof(o));
    o.type = 0;
    o.M = M;
    o.K = K;
    o.A = A;
    o.lda = lda;
    o.sA = sA;
    o.x = x;
    o.sx = sx;
    o.y = y;
    o.sy = sy;
    o.batch = batch;
    o.phase_end = end ? 1 : 0;
    o.ar = ar;
    o.y0 = y0;
    o.sy0 = sy0;
    ops.push_back(o);
  };
  auto leafop = [&](int type, void* y, const void* x) {
    ApplyOp o;
    memset(&o, 0, sizeof(o));
    o.type = type;
    o.M = n;
    o.batch = (int)nleaf;
    o.y = y;
    o.x = x;
    o.phase_end = 1;
    ops.push_back(o);
  };
  // y[b] = X_l^T x[b]: X^T itself, or (I + P_L Q_R)^T = I + Q_R^T P_L^T
  auto xprodT = [&](int l, const cx<R>* x, cx<R>* y, bool end) {
    const int kc = H->lev[l + 1].k, n2 = 2 * kc, P = H->nprob << l, r = H->lev[l].xr;
    if (r <= 0) {
      gemv(n2, n2, H->lev[l].XT, n2, (long long)n2 * n2, x, n2, y, n2, P, end);
      return;
    }
    gemv(2 * r, n2, H->lev[l].XLT, n2, (long long)2 * r * n2, x, n2, ub[l], 2 * r, P, true);  // u = P_L^T x
    gemv(kc, r, H->lev[l + 1].GL, r, 0, ub[l], 2 * r, y, n2, P, false, 1.0, x, n2);          // x_a + L u_a
    gemv(kc, r, H->lev[l + 1].GR, r, 0, ub[l] + r, 2 * r, y + kc, n2, P, end, 1.0, x + kc, n2);
  };
  const LevelData& lf = H->lev[L];
  const int kL = lf.k;
  leafop(1, F, nullptr);                                                              // F <- g
  gemv(kL, n, H->XBUT, n, (long long)kL * n, F, n, wt[L], kL, (int)nleaf, true, -1.0);
  for (int l = L - 1; l >= 1; --l) {
    const int P = H->nprob << l, kc = H->lev[l + 1].k, n2 = 2 * kc, kp = H->lev[l].k;
    const cx<R>* STc = reinterpret_cast<const cx<R>*>(H->lev[l + 1].ST);
    gemv(kc, kc, H->lev[l + 1].Gsib, kc, 0, wt[l + 1] + kc, n2, tmp[l + 1], n2, P, false);       // Gamma w~
    gemv(kc, kc, H->lev[l + 1].GT, kc, 0, wt[l + 1], n2, tmp[l + 1] + kc, n2, P, true);
    xprodT(l, tmp[l + 1], rt[l + 1], true);                                           // t_l
    gemv(kc, kc, STc, kc, 2LL * kc * kc, rt[l + 1], n2, tmp[l + 1], n2, P, false, -1.0, wt[l + 1], n2);
    gemv(kc, kc, STc + (size_t)kc * kc, kc, 2LL * kc * kc, rt[l + 1] + kc, n2, tmp[l + 1] + kc, n2, P, true, -1.0,
         wt[l + 1] + kc, n2);                                                          // w~ - diag(S)^T t_l
    gemv(kp, n2, H->lev[l].UT, n2, 0, tmp[l + 1], n2, wt[l], kp, P, true);            // w~_l
  }
  {
    const int kc = H->lev[1].k, n2 = 2 * kc, G = H->nprob;  // one root per problem
    const long long sX = (long long)n2 * n2;
    gemv(kc, kc, H->lev[1].Gsib, kc, 0, wt[1] + kc, n2, tmp[1], n2, G, false);
    gemv(kc, kc, H->lev[1].GT, kc, 0, wt[1], n2, tmp[1] + kc, n2, G, true);
    // r~_1 = X_0^T v with X_0 kept as [., Y1; Y2, W] (so X_0^T's blocks are [., Y2^T; Y1^T, W^T]):
    // [v_a - Y2^T u; u], u = W^T (v_b - Y1^T v_a)
    if (H->lev[0].xr > 0) {
      xprodT(0, tmp[1], rt[1], true);
    } else {
      const cx<R>* XT0 = reinterpret_cast<const cx<R>*>(H->lev[0].XT);
      gemv(kc, kc, XT0 + (size_t)kc * n2, n2, sX, tmp[1], n2, wt[1], n2, G, true, -1.0, tmp[1] + kc, n2);
      gemv(kc, kc, XT0 + (size_t)kc * n2 + kc, n2, sX, wt[1], n2, rt[1] + kc, n2, G, true);
      gemv(kc, kc, XT0 + kc, n2, sX, rt[1] + kc, n2, rt[1], n2, G, true, -1.0, tmp[1], n2);
    }
  }
  for (int l = 1; l <= L - 1; ++l) {
    const int P = H->nprob << l, kc = H->lev[l + 1].k, n2 = 2 * kc, kp = H->lev[l].k;
    if (H->lev[l].xr > 0) {  // r~_{l+1} = t_l + v + Q_R^T P_L^T v, v = U r~_l
      const int r = H->lev[l].xr;
      gemv(n2, kp, H->lev[l].U, kp, 0, rt[l], kp, tmp[l + 1], n2, P, false);        // v
      gemv(n2, kp, H->lev[l].U, kp, 0, rt[l], kp, rt[l + 1], n2, P, true, 1.0, rt[l + 1], n2);   // t_l + v
      gemv(2 * r, n2, H->lev[l].XLT, n2, (long long)2 * r * n2, tmp[l + 1], n2, ub[l], 2 * r, P, true);
      gemv(kc, r, H->lev[l + 1].GL, r, 0, ub[l], 2 * r, rt[l + 1], n2, P, false, 1.0, rt[l + 1], n2);
      gemv(kc, r, H->lev[l + 1].GR, r, 0, ub[l] + r, 2 * r, rt[l + 1] + kc, n2, P, true, 1.0, rt[l + 1] + kc, n2);
      continue;
    }
    gemv(n2, kp, H->lev[l].U, kp, 0, rt[l], kp, tmp[l + 1], n2, P, true);             // U r~_l
    gemv(n2, n2, H->lev[l].XT, n2, (long long)n2 * n2, tmp[l + 1], n2, rt[l + 1], n2, P, true, 1.0, rt[l + 1],
         n2);                                                                          // r~_{l+1} = t_l + X^T U r~_l
  }
  gemv(n, kL, lf.U, kL, 0, rt[L], kL, Rl, n, (int)nleaf, true, 1.0, F, n);           // g + U r~_L
  gemv(n, n, lf.XT, n, (long long)n * n, Rl, n, F, n, (int)nleaf, true);             // q = X^T (.)
  leafop(2, nullptr, F);                                                              // q -> grid
  return ops;
}

// U^T and G^T of every level (the apply reads every product row-wise).
// U^T and G^T of level l (the build makes them as soon as U and G of the level
// exist, off the end of the build).
// L^T and R^T of level l's sibling factors (the Woodbury apply reads them row-wise).
int lowrank_transpose(ls_handle* H, int l, cudaStream_t st) {
  LevelData& lv = H->lev[l];
  if (lv.gr <= 0 || lv.GLT) return LS_OK;
  const bool fp64 = H->prec == LS_FP64;
  const size_t es = fp64 ? sizeof(z64) : sizeof(c32);
  int rc;
  if ((rc = dalloc(&lv.GLT, es * (size_t)lv.k * lv.gr))) return rc;
  if ((rc = dalloc(&lv.GRT, es * (size_t)lv.k * lv.gr))) return rc;
  if ((rc = transpose_batch(fp64, lv.GL, lv.k, lv.gr, 1, lv.GLT, st))) return rc;
  return transpose_batch(fp64, lv.GR, lv.k, lv.gr, 1, lv.GRT, st);
}

int level_transpose(ls_handle* H, int l, cudaStream_t st) {
  const bool fp64 = H->prec == LS_FP64;
  const size_t es = fp64 ? sizeof(z64) : sizeof(c32);
  LevelData& lv = H->lev[l];
  if (lv.UT) return lowrank_transpose(H, l, st);
  const int m = l == H->L ? H->s * H->s : 2 * H->lev[l + 1].k, k = lv.k;
  int rc;
  if ((rc = dalloc(&lv.UT, es * (size_t)std::max(m * k, 1)))) return rc;
  if ((rc = dalloc(&lv.GT, es * (size_t)std::max(k * k, 1)))) return rc;
  if ((rc = transpose_batch(fp64, lv.U, m, k, 1, lv.UT, st))) return rc;
  if ((rc = transpose_batch(fp64, lv.Gsib, k, k, 1, lv.GT, st))) return rc;
  return lowrank_transpose(H, l, st);
}

int level_transposes(ls_handle* H, cudaStream_t st) {
  int rc;
  for (int l = 1; l <= H->L; ++l)
    if ((rc = level_transpose(H, l, st))) return rc;
  return LS_OK;
}

std::vector<int> phase_ends(const std::vector<ApplyOp>& ops) {
  std::vector<int> e;
  for (int i = 0; i < (int)ops.size(); ++i)
    if (ops[i].phase_end) e.push_back(i);
  return e;
}

int upload_ops(std::vector<ApplyOp>& ops, void** dst, cudaStream_t st) {
  for (auto& o : ops) {
    o.rb = o.K <= 64 ? 8 : o.K <= 160 ? 16 : 32;
    const bool ok = o.type == 0   ? (o.M * (long long)o.batch == 0 || (o.y && (o.K == 0 || (o.A && o.x))))
                    : o.type == 1 ? o.y != nullptr
                    : o.type == 2 ? o.x != nullptr
                    : o.type == 3 ? (o.A && o.y0 && (o.M == 0 || (o.x && o.y)))
                                  : (o.A || o.K == 0) && o.y0 && (o.K == 0 || o.x);
    if (!ok) {  // a factor or buffer the list names was never made
      set_last_error_text("apply operation list refers to a missing buffer");
      return LS_EINVAL;
    }
  }
  int rc;
  if ((rc = dalloc(dst, sizeof(ApplyOp) * ops.size()))) return rc;
  LS_CUDA_TRY(cudaMemcpyAsync(*dst, ops.data(), sizeof(ApplyOp) * ops.size(), cudaMemcpyHostToDevice, st));
  LS_CUDA_TRY(cudaStreamSynchronize(st));  // the host vector is released by the caller
  return LS_OK;
}

// Prepares the persistent apply (transposed U and G, the operation list, the
// barrier); returns LS_OK without preparing it if a cooperative grid of one
// 1024-thread block per SM cannot be co-resident (the graph path is used then).
// Dynamic shared memory of the persistent apply for an operation list of nops
// entries (the attribute is raised as needed).
size_t apply_smem(const void* kfn, int nops, size_t leaf_bytes) {
  const size_t bytes = ((sizeof(ApplyOp) * (size_t)nops + 15) & ~(size_t)15) + leaf_bytes;
  if (bytes > 48 * 1024) cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return bytes;
}

// Scratch of the persistent apply: eight 128-thread groups x 2 s^2 leaf entries,
// or the kSplitParts chunk sums of the split-K rows.
size_t leaf_smem(const ls_handle* H) {
  const size_t e = H->prec == LS_FP64 ? sizeof(z64) : sizeof(c32);
  return e * std::max<size_t>(8 * 2 * (size_t)H->s * H->s, kSplitParts);
}

int apply_persistent_init(ls_handle* H, cudaStream_t st) {
  if (H->apply_ops || H->apply_blocks < 0) return LS_OK;
  if (getenv("LS_APPLY_GRAPH")) {  // diagnostic: the CUDA-graph path, as when the grid cannot be co-resident
    H->apply_blocks = -1;
    return LS_OK;
  }
  const void* kfn = H->prec == LS_FP64 ? (const void*)apply_persistent_kernel<double>
                                       : (const void*)apply_persistent_kernel<float>;
  int rc;
  if ((rc = level_transposes(H, st))) return rc;  // the operation list reads U^T and G^T
  std::vector<ApplyOp> ops = H->prec == LS_FP64 ? apply_ops<double>(H) : apply_ops<float>(H);
  int per_sm = 0;
  if (sizeof(ApplyOp) * ops.size() > 200 * 1024 ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, 1024, apply_smem(kfn, (int)ops.size(), leaf_smem(H))) !=
          cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    H->apply_blocks = -1;  // not co-resident: graph path (forward), one launch per phase (transposed)
    return LS_OK;
  }
  if ((rc = upload_ops(ops, &H->apply_ops, st))) return rc;
  if (!H->apply_bar) {
    if ((rc = dalloc((void**)&H->apply_bar, 2 * sizeof(unsigned)))) return rc;
    LS_CUDA_TRY(cudaMemsetAsync(H->apply_bar, 0, 2 * sizeof(unsigned), st));
    H->apply_epoch = 0;
  }
  H->apply_nops = (int)ops.size();
  H->apply_phases = (int)phase_ends(ops).size();
  H->apply_blocks = H->nsm;
  return check_launch("apply_persistent_init");
}

// Prepares the transposed apply: the transposed factors (once per handle; they
// double the factor memory, so they are made only when a transposed apply is
// asked for) and its operation list.
int apply_transpose_init(ls_handle* H, cudaStream_t st) {
  if (H->apply_ops_t) return LS_OK;
  const bool fp64 = H->prec == LS_FP64;
  const size_t es = fp64 ? sizeof(z64) : sizeof(c32);
  const int L = H->L, n = H->s * H->s;
  int rc;
  if ((rc = level_transposes(H, st))) return rc;
  for (int l = 0; l <= L; ++l) {
    LevelData& lv = H->lev[l];
    const int nx = l == L ? n : 2 * H->lev[l + 1].k, P = H->nprob << l;
    if (lv.xr > 0) {  // factored X: P_L^T per node
      if (!lv.XLT) {
        if ((rc = dalloc(&lv.XLT, es * (size_t)P * nx * 2 * lv.xr))) return rc;
        if ((rc = transpose_batch(fp64, lv.X, nx, 2 * lv.xr, P, lv.XLT, st))) return rc;
      }
    } else if (!lv.XT) {
      if ((rc = dalloc(&lv.XT, es * (size_t)P * std::max(nx * nx, 1)))) return rc;
      if ((rc = transpose_batch(fp64, lv.X, nx, nx, P, lv.XT, st))) return rc;
    }
    if (l >= 2 && !lv.ST) {
      if ((rc = dalloc(&lv.ST, es * (size_t)P * std::max(lv.k * lv.k, 1)))) return rc;
      if ((rc = transpose_batch(fp64, lv.S, lv.k, lv.k, P, lv.ST, st))) return rc;
    }
  }
  const int kL = H->lev[L].k;
  if ((rc = dalloc(&H->XBUT, es * ((size_t)H->nprob << L) * n * std::max(kL, 1)))) return rc;
  if ((rc = transpose_batch(fp64, H->XBU, n, kL, H->nprob << L, H->XBUT, st))) return rc;
  std::vector<ApplyOp> ops = fp64 ? apply_ops_transpose<double>(H) : apply_ops_transpose<float>(H);
  if (sizeof(ApplyOp) * ops.size() > 200 * 1024) {
    set_last_error_text("tree too deep for the transposed apply");
    return LS_EINVAL;
  }
  if ((rc = upload_ops(ops, &H->apply_ops_t, st))) return rc;
  if (!H->apply_bar) {
    if ((rc = dalloc((void**)&H->apply_bar, 2 * sizeof(unsigned)))) return rc;
    LS_CUDA_TRY(cudaMemsetAsync(H->apply_bar, 0, 2 * sizeof(unsigned), st));
    H->apply_epoch = 0;
  }
  H->apply_nops_t = (int)ops.size();
  H->apply_phase_end_t = phase_ends(ops);
  H->apply_phases_t = (int)H->apply_phase_end_t.size();
  return check_launch("apply_transpose_init");
}

// The apply is recorded once per handle as a CUDA graph on a private stream
// (inputs and outputs are passed through two device-side pointer slots), and
// replayed on the caller's stream.
int hbs_apply_graph_init(ls_handle* H) {
  if (H->apply_exec) return LS_OK;
  int rc;
  if (!H->slots && (rc = dalloc((void**)&H->slots, 2 * sizeof(z64*)))) return rc;
  cudaStream_t cs;
  LS_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  long long before = ::ls_kernel_launches();
  cudaGraph_t graph;
  LS_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  cudaError_t e;
  {
    CaptureScope capturing;
    rc = H->prec == LS_FP64 ? apply_core<double>(H, H->slots, cs) : apply_core<float>(H, H->slots, cs);
    e = cudaStreamEndCapture(cs, &graph);
  }
  H->apply_nodes = ::ls_kernel_launches() - before;
  count_launch(-H->apply_nodes);  // recorded, not launched
  if (rc) {
    cudaStreamDestroy(cs);
    return rc;
  }
  LS_CUDA_TRY(e);
  LS_CUDA_TRY(cudaGraphInstantiate(&H->apply_exec, graph, 0));
  cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  return LS_OK;
}

// ------------------------------------------------- apply to a block of right-hand sides
// Algorithm 2 for nb right-hand sides at once.  It runs the operation list of
// the one-vector apply (forward or transposed), every batched matrix-vector
// product y[b] = y0[b] + alpha A[b] x[b] becoming a batched matrix product with
// nb columns, so each factor is read once for the whole block (on the GEMM
// engines of the build: tcgen05 tf32x3 for the large products of a LS_TF32X3
// handle, the SIMT kernels otherwise).  The block workspace stores each entry
// of the one-vector workspace as a row of nb entries, so every vector of the
// list maps to a row block with row stride nb at nb times its offset.

// F[e][r] = f[r][grid index of leaf entry e], 32 entries x 32 right-hand sides
// per block through shared memory (reads follow the grid rows, writes the block rows).
template <class R>
__global__ void __launch_bounds__(256) gather_block_kernel(TreeGeom g, const z64* __restrict__ f, long long N, int nb,
                                                           cx<R>* __restrict__ F) {
  __shared__ cx<R> tile[32][33];
  const int n = g.s * g.s;
  const long long tot = ((long long)g.G << g.L) * n, e0 = (long long)blockIdx.x * 32;
  const int r0 = blockIdx.y * 32, tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const long long e = e0 + tx;
  long long gi = -1;
  if (e < tot) {
    const int leaf = (int)(e / n), i = (int)(e % n);
    int ox, oy;
    leaf_origin(g, leaf, ox, oy);
    gi = (long long)(oy + i / g.s) * g.nx + ox + i % g.s;
  }
  for (int rr = ty; rr < 32; rr += 8)
    if (gi >= 0 && r0 + rr < nb) tile[rr][tx] = cvt<R>(f[(long long)(r0 + rr) * N + gi]);
  __syncthreads();
  for (int ee = ty; ee < 32; ee += 8)
    if (e0 + ee < tot && r0 + tx < nb) F[(e0 + ee) * nb + r0 + tx] = tile[tx][ee];
}

// q[r][grid index of leaf entry e] = Q[e][r] (the inverse of gather_block_kernel).
template <class R>
__global__ void __launch_bounds__(256) scatter_block_kernel(TreeGeom g, const cx<R>* __restrict__ Q, long long N,
                                                            int nb, z64* __restrict__ q) {
  __shared__ cx<R> tile[32][33];
  const int n = g.s * g.s;
  const long long tot = ((long long)g.G << g.L) * n, e0 = (long long)blockIdx.x * 32;
  const int r0 = blockIdx.y * 32, tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int ee = ty; ee < 32; ee += 8)
    if (e0 + ee < tot && r0 + tx < nb) tile[tx][ee] = Q[(e0 + ee) * nb + r0 + tx];
  __syncthreads();
  const long long e = e0 + tx;
  if (e >= tot) return;
  const int leaf = (int)(e / n), i = (int)(e % n);
  int ox, oy;
  leaf_origin(g, leaf, ox, oy);
  const long long gi = (long long)(oy + i / g.s) * g.nx + ox + i % g.s;
  for (int rr = ty; rr < 32; rr += 8)
    if (r0 + rr < nb) q[(long long)(r0 + rr) * N + gi] = cvt<double>(tile[rr][tx]);
}

// Entries of the one-vector apply workspace (its layout is fixed by apply_prepare).
size_t apply_work_entries(const ls_handle* H) {
  size_t vec = (size_t)2 * ((size_t)H->nprob << H->L) * H->s * H->s;
  for (int l = 1; l <= H->L; ++l) vec += (size_t)3 * ((size_t)H->nprob << l) * std::max(1, H->lev[l].k) * 2;
  for (int l = 0; l < H->L; ++l) vec += ((size_t)H->nprob << l) * 2 * std::max(0, H->lev[l].xr);
  return vec;
}

// Sets the calling thread's GEMM engine to the handle's for the lifetime of the object.
struct EngineScope {
  int prev_engine;
  int* prev_err;
  explicit EngineScope(const ls_handle* H) : prev_engine(g_tc_engine), prev_err(g_tc_err) {
    g_tc_engine = tc_engine_of(H);
    g_tc_err = H->d_err;
  }
  ~EngineScope() {
    g_tc_engine = prev_engine;
    g_tc_err = prev_err;
  }
};

// rows x cols row blocks, batch of them: dst[b] = src[b] (src null: zero), strides in entries.
template <class R>
int copy_rows(cx<R>* dst, long long sd, const cx<R>* src, long long ss, long long rows_cols, int batch, cudaStream_t st) {
  const size_t w = sizeof(cx<R>) * (size_t)rows_cols;
  if (w == 0 || batch <= 0) return LS_OK;
  const size_t dp = batch > 1 ? sizeof(cx<R>) * (size_t)sd : w, sp = batch > 1 ? sizeof(cx<R>) * (size_t)ss : w;
  if (src)
    LS_CUDA_TRY(cudaMemcpy2DAsync(dst, dp, src, sp, w, batch, cudaMemcpyDeviceToDevice, st));
  else
    LS_CUDA_TRY(cudaMemset2DAsync(dst, dp, 0, w, batch, st));
  return LS_OK;
}

template <class R>
int apply_block_t(ls_handle* H, const std::vector<ApplyOp>& ops, const z64* f, z64* q, int nb, cudaStream_t st,
                  double* flops) {
  const int L = H->L, n = H->s * H->s;
  const long long nleaf = (long long)H->nprob << L, N = (long long)H->nprob * H->grid.nx * H->grid.ny;
  const size_t went = apply_work_entries(H);
  const size_t need = sizeof(cx<R>) * went * (size_t)nb;
  int rc;
  if (H->bwork_bytes < need) {
    if (H->bwork) dfree(H->bwork);
    H->bwork = nullptr;
    H->bwork_bytes = 0;
    if ((rc = dalloc(&H->bwork, need))) return rc;
    H->bwork_bytes = need;
  }
  const cx<R>* base = reinterpret_cast<const cx<R>*>(H->work);
  cx<R>* W = reinterpret_cast<cx<R>*>(H->bwork);
  auto map = [&](const void* p) -> cx<R>* {
    const cx<R>* c = reinterpret_cast<const cx<R>*>(p);
    if (c >= base && c < base + went) return W + (size_t)(c - base) * nb;
    return const_cast<cx<R>*>(c);  // a factor
  };
  const TreeGeom g = make_geom(H);
  const dim3 tgrid((unsigned)((nleaf * n + 31) / 32), (unsigned)((nb + 31) / 32));
  EngineScope engine(H);
  const cx<R> one_ = mk<R>(R(1), R(0)), zero_ = mk<R>(R(0), R(0));
  double fl = 0;
  for (const ApplyOp& o : ops) {
    const cx<R> alpha = mk<R>((R)o.ar, (R)o.ai);
    switch (o.type) {
      case 1:  // y <- f on the leaves
        count_launch();
        gather_block_kernel<R><<<tgrid, 256, 0, st>>>(g, f, N, nb, map(o.y));
        break;
      case 2:  // grid <- x
        count_launch();
        scatter_block_kernel<R><<<tgrid, 256, 0, st>>>(g, map(o.x), N, nb, q);
        break;
      case 3: {  // leaves: F <- f, r = X F (-> y0), r~ = U^T r (-> y)
        cx<R>* F = W;
        count_launch();
        gather_block_kernel<R><<<tgrid, 256, 0, st>>>(g, f, N, nb, F);
        cx<R>* Rl = map(o.y0);
        gemm<R>(st, false, false, n, nb, n, one_, reinterpret_cast<const cx<R>*>(o.A), n, (long long)n * n, F, nb,
                (long long)n * nb, zero_, Rl, nb, (long long)n * nb, (int)nleaf);
        if (o.M > 0)
          gemm<R>(st, false, false, o.M, nb, n, one_, reinterpret_cast<const cx<R>*>(o.x), n, 0, Rl, nb,
                  (long long)n * nb, zero_, map(o.y), nb, (long long)o.M * nb, (int)nleaf);
        fl += 8.0 * nleaf * nb * ((double)n * n + (double)o.M * n);
        break;
      }
      case 4: {  // grid <- y0 + alpha A x (in place in y0: the list's last use of it)
        cx<R>* Rl = map(o.y0);
        if (o.K > 0)
          gemm<R>(st, false, false, n, nb, o.K, alpha, reinterpret_cast<const cx<R>*>(o.A), o.K, (long long)n * o.K,
                  map(o.x), nb, (long long)o.K * nb, one_, Rl, nb, (long long)n * nb, (int)nleaf);
        count_launch();
        scatter_block_kernel<R><<<tgrid, 256, 0, st>>>(g, Rl, N, nb, q);
        fl += 8.0 * nleaf * nb * (double)n * o.K;
        break;
      }
      default: {  // y = y0 + alpha A x
        if (o.M <= 0 || o.batch <= 0) break;
        cx<R>* y = map(o.y);
        const cx<R>* y0 = o.y0 ? map(o.y0) : nullptr;
        if (y0 != y && (y0 || o.K <= 0) &&
            (rc = copy_rows<R>(y, o.sy * nb, y0, o.sy0 * nb, (long long)o.M * nb, o.batch, st)))
          return rc;
        if (o.K > 0)
          gemm<R>(st, false, false, o.M, nb, o.K, alpha, reinterpret_cast<const cx<R>*>(o.A), o.lda, o.sA, map(o.x),
                  nb, o.sx * nb, y0 ? one_ : zero_, y, nb, o.sy * nb, o.batch);
        fl += 8.0 * o.batch * nb * (double)o.M * o.K;
      }
    }
  }
  if (flops) *flops = fl;
  return check_launch("hbs_apply (block)");
}

// Operation list of the apply on the host (a few hundred entries: made per call).
template <class R>
std::vector<ApplyOp> block_ops(ls_handle* H, int transpose) {
  return transpose ? apply_ops_transpose<R>(H) : apply_ops<R>(H);
}

}  // namespace

int hbs_apply_block(ls_handle* H, const z64* f, z64* q, int nb, int transpose, cudaStream_t st) {
  int rc;
  if ((rc = level_transposes(H, st))) return rc;  // the lists read U^T and G^T
  if (transpose && (rc = apply_transpose_init(H, st))) return rc;
  const int tk = prof_begin(st);
  double fl = 0;
  rc = H->prec == LS_FP64 ? apply_block_t<double>(H, block_ops<double>(H, transpose), f, q, nb, st, &fl)
                          : apply_block_t<float>(H, block_ops<float>(H, transpose), f, q, nb, st, &fl);
  // bytes: every factor once (the inner levels' X twice) and the block's vectors in and out
  prof_end(tk, PR_APPLY_BLOCK, st, H->bytes_apply + 32.0 * (nb - 1) * H->grid.nx * H->grid.ny, fl);
  return rc;
}

int hbs_build(ls_handle* H, cudaStream_t st, const LevelWait& wait_level, const LevelWait& wait_sibling) {
  return H->prec == LS_FP64 ? build_t<double>(H, st, wait_level, wait_sibling)
                            : build_t<float>(H, st, wait_level, wait_sibling);
}

int hbs_finish(ls_handle* H, cudaStream_t st) {
  int rc;
  if (H->prec == LS_FP64) {
    if ((rc = apply_prepare<double>(H, st))) return rc;
    apply_bytes<double>(H);
  } else {
    if ((rc = apply_prepare<float>(H, st))) return rc;
    apply_bytes<float>(H);
  }
  return check_launch("hbs_finish");
}

int sibling_prepare(ls_handle* H, int l, cudaStream_t st) {
  int rc;
  if ((rc = sibling_block(H, l, st))) return rc;
  if ((rc = level_transpose(H, l, st))) return rc;
  return H->prec == LS_FP64 ? sibling_lowrank<double>(H, l, st) : sibling_lowrank<float>(H, l, st);
}

int simt_cgemm(cudaStream_t st, bool ta, bool tb, int M, int N, int K, c32 alpha, const c32* A, int lda, long long sA,
               const c32* B, int ldb, long long sB, c32 beta, c32* C, int ldc, long long sC, int batch) {
  gemm<float>(st, ta, tb, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch);
  return check_launch("simt_cgemm");
}

int simt_zgemm(cudaStream_t st, bool ta, bool tb, int M, int N, int K, z64 alpha, const z64* A, int lda, long long sA,
               const z64* B, int ldb, long long sB, z64 beta, z64* C, int ldc, long long sC, int batch) {
  gemm<double>(st, ta, tb, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch);
  return check_launch("simt_zgemm");
}

int rhs_block_size(const ls_handle* H, int nrhs) {
  if (H->opts.rhs_block > 0) return std::max(1, std::min(nrhs, H->opts.rhs_block));
  // automatic: up to 256, and one slab of the block's vectors within 1 GiB
  const long long N = (long long)H->nprob * H->grid.nx * H->grid.ny;
  const long long fit = (1LL << 30) / (16LL * N);
  return (int)std::max(1LL, std::min<long long>({(long long)nrhs, 256LL, fit}));
}

int hbs_apply(ls_handle* H, const z64* f, z64* q, int nvec, int transpose, cudaStream_t st) {
  // nvec grid vectors = nvec / nprob vectors of the forest (one per problem each)
  if (nvec % H->nprob) {
    set_last_error_text("right-hand sides must come in whole sets of the handle's problems");
    return LS_EINVAL;
  }
  const int nrhs = nvec / H->nprob;
  const long long N = (long long)H->nprob * H->grid.nx * H->grid.ny;
  int rc;
  const int nbk = rhs_block_size(H, nrhs);
  if (nbk > 1) {  // blocks of right-hand sides, each factor read once per block
    for (int r0 = 0; r0 < nrhs; r0 += nbk) {
      const int nb = std::min(nbk, nrhs - r0);
      rc = nb > 1 ? hbs_apply_block(H, f + r0 * N, q + r0 * N, nb, transpose, st)
                  : hbs_apply(H, f + r0 * N, q + r0 * N, H->nprob, transpose, st);
      if (rc) return rc;
    }
    return LS_OK;
  }
  if ((rc = apply_persistent_init(H, st))) return rc;
  if (transpose) {
    if ((rc = apply_transpose_init(H, st))) return rc;
    const TreeGeom g = make_geom(H);
    const void* kfn = H->prec == LS_FP64 ? (const void*)apply_persistent_kernel<double>
                                         : (const void*)apply_persistent_kernel<float>;
    const ApplyOp* ops_all = reinterpret_cast<const ApplyOp*>(H->apply_ops_t);
    unsigned* bar = H->apply_bar;
    int* err = H->d_err;
    for (int r = 0; r < nrhs; ++r) {
      int tk = prof_begin(st);
      const z64* fr = f + r * N;
      z64* qr = q + r * N;
      if (H->apply_ops) {  // one cooperative launch, barriers between the phases
        const ApplyOp* ops = ops_all;
        int nops = H->apply_nops_t;
        unsigned epoch0 = H->apply_epoch;
        long long spin = H->spin_limit;
        void* args[] = {&ops, &nops, (void*)&g, &fr, &qr, &bar, &epoch0, &err, &spin};
        count_launch();
        LS_CUDA_TRY(
            cudaLaunchCooperativeKernel(kfn, dim3(H->apply_blocks), dim3(1024), args, apply_smem(kfn, nops, leaf_smem(H)), st));
        H->apply_epoch += (unsigned)(H->apply_phases_t - 1) * (unsigned)H->apply_blocks;
      } else {  // one launch per phase (no barrier is reached inside a launch)
        int start = 0;
        for (int e : H->apply_phase_end_t) {
          const ApplyOp* ops = ops_all + start;
          int nops = e + 1 - start;
          unsigned epoch0 = 0;
          long long spin = H->spin_limit;
        void* args[] = {&ops, &nops, (void*)&g, &fr, &qr, &bar, &epoch0, &err, &spin};
          count_launch();
          LS_CUDA_TRY(cudaLaunchKernel(kfn, dim3(H->nsm), dim3(1024), args, apply_smem(kfn, nops, leaf_smem(H)), st));
          start = e + 1;
        }
      }
      prof_end(tk, PR_APPLY, st, H->bytes_apply, 0.0);
    }
    return check_launch("hbs_apply (transposed)");
  }
  if (H->apply_ops) {
    const TreeGeom g = make_geom(H);
    const void* kfn = H->prec == LS_FP64 ? (const void*)apply_persistent_kernel<double>
                                         : (const void*)apply_persistent_kernel<float>;
    for (int r = 0; r < nrhs; ++r) {
      int tk = prof_begin(st);
      const ApplyOp* ops = reinterpret_cast<const ApplyOp*>(H->apply_ops);
      int nops = H->apply_nops;
      const z64* fr = f + r * N;
      z64* qr = q + r * N;
      unsigned* bar = H->apply_bar;
      // barrier epochs continue across applies: (phases - 1) barriers of apply_blocks arrivals each
      unsigned epoch0 = H->apply_epoch;
      int* err = H->d_err;
      long long spin = H->spin_limit;
        void* args[] = {&ops, &nops, (void*)&g, &fr, &qr, &bar, &epoch0, &err, &spin};
      count_launch();
      LS_CUDA_TRY(
          cudaLaunchCooperativeKernel(kfn, dim3(H->apply_blocks), dim3(1024), args, apply_smem(kfn, nops, leaf_smem(H)), st));
      H->apply_epoch += (unsigned)(H->apply_phases - 1) * (unsigned)H->apply_blocks;
      prof_end(tk, PR_APPLY, st, H->bytes_apply, 0.0);
    }
    return check_launch("hbs_apply");
  }
  if ((rc = hbs_apply_graph_init(H))) return rc;
  for (int r = 0; r < nrhs; ++r) {
    int tk = prof_begin(st);
    count_launch();
    set_slots_kernel<<<1, 1, 0, st>>>(H->slots, f + r * N, q + r * N);
    LS_CUDA_TRY(cudaGraphLaunch(H->apply_exec, st));
    count_launch(H->apply_nodes);
    prof_end(tk, PR_APPLY, st, H->bytes_apply, 0.0);
  }
  return check_launch("hbs_apply");
}

}  // namespace ls
