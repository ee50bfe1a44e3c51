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
#include <algorithm>

#include "handle.h"
#include "prof.h"

namespace ls {
namespace {

// ---------------------------------------------------------------- GEMM
constexpr int TM = 32, TN = 32, TK = 16;

// C[b] = alpha op(A[b]) op(B[b]) + beta C[b]   (row-major, op = N or T)
template <class R, bool TA, bool TB>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, cx<R> alpha, const cx<R>* __restrict__ A,
                                                   int lda, long long sA, const cx<R>* __restrict__ B, int ldb,
                                                   long long sB, cx<R> beta, cx<R>* __restrict__ C, int ldc,
                                                   long long sC) {
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
      if (gi < M && gj < N) {
        cx<R> v = alpha * acc[i][j];
        if (!zb) v = v + beta * C[(long long)gi * ldc + gj];
        C[(long long)gi * ldc + gj] = v;
      }
    }
}

template <class R>
void gemm(cudaStream_t st, bool ta, bool tb, int M, int N, int K, cx<R> alpha, const cx<R>* A, int lda, long long sA,
          const cx<R>* B, int ldb, long long sB, cx<R> beta, cx<R>* C, int ldc, long long sC, int batch) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  if (K <= 0) {
    // C = beta C; only used with beta = 0 or 1 here
    return;
  }
  dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM, batch);
  if (!ta && !tb)
    {
      count_launch();
      gemm_kernel<R, false, false><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC);
    }
  else if (ta && !tb)
    {
      count_launch();
      gemm_kernel<R, true, false><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC);
    }
  else if (!ta && tb)
    {
      count_launch();
      gemm_kernel<R, false, true><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC);
    }
  else
    {
      count_launch();
      gemm_kernel<R, true, true><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC);
    }
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
  __shared__ int s_p;
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < n; ++k) {
    if (warp == 0) {
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
        if (!(best > R(0))) s_bad = 1;
      }
    }
    __syncthreads();
    if (s_bad) return false;
    const int p = s_p;
    if (p != k)
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        cx<R> t = a[k * lda + j];
        a[k * lda + j] = a[p * lda + j];
        a[p * lda + j] = t;
      }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) col[i] = a[i * lda + k];
    __syncthreads();
    const cx<R> d = inv(col[k]);
    for (int j = threadIdx.x; j < n; j += blockDim.x) a[k * lda + j] = (j == k) ? d : a[k * lda + j] * d;
    __syncthreads();
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
      int i = t / n, j = t % n;
      if (i == k) continue;
      cx<R> f = col[i];
      if (j == k)
        a[i * lda + j] = mk<R>(-(f.re * d.re - f.im * d.im), -(f.re * d.im + f.im * d.re));
      else {
        cx<R> r = a[k * lda + j];
        cx<R> v = a[i * lda + j];
        v.re -= f.re * r.re - f.im * r.im;
        v.im -= f.re * r.im + f.im * r.re;
        a[i * lda + j] = v;
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

struct TreeGeom {
  int L, s, nx;
  int cw[32], ch[32];  // child box dims for the cut l -> l+1
};

__device__ __forceinline__ void leaf_origin(const TreeGeom& g, int leaf, int& ox, int& oy) {
  ox = 0;
  oy = 0;
  for (int l = 0; l < g.L; ++l) {
    int bit = (leaf >> (g.L - 1 - l)) & 1;
    if (l % 2 == 0) {
      if (bit) ox += g.cw[l];
    } else {
      if (!bit) oy += g.ch[l];  // alpha = upper half
    }
  }
}

// Leaf build (Algorithm 1, leaf loop): one block per leaf.
template <class R>
__global__ void __launch_bounds__(256) leaf_build_kernel(TreeGeom g, const double* __restrict__ b, double kap2,
                                                         const cx<R>* __restrict__ Gleaf, const cx<R>* __restrict__ U,
                                                         int k, cx<R>* __restrict__ X, cx<R>* __restrict__ XBU,
                                                         cx<R>* __restrict__ S, int* __restrict__ err) {
  extern __shared__ unsigned char smraw[];
  const int n = g.s * g.s;
  cx<R>* a = reinterpret_cast<cx<R>*>(smraw);  // n x n
  cx<R>* xbu = a + n * n;                      // n x k
  cx<R>* col = xbu + n * k;                    // n
  R* Bv = reinterpret_cast<R*>(col + n);       // n
  int* piv = reinterpret_cast<int*>(Bv + n);   // n
  const int leaf = blockIdx.x;
  int ox, oy;
  leaf_origin(g, leaf, ox, oy);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int lx = i % g.s, ly = i / g.s;
    Bv[i] = (R)(kap2 * b[(long long)(oy + ly) * g.nx + ox + lx]);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    int i = t / n, j = t % n;
    cx<R> v = scale(Gleaf[t], Bv[i]);
    if (i == j) v.re += R(1);
    a[t] = v;
  }
  __syncthreads();
  if (!gj_inverse_smem(a, n, n, piv, col)) {
    if (threadIdx.x == 0) atomicExch(err, LS_ESINGULAR);
    return;
  }
  // XBU = X diag(B) U
  for (int t = threadIdx.x; t < n * k; t += blockDim.x) {
    int i = t / k, c = t % k;
    cx<R> acc = mk<R>(0, 0);
    for (int j = 0; j < n; ++j) fma_(acc, a[i * n + j], scale(U[j * k + c], Bv[j]));
    xbu[t] = acc;
  }
  __syncthreads();
  cx<R>* Xo = X + (long long)leaf * n * n;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) Xo[t] = a[t];
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

// Identity blocks of K = [[I, .],[., I]] (the off-diagonal blocks are written by GEMMs).
template <class R>
__global__ void merge_identity_kernel(cx<R>* X, int kc, int P) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long n2 = 2 * kc;
  if (t >= (long long)P * n2 * kc) return;
  long long node = t / (n2 * kc);
  int r = (int)((t / kc) % n2), c = (int)(t % kc);
  int cc = r < kc ? c : c + kc;  // column within the diagonal block of row r
  X[node * n2 * n2 + (long long)r * n2 + cc] = mk<R>(r % kc == c ? R(1) : R(0), R(0));
}

// Batched in-smem inverse, one block per matrix.
template <class R>
__global__ void __launch_bounds__(256) inverse_smem_kernel(cx<R>* X, int n, int* err) {
  extern __shared__ unsigned char smraw[];
  cx<R>* a = reinterpret_cast<cx<R>*>(smraw);
  cx<R>* col = a + n * n;
  int* piv = reinterpret_cast<int*>(col + n);
  cx<R>* M = X + (long long)blockIdx.x * n * n;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) a[t] = M[t];
  __syncthreads();
  if (!gj_inverse_smem(a, n, n, piv, col)) {
    if (threadIdx.x == 0) atomicExch(err, LS_ESINGULAR);
    return;
  }
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) M[t] = a[t];
}

// Cooperative Gauss-Jordan for large matrices: matrix b uses blocks
// [b*G, (b+1)*G); each step reads buffer src and writes dst (ping-pong), so one
// grid barrier per pivot step suffices.  piv records the row pivots.
template <class R>
__global__ void __launch_bounds__(256) inverse_coop_kernel(cx<R>* X0, cx<R>* X1, int n, int G, int* piv, int* err,
                                                           GridSync gs) {
  extern __shared__ unsigned char smraw[];
  cx<R>* prow = reinterpret_cast<cx<R>*>(smraw);  // n
  __shared__ int s_p;
  __shared__ cx<R> s_d;
  const int mat = blockIdx.x / G, gb = blockIdx.x % G;
  const int rows_per = (n + G - 1) / G;
  const int r0 = gb * rows_per, r1 = min(n, r0 + rows_per);
  const long long nn = (long long)n * n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < n; ++k) {
    const cx<R>* src = ((k & 1) ? X1 : X0) + mat * nn;
    cx<R>* dst = ((k & 1) ? X0 : X1) + mat * nn;
    if (warp == 0) {
      R best = R(-1);
      int bi = n;
      for (int i = k + lane; i < n; i += 32) {
        R v = abs2(src[(long long)i * n + k]);
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
        if (!(best > R(0))) {
          s_p = -1;
          atomicExch(err, LS_ESINGULAR);
        } else {
          s_d = inv(src[(long long)bi * n + k]);
          if (gb == 0) piv[mat * n + k] = bi;
        }
      }
    }
    __syncthreads();
    const int p = s_p;
    if (p < 0) {
      // every block sees the same zero pivot and leaves together
      return;
    }
    const cx<R> d = s_d;
    for (int j = threadIdx.x; j < n; j += blockDim.x) prow[j] = (j == k) ? d : src[(long long)p * n + j] * d;
    __syncthreads();
    for (int i = r0 + warp; i < r1; i += 8) {
      cx<R>* out = dst + (long long)i * n;
      if (i == k) {
        for (int j = lane; j < n; j += 32) out[j] = prow[j];
        continue;
      }
      int si = (i == p) ? k : i;
      const cx<R>* in = src + (long long)si * n;
      cx<R> f = in[k];
      for (int j = lane; j < n; j += 32) {
        if (j == k) {
          out[j] = mk<R>(-(f.re * d.re - f.im * d.im), -(f.re * d.im + f.im * d.re));
        } else {
          cx<R> r = prow[j], v = in[j];
          v.re -= f.re * r.re - f.im * r.im;
          v.im -= f.re * r.im + f.im * r.re;
          out[j] = v;
        }
      }
    }
    if (!grid_sync(gs, gridDim.x)) return;
  }
}

// Undo the row pivoting by column interchanges (in reverse order) while
// copying the result from src to dst.
template <class R>
__global__ void unpivot_kernel(const cx<R>* src, cx<R>* dst, int n, const int* piv) {
  extern __shared__ int idx[];
  const long long nn = (long long)n * n;
  const int mat = blockIdx.y;
  for (int j = threadIdx.x; j < n; j += blockDim.x) idx[j] = j;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int k = n - 1; k >= 0; --k) {
      int p = piv[mat * n + k];
      int t = idx[k];
      idx[k] = idx[p];
      idx[p] = t;
    }
  __syncthreads();
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn; t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t / n), j = (int)(t % n);
    dst[mat * nn + t] = src[mat * nn + (long long)i * n + idx[j]];
  }
}

template <class R>
int invert_batch(ls_handle* H, cx<R>* X, int n, int P, cudaStream_t st) {
  const size_t smem_small = sizeof(cx<R>) * ((size_t)n * n + n) + sizeof(int) * n;
  if (smem_small <= 200 * 1024) {
    LS_CUDA_TRY(cudaFuncSetAttribute(inverse_smem_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem_small));
    count_launch();
    inverse_smem_kernel<R><<<P, 256, smem_small, st>>>(X, n, H->d_err);
    return check_launch("inverse_smem");
  }
  // large: cooperative ping-pong
  cx<R>* X1 = reinterpret_cast<cx<R>*>(H->work);
  int* piv = reinterpret_cast<int*>(X1 + (size_t)P * n * n);
  size_t need = sizeof(cx<R>) * (size_t)P * n * n + sizeof(int) * (size_t)P * n;
  if (need > H->work_bytes) return LS_ENOMEM;
  size_t smem = sizeof(cx<R>) * n;
  LS_CUDA_TRY(cudaFuncSetAttribute(inverse_coop_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  LS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, inverse_coop_kernel<R>, 256, smem));
  int maxblk = std::max(1, per_sm) * H->nsm;
  int G = std::max(1, std::min(maxblk / P, (n + 7) / 8));
  int nblk = G * P;
  if (nblk > maxblk) return LS_EINVAL;
  LS_CUDA_TRY(cudaMemsetAsync(H->sync_buf, 0, 64, st));
  GridSync gs;
  gs.count = reinterpret_cast<unsigned*>(H->sync_buf);
  gs.gen = reinterpret_cast<unsigned*>(H->sync_buf) + 1;
  gs.abort = H->sync_buf + 2;
  void* args[] = {&X, &X1, &n, &G, &piv, &H->d_err, &gs};
  count_launch();
  LS_CUDA_TRY(cudaLaunchCooperativeKernel((void*)inverse_coop_kernel<R>, dim3(nblk), dim3(256), args, smem, st));
  // result is in X (n even) or X1 (n odd)
  const cx<R>* res = (n & 1) ? X1 : X;
  cx<R>* tmp = (n & 1) ? X : X1;
  dim3 g2((unsigned)std::min<long long>(1024, ((long long)n * n + 255) / 256), P);
  count_launch();
  unpivot_kernel<R><<<g2, 256, sizeof(int) * n, st>>>(res, tmp, n, piv);
  if (tmp != X) LS_CUDA_TRY(cudaMemcpyAsync(X, tmp, sizeof(cx<R>) * (size_t)P * n * n, cudaMemcpyDeviceToDevice, st));
  return check_launch("inverse_coop");
}

TreeGeom make_geom(const ls_handle* H) {
  TreeGeom g;
  g.L = H->L;
  g.s = H->s;
  g.nx = H->grid.nx;
  for (int l = 0; l < H->L; ++l) {
    g.cw[l] = H->lev[l + 1].w;
    g.ch[l] = H->lev[l + 1].h;
  }
  return g;
}

template <class R>
int build_t(ls_handle* H, cudaStream_t st) {
  const int L = H->L, n = H->s * H->s;
  int rc;
  // scratch: the largest of (cooperative inverse ping-pong + pivots) and the merge GEMM temporaries
  size_t wb = 0;
  for (int l = 0; l < L; ++l) {
    size_t P = (size_t)1 << l, kc = H->lev[l + 1].k, n2 = 2 * kc, kp = l > 0 ? H->lev[l].k : 0;
    wb = std::max(wb, sizeof(cx<R>) * P * n2 * n2 + sizeof(int) * P * n2);
    wb = std::max(wb, sizeof(cx<R>) * 2 * P * n2 * kp);
  }
  // apply temporaries (one right-hand side): leaf blocks, per-level expansions
  size_t vec = (size_t)2 * ((size_t)1 << L) * n;
  for (int l = 1; l <= L; ++l) vec += (size_t)3 * ((size_t)1 << l) * std::max(1, H->lev[l].k) * 2;
  wb = std::max(wb, sizeof(cx<R>) * vec);
  H->work_bytes = wb;
  if ((rc = dalloc(&H->work, wb))) return rc;

  // leaves
  LevelData& lf = H->lev[L];
  const int kL = lf.k;
  const size_t nleaf = (size_t)1 << L;
  if ((rc = dalloc(&lf.X, sizeof(cx<R>) * nleaf * n * n))) return rc;
  if ((rc = dalloc(&H->XBU, sizeof(cx<R>) * nleaf * n * std::max(kL, 1)))) return rc;
  if ((rc = dalloc(&lf.S, sizeof(cx<R>) * nleaf * std::max(kL * kL, 1)))) return rc;
  H->factor_bytes += sizeof(cx<R>) * nleaf * ((double)n * n + (double)n * kL + (double)kL * kL);
  TreeGeom g = make_geom(H);
  size_t smem = sizeof(cx<R>) * ((size_t)n * n + (size_t)n * kL + n) + sizeof(R) * n + sizeof(int) * n + 64;
  LS_CUDA_TRY(cudaFuncSetAttribute(leaf_build_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int tk = prof_begin(st);
  count_launch();
  leaf_build_kernel<R><<<(unsigned)nleaf, 256, smem, st>>>(g, H->b, H->kappa * H->kappa,
                                                          reinterpret_cast<const cx<R>*>(H->Gleaf),
                                                          reinterpret_cast<const cx<R>*>(lf.U), kL,
                                                          reinterpret_cast<cx<R>*>(lf.X),
                                                          reinterpret_cast<cx<R>*>(H->XBU),
                                                          reinterpret_cast<cx<R>*>(lf.S), H->d_err);
  if ((rc = check_launch("leaf_build"))) return rc;
  {
    double fl = nleaf * (8.0 * n * n * n + 8.0 * n * n * kL + 8.0 * kL * n * kL);
    prof_end(tk, PR_LEAF, st, sizeof(cx<R>) * nleaf * ((double)n * n + (double)n * kL + (double)kL * kL) + 8.0 * nleaf * n,
             fl);
    H->flops_build += fl;
  }

  // merges, level by level
  for (int l = L - 1; l >= 0; --l) {
    LevelData& lv = H->lev[l];
    const LevelData& ch = H->lev[l + 1];
    const int P = 1 << l, kc = ch.k, n2 = 2 * kc;
    if ((rc = dalloc(&lv.X, sizeof(cx<R>) * (size_t)P * std::max(n2 * n2, 1)))) return rc;
    H->factor_bytes += sizeof(cx<R>) * (double)P * n2 * n2;
    cx<R>* X = reinterpret_cast<cx<R>*>(lv.X);
    const cx<R>* Sc = reinterpret_cast<const cx<R>*>(ch.S);
    const cx<R>* Gs = reinterpret_cast<const cx<R>*>(ch.Gsib);
    if (kc > 0) {
      long long tot = (long long)P * n2 * kc;
      int tg = prof_begin(st);
      count_launch();
      merge_identity_kernel<R><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(X, kc, P);
      // X[0:kc, kc:] = S_a G ; X[kc:, 0:kc] = S_b G^T
      gemm<R>(st, false, false, kc, kc, kc, one<R>(), Sc, kc, 2LL * kc * kc, Gs, kc, 0, zero<R>(), X + kc, n2,
              (long long)n2 * n2, P);
      gemm<R>(st, false, true, kc, kc, kc, one<R>(), Sc + (size_t)kc * kc, kc, 2LL * kc * kc, Gs, kc, 0, zero<R>(),
              X + (size_t)kc * n2, n2, (long long)n2 * n2, P);
      if ((rc = check_launch("merge gemm"))) return rc;
      prof_end(tg, PR_MERGE_GEMM, st, sizeof(cx<R>) * P * (3.0 * kc * kc), P * 2.0 * 8.0 * (double)kc * kc * kc);
      int ti = prof_begin(st);
      if ((rc = invert_batch<R>(H, X, n2, P, st))) return rc;
      prof_end(ti, PR_MERGE_INV, st, sizeof(cx<R>) * P * 2.0 * n2 * n2, P * 8.0 * (double)n2 * n2 * n2);
    }
    H->flops_build += P * (2.0 * 8 * (double)kc * kc * kc + 8.0 * (double)n2 * n2 * n2);
    if (l == 0) break;
    const int kp = lv.k;
    if ((rc = dalloc(&lv.S, sizeof(cx<R>) * (size_t)P * std::max(kp * kp, 1)))) return rc;
    H->factor_bytes += sizeof(cx<R>) * (double)P * kp * kp;
    if (kp == 0 || kc == 0) continue;
    const cx<R>* U = reinterpret_cast<const cx<R>*>(lv.U);  // n2 x kp
    cx<R>* D = reinterpret_cast<cx<R>*>(H->work);          // P x n2 x kp
    cx<R>* E = D + (size_t)P * n2 * kp;
    // D = [S_a U_top ; S_b U_bot]
    int ts = prof_begin(st);
    gemm<R>(st, false, false, kc, kp, kc, one<R>(), Sc, kc, 2LL * kc * kc, U, kp, 0, zero<R>(), D, kp,
            (long long)n2 * kp, P);
    gemm<R>(st, false, false, kc, kp, kc, one<R>(), Sc + (size_t)kc * kc, kc, 2LL * kc * kc, U + (size_t)kc * kp, kp,
            0, zero<R>(), D + (size_t)kc * kp, kp, (long long)n2 * kp, P);
    // E = X D ; S = U^T E
    gemm<R>(st, false, false, n2, kp, n2, one<R>(), X, n2, (long long)n2 * n2, D, kp, (long long)n2 * kp, zero<R>(),
            E, kp, (long long)n2 * kp, P);
    gemm<R>(st, true, false, kp, kp, n2, one<R>(), U, kp, 0, E, kp, (long long)n2 * kp, zero<R>(),
            reinterpret_cast<cx<R>*>(lv.S), kp, (long long)kp * kp, P);
    if ((rc = check_launch("merge S"))) return rc;
    {
      double fl = P * (2.0 * 8 * (double)kc * kc * kp + 8.0 * (double)n2 * n2 * kp + 8.0 * (double)kp * n2 * kp);
      prof_end(ts, PR_MERGE_GEMM, st, sizeof(cx<R>) * P * ((double)n2 * n2 + 2.0 * kc * kc + (double)kp * kp), fl);
      H->flops_build += fl;
    }
  }
  int herr = 0;
  LS_CUDA_TRY(cudaMemcpyAsync(&herr, H->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  LS_CUDA_TRY(cudaStreamSynchronize(st));
  if (herr) return herr;
  // bytes of one apply: every X, S, XBU read once, plus the leaf vectors
  double fb = H->factor_bytes;
  H->bytes_apply = fb + (double)H->grid.nx * H->grid.ny * (16.0 * 2);
  return LS_OK;
}

// ------------------------------------------------------------- apply
template <class R>
__global__ void gather_leaves_kernel(TreeGeom g, const z64* __restrict__ f, cx<R>* __restrict__ F) {
  const int n = g.s * g.s;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long nl = 1LL << g.L;
  if (t >= nl * n) return;
  int leaf = (int)(t / n), i = (int)(t % n);
  int ox, oy;
  leaf_origin(g, leaf, ox, oy);
  int lx = i % g.s, ly = i / g.s;
  F[t] = cvt<R>(f[(long long)(oy + ly) * g.nx + ox + lx]);
}

template <class R>
__global__ void scatter_leaves_kernel(TreeGeom g, const cx<R>* __restrict__ Q, z64* __restrict__ q) {
  const int n = g.s * g.s;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long nl = 1LL << g.L;
  if (t >= nl * n) return;
  int leaf = (int)(t / n), i = (int)(t % n);
  int ox, oy;
  leaf_origin(g, leaf, ox, oy);
  int lx = i % g.s, ly = i / g.s;
  q[(long long)(oy + ly) * g.nx + ox + lx] = cvt<double>(Q[t]);
}

template <class R>
int apply_t(ls_handle* H, const z64* f, z64* q, cudaStream_t st) {
  const int L = H->L, n = H->s * H->s;
  const long long nleaf = 1LL << L;
  TreeGeom g = make_geom(H);
  cx<R>* F = reinterpret_cast<cx<R>*>(H->work);  // leaf blocks of f
  cx<R>* Rl = F + nleaf * n;                      // r = X f on the leaves
  cx<R>* p = Rl + nleaf * n;
  std::vector<cx<R>*> rt(L + 1), wt(L + 1), tmp(L + 1);
  for (int l = 1; l <= L; ++l) {
    size_t sz = ((size_t)1 << l) * std::max(1, H->lev[l].k) * 2;
    rt[l] = p;
    p += sz;
    wt[l] = p;
    p += sz;
    tmp[l] = p;
    p += sz;
  }
  count_launch();
  gather_leaves_kernel<R><<<(unsigned)((nleaf * n + 255) / 256), 256, 0, st>>>(g, f, F);
  const LevelData& lf = H->lev[L];
  const int kL = lf.k;
  const cx<R>* XL = reinterpret_cast<const cx<R>*>(lf.X);
  gemm<R>(st, false, false, n, 1, n, one<R>(), XL, n, (long long)n * n, F, 1, n, zero<R>(), Rl, 1, n, (int)nleaf);
  gemm<R>(st, true, false, kL, 1, n, one<R>(), reinterpret_cast<const cx<R>*>(lf.U), kL, 0, Rl, 1, n, zero<R>(), rt[L],
          1, kL, (int)nleaf);
  // upward pass: r_tau = U^T X [r_a; r_b]
  for (int l = L - 1; l >= 1; --l) {
    const int P = 1 << l, kc = H->lev[l + 1].k, n2 = 2 * kc, kp = H->lev[l].k;
    const cx<R>* X = reinterpret_cast<const cx<R>*>(H->lev[l].X);
    // X [r_a; r_b] goes to the child-level scratch, which holds 2 P n2 entries
    gemm<R>(st, false, false, n2, 1, n2, one<R>(), X, n2, (long long)n2 * n2, rt[l + 1], 1, n2, zero<R>(), tmp[l + 1],
            1, n2, P);
    gemm<R>(st, true, false, kp, 1, n2, one<R>(), reinterpret_cast<const cx<R>*>(H->lev[l].U), kp, 0, tmp[l + 1], 1,
            n2, zero<R>(), rt[l], 1, kp, P);
  }
  // root: q = X_0 [r_a; r_b]; w_a = G q_b, w_b = G^T q_a
  {
    const int kc = H->lev[1].k, n2 = 2 * kc;
    cx<R>* qr = tmp[1];
    gemm<R>(st, false, false, n2, 1, n2, one<R>(), reinterpret_cast<const cx<R>*>(H->lev[0].X), n2, 0, rt[1], 1, 0,
            zero<R>(), qr, 1, 0, 1);
    const cx<R>* G1 = reinterpret_cast<const cx<R>*>(H->lev[1].Gsib);
    gemm<R>(st, false, false, kc, 1, kc, one<R>(), G1, kc, 0, qr + kc, 1, 0, zero<R>(), wt[1], 1, 0, 1);
    gemm<R>(st, true, false, kc, 1, kc, one<R>(), G1, kc, 0, qr, 1, 0, zero<R>(), wt[1] + kc, 1, 0, 1);
  }
  // downward pass, l = 1 .. L-1
  for (int l = 1; l <= L - 1; ++l) {
    const int P = 1 << l, kc = H->lev[l + 1].k, n2 = 2 * kc, kp = H->lev[l].k;
    const cx<R>* U = reinterpret_cast<const cx<R>*>(H->lev[l].U);
    const cx<R>* Sc = reinterpret_cast<const cx<R>*>(H->lev[l + 1].S);
    const cx<R>* X = reinterpret_cast<const cx<R>*>(H->lev[l].X);
    const cx<R>* Gs = reinterpret_cast<const cx<R>*>(H->lev[l + 1].Gsib);
    cx<R>* Uw = wt[l + 1];  // U w_tau, laid out as the children's incoming expansions
    cx<R>* t = tmp[l + 1];  // [r_a; r_b] - diag(S_a, S_b) U w_tau
    gemm<R>(st, false, false, n2, 1, kp, one<R>(), U, kp, 0, wt[l], 1, kp, zero<R>(), Uw, 1, n2, P);
    LS_CUDA_TRY(cudaMemcpyAsync(t, rt[l + 1], sizeof(cx<R>) * (size_t)P * n2, cudaMemcpyDeviceToDevice, st));
    const cx<R> mone = mk<R>(R(-1), R(0));
    gemm<R>(st, false, false, kc, 1, kc, mone, Sc, kc, 2LL * kc * kc, Uw, 1, n2, one<R>(), t, 1, n2, P);
    gemm<R>(st, false, false, kc, 1, kc, mone, Sc + (size_t)kc * kc, kc, 2LL * kc * kc, Uw + kc, 1, n2, one<R>(),
            t + kc, 1, n2, P);
    // q = X t overwrites [r_a; r_b], which no later step reads
    cx<R>* qbuf = rt[l + 1];
    gemm<R>(st, false, false, n2, 1, n2, one<R>(), X, n2, (long long)n2 * n2, t, 1, n2, zero<R>(), qbuf, 1, n2, P);
    // w_a = U w_top + G q_b ; w_b = U w_bot + G^T q_a  (Uw already in place)
    gemm<R>(st, false, false, kc, 1, kc, one<R>(), Gs, kc, 0, qbuf + kc, 1, n2, one<R>(), Uw, 1, n2, P);
    gemm<R>(st, true, false, kc, 1, kc, one<R>(), Gs, kc, 0, qbuf, 1, n2, one<R>(), Uw + kc, 1, n2, P);
  }
  // leaves: q = r - XBU w
  gemm<R>(st, false, false, n, 1, kL, mk<R>(R(-1), R(0)), reinterpret_cast<const cx<R>*>(H->XBU), kL,
          (long long)n * kL, wt[L], 1, kL, one<R>(), Rl, 1, n, (int)nleaf);
  count_launch();
  scatter_leaves_kernel<R><<<(unsigned)((nleaf * n + 255) / 256), 256, 0, st>>>(g, Rl, q);
  return check_launch("hbs_apply");
}

}  // namespace

int hbs_build(ls_handle* H, cudaStream_t st) {
  return H->prec == LS_FP64 ? build_t<double>(H, st) : build_t<float>(H, st);
}

int hbs_apply(ls_handle* H, const z64* f, z64* q, int nrhs, cudaStream_t st) {
  const long long N = (long long)H->grid.nx * H->grid.ny;
  for (int r = 0; r < nrhs; ++r) {
    int tk = prof_begin(st);
    int rc = H->prec == LS_FP64 ? apply_t<double>(H, f + r * N, q + r * N, st) : apply_t<float>(H, f + r * N, q + r * N, st);
    if (rc) return rc;
    prof_end(tk, PR_APPLY, st, H->bytes_apply, 0.0);
  }
  return LS_OK;
}

}  // namespace ls
