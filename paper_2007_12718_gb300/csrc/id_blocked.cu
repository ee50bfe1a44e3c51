// Blocked row ID for the per-level compression (Sec. 2.1: the ID from a
// column-pivoted QR of the transposed block; Sec. 3.2: one proxy block per
// level, local tolerance eps * ||block||_F).
//
// The greedy column-pivoted QR picks one pivot per step, each step a global
// agreement over every candidate.  Here the pivots are taken in blocks of up
// to kB, with the trailing matrix updated by GEMM-shaped kernels in between:
//
//   A (m x p, candidate-major) is factored as A(perm) = L Q + A_trail, Q with
//   orthonormal rows, L lower trapezoidal, A_trail the explicit residual of
//   the candidates not yet chosen (kept in place of A).
//
// Per block, with the trailing rows at positions [k, m):
//   1. pool: the kPool trailing rows of largest residual norm (the last block
//      of the previous update kernel chooses them); `outside` is the largest
//      residual norm of the trailing rows not in the pool.
//   2. the pool's Gram matrix G = A_P A_P^H (gram_kernel, partial sums over
//      column slices) and a greedy pivoted Cholesky of G (pchol_kernel): the
//      same pivot order as the column-pivoted QR restricted to the pool.  A
//      pool candidate is accepted only while its residual norm^2 is at least
//      kAlpha2 * outside (norms never grow under projection, so every accepted
//      pivot is within a factor sqrt(kAlpha2) of the largest residual over all
//      candidates), at most kB per block.
//   3. the accepted rows are swapped to positions [k, k + be) (swapq_kernel),
//      and Q_b = L_bb^-1 A(J_b) by forward substitution, L_bb the Cholesky
//      factor of the accepted rows.
//   4. C = A_trail Q_b^H for the other trailing rows (proj_kernel), stored as
//      block column of L.  With ||A_trail||_F^2 known at the block start, the
//      residual after j of the block's pivots is ||A_trail||^2 - sum_{i<j}
//      ||C(:, i)||^2 (the pivot rows contribute their L_bb columns); the first
//      j at which that is <= (eps ||A||_F)^2 ends the factorisation.
//   5. A_trail -= C Q_b over the accepted columns (update_kernel), which also
//      recomputes every trailing row's norm, the exact trailing total (the
//      stopping test is repeated on it: the factorisation ends only when the
//      explicit residual is below the tolerance), and the next pool.
//
// At the end R = L^T in the column-pivoted QR's terms (A^T(:, J) = Q^T L_JJ^T):
// R11 = L(J, :)^T, R12 = L(J^c, :)^T, and the interpolation matrix T =
// R11^-1 R12 is formed by the same blocked back substitution as the greedy
// kernels use (the caller launches it on Rm, RT, sel, rank written here).
//
// Every kernel reads the block's sizes from the device state and returns at
// once when the factorisation is done, so the host queues blocks without
// waiting for each one; it reads the state back two blocks behind.  Sums are
// taken in a fixed order (per-block partials, summed by the last block of a
// launch), so the pivots are the same run after run.
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "handle.h"
#include "prof.h"

namespace ls {
namespace bid {

constexpr int kB = 32;          // pivots per block, at most
constexpr int kPool = 64;       // pool rows per block
constexpr int kUR = 16;         // rows per block of update_kernel
constexpr int kCR = 64;         // rows per block of proj_kernel
constexpr int kGramMax = 32;    // blocks of gram_kernel, at most
constexpr int kGramCols = 32;   // columns per stage of gram_kernel
constexpr double kAlpha2 = 0.25;

struct State {
  int k;        // accepted pivots: the trailing rows are positions [k, m)
  int be;       // pivots chosen in the current block
  int jb;       // of those, the ones the update applies (be, or fewer at the stop)
  int done;     // 1 once the rank is final (k)
  int npool;    // rows in the pool
  unsigned ticket;  // completion counter of the launch in progress (reset by its last block)
  double thr;   // (eps ||A||_F)^2
  double tot;   // ||A_trail||_F^2 at the start of the block
  double outside;   // largest residual norm^2 of a trailing row outside the pool
  int pool[kPool];  // positions of the pool rows, largest norm first
  int swp[kB];      // position k + i is swapped with swp[i], in the order i = 0, 1, ...
};

template <class R>
__device__ __forceinline__ cx<R> czero() {
  return mk<R>(R(0), R(0));
}

// Block-wide sum of one double per thread in a fixed order (blockDim.x = 256).
__device__ double block_sum256(double v, double* sh) {
  const int tid = threadIdx.x;
  for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((tid & 31) == 0) sh[tid >> 5] = v;
  __syncthreads();
  double t = 0;
  if (tid == 0)
    for (int w = 0; w < 8; ++w) t += sh[w];
  __syncthreads();
  if (tid == 0) sh[0] = t;
  __syncthreads();
  const double r = sh[0];
  __syncthreads();
  return r;
}

// Order of candidates for the pool: larger norm first, lower position on ties.
__device__ __forceinline__ bool better(double na, int pa, double nb, int pb) {
  return na > nb || (na == nb && pa < pb);
}

// The last block of a launch: every block fences its results and takes a
// ticket; the block that takes ticket gridDim.x - 1 sees all of them.
__device__ __forceinline__ bool last_block(unsigned* ticket) {
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}

// Pool selection over the trailing norms (last block of update_kernel, 256
// threads): every thread keeps its three best candidates of a strided slice;
// the union of their first two (512 entries) is sorted, the first kPool form
// the pool, and `outside` is the largest norm left out (sorted entries past
// kPool and every thread's third).
__device__ void select_pool(const double* __restrict__ norms, int k, int m, State* S) {
  __shared__ double sn[512];
  __shared__ int sp[512];
  __shared__ double s_third[256];
  const int tid = threadIdx.x;
  double n0 = -1, n1 = -1, n2 = -1;
  int p0 = 0x7fffffff, p1 = 0x7fffffff, p2 = 0x7fffffff;
  for (int q = k + tid; q < m; q += 256) {
    const double v = __ldcg(norms + q);
    if (better(v, q, n0, p0)) {
      n2 = n1; p2 = p1; n1 = n0; p1 = p0; n0 = v; p0 = q;
    } else if (better(v, q, n1, p1)) {
      n2 = n1; p2 = p1; n1 = v; p1 = q;
    } else if (better(v, q, n2, p2)) {
      n2 = v; p2 = q;
    }
  }
  sn[2 * tid] = n0; sp[2 * tid] = p0;
  sn[2 * tid + 1] = n1; sp[2 * tid + 1] = p1;
  s_third[tid] = n2;
  __syncthreads();
  // bitonic sort of 512 entries, best first
  for (int size = 2; size <= 512; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int e = tid; e < 256; e += 256) {
        const int i = 2 * stride * (e / stride) + (e % stride), j = i + stride;
        const bool desc = ((i / size) & 1) == 0;  // best-first runs in even segments
        const bool swap_ = desc ? better(sn[j], sp[j], sn[i], sp[i]) : better(sn[i], sp[i], sn[j], sp[j]);
        if (swap_) {
          double tn = sn[i]; sn[i] = sn[j]; sn[j] = tn;
          int tp = sp[i]; sp[i] = sp[j]; sp[j] = tp;
        }
      }
      __syncthreads();
    }
  if (tid < kPool) S->pool[tid] = sp[tid];
  if (tid == 0) {
    int np = 0;
    while (np < kPool && sn[np] >= 0) ++np;
    double out = np < 512 && sn[kPool] > 0 ? sn[kPool] : 0.0;
    for (int t = 0; t < 256; ++t) out = fmax(out, s_third[t]);
    S->npool = np;
    S->outside = out;
  }
  __syncthreads();
}

// A_trail(r, :) -= sum_{i < jb} L(r, k0 + i) Q(i, :) for the trailing rows
// r >= k0 + jb (nothing to subtract when first), then every such row's norm^2,
// the trailing total and, in the last block, the stopping test and the next
// pool.  kUR rows per block, columns strided over the 256 threads.
template <class R>
__global__ void __launch_bounds__(256) update_kernel(cx<R>* __restrict__ A, int m, int p, int kmax,
                                                     const cx<R>* __restrict__ Lm, int ldl,
                                                     const cx<R>* __restrict__ Q, double* __restrict__ norms,
                                                     double* __restrict__ part, State* __restrict__ S, double eps2,
                                                     int first) {
  __shared__ cx<R> Cs[kUR][kB];
  __shared__ double red[8][kUR];
  __shared__ double sh[8];
  if (S->done) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int k0 = first ? 0 : S->k;
  const int jb = first ? 0 : S->jb;
  const int r0 = k0 + jb + blockIdx.x * kUR;
  const int nr = max(0, min(kUR, m - r0));
  for (int e = tid; e < kUR * kB; e += 256) {
    const int r = e / kB, i = e % kB;
    Cs[r][i] = (r < nr && i < jb) ? Lm[(long long)(r0 + r) * ldl + k0 + i] : czero<R>();
  }
  __syncthreads();
  R nrm[kUR];
#pragma unroll
  for (int r = 0; r < kUR; ++r) nrm[r] = R(0);
  if (nr > 0) {
    for (int c = tid; c < p; c += 256) {
      cx<R> a[kUR];
#pragma unroll
      for (int r = 0; r < kUR; ++r) a[r] = r < nr ? A[(long long)(r0 + r) * p + c] : czero<R>();
      if (jb > 0) {
        for (int i = 0; i < jb; ++i) {
          const cx<R> q = Q[(long long)i * p + c];
#pragma unroll
          for (int r = 0; r < kUR; ++r) {
            const cx<R> cc = Cs[r][i];
            a[r].re -= cc.re * q.re - cc.im * q.im;
            a[r].im -= cc.re * q.im + cc.im * q.re;
          }
        }
#pragma unroll
        for (int r = 0; r < kUR; ++r)
          if (r < nr) A[(long long)(r0 + r) * p + c] = a[r];
      }
#pragma unroll
      for (int r = 0; r < kUR; ++r) nrm[r] += abs2(a[r]);
    }
  }
#pragma unroll
  for (int r = 0; r < kUR; ++r) {
    double v = (double)nrm[r];
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][r] = v;
  }
  __syncthreads();
  if (tid < kUR) {
    double v = 0;
    for (int w = 0; w < 8; ++w) v += red[w][tid];
    red[0][tid] = v;
    if (tid < nr) norms[r0 + tid] = v;
  }
  __syncthreads();
  if (tid == 0) {
    double t = 0;
    for (int r = 0; r < nr; ++r) t += red[0][r];
    part[blockIdx.x] = t;
  }
  if (!last_block(&S->ticket)) return;
  double v = 0;
  for (int b = tid; b < (int)gridDim.x; b += 256) v += __ldcg(part + b);
  const double tot = block_sum256(v, sh);
  const int k = k0 + jb;
  __shared__ int s_done;
  if (tid == 0) {
    S->ticket = 0;
    if (first) S->thr = eps2 * tot;
    const double thr = first ? eps2 * tot : S->thr;
    S->tot = tot;
    S->k = k;
    s_done = (tot <= thr || k >= kmax || k >= m) ? 1 : 0;
    if (s_done) S->done = 1;
  }
  __syncthreads();
  if (s_done) return;
  select_pool(norms, k, m, S);
}

// Partial Gram matrices of the pool rows over column slices:
// gp[b][i * kPool + j] = sum_{t in slice b} A(pool_i, t) conj(A(pool_j, t)).
// 256 threads, a 4 x 4 tile of (i, j) per thread.
template <class R>
__global__ void __launch_bounds__(256) gram_kernel(const cx<R>* __restrict__ A, int p,
                                                   const State* __restrict__ S, cx<R>* __restrict__ gp) {
  __shared__ cx<R> T[kPool][kGramCols + 1];
  __shared__ int pool[kPool];
  if (S->done) return;
  const int tid = threadIdx.x, np = S->npool;
  if (tid < kPool) pool[tid] = tid < np ? S->pool[tid] : -1;
  const int ti = tid >> 4, tj = tid & 15;
  cx<R> acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = czero<R>();
  const int nst = (p + kGramCols - 1) / kGramCols;  // column stages
  const int per = (nst + gridDim.x - 1) / gridDim.x;
  const int s0 = blockIdx.x * per, s1 = min(nst, s0 + per);
  __syncthreads();
  for (int s = s0; s < s1; ++s) {
    const int c0 = s * kGramCols;
    for (int e = tid; e < kPool * kGramCols; e += 256) {
      const int r = e / kGramCols, c = e % kGramCols;
      const int row = pool[r];
      T[r][c] = (row >= 0 && c0 + c < p) ? A[(long long)row * p + c0 + c] : czero<R>();
    }
    __syncthreads();
#pragma unroll 4
    for (int c = 0; c < kGramCols; ++c) {
      cx<R> a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = T[4 * ti + u][c];
#pragma unroll
      for (int v = 0; v < 4; ++v) b[v] = T[4 * tj + v][c];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) fmac_(acc[u][v], b[v], a[u]);  // a_i conj(a_j)
    }
    __syncthreads();
  }
  cx<R>* g = gp + (size_t)blockIdx.x * kPool * kPool;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) g[(4 * ti + u) * kPool + 4 * tj + v] = acc[u][v];
}

// Greedy pivoted Cholesky of the pool's Gram matrix (one block of 256
// threads): the pivot is the pool row of largest residual norm^2 d_i (lowest
// pool index on ties); the block ends at kB pivots, when d_best < kAlpha2 *
// outside, when d_best <= drange * d_first (beyond that the Gram matrix's
// rounding would decide the order), at the rank limit, or at a non-positive d.
// Writes the accepted pivots' Cholesky rows L_bb (be x be, lower), be, and the
// swap sequence that brings the pivots to positions [k, k + be); applies it to perm.
template <class R>
__global__ void __launch_bounds__(256) pchol_kernel(const cx<R>* __restrict__ gp, int ngp, int kmax,
                                                    State* __restrict__ S, int* __restrict__ perm,
                                                    cx<R>* __restrict__ Lbb, double drange) {
  extern __shared__ unsigned char smraw[];
  cx<double>* G = reinterpret_cast<cx<double>*>(smraw);  // kPool x kPool
  cx<double>* Lc = G + kPool * kPool;                     // kPool x kB
  __shared__ double d[kPool];
  __shared__ int chosen[kPool], order[kB];
  __shared__ int s_best, s_stop, s_be;
  __shared__ double s_dbest, s_d0;
  if (S->done) return;
  const int tid = threadIdx.x;
  const int np = S->npool, k = S->k;
  const double outside = S->outside;
  for (int e = tid; e < kPool * kPool; e += 256) {
    cx<double> s = mk<double>(0.0, 0.0);
    for (int b = 0; b < ngp; ++b) s = s + cvt<double>(gp[(size_t)b * kPool * kPool + e]);
    G[e] = s;
  }
  for (int e = tid; e < kPool * kB; e += 256) Lc[e] = mk<double>(0.0, 0.0);
  if (tid < kPool) {
    chosen[tid] = tid < np ? 0 : 1;
    d[tid] = 0;
  }
  __syncthreads();
  if (tid < np) d[tid] = G[tid * kPool + tid].re;
  __syncthreads();
  const int jmax = min(kB, min(np, kmax - k));
  int j = 0;
  for (; j < jmax; ++j) {
    if (tid < 32) {  // warp 0: argmax over the pool
      double bv = -1;
      int bi = 0x7fffffff;
      for (int i = tid; i < kPool; i += 32)
        if (!chosen[i] && (d[i] > bv || (d[i] == bv && i < bi))) {
          bv = d[i];
          bi = i;
        }
      for (int o = 16; o; o >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, bv, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) {
          bv = ov;
          bi = oi;
        }
      }
      if (tid == 0) {
        if (j == 0) s_d0 = bv;
        const bool stop = bi >= kPool || !(bv > 0) || (outside > 0 && bv < kAlpha2 * outside) ||
                          (j > 0 && bv <= drange * s_d0);
        s_stop = stop ? 1 : 0;
        s_best = bi;
        s_dbest = bv;
      }
    }
    __syncthreads();
    if (s_stop) break;
    const int best = s_best;
    const double sd = sqrt(s_dbest);
    if (tid < np) {
      cx<double> v = G[tid * kPool + best];  // <a_i, a_best>
      for (int jj = 0; jj < j; ++jj) {
        const cx<double> a = Lc[tid * kB + jj], bconj = conjz(Lc[best * kB + jj]);
        v = v - a * bconj;
      }
      v = scale(v, 1.0 / sd);
      if (tid == best) v = mk<double>(sd, 0.0);
      Lc[tid * kB + j] = v;
    }
    __syncthreads();
    if (tid < np) d[tid] = chosen[tid] || tid == best ? 0.0 : d[tid] - abs2(Lc[tid * kB + j]);
    if (tid == 0) {
      chosen[best] = 1;
      order[j] = best;
    }
    __syncthreads();
  }
  if (tid == 0) s_be = j;
  __syncthreads();
  const int be = s_be;
  for (int e = tid; e < kB * kB; e += 256) {
    const int i = e / kB, jj = e % kB;
    cx<double> v = mk<double>(0.0, 0.0);
    if (i < be && jj <= i) v = Lc[order[i] * kB + jj];
    Lbb[e] = cvt<R>(v);
  }
  if (tid == 0) {
    // swap sequence: position k + i receives the pivot order[i]; a pivot that
    // sat at k + i' (i' < i) was moved to swp[i'] by swap i'
    for (int i = 0; i < be; ++i) {
      int x = S->pool[order[i]];
      for (int i2 = 0; i2 < i; ++i2)
        if (x == k + i2) x = S->swp[i2];
      S->swp[i] = x;
      const int a = k + i;
      if (x != a) {
        const int t = perm[a];
        perm[a] = perm[x];
        perm[x] = t;
      }
    }
    S->be = be;
    if (be == 0) S->done = 1;  // no admissible pivot left (the Gram matrix is numerically zero)
  }
}

// Swaps of the accepted rows into positions [k, k + be) and Q_b = L_bb^-1 A(J_b)
// (blocks [0, nqa): one column of A per thread), and the same swaps in the
// columns [0, k) of L plus the block's diagonal L_bb (blocks [nqa, ...): one
// column of L per thread).
template <class R>
__global__ void __launch_bounds__(256) swapq_kernel(cx<R>* __restrict__ A, int p, cx<R>* __restrict__ Lm, int ldl,
                                                    const cx<R>* __restrict__ Lbb, cx<R>* __restrict__ Q,
                                                    cx<R>* __restrict__ Qc, const State* __restrict__ S, int nqa) {
  __shared__ int sw[kB];
  __shared__ cx<R> Lb[kB][kB + 1];
  if (S->done) return;
  const int tid = threadIdx.x, k = S->k, be = S->be;
  if (tid < kB) sw[tid] = tid < be ? S->swp[tid] : 0;
  for (int e = tid; e < kB * kB; e += 256) Lb[e / kB][e % kB] = Lbb[e];
  __syncthreads();
  if ((int)blockIdx.x < nqa) {
    const int c = blockIdx.x * 256 + tid;
    if (c >= p) return;
    for (int i = 0; i < be; ++i) {
      const int a = k + i, x = sw[i];
      if (x != a) {
        const cx<R> t = A[(long long)a * p + c];
        A[(long long)a * p + c] = A[(long long)x * p + c];
        A[(long long)x * p + c] = t;
      }
    }
    cx<R> q[kB];
#pragma unroll
    for (int i = 0; i < kB; ++i) {
      if (i < be) {
        cx<R> x = A[(long long)(k + i) * p + c];
#pragma unroll
        for (int jj = 0; jj < i; ++jj) {
          const cx<R> l = Lb[i][jj];
          x.re -= l.re * q[jj].re - l.im * q[jj].im;
          x.im -= l.re * q[jj].im + l.im * q[jj].re;
        }
        q[i] = scale(x, R(1) / Lb[i][i].re);
        Q[(long long)i * p + c] = q[i];
        Qc[(long long)i * p + c] = conjz(q[i]);
      } else {
        q[i] = czero<R>();
      }
    }
  } else {
    const int c = (blockIdx.x - nqa) * 256 + tid;
    if (c < k) {
      for (int i = 0; i < be; ++i) {
        const int a = k + i, x = sw[i];
        if (x != a) {
          const cx<R> t = Lm[(long long)a * ldl + c];
          Lm[(long long)a * ldl + c] = Lm[(long long)x * ldl + c];
          Lm[(long long)x * ldl + c] = t;
        }
      }
    } else if (c < k + be) {
      const int jj = c - k;
      for (int i = 0; i < be; ++i) Lm[(long long)(k + i) * ldl + c] = jj <= i ? Lb[i][jj] : czero<R>();
    }
  }
}

// C = A_trail(rows, :) Q_b^H for the trailing rows after the block's pivots
// (positions [k + be, m)), written to L(rows, k .. k + be).  kCR x kB outputs
// per block, 8 per thread, K (= p) staged 16 columns at a time.  Each block
// also writes the column sums of |C|^2; the last block adds the pivot rows'
// part (the columns of L_bb) and finds the first j at which the residual
// ||A_trail||^2 - sum_{i <= j} ||C(:, i)||^2 is within the tolerance.
template <class R>
__global__ void __launch_bounds__(256) proj_kernel(const cx<R>* __restrict__ A, int m, int p,
                                                   cx<R>* __restrict__ Lm, int ldl, const cx<R>* __restrict__ Qc,
                                                   const cx<R>* __restrict__ Lbb, double* __restrict__ cpart,
                                                   State* __restrict__ S) {
  constexpr int KC = 16;
  __shared__ cx<R> As[KC][kCR + 1];
  __shared__ cx<R> Bs[KC][kB + 1];
  __shared__ double cs[32][kB + 1];
  if (S->done) return;
  const int tid = threadIdx.x, k = S->k, be = S->be;
  const int r0 = k + be + blockIdx.x * kCR;
  const int nr = max(0, min(kCR, m - r0));
  const int tx = tid & 7, ty = tid >> 3;  // rows ty, ty + 32; columns tx + 8 v
  cx<R> acc[2][4];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = czero<R>();
  if (nr > 0) {
    for (int t0 = 0; t0 < p; t0 += KC) {
#pragma unroll
      for (int r = 0; r < (KC * kCR) / 256; ++r) {
        const int e = tid + 256 * r, kk = e % KC, i = e / KC;
        As[kk][i] = (i < nr && t0 + kk < p) ? A[(long long)(r0 + i) * p + t0 + kk] : czero<R>();
      }
#pragma unroll
      for (int r = 0; r < (KC * kB) / 256; ++r) {
        const int e = tid + 256 * r, kk = e % KC, j = e / KC;
        Bs[kk][j] = (j < be && t0 + kk < p) ? Qc[(long long)j * p + t0 + kk] : czero<R>();
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < KC; ++kk) {
        const cx<R> a0 = As[kk][ty], a1 = As[kk][ty + 32];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const cx<R> bb = Bs[kk][tx + 8 * v];
          fma_(acc[0][v], a0, bb);
          fma_(acc[1][v], a1, bb);
        }
      }
      __syncthreads();
    }
  }
  double csum[4] = {0, 0, 0, 0};
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int i = ty + 32 * u;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int j = tx + 8 * v;
      if (i < nr && j < be) {
        Lm[(long long)(r0 + i) * ldl + k + j] = acc[u][v];
        csum[v] += (double)abs2(acc[u][v]);
      }
    }
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) cs[ty][tx + 8 * v] = csum[v];
  __syncthreads();
  if (tid < kB) {
    double t = 0;
    for (int y = 0; y < 32; ++y) t += cs[y][tid];
    cpart[(size_t)blockIdx.x * kB + tid] = t;
  }
  if (!last_block(&S->ticket)) return;
  if (tid < kB) {
    double t = 0;
    for (int b = 0; b < (int)gridDim.x; ++b) t += __ldcg(cpart + (size_t)b * kB + tid);
    for (int i = tid; i < be; ++i) t += (double)abs2(Lbb[i * kB + tid]);
    cs[0][tid] = t;
  }
  __syncthreads();
  if (tid == 0) {
    S->ticket = 0;
    double rem = S->tot;
    const double thr = S->thr;
    int jb = be;
    for (int j = 0; j < be; ++j) {
      rem -= cs[0][j];
      if (rem <= thr) {
        jb = j + 1;
        break;
      }
    }
    S->jb = jb;
  }
}

// R = L^T in the column-pivoted QR's terms, for the back substitution:
// Rm[a][c] = L(pos(c), a) (a < k, candidate c), 32 x 32 tiles through shared memory.
template <class R>
__global__ void finish_rm_kernel(const cx<R>* __restrict__ Lm, int ldl, const int* __restrict__ pos, int m,
                                 const State* __restrict__ S, cx<R>* __restrict__ Rm) {
  __shared__ cx<R> t[32][33];
  const int k = S->k;
  const int c0 = blockIdx.x * 32, a0 = blockIdx.y * 32;
  if (a0 >= k) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  for (int y = ty; y < 32; y += 8) {
    const int c = c0 + y, a = a0 + tx;
    t[y][tx] = (c < m && a < k) ? Lm[(long long)pos[c] * ldl + a] : czero<R>();
  }
  __syncthreads();
  for (int y = ty; y < 32; y += 8) {
    const int a = a0 + y, c = c0 + tx;
    if (a < k && c < m) Rm[(long long)a * m + c] = t[tx][y];
  }
}

// pos = perm^-1, sel, piv, rank; RT[q][r] = L(q, r) (r <= q < k, stride k).
template <class R>
__global__ void finish_meta_kernel(const cx<R>* __restrict__ Lm, int ldl, const int* __restrict__ perm, int m,
                                   const State* __restrict__ S, int* __restrict__ pos, int* __restrict__ sel,
                                   int* __restrict__ piv, int* __restrict__ rank, cx<R>* __restrict__ RT) {
  const int k = S->k;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < m) {
    const int q = (int)t, c = perm[q];
    pos[c] = q;
    sel[c] = q < k ? q : -1;
    if (q < k) piv[q] = c;
  }
  if (t == 0) rank[0] = k;
  if (t < (long long)k * k) {
    const int q = (int)(t / k), r = (int)(t % k);
    RT[t] = r <= q ? Lm[(long long)q * ldl + r] : czero<R>();
  }
}

__global__ void iota_kernel(int* v, int m) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < m) v[t] = t;
}

}  // namespace bid

// Blocked row ID of the candidate-major matrix A (m x p, overwritten by the
// trailing residual).  Writes what the back substitution reads: Rm (kmax x m),
// RT (kmax x kmax, stride k), sel (m), rank (1), and the pivots piv (m, first
// k used) on the device; returns k and the pivots on the host.
template <class R>
int blocked_row_id(cx<R>* A, int m, int p, double eps, cudaStream_t st, cx<R>* Rm, cx<R>* RT, int* sel, int* rank,
                   int* piv, int* k_out, std::vector<int>* hp) {
  using namespace bid;
  const int kmax = std::min(m, p);
  const int ldl = std::max(kmax, 1);
  const int nU = (m + kUR - 1) / kUR, nC = (m + kCR - 1) / kCR;
  const int nst = (p + kGramCols - 1) / kGramCols;
  const int ngp = std::max(1, std::min(kGramMax, nst));
  const int nqa = (p + 255) / 256, nql = (kmax + 255) / 256;
  size_t off = 0;
  auto carve = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  const size_t oL = carve(sizeof(cx<R>) * (size_t)m * ldl), oQ = carve(sizeof(cx<R>) * (size_t)kB * p),
               oQc = carve(sizeof(cx<R>) * (size_t)kB * p), oLbb = carve(sizeof(cx<R>) * kB * kB),
               oN = carve(sizeof(double) * m), oPerm = carve(sizeof(int) * m), oPos = carve(sizeof(int) * m),
               oS = carve(sizeof(State)), oUp = carve(sizeof(double) * nU), oCp = carve(sizeof(double) * nC * kB),
               oG = carve(sizeof(cx<R>) * (size_t)ngp * kPool * kPool);
  char* w = nullptr;
  int rc = dalloc((void**)&w, off);
  if (rc) return rc;
  cx<R>* Lm = reinterpret_cast<cx<R>*>(w + oL);
  cx<R>* Q = reinterpret_cast<cx<R>*>(w + oQ);
  cx<R>* Qc = reinterpret_cast<cx<R>*>(w + oQc);
  cx<R>* Lbb = reinterpret_cast<cx<R>*>(w + oLbb);
  double* norms = reinterpret_cast<double*>(w + oN);
  int* perm = reinterpret_cast<int*>(w + oPerm);
  int* pos = reinterpret_cast<int*>(w + oPos);
  State* S = reinterpret_cast<State*>(w + oS);
  double* upart = reinterpret_cast<double*>(w + oUp);
  double* cpart = reinterpret_cast<double*>(w + oCp);
  cx<R>* gp = reinterpret_cast<cx<R>*>(w + oG);
  const size_t chol_smem = sizeof(cx<double>) * (size_t)kPool * (kPool + kB);
  if (cudaFuncSetAttribute(pchol_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)chol_smem) !=
      cudaSuccess) {
    dfree(w);
    LS_CUDA_TRY(cudaGetLastError());
  }
  const double drange = sizeof(R) == 4 ? 1e-4 : 1e-12;
  auto fail = [&](int r) {
    dfree(w);
    return r;
  };
  if (cudaMemsetAsync(S, 0, sizeof(State), st) != cudaSuccess) return fail(check_launch("blocked ID state"));
  count_launch();
  iota_kernel<<<(m + 255) / 256, 256, 0, st>>>(perm, m);
  count_launch();
  update_kernel<R><<<nU, 256, 0, st>>>(A, m, p, kmax, Lm, ldl, Q, norms, upart, S, eps * eps, 1);
  if ((rc = check_launch("blocked ID norms"))) return fail(rc);
  // host loop: D blocks in flight; the state (k, done) of block n - D is read
  // back (pinned copy recorded behind it) before block n is queued
  constexpr int D = 2;
  int* pin = static_cast<int*>(pinned_scratch(sizeof(int) * 4 * (D + 1)));
  if (!pin) return fail(LS_ENOMEM);
  cudaEvent_t ev[D + 1];
  for (auto& e : ev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return fail(check_launch("event"));
  int k_lb = 0;  // a lower bound of the device's k
  int nblk = 0;
  bool done = false;
  for (; !done; ++nblk) {
    if (nblk >= D) {
      const int s = (nblk - D) % (D + 1);
      if (cudaEventSynchronize(ev[s]) != cudaSuccess) break;
      k_lb = pin[4 * s];
      if (pin[4 * s + 1]) break;
    }
    if (nblk > kmax + D) break;  // every queued block accepts a pivot or ends the factorisation
    const int rows = m - k_lb;
    count_launch(5);
    gram_kernel<R><<<ngp, 256, 0, st>>>(A, p, S, gp);
    pchol_kernel<R><<<1, 256, chol_smem, st>>>(gp, ngp, kmax, S, perm, Lbb, drange);
    swapq_kernel<R><<<nqa + nql, 256, 0, st>>>(A, p, Lm, ldl, Lbb, Q, Qc, S, nqa);
    proj_kernel<R><<<std::max(1, (rows + kCR - 1) / kCR), 256, 0, st>>>(A, m, p, Lm, ldl, Qc, Lbb, cpart, S);
    update_kernel<R><<<std::max(1, (rows + kUR - 1) / kUR), 256, 0, st>>>(A, m, p, kmax, Lm, ldl, Q, norms, upart, S,
                                                                         0.0, 0);
    if ((rc = check_launch("blocked ID block"))) break;
    const int s = nblk % (D + 1);
    if (cudaMemcpyAsync(pin + 4 * s, &S->k, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(pin + 4 * s + 1, &S->done, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaEventRecord(ev[s], st) != cudaSuccess) {
      rc = check_launch("blocked ID state copy");
      break;
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (rc) return fail(rc);
  // k and done, then the outputs
  if (cudaMemcpyAsync(pin, &S->k, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(pin + 1, &S->done, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(check_launch("blocked ID result"));
  const int k = pin[0];
  if (!pin[1] || k < 0 || k > kmax) {
    set_last_error_text("blocked ID did not finish");
    return fail(LS_ECUDA);
  }
  count_launch(2);
  finish_meta_kernel<R><<<(unsigned)((std::max((long long)m, (long long)k * k) + 255) / 256), 256, 0, st>>>(
      Lm, ldl, perm, m, S, pos, sel, piv, rank, RT);
  if (k > 0)
    finish_rm_kernel<R><<<dim3((m + 31) / 32, (k + 31) / 32), 256, 0, st>>>(Lm, ldl, pos, m, S, Rm);
  if ((rc = check_launch("blocked ID finish"))) return fail(rc);
  int* pv = static_cast<int*>(pinned_scratch(sizeof(int) * (size_t)std::max(k, 1)));
  if (!pv) return fail(LS_ENOMEM);
  if (k > 0) LS_CUDA_TRY(cudaMemcpyAsync(pv, piv, sizeof(int) * k, cudaMemcpyDeviceToHost, st));
  LS_CUDA_TRY(cudaStreamSynchronize(st));
  hp->assign(std::max(k, 1), 0);
  for (int a = 0; a < k; ++a) (*hp)[a] = pv[a];
  *k_out = k;
  dfree(w);
  return LS_OK;
}

template int blocked_row_id<float>(c32*, int, int, double, cudaStream_t, c32*, c32*, int*, int*, int*, int*,
                                   std::vector<int>*);
template int blocked_row_id<double>(z64*, int, int, double, cudaStream_t, z64*, z64*, int*, int*, int*, int*,
                                    std::vector<int>*);

}  // namespace ls
