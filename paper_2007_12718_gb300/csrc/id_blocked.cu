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
// R11 = L(J, :)^T, R12 = L(J^c, :)^T, and the interpolation matrix T^T =
// R11^-1 R12, i.e. T = L(J^c, :) L(J, :)^-1, is formed by a blocked back
// substitution in place in L (diagonal blocks solved per row, GEMM updates).
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
constexpr int kTR = 64;         // rows per block of update_kernel
constexpr int kTC = 64;         // columns per chunk of update_kernel
constexpr int kCR = 64;         // rows per block of proj_kernel
constexpr int kGramMax = 32;    // blocks of gram_kernel, at most
constexpr int kGramCols = 32;   // columns per stage of gram_kernel
constexpr int kMaxSplit = 8;    // column slices of proj_kernel, at most
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
  int nu;           // positions the block's swaps touch
  int upos[2 * kB]; // those positions: k .. k + be - 1 first, then the pivots' old positions
  int usrc[2 * kB]; // after the swaps, position upos[t] holds the row that was at upos[usrc[t]]
};

template <class R>
__device__ __forceinline__ cx<R> czero() {
  return mk<R>(R(0), R(0));
}

// L2 load of a complex value written by another block of the same launch.
template <class R>
__device__ __forceinline__ cx<R> __ldcg_cx_any(const cx<R>* p) {
  return ldcg_cx(p);
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
// Norms are compared through their bit patterns (non-negative doubles order like
// the unsigned integers of their bits; integer compares avoid the FP64 pipe);
// key 0 (a zero norm) is never a candidate.
__device__ __forceinline__ bool better(unsigned long long ka, int pa, unsigned long long kb, int pb) {
  return ka > kb || (ka == kb && pa < pb);
}

// Pool selection over the trailing norms (last block of update_kernel, 256
// threads): every thread keeps its three best candidates of a strided slice;
// the union of their first two (512 entries) is sorted, the first kPool form
// the pool, and `outside` is the largest norm left out (sorted entries past
// kPool and every thread's third).
__device__ void select_pool(const double* __restrict__ norms, int k, int m, State* S) {
  typedef unsigned long long u64;
  __shared__ u64 sn[512];
  __shared__ int sp[512];
  __shared__ u64 s_third[256];
  const int tid = threadIdx.x;
  u64 n0 = 0, n1 = 0, n2 = 0;
  int p0 = 0x7fffffff, p1 = 0x7fffffff, p2 = 0x7fffffff;
  for (int q = k + tid; q < m; q += 256) {
    const u64 v = (u64)__double_as_longlong(__ldcg(norms + q));
    if (v == 0) continue;
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
      const int e = tid;
      const int i = 2 * stride * (e / stride) + (e % stride), j = i + stride;
      const bool desc = ((i / size) & 1) == 0;  // best-first runs in even segments
      const bool swap_ = desc ? better(sn[j], sp[j], sn[i], sp[i]) : better(sn[i], sp[i], sn[j], sp[j]);
      if (swap_) {
        const u64 tn = sn[i]; sn[i] = sn[j]; sn[j] = tn;
        const int tp = sp[i]; sp[i] = sp[j]; sp[j] = tp;
      }
      __syncthreads();
    }
  if (tid < kPool) S->pool[tid] = sp[tid];
  if (tid == 0) {
    int np = 0;
    while (np < kPool && sn[np] > 0) ++np;
    u64 out = sn[kPool];
    for (int t = 0; t < 256; ++t) out = out > s_third[t] ? out : s_third[t];
    S->npool = np;
    S->outside = __longlong_as_double((long long)out);
  }
  __syncthreads();
}

// A_trail(r, :) -= sum_{i < jb} L(r, k0 + i) Q(i, :) for the trailing rows
// r >= k0 + jb (nothing to subtract when first), then every such row's norm^2,
// the trailing total and, in the last block, the stopping test and the next
// pool.  Block (x, y): row tile x (kTR rows), slice y of the columns (whole
// 64-column chunks), 4 x 4 entries per thread per chunk; the block's C rows stay
// in shared memory, each chunk of Q is staged there.  Row norms: every slice
// writes its partial sums, the last block of a tile to finish adds them in
// slice order; the last tile to finish takes the total (tiles in order).
template <class R>
__global__ void __launch_bounds__(256) update_kernel(cx<R>* __restrict__ A, int m, int p, int kmax,
                                                     const cx<R>* __restrict__ Lm, int ldl,
                                                     const cx<R>* __restrict__ Q, double* __restrict__ norms,
                                                     double* __restrict__ npart, unsigned* __restrict__ tile_ticket,
                                                     double* __restrict__ part, State* __restrict__ S, double eps2,
                                                     int first) {
  extern __shared__ unsigned char smraw[];
  auto Cs = reinterpret_cast<cx<R>(*)[kB + 1]>(smraw);                                   // kTR x (kB + 1)
  auto Qs = reinterpret_cast<cx<R>(*)[kTC + 1]>(smraw + sizeof(cx<R>) * kTR * (kB + 1));  // kB x (kTC + 1)
  __shared__ double rs[kTR];
  __shared__ double sh[8];
  __shared__ int s_last;
  if (S->done) return;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int k0 = first ? 0 : S->k;
  const int jb = first ? 0 : S->jb;
  const int tile = blockIdx.x, nsl = gridDim.y, sl = blockIdx.y;
  const int r0 = k0 + jb + tile * kTR;
  const int nr = max(0, min(kTR, m - r0));
  const int nch = (p + kTC - 1) / kTC, per = (nch + nsl - 1) / nsl;
  const int c_lo = min(p, sl * per * kTC), c_hi = min(p, c_lo + per * kTC);
  for (int e = tid; e < kTR * kB; e += 256) {
    const int r = e / kB, i = e % kB;
    Cs[r][i] = (r < nr && i < jb) ? Lm[(long long)(r0 + r) * ldl + k0 + i] : czero<R>();
  }
  R nrm[4] = {R(0), R(0), R(0), R(0)};
  if (nr > 0) {
    for (int c0 = c_lo; c0 < c_hi; c0 += kTC) {
      __syncthreads();
      for (int e = tid; e < jb * kTC; e += 256) {
        const int i = e / kTC, c = e % kTC;
        Qs[i][c] = c0 + c < c_hi ? Q[(long long)i * p + c0 + c] : czero<R>();
      }
      cx<R> a[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int r = ty + 16 * u, c = c0 + tx + 16 * v;
          a[u][v] = (r < nr && c < c_hi) ? A[(long long)(r0 + r) * p + c] : czero<R>();
        }
      __syncthreads();
      if (jb > 0) {
        for (int i = 0; i < jb; ++i) {
          cx<R> cu[4], qv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) cu[u] = Cs[ty + 16 * u][i];
#pragma unroll
          for (int v = 0; v < 4; ++v) qv[v] = Qs[i][tx + 16 * v];
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
              a[u][v].re -= cu[u].re * qv[v].re - cu[u].im * qv[v].im;
              a[u][v].im -= cu[u].re * qv[v].im + cu[u].im * qv[v].re;
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const int r = ty + 16 * u, c = c0 + tx + 16 * v;
            if (r < nr && c < c_hi) A[(long long)(r0 + r) * p + c] = a[u][v];
          }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) nrm[u] += abs2(a[u][v]);
    }
  }
  // row partials: the 16 threads of a row (same ty, one half-warp) in a fixed order
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    double v = (double)nrm[u];
    for (int o = 8; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (tx == 0) rs[ty + 16 * u] = v;
  }
  __syncthreads();
  if (nsl > 1) {
    if (tid < nr) npart[(size_t)sl * m + r0 + tid] = rs[tid];
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(tile_ticket + tile, 1u) == (unsigned)nsl - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (tid < kTR) {
      double t = 0;
      if (tid < nr)
        for (int q = 0; q < nsl; ++q) t += __ldcg(npart + (size_t)q * m + r0 + tid);
      rs[tid] = t;
    }
    if (tid == 0) tile_ticket[tile] = 0;
    __syncthreads();
  }
  if (tid < nr) norms[r0 + tid] = rs[tid];
  if (tid == 0) {
    double t = 0;
    for (int r = 0; r < nr; ++r) t += rs[r];
    part[tile] = t;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(&S->ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
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
// Block (x, y): slice x of the columns, quadrant y of the 64 x 64 matrix (32 x 32
// entries, 4 per thread).
template <class R>
__global__ void __launch_bounds__(256) gram_kernel(const cx<R>* __restrict__ A, int p,
                                                   const State* __restrict__ S, cx<R>* __restrict__ gp) {
  constexpr int H = kPool / 2;
  __shared__ cx<R> T[2][H][kGramCols + 1];
  __shared__ int rows[2][H];
  if (S->done) return;
  const int tid = threadIdx.x, np = S->npool;
  const int qi = blockIdx.y >> 1, qj = blockIdx.y & 1;  // quadrant: rows qi * H.., columns qj * H..
  if (tid < 2 * H) {
    const int side = tid / H, r = tid % H, idx = (side ? qj : qi) * H + r;
    rows[side][r] = idx < np ? S->pool[idx] : -1;
  }
  const int ti = tid >> 4, tj = tid & 15;  // entries (ti + 16 u, tj + 16 v), u, v < 2
  cx<R> acc[2][2];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) acc[u][v] = czero<R>();
  const int nst = (p + kGramCols - 1) / kGramCols;  // column stages
  const int per = (nst + gridDim.x - 1) / gridDim.x;
  const int s0 = blockIdx.x * per, s1 = min(nst, s0 + per);
  __syncthreads();
  for (int st = s0; st < s1; ++st) {
    const int c0 = st * kGramCols;
    for (int e = tid; e < 2 * H * kGramCols; e += 256) {
      const int side = e / (H * kGramCols), r = (e / kGramCols) % H, c = e % kGramCols;
      const int row = rows[side][r];
      T[side][r][c] = (row >= 0 && c0 + c < p) ? A[(long long)row * p + c0 + c] : czero<R>();
    }
    __syncthreads();
#pragma unroll 8
    for (int c = 0; c < kGramCols; ++c) {
      const cx<R> a0 = T[0][ti][c], a1 = T[0][ti + 16][c];
      const cx<R> b0 = T[1][tj][c], b1 = T[1][tj + 16][c];
      fmac_(acc[0][0], b0, a0);  // a_i conj(a_j)
      fmac_(acc[0][1], b1, a0);
      fmac_(acc[1][0], b0, a1);
      fmac_(acc[1][1], b1, a1);
    }
    __syncthreads();
  }
  cx<R>* g = gp + (size_t)blockIdx.x * kPool * kPool;
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) g[(qi * H + ti + 16 * u) * kPool + qj * H + tj + 16 * v] = acc[u][v];
}

// Greedy pivoted Cholesky of the pool's Gram matrix (one block of 1024
// threads): the pivot is the pool row of largest residual norm^2 d_i (lowest
// pool index on ties); the block ends at kB pivots, when d_best < kAlpha2 *
// outside, when d_best <= drange * d_first (beyond that the Gram matrix's
// rounding would decide the order), at the rank limit, or at a non-positive d.
// The partial Gram matrices are summed in a fixed order (four entries per
// thread, the loads of eight partials in flight) and the factorisation runs in
// the working precision R: its rounding only perturbs the pivot order among
// nearly equal candidates and the orthonormality of Q_b, which the explicit
// trailing update absorbs (FP64 arithmetic here would cost more than the rest
// of the block on a GPU whose FP64 rate is a small fraction of its FP32 rate).  Writes the accepted
// pivots' Cholesky rows L_bb (be x be, lower), be, and the swap sequence that
// brings the pivots to positions [k, k + be); applies it to perm.
template <class R>
__global__ void __launch_bounds__(1024) pchol_kernel(const cx<R>* __restrict__ gp, int ngp, int kmax,
                                                     State* __restrict__ S, int* __restrict__ perm,
                                                     cx<R>* __restrict__ Lbb, double drange) {
  extern __shared__ unsigned char smraw[];
  constexpr int LG = kPool + 1, LL = kB + 1;    // padded row strides (no bank conflicts down a column)
  cx<R>* G = reinterpret_cast<cx<R>*>(smraw);  // kPool x LG
  cx<R>* Lc = G + kPool * LG;                   // kPool x LL
  __shared__ R d[kPool];
  __shared__ int chosen[kPool], order[kB];
  __shared__ int s_be;
  if (S->done) return;
  const int tid = threadIdx.x;
  const int np = S->npool, k = S->k;
  const double outside = S->outside;
  {
    constexpr int E = kPool * kPool / 1024;  // entries per thread
    cx<R> acc[E];
#pragma unroll
    for (int u = 0; u < E; ++u) acc[u] = czero<R>();
    int b = 0;
    for (; b + 8 <= ngp; b += 8) {
      cx<R> v[8][E];
#pragma unroll
      for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int u = 0; u < E; ++u) v[q][u] = gp[(size_t)(b + q) * kPool * kPool + tid + 1024 * u];
#pragma unroll
      for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int u = 0; u < E; ++u) acc[u] = acc[u] + v[q][u];
    }
    for (; b < ngp; ++b)
#pragma unroll
      for (int u = 0; u < E; ++u) acc[u] = acc[u] + gp[(size_t)b * kPool * kPool + tid + 1024 * u];
#pragma unroll
    for (int u = 0; u < E; ++u) {
      const int e = tid + 1024 * u;
      G[(e / kPool) * LG + e % kPool] = acc[u];
    }
  }
  for (int e = tid; e < kPool * LL; e += 1024) Lc[e] = czero<R>();
  if (tid < kPool) chosen[tid] = tid < np ? 0 : 1;
  __syncthreads();
  if (tid < kPool) d[tid] = tid < np ? G[tid * LG + tid].re : R(0);
  __syncthreads();
  const int jmax = min(kB, min(np, kmax - k));
  // the greedy steps in warp 0 alone (lane i owns candidates i and i + 32): no block barrier
  // per step; the same operations in the same order as a block-wide loop would take
  if (tid < 32) {
    const int lane = tid;
    int j = 0;
    R d0 = R(0);
    for (; j < jmax; ++j) {
      R bv = R(-1);
      int bi = 0x7fffffff;
      for (int i = lane; i < kPool; i += 32)
        if (!chosen[i] && (d[i] > bv || (d[i] == bv && i < bi))) {
          bv = d[i];
          bi = i;
        }
      for (int o = 16; o; o >>= 1) {  // every lane ends with the largest d (lowest index on ties)
        const R ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) {
          bv = ov;
          bi = oi;
        }
      }
      if (j == 0) d0 = bv;
      const bool stop = bi >= kPool || !(bv > R(0)) || (outside > 0 && (double)bv < kAlpha2 * outside) ||
                        (j > 0 && (double)bv <= drange * (double)d0);
      if (stop) break;
      const int best = bi;
      const R sd = sqrt(bv);
      for (int i = lane; i < np; i += 32) {
        cx<R> v = G[i * LG + best];  // <a_i, a_best>
        for (int jj = 0; jj < j; ++jj) {
          const cx<R> a = Lc[i * LL + jj], bc = Lc[best * LL + jj];
          v.re -= a.re * bc.re + a.im * bc.im;  // v -= a conj(bc)
          v.im -= a.im * bc.re - a.re * bc.im;
        }
        v = scale(v, R(1) / sd);
        if (i == best) v = mk<R>(sd, R(0));
        Lc[i * LL + j] = v;
      }
      __syncwarp();
      for (int i = lane; i < np; i += 32) d[i] = chosen[i] || i == best ? R(0) : d[i] - abs2(Lc[i * LL + j]);
      if (lane == 0) {
        chosen[best] = 1;
        order[j] = best;
      }
      __syncwarp();
    }
    if (lane == 0) s_be = j;
  }
  __syncthreads();
  const int be = s_be;
  for (int e = tid; e < kB * kB; e += 1024) {
    const int i = e / kB, jj = e % kB;
    Lbb[e] = (i < be && jj <= i) ? Lc[order[i] * LL + jj] : czero<R>();
  }
  // swap sequence in shared memory: position k + i receives the pivot order[i]
  // (a pivot that sat at k + i', i' < i, was moved to the partner of swap i');
  // the positions it touches, and where each of their final rows comes from
  __shared__ int s_swp[kB], s_upos[2 * kB], s_cur[2 * kB], s_ia[kB], s_ix[kB], s_val[2 * kB], s_nu;
  __shared__ int s_pool[kPool];
  if (tid < kPool) s_pool[tid] = S->pool[tid];
  __syncthreads();
  if (tid < 32) {  // warp 0; every lane follows the same (uniform) control flow
    const int lane = tid;
    int nu = be;
    if (lane < be) s_upos[lane] = k + lane;  // be <= kB = 32
    __syncwarp();
    for (int i = 0; i < be; ++i) {
      // follow the earlier swaps: position k + t (t < i) now holds the row that sat at swp[t],
      // and only later swaps can move it again
      int x = s_pool[order[i]];
      for (int lo = 0;;) {
        const int t = x - k;
        if (t < lo || t >= i) break;
        x = s_swp[t];
        lo = t + 1;
      }
      int ix = -1;  // x among the touched positions (a warp-wide search)
      for (int base = 0; base < nu && ix < 0; base += 32) {
        const int t = base + lane;
        const unsigned hit = __ballot_sync(0xffffffffu, t < nu && s_upos[t] == x);
        if (hit) ix = base + __ffs(hit) - 1;
      }
      __syncwarp();
      if (lane == 0) {
        s_swp[i] = x;
        if (ix < 0) s_upos[nu] = x;
        s_ia[i] = i;  // position k + i is upos[i]
        s_ix[i] = ix < 0 ? nu : ix;
      }
      if (ix < 0) ++nu;
      __syncwarp();
    }
    if (lane == 0) {
      for (int t = 0; t < nu; ++t) s_cur[t] = t;
      for (int i = 0; i < be; ++i) {
        const int a = s_ia[i], b = s_ix[i];
        const int tmp = s_cur[a];
        s_cur[a] = s_cur[b];
        s_cur[b] = tmp;
      }
      s_nu = nu;
      S->be = be;
      S->nu = nu;
      if (be == 0) S->done = 1;  // no admissible pivot left (the Gram matrix is numerically zero)
    }
  }
  __syncthreads();
  const int nu = s_nu;
  if (tid < nu) {
    S->upos[tid] = s_upos[tid];
    S->usrc[tid] = s_cur[tid];
    s_val[tid] = perm[s_upos[tid]];
  }
  __syncthreads();
  if (tid < nu) perm[s_upos[tid]] = s_val[s_cur[tid]];
}

// The block's row permutation and Q_b = L_bb^-1 A(J_b): blocks [0, nqa) take
// 128 columns of A each -- the rows at the touched positions are staged in
// shared memory and written back permuted (position upos[t] receives the row
// from upos[usrc[t]]), then one thread per column forward-substitutes the
// pivot rows (now at k .. k + be - 1).  Blocks [nqa, ...) do the same
// permutation in columns [0, k) of L, 128 columns each, and the first of them
// writes the block's diagonal L_bb.
template <class R>
__global__ void __launch_bounds__(256) swapq_kernel(cx<R>* __restrict__ A, int p, cx<R>* __restrict__ Lm, int ldl,
                                                    const cx<R>* __restrict__ Lbb, cx<R>* __restrict__ Q,
                                                    cx<R>* __restrict__ Qc, const State* __restrict__ S, int nqa) {
  constexpr int CW = 128;
  extern __shared__ unsigned char smraw[];
  cx<R>* stage = reinterpret_cast<cx<R>*>(smraw);  // 2 kB x CW
  __shared__ int upos[2 * kB], usrc[2 * kB];
  __shared__ cx<R> Lb[kB][kB + 1];
  if (S->done) return;
  const int tid = threadIdx.x, k = S->k, be = S->be, nu = S->nu;
  if (tid < nu) {
    upos[tid] = S->upos[tid];
    usrc[tid] = S->usrc[tid];
  }
  for (int e = tid; e < kB * kB; e += 256) Lb[e / kB][e % kB] = Lbb[e];
  __syncthreads();
  if ((int)blockIdx.x < nqa) {
    const int c0 = blockIdx.x * CW;
    for (int e = tid; e < nu * CW; e += 256) {
      const int t = e / CW, c = e % CW;
      if (c0 + c < p) stage[t * CW + c] = A[(long long)upos[t] * p + c0 + c];
    }
    __syncthreads();
    for (int e = tid; e < nu * CW; e += 256) {
      const int t = e / CW, c = e % CW;
      if (c0 + c < p) A[(long long)upos[t] * p + c0 + c] = stage[usrc[t] * CW + c];
    }
    if (tid >= CW) return;
    const int c = c0 + tid;
    if (c >= p) return;
    cx<R> q[kB];
#pragma unroll
    for (int i = 0; i < kB; ++i) {
      if (i < be) {
        cx<R> x = stage[usrc[i] * CW + tid];  // the row now at position k + i (upos[i] = k + i)
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
    const int c0 = (blockIdx.x - nqa) * CW;
    for (int e = tid; e < nu * CW; e += 256) {
      const int t = e / CW, c = e % CW;
      if (c0 + c < k) stage[t * CW + c] = Lm[(long long)upos[t] * ldl + c0 + c];
    }
    __syncthreads();
    for (int e = tid; e < nu * CW; e += 256) {
      const int t = e / CW, c = e % CW;
      if (c0 + c < k) Lm[(long long)upos[t] * ldl + c0 + c] = stage[usrc[t] * CW + c];
    }
    if (blockIdx.x == nqa)  // the block's diagonal L_bb in columns [k, k + be)
      for (int e = tid; e < be * be; e += 256) {
        const int i = e / be, jj = e % be;
        Lm[(long long)(k + i) * ldl + k + jj] = jj <= i ? Lb[i][jj] : czero<R>();
      }
  }
}

// C = A_trail(rows, :) Q_b^H for the trailing rows after the block's pivots
// (positions [k + be, m)), written to L(rows, k .. k + be).  Block (x, y):
// row tile x (kCR rows), slice y of the p columns (split K; gridDim.y slices,
// multiples of 16 columns), kCR x kB outputs per block, 8 per thread.  With
// more than one slice the partial products go to Cp and the last block of a
// tile to finish adds them in slice order; the tile's finishing block writes
// L and the column sums of |C|^2 of its rows.  The last tile to finish adds
// the pivot rows' part (the columns of L_bb) and finds the first j at which the
// residual ||A_trail||^2 - sum_{i <= j} ||C(:, i)||^2 is within the tolerance.
template <class R>
__global__ void __launch_bounds__(256) proj_kernel(const cx<R>* __restrict__ A, int m, int p,
                                                   cx<R>* __restrict__ Lm, int ldl, const cx<R>* __restrict__ Qc,
                                                   const cx<R>* __restrict__ Lbb, cx<R>* __restrict__ Cp,
                                                   unsigned* __restrict__ tile_ticket, double* __restrict__ cpart,
                                                   State* __restrict__ S) {
  constexpr int KC = 16;
  __shared__ cx<R> As[KC][kCR + 1];
  __shared__ cx<R> Bs[KC][kB + 1];
  __shared__ double cs[32][kB + 1];
  __shared__ int s_last;
  if (S->done) return;
  const int tid = threadIdx.x, k = S->k, be = S->be;
  const int tile = blockIdx.x, nsl = gridDim.y, sl = blockIdx.y;
  const int r0 = k + be + tile * kCR;
  const int nr = max(0, min(kCR, m - r0));
  const int kc = ((p + nsl - 1) / nsl + KC - 1) / KC * KC;
  const int t_lo = min(p, sl * kc), t_hi = min(p, t_lo + kc);
  const int tx = tid & 7, ty = tid >> 3;  // rows ty, ty + 32; columns tx + 8 v
  cx<R> acc[2][4];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = czero<R>();
  if (nr > 0) {
    for (int t0 = t_lo; t0 < t_hi; t0 += KC) {
#pragma unroll
      for (int r = 0; r < (KC * kCR) / 256; ++r) {
        const int e = tid + 256 * r, kk = e % KC, i = e / KC;
        As[kk][i] = (i < nr && t0 + kk < t_hi) ? A[(long long)(r0 + i) * p + t0 + kk] : czero<R>();
      }
#pragma unroll
      for (int r = 0; r < (KC * kB) / 256; ++r) {
        const int e = tid + 256 * r, kk = e % KC, j = e / KC;
        Bs[kk][j] = (j < be && t0 + kk < t_hi) ? Qc[(long long)j * p + t0 + kk] : czero<R>();
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
  if (nsl > 1) {
    // partial products of this slice; the tile's last block adds them in slice order
    cx<R>* cp = Cp + ((size_t)sl * gridDim.x + tile) * kCR * kB;
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) cp[(ty + 32 * u) * kB + tx + 8 * v] = acc[u][v];
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(tile_ticket + tile, 1u) == (unsigned)nsl - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        cx<R> a = czero<R>();
        for (int q = 0; q < nsl; ++q)
          a = a + __ldcg_cx_any(Cp + ((size_t)q * gridDim.x + tile) * kCR * kB + (ty + 32 * u) * kB + tx + 8 * v);
        acc[u][v] = a;
      }
    if (tid == 0) tile_ticket[tile] = 0;
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
    cpart[(size_t)tile * kB + tid] = t;
  }
  // the last tile: the stopping test
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(&S->ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
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

// The interpolation matrix by blocked back substitution on L: the rows of the
// candidates that are not pivots, T = L(J^c, :) L(J, :)^-1 (L(J, :) lower
// triangular), in place in rows [k, m) of L, 64 columns at a time from the
// right.  trsm_diag_kernel solves the diagonal block: 128 rows per block, one
// thread per row, the block of L and the rows' segments in shared memory (row
// stride 65); the GEMM update of the columns on the left follows on the host.
constexpr int kTN = 64;
template <class R>
__global__ void __launch_bounds__(128) trsm_diag_kernel(cx<R>* __restrict__ Lm, int ldl, int m, int k, int j0,
                                                        int w) {
  extern __shared__ unsigned char smraw[];
  cx<R>* Ld = reinterpret_cast<cx<R>*>(smraw);  // kTN x (kTN + 1)
  cx<R>* Bt = Ld + kTN * (kTN + 1);              // 128 x (kTN + 1)
  const int tid = threadIdx.x, r0 = k + blockIdx.x * 128;
  const int nr = min(128, m - r0);
  for (int e = tid; e < w * w; e += 128) {
    const int i = e / w, c = e % w;
    Ld[i * (kTN + 1) + c] = c <= i ? Lm[(long long)(j0 + i) * ldl + j0 + c] : czero<R>();
  }
  for (int e = tid; e < nr * w; e += 128) {
    const int rr = e / w, c = e % w;
    Bt[rr * (kTN + 1) + c] = Lm[(long long)(r0 + rr) * ldl + j0 + c];
  }
  __syncthreads();
  if (tid < nr) {
    cx<R>* b = Bt + tid * (kTN + 1);
    for (int j = w - 1; j >= 0; --j) {
      cx<R> x = b[j];
      for (int i = j + 1; i < w; ++i) {
        const cx<R> t = b[i], l = Ld[i * (kTN + 1) + j];
        x.re -= t.re * l.re - t.im * l.im;
        x.im -= t.re * l.im + t.im * l.re;
      }
      b[j] = x * inv(Ld[j * (kTN + 1) + j]);
    }
  }
  __syncthreads();
  for (int e = tid; e < nr * w; e += 128) {
    const int rr = e / w, c = e % w;
    Lm[(long long)(r0 + rr) * ldl + j0 + c] = Bt[rr * (kTN + 1) + c];
  }
}

// U (m x k, row-major, candidate order): the pivot at position q < k has the
// unit row e_q; the candidate at position q >= k has row T(q - k, :).
template <class R>
__global__ void scatter_u_kernel(const cx<R>* __restrict__ Lm, int ldl, const int* __restrict__ perm, int m, int k,
                                 cx<R>* __restrict__ U) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)m * k) return;
  const int q = (int)(t / k), a = (int)(t % k);
  const int c = perm[q];
  U[(long long)c * k + a] = q < k ? mk<R>(a == q ? R(1) : R(0), R(0)) : Lm[(long long)q * ldl + a];
}

__global__ void iota_kernel(int* v, int m) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < m) v[t] = t;
}

}  // namespace bid

// Blocked row ID of the candidate-major matrix A (m x p, overwritten by the
// trailing residual): returns k and the pivots (host); with U non-null writes U
// (m x k, row-major, device) on su (after the factorisation on st), or on st.
template <class R>
int blocked_row_id(cx<R>* A, int m, int p, double eps, cudaStream_t st, cudaStream_t su, cx<R>* U, int* k_out,
                   std::vector<int>* hp) {
  using namespace bid;
  int dev = 0, nsm = 148;
  LS_CUDA_TRY(cudaGetDevice(&dev));
  LS_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int kmax = std::min(m, p);
  const int ldl = std::max(kmax, 1);
  const int nU = (m + kTR - 1) / kTR, nC = (m + kCR - 1) / kCR;
  const int nst = (p + kGramCols - 1) / kGramCols;
  const int ngp = std::max(1, std::min(kGramMax, nst));
  const int nqa = (p + 127) / 128, nql = (kmax + 127) / 128;
  size_t off = 0;
  auto carve = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  const size_t oL = carve(sizeof(cx<R>) * (size_t)m * ldl), oQ = carve(sizeof(cx<R>) * (size_t)kB * p),
               oQc = carve(sizeof(cx<R>) * (size_t)kB * p), oLbb = carve(sizeof(cx<R>) * kB * kB),
               oN = carve(sizeof(double) * m), oPerm = carve(sizeof(int) * m),
               oS = carve(sizeof(State)), oUp = carve(sizeof(double) * nU), oCp = carve(sizeof(double) * nC * kB),
               oG = carve(sizeof(cx<R>) * (size_t)ngp * kPool * kPool),
               oCs = carve(sizeof(cx<R>) * (size_t)kMaxSplit * nC * kCR * kB), oTk = carve(sizeof(unsigned) * nC),
               oNp = carve(sizeof(double) * (size_t)kMaxSplit * m), oTu = carve(sizeof(unsigned) * nU);
  char* w = nullptr;
  int rc = dalloc((void**)&w, off);
  if (rc) return rc;
  cx<R>* Lm = reinterpret_cast<cx<R>*>(w + oL);
  cx<R>* Q = reinterpret_cast<cx<R>*>(w + oQ);
  cx<R>* Qc = reinterpret_cast<cx<R>*>(w + oQc);
  cx<R>* Lbb = reinterpret_cast<cx<R>*>(w + oLbb);
  double* norms = reinterpret_cast<double*>(w + oN);
  int* perm = reinterpret_cast<int*>(w + oPerm);
  State* S = reinterpret_cast<State*>(w + oS);
  double* upart = reinterpret_cast<double*>(w + oUp);
  double* cpart = reinterpret_cast<double*>(w + oCp);
  cx<R>* gp = reinterpret_cast<cx<R>*>(w + oG);
  cx<R>* Cs = reinterpret_cast<cx<R>*>(w + oCs);
  unsigned* tickets = reinterpret_cast<unsigned*>(w + oTk);
  double* npart = reinterpret_cast<double*>(w + oNp);
  unsigned* uticket = reinterpret_cast<unsigned*>(w + oTu);
  // column slices of the update: about two blocks per SM, at least four 64-column chunks each
  const size_t upd_smem = sizeof(cx<R>) * ((size_t)kTR * (kB + 1) + (size_t)kB * (kTC + 1));
  if (cudaFuncSetAttribute(update_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)upd_smem) !=
      cudaSuccess) {
    dfree(w);
    LS_CUDA_TRY(cudaGetLastError());
  }
  const size_t swap_smem = sizeof(cx<R>) * 2 * kB * 128;
  if (cudaFuncSetAttribute(swapq_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)swap_smem) !=
      cudaSuccess) {
    dfree(w);
    LS_CUDA_TRY(cudaGetLastError());
  }
  auto usplit = [&](int tiles) {
    return std::max(1, std::min({kMaxSplit, (2 * nsm + tiles - 1) / tiles, (p + 4 * kTC - 1) / (4 * kTC)}));
  };
  const size_t chol_smem = sizeof(cx<R>) * (size_t)kPool * (kPool + 1 + kB + 1);
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
  if (cudaMemsetAsync(S, 0, sizeof(State), st) != cudaSuccess ||
      cudaMemsetAsync(tickets, 0, sizeof(unsigned) * nC, st) != cudaSuccess ||
      cudaMemsetAsync(uticket, 0, sizeof(unsigned) * nU, st) != cudaSuccess)
    return fail(check_launch("blocked ID state"));
  count_launch();
  iota_kernel<<<(m + 255) / 256, 256, 0, st>>>(perm, m);
  count_launch();
  update_kernel<R><<<dim3(nU, usplit(nU)), 256, upd_smem, st>>>(A, m, p, kmax, Lm, ldl, Q, norms, npart, uticket, upart, S,
                                                         eps * eps, 1);
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
    gram_kernel<R><<<dim3(ngp, 4), 256, 0, st>>>(A, p, S, gp);
    pchol_kernel<R><<<1, 1024, chol_smem, st>>>(gp, ngp, kmax, S, perm, Lbb, drange);
    swapq_kernel<R><<<nqa + nql, 256, swap_smem, st>>>(A, p, Lm, ldl, Lbb, Q, Qc, S, nqa);
    {
      // split K so that the projection fills about two blocks per SM (slices of at least 512 columns)
      const int tiles = std::max(1, (rows + kCR - 1) / kCR);
      const int nsl = std::max(1, std::min({kMaxSplit, (2 * nsm + tiles - 1) / tiles, (p + 511) / 512}));
      proj_kernel<R><<<dim3(tiles, nsl), 256, 0, st>>>(A, m, p, Lm, ldl, Qc, Lbb, Cs, tickets, cpart, S);
    }
    {
      const int tiles = std::max(1, (rows + kTR - 1) / kTR);
      update_kernel<R><<<dim3(tiles, usplit(tiles)), 256, upd_smem, st>>>(A, m, p, kmax, Lm, ldl, Q, norms, npart, uticket,
                                                                   upart, S, 0.0, 0);
    }
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
  int* pv = static_cast<int*>(pinned_scratch(sizeof(int) * (size_t)std::max(k, 1)));
  if (!pv) return fail(LS_ENOMEM);
  if (k > 0) LS_CUDA_TRY(cudaMemcpyAsync(pv, perm, sizeof(int) * k, cudaMemcpyDeviceToHost, st));
  LS_CUDA_TRY(cudaStreamSynchronize(st));
  hp->assign(std::max(k, 1), 0);
  for (int a = 0; a < k; ++a) (*hp)[a] = pv[a];
  *k_out = k;
  if (!U || k == 0) {
    dfree(w);
    return LS_OK;
  }
  // T and U on su (beside the next ID) when given; the workspace is released there
  cudaStream_t sb = st;
  if (su) {
    cudaEvent_t e;
    LS_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    LS_CUDA_TRY(cudaEventRecord(e, st));
    LS_CUDA_TRY(cudaStreamWaitEvent(su, e, 0));
    cudaEventDestroy(e);
    sb = su;
  }
  StreamScope scope(sb);
  if (m > k) {
    const size_t dsm = sizeof(cx<R>) * (size_t)(kTN + 128) * (kTN + 1);
    LS_CUDA_TRY(cudaFuncSetAttribute(trsm_diag_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm));
    const cx<R> mone = mk<R>(R(-1), R(0)), one = mk<R>(R(1), R(0));
    cx<R>* T = Lm + (size_t)k * ldl;
    for (int j0 = ((k - 1) / kTN) * kTN; j0 >= 0; j0 -= kTN) {
      const int wd = std::min(kTN, k - j0);
      count_launch();
      trsm_diag_kernel<R><<<(m - k + 127) / 128, 128, dsm, sb>>>(Lm, ldl, m, k, j0, wd);
      if (j0 > 0) {  // T(:, 0:j0) -= T(:, j0:j0+w) L(j0:j0+w, 0:j0)
        if constexpr (sizeof(R) == 4)
          rc = simt_cgemm(sb, false, false, m - k, j0, wd, mone, T + j0, ldl, 0, Lm + (size_t)j0 * ldl, ldl, 0, one, T,
                          ldl, 0, 1);
        else
          rc = simt_zgemm(sb, false, false, m - k, j0, wd, mone, T + j0, ldl, 0, Lm + (size_t)j0 * ldl, ldl, 0, one, T,
                          ldl, 0, 1);
        if (rc) return rc;
      }
    }
  }
  count_launch();
  scatter_u_kernel<R><<<(unsigned)(((long long)m * k + 255) / 256), 256, 0, sb>>>(Lm, ldl, perm, m, k, U);
  if ((rc = check_launch("blocked ID interpolation matrix"))) return rc;
  dfree(w);
  return LS_OK;
}

template int blocked_row_id<float>(c32*, int, int, double, cudaStream_t, cudaStream_t, c32*, int*,
                                   std::vector<int>*);
template int blocked_row_id<double>(z64*, int, int, double, cudaStream_t, cudaStream_t, z64*, int*,
                                    std::vector<int>*);

}  // namespace ls
