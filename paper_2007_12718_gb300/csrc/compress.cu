// HBS compression of G (Sec. 3.2): one row ID per tree level.
//
// For each level l = L..1 the rows are the points of one box (leaves) or the
// two children's skeletons (Eq. 14), the columns the proxy ring of lattice
// points at Chebyshev distance 1..w outside the box (Eq. 13).  The proxy
// block is the same for every box of a level (translation invariance), so one
// ID per level serves all 2^l boxes.  The ID is a column-pivoted QR of the
// transposed block (Sec. 2.1): candidates are the rows, pivoting picks the
// skeleton, U = P^T [I; (R11^-1 R12)^T] (U(skel,:) = I).  The rank is the
// first k whose remaining residual has Frobenius norm <= eps ||block||_F
// (the local tolerance rule, remark in Sec. 3.2).
//
// The CPQR runs as one cooperative kernel across many SMs: each block owns a
// slice of candidate columns, one bounded grid barrier per pivot step; the
// pivot column is read by every block straight from L2 (no broadcast copy).
// Sibling blocks G_ab = G(skel_a, skel_b) (Eq. 15) and the leaf block
// G(I_tau, I_tau) are evaluated on the device at the end.
#include <cooperative_groups.h>
#include <string.h>

#include <algorithm>

#include "handle.h"
#include "prof.h"

namespace ls {
namespace {

template <class R>
__global__ void block_kernel(const int* __restrict__ rx, const int* __restrict__ ry, int m,
                             const int* __restrict__ px, const int* __restrict__ py, int p, cx<R>* __restrict__ out,
                             long long ld, KernelTable kt, KernelSpec ks) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)m * p) return;
  int c = (int)(t / p), q = (int)(t % p);
  z64 v = table_entry(kt, ks, px[q] - rx[c], py[q] - ry[c]);
  out[(long long)c * ld + q] = cvt<R>(v);
}

template <class R>
struct IdSlot {
  R best;   // largest residual norm^2 among the block's active candidates
  R total;  // sum of residual norm^2 over the block's active candidates
  int idx;  // candidate index of best (lowest index on ties), -1 if none
  int pad;
};

// Warp-level helpers of one projection a -= q (q^H a) / |q|^2 (two independent
// accumulators per lane for instruction-level parallelism).
template <class R>
__device__ __forceinline__ cx<R> project_coeff(const cx<R>* q, const cx<R>* a, int p, int lane, R inu2) {
  cx<R> d0 = mk<R>(0, 0), d1 = mk<R>(0, 0);
  int i = lane;
  for (; i + 32 < p; i += 64) {
    fmac_(d0, q[i], a[i]);
    fmac_(d1, q[i + 32], a[i + 32]);
  }
  if (i < p) fmac_(d0, q[i], a[i]);
  return scale(warp_sum(d0 + d1), inu2);
}

template <class R>
__device__ __forceinline__ R project_update(const cx<R>* q, cx<R>* a, int p, int lane, cx<R> d) {
  R n0 = 0, n1 = 0;
  int i = lane;
  for (; i + 32 < p; i += 64) {
    cx<R> v0 = a[i], q0 = q[i], v1 = a[i + 32], q1 = q[i + 32];
    v0.re -= q0.re * d.re - q0.im * d.im;
    v0.im -= q0.re * d.im + q0.im * d.re;
    v1.re -= q1.re * d.re - q1.im * d.im;
    v1.im -= q1.re * d.im + q1.im * d.re;
    a[i] = v0;
    a[i + 32] = v1;
    n0 += abs2(v0);
    n1 += abs2(v1);
  }
  if (i < p) {
    cx<R> v = a[i], q0 = q[i];
    v.re -= q0.re * d.re - q0.im * d.im;
    v.im -= q0.re * d.im + q0.im * d.re;
    a[i] = v;
    n0 += abs2(v);
  }
  return warp_sum_r(n0 + n1);
}

// 64-bit pivot key: the residual norm's leading bits (all 32 of a float, the
// top 44 of a double; non-negative, so integer order is numeric order) above
// 20 bits of (2^20 - 1 - index).  The integer maximum of the keys is the
// largest norm, lowest index on ties; key 0 means "no candidate".
__device__ __forceinline__ unsigned long long piv_key(float nrm, int idx) {
  return ((unsigned long long)__float_as_uint(nrm) << 20) | (unsigned long long)(0xFFFFF - idx);
}
__device__ __forceinline__ unsigned long long piv_key(double nrm, int idx) {
  return (((unsigned long long)__double_as_longlong(nrm) >> 20) << 20) | (unsigned long long)(0xFFFFF - idx);
}
__device__ __forceinline__ int piv_key_index(unsigned long long key) { return 0xFFFFF - (int)(key & 0xFFFFF); }
// Warp-wide maximum of 64-bit keys: redux.sync on the high words, then on the
// low words of the lanes that hold the maximal high word.
__device__ __forceinline__ unsigned long long warp_max_key(unsigned long long key) {
  const unsigned hi = (unsigned)(key >> 32);
  const unsigned mhi = __reduce_max_sync(0xffffffffu, hi);
  const unsigned lo = hi == mhi ? (unsigned)key : 0u;
  const unsigned mlo = __reduce_max_sync(0xffffffffu, lo);
  return ((unsigned long long)mhi << 32) | mlo;
}
// The residual norm a float key carries (exact).
__device__ __forceinline__ float piv_key_norm(unsigned long long key) { return __uint_as_float((unsigned)(key >> 20)); }

// Column-pivoted QR ID of the candidate-major matrix A (m candidates, each a
// length-p vector at A + c*p).  Block b owns candidates [c0, c0 + mc) and keeps
// their residual vectors in shared memory when they fit (else in the global
// working copy Aw).  Per pivot step: every block publishes its best local
// candidate (norm and block total in a parity slot, vector in a parity vector
// slot) and folds its key into the step's global key (atomic max); one bounded
// grid barrier; every block reads the step's key, the winner's slot and vector
// and the block totals (fixed order: every block takes the same stopping
// decision), and projects the winner out of its own candidates (one warp per
// candidate: a_c -= q (q^H a_c) / |q|^2, then the exact new norm, folded into
// the block's next key with a shared-memory atomic max).  gkey[0..kmax] must
// be zero at launch; m < 2^20.
// Outputs: piv[0..k), rank[0] = k, U (m x k, row-major, stride k).
template <class R>
__global__ void __launch_bounds__(256) cpqr_id_kernel(const cx<R>* __restrict__ A, int m, int p, int kmax,
                                                      double eps, int use_smem, cx<R>* __restrict__ Aw,
                                                      cx<R>* __restrict__ Rm, int* __restrict__ sel,
                                                      IdSlot<R>* __restrict__ slots, cx<R>* __restrict__ pslots,
                                                      unsigned long long* __restrict__ gkey, int* __restrict__ piv,
                                                      int* __restrict__ rank, cx<R>* __restrict__ U,
                                                      cx<R>* __restrict__ RT, GridSync gs, int* __restrict__ err) {
  extern __shared__ unsigned char smraw[];
  cx<R>* pvec = reinterpret_cast<cx<R>*>(smraw);  // p
  const int nblk = gridDim.x, blk = blockIdx.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarp = blockDim.x >> 5;
  const int per = (m + nblk - 1) / nblk;
  const int c0 = min(m, blk * per), c1 = min(m, c0 + per), mc = c1 - c0;
  cx<R>* cand = use_smem ? pvec + p : Aw + (long long)c0 * p;
  __shared__ unsigned long long s_key[2];
  __shared__ R s_nrm[64];
  __shared__ int s_sel[64];
  __shared__ R s_best, s_tol2;
  __shared__ int s_stop;
  unsigned int epoch = 0;

  if (tid < 2) s_key[tid] = 0ULL;
  for (long long t = tid; t < (long long)mc * p; t += blockDim.x) cand[t] = A[(long long)c0 * p + t];
  __syncthreads();
  for (int c = warp; c < mc; c += nwarp) {
    R acc = 0;
    for (int i = lane; i < p; i += 32) acc += abs2(cand[(long long)c * p + i]);
    acc = warp_sum_r(acc);
    if (lane == 0) {
      s_nrm[c] = acc;
      s_sel[c] = -1;
      sel[c0 + c] = -1;
      atomicMax(&s_key[0], piv_key(acc, c0 + c));
    }
  }
  __syncthreads();

  int k = 0;
  for (int j = 0;; ++j) {
    const int par = j & 1;
    const unsigned long long kb = s_key[par];
    const int lb = kb ? piv_key_index(kb) - c0 : -1;  // this block's best candidate (local index)
    if (warp == 0) {
      R total = R(0);
      for (int c = lane; c < mc; c += 32)
        if (s_sel[c] == -1) total += s_nrm[c];
      total = warp_sum_r(total);
      if (lane == 0) {
        IdSlot<R> sl;
        sl.best = lb >= 0 ? s_nrm[lb] : R(0);
        sl.total = total;
        sl.idx = lb >= 0 ? c0 + lb : -1;
        sl.pad = 0;
        slots[par * nblk + blk] = sl;
        if (kb) atomicMax(&gkey[j], kb);
      }
    }
    if (lb >= 0) {
      cx<R>* dst = pslots + ((long long)par * nblk + blk) * p;
      const cx<R>* src = cand + (long long)lb * p;
      for (int i = tid; i < p; i += blockDim.x) dst[i] = src[i];
    }
    if (!grid_sync(gs, nblk, epoch)) return;
    const unsigned long long key = __ldcg(&gkey[j]);
    int idx = key ? piv_key_index(key) : -1;
    const int bw = idx >= 0 ? idx / per : 0;
    if (idx >= m || (idx >= 0 && (bw >= nblk || idx - bw * per >= 64))) {  // cannot happen; uniform over the grid
      if (tid == 0) atomicExch(err, 1);
      idx = -1;
    }
    if (warp == 0) {
      R total = R(0);
      for (int b = lane; b < nblk; b += 32) total += __ldcg(&slots[par * nblk + b].total);
      total = warp_sum_r(total);
      if (lane == 0) {
        if (j == 0) s_tol2 = (R)(eps * eps) * total;
        const R best = idx >= 0 ? __ldcg(&slots[par * nblk + bw].best) : R(0);
        s_best = best;
        s_stop = (j == kmax) || idx < 0 || !(best > R(0)) || total <= s_tol2;
        s_key[par] = 0ULL;  // published; reused for step j + 2
      }
    }
    if (idx >= 0) {
      const cx<R>* src = pslots + ((long long)par * nblk + bw) * p;
      for (int i = tid; i < p; i += blockDim.x) pvec[i] = ldcg_cx(src + i);
    }
    __syncthreads();
    if (s_stop) {
      k = j;
      break;
    }
    const R best = s_best;
    const R nu = sqrt(best);
    const R inu2 = R(1) / best;
    if (blk == bw && tid == 0) {
      s_sel[idx - c0] = j;
      sel[idx] = j;
      piv[j] = idx;
      Rm[(long long)j * m + idx] = mk<R>(nu, R(0));
    }
    for (int c = warp; c < mc; c += nwarp) {
      if (c0 + c == idx || s_sel[c] != -1) continue;
      cx<R>* a = cand + (long long)c * p;
      cx<R> d = project_coeff(pvec, a, p, lane, inu2);  // coefficient of the pivot vector
      R nr = project_update(pvec, a, p, lane, d);
      if (lane == 0) {
        s_nrm[c] = nr;
        Rm[(long long)j * m + c0 + c] = scale(d, nu);  // R(j, c) = q^H a = (a_pv^H a) / nu
        atomicMax(&s_key[par ^ 1], piv_key(nr, c0 + c));
      }
    }
    __syncthreads();
  }
  if (blk == 0 && tid == 0) rank[0] = k;
  if (!grid_sync(gs, nblk, epoch)) return;  // piv and Rm complete
  // R11 gathered by columns: RT[a][b] = R(b, piv[a]) for b <= a (rows of RT contiguous)
  for (long long t = (long long)blk * blockDim.x + tid; t < (long long)k * k; t += (long long)nblk * blockDim.x) {
    int a = (int)(t / k), bb = (int)(t % k);
    RT[t] = bb <= a ? ldcg_cx(Rm + (long long)bb * m + __ldcg(piv + a)) : mk<R>(0, 0);
  }
  if (!grid_sync(gs, nblk, epoch)) return;
  // U rows: identity on the skeleton, T = R11^-1 R12 on the rest: one warp per
  // candidate, column-oriented back substitution in shared memory (the
  // candidate vectors' space is reused).
  cx<R>* t = pvec + (long long)warp * kmax;
  for (int c = c0 + warp; c < c1; c += nwarp) {
    int sc = s_sel[c - c0];
    if (sc >= 0) {
      for (int a = lane; a < k; a += 32) U[(long long)c * k + a] = mk<R>(a == sc ? R(1) : R(0), R(0));
      continue;
    }
    for (int a = lane; a < k; a += 32) t[a] = ldcg_cx(Rm + (long long)a * m + c);
    __syncwarp();
    for (int a = k - 1; a >= 0; --a) {
      const cx<R>* col = RT + (long long)a * k;
      const cx<R> ta = t[a] * inv(ldcg_cx(col + a));
      __syncwarp();
      for (int bb = lane; bb < a; bb += 32) {
        cx<R> v = t[bb], r = ldcg_cx(col + bb);
        v.re -= r.re * ta.re - r.im * ta.im;
        v.im -= r.re * ta.im + r.im * ta.re;
        t[bb] = v;
      }
      if (lane == 0) t[a] = ta;
      __syncwarp();
    }
    for (int a = lane; a < k; a += 32) U[(long long)c * k + a] = t[a];
    __syncwarp();
  }
}

// The same ID on one thread-block cluster (CL <= 16 blocks of 1024 threads,
// candidates resident in shared memory, normally one candidate per warp).
// Per pivot step the critical path is: each warp projects its candidate and
// folds the new norm's key into the block's key with a shared-memory atomic
// max; one block barrier; lanes r < CL of warp 0 store the block's key and its
// best norm, and lanes of warp 1 the block's residual total, into slot
// [this block] of block r (distributed shared memory stores); one cluster
// barrier; every block then finds the winner, its norm and the cluster total
// in its own shared memory (fixed summation order, so every block takes the
// same stopping decision) and copies the winning vector from the owner; one
// block barrier.  Same outputs as cpqr_id_kernel.  Needs m < 2^20.
template <class R>
__global__ void __launch_bounds__(1024) cpqr_id_cluster_kernel(const cx<R>* __restrict__ A, int m, int p, int kmax,
                                                               double eps, cx<R>* __restrict__ Rm,
                                                               int* __restrict__ sel, int* __restrict__ piv,
                                                               int* __restrict__ rank, cx<R>* __restrict__ U,
                                                               cx<R>* __restrict__ RT, int* __restrict__ err) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ unsigned char smraw[];
  cx<R>* pvec = reinterpret_cast<cx<R>*>(smraw);  // p
  cx<R>* cand = pvec + p;                          // per x p
  const int CL = (int)cluster.num_blocks(), crank = (int)cluster.block_rank();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarp = blockDim.x >> 5;
  const int per = (m + CL - 1) / CL;
  const int c0 = min(m, crank * per), c1 = min(m, c0 + per), mc = c1 - c0;
  __shared__ unsigned long long s_key[2];     // this block's best key, by step parity
  __shared__ unsigned long long s_ck[2][16];  // every block's best key, by step parity and block
  __shared__ R s_cb[2][16];                   // every block's best norm
  __shared__ R s_ct[2][16];                   // every block's residual total
  __shared__ R s_best;                        // winner's residual norm^2
  __shared__ int s_stop;
  __shared__ R s_nrm[64];
  __shared__ int s_sel[64];

  if (tid < 2) s_key[tid] = 0ULL;
  for (long long t = tid; t < (long long)mc * p; t += blockDim.x) cand[t] = A[(long long)c0 * p + t];
  __syncthreads();
  for (int c = warp; c < mc; c += nwarp) {
    R acc = 0;
    for (int i = lane; i < p; i += 32) acc += abs2(cand[(long long)c * p + i]);
    acc = warp_sum_r(acc);
    if (lane == 0) {
      s_nrm[c] = acc;
      s_sel[c] = -1;
      sel[c0 + c] = -1;
      atomicMax(&s_key[0], piv_key(acc, c0 + c));
    }
  }
  __syncthreads();
  R tol2 = 0;
  int k = 0;
  for (int j = 0;; ++j) {
    const int par = j & 1;
    // this block's key, best norm and total for step j, stored into every block
    if (warp == 0) {
      const unsigned long long kb = s_key[par];
      const int lb = kb ? piv_key_index(kb) - c0 : -1;
      const R nb = (lb >= 0 && lb < mc) ? s_nrm[lb] : R(0);
      if (lane < CL) {
        *cluster.map_shared_rank(&s_ck[par][crank], lane) = kb;
        *cluster.map_shared_rank(&s_cb[par][crank], lane) = nb;
      }
    } else if (warp == 1) {
      R tot = 0;
      for (int c = lane; c < mc; c += 32)
        if (s_sel[c] == -1) tot += s_nrm[c];
      tot = warp_sum_r(tot);
      if (lane < CL) *cluster.map_shared_rank(&s_ct[par][crank], lane) = tot;
    }
    cluster.sync();
    // winner: the largest key over the CL slots (every lane of every warp ends with it)
    unsigned long long key = lane < CL ? s_ck[par][lane] : 0ULL;
    for (int o = 16; o; o >>= 1) {
      const unsigned long long ok = __shfl_xor_sync(0xffffffffu, key, o);
      key = ok > key ? ok : key;
    }
    int idx = key ? piv_key_index(key) : -1;
    const int bw = idx >= 0 ? idx / per : 0;
    if (idx >= m || (idx >= 0 && (bw >= CL || idx - bw * per >= 64))) {  // cannot happen; uniform over the cluster
      if (tid == 0) atomicExch(err, 1);
      idx = -1;
    }
    if (warp == 0) {
      R tot = lane < CL ? s_ct[par][lane] : R(0);
      tot = warp_sum_r(tot);
      if (lane == 0) {
        if (j == 0) tol2 = (R)(eps * eps) * tot;
        const R best = idx >= 0 ? s_cb[par][bw] : R(0);
        s_best = best;
        s_stop = (j == kmax) || idx < 0 || !(best > R(0)) || tot <= tol2;
        s_key[par] = 0ULL;  // this block's key for step j has been published
      }
    }
    if (idx >= 0) {
      const cx<R>* src = cluster.map_shared_rank(cand + (long long)(idx - bw * per) * p, bw);
      for (int i = tid; i < p; i += blockDim.x) pvec[i] = src[i];
    }
    __syncthreads();
    if (s_stop) {
      k = j;
      break;
    }
    const R best = s_best;
    const R nu = sqrt(best);
    const R inu2 = R(1) / best;
    if (crank == bw && tid == 0) {
      s_sel[idx - c0] = j;
      sel[idx] = j;
      piv[j] = idx;
      Rm[(long long)j * m + idx] = mk<R>(nu, R(0));
    }
    for (int c = warp; c < mc; c += nwarp) {
      if (c0 + c == idx || s_sel[c] != -1) continue;
      cx<R>* a = cand + (long long)c * p;
      cx<R> d = project_coeff(pvec, a, p, lane, inu2);  // coefficient of the pivot vector
      R nr = project_update(pvec, a, p, lane, d);
      if (lane == 0) {
        s_nrm[c] = nr;
        Rm[(long long)j * m + c0 + c] = scale(d, nu);  // R(j, c) = q^H a = (a_pv^H a) / nu
        atomicMax(&s_key[par ^ 1], piv_key(nr, c0 + c));
      }
    }
    __syncthreads();
  }
  if (crank == 0 && tid == 0) rank[0] = k;
  cluster.sync();  // every remote read is done; piv and Rm are complete and visible
  for (long long t = (long long)crank * blockDim.x + tid; t < (long long)k * k; t += (long long)CL * blockDim.x) {
    int a = (int)(t / k), bb = (int)(t % k);
    RT[t] = bb <= a ? ldcg_cx(Rm + (long long)bb * m + __ldcg(piv + a)) : mk<R>(0, 0);
  }
  cluster.sync();
  cx<R>* t = pvec + (long long)warp * kmax;
  for (int c = c0 + warp; c < c1; c += nwarp) {
    int sc = s_sel[c - c0];
    if (sc >= 0) {
      for (int a = lane; a < k; a += 32) U[(long long)c * k + a] = mk<R>(a == sc ? R(1) : R(0), R(0));
      continue;
    }
    for (int a = lane; a < k; a += 32) t[a] = ldcg_cx(Rm + (long long)a * m + c);
    __syncwarp();
    for (int a = k - 1; a >= 0; --a) {
      const cx<R>* col = RT + (long long)a * k;
      const cx<R> ta = t[a] * inv(ldcg_cx(col + a));
      __syncwarp();
      for (int bb = lane; bb < a; bb += 32) {
        cx<R> v = t[bb], r = ldcg_cx(col + bb);
        v.re -= r.re * ta.re - r.im * ta.im;
        v.im -= r.re * ta.im + r.im * ta.re;
        t[bb] = v;
      }
      if (lane == 0) t[a] = ta;
      __syncwarp();
    }
    for (int a = lane; a < k; a += 32) U[(long long)c * k + a] = t[a];
    __syncwarp();
  }
}

// ---------------------------------------------------------------- register-resident ID
// In the two kernels below every warp owns one candidate and keeps its residual
// vector in registers (lane l holds entries l, l + 32, ..., l + 32 (T - 1)).
// A pivot step then touches shared memory only to read the pivot vector q;
// the block's best candidate is published by its warp (double-buffered by step
// parity).  The coefficients R(j, c) are collected in registers (lane j mod 32
// holds step j) and written to global memory every 32 steps, so that no global
// store is in flight at the per-step barrier; pivots and selections are
// written once at the end.

// Projection of the pivot vector q (shared memory) out of a register vector:
// d = q^H a / |q|^2, a -= q d; returns the new |a|^2 (warp-wide) and d.
template <class R, int T>
__device__ __forceinline__ R reg_project(cx<R> (&a)[T], const cx<R>* q, int p, int lane, R inu2, cx<R>& dout) {
  cx<R> s0 = mk<R>(0, 0), s1 = mk<R>(0, 0);
#pragma unroll
  for (int t = 0; t < T; t += 2) {
    const int i0 = lane + 32 * t;
    if (i0 < p) fmac_(s0, q[i0], a[t]);
    if (t + 1 < T) {
      const int i1 = i0 + 32;
      if (i1 < p) fmac_(s1, q[i1], a[t + 1]);
    }
  }
  const cx<R> d = scale(warp_sum(s0 + s1), inu2);
  R n0 = 0, n1 = 0;
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int i = lane + 32 * t;
    if (i < p) {
      const cx<R> qi = q[i];
      a[t].re -= qi.re * d.re - qi.im * d.im;
      a[t].im -= qi.re * d.im + qi.im * d.re;
      if (t & 1)
        n1 += abs2(a[t]);
      else
        n0 += abs2(a[t]);
    }
  }
  dout = d;
  return warp_sum_r(n0 + n1);
}

// Deferred write of the register-held coefficients R(t, c), steps [t0, t1).
template <class R>
__device__ __forceinline__ void flush_coeffs(cx<R>* Rm, int m, int c, int lane, int t0, int t1, int rsel, cx<R> rbuf) {
  const int t = t0 + lane;
  if (t < t1 && (rsel < 0 || t <= rsel)) Rm[(long long)t * m + c] = rbuf;
}

// U rows (identity on the skeleton, R11^-1 R12 elsewhere) by column-oriented
// back substitution, one warp per candidate; tbuf: kmax entries per warp.
template <class R>
__device__ __forceinline__ void id_back_substitution(const cx<R>* Rm, const cx<R>* RT, int m, int k, int c, int sc,
                                                     int lane, cx<R>* tbuf, cx<R>* U) {
  if (sc >= 0) {
    for (int a = lane; a < k; a += 32) U[(long long)c * k + a] = mk<R>(a == sc ? R(1) : R(0), R(0));
    return;
  }
  for (int a = lane; a < k; a += 32) tbuf[a] = ldcg_cx(Rm + (long long)a * m + c);
  __syncwarp();
  for (int a = k - 1; a >= 0; --a) {
    const cx<R>* col = RT + (long long)a * k;
    const cx<R> ta = tbuf[a] * inv(ldcg_cx(col + a));
    __syncwarp();
    for (int bb = lane; bb < a; bb += 32) {
      cx<R> v = tbuf[bb], r = ldcg_cx(col + bb);
      v.re -= r.re * ta.re - r.im * ta.im;
      v.im -= r.re * ta.im + r.im * ta.re;
      tbuf[bb] = v;
    }
    if (lane == 0) tbuf[a] = ta;
    __syncwarp();
  }
  for (int a = lane; a < k; a += 32) U[(long long)c * k + a] = tbuf[a];
  __syncwarp();
}

// U rows of the ID by a blocked back substitution: U(c, :) = (R11^-1 R(:, c))^T
// for a candidate c that is not a pivot, e_sel(c) for a pivot (Sec. 2.1, the
// interpolation matrix T = R11^-1 R12).  CB candidates per block, one warp
// each for the triangular panel solves, all kTrsmThreads threads for the
// updates; the right-hand sides (column c of R, k entries) live in shared
// memory.  Panels of kTrsmNB rows are taken from the bottom: the panel's
// diagonal block (read from RT = R11^T, so a row of RT is a column of R11) is
// staged in shared memory (the next panel's block is fetched during the
// current panel's update) and each warp solves its candidate's panel rows with
// warp-synchronous steps (one lane per row); then the block updates the rows
// above the panel with the panel's solved unknowns, reading kTrsmNB rows of RT
// (coalesced, sixteen loads in flight per thread).  k is read on the device
// (rank[0]).
constexpr int kTrsmNB = 32, kTrsmThreads = 256;
template <class R, int CB>
__global__ void __launch_bounds__(kTrsmThreads) id_trsm_kernel(const cx<R>* __restrict__ Rm,
                                                               const cx<R>* __restrict__ RT,
                                                               const int* __restrict__ sel,
                                                               const int* __restrict__ rank, int m, int kmax,
                                                               cx<R>* __restrict__ U) {
  extern __shared__ unsigned char smraw[];
  cx<R>* tv = reinterpret_cast<cx<R>*>(smraw);  // CB x kmax
  cx<R>* Db = tv + (size_t)CB * kmax;            // 2 x kTrsmNB^2: D[q][r] = R11(i0 + r, i0 + q), r <= q
  const int k = min(*rank, kmax);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int c = blockIdx.x * CB + warp;
  const bool solver = warp < CB;
  const bool own = solver && c < m;
  const int sc = own ? sel[c] : 0;
  const bool solve = own && sc < 0;
  cx<R>* t = tv + (size_t)(solver ? warp : 0) * kmax;
  for (int e = tid; e < CB * k; e += kTrsmThreads) {
    const int j = e / k, a = e % k, cj = blockIdx.x * CB + j;
    const bool sj = cj < m && sel[cj] < 0;
    tv[(size_t)j * kmax + a] = sj ? ldcg_cx(Rm + (long long)a * m + cj) : mk<R>(0, 0);
  }
  auto load_diag = [&](int i1, cx<R>* D) {
    const int i0 = max(0, i1 - kTrsmNB), w = i1 - i0;
    for (int e = tid; e < w * w; e += kTrsmThreads) {
      const int q = e / w, r = e % w;
      D[q * kTrsmNB + r] = r <= q ? ldcg_cx(RT + (long long)(i0 + q) * k + i0 + r) : mk<R>(0, 0);
    }
  };
  if (k > 0) load_diag(k, Db);
  __syncthreads();
  int buf = 0;
  for (int i1 = k; i1 > 0; i1 -= kTrsmNB) {
    const int i0 = max(0, i1 - kTrsmNB), w = i1 - i0;
    const cx<R>* D = Db + buf * kTrsmNB * kTrsmNB;
    if (solve) {  // rows i1 - 1 .. i0 of this candidate; lane r holds row i0 + r
      cx<R> x = lane < w ? t[i0 + lane] : mk<R>(0, 0);
      for (int q = w - 1; q >= 0; --q) {
        const cx<R> xq = mk<R>(__shfl_sync(0xffffffffu, x.re, q), __shfl_sync(0xffffffffu, x.im, q));
        const cx<R> tq = xq * inv(D[q * kTrsmNB + q]);
        if (lane == q) x = tq;
        if (lane < q) {
          const cx<R> r = D[q * kTrsmNB + lane];
          x.re -= r.re * tq.re - r.im * tq.im;
          x.im -= r.re * tq.im + r.im * tq.re;
        }
      }
      if (lane < w) t[i0 + lane] = x;
    }
    __syncthreads();
    if (i0 > 0) load_diag(i0, Db + (buf ^ 1) * kTrsmNB * kTrsmNB);  // next panel's block, during the update
    // rows above the panel: t[b] -= sum_{a in panel} R11(b, a) t[a] = RT[a][b] t[a]
    for (int b = tid; b < i0; b += kTrsmThreads) {
      cx<R> acc[CB];
#pragma unroll
      for (int j = 0; j < CB; ++j) acc[j] = mk<R>(0, 0);
      for (int a0 = i0; a0 < i1; a0 += 16) {
        cx<R> rv[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) rv[u] = a0 + u < i1 ? ldcg_cx(RT + (long long)(a0 + u) * k + b) : mk<R>(0, 0);
#pragma unroll
        for (int u = 0; u < 16; ++u)
          if (a0 + u < i1) {
#pragma unroll
            for (int j = 0; j < CB; ++j) fma_(acc[j], rv[u], tv[(size_t)j * kmax + a0 + u]);
          }
      }
#pragma unroll
      for (int j = 0; j < CB; ++j) tv[(size_t)j * kmax + b] = tv[(size_t)j * kmax + b] - acc[j];
    }
    __syncthreads();
    buf ^= 1;
  }
  if (own)
    for (int a = lane; a < k; a += 32)
      U[(long long)c * k + a] = solve ? t[a] : mk<R>(a == sc ? R(1) : R(0), R(0));
}

// Launch of id_trsm_kernel with as many candidates per block (4, 2 or 1) as
// their right-hand sides (kmax entries each) leave room for in shared memory.
template <class R>
int launch_id_trsm(const cx<R>* Rm, const cx<R>* RT, const int* sel, const int* rank, int m, int kmax, cx<R>* U,
                   cudaStream_t sb) {
  const size_t diag = sizeof(cx<R>) * (size_t)2 * kTrsmNB * kTrsmNB;
  auto smem = [&](int cb) { return sizeof(cx<R>) * (size_t)cb * kmax + diag; };
  const size_t limit = 227 * 1024;
  const int CB = smem(4) <= limit ? 4 : smem(2) <= limit ? 2 : smem(1) <= limit ? 1 : 0;
  if (!CB) {
    set_last_error_text("ID rank too large for the back substitution's shared memory");
    return LS_EINVAL;
  }
  const size_t smt = smem(CB);
  const void* fn = CB == 4 ? (const void*)id_trsm_kernel<R, 4> : CB == 2 ? (const void*)id_trsm_kernel<R, 2>
                                                                          : (const void*)id_trsm_kernel<R, 1>;
  if (smt > 48 * 1024) LS_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smt));
  count_launch();
  const unsigned grid = (unsigned)((m + CB - 1) / CB);
  if (CB == 4)
    id_trsm_kernel<R, 4><<<grid, kTrsmThreads, smt, sb>>>(Rm, RT, sel, rank, m, kmax, U);
  else if (CB == 2)
    id_trsm_kernel<R, 2><<<grid, kTrsmThreads, smt, sb>>>(Rm, RT, sel, rank, m, kmax, U);
  else
    id_trsm_kernel<R, 1><<<grid, kTrsmThreads, smt, sb>>>(Rm, RT, sel, rank, m, kmax, U);
  return check_launch("ID back substitution");
}

// Cluster version: CL <= 16 blocks of 1024 threads, at most 32 candidates per
// block (block r owns candidates [r per, r per + per)), p <= 32 T.  Each warp
// keeps its candidate's key (0 once the candidate is a pivot) in a per-warp
// slot; per step every warp reduces the block's key from the 32 slots
// (redux.sync), the best warp publishes its vector, lanes r < CL of warp 0
// store the block key (FP64: and the best norm), lanes of warp 1 the block
// total, into slot [this block] of block r; one cluster barrier; every warp
// reduces the winner from the CL slots of its own block; thread 0 sums the CL
// totals in a fixed order and decides whether to stop (the same decision in
// every block); the block copies the winner's vector from its owner; one
// block barrier.  Dynamic shared memory: max(3 p, 32 kmax) entries.
template <class R, int T>
__global__ void __launch_bounds__(1024) cpqr_reg_cluster_kernel(const cx<R>* __restrict__ A, int m, int p, int kmax,
                                                                double eps, cx<R>* __restrict__ Rm,
                                                                int* __restrict__ sel, int* __restrict__ piv,
                                                                int* __restrict__ rank, cx<R>* __restrict__ U,
                                                                cx<R>* __restrict__ RT, int* __restrict__ err) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ unsigned char smraw[];
  cx<R>* stage = reinterpret_cast<cx<R>*>(smraw);  // 2 x p: the block's best vector, by step parity
  cx<R>* pvec = stage + 2 * p;                      // p: the winner's vector
  const int CL = (int)cluster.num_blocks(), crank = (int)cluster.block_rank();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int per = (m + CL - 1) / CL;
  const int c0 = min(m, crank * per), mc = min(m, c0 + per) - c0;
  __shared__ unsigned long long s_wkey[32];   // each warp's candidate key, 0 if none
  __shared__ unsigned long long s_ck[2][16];  // every block's key, by step parity and block
  __shared__ R s_cb[2][16], s_ct[2][16];      // every block's best norm (FP64) and total
  __shared__ R s_nrm[32];
  __shared__ int s_stop;

  const bool own = warp < mc;
  const int c = c0 + warp;
  cx<R> a[T];
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int i = lane + 32 * t;
    a[t] = (own && i < p) ? A[(long long)c * p + i] : mk<R>(0, 0);
  }
  R nrm = 0;
#pragma unroll
  for (int t = 0; t < T; ++t) nrm += abs2(a[t]);
  nrm = warp_sum_r(nrm);
  if (lane == 0) {
    s_nrm[warp] = own ? nrm : R(0);
    s_wkey[warp] = own ? piv_key(nrm, c) : 0ULL;
  }
  __syncthreads();
  cx<R> rbuf = mk<R>(0, 0);
  int rsel = -1;  // step at which this warp's candidate became a pivot
  R tol2 = 0;
  int k = 0;
  for (int j = 0;; ++j) {
    const int par = j & 1;
    const unsigned long long kw = s_wkey[lane];
    const unsigned long long kb = warp_max_key(kw);
    const int lb = kb ? piv_key_index(kb) - c0 : -1;
    if (warp == lb) {
      cx<R>* st = stage + par * p;
#pragma unroll
      for (int t = 0; t < T; ++t) {
        const int i = lane + 32 * t;
        if (i < p) st[i] = a[t];
      }
    }
    if (warp == 0) {
      if (lane < CL) {
        *cluster.map_shared_rank(&s_ck[par][crank], lane) = kb;
        if constexpr (sizeof(R) == 8) *cluster.map_shared_rank(&s_cb[par][crank], lane) = lb >= 0 ? s_nrm[lb] : R(0);
      }
    } else if (warp == 1) {
      R tot = kw ? s_nrm[lane] : R(0);
      tot = warp_sum_r(tot);
      if (lane < CL) *cluster.map_shared_rank(&s_ct[par][crank], lane) = tot;
    }
    cluster.sync();
    const unsigned long long key = warp_max_key(lane < CL ? s_ck[par][lane] : 0ULL);
    int idx = key ? piv_key_index(key) : -1;
    const int bw = idx >= 0 ? idx / per : 0;
    if (idx >= m || (idx >= 0 && (bw >= CL || idx - bw * per >= 32))) {  // cannot happen; uniform
      if (tid == 0) atomicExch(err, 1);
      idx = -1;
    }
    R best;
    if constexpr (sizeof(R) == 4)
      best = piv_key_norm(key);
    else
      best = idx >= 0 ? s_cb[par][bw] : R(0);
    if (tid == 0) {
      R tot = 0;
      for (int r = 0; r < CL; ++r) tot += s_ct[par][r];
      if (j == 0) tol2 = (R)(eps * eps) * tot;
      s_stop = (j == kmax) || idx < 0 || !(best > R(0)) || tot <= tol2;
    }
    if (idx >= 0) {
      const cx<R>* src = cluster.map_shared_rank(stage + par * p, bw);
      for (int i = tid; i < p; i += blockDim.x) pvec[i] = src[i];
    }
    __syncthreads();
    if (s_stop) {
      k = j;
      break;
    }
    const R nu = sqrt(best);
    if (own && c == idx) {
      rsel = j;
      if (lane == (j & 31)) rbuf = mk<R>(nu, R(0));
      if (lane == 0) s_wkey[warp] = 0ULL;
    }
    if (own && rsel < 0) {
      cx<R> d;
      const R nr = reg_project<R, T>(a, pvec, p, lane, R(1) / best, d);
      if (lane == (j & 31)) rbuf = scale(d, nu);  // R(j, c) = q^H a = (a_pv^H a) / nu
      if (lane == 0) {
        s_nrm[warp] = nr;
        s_wkey[warp] = piv_key(nr, c);
      }
    }
    if ((j & 31) == 31 && own) flush_coeffs(Rm, m, c, lane, j - 31, j + 1, rsel, rbuf);
    __syncthreads();
  }
  if (own) {
    flush_coeffs(Rm, m, c, lane, k & ~31, k, rsel, rbuf);
    if (lane == 0) {
      sel[c] = rsel;
      if (rsel >= 0) piv[rsel] = c;
    }
  }
  if (crank == 0 && tid == 0) rank[0] = k;
  cluster.sync();  // Rm, piv complete and visible in the cluster
  for (long long t = (long long)crank * blockDim.x + tid; t < (long long)k * k; t += (long long)CL * blockDim.x) {
    int aa = (int)(t / k), bb = (int)(t % k);
    RT[t] = bb <= aa ? ldcg_cx(Rm + (long long)bb * m + __ldcg(piv + aa)) : mk<R>(0, 0);
  }
  // U follows from RT and R in id_trsm_kernel
}

// Dynamic shared memory the grid ID kernel asks for at least: with it no block
// of the merge kernels (>= 8 KB of shared memory each) fits on the same SM.
constexpr size_t kIdSmemReserve = 220 * 1024;

// Per-step exchange record of the grid ID kernel.  word: bits 52..63 count the
// blocks that have arrived, bits 0..51 hold the sum of their residual totals in
// fixed point, unit = (eps^2 total_0) 2^-20 (the stopping threshold is 2^20
// units; each block's term saturates at 2^40, far above it), so the barrier
// and the total are one atomic add, and integer addition makes the sum
// independent of the arrival order (every block takes the same stopping
// decision, run after run).
struct StepExchange {
  unsigned long long key;   // largest pivot key of the step
  unsigned long long word;  // arrivals and fixed-point total
};
__device__ __forceinline__ void red_release_add(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Cooperative-grid version: blocks of 1024 threads holding 8 candidates, four
// warps per candidate (warp part w holds entries lane + 32 (w + 4 t), t < T4,
// p <= 128 T4), so that each warp's dependent chain per step is a quarter of
// the vector.  The coefficient and the new norm of a candidate are reduced
// over its four warps through shared memory (fixed order) behind a named
// barrier of the 128 threads.  The initial total (the scale of the fixed-point
// totals) is reduced once through the slots.  Per step: the block's best
// candidate publishes its vector to a parity vector slot; thread 0 folds the
// block key into the step's key (atomic max) and arrives with the block total
// (release add on the step's word), then polls the word (acquire, bounded)
// until every block has arrived; every thread reads the step's key, the block
// copies the winner's vector.  ex[0..kmax] zero at launch.  Dynamic shared
// memory: max(p, 8 kmax) entries.
template <class R, int T4>
__global__ void __launch_bounds__(1024) cpqr_reg_grid_kernel(const cx<R>* __restrict__ A, int m, int p, int kmax,
                                                             double eps, cx<R>* __restrict__ Rm, int* __restrict__ sel,
                                                             int* __restrict__ piv, int* __restrict__ rank,
                                                             cx<R>* __restrict__ U, cx<R>* __restrict__ RT,
                                                             IdSlot<R>* __restrict__ slots, cx<R>* __restrict__ pslots,
                                                             StepExchange* __restrict__ ex, GridSync gs,
                                                             int* __restrict__ err) {
  extern __shared__ unsigned char smraw[];
  cx<R>* pvec = reinterpret_cast<cx<R>*>(smraw);
  const int nblk = gridDim.x, blk = blockIdx.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int cand = warp >> 2, part = warp & 3;
  const int cpb = blockDim.x >> 7;  // candidates per block (four warps each, at most 8)
  const int c0 = min(m, blk * cpb), mc = min(m, c0 + cpb) - c0;
  __shared__ unsigned long long s_wkey[8];
  __shared__ R s_nrm[8];
  __shared__ cx<R> s_part[8][4];
  __shared__ R s_npart[8][4];
  __shared__ unsigned long long s_word;
  __shared__ R s_scale;
  __shared__ int s_fail;
  unsigned int epoch = 0;
  const unsigned bar_id = 1 + cand;  // named barrier of this candidate's four warps

  const bool own = cand < mc;
  const int c = c0 + cand;
  cx<R> a[T4];
#pragma unroll
  for (int t = 0; t < T4; ++t) {
    const int i = lane + 32 * (part + 4 * t);
    a[t] = (own && i < p) ? A[(long long)c * p + i] : mk<R>(0, 0);
  }
  {
    R nrm = 0;
#pragma unroll
    for (int t = 0; t < T4; ++t) nrm += abs2(a[t]);
    nrm = warp_sum_r(nrm);
    if (lane == 0) s_npart[cand][part] = nrm;
  }
  if (tid == 0) s_fail = 0;
  if (tid < 8) {  // slots of absent candidates stay empty
    s_wkey[tid] = 0ULL;
    s_nrm[tid] = R(0);
  }
  __syncthreads();
  if (part == 0 && lane == 0) {
    const R nrm = ((s_npart[cand][0] + s_npart[cand][1]) + s_npart[cand][2]) + s_npart[cand][3];
    s_nrm[cand] = own ? nrm : R(0);
    s_wkey[cand] = own ? piv_key(nrm, c) : 0ULL;
  }
  __syncthreads();
  // initial total through the slots: the fixed-point unit and the tolerance
  if (warp == 0) {
    R tot = lane < 8 ? s_nrm[lane] : R(0);
    tot = warp_sum_r(tot);
    if (lane == 0) {
      IdSlot<R> sl;
      sl.best = R(0);
      sl.total = tot;
      sl.idx = -1;
      sl.pad = 0;
      slots[blk] = sl;
    }
  }
  if (!grid_sync(gs, nblk, epoch)) return;
  if (warp == 0) {
    R tot = 0;
    for (int b = lane; b < nblk; b += 32) tot += __ldcg(&slots[b].total);
    tot = warp_sum_r(tot);
    if (lane == 0) s_scale = tot;
  }
  __syncthreads();
  const double thresh = eps * eps * (double)s_scale;          // stop when the residual total <= thresh
  const double fx_inv = thresh > 0.0 ? 1048576.0 / thresh : 0.0;  // fixed-point units per unit total
  const unsigned long long tol_fx = 1ULL << 20, fx_cap = 1ULL << 40;
  cx<R> rbuf = mk<R>(0, 0);
  int rsel = -1;
  int k = 0;
  for (int j = 0;; ++j) {
    const int par = j & 1;
    const unsigned long long kw = lane < 8 ? s_wkey[lane] : 0ULL;
    const unsigned long long kb = warp_max_key(kw);
    const int lb = kb ? piv_key_index(kb) - c0 : -1;
    if (cand == lb) {
      cx<R>* dst = pslots + ((long long)par * nblk + blk) * p;
#pragma unroll
      for (int t = 0; t < T4; ++t) {
        const int i = lane + 32 * (part + 4 * t);
        if (i < p) dst[i] = a[t];
      }
    }
    R btot = 0;
    if (warp == 0) {
      btot = kw ? s_nrm[lane & 7] : R(0);
      btot = warp_sum_r(btot);
      if constexpr (sizeof(R) == 8)
        if (lane == 0) slots[par * nblk + blk].best = lb >= 0 ? s_nrm[lb] : R(0);
    }
    __syncthreads();  // the block's vector and slot are written
    if (tid == 0) {
      if (kb) atomicMax(&ex[j].key, kb);
      const double fxd = (double)btot * fx_inv + 0.5;
      const unsigned long long fx =
          thresh > 0.0 ? (fxd >= (double)fx_cap ? fx_cap : (unsigned long long)fxd) : (btot > R(0) ? fx_cap : 0ULL);
      red_release_add(&ex[j].word, (1ULL << 52) + fx);
      unsigned long long v;
      long long spins = 0;
      while (((v = ld_acquire_u64(&ex[j].word)) >> 52) < (unsigned long long)nblk) {
        if (++spins >= gs.limit || ((spins & 4095) == 0 && *(volatile int*)gs.abort)) {
          atomicExch(gs.abort, 1);
          s_fail = 1;
          break;
        }
      }
      s_word = v;
    }
    __syncthreads();
    if (s_fail) return;
    const unsigned long long key = __ldcg(&ex[j].key);
    int idx = key ? piv_key_index(key) : -1;
    const int bw = idx >= 0 ? idx / cpb : 0;
    if (idx >= m || (idx >= 0 && bw >= nblk)) {  // cannot happen; uniform
      if (tid == 0) atomicExch(err, 1);
      idx = -1;
    }
    R best;
    if constexpr (sizeof(R) == 4)
      best = piv_key_norm(key);
    else
      best = idx >= 0 ? __ldcg(&slots[par * nblk + bw].best) : R(0);
    const unsigned long long tot_fx = s_word & ((1ULL << 52) - 1);
    if ((j == kmax) || idx < 0 || !(best > R(0)) || tot_fx <= tol_fx) {  // the same decision everywhere
      k = j;
      break;
    }
    {
      const cx<R>* src = pslots + ((long long)par * nblk + bw) * p;
      for (int i = tid; i < p; i += blockDim.x) pvec[i] = ldcg_cx(src + i);
    }
    const R nu = sqrt(best);
    if (own && c == idx) {
      rsel = j;
      if (part == 0 && lane == (j & 31)) rbuf = mk<R>(nu, R(0));
      if (part == 0 && lane == 0) s_wkey[cand] = 0ULL;
    }
    __syncthreads();  // the winner's vector is in shared memory
    if (own && rsel < 0) {
      cx<R> s0 = mk<R>(0, 0), s1 = mk<R>(0, 0);
#pragma unroll
      for (int t = 0; t < T4; ++t) {
        const int i = lane + 32 * (part + 4 * t);
        if (i < p) {
          if (t & 1)
            fmac_(s1, pvec[i], a[t]);
          else
            fmac_(s0, pvec[i], a[t]);
        }
      }
      const cx<R> ps = warp_sum(s0 + s1);
      if (lane == 0) s_part[cand][part] = ps;
      asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory");
      const cx<R> d = scale(((s_part[cand][0] + s_part[cand][1]) + s_part[cand][2]) + s_part[cand][3], R(1) / best);
      R n0 = 0, n1 = 0;
#pragma unroll
      for (int t = 0; t < T4; ++t) {
        const int i = lane + 32 * (part + 4 * t);
        if (i < p) {
          const cx<R> qi = pvec[i];
          a[t].re -= qi.re * d.re - qi.im * d.im;
          a[t].im -= qi.re * d.im + qi.im * d.re;
          if (t & 1)
            n1 += abs2(a[t]);
          else
            n0 += abs2(a[t]);
        }
      }
      const R pn = warp_sum_r(n0 + n1);
      if (lane == 0) s_npart[cand][part] = pn;
      if (part == 0 && lane == (j & 31)) rbuf = scale(d, nu);  // R(j, c) = q^H a = (a_pv^H a) / nu
      asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory");
      if (part == 0 && lane == 0) {
        const R nr = ((s_npart[cand][0] + s_npart[cand][1]) + s_npart[cand][2]) + s_npart[cand][3];
        s_nrm[cand] = nr;
        s_wkey[cand] = piv_key(nr, c);
      }
    }
    if ((j & 31) == 31 && own && part == 0) flush_coeffs(Rm, m, c, lane, j - 31, j + 1, rsel, rbuf);
    __syncthreads();
  }
  if (own && part == 0) {
    flush_coeffs(Rm, m, c, lane, k & ~31, k, rsel, rbuf);
    if (lane == 0) {
      sel[c] = rsel;
      if (rsel >= 0) piv[rsel] = c;
    }
  }
  if (blk == 0 && tid == 0) rank[0] = k;
  if (!grid_sync(gs, nblk, epoch)) return;
  for (long long t = (long long)blk * blockDim.x + tid; t < (long long)k * k; t += (long long)nblk * blockDim.x) {
    int aa = (int)(t / k), bb = (int)(t % k);
    RT[t] = bb <= aa ? ldcg_cx(Rm + (long long)bb * m + __ldcg(piv + aa)) : mk<R>(0, 0);
  }
  // U follows from RT and R in id_trsm_kernel
}

template <class R>
__global__ void identity_kernel(cx<R>* U, int m) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)m * m) return;
  U[t] = mk<R>((t / m) == (t % m) ? R(1) : R(0), R(0));
}

template <class R>
int upload_block(const std::vector<int>& rx, const std::vector<int>& ry, const std::vector<int>& px,
                 const std::vector<int>& py, cx<R>* out, int* dtmp, cudaStream_t st, const KernelSpec& ks,
                 const KernelTable& kt) {
  int m = (int)rx.size(), p = (int)px.size();
  std::vector<int> host(2 * m + 2 * p);
  std::copy(rx.begin(), rx.end(), host.begin());
  std::copy(ry.begin(), ry.end(), host.begin() + m);
  std::copy(px.begin(), px.end(), host.begin() + 2 * m);
  std::copy(py.begin(), py.end(), host.begin() + 2 * m + p);
  int* pin = static_cast<int*>(pinned_scratch(sizeof(int) * host.size()));
  if (!pin) return LS_ENOMEM;
  std::copy(host.begin(), host.end(), pin);
  LS_CUDA_TRY(cudaMemcpyAsync(dtmp, pin, sizeof(int) * host.size(), cudaMemcpyHostToDevice, st));
  long long tot = (long long)m * p;
  if (tot > 0)
    {
      count_launch();
      block_kernel<R><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(dtmp, dtmp + m, m, dtmp + 2 * m, dtmp + 2 * m + p,
                                                                     p, out, p, kt, ks);
    }
  // host vector must outlive the copy
  LS_CUDA_TRY(cudaStreamSynchronize(st));
  return check_launch("kernel block");
}

// Row ID by blocks of pivots (id_blocked.cu), its interpolation matrix by a
// blocked back substitution (on su when given, like the greedy kernels' U).  A
// is overwritten.
template <class R>
int run_row_id_blocked(cx<R>* A, int m, int p, double eps, cudaStream_t st, int* k_out, std::vector<int>* hp,
                       cx<R>* Uout, cudaStream_t su) {
  int tk = prof_begin(st);
  int k = 0;
  int rc = blocked_row_id<R>(A, m, p, eps, st, su, Uout, &k, hp);
  // algorithmic work of the ID: ~8 m p k real flops (one projection of every
  // candidate on every pivot direction); one read of the block
  prof_end(tk, PR_CPQR, st, sizeof(cx<R>) * (double)m * p, 8.0 * m * (double)p * k);
  if (rc) return rc;
  *k_out = k;
  return LS_OK;
}

// Candidates from which the blocked ID takes over from the greedy kernels
// (ID_AUTO), and above which only the blocked ID applies (the greedy kernels
// keep a candidate's residual in registers or one block's shared memory).
constexpr int kBlockedMinRows = 1024;

// Row ID of the device matrix A (m candidates x p, candidate-major) by the
// column-pivoted QR kernels above: one thread-block cluster when the
// candidates fit in the shared memory of at most 16 blocks, else one
// cooperative grid.  Returns k, the pivots (host) and, if Uout is not null,
// U (m x k, device, row-major).  sync_buf: 64 zeroed-on-entry bytes of device
// scratch for the grid barrier and the kernels' status words.
template <class R>
int run_row_id(const cx<R>* A, int m, int p, double eps_in, int nsm, int* sync_buf, cudaStream_t st, int* k_out,
               std::vector<int>* hp_out, cx<R>* Uout, cudaStream_t su = nullptr, int method = ID_GREEDY,
               bool a_mutable = false) {
  int rc;
  const bool greedy_fits = (p + 127) / 128 <= (sizeof(R) == 4 ? 16 : 8);
  if (method == ID_BLOCKED || (method == ID_AUTO && (m >= kBlockedMinRows || !greedy_fits))) {
    if (a_mutable) return run_row_id_blocked<R>(const_cast<cx<R>*>(A), m, p, eps_in, st, k_out, hp_out, Uout, su);
    cx<R>* Aw = nullptr;
    if ((rc = dalloc((void**)&Aw, sizeof(cx<R>) * (size_t)m * p))) return rc;
    LS_CUDA_TRY(cudaMemcpyAsync(Aw, A, sizeof(cx<R>) * (size_t)m * p, cudaMemcpyDeviceToDevice, st));
    rc = run_row_id_blocked<R>(Aw, m, p, eps_in, st, k_out, hp_out, Uout, su);
    dfree(Aw);
    return rc;
  }
  std::vector<int>& hp = *hp_out;
  const int kmax = std::min(m, p);
  if (m >= (1 << 20)) {  // pivot keys carry 20 index bits
    set_last_error_text("too many ID candidates");
    return LS_EINVAL;
  }
  // blocks and candidates per block (at most 64 per block)
  int nblk = std::max(1, std::min(nsm, (m + 1) / 2));
  int per = (m + nblk - 1) / nblk;
  if (per > 64) {
    per = 64;
    nblk = (m + per - 1) / per;
  }
  const int nslot = std::max(nblk, (m + std::min(8, std::max(1, (m + nsm - 1) / nsm)) - 1) /
                                        std::min(8, std::max(1, (m + nsm - 1) / nsm)));  // slots for either grid kernel
  size_t loop_smem = sizeof(cx<R>) * ((size_t)p + (size_t)per * p);
  size_t tail_smem = sizeof(cx<R>) * (size_t)8 * kmax;
  int use_smem = loop_smem <= 200 * 1024;
  size_t smem = std::max(use_smem ? loop_smem : sizeof(cx<R>) * (size_t)p, tail_smem);
  if (smem > 220 * 1024) {
    set_last_error_text("proxy block too large for the ID kernel");
    return LS_EINVAL;
  }
  size_t need = 64 * 256 + sizeof(cx<R>) * ((size_t)m * p * (use_smem ? 0 : 1) + (size_t)m * kmax +
                                 (size_t)2 * nslot * p) +
                sizeof(int) * (m + 8) + sizeof(IdSlot<R>) * 2 * (nslot + 1) +
                2 * sizeof(unsigned long long) * ((size_t)kmax + 1) + 2048;
  // R, R11^T, the selection and the rank (what the back substitution reads) in an
  // allocation of their own: with an auxiliary stream su the back substitution runs
  // there, beside the next level's ID, and this allocation is released on su
  const size_t need_t = 4 * 256 + sizeof(cx<R>) * ((size_t)kmax * m + (size_t)kmax * kmax) + sizeof(int) * (m + 8);
  char* wsp = nullptr;
  char* tsp = nullptr;
  if ((rc = dalloc((void**)&wsp, need))) return rc;
  if ((rc = dalloc((void**)&tsp, need_t))) {
    dfree(wsp);
    return rc;
  }
  char* cur = nullptr;
  auto carve = [&](size_t bytes) {
    char* r = cur;
    cur += (bytes + 255) & ~(size_t)255;
    return r;
  };
  cur = tsp;
  cx<R>* Rm = reinterpret_cast<cx<R>*>(carve(sizeof(cx<R>) * (size_t)kmax * m));
  cx<R>* RT = reinterpret_cast<cx<R>*>(carve(sizeof(cx<R>) * (size_t)kmax * kmax));
  int* sel = reinterpret_cast<int*>(carve(sizeof(int) * m));
  int* rank = reinterpret_cast<int*>(carve(sizeof(int) * 8));
  cur = wsp;
  cx<R>* Aw = use_smem ? nullptr : reinterpret_cast<cx<R>*>(carve(sizeof(cx<R>) * (size_t)m * p));
  cx<R>* Ut = reinterpret_cast<cx<R>*>(carve(sizeof(cx<R>) * (size_t)m * kmax));
  cx<R>* pslots = reinterpret_cast<cx<R>*>(carve(sizeof(cx<R>) * (size_t)2 * nslot * p));
  int* piv = reinterpret_cast<int*>(carve(sizeof(int) * m));
  IdSlot<R>* slots = reinterpret_cast<IdSlot<R>*>(carve(sizeof(IdSlot<R>) * 2 * (nslot + 1)));
  unsigned long long* gkey =
      reinterpret_cast<unsigned long long*>(carve(2 * sizeof(unsigned long long) * ((size_t)kmax + 1)));
  // one cluster when the candidates fit in the shared memory of CL blocks: the
  // smallest CL with at most 32 candidates per block (4 per warp), else at most 64
  int maxcl = 16;
  if (cudaFuncSetAttribute(cpqr_id_cluster_kernel<R>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
      cudaSuccess) {
    cudaGetLastError();
    maxcl = 8;
  }
  const size_t cl_tail_smem = sizeof(cx<R>) * (size_t)32 * kmax;
  auto cl_smem = [&](int cl) {
    const int pc = (m + cl - 1) / cl;
    return std::max(sizeof(cx<R>) * ((size_t)p + (size_t)pc * p), cl_tail_smem);
  };
  // the smallest cluster with at most one candidate per warp (32 per block), else at most 64 per block
  int CL = 0;
  for (int lim : {32, 64}) {
    for (int cl = 1; cl <= maxcl && !CL; ++cl)
      if ((m + cl - 1) / cl <= lim && cl_smem(cl) <= 220 * 1024) CL = cl;
    if (CL) break;
  }
  bool use_cluster = CL > 0;
  if (!use_cluster) CL = 1;
  const size_t smem_cl = cl_smem(CL);
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  if (use_cluster) {
    LS_CUDA_TRY(cudaFuncSetAttribute(cpqr_id_cluster_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem_cl));
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(1024);
    cfg.dynamicSmemBytes = smem_cl;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, (void*)cpqr_id_cluster_kernel<R>, &cfg) != cudaSuccess || ncl < 1) {
      cudaGetLastError();
      use_cluster = false;
    }
  }
  double eps = eps_in;
  LS_CUDA_TRY(cudaMemsetAsync(sync_buf, 0, 64, st));
  int tk = prof_begin(st);
  // register-resident kernels (one candidate per warp) when the vectors fit in registers
  const int tneed = (p + 31) / 32;
  const int t_cl_max = sizeof(R) == 4 ? 20 : 8;
  int reg_mode = 0;  // 1 cluster, 2 grid
  // grid kernel: spread the candidates over two fifths of the SMs (cpb per block,
  // at most 8, four warps each).  The build runs the merges of lower levels beside
  // the ID, and with the back substitution moved beside the next level's ID the
  // merge chain became the longer path: leaving three fifths of the SMs to the
  // merges measured best (15.0 -> 14.7 ms per build + solve at 256^2; a third:
  // slower merges, three quarters: slower IDs).  A merge block placed on an SM of
  // this latency-bound kernel runs many times slower and holds up its whole
  // launch, so the kernel also takes nearly all of its SMs' shared memory.
  const int nsm_id = std::max(1, nsm - (nsm * 3) / 5);
  const int cpb = std::min(8, std::max(1, (m + nsm_id - 1) / nsm_id));
  int treg = 0, clr = (m + 31) / 32, nblk_r = (m + cpb - 1) / cpb;
  const void* kreg = nullptr;
  size_t smem_r = 0;
  // clusters win while they are small (<= 6 blocks: levels with <= 192 candidates,
  // measured ~3.5-4 us per pivot against ~4.6-5.6 on the grid); above, the grid
  // kernel's spread over more SMs wins (~5 against ~6-8 us per pivot)
  if (tneed <= t_cl_max && clr <= std::min(maxcl, 6)) {
    treg = tneed <= 4 ? 4 : tneed <= 8 ? 8 : tneed <= 12 ? 12 : tneed <= 16 ? 16 : 20;
    if constexpr (sizeof(R) == 4)
      kreg = treg == 4 ? (const void*)cpqr_reg_cluster_kernel<R, 4> : treg == 8 ? (const void*)cpqr_reg_cluster_kernel<R, 8>
           : treg == 12 ? (const void*)cpqr_reg_cluster_kernel<R, 12> : treg == 16 ? (const void*)cpqr_reg_cluster_kernel<R, 16>
           : (const void*)cpqr_reg_cluster_kernel<R, 20>;
    else
      kreg = treg == 4 ? (const void*)cpqr_reg_cluster_kernel<R, 4> : (const void*)cpqr_reg_cluster_kernel<R, 8>;
    smem_r = sizeof(cx<R>) * std::max((size_t)3 * p, (size_t)32 * kmax);
    if (smem_r <= 220 * 1024) reg_mode = 1;
  }
  const int t4need = (p + 127) / 128;
  if (!reg_mode && t4need <= (sizeof(R) == 4 ? 16 : 8)) {
    treg = t4need <= 4 ? 4 : t4need <= 8 ? 8 : t4need <= 12 ? 12 : 16;
    if constexpr (sizeof(R) == 4)
      kreg = treg == 4 ? (const void*)cpqr_reg_grid_kernel<R, 4> : treg == 8 ? (const void*)cpqr_reg_grid_kernel<R, 8>
           : treg == 12 ? (const void*)cpqr_reg_grid_kernel<R, 12> : (const void*)cpqr_reg_grid_kernel<R, 16>;
    else
      kreg = treg == 4 ? (const void*)cpqr_reg_grid_kernel<R, 4> : (const void*)cpqr_reg_grid_kernel<R, 8>;
    smem_r = std::max(sizeof(cx<R>) * std::max((size_t)p, (size_t)cpb * kmax), (size_t)kIdSmemReserve);
    int per_sm = 0;
    if (smem_r <= 220 * 1024 && nblk_r <= nsm &&
        cudaFuncSetAttribute(kreg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_r) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kreg, 128 * cpb, smem_r) == cudaSuccess &&
        nblk_r <= per_sm * nsm)
      reg_mode = 2;
    cudaGetLastError();
  }
  if (reg_mode == 1) {
    LS_CUDA_TRY(cudaFuncSetAttribute(kreg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_r));
    if (maxcl == 16) LS_CUDA_TRY(cudaFuncSetAttribute(kreg, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t rc_cfg;
    cudaLaunchAttribute rc_attr[1];
    memset(&rc_cfg, 0, sizeof(rc_cfg));
    rc_cfg.gridDim = dim3(clr);
    rc_cfg.blockDim = dim3(1024);
    rc_cfg.dynamicSmemBytes = smem_r;
    rc_cfg.stream = st;
    rc_attr[0].id = cudaLaunchAttributeClusterDimension;
    rc_attr[0].val.clusterDim.x = clr;
    rc_attr[0].val.clusterDim.y = 1;
    rc_attr[0].val.clusterDim.z = 1;
    rc_cfg.attrs = rc_attr;
    rc_cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, kreg, &rc_cfg) != cudaSuccess || ncl < 1) {
      cudaGetLastError();
      reg_mode = 0;
    } else {
      const cx<R>* Ac = A;
      int* ierr = sync_buf + 3;
      void* args[] = {&Ac, (void*)&m, (void*)&p, (void*)&kmax, &eps, &Rm, &sel, &piv, &rank, &Ut, &RT, &ierr};
      count_launch();
      LS_CUDA_TRY(cudaLaunchKernelExC(&rc_cfg, kreg, args));
    }
  } else if (reg_mode == 2) {
    GridSync gs;
    gs.count = reinterpret_cast<unsigned*>(sync_buf);
    gs.gen = reinterpret_cast<unsigned*>(sync_buf) + 1;
    gs.abort = sync_buf + 2;
    gs.limit = spin_limit();
    const cx<R>* Ac = A;
    int* ierr = sync_buf + 3;
    StepExchange* ex = reinterpret_cast<StepExchange*>(gkey);
    LS_CUDA_TRY(cudaMemsetAsync(ex, 0, sizeof(StepExchange) * ((size_t)kmax + 1), st));
    void* args[] = {&Ac, (void*)&m, (void*)&p, (void*)&kmax, &eps, &Rm, &sel, &piv, &rank, &Ut, &RT,
                    &slots, &pslots, &ex, &gs, &ierr};
    count_launch();
    LS_CUDA_TRY(cudaLaunchCooperativeKernel(kreg, dim3(nblk_r), dim3(128 * cpb), args, smem_r, st));
  }
  bool u_on_aux = false;  // U written by the back substitution on su
  if (reg_mode) {
    cudaStream_t sb = st;
    cx<R>* Udst = Ut;
    if (su && Uout) {  // U straight into Uout on the auxiliary stream, after the ID kernel
      cudaEvent_t e;
      LS_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      LS_CUDA_TRY(cudaEventRecord(e, st));
      LS_CUDA_TRY(cudaStreamWaitEvent(su, e, 0));
      cudaEventDestroy(e);
      sb = su;
      Udst = Uout;
      u_on_aux = true;
    }
    if ((rc = launch_id_trsm<R>(Rm, RT, sel, rank, m, kmax, Udst, sb))) return rc;
  } else if (use_cluster) {
    count_launch();
    LS_CUDA_TRY(cudaLaunchKernelEx(&cfg, cpqr_id_cluster_kernel<R>, (const cx<R>*)A, m, p, kmax, eps, Rm, sel, piv,
                                   rank, Ut, RT, sync_buf + 3));
  } else {
    const void* kfn = (const void*)cpqr_id_kernel<R>;
    LS_CUDA_TRY(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    LS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, 256, smem));
    if (per_sm < 1 || nblk > per_sm * nsm) {
      set_last_error_text("ID kernel cannot be co-resident");
      return LS_EINVAL;
    }
    GridSync gs;
    gs.count = reinterpret_cast<unsigned*>(sync_buf);
    gs.gen = reinterpret_cast<unsigned*>(sync_buf) + 1;
    gs.abort = sync_buf + 2;
    gs.limit = spin_limit();
    const cx<R>* Ac = A;
    int* ierr = sync_buf + 3;
    LS_CUDA_TRY(cudaMemsetAsync(gkey, 0, sizeof(unsigned long long) * ((size_t)kmax + 1), st));
    void* args[] = {&Ac, (void*)&m, (void*)&p, (void*)&kmax, &eps, &use_smem, &Aw, &Rm, &sel, &slots, &pslots,
                    &gkey, &piv, &rank, &Ut, &RT, &gs, &ierr};
    count_launch();
    LS_CUDA_TRY(cudaLaunchCooperativeKernel(kfn, dim3(nblk), dim3(256), args, smem, st));
  }
  int* pin = static_cast<int*>(pinned_scratch(sizeof(int) * (4 + (size_t)kmax)));
  if (!pin) return LS_ENOMEM;
  // rank, status words and all kmax pivot slots (entries past the rank are unused) in one round trip
  LS_CUDA_TRY(cudaMemcpyAsync(pin, rank, sizeof(int), cudaMemcpyDeviceToHost, st));
  LS_CUDA_TRY(cudaMemcpyAsync(pin + 1, sync_buf + 2, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  if (kmax > 0) LS_CUDA_TRY(cudaMemcpyAsync(pin + 4, piv, sizeof(int) * kmax, cudaMemcpyDeviceToHost, st));
  LS_CUDA_TRY(cudaStreamSynchronize(st));
  const int k = pin[0], abort_flag = pin[1];  // rank, barrier timeout
  if (pin[2]) {  // index check
    set_last_error_text("ID kernel: pivot index check failed");
    return LS_ECUDA;
  }
  // CPQR work: two projections and a norm (36 p real flops) per active candidate and step
  prof_end(tk, PR_CPQR, st, sizeof(cx<R>) * (double)m * p * 2.0 * k,
           36.0 * p * ((double)m * k - 0.5 * (double)k * k));
  auto release_tsp = [&] {
    if (u_on_aux) {
      ls::StreamScope scope(su);
      ls::dfree(tsp);
    } else {
      ls::dfree(tsp);
    }
  };
  if (abort_flag) {
    ls::dfree(wsp);
    release_tsp();
    return LS_ETIMEOUT;
  }
  if (k < 0 || k > kmax) {
    set_last_error_text("ID kernel returned an invalid rank");
    return LS_ECUDA;
  }
  hp.assign(k > 0 ? k : 1, 0);
  for (int a = 0; a < k; ++a) hp[a] = pin[4 + a];
  if (k > 0 && Uout && !u_on_aux)  // stream-ordered: later users of U run after this copy
    LS_CUDA_TRY(cudaMemcpyAsync(Uout, Ut, sizeof(cx<R>) * (size_t)m * k, cudaMemcpyDeviceToDevice, st));
  ls::dfree(wsp);
  release_tsp();
  for (int a = 0; a < k; ++a)
    if (hp[a] < 0 || hp[a] >= m) {
      set_last_error_text("ID kernel returned an invalid pivot");
      return LS_ECUDA;
    }
  *k_out = k;
  return LS_OK;
}

template <class R>
int compress_t(ls_handle* H, cudaStream_t st, const LevelDone& level_done, cudaStream_t su) {
  const int L = H->L, s = H->s, w = H->ring;
  int rc;
  // with an auxiliary stream the U of a level is finished there; the level is
  // reported done once su has also passed everything issued on st so far
  auto done = [&](int l) -> int {
    if (su) {
      cudaEvent_t e;
      LS_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      LS_CUDA_TRY(cudaEventRecord(e, st));
      LS_CUDA_TRY(cudaStreamWaitEvent(su, e, 0));
      cudaEventDestroy(e);
    }
    {
      char mark[48];
      snprintf(mark, sizeof(mark), "compressed_level_%d", l);
      host_mark(mark);
    }
    if (level_done) level_done(l);
    return LS_OK;
  };
  std::vector<int> rows_x, rows_y;
  int* dint = nullptr;
  for (int l = L; l >= 1; --l) {
    LevelData& lv = H->lev[l];
    rows_x.clear();
    rows_y.clear();
    if (l == L) {
      for (int y = 0; y < s; ++y)
        for (int x = 0; x < s; ++x) {
          rows_x.push_back(x);
          rows_y.push_back(y);
        }
    } else {
      const LevelData& ch = H->lev[l + 1];
      int oax, oay, obx, oby;
      if (l % 2 == 0) {  // vertical cut: alpha left, beta right
        oax = 0; oay = 0; obx = ch.w; oby = 0;
      } else {           // horizontal cut: alpha upper (larger y), beta lower
        oax = 0; oay = ch.h; obx = 0; oby = 0;
      }
      for (size_t i = 0; i < ch.skel_x.size(); ++i) {
        rows_x.push_back(ch.skel_x[i] + oax);
        rows_y.push_back(ch.skel_y[i] + oay);
      }
      for (size_t i = 0; i < ch.skel_x.size(); ++i) {
        rows_x.push_back(ch.skel_x[i] + obx);
        rows_y.push_back(ch.skel_y[i] + oby);
      }
    }
    std::vector<int> px, py;
    for (int y = -w; y < lv.h + w; ++y)
      for (int x = -w; x < lv.w + w; ++x)
        if (x < 0 || x >= lv.w || y < 0 || y >= lv.h) {
          px.push_back(x);
          py.push_back(y);
        }
    const int m = (int)rows_x.size(), p = (int)px.size();
    lv.m = m;
    lv.ring = p;
    if (l <= H->opts.top_uncompressed) {
      // top level kept uncompressed: every row is a skeleton point and U = I
      lv.k = m;
      lv.skel_x = rows_x;
      lv.skel_y = rows_y;
      if ((rc = dalloc(&lv.U, sizeof(cx<R>) * (size_t)m * m))) return rc;
      long long tot = (long long)m * m;
      count_launch();
      identity_kernel<R><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(reinterpret_cast<cx<R>*>(lv.U), m);
      if ((rc = check_launch("identity U"))) return rc;
      if ((rc = done(l))) return rc;
      continue;
    }
    int k = 0;
    std::vector<int> hp;
    cx<R>* A = nullptr;
    if ((rc = dalloc((void**)&A, sizeof(cx<R>) * (size_t)m * p))) return rc;
    if (dint) ls::dfree(dint);
    dint = nullptr;
    if ((rc = dalloc((void**)&dint, sizeof(int) * (2 * m + 2 * p + 8)))) return rc;
    if ((rc = upload_block<R>(rows_x, rows_y, px, py, A, dint, st, H->ks_prec, KernelTable{H->ktab, H->ktx, H->kty}))) return rc;
    if ((rc = dalloc(&lv.U, sizeof(cx<R>) * (size_t)m * std::max(std::min(m, p), 1)))) return rc;
    if ((rc = run_row_id<R>(A, m, p, H->tol, H->nsm, H->sync_buf, st, &k, &hp, reinterpret_cast<cx<R>*>(lv.U), su,
                            H->opts.id_method, true)))
      return rc;
    ls::dfree(A);
    lv.k = k;
    lv.piv.assign(hp.begin(), hp.begin() + k);
    lv.skel_x.resize(k);
    lv.skel_y.resize(k);
    for (int a = 0; a < k; ++a) {
      lv.skel_x[a] = rows_x[hp[a]];
      lv.skel_y[a] = rows_y[hp[a]];
    }
    H->flops_compress += 8.0 * 2.0 * (double)m * p * k;  // two projections per pivot step
    if ((rc = done(l))) return rc;
  }
  if (dint) ls::dfree(dint);
  return LS_OK;
}

}  // namespace

namespace {
template <class Ro, class Ri>
__global__ void convert_kernel(cx<Ro>* out, const cx<Ri>* in, long long n) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < n) out[t] = cvt<Ro>(in[t]);
}
}  // namespace

int row_id(const z64* A, int m, int p, double eps, int precision, int method, int nsm, int* sync_buf,
           cudaStream_t st, int* k, int* piv, z64* U) {
  *k = 0;
  if (m <= 0 || p <= 0) return LS_OK;
  std::vector<int> hp;
  int rc;
  if (precision == LS_FP64) {
    rc = run_row_id<double>(A, m, p, eps, nsm, sync_buf, st, k, &hp, U, nullptr, method, false);
  } else {
    const long long nA = (long long)m * p, nU = (long long)m * std::min(m, p);
    c32* A32 = nullptr;
    c32* U32 = nullptr;
    if ((rc = dalloc((void**)&A32, sizeof(c32) * nA))) return rc;
    if ((rc = dalloc((void**)&U32, sizeof(c32) * nU))) return rc;
    count_launch();
    convert_kernel<float, double><<<(unsigned)((nA + 255) / 256), 256, 0, st>>>(A32, A, nA);
    rc = run_row_id<float>(A32, m, p, eps, nsm, sync_buf, st, k, &hp, U ? U32 : nullptr, nullptr, method, true);
    if (!rc && U && *k > 0) {
      const long long nk = (long long)m * *k;
      count_launch();
      convert_kernel<double, float><<<(unsigned)((nk + 255) / 256), 256, 0, st>>>(U, U32, nk);
      LS_CUDA_TRY(cudaStreamSynchronize(st));
    }
    ls::dfree(A32);
    ls::dfree(U32);
  }
  if (rc) return rc;
  for (int a = 0; a < *k; ++a) piv[a] = hp[a];
  return check_launch("row_id");
}

namespace {
template <class R>
int device_block_t(ls_handle* H, const std::vector<int>& rx, const std::vector<int>& ry, const std::vector<int>& cx_,
                   const std::vector<int>& cy_, void** out, cudaStream_t st) {
  int r;
  if ((r = dalloc(out, sizeof(cx<R>) * std::max<size_t>(rx.size() * cx_.size(), 1)))) return r;
  int* dint = nullptr;
  if ((r = dalloc((void**)&dint, sizeof(int) * (2 * rx.size() + 2 * cx_.size() + 8)))) return r;
  r = upload_block<R>(rx, ry, cx_, cy_, reinterpret_cast<cx<R>*>(*out), dint, st, H->ks_prec,
                      KernelTable{H->ktab, H->ktx, H->kty});
  ls::dfree(dint);
  return r;
}
}  // namespace

// Leaf self-interaction block G(I_tau, I_tau), the same for every leaf.
int leaf_block(ls_handle* H, cudaStream_t st) {
  std::vector<int> lx, ly;
  for (int y = 0; y < H->s; ++y)
    for (int x = 0; x < H->s; ++x) {
      lx.push_back(x);
      ly.push_back(y);
    }
  return H->prec == LS_FP64 ? device_block_t<double>(H, lx, ly, lx, ly, &H->Gleaf, st)
                            : device_block_t<float>(H, lx, ly, lx, ly, &H->Gleaf, st);
}

// Sibling block G(skel_a, skel_b) of the two children on level l (Eq. 15); needs the
// level's skeleton (host), not its compression kernels.
int sibling_block(ls_handle* H, int l, cudaStream_t st) {
  LevelData& lv = H->lev[l];
  if (lv.Gsib) return LS_OK;  // made already (a reused compression)
  const int kk = lv.k;
  int oax, oay, obx, oby;
  if ((l - 1) % 2 == 0) {
    oax = 0; oay = 0; obx = lv.w; oby = 0;
  } else {
    oax = 0; oay = lv.h; obx = 0; oby = 0;
  }
  std::vector<int> ax(kk), ay(kk), bx(kk), by(kk);
  for (int i = 0; i < kk; ++i) {
    ax[i] = lv.skel_x[i] + oax;
    ay[i] = lv.skel_y[i] + oay;
    bx[i] = lv.skel_x[i] + obx;
    by[i] = lv.skel_y[i] + oby;
  }
  return H->prec == LS_FP64 ? device_block_t<double>(H, ax, ay, bx, by, &lv.Gsib, st)
                            : device_block_t<float>(H, ax, ay, bx, by, &lv.Gsib, st);
}

int compress(ls_handle* H, cudaStream_t st, const LevelDone& level_done, cudaStream_t su) {
  return H->prec == LS_FP64 ? compress_t<double>(H, st, level_done, su) : compress_t<float>(H, st, level_done, su);
}

}  // namespace ls
