// Right-preconditioned GMRES on the device (Sec. 5): solve A sigma = f with
// A = I + B (G + T) applied by the FFT convolution and M the HBS inverse, as
// A M y = f, sigma = M y; or the transposed system A^T sigma = f with M^T
// (the adjoint solve of a misfit gradient).  The preconditioned vectors z_j = M v_j are kept
// (flexible form, sigma = sum z_j y_j): an FP32 preconditioner is not exactly
// linear in floating point, and re-applying it to V y at the end would leave
// a residual at its rounding level.  Zero initial guess, no restart, classical
// Gram-Schmidt applied twice, complex Givens rotations
// Q = [[conj(c), conj(s)], [-s, c]].  All vectors and the Hessenberg matrix
// live on the device; the host reads one residual estimate per iteration to
// decide when to stop (gmres_tol or gmres_maxit, Sec. 6.3).  Reductions are
// two-stage with a fixed order, so runs are bitwise reproducible.
#include <algorithm>
#include <vector>

#include "handle.h"
#include "prof.h"

namespace ls {
namespace {

constexpr int kChunks = 256;  // first-stage partial sums per vector

// partial[i][c] = sum over chunk c of conj(V_i[n]) w[n], i < nvec
__global__ void dot_partials_kernel(const z64* __restrict__ V, long long ldv, const z64* __restrict__ w, long long N,
                                    z64* __restrict__ partial) {
  const int c = blockIdx.x, i = blockIdx.y;
  const long long per = (N + gridDim.x - 1) / gridDim.x;
  const long long n0 = c * per, n1 = min(N, n0 + per);
  const z64* v = V + i * ldv;
  z64 acc = mk<double>(0.0, 0.0);
  for (long long n = n0 + threadIdx.x; n < n1; n += blockDim.x) fmac_(acc, v[n], w[n]);
  acc = warp_sum(acc);
  __shared__ z64 red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    z64 v2 = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : mk<double>(0.0, 0.0);
    v2 = warp_sum(v2);
    if (threadIdx.x == 0) partial[(long long)i * gridDim.x + c] = v2;
  }
}

// s_i = sum_c partial[i][c]; out[i] = s_i; if acc: acc[i * ld] += s_i
__global__ void reduce_partials_kernel(const z64* __restrict__ partial, int nchunk, z64* __restrict__ out,
                                       z64* __restrict__ acc, int ld) {
  const int i = blockIdx.x;
  z64 a = mk<double>(0.0, 0.0);
  for (int c = threadIdx.x; c < nchunk; c += blockDim.x) a = a + partial[(long long)i * nchunk + c];
  a = warp_sum(a);
  __shared__ z64 red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    z64 s = mk<double>(0.0, 0.0);
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s = s + red[k];
    out[i] = s;
    if (acc) acc[(long long)i * ld] = acc[(long long)i * ld] + s;
  }
}

// w -= sum_{i<nvec} V_i h_i
__global__ void axpy_multi_kernel(const z64* __restrict__ V, long long ldv, int nvec, const z64* __restrict__ h,
                                  z64* __restrict__ w, long long N) {
  long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= N) return;
  z64 acc = w[n];
  for (int i = 0; i < nvec; ++i) {
    z64 c = h[i], v = V[i * ldv + n];
    acc.re -= v.re * c.re - v.im * c.im;
    acc.im -= v.re * c.im + v.im * c.re;
  }
  w[n] = acc;
}

// v = w / ||w||, with ||w||^2 in nrm2->re; optionally records ||w|| in *hout.
__global__ void normalize_kernel(const z64* __restrict__ w, z64* __restrict__ v, long long N, const z64* nrm2,
                                 z64* hout) {
  long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double nr = sqrt(nrm2->re);
  if (n == 0 && hout) *hout = mk<double>(nr, 0.0);
  if (n >= N) return;
  double s = nr > 0 ? 1.0 / nr : 0.0;
  z64 x = w[n];
  v[n] = mk<double>(x.re * s, x.im * s);
}

struct GmState {
  double fnorm;
  double resid;
  int k;
};

// GMRES start on the device: ||f|| from nrm2->re, residual estimate 1, g = (||f||, 0, ...).
__global__ void gmres_init_kernel(const z64* nrm2, GmState* st, z64* g) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double fnorm = sqrt(nrm2->re);
  st->fnorm = fnorm;
  st->resid = 1.0;
  st->k = 0;
  g[0] = mk<double>(fnorm, 0.0);
}

// Column j of H: apply the earlier rotations, form the new one, update g.
__device__ void givens_step(z64* H, int ldh, z64* cs, z64* sn, z64* g, int j, GmState* st) {
  z64* col = H + j;  // H[i][j] at H[i*ldh + j]
  for (int i = 0; i < j; ++i) {
    z64 a = col[(long long)i * ldh], b = col[(long long)(i + 1) * ldh];
    z64 c = cs[i], s = sn[i];
    z64 top = conjz(c) * a + conjz(s) * b;
    z64 bot = mk<double>(0.0, 0.0) - s * a + c * b;
    col[(long long)i * ldh] = top;
    col[(long long)(i + 1) * ldh] = bot;
  }
  z64 a = col[(long long)j * ldh], b = col[(long long)(j + 1) * ldh];
  double rho = sqrt(abs2(a) + abs2(b));
  z64 c, s;
  if (rho > 0) {
    c = mk<double>(a.re / rho, a.im / rho);
    s = mk<double>(b.re / rho, b.im / rho);
  } else {
    c = mk<double>(1.0, 0.0);
    s = mk<double>(0.0, 0.0);
  }
  cs[j] = c;
  sn[j] = s;
  col[(long long)j * ldh] = mk<double>(rho, 0.0);
  col[(long long)(j + 1) * ldh] = mk<double>(0.0, 0.0);
  z64 gj = g[j];
  g[j + 1] = mk<double>(0.0, 0.0) - s * gj;
  g[j] = conjz(c) * gj;
  st->resid = st->fnorm > 0.0 ? sqrt(abs2(g[j + 1])) / st->fnorm : 0.0;
  st->k = j + 1;
}

__global__ void givens_kernel(z64* H, int ldh, z64* cs, z64* sn, z64* g, int j, GmState* st) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  givens_step(H, ldh, cs, sn, g, j, st);
}

// Block sum in the order of dot_partials_kernel (warp sums, then the warp
// totals by the first warp); the result is valid in thread 0.
__device__ __forceinline__ z64 block_sum_dp(z64 acc, z64* red) {
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  z64 v2 = mk<double>(0.0, 0.0);
  if (threadIdx.x < 32) {
    v2 = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : mk<double>(0.0, 0.0);
    v2 = warp_sum(v2);
  }
  __syncthreads();  // red is reused
  return v2;
}

// One iteration's orthogonalisation in one cooperative launch of kChunks
// blocks (block b owns the entries of chunk b, as in dot_partials_kernel):
// classical Gram-Schmidt twice against V_0..V_j, ||w||, V_{j+1} = w / ||w||,
// and the Givens step in block 0 (the only writer of column j of H).  Warp q of
// a block takes the vectors i = q (mod warps): their dot products over the
// block's chunk, then (after the grid barrier) their sums over all chunks in a
// fixed order (read through L2: other blocks wrote them), so no block barrier
// is needed per vector and runs are bitwise reproducible.  Three grid barriers (bounded waits: a block that gives up
// sets *err = LS_ETIMEOUT).  Dynamic shared memory: (j + 1) coefficients.
__global__ void __launch_bounds__(256) gmres_orth_kernel(const z64* __restrict__ V, long long ldv, int j, z64* w,
                                                         long long N, z64* Hm, int ldh, z64* part0, z64* part1,
                                                         z64* cs, z64* sn, z64* g, GmState* st, GridSync gs,
                                                         unsigned epoch0, int* err) {
  extern __shared__ z64 hc[];
  __shared__ z64 red[32];
  __shared__ z64 bc;
  const int b = blockIdx.x, G = gridDim.x, nvec = j + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const long long per = (N + G - 1) / G;
  const long long n0 = b * per, n1 = min(N, n0 + per);
  unsigned epoch = epoch0;
  for (int pass = 0; pass < 2; ++pass) {
    z64* part = pass ? part1 : part0;
    for (int i = warp; i < nvec; i += nw) {
      const z64* v = V + i * ldv;
      z64 acc = mk<double>(0.0, 0.0);
      for (long long n = n0 + lane; n < n1; n += 32) fmac_(acc, v[n], w[n]);
      acc = warp_sum(acc);
      if (lane == 0) part[(long long)i * G + b] = acc;
    }
    if (!grid_sync(gs, G, epoch)) {
      if (threadIdx.x == 0) atomicExch(err, LS_ETIMEOUT);
      return;
    }
    for (int i = warp; i < nvec; i += nw) {
      z64 a = mk<double>(0.0, 0.0);
      for (int c = lane; c < G; c += 32) a = a + ldcg_cx(part + (long long)i * G + c);
      a = warp_sum(a);
      if (lane == 0) {
        hc[i] = a;
        if (b == 0) Hm[(long long)i * ldh + j] = Hm[(long long)i * ldh + j] + a;
      }
    }
    __syncthreads();
    for (long long n = n0 + threadIdx.x; n < n1; n += blockDim.x) {
      z64 acc = w[n];
      for (int i = 0; i < nvec; ++i) {
        const z64 c = hc[i], v = V[i * ldv + n];
        acc.re -= v.re * c.re - v.im * c.im;
        acc.im -= v.re * c.im + v.im * c.re;
      }
      w[n] = acc;
    }
    __syncthreads();
  }
  // ||w||^2: part0 is free again (every block read it before the second barrier)
  {
    z64 acc = mk<double>(0.0, 0.0);
    for (long long n = n0 + threadIdx.x; n < n1; n += blockDim.x) fmac_(acc, w[n], w[n]);
    const z64 t = block_sum_dp(acc, red);
    if (threadIdx.x == 0) part0[b] = t;
  }
  if (!grid_sync(gs, G, epoch)) {
    if (threadIdx.x == 0) atomicExch(err, LS_ETIMEOUT);
    return;
  }
  if (warp == 0) {
    z64 a = mk<double>(0.0, 0.0);
    for (int c = lane; c < G; c += 32) a = a + ldcg_cx(part0 + c);
    a = warp_sum(a);
    if (lane == 0) bc = a;
  }
  __syncthreads();
  const double nr = sqrt(bc.re);
  const double sc = nr > 0 ? 1.0 / nr : 0.0;
  z64* vn = const_cast<z64*>(V) + (long long)(j + 1) * ldv;
  for (long long n = n0 + threadIdx.x; n < n1; n += blockDim.x) {
    const z64 x = w[n];
    vn[n] = mk<double>(x.re * sc, x.im * sc);
  }
  if (b == 0 && threadIdx.x == 0) {
    Hm[(long long)(j + 1) * ldh + j] = mk<double>(nr, 0.0);
    givens_step(Hm, ldh, cs, sn, g, j, st);
  }
}

// Back substitution H(0:k,0:k) y = g(0:k), one thread (k <= maxit).
__global__ void backsolve_kernel(const z64* H, int ldh, const z64* g, z64* y, int k) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    z64 s = g[i];
    for (int c = i + 1; c < k; ++c) s = s - H[(long long)i * ldh + c] * y[c];
    y[i] = s * inv(H[(long long)i * ldh + i]);
  }
}

// x = sum_i V_i y_i
__global__ void combine_kernel(const z64* __restrict__ V, long long ldv, int k, const z64* __restrict__ y,
                               z64* __restrict__ x, long long N) {
  long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= N) return;
  z64 acc = mk<double>(0.0, 0.0);
  for (int i = 0; i < k; ++i) fma_(acc, V[i * ldv + n], y[i]);
  x[n] = acc;
}

__global__ void sub_kernel(const z64* a, const z64* b, z64* c, long long N) {
  long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n < N) c[n] = a[n] - b[n];
}

struct Ws {
  z64 *V, *Z, *w, *z, *Hm, *cs, *sn, *g, *y, *partial, *partial1, *scal;
  GmState* st;
  unsigned* sync;  // grid barrier of gmres_orth_kernel: arrival count, abort flag
};

Ws carve(ls_handle* H, long long N, int m) {
  Ws ws;
  char* p = reinterpret_cast<char*>(H->gm);
  auto take = [&](size_t bytes) {
    char* r = p;
    p += (bytes + 255) & ~(size_t)255;
    return r;
  };
  ws.V = reinterpret_cast<z64*>(take(sizeof(z64) * N * (m + 1)));
  ws.Z = reinterpret_cast<z64*>(take(sizeof(z64) * N * m));
  ws.w = reinterpret_cast<z64*>(take(sizeof(z64) * N));
  ws.z = reinterpret_cast<z64*>(take(sizeof(z64) * N));
  ws.Hm = reinterpret_cast<z64*>(take(sizeof(z64) * (m + 1) * m));
  ws.cs = reinterpret_cast<z64*>(take(sizeof(z64) * m));
  ws.sn = reinterpret_cast<z64*>(take(sizeof(z64) * m));
  ws.g = reinterpret_cast<z64*>(take(sizeof(z64) * (m + 1)));
  ws.y = reinterpret_cast<z64*>(take(sizeof(z64) * (m + 1)));
  ws.partial = reinterpret_cast<z64*>(take(sizeof(z64) * kChunks * (m + 1)));
  ws.partial1 = reinterpret_cast<z64*>(take(sizeof(z64) * kChunks * (m + 1)));
  ws.scal = reinterpret_cast<z64*>(take(sizeof(z64) * 8));
  ws.st = reinterpret_cast<GmState*>(take(sizeof(GmState)));
  ws.sync = reinterpret_cast<unsigned*>(take(4 * sizeof(unsigned)));
  return ws;
}

size_t ws_bytes(long long N, int m) {
  size_t b = 0;
  auto add = [&](size_t x) { b += (x + 255) & ~(size_t)255; };
  add(sizeof(z64) * N * (m + 1));
  add(sizeof(z64) * N * m);
  add(sizeof(z64) * N);
  add(sizeof(z64) * N);
  add(sizeof(z64) * (m + 1) * m);
  add(sizeof(z64) * m);
  add(sizeof(z64) * m);
  add(sizeof(z64) * (m + 1));
  add(sizeof(z64) * (m + 1));
  add(sizeof(z64) * kChunks * (m + 1));
  add(sizeof(z64) * kChunks * (m + 1));
  add(sizeof(z64) * 8);
  add(sizeof(GmState));
  add(4 * sizeof(unsigned));
  return b;
}

// ||x||^2 into out->re (deterministic two-stage reduction)
void norm2(const z64* x, long long N, z64* partial, z64* out, cudaStream_t st) {
  count_launch();
  dot_partials_kernel<<<dim3(kChunks, 1), 256, 0, st>>>(x, 0, x, N, partial);
  count_launch();
  reduce_partials_kernel<<<1, 256, 0, st>>>(partial, kChunks, out, nullptr, 0);
}

int solve_one(ls_handle* H, const z64* f, z64* sigma, ls_solve_info* info, int transpose, cudaStream_t st) {
  const int mode = transpose ? CONV_TRANSPOSE : CONV_FORWARD;
  const long long N = (long long)H->grid.nx * H->grid.ny;
  const int m = H->opts.gmres_maxit;
  Ws ws = carve(H, N, m);
  const unsigned nb = (unsigned)((N + 255) / 256);
  int rc;
  LS_CUDA_TRY(cudaMemsetAsync(ws.Hm, 0, sizeof(z64) * (m + 1) * m, st));
  LS_CUDA_TRY(cudaMemsetAsync(ws.g, 0, sizeof(z64) * (m + 1), st));
  // the orthogonalisation as one cooperative launch per iteration when its
  // kChunks blocks can all be resident (else the separate kernels)
  bool fused = false;
  {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gmres_orth_kernel, 256,
                                                      sizeof(z64) * (size_t)(m + 1)) == cudaSuccess)
      fused = (long long)per_sm * H->nsm >= kChunks;
    cudaGetLastError();
  }
  if (fused) LS_CUDA_TRY(cudaMemsetAsync(ws.sync, 0, 4 * sizeof(unsigned), st));
  unsigned orth_epoch = 0;  // grid barriers passed so far (three per launch)
  norm2(f, N, ws.partial, ws.scal, st);
  // small host<->device transfers go through page-locked scratch
  unsigned char* pin = static_cast<unsigned char*>(pinned_scratch(256));
  if (!pin) return LS_ENOMEM;
  static_assert(sizeof(GmState) + sizeof(z64) <= 256, "pinned scratch too small");
  // ||f|| stays on the device (state and g_0 set there, v_0 = f / ||f||, zero for
  // f = 0); the host learns it with the first iteration's state
  count_launch();
  gmres_init_kernel<<<1, 32, 0, st>>>(ws.scal, ws.st, ws.g);
  count_launch();
  normalize_kernel<<<nb, 256, 0, st>>>(f, ws.V, N, ws.scal, nullptr);
  GmState* hs = reinterpret_cast<GmState*>(pin);
  double fnorm = 0.0;
  ls_solve_info inf;
  inf.iterations = 0;
  inf.converged = 1;
  inf.resid_est = 0.0;
  inf.resid_true = 0.0;
  int k = 0;
  double resid = 1.0;
  const double tol = H->opts.gmres_tol;
  for (int j = 0; j < m; ++j) {
    z64* vj = ws.V + (long long)j * N;
    z64* zj = ws.Z + (long long)j * N;
    if ((rc = hbs_apply(H, vj, zj, 1, transpose, st))) return rc;
    if ((rc = conv_apply(H, zj, ws.w, 1, mode, st))) return rc;
    int tk = prof_begin(st);
    if (fused) {
      const z64* Vc = ws.V;
      z64* wv = ws.w;
      long long ldv = N, Nn = N;
      int jj = j, ldh = m;
      GridSync gs{ws.sync, ws.sync + 1, reinterpret_cast<int*>(ws.sync + 2), H->spin_limit};
      unsigned e0 = orth_epoch;
      int* err = H->d_err;
      void* args[] = {&Vc, &ldv, &jj, &wv, &Nn, &ws.Hm, &ldh, &ws.partial, &ws.partial1, &ws.cs, &ws.sn, &ws.g, &ws.st,
                      &gs, &e0, &err};
      count_launch();
      LS_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)gmres_orth_kernel, dim3(kChunks), dim3(256), args,
                                              sizeof(z64) * (size_t)(j + 1), st));
      orth_epoch += 3;
    } else {
      for (int pass = 0; pass < 2; ++pass) {  // classical Gram-Schmidt, twice
        count_launch();
        dot_partials_kernel<<<dim3(kChunks, j + 1), 256, 0, st>>>(ws.V, N, ws.w, N, ws.partial);
        count_launch();
        reduce_partials_kernel<<<j + 1, 256, 0, st>>>(ws.partial, kChunks, ws.y, ws.Hm + j, m);
        count_launch();
        axpy_multi_kernel<<<nb, 256, 0, st>>>(ws.V, N, j + 1, ws.y, ws.w, N);
      }
      norm2(ws.w, N, ws.partial, ws.scal, st);
      count_launch();
      normalize_kernel<<<nb, 256, 0, st>>>(ws.w, ws.V + (long long)(j + 1) * N, N, ws.scal,
                                           ws.Hm + (long long)(j + 1) * m + j);
      count_launch();
      givens_kernel<<<1, 32, 0, st>>>(ws.Hm, m, ws.cs, ws.sn, ws.g, j, ws.st);
    }
    // CGS2: per pass j+1 dot products and j+1 axpys over N complex entries, plus the norm
    prof_end(tk, PR_GMRES_ORTH, st, 16.0 * N * (2.0 * (2.0 * (j + 1) + 2.0) + 3.0),
             8.0 * N * (4.0 * (j + 1) + 1.0));
    if ((rc = check_launch("gmres iteration"))) return rc;
    LS_CUDA_TRY(cudaMemcpyAsync(hs, ws.st, sizeof(GmState), cudaMemcpyDeviceToHost, st));
    LS_CUDA_TRY(cudaStreamSynchronize(st));
    if (j == 0) {
      fnorm = hs->fnorm;
      if (fnorm == 0.0) {  // f = 0: sigma = 0 (the iteration ran on zero vectors)
        LS_CUDA_TRY(cudaMemsetAsync(sigma, 0, sizeof(z64) * N, st));
        int* derr = reinterpret_cast<int*>(pin + 192);  // status of that iteration's apply
        LS_CUDA_TRY(cudaMemcpyAsync(derr, H->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
        LS_CUDA_TRY(cudaStreamSynchronize(st));
        if (*derr) return *derr;
        if (info) *info = inf;
        return LS_OK;
      }
    }
    k = j + 1;
    resid = hs->resid;
    if (resid <= tol) break;
  }
  count_launch();
  backsolve_kernel<<<1, 32, 0, st>>>(ws.Hm, m, ws.g, ws.y, k);
  count_launch();
  combine_kernel<<<nb, 256, 0, st>>>(ws.Z, N, k, ws.y, sigma, N);
  // true residual ||f - A sigma|| / ||f||
  if ((rc = conv_apply(H, sigma, ws.w, 1, mode, st))) return rc;
  count_launch();
  sub_kernel<<<nb, 256, 0, st>>>(f, ws.w, ws.w, N);
  norm2(ws.w, N, ws.partial, ws.scal, st);
  z64* rn2 = reinterpret_cast<z64*>(pin + 128);
  int* derr = reinterpret_cast<int*>(pin + 192);  // status of the preconditioner applies
  LS_CUDA_TRY(cudaMemcpyAsync(rn2, ws.scal, sizeof(z64), cudaMemcpyDeviceToHost, st));
  LS_CUDA_TRY(cudaMemcpyAsync(derr, H->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  LS_CUDA_TRY(cudaStreamSynchronize(st));
  if (*derr) return *derr;
  if ((rc = check_launch("gmres finish"))) return rc;
  inf.iterations = k;
  inf.resid_est = resid;
  inf.resid_true = sqrt(rn2->re) / fnorm;
  inf.converged = resid <= tol;
  if (info) *info = inf;
  return inf.converged ? LS_OK : LS_ENOCONV;
}


// ------------------------------------------------- block GMRES
// nb right-hand sides, each with its own Krylov space: the one-vector solver's
// arithmetic (flexible right preconditioning, CGS2, complex Givens rotations,
// zero initial guess, no restart) run side by side.  Each iteration applies the
// preconditioner and the operator to the nb current vectors at once
// (hbs_apply, conv_apply with nrhs = nb), so every factor and the kernel
// spectrum are read once per iteration for the block.  On a handle of several
// problems the block holds whole sets of them, right-hand side r belonging to
// problem r mod nprob (its own potential in the matvec, its own tree in the
// apply).  A right-hand side whose
// residual estimate reaches the tolerance is frozen (its later vectors are
// zero, its kernels return early); the block stops when all are frozen or at
// gmres_maxit.  Vectors: one slab of nb grid vectors per Krylov vector V_j and
// per preconditioned vector Z_j, allocated as the iterations reach them; the
// kernels find them through device tables of slab pointers.  Right-hand side r
// is split into C chunks (block (c, r) of every grid); reductions run in a
// fixed order, so results are reproducible.

constexpr int kVG = 4;  // Krylov vectors per pass of the dot-product kernel

struct BState {
  double fnorm;
  double resid;
  int k;     // iterations taken (columns of H in use)
  int done;  // frozen
};

__device__ __forceinline__ void chunk_of(long long N, int C, int c, long long& n0, long long& n1) {
  const long long per = (N + C - 1) / C;
  n0 = c * per;
  n1 = min(N, n0 + per);
}

// block sum of a complex value over 256 threads in a fixed order; valid in thread 0
__device__ __forceinline__ z64 block_sum256(z64 a, z64* red) {
  a = warp_sum(a);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  z64 s = mk<double>(0.0, 0.0);
  if (threadIdx.x == 0)
    for (int w = 0; w < 8; ++w) s = s + red[w];
  __syncthreads();
  return s;
}

// nrm[r * C + c] = ||x_r||^2 over chunk c
__global__ void __launch_bounds__(256) bnorm_kernel(const z64* __restrict__ x, long long N, int C, z64* __restrict__ nrm) {
  __shared__ z64 red[8];
  const int c = blockIdx.x, r = blockIdx.y;
  long long n0, n1;
  chunk_of(N, C, c, n0, n1);
  const z64* xr = x + r * N;
  z64 acc = mk<double>(0.0, 0.0);
  for (long long n = n0 + threadIdx.x; n < n1; n += 256) fmac_(acc, xr[n], xr[n]);
  const z64 s = block_sum256(acc, red);
  if (threadIdx.x == 0) nrm[(long long)r * C + c] = s;
}

// ||f_r|| from the partials, state and g_r = (||f_r||, 0, ...); f_r = 0 is frozen at k = 0
__global__ void binit_kernel(const z64* __restrict__ nrm, int C, BState* st, z64* g, int ldg) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= gridDim.x * blockDim.x) return;
  double s = 0.0;
  for (int c = 0; c < C; ++c) s += nrm[(long long)r * C + c].re;
  const double fn = sqrt(s);
  st[r].fnorm = fn;
  st[r].resid = fn > 0.0 ? 1.0 : 0.0;
  st[r].k = 0;
  st[r].done = fn > 0.0 ? 0 : 1;
  g[(long long)r * ldg] = mk<double>(fn, 0.0);
}

// V_0[r] = f_r / ||f_r|| (zero for f_r = 0)
__global__ void __launch_bounds__(256) bscale_kernel(const z64* __restrict__ f, z64* __restrict__ v, long long N, int C,
                                                     const BState* __restrict__ st) {
  const int c = blockIdx.x, r = blockIdx.y;
  long long n0, n1;
  chunk_of(N, C, c, n0, n1);
  const double fn = st[r].fnorm, s = fn > 0.0 ? 1.0 / fn : 0.0;
  for (long long n = n0 + threadIdx.x; n < n1; n += 256) {
    const z64 x = f[r * N + n];
    v[r * N + n] = mk<double>(x.re * s, x.im * s);
  }
}

// part[(r * ldp + i) * C + c] = sum over chunk c of conj(V_i[r]) w_r, i <= j
__global__ void __launch_bounds__(256) bdots_kernel(const z64* const* __restrict__ Vt, int j, const z64* __restrict__ w,
                                                    long long N, int C, int ldp, z64* __restrict__ part,
                                                    const BState* __restrict__ st) {
  __shared__ z64 red[kVG][8];
  const int c = blockIdx.x, r = blockIdx.y;
  if (st[r].done) return;
  long long n0, n1;
  chunk_of(N, C, c, n0, n1);
  const z64* wr = w + r * N;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i0 = 0; i0 <= j; i0 += kVG) {
    const int ng = min(kVG, j + 1 - i0);
    const z64* v[kVG];
#pragma unroll
    for (int q = 0; q < kVG; ++q) v[q] = (q < ng ? Vt[i0 + q] : Vt[i0]) + r * N;
    z64 acc[kVG];
#pragma unroll
    for (int q = 0; q < kVG; ++q) acc[q] = mk<double>(0.0, 0.0);
    for (long long n = n0 + threadIdx.x; n < n1; n += 256) {
      const z64 x = wr[n];
#pragma unroll
      for (int q = 0; q < kVG; ++q)
        if (q < ng) fmac_(acc[q], v[q][n], x);
    }
#pragma unroll
    for (int q = 0; q < kVG; ++q) {
      const z64 a = warp_sum(acc[q]);
      if (lane == 0) red[q][warp] = a;
    }
    __syncthreads();
    if (threadIdx.x < ng) {
      z64 s = mk<double>(0.0, 0.0);
      for (int w2 = 0; w2 < 8; ++w2) s = s + red[threadIdx.x][w2];
      part[((long long)r * ldp + i0 + threadIdx.x) * C + c] = s;
    }
    __syncthreads();
  }
}

// h_i = sum_c part[r][i][c] (fixed order; block c = 0 adds it to column j of H_r),
// then w_r -= sum_i V_i[r] h_i on chunk c; with nrm, the chunk's ||w_r||^2 -> nrm[r * C + c]
__global__ void __launch_bounds__(256) bupdate_kernel(const z64* const* __restrict__ Vt, int j, z64* __restrict__ w,
                                                      long long N, int C, int ldp, const z64* __restrict__ part,
                                                      z64* __restrict__ Hm, int m, z64* __restrict__ nrm,
                                                      const BState* __restrict__ st) {
  extern __shared__ z64 h[];  // j + 1
  __shared__ z64 red[8];
  const int c = blockIdx.x, r = blockIdx.y;
  if (st[r].done) return;
  for (int i = threadIdx.x; i <= j; i += 256) {
    z64 s = mk<double>(0.0, 0.0);
    for (int cc = 0; cc < C; ++cc) s = s + part[((long long)r * ldp + i) * C + cc];
    h[i] = s;
    if (c == 0) {
      z64* e = Hm + (long long)r * (m + 1) * m + (long long)i * m + j;
      *e = *e + s;
    }
  }
  __syncthreads();
  long long n0, n1;
  chunk_of(N, C, c, n0, n1);
  z64* wr = w + r * N;
  z64 acc = mk<double>(0.0, 0.0);
  for (long long n = n0 + threadIdx.x; n < n1; n += 256) {
    z64 x = wr[n];
    for (int i = 0; i <= j; ++i) {
      const z64 a = h[i], v = Vt[i][r * N + n];
      x.re -= v.re * a.re - v.im * a.im;
      x.im -= v.re * a.im + v.im * a.re;
    }
    wr[n] = x;
    fmac_(acc, x, x);
  }
  if (nrm) {
    const z64 s = block_sum256(acc, red);
    if (threadIdx.x == 0) nrm[(long long)r * C + c] = s;
  }
}

// ||w_r|| from the partials into H_r(j+1, j), the Givens step of column j, and the
// freeze decision (residual estimate <= tol); one thread per right-hand side.
__global__ void bgivens_kernel(const z64* __restrict__ nrm, int C, z64* Hm, int m, z64* cs, z64* sn, z64* g, BState* st,
                               int j, double tol, int nb) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nb || st[r].done) return;
  double s = 0.0;
  for (int c = 0; c < C; ++c) s += nrm[(long long)r * C + c].re;
  z64* H = Hm + (long long)r * (m + 1) * m;
  H[(long long)(j + 1) * m + j] = mk<double>(sqrt(s), 0.0);
  GmState gs{st[r].fnorm, st[r].resid, st[r].k};
  givens_step(H, m, cs + (long long)r * m, sn + (long long)r * m, g + (long long)r * (m + 1), j, &gs);
  st[r].resid = gs.resid;
  st[r].k = gs.k;
  if (gs.resid <= tol) st[r].done = 1;
}

// V_{j+1}[r] = w_r / ||w_r|| (the norm summed from the partials in the order of
// bgivens_kernel: the Givens step has already rotated H_r(j+1, j) to zero);
// zero for a frozen right-hand side
__global__ void __launch_bounds__(256) bnormalize_kernel(const z64* __restrict__ w, z64* __restrict__ vn, long long N,
                                                         int C, const z64* __restrict__ nrm,
                                                         const BState* __restrict__ st) {
  __shared__ double nr_s;
  const int c = blockIdx.x, r = blockIdx.y;
  long long n0, n1;
  chunk_of(N, C, c, n0, n1);
  if (threadIdx.x == 0) {
    double s2 = 0.0;
    for (int cc = 0; cc < C; ++cc) s2 += nrm[(long long)r * C + cc].re;
    nr_s = sqrt(s2);
  }
  __syncthreads();
  const double nr = nr_s;
  const double s = (!st[r].done && nr > 0.0) ? 1.0 / nr : 0.0;
  for (long long n = n0 + threadIdx.x; n < n1; n += 256) {
    const z64 x = w[r * N + n];
    vn[r * N + n] = mk<double>(x.re * s, x.im * s);
  }
}

// y_r = H_r(0:k, 0:k)^-1 g_r(0:k), k = the right-hand side's iterations
__global__ void bbacksolve_kernel(const z64* Hm, int m, const z64* g, z64* y, const BState* st, int nb) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nb) return;
  const z64* H = Hm + (long long)r * (m + 1) * m;
  const z64* gr = g + (long long)r * (m + 1);
  z64* yr = y + (long long)r * (m + 1);
  const int k = st[r].k;
  for (int i = k - 1; i >= 0; --i) {
    z64 s = gr[i];
    for (int c = i + 1; c < k; ++c) s = s - H[(long long)i * m + c] * yr[c];
    yr[i] = s * inv(H[(long long)i * m + i]);
  }
}

// sigma_r = sum_{i < k_r} Z_i[r] y_r[i]
__global__ void __launch_bounds__(256) bcombine_kernel(const z64* const* __restrict__ Zt, const z64* __restrict__ y,
                                                       int m, z64* __restrict__ sigma, long long N, int C,
                                                       const BState* __restrict__ st) {
  const int c = blockIdx.x, r = blockIdx.y, k = st[r].k;
  long long n0, n1;
  chunk_of(N, C, c, n0, n1);
  const z64* yr = y + (long long)r * (m + 1);
  for (long long n = n0 + threadIdx.x; n < n1; n += 256) {
    z64 acc = mk<double>(0.0, 0.0);
    for (int i = 0; i < k; ++i) fma_(acc, Zt[i][r * N + n], yr[i]);
    sigma[r * N + n] = acc;
  }
}

// w = f - w and its chunk norms
__global__ void __launch_bounds__(256) bresid_kernel(const z64* __restrict__ f, z64* __restrict__ w, long long N, int C,
                                                     z64* __restrict__ nrm) {
  __shared__ z64 red[8];
  const int c = blockIdx.x, r = blockIdx.y;
  long long n0, n1;
  chunk_of(N, C, c, n0, n1);
  z64 acc = mk<double>(0.0, 0.0);
  for (long long n = n0 + threadIdx.x; n < n1; n += 256) {
    const z64 d = f[r * N + n] - w[r * N + n];
    w[r * N + n] = d;
    fmac_(acc, d, d);
  }
  const z64 s = block_sum256(acc, red);
  if (threadIdx.x == 0) nrm[(long long)r * C + c] = s;
}

// out[r] = sum_c nrm[r * C + c] (real part), fixed order
__global__ void bsum_kernel(const z64* __restrict__ nrm, int C, double* __restrict__ out, int nb) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nb) return;
  double s = 0.0;
  for (int c = 0; c < C; ++c) s += nrm[(long long)r * C + c].re;
  out[r] = s;
}

int solve_block(ls_handle* H, const z64* f, z64* sigma, int nb, ls_solve_info* info, int transpose, cudaStream_t st) {
  const int mode = transpose ? CONV_TRANSPOSE : CONV_FORWARD;
  const long long N = (long long)H->grid.nx * H->grid.ny;
  const int m = H->opts.gmres_maxit;
  // chunks per right-hand side: about eight blocks per SM over the block, at least 256 entries each
  const int C = (int)std::max(1LL, std::min({(long long)kChunks, (8LL * H->nsm + nb - 1) / nb, (N + 255) / 256}));
  const int ldp = m + 1;
  // small state: H, cs, sn, g, y, dot partials, norm partials, states, slab tables, residual norms
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  const size_t oH = take(sizeof(z64) * nb * (size_t)(m + 1) * m), ocs = take(sizeof(z64) * nb * (size_t)m),
               osn = take(sizeof(z64) * nb * (size_t)m), og = take(sizeof(z64) * nb * (size_t)(m + 1)),
               oy = take(sizeof(z64) * nb * (size_t)(m + 1)), op = take(sizeof(z64) * nb * (size_t)ldp * C),
               onr = take(sizeof(z64) * nb * (size_t)C), ost = take(sizeof(BState) * nb),
               oVt = take(sizeof(z64*) * (size_t)(m + 1)), oZt = take(sizeof(z64*) * (size_t)m),
               orn = take(sizeof(double) * nb), ow = take(sizeof(z64) * nb * (size_t)N);
  int rc;
  if (H->bgm_bytes < off) {
    if (H->bgm) dfree(H->bgm);
    H->bgm = nullptr;
    H->bgm_bytes = 0;
    if ((rc = dalloc(&H->bgm, off))) return rc;
    H->bgm_bytes = off;
  }
  char* base = static_cast<char*>(H->bgm);
  z64* Hm = reinterpret_cast<z64*>(base + oH);
  z64* cs = reinterpret_cast<z64*>(base + ocs);
  z64* sn = reinterpret_cast<z64*>(base + osn);
  z64* g = reinterpret_cast<z64*>(base + og);
  z64* y = reinterpret_cast<z64*>(base + oy);
  z64* part = reinterpret_cast<z64*>(base + op);
  z64* nrm = reinterpret_cast<z64*>(base + onr);
  BState* bst = reinterpret_cast<BState*>(base + ost);
  z64** Vt = reinterpret_cast<z64**>(base + oVt);
  z64** Zt = reinterpret_cast<z64**>(base + oZt);
  double* rn = reinterpret_cast<double*>(base + orn);
  z64* w = reinterpret_cast<z64*>(base + ow);
  // slabs of nb vectors: V_i at bslab[2 i], Z_i at bslab[2 i + 1]
  const size_t slab = sizeof(z64) * (size_t)nb * N;
  if (H->bslab_bytes < slab) {
    for (void* p : H->bslab) dfree(p);
    H->bslab.clear();
    H->bslab_bytes = slab;
  }
  // pinned host scratch: the slab tables, the states, the residual norms
  const size_t pin_tab = sizeof(z64*) * (size_t)(2 * m + 2), pin_st = sizeof(BState) * nb;
  unsigned char* pin = static_cast<unsigned char*>(pinned_scratch(pin_tab + pin_st + sizeof(double) * nb + 64));
  if (!pin) return LS_ENOMEM;
  z64** hVt = reinterpret_cast<z64**>(pin);
  z64** hZt = hVt + (m + 1);
  BState* hst = reinterpret_cast<BState*>(pin + pin_tab);
  double* hrn = reinterpret_cast<double*>(pin + pin_tab + pin_st);
  int* derr = reinterpret_cast<int*>(pin + pin_tab + pin_st + sizeof(double) * nb);
  auto slab_at = [&](int idx, z64** out) -> int {
    while ((int)H->bslab.size() <= idx) {
      void* p = nullptr;
      int rc2 = dalloc(&p, slab);
      if (rc2) return rc2;
      H->bslab.push_back(p);
    }
    *out = static_cast<z64*>(H->bslab[idx]);
    return LS_OK;
  };
  auto table = [&](z64** dtab, z64** htab, int i, z64* p) -> int {  // one entry, copied from pinned memory
    htab[i] = p;
    LS_CUDA_TRY(cudaMemcpyAsync(dtab + i, htab + i, sizeof(z64*), cudaMemcpyHostToDevice, st));
    return LS_OK;
  };
  const dim3 grid(C, nb), g1((nb + 127) / 128);
  LS_CUDA_TRY(cudaMemsetAsync(Hm, 0, sizeof(z64) * nb * (size_t)(m + 1) * m, st));
  LS_CUDA_TRY(cudaMemsetAsync(g, 0, sizeof(z64) * nb * (size_t)(m + 1), st));
  z64* V0;
  if ((rc = slab_at(0, &V0)) || (rc = table(Vt, hVt, 0, V0))) return rc;
  count_launch();
  bnorm_kernel<<<grid, 256, 0, st>>>(f, N, C, nrm);
  count_launch();
  binit_kernel<<<nb, 1, 0, st>>>(nrm, C, bst, g, m + 1);
  count_launch();
  bscale_kernel<<<grid, 256, 0, st>>>(f, V0, N, C, bst);
  int k_all = 0;
  for (int j = 0; j < m; ++j) {
    z64 *Vj = hVt[j], *Zj, *Vn;
    if ((rc = slab_at(2 * j + 1, &Zj)) || (rc = table(Zt, hZt, j, Zj))) return rc;
    if ((rc = slab_at(2 * j + 2, &Vn)) || (rc = table(Vt, hVt, j + 1, Vn))) return rc;
    if ((rc = hbs_apply(H, Vj, Zj, nb, transpose, st))) return rc;
    if ((rc = conv_apply(H, Zj, w, nb, mode, st))) return rc;
    const int tk = prof_begin(st);
    const z64* const* Vc = Vt;
    for (int pass = 0; pass < 2; ++pass) {  // classical Gram-Schmidt, twice
      count_launch();
      bdots_kernel<<<grid, 256, 0, st>>>(Vc, j, w, N, C, ldp, part, bst);
      count_launch();
      bupdate_kernel<<<grid, 256, sizeof(z64) * (size_t)(j + 1), st>>>(Vc, j, w, N, C, ldp, part, Hm, m,
                                                                       pass ? nrm : nullptr, bst);
    }
    count_launch();
    bgivens_kernel<<<g1, 128, 0, st>>>(nrm, C, Hm, m, cs, sn, g, bst, j, H->opts.gmres_tol, nb);
    count_launch();
    bnormalize_kernel<<<grid, 256, 0, st>>>(w, Vn, N, C, nrm, bst);
    prof_end(tk, PR_GMRES_BLOCK, st, 16.0 * N * nb * (4.0 * (j + 1) + 5.0), 16.0 * N * nb * (4.0 * (j + 1) + 1.0));
    if ((rc = check_launch("block gmres iteration"))) return rc;
    LS_CUDA_TRY(cudaMemcpyAsync(hst, bst, sizeof(BState) * nb, cudaMemcpyDeviceToHost, st));
    LS_CUDA_TRY(cudaStreamSynchronize(st));
    k_all = j + 1;
    bool all = true;
    for (int r = 0; r < nb; ++r) all = all && hst[r].done;
    if (all) break;
  }
  (void)k_all;
  count_launch();
  bbacksolve_kernel<<<g1, 128, 0, st>>>(Hm, m, g, y, bst, nb);
  count_launch();
  bcombine_kernel<<<grid, 256, 0, st>>>(Zt, y, m, sigma, N, C, bst);
  // true residuals ||f_r - A sigma_r|| / ||f_r||
  if ((rc = conv_apply(H, sigma, w, nb, mode, st))) return rc;
  count_launch();
  bresid_kernel<<<grid, 256, 0, st>>>(f, w, N, C, nrm);
  count_launch();
  bsum_kernel<<<g1, 128, 0, st>>>(nrm, C, rn, nb);
  LS_CUDA_TRY(cudaMemcpyAsync(hrn, rn, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
  LS_CUDA_TRY(cudaMemcpyAsync(hst, bst, sizeof(BState) * nb, cudaMemcpyDeviceToHost, st));
  LS_CUDA_TRY(cudaMemcpyAsync(derr, H->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  LS_CUDA_TRY(cudaStreamSynchronize(st));
  if (*derr) return *derr;
  if ((rc = check_launch("block gmres finish"))) return rc;
  int worst = LS_OK;
  for (int r = 0; r < nb; ++r) {
    ls_solve_info inf;
    const double fn = hst[r].fnorm;
    inf.iterations = hst[r].k;
    inf.resid_est = fn > 0.0 ? hst[r].resid : 0.0;
    inf.resid_true = fn > 0.0 ? sqrt(hrn[r]) / fn : 0.0;
    inf.converged = fn > 0.0 ? hst[r].resid <= H->opts.gmres_tol : 1;
    if (!inf.converged) worst = LS_ENOCONV;
    if (info) info[r] = inf;
  }
  return worst;
}
}  // namespace

int gmres_solve(ls_handle* H, const z64* f, z64* sigma, int nrhs, ls_solve_info* info, int transpose,
                cudaStream_t st) {
  const long long N = (long long)H->grid.nx * H->grid.ny;
  const int m = H->opts.gmres_maxit;
  size_t need = ws_bytes(N, m);
  if (!H->gm || H->gm_bytes < need) {
    if (H->gm) ls::dfree(H->gm);
    H->gm = nullptr;
    int rc = dalloc(&H->gm, need);
    if (rc) return rc;
    H->gm_bytes = need;
  }
  host_mark("gmres_workspace");
  int worst = LS_OK;
  // blocks of whole sets of the handle's problems (one right-hand side per problem each)
  if (nrhs % H->nprob) {
    set_last_error_text("right-hand sides must come in whole sets of the handle's problems");
    return LS_EINVAL;
  }
  const int nbk = H->nprob * rhs_block_size(H, nrhs / H->nprob);
  for (int r = 0; r < nrhs; r += nbk) {
    const int nb = std::min(nbk, nrhs - r);
    int rc = nb > 1 ? solve_block(H, f + r * N, sigma + r * N, nb, info ? info + r : nullptr, transpose, st)
                    : solve_one(H, f + r * N, sigma + r * N, info ? info + r : nullptr, transpose, st);
    if (rc == LS_ENOCONV)
      worst = LS_ENOCONV;
    else if (rc)
      return rc;
  }
  return worst;
}

}  // namespace ls
