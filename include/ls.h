/* ls.h -- C ABI of the GB300 (sm_103a) Lippmann-Schwinger HBS solver.
 *
 * Method: Gopal & Martinsson, "An accelerated, high-order accurate direct
 * solver for the Lippmann-Schwinger equation for acoustic scattering in the
 * plane" (arXiv 2007.12718).
 *
 *   sigma + kappa^2 b(x) int_Omega G(x,y) sigma(y) dy = -kappa^2 b(x) u_inc(x)   (Eq. 3)
 *   G(x,y) = (i/4) H0^(1)(kappa |x-y|)                                            (Eq. 2)
 *
 * discretised on a regular grid with the corrected trapezoidal rule (Sec. 2.2,
 * Eq. 8) into (I + B G_p) q = f  (Eqs. 9-10), B = diag(kappa^2 b).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Grid: nx * ny cell-centred nodes x_ij = (x0 + (i+1/2) h, y0 + (j+1/2) h).
 *    Grid arrays are row-major [ny][nx] (x fastest).  Several right-hand
 *    sides are stacked as [nrhs][ny][nx].
 *  - Complex vectors are interleaved complex128 {re, im} (16 bytes/entry).
 *  - Pointers to vectors may be device pointers or host pointers (pageable or
 *    pinned); the library queries the pointer and stages host data through
 *    device memory itself.  All work is ordered on `stream` (a cudaStream_t,
 *    NULL = the legacy default stream); calls return after the work is
 *    enqueued, except where a result must come back to the host (ranks in
 *    ls_build, the convergence test in ls_solve, host output buffers).
 *  - Ownership: the caller owns every buffer it passes; the library copies b
 *    during ls_build and owns the handle's memory until ls_free.
 *  - Errors: every int-returning call returns LS_OK (0) or a negative LS_E*
 *    code; no call aborts the process or throws across the ABI.  The text of
 *    the last error of the calling thread is available from ls_last_error().
 */
#ifndef LS_H_
#define LS_H_

#ifdef __cplusplus
extern "C" {
#endif

enum {
  LS_OK = 0,
  LS_EINVAL = -1,     /* bad argument (sizes, b not finite, ...) */
  LS_ENOMEM = -2,     /* device allocation failed */
  LS_ECUDA = -3,      /* CUDA runtime error (see ls_last_error) */
  LS_ESINGULAR = -4,  /* zero pivot in a local inverse */
  LS_ENOCONV = -5,    /* GMRES hit maxit; sigma and info are still written */
  LS_ETIMEOUT = -6    /* a bounded device-side wait gave up */
};

/* Precision of the HBS preconditioner (compression, inverse build, apply).
 * The FFT matvec and GMRES are FP64 in every mode.  LS_FP32, LS_TF32X3 and
 * LS_FP16SPLIT store the factors in FP32; they differ in the engine of the
 * large merge GEMMs (Eqs. 26-27): FP32 SIMT cores; tensor cores with each
 * operand split into two tf32 terms (three products, ~FP32 accuracy); tensor
 * cores with each operand scaled by a power of two and split into two FP16
 * terms (the FP16 split product: three kind::f16 products at twice the tf32
 * rate, the same ~22 bits of each operand).  LS_TF32 (one tf32 product, ~1e-3
 * relative error) names a GEMM engine of ls_cgemm_c64 only: its
 * preconditioner misses the HBS tolerance by orders of magnitude, so ls_build
 * rejects it (LS_EINVAL). */
enum { LS_FP64 = 0, LS_FP32 = 1, LS_TF32 = 2, LS_TF32X3 = 3, LS_FP16SPLIT = 4 };

typedef struct {
  int nx, ny;        /* grid size; a tree of square leaves must fit (see ls_build) */
  double h;          /* mesh width */
  double x0, y0;     /* lower-left corner of the domain */
} ls_grid;

typedef struct {
  int order_matvec;  /* corrected-quadrature order of the FFT matvec: 2,4,6,8,10 (default 10) */
  int order_precond; /* order used inside the HBS compression: 4,6,8,10 (default 4)      */
  int leaf_side;     /* leaf box side s (s*s points per leaf, default 8)                  */
  int proxy_width;   /* proxy ring width in grid cells; 0 = from tol and order (default)  */
  int precision;     /* LS_FP64, LS_FP32, LS_TF32X3 or LS_FP16SPLIT (default LS_FP32)       */
  int gmres_maxit;   /* default 100 (Sec. 6.3)                                            */
  double gmres_tol;  /* relative residual, default 1e-10 (Sec. 6.3)                       */
  int merge_pivoting; /* merge inverses: 0 = blocks without interchanges, checked, with the
                         row-pivoted inverse as fallback (default); 1 = always row-pivoted   */
  int top_uncompressed; /* levels 1..top_uncompressed keep every row as skeleton (U = I,
                         no ID); 0 = every level compressed as in Sec. 3.2 (default)      */
  int id_method;      /* per-level ID (Sec. 2.1): LS_ID_AUTO (default), LS_ID_GREEDY or
                         LS_ID_BLOCKED, see ls_row_id_ex                                  */
  int wait_limit;     /* polls of a device-side wait (grid barriers of the ID, apply and GMRES
                         kernels) before it gives up and the call returns LS_ETIMEOUT; 0 =
                         default (2e7 polls, about a second).  After LS_ETIMEOUT the handle's
                         barrier state is spent: free the handle.                          */
  int woodbury;       /* merges (Eq. 26): 1 = the Woodbury form where it pays (default): each
                         level's sibling block is factored once, G ~ L R^T by a row ID at
                         tolerance tol, and the merge inverts an r x r matrix instead of a
                         k x k one (Sec. 4.1, the remark on the rank of G); used where
                         k >= 48 and r <= k / 2.  0 = the Schur form everywhere; 2 = the
                         Woodbury form at every level with r < k (small grids, tests).      */
  int reuse_compression; /* 1 = keep the compression (per-level skeletons, U, sibling blocks and
                         their factors) in a process-wide cache and take it from there when a
                         later ls_build on the same device has the same kappa, h, grid, leaf
                         side, tol, order_precond, ring, precision, top_uncompressed,
                         id_method and woodbury: it does not depend on b (Sec. 3.2), so only
                         the leaf build and the merges run.  0 = compress every time
                         (default).  ls_compression_cache_clear releases the cache.       */
  int rhs_block;      /* right-hand sides that ls_apply / ls_solve / ls_solve_transpose treat
                         as one block: the apply runs each product as a GEMM over the block
                         (every factor read once per block), GMRES keeps one Krylov space per
                         right-hand side and applies the preconditioner and the operator to
                         the block's current vectors together.  0 = automatic (up to 256, and
                         nb * nx * ny * 16 bytes within 1 GiB); 1 = one right-hand side at a
                         time (the persistent one-vector apply).  Block GMRES allocates one
                         slab of nb grid vectors per Krylov vector and per preconditioned
                         vector as the iterations reach them (kept by the handle).         */
} ls_opts;

/* Pivot selection of the row ID (ls_opts.id_method, ls_row_id_ex).
 *  LS_ID_GREEDY : one pivot per step, the candidate of largest residual norm --
 *                 the pivots of a column-pivoted QR (Sec. 2.1).
 *  LS_ID_BLOCKED: pivots in blocks of up to 32.  Each block considers the 64
 *                 candidates of largest residual norm, orders them by a greedy
 *                 pivoted Cholesky of their Gram matrix (the column-pivoted QR
 *                 restricted to those 64) and accepts a candidate while its
 *                 residual norm is at least half the largest residual norm of
 *                 the candidates left out; the other candidates are then updated
 *                 by GEMM-shaped kernels.  The rank is decided by the same
 *                 Frobenius-norm rule, on the explicit residual.
 *  LS_ID_AUTO   : blocked above 1024 candidates (and wherever a candidate's
 *                 vector is too long for the greedy kernels), greedy below. */
enum { LS_ID_AUTO = 0, LS_ID_GREEDY = 1, LS_ID_BLOCKED = 2 };

typedef struct {
  int iterations;     /* GMRES iterations taken */
  int converged;      /* 1 if the residual estimate reached gmres_tol */
  double resid_est;   /* Arnoldi residual estimate ||f - A sigma|| / ||f|| */
  double resid_true;  /* recomputed ||f - A sigma|| / ||f|| with the FFT matvec */
} ls_solve_info;

typedef struct {
  int levels;               /* L: the tree has 2^L leaves */
  int ranks[32];            /* ranks[l] = skeleton size k_l of level l (ranks[0] = 0) */
  int proxy_width;          /* ring width actually used */
  double flops_build;       /* algorithmic real flops of the inverse build (Alg. 1) */
  double flops_compress;    /* algorithmic real flops of the per-level IDs */
  double bytes_apply;       /* algorithmic bytes read+written by one HBS apply */
  double factor_bytes;      /* device bytes held by the factors */
  int pivot_fallbacks;      /* merge levels whose check sent them to the row-pivoted inverse */
  int sibling_ranks[32];    /* sibling_ranks[l] = r_l of the level's factored sibling block
                               G ~ L R^T (Woodbury merge), 0 where the level keeps the Schur form */
  double probe_resid_max;   /* largest max_i |(Z W v - v)_i| over the merge inverses W = Z^-1
                               formed without interchanges, v a unit-modulus probe; W is accepted
                               when it is <= max(tol, 10 u k), u the unit roundoff, k the order */
  int compression_reused;   /* 1 if the compression came from the cache (reuse_compression)
                               or from a file (ls_load) */
  int nx, ny;               /* the grid */
  int nprob;                /* problems on the grid (ls_build_many) */
} ls_build_info;

typedef struct ls_handle ls_handle; /* opaque, library-owned */

/* Fill *o with the defaults listed above. */
void ls_default_opts(ls_opts* o);

/* ls_build -- compress G_p (Sec. 3.2) and build the HBS inverse of I + B G_p
 * (Algorithm 1, Sec. 4.1), and set up the FFT matvec of the order_matvec
 * operator (Sec. 5).
 *   grid   : geometry.  nx = s * 2^ceil(L/2), ny = s * 2^floor(L/2) for the
 *            leaf side s and some L >= 1 (cuts alternate vertical/horizontal,
 *            Sec. 3.2), e.g. nx = ny = s * 2^(L/2).
 *   kappa  : wavenumber > 0.
 *   b      : scattering potential, ny*nx doubles (host or device), finite.
 *            b <= 1 guarantees existence and uniqueness (Sec. 1); larger
 *            values are accepted (the lens of Sec. 6.2 reaches 1.18), and a
 *            singular system shows as LS_ENOCONV of the solve.
 *   tol    : HBS compression tolerance eps in (0, 1) (Eq. 11, with the local
 *            tolerance eps * ||proxy block||_F).
 *   opts   : NULL for defaults.
 *   out    : receives the handle.
 * Returns LS_EINVAL for a bad argument, LS_ESINGULAR when a local inverse
 * meets a zero pivot, LS_ETIMEOUT if a device-side wait gave up. */
int ls_build(const ls_grid* grid, double kappa, const double* b, double tol,
             const ls_opts* opts, void* stream, ls_handle** out);

/* ls_build_many -- nprob independent problems on the same grid and kappa
 * (potentials b_0 .. b_{nprob-1}, nprob * ny * nx doubles, host or device, in
 * that order) in one handle: the compression does not depend on b and is made
 * once (Sec. 3.2); the leaf builds and merges of all problems run as one
 * forest of nprob trees, every level's nodes of every problem in the same
 * batched launches, and so does the apply.  On such a handle every vector
 * argument of ls_apply, ls_matvec, ls_field, ls_solve, ls_solve_transpose and
 * ls_rhs_plane_wave holds nrhs sets of nprob grid vectors, [nrhs][nprob][ny][nx]
 * (vector g of a set belongs to problem g), and ls_solve's info has nrhs *
 * nprob entries in the same order; each problem is solved with its own
 * operator and its own Krylov space (block GMRES).  The receiver calls and
 * ls_matvec_noalloc take handles of one problem only (LS_EINVAL).  ls_build is
 * ls_build_many with nprob = 1. */
int ls_build_many(const ls_grid* grid, int nprob, double kappa, const double* b, double tol,
                  const ls_opts* opts, void* stream, ls_handle** out);

/* ls_apply -- q = M f, M ~ (I + B G_p)^-1 the HBS inverse (Algorithm 2,
 * Sec. 4.1); with transpose = 1, q = M^T f: the steps of Algorithm 2 in
 * reverse order with every factor transposed (plain transpose, no
 * conjugate), the preconditioner of the adjoint solve.  The first transposed
 * apply on a handle makes transposed copies of the factors (as much device
 * memory again as the factors).  f, q: nrhs complex128 grid vectors.
 * transpose: 0 or 1, else LS_EINVAL.  Applies on one handle must not run
 * concurrently (they share the handle's scratch).  The call is asynchronous: a
 * device-side timeout of its barriers shows in ls_sync or the next ls_solve. */
int ls_apply(ls_handle* h, const void* f, void* q, int nrhs, int transpose, void* stream);

/* ls_matvec -- y = (I + B (G + T)) x, the order_matvec operator applied by a
 * zero-padded 2D FFT convolution (Sec. 2.2 last paragraph, Sec. 5); with
 * transpose = 1, y = (I + B (G + T))^T x = x + (G + T)(B x) (G + T is
 * complex symmetric: its entries depend on |x_i - x_j| and the correction
 * stencil is symmetric, Eqs. 8, 10).  x, y: nrhs complex128 grid vectors (may
 * not alias).  transpose: 0 or 1, else LS_EINVAL. */
int ls_matvec(ls_handle* h, const void* x, void* y, int nrhs, int transpose, void* stream);

/* ls_field -- u = (G + T) sigma on the grid: the scattered field at the nodes
 * of a density sigma (Eq. 1 with the order_matvec corrected quadrature,
 * Eqs. 8, 10), by the same FFT convolution.  sigma, u: nrhs complex128 grid
 * vectors, host or device (may not alias). */
int ls_field(ls_handle* h, const void* sigma, void* u, int nrhs, void* stream);

/* ls_solve -- GMRES on (I + B (G+T)) sigma = f, right-preconditioned by the
 * HBS inverse (Sec. 5), from sigma = 0, no restart, stopping at
 * gmres_tol or gmres_maxit (Sec. 6.3).  f, sigma: nrhs complex128 grid
 * vectors; info: nrhs entries (may be NULL).  Returns LS_ENOCONV if some
 * right-hand side did not converge (sigma is still written). */
int ls_solve(ls_handle* h, const void* f, void* sigma, int nrhs, ls_solve_info* info, void* stream);

/* ls_solve_transpose -- the same GMRES on the transposed system
 * (I + B (G+T))^T sigma = f, right-preconditioned by M^T (ls_apply with
 * transpose = 1): the adjoint solve of a gradient.  Arguments and return
 * codes as ls_solve. */
int ls_solve_transpose(ls_handle* h, const void* f, void* sigma, int nrhs, ls_solve_info* info, void* stream);

/* ls_set_receivers -- receivers r_k for the calls below: the handle evaluates
 * and keeps R[k][j] = h^2 G(|r_k - x_j|) (Eq. 1 by the trapezoidal rule, which
 * is spectrally accurate for receivers outside the support of sigma;
 * G = (i/4) H0(kappa r), Eq. 2), nr * N complex128 on the device.
 *   rx: host, nr pairs (x, y).  nr = 0 clears.  A receiver on a grid node
 *   returns LS_EINVAL.  Synchronises the stream. */
int ls_set_receivers(ls_handle* h, const double* rx, int nr, void* stream);

/* ls_receiver_field -- u[r][k] = sum_j R[k][j] sigma[r][j]: the field of
 * nrhs densities at the receivers.  sigma: nrhs complex128 grid vectors; u:
 * nrhs * nr complex128 ([nrhs][nr]); host or device.  LS_EINVAL without
 * receivers. */
int ls_receiver_field(ls_handle* h, const void* sigma, void* u, int nrhs, void* stream);

/* ls_receiver_adjoint -- g[r][j] = sum_k R[k][j] v[r][k] (R^T v, no
 * conjugate).  v: nrhs * nr complex128; g: nrhs complex128 grid vectors. */
int ls_receiver_adjoint(ls_handle* h, const void* v, void* g, int nrhs, void* stream);

/* ls_misfit_gradient -- for plane waves thetas[r] (host, nrhs angles) and
 * data d ([nrhs][nr] complex128, host or device) at the handle's receivers:
 *   J = sum_{r,k} |u_r(r_k) - d[r][k]|^2,  sigma_r = A^-1 f_r (ls_solve),
 *   u_r = R sigma_r,  A = I + B (G+T),  f_r = -kappa^2 b u_inc,r (Eq. 3),
 * and dJ/db by the adjoint method: lambda_r = A^-T R^T conj(u_r - d_r)
 * (ls_solve_transpose), then
 *   dJ/db_j = -2 kappa^2 sum_r Re(lambda_r[j] ((G+T) sigma_r + u_inc,r)[j]).
 *   J: out, host double.  grad: out, ny*nx doubles, host or device; NULL
 *   computes J alone (the forward solves only, no adjoint solve).
 *   info: NULL or 2 nrhs entries (the forward solves, then the adjoint ones).
 * The gradient is that of the discrete system solved to gmres_tol; the HBS
 * inverse only preconditions.  Returns LS_ENOCONV (outputs still written) if
 * a solve did not converge, LS_EINVAL without receivers. */
int ls_misfit_gradient(ls_handle* h, const double* thetas, int nrhs, const void* d, double* J, void* grad,
                       ls_solve_info* info, void* stream);

/* ls_rhs_plane_wave -- f = -kappa^2 b u_inc with u_inc = exp(i kappa (x1 cos theta
 * + x2 sin theta)) (right-hand side of Eq. 3), one complex128 grid vector per
 * angle.  thetas: nrhs doubles on the host. */
int ls_rhs_plane_wave(ls_handle* h, const double* thetas, void* f, int nrhs, void* stream);

/* ls_matvec_noalloc -- ls_matvec for callers that must not allocate device
 * memory when they apply the operator.  The paper has no counterpart: this is
 * a deployment variant.  Such callers include frameworks whose memory pool
 * already holds the free device memory (a cudaMalloc would fail or fragment
 * it), latency-critical loops that cannot take the implicit device
 * synchronisation of cudaMalloc/cudaFree, and programs whose memory budget is
 * fixed at start-up.  ls_matvec may allocate (its FFT buffer grows with nrhs,
 * host vectors are staged); this call calls no cudaMalloc, cudaFree or other
 * allocating routine.  Its FFT scratch is a fixed file-scope device array of
 * ls_matvec_noalloc_max_elems() = 2^18 complex128 entries (4 MiB), held by
 * every GPU that loads the library until the process exits.
 *   x, y : device pointers of the current device (the handle's), nrhs
 *   complex128 grid vectors (x, y may not alias).
 *   Requires nrhs * ny * 2 * nx <= 2^18; larger sizes return LS_EINVAL with a
 *   message, as do host pointers and pointers of another device.  The handle
 *   must come from ls_build (which does allocate, at set-up time).
 *   The first call on a device looks up the scratch array's device address
 *   (cudaGetSymbolAddress, with that device current) and keeps it for the life
 *   of the process; make that first call before any stream capture.  The kept
 *   address does not survive a cudaDeviceReset of that device (the library's
 *   module is loaded anew there): such a program must not call this entry point
 *   after the reset.  Every call shares the one array and leaves its
 *   contents behind; nothing in it needs to start at zero (each call writes
 *   every entry before reading it), but calls that overlap on the GPU (two
 *   streams at once) race on it. */
int ls_matvec_noalloc(ls_handle* h, const void* x, void* y, int nrhs, void* stream);
long long ls_matvec_noalloc_max_elems(void);

/* ls_sync -- wait for the work queued on `stream` and return the handle's
 * device status: LS_OK, or LS_ETIMEOUT / LS_ESINGULAR if a device-side wait or
 * a local inverse of an earlier asynchronous call (ls_apply, ls_matvec, ...)
 * failed.  ls_solve and ls_build report the status themselves.  The status is
 * not cleared: a handle whose wait timed out is spent. */
int ls_sync(ls_handle* h, void* stream);

/* ls_build_info -- ranks, flop and byte counts of the built handle. */
int ls_get_build_info(const ls_handle* h, ls_build_info* info);

/* ls_compression_cache_clear -- release every compression kept by
 * reuse_compression (device memory of every device that holds one). */
void ls_compression_cache_clear(void);

/* ls_save -- write a built handle to the file `path`: the inputs (grid, kappa,
 * tol, options, b) and every factor (per level the skeleton, U, the sibling
 * block and its low-rank factors, X and S; X B U of the leaves), so that
 * ls_load can restore it without compressing or merging.  Binary, this
 * library's layout (little-endian, native sizes), version-checked.
 * Synchronises the stream.  LS_EINVAL if the file cannot be written. */
int ls_save(const ls_handle* h, const char* path, void* stream);

/* ls_load -- a handle from a file written by ls_save, on the current device:
 * the set-up of ls_build (kernel table, FFT spectrum, b checked) and the
 * stored factors uploaded; the apply and solve calls then behave as on the
 * saved handle.  LS_EINVAL for a missing, truncated or foreign file. */
int ls_load(const char* path, void* stream, ls_handle** out);

/* ls_free -- release every resource of the handle (NULL is allowed). */
void ls_free(ls_handle* h);

/* Every call taking a handle must run with the handle's device current (the
 * device current at ls_build); otherwise it returns LS_EINVAL without touching
 * the GPU.  ls_free releases the handle on its own device. */

/* Per-kernel timing (not part of the method; used by the benchmark).
 * When enabled, the library records a CUDA event pair around each launch of
 * the listed kernel families on the stream it launches them on, and
 * accumulates launches, device milliseconds and the algorithmic bytes and
 * flops of each launch.  ls_profile_get synchronises on the recorded events
 * and fills up to max_entries entries; it returns the number written. */
typedef struct {
  char name[32];
  long long launches;
  double total_ms;
  double bytes;   /* algorithmic bytes moved, summed over launches */
  double flops;   /* algorithmic real flops, summed over launches */
} ls_profile_entry;
int ls_profile_enable(int on);
int ls_profile_reset(void);
int ls_profile_get(ls_profile_entry* out, int max_entries);

/* ls_measure_peak -- arithmetic rate of this GPU for the roofline denominators
 * (not part of the method): long chains of independent fused multiply-adds,
 * timed with CUDA events on `stream` (best of three launches after one warm-up).
 *   kind: 0 = FP64 FMA, 1 = FP32 FMA, 2 = packed FP32 FMA (two lanes per
 *         instruction, the form the FP32 GEMMs use).  tflops: out, 2 flops/FMA.
 * Returns LS_EINVAL for a bad kind.  Synchronises the stream. */
int ls_measure_peak(int kind, double* tflops, void* stream);

/* Device and page-locked host allocations this library has made in this
 * process so far (every stream-ordered pool allocation counts, also when the
 * pool serves it from memory it already holds). */
long long ls_allocations(void);

/* ls_fault_inject -- host-side failure injection for tests of the error paths
 * (not part of the method; no GPU fault is ever caused).  spec:
 *   "alloc:N"  the N-th device allocation from now on (N >= 1) fails as if the
 *              device were out of memory (LS_ENOMEM), once;
 *   "nan_b"    the next ls_build sees a NaN in b, as if the caller had passed
 *              one (LS_EINVAL from the finiteness check), once;
 *   "" or NULL clears a pending injection.
 * The environment variable LS_FAULT, read once when the library loads, takes
 * the same spec.  Returns LS_EINVAL for a spec it does not know. */
int ls_fault_inject(const char* spec);

/* Number of CUDA kernels this library has launched in this process so far. */
long long ls_kernel_launches(void);

/* ls_cgemm_c64 -- building block exposed for testing: the batched complex
 * FP32 GEMM the HBS build uses for its merge products,
 *   C[b] = alpha op(A[b]) op(B[b]) + beta C[b],   b < batch,
 * row-major interleaved complex64, op = transpose (no conjugate) when ta/tb.
 * engine: 0 = FP32 SIMT, 1 = tcgen05 tf32, 2 = tcgen05 tf32x3, 3 = tcgen05
 * f16x3 (the FP16 split product; A and B each scaled by one power of two from
 * their largest entry over the batch).  alpha, beta:
 * {re, im} pairs.  All pointers on the device.  Returns LS_EINVAL for a bad
 * engine or size, LS_ETIMEOUT if a tensor-core wait gave up. */
int ls_cgemm_c64(int engine, int ta, int tb, int M, int N, int K, const float* alpha, const void* A, int lda,
                 long long sA, const void* B, int ldb, long long sB, const float* beta, void* C, int ldc,
                 long long sC, int batch, void* stream);

/* ls_row_id -- the interpolative decomposition of Sec. 2.1 as the compression
 * uses it (Sec. 3.2): A ~ U A(J, :) for an m x p complex matrix whose rows are
 * the candidates, by column-pivoted QR of A^T.  Pivot j is the candidate with
 * the largest residual norm (lowest index on ties); k is the first j at which
 * the Frobenius norm of the remaining residual is <= eps ||A||_F.
 *   A:    m * p complex128, row-major (row c = candidate c), host or device.
 *   precision: LS_FP64 or LS_FP32 (the arithmetic of the device kernels; with
 *         LS_FP32, A is rounded to complex64 on the device).
 *   k:    out, the rank.  piv: out, host array of at least min(m, p) ints,
 *         piv[0..k) the skeleton rows in pivot order.
 *   U:    out (may be NULL), m * k complex128 row-major, host or device,
 *         sized by the caller for m * min(m, p) entries; U(piv[a], a') = [a = a'].
 * Requires 1 <= m < 2^20, p >= 1, 0 < eps < 1.  Returns LS_EINVAL for a bad
 * argument, LS_ENOMEM, LS_ECUDA, or LS_ETIMEOUT if a grid barrier wait gave up.
 * Synchronises the stream before returning. */
int ls_row_id(const void* A, int m, int p, double eps, int precision, int* k, int* piv, void* U, void* stream);

/* ls_row_id_ex -- ls_row_id with the pivot selection chosen by method
 * (LS_ID_AUTO, LS_ID_GREEDY or LS_ID_BLOCKED; ls_row_id is LS_ID_GREEDY).  With
 * LS_ID_BLOCKED the pivots are a valid skeleton but need not be the greedy
 * ones; the rank rule and the outputs are the same.  A is not modified. */
int ls_row_id_ex(const void* A, int m, int p, double eps, int precision, int method, int* k, int* piv, void* U,
                 void* stream);

/* Static text for an LS_E* code, and the last error message of this thread. */
const char* ls_strerror(int code);
const char* ls_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LS_H_ */
