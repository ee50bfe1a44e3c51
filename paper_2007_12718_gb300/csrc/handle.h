// Internal state of an ls_handle and the host-side entry points of each
// kernel family.  Not part of the public ABI.
#pragma once
#include <functional>
#include <vector>

#include "common.cuh"
#include "hankel.cuh"

struct LevelData {
  int w = 0, h = 0;  // box dimensions (grid cells) of a node on this level
  int m = 0;         // rows of this level's ID: s*s on the leaf level, 2*k_{l+1} above
  int k = 0;         // skeleton rank k_l
  int ring = 0;      // proxy points of this level's ring
  std::vector<int> skel_x, skel_y;  // skeleton, local coordinates in a level-l box
  std::vector<int> piv;              // the skeleton's rows among the level's m candidates (U(piv, :) = I)
  void* U = nullptr;     // m x k, row-major (precision of the preconditioner)
  void* Gsib = nullptr;  // k x k: G(skel_alpha, skel_beta) of two children on this level
  void* X = nullptr;     // per node: (s^2)^2 on the leaf level, (2 k_{l+1})^2 above
  void* S = nullptr;     // per node: k x k (levels >= 1)
  void* UT = nullptr;    // k x m: U transposed (the apply reads every product row-wise)
  void* GT = nullptr;    // k x k: Gsib transposed
  void* XT = nullptr;    // per node: X transposed (made on the first transposed apply)
  void* ST = nullptr;    // per node: S transposed (idem)
  int gr = 0;            // rank of Gsib ~ GL GR^T (Woodbury merge); -1: the level keeps the Schur form
  void* GL = nullptr;    // k x gr
  void* GR = nullptr;    // k x gr
  void* GLT = nullptr;   // gr x k: GL transposed (the apply reads every product row-wise)
  void* GRT = nullptr;   // gr x k: GR transposed
  int xr = 0;            // > 0: X of this level is kept as I + P_L Q_R, X holding P_L (2k' x 2xr per
                         // node, k' the children's rank), Q_R = diag(GL^T, GR^T) of the children's level
  void* XLT = nullptr;   // per node: P_L transposed (2xr x 2k'), for the transposed apply
};

struct ls_handle {
  cudaStream_t stream = nullptr;  // stream of the most recent call (ls_free orders on it)
  int device = -1;                // the device the handle was built on (every call must have it current)
  ls_grid grid;
  double kappa = 0, tol = 0;
  ls_opts opts;
  int L = 0, s = 0, ring = 0;
  int nprob = 1;  // problems on the grid (a forest of nprob trees sharing one compression)
  int prec = LS_FP32;
  int nsm = 0;  // SMs on the device
  ls::KernelSpec ks_prec, ks_mv;

  // FFT matvec (Sec. 5): quarter spectrum (nx+1) x (ny+1), scaled by 1/(4 nx ny)
  ls::z64* spec = nullptr;
  ls::z64 *tw_x = nullptr, *tw_y = nullptr;  // exp(-2 pi i k / L) for the two padded lengths
  int Lx = 0, Ly = 0, logLx = 0, logLy = 0;
  double* b = nullptr;          // device copy of b [ny][nx]
  ls::z64* ktab = nullptr;      // h^2 G(h |d|) for lattice offsets 0 <= d1 < ktx, 0 <= d2 < kty
  int ktx = 0, kty = 0;
  ls::z64* convbuf = nullptr;   // ny x 2nx complex per right-hand side
  int convbuf_rhs = 0;

  // HBS (Secs. 3-4)
  std::vector<LevelData> lev;   // lev[0..L]
  void* Gleaf = nullptr;        // s^2 x s^2
  void* XBU = nullptr;          // per leaf s^2 x k_L: X B U (Algorithm 2, last step)
  void* work = nullptr;         // scratch for build and apply
  size_t work_bytes = 0;
  void* bwork = nullptr;        // scratch of the apply to a block of right-hand sides (nb x work)
  size_t bwork_bytes = 0;
  int* sync_buf = nullptr;      // grid-barrier counters + error flags
  int* d_err = nullptr;         // device status word (LS_ESINGULAR / LS_ETIMEOUT)
  cudaGraphExec_t apply_exec = nullptr;  // Algorithm 2 recorded as a CUDA graph
  ls::z64** slots = nullptr;    // device-side input/output pointers of the apply graph
  long long apply_nodes = 0;    // kernels in the apply graph
  void* apply_ops = nullptr;    // the apply as one persistent kernel: operation list (device)
  int apply_nops = 0, apply_phases = 0, apply_blocks = 0;
  unsigned* apply_bar = nullptr;     // its grid barrier: arrival counter and abort flag
  unsigned apply_epoch = 0;     // barrier arrivals so far (epochs continue across applies)
  // the transposed apply (Algorithm 2 reversed): factors transposed, its operation list
  void* XBUT = nullptr;         // per leaf k_L x s^2
  void* apply_ops_t = nullptr;
  int apply_nops_t = 0, apply_phases_t = 0;
  std::vector<int> apply_phase_end_t;  // host copy: index of the last operation of each phase
  double flops_build = 0, flops_compress = 0, bytes_apply = 0, factor_bytes = 0;
  double flops_sibling = 0;     // the sibling blocks' low-rank factorisations (counted in flops_build)
  int compression_reused = 0;   // the compression came from the cache or a file
  int pivot_fallbacks = 0;      // merge levels that needed the row-pivoted inverse
  double probe_resid_max = 0;   // largest probe residual max_i |(Z W v - v)_i| of the merge inverses
  long long spin_limit = ls::kSpinLimit;  // polls of a bounded device wait (ls_opts.wait_limit)
  cudaStream_t inv_stream = nullptr;  // second stream of the blocked inverse (panel updates)
  cudaStream_t ext_stream = nullptr;  // third stream of the blocked inverse (panel operands)
  cudaStream_t side_stream = nullptr; // the FFT spectrum set-up beside the build

  // receivers (Eq. (1)): positions (device, nr x 2) and R[k][j] = h^2 G(|r_k - x_j|)
  double* rx = nullptr;
  int nrec = 0;
  ls::z64* Rrec = nullptr;      // nr x N complex128

  // GMRES workspace (Sec. 5)
  int gm_maxit = 0, gm_rhs = 0;
  void* gm = nullptr;
  size_t gm_bytes = 0;
  // block GMRES (gmres_block.cu): small state, then one slab of nb vectors per
  // Krylov vector V_j and preconditioned vector Z_j, allocated as iterations need them
  void* bgm = nullptr;
  size_t bgm_bytes = 0;
  std::vector<void*> bslab;
  size_t bslab_bytes = 0;
};

namespace ls {

// conv.cu
int kernel_table_setup(ls_handle* H, cudaStream_t st);
int conv_setup(ls_handle* H, cudaStream_t st);
// mode CONV_FORWARD: y = x + kappa^2 b .* (K * x) = A x;  CONV_TRANSPOSE:
// y = x + K * (kappa^2 b .* x) = A^T x (K is complex symmetric);  CONV_FIELD: y = K * x.
enum ConvMode { CONV_FORWARD = 0, CONV_TRANSPOSE = 1, CONV_FIELD = 2 };
int conv_apply(ls_handle* H, const z64* x, z64* y, int nrhs, int mode, cudaStream_t st);

// Build pipeline hooks: the compression reports each finished level (its U,
// rank, skeleton and sibling block are in place and recorded on its stream);
// the merge stage waits for the level it needs.  Empty hooks: no pipelining.
typedef std::function<int(int level)> LevelWait;
typedef std::function<void(int level)> LevelDone;

// Page-locked host scratch of at least `bytes` bytes, private to the calling
// thread (grown on demand, released when the thread exits).  Small device-to-
// host reads go through it: a copy to pageable memory is synchronous inside
// the driver and would stall the other build thread's launches.
void* pinned_scratch(size_t bytes);
// LS_TRACE=1: prints "ls host <label> <ms since the last ls_build started>" to stderr.
void host_mark(const char* label);

// compress.cu
// With an auxiliary stream su, each level's U (the ID's back substitution) is
// finished on su, beside the next level's ID; level_done must then order its
// users after su.
int compress(ls_handle* H, cudaStream_t st, const LevelDone& level_done = LevelDone(), cudaStream_t su = nullptr);
// Kernel blocks the merges need: the leaf self-interaction block, and the sibling
// block of level l (once the level's skeleton is known).
int leaf_block(ls_handle* H, cudaStream_t st);
int sibling_block(ls_handle* H, int l, cudaStream_t st);
// Row ID of the device matrix A (m x p, candidate-major) in the given precision;
// piv (host, m entries) and U (device, m x min(m, p) entries) receive k pivots / columns.
// method: ID_AUTO (blocked above a size threshold), ID_GREEDY (one pivot per
// step, the same pivots as a column-pivoted QR), ID_BLOCKED (id_blocked.cu).
enum IdMethod { ID_AUTO = 0, ID_GREEDY = 1, ID_BLOCKED = 2 };
int row_id(const z64* A, int m, int p, double eps, int precision, int method, int nsm, int* sync_buf,
           cudaStream_t st, int* k, int* piv, z64* U);

// id_blocked.cu: the row ID in blocks of pivots (A is overwritten by the trailing
// residual).  Returns k and the pivots (host); with U non-null also U (m x k,
// row-major, device), written on su when given (else on st).
template <class R>
int blocked_row_id(cx<R>* A, int m, int p, double eps, cudaStream_t st, cudaStream_t su, cx<R>* U, int* k_out,
                   std::vector<int>* hp);

// build.cu (Algorithm 1) and apply (Algorithm 2)
// wait_level(l): the compression of level l is done; wait_sibling(l): level l's
// sibling block, U^T, G^T and low-rank factors are made (sibling_prepare, by the
// caller's worker); an empty hook makes the build wait or make them itself.
int hbs_build(ls_handle* H, cudaStream_t st, const LevelWait& wait_level = LevelWait(),
              const LevelWait& wait_sibling = LevelWait());
int sibling_prepare(ls_handle* H, int l, cudaStream_t st);
// After the factors are in place (ls_load): the apply's workspace and operation
// list, and the apply's byte count.
int hbs_finish(ls_handle* H, cudaStream_t st);

// persist.cu: the compression cache of reuse_compression.  cache_fetch copies a
// matching entry's levels into H (*found = true); cache_store keeps a copy of H's.
int cache_fetch(ls_handle* H, cudaStream_t st, bool* found);
int cache_store(ls_handle* H, cudaStream_t st);
int setup_handle(ls_handle* H, const ls_grid* grid, double kappa, const double* b, double tol, const ls_opts* opts,
                 cudaStream_t st);
// q = M f, or q = M^T f when transpose (Algorithm 2 reversed, every factor transposed)
int hbs_apply(ls_handle* H, const z64* f, z64* q, int nrhs, int transpose, cudaStream_t st);
// the same for a block of nb right-hand sides at once (each factor read once for
// the block, every product a batched GEMM with nb columns)
int hbs_apply_block(ls_handle* H, const z64* f, z64* q, int nb, int transpose, cudaStream_t st);
// right-hand sides per block of ls_apply / ls_solve (ls_opts.rhs_block; 0 = automatic)
int rhs_block_size(const ls_handle* H, int nrhs);

// tc_gemm.cu: complex FP32 GEMM on tcgen05 tensor cores (split: 0 tf32, 1 tf32x3)
int tc_cgemm(cudaStream_t st, bool ta, bool tb, int M, int N, int K, c32 alpha, const c32* A, int lda, long long sA,
             const c32* B, int ldb, long long sB, c32 beta, c32* C, int ldc, long long sC, int batch, int split,
             int* err, int band_lo = 0, int band_hi = 0);
int simt_cgemm(cudaStream_t st, bool ta, bool tb, int M, int N, int K, c32 alpha, const c32* A, int lda, long long sA,
               const c32* B, int ldb, long long sB, c32 beta, c32* C, int ldc, long long sC, int batch);
int simt_zgemm(cudaStream_t st, bool ta, bool tb, int M, int N, int K, z64 alpha, const z64* A, int lda, long long sA,
               const z64* B, int ldb, long long sB, z64 beta, z64* C, int ldc, long long sC, int batch);

// adjoint.cu: u (nrhs x nr) = sigma R^T and g (nrhs x N) = v R with the handle's receivers
int receiver_field(ls_handle* H, const z64* sigma, z64* u, int nrhs, cudaStream_t st);
int receiver_adjoint(ls_handle* H, const z64* v, z64* g, int nrhs, cudaStream_t st);

// gmres.cu
int gmres_solve(ls_handle* H, const z64* f, z64* sigma, int nrhs, ls_solve_info* info, int transpose,
                cudaStream_t st);

// Host or device vectors at the C ABI: device pointers are used in place;
// host vectors are staged through a device buffer (copied in on the stream,
// copied out and synchronised by stage_out_finish).
struct Staged {
  z64* dev = nullptr;
  bool owned = false;
};
bool is_device_pointer(const void* p);
int stage_in(const void* p, size_t bytes, cudaStream_t st, Staged* s);
int stage_out_alloc(void* p, size_t bytes, Staged* s);
int stage_out_finish(void* p, size_t bytes, cudaStream_t st, Staged* s);
void release(Staged* s);

// Device allocation from the library's stream-ordered memory pool (one per
// device, memory kept in the pool between calls), ordered on the stream of the
// current entry point; failures are recorded as LS_ENOMEM.
int dalloc(void** p, size_t bytes);
void dfree(void* p);
// Sets the stream dalloc/dfree order on for the lifetime of the object.
struct StreamScope {
  cudaStream_t prev;
  explicit StreamScope(cudaStream_t s);
  ~StreamScope();
};
void set_last_error_text(const char* msg);
int check_launch(const char* what);

}  // namespace ls

namespace ls {
// LS_OK when the calling thread's current device is the handle's, else LS_EINVAL
// with a message (the handle's memory and kernels belong to its device).
int check_device(const ls_handle* H);
// Device and pinned host allocations made by the library so far (ls_allocations).
long long allocation_count();
// Failure injection (ls_fault_inject): parse a spec; consume a pending NaN-in-b fault.
int parse_fault(const char* spec);
bool take_nan_b_fault();
}  // namespace ls
