// C ABI of the Lippmann-Schwinger HBS solver (declared in include/ls.h).
// Argument checking, host/device staging, and the order of the phases:
// corrected-quadrature weights (host), FFT matvec set-up, per-level
// compression, Algorithm 1, then apply / matvec / GMRES on request.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <mutex>
#include <vector>
#include <thread>
#include <condition_variable>
#include <string>
#include <limits>

#include "handle.h"
#include "quad.h"

namespace {
thread_local std::string g_last_error;

void set_error(const char* msg) { g_last_error = msg; }

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int valid_order(int o) { return o == 2 || o == 4 || o == 6 || o == 8 || o == 10; }


__global__ void rhs_kernel(const double* b, int nx, int ny, double h, double x0, double y0, double kappa, double ct,
                           double stt, ls::z64* f) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)nx * ny) return;
  int i = (int)(t % nx), j = (int)(t / nx);
  double x1 = x0 + (i + 0.5) * h, x2 = y0 + (j + 0.5) * h;
  double sn, cs;
  sincos(kappa * (x1 * ct + x2 * stt), &sn, &cs);
  double a = -kappa * kappa * b[t];
  f[t] = ls::mk<double>(a * cs, a * sn);
}

__global__ void check_b_kernel(const double* b, long long n, int* bad) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  if (!isfinite(b[t])) atomicExch(bad, 1);
}

}  // namespace

namespace ls {

bool is_device_pointer(const void* p) { return is_device_ptr(p); }

// Staging of host vectors through device memory.
int stage_in(const void* p, size_t bytes, cudaStream_t st, Staged* s) {
  if (is_device_ptr(p)) {
    s->dev = (ls::z64*)p;
    s->owned = false;
    return LS_OK;
  }
  int rc = ls::dalloc((void**)&s->dev, bytes);
  if (rc) return rc;
  s->owned = true;
  LS_CUDA_TRY(cudaMemcpyAsync(s->dev, p, bytes, cudaMemcpyHostToDevice, st));
  return LS_OK;
}

int stage_out_alloc(void* p, size_t bytes, Staged* s) {
  if (is_device_ptr(p)) {
    s->dev = (ls::z64*)p;
    s->owned = false;
    return LS_OK;
  }
  int rc = ls::dalloc((void**)&s->dev, bytes);
  if (rc) return rc;
  s->owned = true;
  return LS_OK;
}

int stage_out_finish(void* p, size_t bytes, cudaStream_t st, Staged* s) {
  if (s->owned) {
    LS_CUDA_TRY(cudaMemcpyAsync(p, s->dev, bytes, cudaMemcpyDeviceToHost, st));
    LS_CUDA_TRY(cudaStreamSynchronize(st));
  }
  return LS_OK;
}

void release(Staged* s) {
  if (s->owned && s->dev) ls::dfree(s->dev);
  s->dev = nullptr;
  s->owned = false;
}

}  // namespace ls

using ls::release;
using ls::stage_in;
using ls::stage_out_alloc;
using ls::stage_out_finish;
using ls::Staged;

void ls_set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  char buf[512];
  snprintf(buf, sizeof(buf), "CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e), what, file, line);
  set_error(buf);
}

namespace ls {

void set_last_error_text(const char* msg) { set_error(msg); }

static std::atomic<long long> g_launches{0};
static std::atomic<long long> g_allocs{0};  // device and pinned host allocations (ls_allocations)
namespace {
bool debug_sync_enabled() {
  static const bool on = [] {
    const char* v = getenv("LS_DEBUG_SYNC");
    return v && v[0] && v[0] != '0';
  }();
  return on;
}
thread_local int g_capture_depth = 0;
thread_local const char* g_prev_file = "(none)";
thread_local int g_prev_line = 0;
std::atomic<bool> g_debug_reported{false};

void debug_sync(const char* file, int line, const char* what) {
  if (!debug_sync_enabled() || g_capture_depth > 0) return;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess && !g_debug_reported.exchange(true))
    fprintf(stderr, "[ls debug] device error '%s' detected at %s:%d (%s); previous launch site %s:%d\n",
            cudaGetErrorString(e), file, line, what, g_prev_file, g_prev_line);
}
}  // namespace
CaptureScope::CaptureScope() { ++g_capture_depth; }
CaptureScope::~CaptureScope() { --g_capture_depth; }
void count_launch_at(const char* file, int line, LaunchCount c) {
  g_launches.fetch_add(c.n, std::memory_order_relaxed);
  debug_sync(file, line, "before launch");
  g_prev_file = file;
  g_prev_line = line;
}

namespace {
thread_local cudaStream_t g_alloc_stream = nullptr;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[64] = {nullptr};

int pool_for_current_device(cudaMemPool_t* out) {
  int dev = 0;
  LS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return LS_EINVAL;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pools[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    LS_CUDA_TRY(cudaMemPoolCreate(&g_pools[dev], &props));
    unsigned long long keep = ~0ULL;  // keep freed memory in the pool
    LS_CUDA_TRY(cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolAttrReleaseThreshold, &keep));
    int no = 0;  // reuse across streams only without inserted dependencies (the build runs on two streams)
    LS_CUDA_TRY(cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolReuseAllowInternalDependencies, &no));
  }
  *out = g_pools[dev];
  return LS_OK;
}
}  // namespace

namespace {
// Page-locked scratch, one buffer per thread.  Each build runs its merges on a
// thread of its own, so a thread's buffer goes back to a process-wide free
// list when the thread ends (cudaFreeHost there would stall the end of every
// build) and the next thread takes it from there.
struct PinnedBuf {
  void* p = nullptr;
  size_t bytes = 0;
};
std::mutex g_pinned_mu;
std::vector<PinnedBuf>& pinned_free_list() {
  static std::vector<PinnedBuf>* v = new std::vector<PinnedBuf>();  // kept until process exit
  return *v;
}
struct PinnedScratch {
  PinnedBuf b;
  ~PinnedScratch() {
    if (!b.p) return;
    std::lock_guard<std::mutex> lk(g_pinned_mu);
    pinned_free_list().push_back(b);
  }
};
thread_local PinnedScratch g_pinned;
}  // namespace

void* pinned_scratch(size_t bytes) {
  PinnedBuf& b = g_pinned.b;
  if (!b.p) {
    std::lock_guard<std::mutex> lk(g_pinned_mu);
    auto& fl = pinned_free_list();
    if (!fl.empty()) {
      b = fl.back();
      fl.pop_back();
    }
  }
  if (bytes > b.bytes) {
    if (b.p) cudaFreeHost(b.p);
    b.p = nullptr;
    b.bytes = 0;
    size_t want = std::max(bytes, (size_t)1 << 16);
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    if (cudaMallocHost(&b.p, want) != cudaSuccess) {
      cudaGetLastError();
      b.p = nullptr;
      return nullptr;
    }
    b.bytes = want;
  }
  return b.p;
}

// Host-side build timeline (LS_TRACE=1): "ls host <label> <ms since the build started>".
std::chrono::steady_clock::time_point g_build_t0;

void host_mark(const char* label) {
  static const bool on = [] {
    const char* v = getenv("LS_TRACE");
    return v && v[0] && v[0] != '0';
  }();
  if (!on) return;
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - g_build_t0).count();
  fprintf(stderr, "ls host %s %.3f\n", label, ms);
}

namespace {
thread_local long long g_spin_limit = kSpinLimit;
}
long long spin_limit() { return g_spin_limit; }
SpinLimitScope::SpinLimitScope(long long limit) : prev(g_spin_limit) { g_spin_limit = limit; }
SpinLimitScope::~SpinLimitScope() { g_spin_limit = prev; }

StreamScope::StreamScope(cudaStream_t s) : prev(g_alloc_stream) { g_alloc_stream = s; }
StreamScope::~StreamScope() { g_alloc_stream = prev; }

long long allocation_count() { return g_allocs.load(); }

// Host-side failure injection (ls_fault_inject, LS_FAULT): the countdown of
// device allocations to the one that fails (0 = none), and a pending NaN in b.
static std::atomic<long long> g_fail_alloc_in{0};
static std::atomic<int> g_fail_nan_b{0};
int parse_fault(const char* spec) {
  if (!spec || !spec[0]) {
    g_fail_alloc_in = 0;
    g_fail_nan_b = 0;
    return LS_OK;
  }
  if (!strncmp(spec, "alloc:", 6)) {
    char* end = nullptr;
    const long long nth = strtoll(spec + 6, &end, 10);
    if (nth < 1 || !end || *end) return LS_EINVAL;
    g_fail_alloc_in = nth;
    return LS_OK;
  }
  if (!strcmp(spec, "nan_b")) {
    g_fail_nan_b = 1;
    return LS_OK;
  }
  return LS_EINVAL;
}
bool take_nan_b_fault() { return g_fail_nan_b.exchange(0) != 0; }
namespace {
struct FaultFromEnv {
  FaultFromEnv() {
    if (const char* v = getenv("LS_FAULT")) parse_fault(v);
  }
} g_fault_from_env;
// True when this allocation is the injected failure.
bool injected_alloc_failure() {
  long long c = g_fail_alloc_in.load();
  while (c > 0) {
    if (g_fail_alloc_in.compare_exchange_weak(c, c - 1)) return c == 1;
  }
  return false;
}
}  // namespace

int check_device(const ls_handle* H) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    set_error("no current CUDA device");
    return LS_ECUDA;
  }
  if (dev != H->device) {
    char buf[128];
    snprintf(buf, sizeof(buf), "handle was built on device %d but device %d is current", H->device, dev);
    set_error(buf);
    return LS_EINVAL;
  }
  return LS_OK;
}

int dalloc(void** p, size_t bytes) {
  *p = nullptr;
  g_allocs.fetch_add(1, std::memory_order_relaxed);
  if (injected_alloc_failure()) {
    char buf[96];
    snprintf(buf, sizeof(buf), "device allocation of %zu bytes failed (injected)", bytes);
    set_error(buf);
    return LS_ENOMEM;
  }
  if (bytes == 0) bytes = 16;
  cudaMemPool_t pool;
  int rc = pool_for_current_device(&pool);
  if (rc) return rc;
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, g_alloc_stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    char buf[128];
    snprintf(buf, sizeof(buf), "device allocation of %zu bytes failed", bytes);
    set_error(buf);
    *p = nullptr;
    return LS_ENOMEM;
  }
  return LS_OK;
}

void dfree(void* p) {
  if (p) cudaFreeAsync(p, g_alloc_stream);
}

int check_launch(const char* what) {
  debug_sync(__FILE__, __LINE__, what);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    ls_set_last_cuda_error(e, what, __FILE__, __LINE__);
    return LS_ECUDA;
  }
  return LS_OK;
}

}  // namespace ls

extern "C" {

void ls_default_opts(ls_opts* o) {
  o->order_matvec = 10;
  o->order_precond = 4;
  o->leaf_side = 8;
  o->proxy_width = 0;
  o->precision = LS_FP32;
  o->gmres_maxit = 100;
  o->gmres_tol = 1e-10;
  o->merge_pivoting = 0;
  o->top_uncompressed = 0;
  o->id_method = LS_ID_AUTO;
  o->wait_limit = 0;
  o->woodbury = 1;
  o->rhs_block = 0;
  o->reuse_compression = 0;
}

const char* ls_strerror(int code) {
  switch (code) {
    case LS_OK: return "ok";
    case LS_EINVAL: return "invalid argument";
    case LS_ENOMEM: return "device out of memory";
    case LS_ECUDA: return "CUDA error";
    case LS_ESINGULAR: return "zero pivot in a local inverse";
    case LS_ENOCONV: return "GMRES did not reach the tolerance";
    case LS_ETIMEOUT: return "device-side wait timed out";
    default: return "unknown error";
  }
}

const char* ls_last_error(void) { return g_last_error.c_str(); }

long long ls_kernel_launches(void) { return ls::g_launches.load(); }

long long ls_allocations(void) { return ls::allocation_count(); }

int ls_fault_inject(const char* spec) {
  if (ls::parse_fault(spec)) {
    set_error("unknown fault spec");
    return LS_EINVAL;
  }
  return LS_OK;
}

int ls_row_id(const void* A, int m, int p, double eps, int precision, int* k, int* piv, void* U, void* stream) {
  return ls_row_id_ex(A, m, p, eps, precision, LS_ID_GREEDY, k, piv, U, stream);
}

int ls_row_id_ex(const void* A, int m, int p, double eps, int precision, int method, int* k, int* piv, void* U,
                 void* stream) {
  if (!A || !k || !piv || m < 1 || m >= (1 << 20) || p < 1 || !(eps > 0 && eps < 1) ||
      (precision != LS_FP64 && precision != LS_FP32) || method < LS_ID_AUTO || method > LS_ID_BLOCKED) {
    set_error("invalid ls_row_id argument");
    return LS_EINVAL;
  }
  *k = 0;
  ls::StreamScope scope((cudaStream_t)stream);
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  LS_CUDA_TRY(cudaGetDevice(&dev));
  LS_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const size_t bytesA = sizeof(ls::z64) * (size_t)m * p, bytesU = sizeof(ls::z64) * (size_t)m * std::min(m, p);
  Staged sa, su;
  int* sync_buf = nullptr;
  int rc = stage_in(A, bytesA, st, &sa);
  if (!rc && U) rc = stage_out_alloc(U, bytesU, &su);
  if (!rc) rc = ls::dalloc((void**)&sync_buf, 256);
  if (!rc) rc = ls::row_id(sa.dev, m, p, eps, precision, method, nsm, sync_buf, st, k, piv, U ? su.dev : nullptr);
  if (!rc && U && su.owned && *k > 0) {
    cudaError_t e = cudaMemcpyAsync(U, su.dev, sizeof(ls::z64) * (size_t)m * *k, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) {
      ls_set_last_cuda_error(e, "ls_row_id U copy", __FILE__, __LINE__);
      rc = LS_ECUDA;
    }
  }
  cudaStreamSynchronize(st);
  release(&sa);
  release(&su);
  if (sync_buf) ls::dfree(sync_buf);
  cudaStreamSynchronize(st);
  return rc;
}

int ls_cgemm_c64(int engine, int ta, int tb, int M, int N, int K, const float* alpha, const void* A, int lda,
                 long long sA, const void* B, int ldb, long long sB, const float* beta, void* C, int ldc,
                 long long sC, int batch, void* stream) {
  if (engine < 0 || engine > 3 || M < 0 || N < 0 || K < 0 || batch < 0 || !alpha || !beta || !A || !B || !C)
    return LS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  ls::StreamScope scope(st);
  ls::c32 al = ls::mk<float>(alpha[0], alpha[1]), be = ls::mk<float>(beta[0], beta[1]);
  const ls::c32* a = static_cast<const ls::c32*>(A);
  const ls::c32* b = static_cast<const ls::c32*>(B);
  ls::c32* c = static_cast<ls::c32*>(C);
  if (engine == 0) return ls::simt_cgemm(st, ta, tb, M, N, K, al, a, lda, sA, b, ldb, sB, be, c, ldc, sC, batch);
  static int* d_flag = nullptr;  // per-process timeout flag of the tensor-core kernel
  if (!d_flag) {
    if (cudaMalloc(&d_flag, sizeof(int)) != cudaSuccess) return LS_ENOMEM;
    cudaMemset(d_flag, 0, sizeof(int));
  }
  int rc = ls::tc_cgemm(st, ta, tb, M, N, K, al, a, lda, sA, b, ldb, sB, be, c, ldc, sC, batch, engine - 1, d_flag);
  if (rc) return rc;
  int flag = 0;
  LS_CUDA_TRY(cudaMemcpyAsync(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  LS_CUDA_TRY(cudaStreamSynchronize(st));
  return flag ? flag : LS_OK;
}

void ls_free(ls_handle* H) {
  if (!H) return;
  int cur = -1;
  if (H->device >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != H->device) cudaSetDevice(H->device);
  if (H->side_stream) {  // the spectrum set-up may still run after a failed build
    cudaStreamSynchronize(H->side_stream);
    cudaStreamDestroy(H->side_stream);
    H->side_stream = nullptr;
  }
  ls::StreamScope scope(H->stream);
  auto f = [](void* p) { ls::dfree(p); };
  f(H->spec);
  f(H->tw_x);
  f(H->tw_y);
  f(H->b);
  f(H->ktab);
  f(H->convbuf);
  for (auto& lv : H->lev) {
    f(lv.U);
    f(lv.Gsib);
    f(lv.X);
    f(lv.S);
    f(lv.UT);
    f(lv.GT);
    f(lv.XT);
    f(lv.ST);
    f(lv.GL);
    f(lv.GR);
    f(lv.GLT);
    f(lv.GRT);
    f(lv.XLT);
  }
  f(H->Gleaf);
  f(H->XBU);
  f(H->XBUT);
  f(H->apply_ops_t);
  f(H->work);
  f(H->bwork);
  f(H->sync_buf);
  f(H->d_err);
  f(H->gm);
  f(H->bgm);
  for (void* p : H->bslab) f(p);
  f(H->slots);
  f(H->apply_ops);
  f(H->apply_bar);
  f(H->rx);
  f(H->Rrec);
  if (H->apply_exec) cudaGraphExecDestroy(H->apply_exec);
  if (H->inv_stream) cudaStreamDestroy(H->inv_stream);
  if (H->ext_stream) cudaStreamDestroy(H->ext_stream);
  const int dev = H->device;
  delete H;
  if (dev >= 0 && cur >= 0 && cur != dev) cudaSetDevice(cur);  // the caller's current device is left as it was
}

// Compression and merges run as a two-stage pipeline: this thread compresses
// the levels L..1 on the caller's stream (the ID kernels occupy at most one
// thread-block cluster or one cooperative grid); a worker thread runs the leaf
// build and the merges on a second stream, each level starting as soon as the
// compression of the level it needs has been recorded, so that the merges of
// the lower levels overlap the IDs of the upper ones.  The caller's stream
// waits for the last merge.
static int build_pipelined(ls_handle* H, cudaStream_t st) {
  const int L = H->L;
  // the compression is the critical path: its stream gets the highest priority, so
  // that its blocks are scheduled first when the merges occupy the SMs
  int prio_low = 0, prio_high = 0;
  LS_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
  // su: the ID back substitutions (a level's U), beside the next level's ID on sc
  cudaStream_t sm = nullptr, sc = nullptr, su = nullptr;
  LS_CUDA_TRY(cudaStreamCreateWithPriority(&sm, cudaStreamNonBlocking, prio_low));
  LS_CUDA_TRY(cudaStreamCreateWithPriority(&sc, cudaStreamNonBlocking, prio_high));
  LS_CUDA_TRY(cudaStreamCreateWithPriority(&su, cudaStreamNonBlocking, prio_high));
  std::vector<cudaEvent_t> ev(L + 4, nullptr);
  for (auto& e : ev) LS_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  LS_CUDA_TRY(cudaEventRecord(ev[0], st));  // kernel table, spectrum, b: ready for both stages
  LS_CUDA_TRY(cudaStreamWaitEvent(sc, ev[0], 0));
  LS_CUDA_TRY(cudaStreamWaitEvent(sm, ev[0], 0));
  // ss[0], ss[1]: each level's sibling block, transposes and low-rank factors
  // (sibling_prepare), made as soon as the level is compressed by two more
  // threads, one for the even and one for the odd levels: the levels kept
  // uncompressed at the top are ready together with the first compressed one
  // below them, and their factorisations then run side by side
  cudaStream_t ss[2] = {nullptr, nullptr};
  for (auto& q : ss) LS_CUDA_TRY(cudaStreamCreateWithPriority(&q, cudaStreamNonBlocking, prio_low));
  std::vector<cudaEvent_t> evs(L + 1, nullptr);
  for (auto& e : evs) LS_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  std::mutex mu;
  std::condition_variable cv;
  int ready = L + 1;                    // the lowest level index compressed so far (levels finish from L down to 1)
  std::vector<char> sib_done(L + 2, 0);  // the levels whose sibling data are made
  bool abort = false;
  int mrc = LS_OK, src = LS_OK;
  std::string merr, serr;
  auto sibling_worker = [&](int parity) {
    cudaStream_t q = ss[parity];
    ls::StreamScope scope(q);
    for (int l = L; l >= 1; --l) {
      if ((l & 1) != parity) continue;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] { return abort || ready <= l; });
        if (abort) return;
      }
      int r = cudaStreamWaitEvent(q, ev[l], 0) == cudaSuccess ? ls::sibling_prepare(H, l, q) : LS_ECUDA;
      if (!r && cudaEventRecord(evs[l], q) != cudaSuccess) r = LS_ECUDA;
      std::lock_guard<std::mutex> lk(mu);
      if (r) {
        if (!src) {
          src = r;
          serr = ls_last_error();
        }
        abort = true;
      } else {
        sib_done[l] = 1;
      }
      cv.notify_all();
      if (r) return;
    }
  };
  std::thread sibling_even(sibling_worker, 0), sibling_odd(sibling_worker, 1);
  std::thread merger([&] {
    ls::StreamScope scope(sm);
    auto wait_level = [&](int level) -> int {
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] { return abort || ready <= level; });
        if (abort) return LS_EINVAL;
      }
      LS_CUDA_TRY(cudaStreamWaitEvent(sm, ev[level], 0));
      return LS_OK;
    };
    auto wait_sibling = [&](int level) -> int {
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] { return abort || sib_done[level]; });
        if (abort) return LS_EINVAL;
      }
      LS_CUDA_TRY(cudaStreamWaitEvent(sm, evs[level], 0));
      return LS_OK;
    };
    int r = ls::hbs_build(H, sm, wait_level, wait_sibling);
    if (r) merr = ls_last_error();
    std::lock_guard<std::mutex> lk(mu);
    mrc = r;
    if (r) abort = true;
    cv.notify_all();
  });
  auto level_done = [&](int level) {
    cudaEventRecord(ev[level], su);  // su has passed sc's work of this level (compress orders it)
    {
      std::lock_guard<std::mutex> lk(mu);
      ready = level;
    }
    cv.notify_all();
  };
  int rc;
  ls::host_mark("pipeline_started");
  {
    ls::StreamScope scope(sc);
    rc = ls::compress(H, sc, level_done, su);
  }
  ls::host_mark("compress_returned");
  if (rc) {
    std::lock_guard<std::mutex> lk(mu);
    abort = true;
  }
  cv.notify_all();
  merger.join();
  sibling_even.join();
  sibling_odd.join();
  ls::host_mark("merges_joined");
  if (!rc && src) {  // the sibling worker's failure aborted the merges
    rc = src;
    set_error(serr.c_str());
  }
  if (!rc && mrc) {
    rc = mrc;
    set_error(merr.c_str());
  }
  cudaEventRecord(ev[L + 1], sm);
  cudaEventRecord(ev[L + 2], sc);
  cudaEventRecord(ev[L + 3], su);
  cudaStreamWaitEvent(st, ev[L + 3], 0);
  cudaStreamWaitEvent(st, ev[L + 1], 0);
  cudaStreamWaitEvent(st, ev[L + 2], 0);
  for (auto q : ss) {  // the wait takes the event's state at the call: one event serves both
    cudaEventRecord(evs[0], q);
    cudaStreamWaitEvent(st, evs[0], 0);
  }
  for (auto& e : ev) cudaEventDestroy(e);
  for (auto& e : evs) cudaEventDestroy(e);
  cudaStreamDestroy(sm);
  cudaStreamDestroy(sc);
  cudaStreamDestroy(su);
  for (auto q : ss) cudaStreamDestroy(q);
  return rc;
}

static int build_impl(const ls_grid* grid, int nprob, double kappa, const double* b, double tol, const ls_opts* opts,
                      cudaStream_t st, ls_handle** out) {
  ls::g_build_t0 = std::chrono::steady_clock::now();
  ls_handle* H = new ls_handle();
  *out = H;
  H->nprob = nprob;
  int rc = ls::setup_handle(H, grid, kappa, b, tol, opts, st);
  if (rc) return rc;
  ls::SpinLimitScope spin_scope(H->spin_limit);
  // the compression depends on kappa, h, the tree, tol, order and ring only: with
  // reuse_compression a cached one replaces the IDs (Sec. 3.2)
  bool reused = false;
  if (H->opts.reuse_compression && (rc = ls::cache_fetch(H, st, &reused))) return rc;
  ls::host_mark("setup_done");
  if (reused) {
    H->compression_reused = 1;
    rc = ls::hbs_build(H, st);
  } else {
    rc = build_pipelined(H, st);
    if (!rc && H->opts.reuse_compression) rc = ls::cache_store(H, st);
  }
  ls::host_mark("pipeline_done");
  return rc;
}

}  // extern "C"

// Everything of ls_build up to the factors: options, tree, ring, quadrature
// corrections, b on the device (checked), kernel table, FFT spectrum (on a side
// stream, waited for before returning).  ls_load uses it too.
int ls::setup_handle(ls_handle* H, const ls_grid* grid, double kappa, const double* b, double tol,
                     const ls_opts* opts, cudaStream_t st) {
  H->stream = st;
  H->grid = *grid;
  H->kappa = kappa;
  H->tol = tol;
  if (opts)
    H->opts = *opts;
  else
    ls_default_opts(&H->opts);
  const ls_opts& o = H->opts;
  if (!valid_order(o.order_matvec) || !valid_order(o.order_precond) || o.order_precond == 2 || o.leaf_side < 2 ||
      o.gmres_maxit < 1 || !(o.gmres_tol > 0) || (o.precision < LS_FP64 || o.precision > LS_FP16SPLIT) ||
      o.precision == LS_TF32 ||
      o.proxy_width < 0 || o.merge_pivoting < 0 || o.merge_pivoting > 1 ||
      o.top_uncompressed < 0 || o.id_method < LS_ID_AUTO || o.id_method > LS_ID_BLOCKED || o.wait_limit < 0 ||
      o.rhs_block < 0 || o.woodbury < 0 || o.woodbury > 2 || o.reuse_compression < 0 || o.reuse_compression > 1) {
    set_error("invalid ls_opts");
    return LS_EINVAL;
  }
  H->prec = o.precision;
  H->s = o.leaf_side;
  H->spin_limit = o.wait_limit > 0 ? (long long)o.wait_limit : ls::kSpinLimit;
  ls::SpinLimitScope spin_scope(H->spin_limit);
  // tree: cuts alternate vertical / horizontal until square leaves of side s
  {
    int w = grid->nx, h = grid->ny, L = 0;
    H->lev.clear();
    LevelData root;
    root.w = w;
    root.h = h;
    H->lev.push_back(root);
    while (!(w == H->s && h == H->s)) {
      if (L % 2 == 0) {
        if (w % 2 || w / 2 < H->s) break;
        w /= 2;
      } else {
        if (h % 2 || h / 2 < H->s) break;
        h /= 2;
      }
      ++L;
      LevelData lv;
      lv.w = w;
      lv.h = h;
      H->lev.push_back(lv);
      if (L > 30) break;
    }
    if (!(w == H->s && h == H->s) || L < 1) {
      set_error("grid does not split into 2^L square leaves of side leaf_side with alternating cuts");
      return LS_EINVAL;
    }
    H->L = L;
  }
  // proxy ring width: Table 1 (1: ~1e-4, 2: ~1e-10, 3: full precision), and at
  // least one uncorrected layer beyond the correction stencil radius
  int ring = o.proxy_width;
  if (ring == 0) {
    ring = tol >= 1e-3 ? 1 : (tol >= 1e-9 ? 2 : 3);
    if (tol < 1e-3 && ring < 2) ring = 2;
    int r = o.order_precond == 4 ? 0 : o.order_precond == 6 ? 1 : o.order_precond == 8 ? 2 : 3;
    ring = std::max(ring, r + 1);
  }
  H->ring = ring;
  {
    int dev = 0;
    LS_CUDA_TRY(cudaGetDevice(&dev));
    LS_CUDA_TRY(cudaDeviceGetAttribute(&H->nsm, cudaDevAttrMultiProcessorCount, dev));
    H->device = dev;
  }
  // corrected-quadrature weights (host, Sec. 2.2)
  const double kh = kappa * grid->h;
  for (int which = 0; which < 2; ++which) {
    ls::QuadCorr q;
    int order = which == 0 ? o.order_precond : o.order_matvec;
    if (ls::quad_corrections(order, kh, &q)) {
      set_error("unsupported quadrature order");
      return LS_EINVAL;
    }
    ls::KernelSpec& ks = which == 0 ? H->ks_prec : H->ks_mv;
    ks.kappa = kappa;
    ks.h = grid->h;
    ks.npts = q.npts;
    for (int i = 0; i < 25; ++i) {
      ks.m1[i] = q.m1[i];
      ks.m2[i] = q.m2[i];
      ks.wr[i] = q.wr[i];
      ks.wi[i] = q.wi[i];
    }
  }
  int rc;
  const long long N = (long long)grid->nx * grid->ny * H->nprob;  // the problems' potentials, stacked
  if ((rc = ls::dalloc((void**)&H->b, sizeof(double) * N))) return rc;
  LS_CUDA_TRY(cudaMemcpyAsync(H->b, b, sizeof(double) * N, cudaMemcpyDefault, st));
  if (ls::take_nan_b_fault()) {  // injected: as if b held a NaN
    const double nan = std::numeric_limits<double>::quiet_NaN();
    LS_CUDA_TRY(cudaMemcpyAsync(H->b, &nan, sizeof(double), cudaMemcpyHostToDevice, st));
    LS_CUDA_TRY(cudaStreamSynchronize(st));
  }
  if ((rc = ls::dalloc((void**)&H->sync_buf, 256))) return rc;
  if ((rc = ls::dalloc((void**)&H->d_err, sizeof(int) * 4))) return rc;
  LS_CUDA_TRY(cudaMemsetAsync(H->d_err, 0, sizeof(int) * 4, st));
  count_launch();
  check_b_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(H->b, N, H->d_err + 1);
  if ((rc = ls::kernel_table_setup(H, st))) return rc;
  // the FFT matvec's kernel spectrum is needed by the solve, not by the build:
  // it is computed on a side stream beside the build
  LS_CUDA_TRY(cudaStreamCreateWithFlags(&H->side_stream, cudaStreamNonBlocking));
  cudaEvent_t ev_side;
  LS_CUDA_TRY(cudaEventCreateWithFlags(&ev_side, cudaEventDisableTiming));
  LS_CUDA_TRY(cudaEventRecord(ev_side, st));
  LS_CUDA_TRY(cudaStreamWaitEvent(H->side_stream, ev_side, 0));
  {
    ls::StreamScope side(H->side_stream);
    rc = ls::conv_setup(H, H->side_stream);
  }
  if (rc) {
    cudaEventDestroy(ev_side);
    return rc;
  }
  int* pin = static_cast<int*>(ls::pinned_scratch(sizeof(int)));
  if (!pin) return LS_ENOMEM;
  LS_CUDA_TRY(cudaMemcpyAsync(pin, H->d_err + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
  LS_CUDA_TRY(cudaStreamSynchronize(st));
  const int bad = pin[0];
  if (bad) {
    cudaEventDestroy(ev_side);
    set_error("b must be finite");
    return LS_EINVAL;
  }
  // the spectrum is short next to any build: the handle is complete on return, for any stream
  LS_CUDA_TRY(cudaStreamSynchronize(H->side_stream));
  cudaEventDestroy(ev_side);
  return LS_OK;
}

extern "C" {

int ls_build(const ls_grid* grid, double kappa, const double* b, double tol, const ls_opts* opts, void* stream,
             ls_handle** out) {
  return ls_build_many(grid, 1, kappa, b, tol, opts, stream, out);
}

int ls_build_many(const ls_grid* grid, int nprob, double kappa, const double* b, double tol, const ls_opts* opts,
                  void* stream, ls_handle** out) {
  if (!out) return LS_EINVAL;
  *out = nullptr;
  if (!grid || !b || !(kappa > 0) || !(tol > 0 && tol < 1) || grid->nx < 2 || grid->ny < 2 || !(grid->h > 0) ||
      nprob < 1 || nprob > 65535) {
    set_error("invalid ls_build argument");
    return LS_EINVAL;
  }
  ls::StreamScope scope((cudaStream_t)stream);
  ls_handle* H = nullptr;
  int rc = build_impl(grid, nprob, kappa, b, tol, opts, (cudaStream_t)stream, &H);
  if (rc) {
    cudaStreamSynchronize((cudaStream_t)stream);
    ls_free(H);
    return rc;
  }
  *out = H;
  return LS_OK;
}

static int conv_entry(ls_handle* H, const void* x, void* y, int nrhs, int mode, void* stream) {
  if (int rc = ls::check_device(H)) return rc;
  ls::StreamScope scope((cudaStream_t)stream);
  H->stream = (cudaStream_t)stream;
  cudaStream_t st = (cudaStream_t)stream;
  const int nvec = nrhs * H->nprob;  // grid vectors: nrhs sets of the handle's problems
  size_t bytes = sizeof(ls::z64) * (size_t)H->grid.nx * H->grid.ny * nvec;
  Staged sx, sy;
  int rc = stage_in(x, bytes, st, &sx);
  if (!rc) rc = stage_out_alloc(y, bytes, &sy);
  if (!rc) rc = ls::conv_apply(H, sx.dev, sy.dev, nvec, mode, st);
  if (!rc) rc = stage_out_finish(y, bytes, st, &sy);
  if (sx.owned || sy.owned) cudaStreamSynchronize(st);
  release(&sx);
  release(&sy);
  return rc;
}

int ls_matvec(ls_handle* H, const void* x, void* y, int nrhs, int transpose, void* stream) {
  if (!H || !x || !y || nrhs < 1 || (transpose != 0 && transpose != 1)) return LS_EINVAL;
  return conv_entry(H, x, y, nrhs, transpose ? ls::CONV_TRANSPOSE : ls::CONV_FORWARD, stream);
}

int ls_field(ls_handle* H, const void* sigma, void* u, int nrhs, void* stream) {
  if (!H || !sigma || !u || nrhs < 1) return LS_EINVAL;
  return conv_entry(H, sigma, u, nrhs, ls::CONV_FIELD, stream);
}

int ls_apply(ls_handle* H, const void* f, void* q, int nrhs, int transpose, void* stream) {
  if (!H || !f || !q || nrhs < 1 || (transpose != 0 && transpose != 1)) return LS_EINVAL;
  if (int rc = ls::check_device(H)) return rc;
  ls::StreamScope scope((cudaStream_t)stream);
  H->stream = (cudaStream_t)stream;
  cudaStream_t st = (cudaStream_t)stream;
  const int nvec = nrhs * H->nprob;  // grid vectors: nrhs sets of the handle's problems
  size_t bytes = sizeof(ls::z64) * (size_t)H->grid.nx * H->grid.ny * nvec;
  Staged sf, sq;
  int rc = stage_in(f, bytes, st, &sf);
  if (!rc) rc = stage_out_alloc(q, bytes, &sq);
  if (!rc) rc = ls::hbs_apply(H, sf.dev, sq.dev, nvec, transpose, st);
  if (!rc) rc = stage_out_finish(q, bytes, st, &sq);
  if (sf.owned || sq.owned) cudaStreamSynchronize(st);
  release(&sf);
  release(&sq);
  return rc;
}

static int solve_entry(ls_handle* H, const void* f, void* sigma, int nrhs, ls_solve_info* info, int transpose,
                       void* stream) {
  if (!H || !f || !sigma || nrhs < 1) return LS_EINVAL;
  if (int rc = ls::check_device(H)) return rc;
  ls::host_mark("solve_entered");
  ls::StreamScope scope((cudaStream_t)stream);
  H->stream = (cudaStream_t)stream;
  cudaStream_t st = (cudaStream_t)stream;
  const int nvec = nrhs * H->nprob;  // grid vectors: nrhs sets of the handle's problems
  size_t bytes = sizeof(ls::z64) * (size_t)H->grid.nx * H->grid.ny * nvec;
  Staged sf, ss;
  int rc = stage_in(f, bytes, st, &sf);
  if (!rc) rc = stage_out_alloc(sigma, bytes, &ss);
  int solve_rc = LS_OK;
  if (!rc) {
    solve_rc = ls::gmres_solve(H, sf.dev, ss.dev, nvec, info, transpose, st);
    if (solve_rc != LS_OK && solve_rc != LS_ENOCONV) rc = solve_rc;
  }
  if (!rc) rc = stage_out_finish(sigma, bytes, st, &ss);
  if (sf.owned || ss.owned) cudaStreamSynchronize(st);
  release(&sf);
  release(&ss);
  return rc ? rc : solve_rc;
}

int ls_solve(ls_handle* H, const void* f, void* sigma, int nrhs, ls_solve_info* info, void* stream) {
  return solve_entry(H, f, sigma, nrhs, info, 0, stream);
}

int ls_solve_transpose(ls_handle* H, const void* f, void* sigma, int nrhs, ls_solve_info* info, void* stream) {
  return solve_entry(H, f, sigma, nrhs, info, 1, stream);
}

int ls_rhs_plane_wave(ls_handle* H, const double* thetas, void* f, int nrhs, void* stream) {
  if (!H || !thetas || !f || nrhs < 1) return LS_EINVAL;
  if (int rc = ls::check_device(H)) return rc;
  ls::StreamScope scope((cudaStream_t)stream);
  H->stream = (cudaStream_t)stream;
  cudaStream_t st = (cudaStream_t)stream;
  const long long N = (long long)H->grid.nx * H->grid.ny;
  const int G = H->nprob;  // each angle gives one right-hand side per problem, with that problem's b
  size_t bytes = sizeof(ls::z64) * N * G * nrhs;
  Staged sf;
  int rc = stage_out_alloc(f, bytes, &sf);
  for (int r = 0; !rc && r < nrhs; ++r)
    for (int g = 0; !rc && g < G; ++g) {
      count_launch();
      rhs_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(H->b + g * N, H->grid.nx, H->grid.ny, H->grid.h,
                                                            H->grid.x0, H->grid.y0, H->kappa, cos(thetas[r]),
                                                            sin(thetas[r]), sf.dev + ((long long)r * G + g) * N);
      rc = ls::check_launch("rhs");
    }
  if (!rc) rc = stage_out_finish(f, bytes, st, &sf);
  release(&sf);
  return rc;
}

int ls_sync(ls_handle* H, void* stream) {
  if (!H) return LS_EINVAL;
  if (int rc = ls::check_device(H)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  int* pin = static_cast<int*>(ls::pinned_scratch(sizeof(int)));
  if (!pin) return LS_ENOMEM;
  LS_CUDA_TRY(cudaMemcpyAsync(pin, H->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  LS_CUDA_TRY(cudaStreamSynchronize(st));
  if (pin[0]) set_error("a device-side wait or local inverse of this handle failed");
  return pin[0];
}

int ls_get_build_info(const ls_handle* H, ls_build_info* info) {
  if (!H || !info) return LS_EINVAL;
  memset(info, 0, sizeof(*info));
  info->levels = H->L;
  for (int l = 0; l <= H->L && l < 32; ++l) info->ranks[l] = H->lev[l].k;
  info->proxy_width = H->ring;
  info->flops_build = H->flops_build + H->flops_sibling;
  info->flops_compress = H->flops_compress;
  info->bytes_apply = H->bytes_apply;
  info->factor_bytes = H->factor_bytes;
  info->pivot_fallbacks = H->pivot_fallbacks;
  for (int l = 0; l <= H->L && l < 32; ++l) info->sibling_ranks[l] = std::max(0, H->lev[l].gr);
  info->probe_resid_max = H->probe_resid_max;
  info->compression_reused = H->compression_reused;
  info->nx = H->grid.nx;
  info->ny = H->grid.ny;
  info->nprob = H->nprob;
  return LS_OK;
}

}  // extern "C"
