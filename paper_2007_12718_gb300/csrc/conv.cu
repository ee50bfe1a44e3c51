// FFT application of the corrected Nystrom operator (Sec. 2.2 last paragraph,
// Sec. 5): y = x + kappa^2 b .* (K * x), K the discrete kernel on lattice
// offsets |m1| < nx, |m2| < ny embedded in an Ly x Lx circulant, Lx and Ly the
// powers of two >= 2nx, 2ny (any length >= 2n - 1 holds the linear convolution;
// zeros between the positive and the negative offsets).
//
// Three passes over the padded array, FP64 throughout, no cuFFT:
//   1. rows:    zero-pad each grid row to Lx, forward DIF FFT
//               (natural order in, bit-reversed order out)  -> W[ny][Lx]
//   2. columns: each block takes C adjacent columns of W, zero-pads them to
//               Ly, forward DIF FFT, multiplies by the kernel spectrum
//               (looked up at the bit-reversed frequencies), inverse DIT FFT
//               (bit-reversed in, natural out), keeps the first ny rows
//   3. rows:    inverse DIT FFT of each W row, keeps the first nx entries and
//               writes y = x + kappa^2 b .* conv in the same pass.
// DIF-forward / DIT-inverse pairs need no bit-reversal permutations.  K is
// even in m1 and m2, so its spectrum is even too and only the quarter
// (Lx/2 + 1) x (Ly/2 + 1) is stored (1/(Lx Ly) folded in).
#include <mutex>

#include "handle.h"
#include "prof.h"

namespace ls {
namespace {

__device__ __forceinline__ int brev(int i, int logL) { return (int)(__brev((unsigned)i) >> (32 - logL)); }

// COUNT interleaved length-L transforms s[i*stride + c]; forward DIF.  COUNT is
// a compile-time constant so that the transform index needs no division.
template <int COUNT>
__device__ void fft_dif(z64* s, int L, int logL, int stride, const z64* tw) {
  constexpr int count = COUNT;
  for (int lh = logL - 1; lh >= 0; --lh) {
    int half = 1 << lh;
    int tstep = L >> (lh + 1);
    int nb = (L >> 1) * count;
    for (int t = threadIdx.x; t < nb; t += blockDim.x) {
      int c = t % count, b = t / count;
      int j = b & (half - 1), g = b >> lh;
      int i0 = (g << (lh + 1)) + j, i1 = i0 + half;
      z64 a = s[i0 * stride + c], bb = s[i1 * stride + c];
      s[i0 * stride + c] = a + bb;
      const z64 d = a - bb;
      // the last two stages' twiddles are 1 and e^{-i pi/2} = -i: no multiply
      if (lh == 0)
        s[i1 * stride + c] = d;
      else if (lh == 1)
        s[i1 * stride + c] = j ? mk<double>(d.im, -d.re) : d;
      else
        s[i1 * stride + c] = tw[j * tstep] * d;
    }
    __syncthreads();
  }
}

// inverse DIT (unnormalised), bit-reversed input, natural output.
template <int COUNT>
__device__ void fft_dit_inv(z64* s, int L, int logL, int stride, const z64* tw) {
  constexpr int count = COUNT;
  for (int lh = 0; lh < logL; ++lh) {
    int half = 1 << lh;
    int tstep = L >> (lh + 1);
    int nb = (L >> 1) * count;
    for (int t = threadIdx.x; t < nb; t += blockDim.x) {
      int c = t % count, b = t / count;
      int j = b & (half - 1), g = b >> lh;
      int i0 = (g << (lh + 1)) + j, i1 = i0 + half;
      const z64 a = s[i0 * stride + c], x = s[i1 * stride + c];
      // the first two stages' twiddles are 1 and e^{i pi/2} = i: no multiply
      z64 tt;
      if (lh == 0)
        tt = x;
      else if (lh == 1)
        tt = j ? mk<double>(-x.im, x.re) : x;
      else
        tt = conjz(tw[j * tstep]) * x;
      s[i0 * stride + c] = a + tt;
      s[i1 * stride + c] = a - tt;
    }
    __syncthreads();
  }
}

__global__ void twiddle_kernel(z64* tw, int L) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < L / 2) {
    double sn, cs;
    sincospi(-2.0 * (double)k / (double)L, &sn, &cs);
    tw[k] = mk<double>(cs, sn);
  }
}

// Pass 1: rows. in: [rhs][nrow][ld_in] (first nvalid entries used); out: [rhs][nrow][L].
// bsc (may be null): the input is scaled by kap2 * bsc[row][i] (the transposed
// operator convolves B x); right-hand side r takes the b of problem r mod nprob
// (bsc holds nprob potentials of nrow x nvalid).
__global__ void rows_fwd_kernel(const z64* in, int ld_in, int nvalid, long long in_rhs_stride, z64* out, long long out_rhs_stride, int L, int logL,
                                const z64* __restrict__ tw, const double* __restrict__ bsc, double kap2, int nprob) {
  extern __shared__ z64 sm[];
  z64* s = sm;
  z64* stw = sm + L;
  int row = blockIdx.x, rhs = blockIdx.y;
  const z64* src = in + rhs * in_rhs_stride + (long long)row * ld_in;
  if (bsc) bsc += (long long)(rhs % nprob) * gridDim.x * nvalid;
  for (int i = threadIdx.x; i < L / 2; i += blockDim.x) stw[i] = tw[i];
  for (int i = threadIdx.x; i < L; i += blockDim.x) {
    z64 v = i < nvalid ? src[i] : mk<double>(0.0, 0.0);
    if (bsc && i < nvalid) {
      const double bb = kap2 * bsc[(long long)row * nvalid + i];
      v = mk<double>(bb * v.re, bb * v.im);
    }
    s[i] = v;
  }
  __syncthreads();
  fft_dif<1>(s, L, logL, 1, stw);
  z64* dst = out + rhs * out_rhs_stride + (long long)row * L;
  for (int i = threadIdx.x; i < L; i += blockDim.x) dst[i] = s[i];
}

// Pass 2: C columns per block (C = 2: a 512-column array is 256 blocks, so every
// SM takes part in the FP64 butterflies).  W: [rhs][nrow_valid][Lx] (bit-reversed column order).
// mode 0: forward, multiply by the quarter spectrum, inverse, keep first nrow rows.
// mode 1: forward only over all Ly rows (spectrum set-up), output bit-reversed rows.
template <int C>
__global__ void cols_kernel(z64* __restrict__ W, long long rhs_stride, int Lx, int logLx, int nrow, int Ly,
                            int logLy, const z64* __restrict__ tw, const z64* __restrict__ spec, int nxq, int nyq,
                            int mode) {
  extern __shared__ z64 sm[];
  z64* s = sm;             // Ly * C
  z64* stw = sm + Ly * C;  // Ly / 2
  int c0 = blockIdx.x * C, rhs = blockIdx.y;
  z64* base = W + rhs * rhs_stride;
  for (int i = threadIdx.x; i < Ly / 2; i += blockDim.x) stw[i] = tw[i];
  for (int t = threadIdx.x; t < Ly * C; t += blockDim.x) {
    int i = t / C, c = t % C;
    s[t] = i < nrow ? base[(long long)i * Lx + c0 + c] : mk<double>(0.0, 0.0);
  }
  __syncthreads();
  fft_dif<C>(s, Ly, logLy, C, stw);
  if (mode == 1) {
    for (int t = threadIdx.x; t < Ly * C; t += blockDim.x) {
      int i = t / C, c = t % C;
      base[(long long)i * Lx + c0 + c] = s[t];
    }
    return;
  }
  for (int t = threadIdx.x; t < Ly * C; t += blockDim.x) {
    int i = t / C, c = t % C;
    int ky = brev(i, logLy), kx = brev(c0 + c, logLx);
    if (ky > nyq) ky = Ly - ky;
    if (kx > nxq) kx = Lx - kx;
    s[t] = s[t] * spec[(long long)ky * (nxq + 1) + kx];
  }
  __syncthreads();
  fft_dit_inv<C>(s, Ly, logLy, C, stw);
  for (int t = threadIdx.x; t < nrow * C; t += blockDim.x) {
    int i = t / C, c = t % C;
    base[(long long)i * Lx + c0 + c] = s[t];
  }
}

// Pass 3: rows inverse + epilogue (ConvMode): y = x + kappa^2 b .* conv
// (forward), y = x + conv (transpose: B was applied to the input), y = conv (field).
__global__ void rows_inv_kernel(const z64* __restrict__ W, long long w_rhs_stride, int L, int logL,
                                const z64* __restrict__ tw, const z64* __restrict__ x, const double* __restrict__ b,
                                double kap2, int nx, long long g_rhs_stride, z64* __restrict__ y, int mode, int nprob) {
  extern __shared__ z64 sm[];
  z64* s = sm;
  z64* stw = sm + L;
  int row = blockIdx.x, rhs = blockIdx.y;
  const z64* src = W + rhs * w_rhs_stride + (long long)row * L;
  b += (long long)(rhs % nprob) * gridDim.x * nx;  // the potential of this right-hand side's problem
  for (int i = threadIdx.x; i < L / 2; i += blockDim.x) stw[i] = tw[i];
  for (int i = threadIdx.x; i < L; i += blockDim.x) s[i] = src[i];
  __syncthreads();
  fft_dit_inv<1>(s, L, logL, 1, stw);
  long long off = rhs * g_rhs_stride + (long long)row * nx;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    z64 cv = s[i];
    if (mode == CONV_FIELD) {
      y[off + i] = cv;
    } else {
      const double bb = mode == CONV_FORWARD ? kap2 * b[(long long)row * nx + i] : 1.0;
      z64 xv = x[off + i];
      y[off + i] = mk<double>(xv.re + bb * cv.re, xv.im + bb * cv.im);
    }
  }
}

__global__ void kernel_table_kernel(z64* T, int tx, int ty, double kh, double h2) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)tx * ty) return;
  int i = (int)(t % tx), j = (int)(t / tx);
  z64 v = mk<double>(0.0, 0.0);
  if (i || j) {
    z64 g = green(kh * sqrt((double)i * i + (double)j * j));
    v = mk<double>(g.re * h2, g.im * h2);
  }
  T[t] = v;
}

// Fill the Ly x Lx circulant with K(m): index i <-> m1 = i (i < nx), i - Lx
// (i > Lx - nx), no offset (zero) in between.
__global__ void circulant_kernel(z64* C, int nx, int ny, int Lx, int Ly, KernelTable kt, KernelSpec ks) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)Lx * Ly) return;
  int i = (int)(t % Lx), j = (int)(t / Lx);
  z64 v = mk<double>(0.0, 0.0);
  const bool ix = i < nx || i > Lx - nx, jy = j < ny || j > Ly - ny;
  if (ix && jy) {
    int m1 = i < nx ? i : i - Lx;
    int m2 = j < ny ? j : j - Ly;
    v = table_entry(kt, ks, m1, m2);
  }
  C[t] = v;
}

// Quarter spectrum (frequencies 0..nxq, 0..nyq; nxq = Lx / 2, nyq = Ly / 2) in
// natural order from the bit-reversed full transform.
__global__ void quarter_kernel(const z64* F, int Lx, int logLx, int Ly, int logLy, int nxq, int nyq, z64* Q,
                               double scale) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)(nxq + 1) * (nyq + 1)) return;
  int kx = (int)(t % (nxq + 1)), ky = (int)(t / (nxq + 1));
  z64 v = F[(long long)brev(ky, logLy) * Lx + brev(kx, logLx)];
  Q[t] = mk<double>(v.re * scale, v.im * scale);
}

int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

int cols_per_block(int Ly) { return (size_t)Ly * 2 * sizeof(z64) <= 96 * 1024 ? 2 : 1; }

cudaError_t launch_cols(int C, unsigned nblk, unsigned nrhs, cudaStream_t st, z64* W, long long rhs_stride, int Lx,
                        int logLx, int nrow, int Ly, int logLy, const z64* tw, const z64* spec, int nxq, int nyq,
                        int mode) {
  const size_t smc = sizeof(z64) * ((size_t)Ly * C + Ly / 2);
  auto kfn = C == 2 ? cols_kernel<2> : cols_kernel<1>;
  cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smc);
  if (e != cudaSuccess) return e;
  count_launch();
  kfn<<<dim3(nblk, nrhs), 256, smc, st>>>(W, rhs_stride, Lx, logLx, nrow, Ly, logLy, tw, spec, nxq, nyq, mode);
  return cudaGetLastError();
}

}  // namespace

int kernel_table_setup(ls_handle* H, cudaStream_t st) {
  // offsets up to the grid size plus the proxy ring on both sides
  H->ktx = H->grid.nx + 2 * H->ring + 2;
  H->kty = H->grid.ny + 2 * H->ring + 2;
  int rc;
  if ((rc = dalloc((void**)&H->ktab, sizeof(z64) * (size_t)H->ktx * H->kty))) return rc;
  long long tot = (long long)H->ktx * H->kty;
  count_launch();
  kernel_table_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(H->ktab, H->ktx, H->kty, H->kappa * H->grid.h,
                                                                      H->grid.h * H->grid.h);
  return check_launch("kernel table");
}

int conv_setup(ls_handle* H, cudaStream_t st) {
  const int nx = H->grid.nx, ny = H->grid.ny;
  H->logLx = ilog2(2 * nx);
  H->logLy = ilog2(2 * ny);
  H->Lx = 1 << H->logLx;
  H->Ly = 1 << H->logLy;
  // one padded row (and column) with its twiddles must fit in a block's shared memory
  if (sizeof(z64) * ((size_t)std::max(H->Lx, H->Ly) * 3 / 2) > 200 * 1024) {
    set_last_error_text("grid too large for the FFT matvec (padded length above 8192)");
    return LS_EINVAL;
  }
  const int nxq = H->Lx / 2, nyq = H->Ly / 2;
  int rc;
  if ((rc = dalloc((void**)&H->tw_x, sizeof(z64) * H->Lx / 2))) return rc;
  if ((rc = dalloc((void**)&H->tw_y, sizeof(z64) * H->Ly / 2))) return rc;
  if ((rc = dalloc((void**)&H->spec, sizeof(z64) * (size_t)(nxq + 1) * (nyq + 1)))) return rc;
  count_launch();
  twiddle_kernel<<<(H->Lx / 2 + 255) / 256, 256, 0, st>>>(H->tw_x, H->Lx);
  count_launch();
  twiddle_kernel<<<(H->Ly / 2 + 255) / 256, 256, 0, st>>>(H->tw_y, H->Ly);
  z64* full = nullptr;
  size_t nfull = (size_t)H->Lx * H->Ly;
  if ((rc = dalloc((void**)&full, sizeof(z64) * nfull))) return rc;
  count_launch();
  circulant_kernel<<<(unsigned)((nfull + 255) / 256), 256, 0, st>>>(full, nx, ny, H->Lx, H->Ly,
                                                                   KernelTable{H->ktab, H->ktx, H->kty}, H->ks_mv);
  // rows: full length, in place through the same buffer (each block owns one row)
  size_t smr = sizeof(z64) * (H->Lx + H->Lx / 2);
  cudaFuncSetAttribute(rows_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smr);
  count_launch();
  rows_fwd_kernel<<<dim3(H->Ly, 1), 256, smr, st>>>(full, H->Lx, H->Lx, 0, full, 0, H->Lx, H->logLx, H->tw_x,
                                                    nullptr, 0.0, 1);
  int C = cols_per_block(H->Ly);
  LS_CUDA_TRY(launch_cols(C, H->Lx / C, 1, st, full, 0, H->Lx, H->logLx, H->Ly, H->Ly, H->logLy, H->tw_y, nullptr,
                          nxq, nyq, 1));
  size_t nq = (size_t)(nxq + 1) * (nyq + 1);
  count_launch();
  quarter_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(full, H->Lx, H->logLx, H->Ly, H->logLy, nxq, nyq,
                                                              H->spec, 1.0 / ((double)H->Lx * H->Ly));
  if ((rc = check_launch("conv_setup"))) return rc;
  ls::dfree(full);  // stream-ordered: released after the kernels above
  return LS_OK;
}

int conv_apply(ls_handle* H, const z64* x, z64* y, int nrhs, int mode, cudaStream_t st) {
  const int nx = H->grid.nx, ny = H->grid.ny;
  int rc;
  if (H->convbuf_rhs < nrhs) {
    if (H->convbuf) ls::dfree(H->convbuf);
    H->convbuf = nullptr;
    H->convbuf_rhs = 0;
    if ((rc = dalloc((void**)&H->convbuf, sizeof(z64) * (size_t)ny * H->Lx * nrhs))) return rc;
    H->convbuf_rhs = nrhs;
  }
  long long g_stride = (long long)nx * ny, w_stride = (long long)ny * H->Lx;
  size_t smr = sizeof(z64) * (H->Lx + H->Lx / 2);
  cudaFuncSetAttribute(rows_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smr);
  cudaFuncSetAttribute(rows_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smr);
  // algorithmic counts per launch: 5 L log2 L flops per length-L FFT, 16-byte complex entries
  const double N = (double)nx * ny, W = (double)ny * H->Lx, R = nrhs;
  int tk = prof_begin(st);
  count_launch();
  rows_fwd_kernel<<<dim3(ny, nrhs), 256, smr, st>>>(x, nx, nx, g_stride, H->convbuf, w_stride, H->Lx, H->logLx,
                                                    H->tw_x, mode == CONV_TRANSPOSE ? H->b : nullptr,
                                                    H->kappa * H->kappa, H->nprob);
  prof_end(tk, PR_MV_ROWS_FWD, st, R * (16.0 * N + 16.0 * W) + (mode == CONV_TRANSPOSE ? 8.0 * N : 0.0),
           R * 5.0 * W * H->logLx);
  int C = cols_per_block(H->Ly);
  tk = prof_begin(st);
  LS_CUDA_TRY(launch_cols(C, H->Lx / C, nrhs, st, H->convbuf, w_stride, H->Lx, H->logLx, ny, H->Ly, H->logLy, H->tw_y,
                          H->spec, H->Lx / 2, H->Ly / 2, 0));
  prof_end(tk, PR_MV_COLS, st, R * 32.0 * W + 16.0 * (H->Lx / 2 + 1.0) * (H->Ly / 2 + 1.0),
           R * (2.0 * 5.0 * H->Lx * (double)H->Ly * H->logLy + 6.0 * H->Lx * (double)H->Ly));
  tk = prof_begin(st);
  count_launch();
  rows_inv_kernel<<<dim3(ny, nrhs), 256, smr, st>>>(H->convbuf, w_stride, H->Lx, H->logLx, H->tw_x, x, H->b,
                                                    H->kappa * H->kappa, nx, g_stride, y, mode, H->nprob);
  prof_end(tk, PR_MV_ROWS_INV, st,
           R * (16.0 * W + (mode == CONV_FIELD ? 16.0 : mode == CONV_TRANSPOSE ? 32.0 : 40.0) * N),
           R * 5.0 * W * H->logLx);
  return check_launch("conv_apply");
}

}  // namespace ls

// ---------------------------------------------------------------------------
// ls_matvec_noalloc: the FFT matvec with its scratch in a fixed device array.
//
// Some callers cannot allocate device memory at the point where they apply
// the operator: code whose framework has already reserved the free device
// memory in its own pool (a cudaMalloc there fails or fragments the pool),
// latency-critical loops that cannot afford the implicit device
// synchronisation of cudaMalloc/cudaFree, and programs that must stay within a
// memory budget fixed at start-up.  ls_matvec may allocate (its padded FFT
// buffer grows with nrhs, and host vectors are staged through device memory);
// this entry point allocates nothing: the padded buffer lives in the
// file-scope array below, which every GPU that loads the library holds until
// the process exits.
namespace {

constexpr long long kNoAllocScratchElems = 1LL << 18;  // complex128 entries: 4 MiB
static __device__ __align__(256) ls::z64 g_noalloc_scratch[kNoAllocScratchElems];

constexpr int kMaxDevices = 64;
ls::z64* g_noalloc_ptr[kMaxDevices] = {nullptr};
std::mutex g_noalloc_mu;

// Device address of the scratch array on the current device (host code only
// sees a host-side stand-in for the symbol, so the address is looked up once
// per device, with that device current).
int noalloc_scratch(ls::z64** out) {
  int dev = 0;
  LS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return LS_EINVAL;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    LS_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = static_cast<ls::z64*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return LS_OK;
}

// Device (or managed) memory of the current device, the device the scratch
// array's address belongs to.
bool on_device(const void* p) {
  cudaPointerAttributes a;
  int dev = -1;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" long long ls_matvec_noalloc_max_elems(void) { return kNoAllocScratchElems; }

extern "C" int ls_matvec_noalloc(ls_handle* H, const void* xv, void* yv, int nrhs, void* stream) {
  using namespace ls;
  if (!H || !xv || !yv || nrhs < 1) return LS_EINVAL;
  if (int rc = check_device(H)) return rc;
  if (H->nprob != 1) {
    set_last_error_text("ls_matvec_noalloc: handles of one problem only");
    return LS_EINVAL;
  }
  const int nx = H->grid.nx, ny = H->grid.ny;
  const long long need = (long long)nrhs * ny * H->Lx;
  if (need > kNoAllocScratchElems) {
    set_last_error_text("ls_matvec_noalloc: nrhs * ny * 2 nx exceeds the fixed scratch (2^18 complex128 entries)");
    return LS_EINVAL;
  }
  if (!on_device(xv) || !on_device(yv)) {
    set_last_error_text("ls_matvec_noalloc: x and y must be device pointers of the current device");
    return LS_EINVAL;
  }
  z64* W = nullptr;
  int rc = noalloc_scratch(&W);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const z64* x = static_cast<const z64*>(xv);
  z64* y = static_cast<z64*>(yv);
  long long g_stride = (long long)nx * ny, w_stride = (long long)ny * H->Lx;
  size_t smr = sizeof(z64) * (H->Lx + H->Lx / 2);
  LS_CUDA_TRY(cudaFuncSetAttribute(rows_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smr));
  LS_CUDA_TRY(cudaFuncSetAttribute(rows_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smr));
  count_launch();
  rows_fwd_kernel<<<dim3(ny, nrhs), 256, smr, st>>>(x, nx, nx, g_stride, W, w_stride, H->Lx, H->logLx, H->tw_x,
                                                    nullptr, 0.0, 1);
  int C = cols_per_block(H->Ly);
  LS_CUDA_TRY(launch_cols(C, H->Lx / C, nrhs, st, W, w_stride, H->Lx, H->logLx, ny, H->Ly, H->logLy, H->tw_y, H->spec,
                          H->Lx / 2, H->Ly / 2, 0));
  count_launch();
  rows_inv_kernel<<<dim3(ny, nrhs), 256, smr, st>>>(W, w_stride, H->Lx, H->logLx, H->tw_x, x, H->b, H->kappa * H->kappa,
                                                    nx, g_stride, y, ls::CONV_FORWARD, 1);
  return check_launch("ls_matvec_noalloc");
}
