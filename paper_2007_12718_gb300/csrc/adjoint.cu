// Receiver fields and the gradient of a receiver misfit with respect to b.
//
// The paper's discretisation (Eq. (1) for the field of the density, Eqs.
// (9)-(10) for the system (I + B (G + T)) sigma = f, f = -kappa^2 b u_inc)
// gives, for plane waves theta_r and receivers r_k outside the domain,
//   u_r(r_k) = sum_j R[k][j] sigma_r[j],   R[k][j] = h^2 G(|r_k - x_j|)
// (trapezoidal rule), and for J(b) = sum_{r,k} |u_r(r_k) - d_rk|^2
//   dJ/db_j = -2 kappa^2 sum_r Re(lambda_r[j] ((G + T) sigma_r + u_inc,r)[j]),
// where the adjoint state solves A^T lambda_r = R^T conj(u_r - d_r) (plain
// transpose: G + T is complex symmetric).  Both solves are the GMRES of
// gmres.cu, the adjoint one with A^T (FFT matvec, transpose mode) and the
// transposed HBS apply as preconditioner.
//
// R is evaluated once per handle by ls_set_receivers (nr x N complex128, one
// Hankel evaluation per entry, FP64).  u = sigma R^T is a long-K complex GEMM
// (K = N): it runs as S independent K-slices (the batch index of the SIMT
// GEMM) whose partial products are summed in a fixed order, so the result
// does not depend on the schedule.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "handle.h"

namespace ls {
namespace {

// R[k][j] = h^2 (i/4) H0(kappa |r_k - x_j|), x_j = (x0 + (i + 1/2) h, y0 + (j + 1/2) h).
__global__ void receiver_matrix_kernel(const double* __restrict__ rx, int nr, int nx, int ny, double h, double x0,
                                       double y0, double kappa, z64* __restrict__ R) {
  const long long N = (long long)nx * ny;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= N * nr) return;
  const int k = (int)(t / N);
  const long long j = t - (long long)k * N;
  const int ix = (int)(j % nx), iy = (int)(j / nx);
  const double dx = rx[2 * k] - (x0 + (ix + 0.5) * h), dy = rx[2 * k + 1] - (y0 + (iy + 0.5) * h);
  const z64 g = green(kappa * sqrt(dx * dx + dy * dy));
  R[t] = mk<double>(h * h * g.re, h * h * g.im);
}

// out[i] = sum_{c < S} part[c][i], i < n, summed in order c = 0, 1, ...
__global__ void sum_slices_kernel(const z64* __restrict__ part, int S, long long n, z64* __restrict__ out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  z64 a = mk<double>(0.0, 0.0);
  for (int c = 0; c < S; ++c) a = a + part[(long long)c * n + i];
  out[i] = a;
}

// rc = conj(u - d), *J = sum |u - d|^2 (one block, fixed reduction order).
__global__ void __launch_bounds__(1024) residual_kernel(const z64* __restrict__ u, const z64* __restrict__ d,
                                                        long long n, z64* __restrict__ rc, double* __restrict__ J) {
  double acc = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    const z64 r = u[i] - d[i];
    rc[i] = conjz(r);
    acc += abs2(r);
  }
  acc = warp_sum_r(acc);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    *J = s;
  }
}

// grad[j] = -2 kappa^2 sum_r Re(lam_r[j] (v_r[j] + u_inc,r[j])), u_inc = e^{i kappa (x1 cos + x2 sin)}.
__global__ void gradient_kernel(const z64* __restrict__ lam, const z64* __restrict__ v, const double* __restrict__ cs,
                                int nrhs, int nx, int ny, double h, double x0, double y0, double kappa,
                                double* __restrict__ grad) {
  const long long N = (long long)nx * ny;
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= N) return;
  const double x1 = x0 + ((int)(j % nx) + 0.5) * h, x2 = y0 + ((int)(j / nx) + 0.5) * h;
  double acc = 0.0;
  for (int r = 0; r < nrhs; ++r) {
    double sn, c;
    sincos(kappa * (x1 * cs[2 * r] + x2 * cs[2 * r + 1]), &sn, &c);
    const z64 w = v[r * N + j] + mk<double>(c, sn);
    const z64 l = lam[r * N + j];
    acc += l.re * w.re - l.im * w.im;
  }
  grad[j] = -2.0 * kappa * kappa * acc;
}

// K-slices of the long GEMM u = sigma R^T: S divides N, slices of at least 512.
int k_slices(long long N) {
  int S = 1;
  while (S < 256 && N % (2LL * S) == 0 && N / (2LL * S) >= 512) S *= 2;
  return S;
}

}  // namespace

int receiver_field(ls_handle* H, const z64* sigma, z64* u, int nrhs, cudaStream_t st) {
  const long long N = (long long)H->grid.nx * H->grid.ny;
  const int nr = H->nrec, S = k_slices(N);
  const long long Kc = N / S, n = (long long)nrhs * nr;
  z64* part = nullptr;
  int rc;
  if ((rc = dalloc((void**)&part, sizeof(z64) * (size_t)S * n))) return rc;
  // part[c] (nrhs x nr) = sigma[:, c Kc : (c+1) Kc] R[:, c Kc : (c+1) Kc]^T
  rc = simt_zgemm(st, false, true, nrhs, nr, (int)Kc, mk<double>(1.0, 0.0), sigma, (int)N, Kc, H->Rrec, (int)N, Kc,
                  mk<double>(0.0, 0.0), part, nr, n, S);
  if (!rc) {
    count_launch();
    sum_slices_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(part, S, n, u);
    rc = check_launch("receiver_field");
  }
  dfree(part);
  return rc;
}

int receiver_adjoint(ls_handle* H, const z64* v, z64* g, int nrhs, cudaStream_t st) {
  const long long N = (long long)H->grid.nx * H->grid.ny;
  // g (nrhs x N) = v (nrhs x nr) R (nr x N)
  return simt_zgemm(st, false, false, nrhs, (int)N, H->nrec, mk<double>(1.0, 0.0), v, H->nrec, 0, H->Rrec, (int)N, 0,
                    mk<double>(0.0, 0.0), g, (int)N, 0, 1);
}

}  // namespace ls

using ls::z64;

int ls_set_receivers(ls_handle* H, const double* rx, int nr, void* stream) {
  if (H && H->nprob != 1) {
    ls::set_last_error_text("receivers: handles of one problem only");
    return LS_EINVAL;
  }
  if (!H || nr < 0 || (nr > 0 && !rx)) return LS_EINVAL;
  if (int rc = ls::check_device(H)) return rc;
  ls::StreamScope scope((cudaStream_t)stream);
  H->stream = (cudaStream_t)stream;
  cudaStream_t st = (cudaStream_t)stream;
  const ls_grid& g = H->grid;
  for (int k = 0; k < nr; ++k) {  // a receiver on a grid node would need G(0)
    const double fx = (rx[2 * k] - g.x0) / g.h - 0.5, fy = (rx[2 * k + 1] - g.y0) / g.h - 0.5;
    if (!std::isfinite(fx) || !std::isfinite(fy)) return LS_EINVAL;
    if (fabs(fx - nearbyint(fx)) < 1e-9 && fabs(fy - nearbyint(fy)) < 1e-9 && nearbyint(fx) >= 0 &&
        nearbyint(fx) < g.nx && nearbyint(fy) >= 0 && nearbyint(fy) < g.ny) {
      ls::set_last_error_text("a receiver lies on a grid node");
      return LS_EINVAL;
    }
  }
  if (H->Rrec) ls::dfree(H->Rrec);
  if (H->rx) ls::dfree(H->rx);
  H->Rrec = nullptr;
  H->rx = nullptr;
  H->nrec = 0;
  if (nr == 0) return LS_OK;
  const long long N = (long long)g.nx * g.ny;
  int rc;
  if ((rc = ls::dalloc((void**)&H->rx, sizeof(double) * 2 * nr))) return rc;
  if ((rc = ls::dalloc((void**)&H->Rrec, sizeof(z64) * (size_t)N * nr))) return rc;
  LS_CUDA_TRY(cudaMemcpyAsync(H->rx, rx, sizeof(double) * 2 * nr, cudaMemcpyHostToDevice, st));
  count_launch();
  ls::receiver_matrix_kernel<<<(unsigned)((N * nr + 255) / 256), 256, 0, st>>>(H->rx, nr, g.nx, g.ny, g.h, g.x0, g.y0,
                                                                               H->kappa, H->Rrec);
  if ((rc = ls::check_launch("ls_set_receivers"))) return rc;
  LS_CUDA_TRY(cudaStreamSynchronize(st));  // rx (host) may be released on return
  H->nrec = nr;
  return LS_OK;
}

int ls_receiver_field(ls_handle* H, const void* sigma, void* u, int nrhs, void* stream) {
  if (H && H->nprob != 1) {
    ls::set_last_error_text("receivers: handles of one problem only");
    return LS_EINVAL;
  }
  if (!H || !sigma || !u || nrhs < 1 || H->nrec < 1) return LS_EINVAL;
  if (int rc = ls::check_device(H)) return rc;
  ls::StreamScope scope((cudaStream_t)stream);
  H->stream = (cudaStream_t)stream;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bs = sizeof(z64) * (size_t)H->grid.nx * H->grid.ny * nrhs, bu = sizeof(z64) * (size_t)H->nrec * nrhs;
  ls::Staged ss, su;
  int rc = ls::stage_in(sigma, bs, st, &ss);
  if (!rc) rc = ls::stage_out_alloc(u, bu, &su);
  if (!rc) rc = ls::receiver_field(H, ss.dev, su.dev, nrhs, st);
  if (!rc) rc = ls::stage_out_finish(u, bu, st, &su);
  if (ss.owned || su.owned) cudaStreamSynchronize(st);
  ls::release(&ss);
  ls::release(&su);
  return rc;
}

int ls_receiver_adjoint(ls_handle* H, const void* v, void* g, int nrhs, void* stream) {
  if (H && H->nprob != 1) {
    ls::set_last_error_text("receivers: handles of one problem only");
    return LS_EINVAL;
  }
  if (!H || !v || !g || nrhs < 1 || H->nrec < 1) return LS_EINVAL;
  if (int rc = ls::check_device(H)) return rc;
  ls::StreamScope scope((cudaStream_t)stream);
  H->stream = (cudaStream_t)stream;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bg = sizeof(z64) * (size_t)H->grid.nx * H->grid.ny * nrhs, bv = sizeof(z64) * (size_t)H->nrec * nrhs;
  ls::Staged sv, sg;
  int rc = ls::stage_in(v, bv, st, &sv);
  if (!rc) rc = ls::stage_out_alloc(g, bg, &sg);
  if (!rc) rc = ls::receiver_adjoint(H, sv.dev, sg.dev, nrhs, st);
  if (!rc) rc = ls::check_launch("ls_receiver_adjoint");
  if (!rc) rc = ls::stage_out_finish(g, bg, st, &sg);
  if (sv.owned || sg.owned) cudaStreamSynchronize(st);
  ls::release(&sv);
  ls::release(&sg);
  return rc;
}

int ls_misfit_gradient(ls_handle* H, const double* thetas, int nrhs, const void* d, double* J, void* grad,
                       ls_solve_info* info, void* stream) {
  if (H && H->nprob != 1) {
    ls::set_last_error_text("misfit gradient: handles of one problem only");
    return LS_EINVAL;
  }
  if (!H || !thetas || nrhs < 1 || !d || !J || H->nrec < 1) return LS_EINVAL;
  if (int rc = ls::check_device(H)) return rc;
  const bool want_grad = grad != nullptr;  // without it only J: no adjoint solve
  ls::StreamScope scope((cudaStream_t)stream);
  H->stream = (cudaStream_t)stream;
  cudaStream_t st = (cudaStream_t)stream;
  const ls_grid& gr = H->grid;
  const long long N = (long long)gr.nx * gr.ny, n = (long long)H->nrec * nrhs;
  const size_t bvec = sizeof(z64) * (size_t)N * nrhs;
  z64 *f = nullptr, *sig = nullptr, *lam = nullptr, *v = nullptr, *u = nullptr, *res = nullptr;
  double* dev_small = nullptr;  // J, then (cos, sin) per direction
  ls::Staged sd, sg;
  int rc = LS_OK, solve_rc = LS_OK;
  auto fail = [&](int r) {
    if (!rc) rc = r;
  };
  fail(ls::dalloc((void**)&f, bvec));
  if (!rc) fail(ls::dalloc((void**)&sig, bvec));
  if (!rc && want_grad) fail(ls::dalloc((void**)&lam, bvec));
  if (!rc && want_grad) fail(ls::dalloc((void**)&v, bvec));
  if (!rc) fail(ls::dalloc((void**)&u, sizeof(z64) * (size_t)n));
  if (!rc) fail(ls::dalloc((void**)&res, sizeof(z64) * (size_t)n));
  if (!rc) fail(ls::dalloc((void**)&dev_small, sizeof(double) * (1 + 2 * (size_t)nrhs)));
  if (!rc) fail(ls::stage_in(d, sizeof(z64) * (size_t)n, st, &sd));
  if (!rc && want_grad) fail(ls::stage_out_alloc(grad, sizeof(double) * (size_t)N, &sg));
  double* pin = nullptr;
  if (!rc) {
    pin = static_cast<double*>(ls::pinned_scratch(sizeof(double) * (1 + 2 * (size_t)nrhs)));
    if (!pin) fail(LS_ENOMEM);
  }
  if (!rc) {
    for (int r = 0; r < nrhs; ++r) {
      pin[1 + 2 * r] = cos(thetas[r]);
      pin[2 + 2 * r] = sin(thetas[r]);
    }
    cudaError_t e = cudaMemcpyAsync(dev_small + 1, pin + 1, sizeof(double) * 2 * nrhs, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // pin is reused below
    if (e != cudaSuccess) fail(LS_ECUDA);
  }
  // forward: sigma_r = A^-1 f_r, u = R sigma
  if (!rc) fail(ls_rhs_plane_wave(H, thetas, f, nrhs, stream));
  if (!rc) {
    int s = ls::gmres_solve(H, f, sig, nrhs, info, 0, st);
    if (s == LS_ENOCONV)
      solve_rc = s;
    else
      fail(s);
  }
  if (!rc) fail(ls::receiver_field(H, sig, u, nrhs, st));
  // J and the adjoint right-hand sides R^T conj(u - d)
  if (!rc) {
    count_launch();
    ls::residual_kernel<<<1, 1024, 0, st>>>(u, sd.dev, n, res, dev_small);
    fail(ls::check_launch("misfit residual"));
  }
  if (!rc && want_grad) fail(ls::receiver_adjoint(H, res, f, nrhs, st));
  if (!rc && want_grad) {
    int s = ls::gmres_solve(H, f, lam, nrhs, info ? info + nrhs : nullptr, 1, st);
    if (s == LS_ENOCONV)
      solve_rc = s;
    else
      fail(s);
  }
  // dJ/db = -2 kappa^2 sum_r Re(lambda_r ((G + T) sigma_r + u_inc,r))
  if (!rc && want_grad) fail(ls::conv_apply(H, sig, v, nrhs, ls::CONV_FIELD, st));
  if (!rc && want_grad) {
    count_launch();
    ls::gradient_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(lam, v, dev_small + 1, nrhs, gr.nx, gr.ny, gr.h,
                                                                     gr.x0, gr.y0, H->kappa,
                                                                     reinterpret_cast<double*>(sg.dev));
    fail(ls::check_launch("misfit gradient"));
  }
  if (!rc) {
    cudaError_t e = cudaMemcpyAsync(pin, dev_small, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
      fail(LS_ECUDA);
    else
      *J = pin[0];
  }
  if (!rc && want_grad) fail(ls::stage_out_finish(grad, sizeof(double) * (size_t)N, st, &sg));
  cudaStreamSynchronize(st);
  ls::release(&sd);
  ls::release(&sg);
  for (void* p : {(void*)f, (void*)sig, (void*)lam, (void*)v, (void*)u, (void*)res, (void*)dev_small})
    if (p) ls::dfree(p);
  return rc ? rc : solve_rc;
}
