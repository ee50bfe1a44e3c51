"""GB300 (sm_103a) HBS-preconditioned solver for the 2D Lippmann-Schwinger equation.

Method: Gopal & Martinsson, arXiv 2007.12718.  The compute path lives in the
C-ABI library ``_lib/libls.so`` (CUDA kernels, see ``include/ls.h``); this
module only marshals arguments to it through ctypes.  There is no CPU
fallback: if the library is missing or cannot load, every call raises.

Entry points (same names as the C ABI):
  ls_build(grid_n, h, kappa, b, tol, **opts) -> Handle
  ls_apply(handle, f, q, transpose=False)   q = M f or M^T f  (HBS inverse, Algorithm 2)
  ls_matvec(handle, x, y, transpose=False)  y = A x or A^T x, A = I + B(G+T)  (FFT, Sec. 5)
  ls_field(handle, sigma, u)                u = (G+T) sigma on the grid
  ls_solve(handle, f, sigma)                GMRES on A, right-preconditioned by M (Sec. 5)
  ls_solve_transpose(handle, f, sigma)      GMRES on A^T with M^T (adjoint solve)
  ls_rhs_plane_wave(handle, thetas, f)
  ls_set_receivers / ls_receiver_field / ls_receiver_adjoint / ls_misfit_gradient
  LSMisfit                                  torch.autograd.Function: J(b) and dJ/db
  ls_free(handle)
Vectors are complex128 arrays [nrhs][ny][nx] (or [ny][nx]); torch tensors on
the GPU are passed as device pointers, numpy arrays / CPU tensors as host
pointers (the library stages those itself).
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libls.so")

LS_OK, LS_EINVAL, LS_ENOMEM, LS_ECUDA, LS_ESINGULAR, LS_ENOCONV, LS_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
LS_FP64, LS_FP32, LS_TF32, LS_TF32X3, LS_FP16SPLIT = 0, 1, 2, 3, 4
LS_ID_AUTO, LS_ID_GREEDY, LS_ID_BLOCKED = 0, 1, 2

EXPORTED = ["ls_default_opts", "ls_build", "ls_apply", "ls_matvec", "ls_solve", "ls_rhs_plane_wave",
            "ls_get_build_info", "ls_free", "ls_strerror", "ls_last_error", "ls_profile_enable",
            "ls_profile_reset", "ls_profile_get", "ls_kernel_launches", "ls_matvec_noalloc",
            "ls_matvec_noalloc_max_elems", "ls_cgemm_c64", "ls_row_id", "ls_row_id_ex", "ls_field", "ls_solve_transpose",
            "ls_set_receivers", "ls_receiver_field", "ls_receiver_adjoint", "ls_misfit_gradient",
            "ls_measure_peak", "ls_allocations", "ls_fault_inject", "ls_sync"]


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("h", ctypes.c_double),
                ("x0", ctypes.c_double), ("y0", ctypes.c_double)]


class Opts(ctypes.Structure):
    _fields_ = [("order_matvec", ctypes.c_int), ("order_precond", ctypes.c_int), ("leaf_side", ctypes.c_int),
                ("proxy_width", ctypes.c_int), ("precision", ctypes.c_int), ("gmres_maxit", ctypes.c_int),
                ("gmres_tol", ctypes.c_double), ("merge_pivoting", ctypes.c_int),
                ("top_uncompressed", ctypes.c_int), ("id_method", ctypes.c_int), ("wait_limit", ctypes.c_int),
                ("woodbury", ctypes.c_int), ("reuse_compression", ctypes.c_int), ("rhs_block", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("resid_est", ctypes.c_double),
                ("resid_true", ctypes.c_double)]


class BuildInfo(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("ranks", ctypes.c_int * 32), ("proxy_width", ctypes.c_int),
                ("flops_build", ctypes.c_double), ("flops_compress", ctypes.c_double),
                ("bytes_apply", ctypes.c_double), ("factor_bytes", ctypes.c_double),
                ("pivot_fallbacks", ctypes.c_int), ("sibling_ranks", ctypes.c_int * 32),
                ("probe_resid_max", ctypes.c_double), ("compression_reused", ctypes.c_int),
                ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nprob", ctypes.c_int)]


class ProfileEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_longlong), ("total_ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("flops", ctypes.c_double)]


_lib = None


def load_library(path=LIB_PATH):
    """Load libls.so (raises if it is not built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is not built; run __graft_entry__.build() "
                           "or python -m paper_2007_12718_gb300.build")
    lib = ctypes.CDLL(path)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.ls_default_opts.argtypes = [ctypes.POINTER(Opts)]
    lib.ls_default_opts.restype = None
    lib.ls_build.argtypes = [ctypes.POINTER(Grid), dp, vp, dp, ctypes.POINTER(Opts), vp, ctypes.POINTER(vp)]
    lib.ls_build.restype = ip
    lib.ls_build_many.argtypes = [ctypes.POINTER(Grid), ip, dp, vp, dp, ctypes.POINTER(Opts), vp, ctypes.POINTER(vp)]
    lib.ls_build_many.restype = ip
    for name in ("ls_apply", "ls_matvec"):
        getattr(lib, name).argtypes = [vp, vp, vp, ip, ip, vp]
        getattr(lib, name).restype = ip
    for name in ("ls_solve", "ls_solve_transpose"):
        getattr(lib, name).argtypes = [vp, vp, vp, ip, ctypes.POINTER(SolveInfo), vp]
        getattr(lib, name).restype = ip
    for name in ("ls_field", "ls_receiver_field", "ls_receiver_adjoint"):
        getattr(lib, name).argtypes = [vp, vp, vp, ip, vp]
        getattr(lib, name).restype = ip
    lib.ls_set_receivers.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ip, vp]
    lib.ls_set_receivers.restype = ip
    lib.ls_misfit_gradient.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ip, vp, ctypes.POINTER(ctypes.c_double),
                                       vp, ctypes.POINTER(SolveInfo), vp]
    lib.ls_misfit_gradient.restype = ip
    lib.ls_rhs_plane_wave.argtypes = [vp, ctypes.POINTER(ctypes.c_double), vp, ip, vp]
    lib.ls_rhs_plane_wave.restype = ip
    lib.ls_get_build_info.argtypes = [vp, ctypes.POINTER(BuildInfo)]
    lib.ls_get_build_info.restype = ip
    lib.ls_free.argtypes = [vp]
    lib.ls_free.restype = None
    lib.ls_save.argtypes = [vp, ctypes.c_char_p, vp]
    lib.ls_save.restype = ip
    lib.ls_load.argtypes = [ctypes.c_char_p, vp, ctypes.POINTER(vp)]
    lib.ls_load.restype = ip
    lib.ls_compression_cache_clear.argtypes = []
    lib.ls_compression_cache_clear.restype = None
    lib.ls_strerror.argtypes = [ip]
    lib.ls_strerror.restype = ctypes.c_char_p
    lib.ls_last_error.argtypes = []
    lib.ls_last_error.restype = ctypes.c_char_p
    lib.ls_profile_enable.argtypes = [ip]
    lib.ls_profile_enable.restype = ip
    lib.ls_profile_reset.argtypes = []
    lib.ls_profile_reset.restype = ip
    lib.ls_profile_get.argtypes = [ctypes.POINTER(ProfileEntry), ip]
    lib.ls_profile_get.restype = ip
    lib.ls_matvec_noalloc.argtypes = [vp, vp, vp, ip, vp]
    lib.ls_matvec_noalloc.restype = ip
    lib.ls_matvec_noalloc_max_elems.argtypes = []
    lib.ls_matvec_noalloc_max_elems.restype = ctypes.c_longlong
    lib.ls_cgemm_c64.argtypes = [ip, ip, ip, ip, ip, ip, ctypes.POINTER(ctypes.c_float), vp, ip, ctypes.c_longlong,
                                 vp, ip, ctypes.c_longlong, ctypes.POINTER(ctypes.c_float), vp, ip, ctypes.c_longlong,
                                 ip, vp]
    lib.ls_cgemm_c64.restype = ip
    lib.ls_row_id.argtypes = [vp, ip, ip, dp, ip, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), vp, vp]
    lib.ls_row_id.restype = ip
    lib.ls_row_id_ex.argtypes = [vp, ip, ip, dp, ip, ip, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                 vp, vp]
    lib.ls_row_id_ex.restype = ip
    lib.ls_measure_peak.argtypes = [ip, ctypes.POINTER(ctypes.c_double), vp]
    lib.ls_measure_peak.restype = ip
    lib.ls_sync.argtypes = [vp, vp]
    lib.ls_sync.restype = ip
    lib.ls_allocations.argtypes = []
    lib.ls_allocations.restype = ctypes.c_longlong
    lib.ls_fault_inject.argtypes = [ctypes.c_char_p]
    lib.ls_fault_inject.restype = ip
    lib.ls_kernel_launches.argtypes = []
    lib.ls_kernel_launches.restype = ctypes.c_longlong
    _lib = lib
    return lib


class LSError(RuntimeError):
    def __init__(self, code, where):
        lib = load_library()
        msg = lib.ls_strerror(code).decode()
        last = lib.ls_last_error().decode()
        super().__init__(f"{where}: {msg} ({code}) {last}")
        self.code = code


def _check(code, where, allow=()):
    if code != LS_OK and code not in allow:
        raise LSError(code, where)
    return code


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(stream)
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return ctypes.c_void_p(0)


def _ptr(a, dtype, writable=False):
    """(pointer, keepalive, nelem) for a torch tensor or numpy array."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            want = {np.complex128: torch.complex128, np.float64: torch.float64}[dtype]
            if a.dtype != want or not a.is_contiguous():
                raise TypeError(f"expected a contiguous {want} tensor")
            return ctypes.c_void_p(a.data_ptr()), a, a.numel()
    except ImportError:
        pass
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise TypeError(f"expected a C-contiguous numpy array of {np.dtype(dtype)}")
    if writable and not a.flags["WRITEABLE"]:
        raise TypeError("output array is read-only")
    return ctypes.c_void_p(a.ctypes.data), a, a.size


class Handle:
    def __init__(self, ptr, n):
        self.ptr = ptr
        self.n = n        # grid points of one problem
        self.nprob = 1    # problems in the handle (ls_build with b of shape (nprob, ny, nx))

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.ls_free(self.ptr)
            self.ptr = None

    def info(self):
        bi = BuildInfo()
        _check(load_library().ls_get_build_info(self.ptr, ctypes.byref(bi)), "ls_get_build_info")
        return {"levels": bi.levels, "ranks": list(bi.ranks[: bi.levels + 1]), "proxy_width": bi.proxy_width,
                "flops_build": bi.flops_build, "flops_compress": bi.flops_compress,
                "bytes_apply": bi.bytes_apply, "factor_bytes": bi.factor_bytes,
                "pivot_fallbacks": bi.pivot_fallbacks, "probe_resid_max": bi.probe_resid_max,
                "sibling_ranks": list(bi.sibling_ranks[: bi.levels + 1]),
                "compression_reused": bool(bi.compression_reused), "nprob": bi.nprob}


def default_opts():
    o = Opts()
    load_library().ls_default_opts(ctypes.byref(o))
    return o


def ls_build(n, h, kappa, b, tol, order_matvec=10, order_precond=4, leaf_side=8, proxy_width=0,
             precision=LS_FP32, gmres_maxit=100, gmres_tol=1e-10, x0=0.0, y0=0.0, ny=None, stream=None,
             merge_pivoting=0, top_uncompressed=0, id_method=LS_ID_AUTO, wait_limit=0, rhs_block=0, woodbury=1, reuse_compression=0):
    """Compress G and build the HBS inverse (Sec. 3.2, Algorithm 1); b is [ny][nx] float64.
    rhs_block: right-hand sides per block of ls_apply / ls_solve (0 automatic, 1 one at a time).
    woodbury: 1 = merges in the Woodbury form where the sibling block's rank is low, 0 = Schur form.
    reuse_compression: 1 = take the compression from (and keep it in) the process-wide cache."""
    lib = load_library()
    g = Grid(n, n if ny is None else ny, h, x0, y0)
    o = Opts(order_matvec, order_precond, leaf_side, proxy_width, precision, gmres_maxit, gmres_tol,
             merge_pivoting, top_uncompressed, id_method, wait_limit, woodbury, reuse_compression, rhs_block)
    bp, keep, nb = _ptr(b, np.float64)
    if nb % (g.nx * g.ny):
        raise ValueError("b must hold whole grids")
    nprob = nb // (g.nx * g.ny)  # b of shape (nprob, ny, nx): nprob problems in one handle
    out = ctypes.c_void_p()
    _check(lib.ls_build_many(ctypes.byref(g), nprob, kappa, bp, tol, ctypes.byref(o), _stream(stream),
                             ctypes.byref(out)), "ls_build_many")
    H = Handle(out, g.nx * g.ny)
    H.nprob = nprob
    return H


def ls_save(handle, path, stream=None):
    """Write the built handle (inputs and every factor) to a file."""
    _check(load_library().ls_save(handle.ptr, str(path).encode(), _stream(stream)), "ls_save")


def ls_load(path, stream=None):
    """A handle restored from a file of ls_save, on the current device."""
    lib = load_library()
    out = ctypes.c_void_p()
    _check(lib.ls_load(str(path).encode(), _stream(stream), ctypes.byref(out)), "ls_load")
    H = Handle(out, 0)
    bi = BuildInfo()
    _check(lib.ls_get_build_info(H.ptr, ctypes.byref(bi)), "ls_get_build_info")
    H.n = bi.nx * bi.ny
    H.nprob = bi.nprob
    return H


def ls_compression_cache_clear():
    load_library().ls_compression_cache_clear()


def _nrhs(handle, nelem):
    """Sets of the handle's problems in a vector argument ([nrhs][nprob][ny][nx])."""
    per = handle.n * getattr(handle, "nprob", 1)
    if nelem % per:
        raise ValueError("vector size is not a multiple of the grid size times the number of problems")
    return nelem // per


def ls_apply(handle, f, q, transpose=False, stream=None):
    fp, k1, n = _ptr(f, np.complex128)
    qp, k2, _ = _ptr(q, np.complex128, True)
    _check(load_library().ls_apply(handle.ptr, fp, qp, _nrhs(handle, n), int(bool(transpose)), _stream(stream)),
           "ls_apply")
    return q


def ls_matvec(handle, x, y, transpose=False, stream=None):
    xp, k1, n = _ptr(x, np.complex128)
    yp, k2, _ = _ptr(y, np.complex128, True)
    _check(load_library().ls_matvec(handle.ptr, xp, yp, _nrhs(handle, n), int(bool(transpose)), _stream(stream)),
           "ls_matvec")
    return y


def ls_field(handle, sigma, u, stream=None):
    """u = (G+T) sigma on the grid (the scattered field of the density at the nodes)."""
    sp_, k1, n = _ptr(sigma, np.complex128)
    up, k2, _ = _ptr(u, np.complex128, True)
    _check(load_library().ls_field(handle.ptr, sp_, up, _nrhs(handle, n), _stream(stream)), "ls_field")
    return u


def _infos(infos):
    return [{"iterations": i.iterations, "converged": bool(i.converged), "resid_est": i.resid_est,
             "resid_true": i.resid_true} for i in infos]


def ls_solve(handle, f, sigma, stream=None, allow_noconv=False):
    fp, k1, n = _ptr(f, np.complex128)
    sp_, k2, _ = _ptr(sigma, np.complex128, True)
    nr = _nrhs(handle, n)
    infos = (SolveInfo * (nr * getattr(handle, "nprob", 1)))()
    _check(load_library().ls_solve(handle.ptr, fp, sp_, nr, infos, _stream(stream)), "ls_solve",
           allow=(LS_ENOCONV,) if allow_noconv else ())
    return _infos(infos)


def ls_solve_transpose(handle, f, sigma, stream=None, allow_noconv=False):
    """GMRES on A^T sigma = f, right-preconditioned by M^T (the adjoint solve)."""
    fp, k1, n = _ptr(f, np.complex128)
    sp_, k2, _ = _ptr(sigma, np.complex128, True)
    nr = _nrhs(handle, n)
    infos = (SolveInfo * (nr * getattr(handle, "nprob", 1)))()
    _check(load_library().ls_solve_transpose(handle.ptr, fp, sp_, nr, infos, _stream(stream)), "ls_solve_transpose",
           allow=(LS_ENOCONV,) if allow_noconv else ())
    return _infos(infos)


def ls_set_receivers(handle, receivers, stream=None):
    """Receivers (nr x 2 array of positions, host) for the receiver calls below."""
    rx = np.ascontiguousarray(receivers, dtype=np.float64).reshape(-1, 2)
    _check(load_library().ls_set_receivers(handle.ptr, rx.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(rx),
                                           _stream(stream)), "ls_set_receivers")
    handle.nrec = len(rx)


def ls_receiver_field(handle, sigma, u, stream=None):
    """u[r][k] = h^2 sum_j G(|r_k - x_j|) sigma[r][j] (Eq. (1)); u has nrhs * nr entries."""
    sp_, k1, n = _ptr(sigma, np.complex128)
    up, k2, _ = _ptr(u, np.complex128, True)
    _check(load_library().ls_receiver_field(handle.ptr, sp_, up, _nrhs(handle, n), _stream(stream)),
           "ls_receiver_field")
    return u


def ls_receiver_adjoint(handle, v, g, stream=None):
    """g[r][j] = h^2 sum_k G(|r_k - x_j|) v[r][k] (the transpose of ls_receiver_field)."""
    vp_, k1, _ = _ptr(v, np.complex128)
    gp, k2, n = _ptr(g, np.complex128, True)
    _check(load_library().ls_receiver_adjoint(handle.ptr, vp_, gp, _nrhs(handle, n), _stream(stream)),
           "ls_receiver_adjoint")
    return g


def ls_misfit_gradient(handle, thetas, data, grad, stream=None, allow_noconv=False):
    """J = sum |u - data|^2 over plane waves `thetas` and the handle's receivers, and
    dJ/db into `grad` (ny*nx float64) by the adjoint method; grad=None computes J
    alone (no adjoint solve).  Returns (J, infos)."""
    th = np.ascontiguousarray(thetas, dtype=np.float64)
    dp_, k1, _ = _ptr(data, np.complex128)
    gp, k2 = (ctypes.c_void_p(None), None) if grad is None else _ptr(grad, np.float64, True)[:2]
    J = ctypes.c_double(0.0)
    infos = (SolveInfo * (2 * len(th)))()
    _check(load_library().ls_misfit_gradient(handle.ptr, th.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                             len(th), dp_, ctypes.byref(J), gp, infos, _stream(stream)),
           "ls_misfit_gradient", allow=(LS_ENOCONV,) if allow_noconv else ())
    return J.value, _infos(infos)


def _make_misfit_function():
    import torch

    class LSMisfit(torch.autograd.Function):
        """J(b) = sum over directions and receivers of |u(r_k) - d|^2 as a torch
        function of the potential b (float64 [ny][nx], CUDA).  forward builds the
        HBS preconditioner for b and runs the forward solves; when b requires a
        gradient it also runs the adjoint solves and keeps dJ/db, which backward
        returns times grad_output.  Usage:
            J = LSMisfit.apply(b, h, kappa, thetas, receivers, data, build_kwargs)"""

        @staticmethod
        def forward(ctx, b, h, kappa, thetas, receivers, data, build_kwargs=None):
            kw = dict(build_kwargs or {})
            tol = kw.pop("tol", 1e-4)
            H = ls_build(b.shape[1], h, kappa, b.detach().contiguous(), tol, ny=b.shape[0], **kw)
            want_grad = bool(ctx.needs_input_grad[0])
            try:
                ls_set_receivers(H, receivers)
                grad = torch.empty_like(b, dtype=torch.float64) if want_grad else None
                J, _ = ls_misfit_gradient(H, thetas, data, grad)
            finally:
                ls_free(H)
            ctx.save_for_backward(grad if want_grad else torch.zeros(0, dtype=torch.float64, device=b.device))
            return torch.tensor(J, dtype=torch.float64, device=b.device)

        @staticmethod
        def backward(ctx, gout):
            (grad,) = ctx.saved_tensors
            return gout * grad, None, None, None, None, None, None

    return LSMisfit


def __getattr__(name):
    if name == "LSMisfit":
        fn = _make_misfit_function()
        globals()["LSMisfit"] = fn
        return fn
    raise AttributeError(name)


def ls_matvec_noalloc(handle, x, y, stream=None):
    """y = (I + B(G+T)) x without any device allocation (device tensors only;
    the FFT scratch is a fixed 2^18-entry array inside the library)."""
    xp, k1, n = _ptr(x, np.complex128)
    yp, k2, _ = _ptr(y, np.complex128, True)
    _check(load_library().ls_matvec_noalloc(handle.ptr, xp, yp, _nrhs(handle, n), _stream(stream)),
           "ls_matvec_noalloc")
    return y


def ls_rhs_plane_wave(handle, thetas, f, stream=None):
    th = np.ascontiguousarray(thetas, dtype=np.float64)
    fp, k1, n = _ptr(f, np.complex128, True)
    _check(load_library().ls_rhs_plane_wave(handle.ptr, th.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), fp,
                                            len(th), _stream(stream)), "ls_rhs_plane_wave")
    return f


def ls_profile_enable(on=True):
    _check(load_library().ls_profile_enable(1 if on else 0), "ls_profile_enable")


def ls_profile_reset():
    _check(load_library().ls_profile_reset(), "ls_profile_reset")


def ls_profile_get():
    """{name: {launches, total_ms, bytes, flops}} of the timed kernel families."""
    buf = (ProfileEntry * 32)()
    n = load_library().ls_profile_get(buf, 32)
    return {e.name.decode(): {"launches": e.launches, "total_ms": e.total_ms, "bytes": e.bytes,
                              "flops": e.flops} for e in buf[:n]}


def ls_cgemm_c64(engine, A, B, C, ta=False, tb=False, alpha=1.0, beta=0.0, stream=None):
    """C = alpha op(A) op(B) + beta C on batched complex64 device tensors [batch, rows, cols]
    (engine 0 SIMT, 1 tcgen05 tf32, 2 tcgen05 tf32x3, 3 tcgen05 f16x3, the FP16 split product)."""
    import torch
    for t in (A, B, C):
        if not (isinstance(t, torch.Tensor) and t.dtype == torch.complex64 and t.is_cuda and t.is_contiguous()):
            raise TypeError("expected contiguous complex64 CUDA tensors")
    batch = C.shape[0]
    M, N = C.shape[1], C.shape[2]
    K = A.shape[1] if ta else A.shape[2]
    al = (ctypes.c_float * 2)(complex(alpha).real, complex(alpha).imag)
    be = (ctypes.c_float * 2)(complex(beta).real, complex(beta).imag)
    sa = A.shape[1] * A.shape[2] if A.shape[0] > 1 else 0
    sb = B.shape[1] * B.shape[2] if B.shape[0] > 1 else 0
    _check(load_library().ls_cgemm_c64(engine, int(ta), int(tb), M, N, K, al, ctypes.c_void_p(A.data_ptr()),
                                       A.shape[2], sa, ctypes.c_void_p(B.data_ptr()), B.shape[2], sb, be,
                                       ctypes.c_void_p(C.data_ptr()), C.shape[2], M * N, batch, _stream(stream)),
           "ls_cgemm_c64")
    return C


def ls_row_id(A, eps, precision=LS_FP64, stream=None, method=LS_ID_GREEDY):
    """Row ID A ~ U A(J, :) of an m x p complex128 matrix (rows = candidates) by
    the device column-pivoted QR (Sec. 2.1), greedy (one pivot per step) or in
    blocks of pivots (method).  A: numpy array or torch tensor (host or CUDA).
    Returns (k, piv[:k] as numpy int array, U as an m x k numpy array)."""
    lib = load_library()
    m, p = A.shape
    ap, keep, _ = _ptr(A, np.complex128)
    kmax = min(m, p)
    piv = (ctypes.c_int * max(kmax, 1))()
    U = np.zeros((m, kmax), np.complex128)
    k = ctypes.c_int(0)
    _check(lib.ls_row_id_ex(ap, m, p, eps, precision, method, ctypes.byref(k), piv, ctypes.c_void_p(U.ctypes.data),
                            _stream(stream)), "ls_row_id_ex")
    kk = k.value
    Uk = U.reshape(-1)[: m * kk].reshape(m, kk).copy()
    return kk, np.array(piv[:kk], dtype=np.int64), Uk


def ls_measure_peak(kind, stream=None):
    """Measured arithmetic rate in TFLOP/s: kind 0 FP64 FMA, 1 FP32 FMA, 2 packed FP32 FMA."""
    v = ctypes.c_double(0.0)
    _check(load_library().ls_measure_peak(kind, ctypes.byref(v), _stream(stream)), "ls_measure_peak")
    return v.value


def ls_sync(handle, stream=None):
    """Wait for the stream; raise LSError if an earlier asynchronous call of the
    handle failed on the device (LS_ETIMEOUT, LS_ESINGULAR)."""
    _check(load_library().ls_sync(handle.ptr, _stream(stream)), "ls_sync")


def ls_allocations():
    """Device and page-locked host allocations the library has made so far."""
    return int(load_library().ls_allocations())


def ls_fault_inject(spec):
    """Host-side failure injection for error-path tests: "alloc:N", "nan_b" or ""."""
    _check(load_library().ls_fault_inject(spec.encode() if spec is not None else None), "ls_fault_inject")


def ls_kernel_launches():
    return int(load_library().ls_kernel_launches())


def ls_free(handle):
    if handle.ptr:
        load_library().ls_free(handle.ptr)
        handle.ptr = None
