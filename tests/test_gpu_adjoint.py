"""GPU parity of the adjoint path (transposed operator, transposed HBS apply,
transposed solve, receiver fields, misfit gradient) against the CPU oracle.

Tolerances (relative, 2-norm unless stated):
* transposed matvec and the grid field (FP64 FFT convolution vs the oracle's
  dense matrices): 1e-12, as the forward matvec.
* M^T against the GPU's own M (bilinear identity y^T (M x) = (M^T y)^T x):
  1e-12 with FP64 factors, 1e-5 with FP32 factors (two summation orders of
  the same FP32 products).  M^T f against the dense (A^T)^-1 f: 5 eps, as M.
* transposed GMRES to 1e-10 vs dense LU of A^T: 1e-9.
* receiver fields (FP64, R evaluated by the device Hankel routine, |error|
  ~1e-15 relative per entry): 1e-12.
* J and dJ/db vs the oracle's dense adjoint: both solves stop at 1e-10, so
  J and the gradient agree to ~1e-9; the test allows 1e-8.
"""
import numpy as np
import pytest

import paper_2007_12718_gb300 as ls
from oracle import adjoint as oadj
from oracle import nystrom
from paper_2007_12718_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def zeros(*shape):
    return torch.zeros(*shape, dtype=torch.complex128, device=DEV)


def build(n, kappa, b, eps, precision=ls.LS_FP64, **kw):
    return ls.ls_build(n, 1.0 / n, kappa, b, eps, order_matvec=10, order_precond=4, precision=precision, **kw)


@pytest.mark.parametrize("n,nrhs", [(32, 1), (64, 2)])
def test_matvec_transpose_and_field_vs_oracle(n, nrhs):
    kappa = 25.0
    b = inputs.gaussian_family(n, 2)
    H = build(n, kappa, b, 1e-4)
    x = inputs.random_complex((nrhs, n, n), 3)
    yt = host(ls.ls_matvec(H, dev(x), zeros(nrhs, n, n), transpose=True))
    u = host(ls.ls_field(H, dev(x), zeros(nrhs, n, n)))
    spec = nystrom.conv_kernel_spectrum(kappa, 1.0 / n, n, n, 10)
    A = nystrom.dense_operator(kappa, 1.0 / n, b, 10) if n <= 32 else None
    for r in range(nrhs):
        xr = x[r].ravel()
        ref_t = A.T @ xr if A is not None else nystrom.matvec_fft_transpose(spec, kappa, b, xr)
        assert rel(yt[r].ravel(), ref_t) < 1e-12
        assert rel(u[r].ravel(), nystrom.apply_conv(spec, xr, n, n)) < 1e-12
    # host buffers give the same bytes as device buffers
    yh = ls.ls_matvec(H, x, np.zeros_like(x), transpose=True)
    np.testing.assert_array_equal(yh, yt)


@pytest.mark.parametrize("precision,tol", [(ls.LS_FP64, 1e-12), (ls.LS_FP32, 1e-5)])
def test_apply_transpose_is_transpose_of_apply(precision, tol):
    n, kappa = 64, 40.0
    b = inputs.gaussian_family(n, 0)
    H = build(n, kappa, b, 1e-4, precision=precision)
    for s in range(2):
        x = inputs.random_complex((n, n), 40 + s)
        y = inputs.random_complex((n, n), 50 + s)
        Mx = host(ls.ls_apply(H, dev(x), zeros(n, n)))
        MTy = host(ls.ls_apply(H, dev(y), zeros(n, n), transpose=True))
        lhs = np.sum(y * Mx)
        rhs = np.sum(MTy * x)
        assert abs(lhs - rhs) < tol * abs(lhs), (lhs, rhs)


@pytest.mark.parametrize("precision", [ls.LS_FP64, ls.LS_FP32])
def test_apply_transpose_vs_dense_inverse(precision):
    n, kappa, eps = 32, 20.0, 1e-4
    b = inputs.gaussian_bump(n)
    H = build(n, kappa, b, eps, precision=precision)
    A = nystrom.dense_operator(kappa, 1.0 / n, b, 4)
    for seed in (1, 2):
        f = inputs.random_complex((n, n), seed)
        q = host(ls.ls_apply(H, dev(f), zeros(n, n), transpose=True))
        ref = nystrom.solve_dense(A.T, f.ravel()).reshape(n, n)
        assert rel(q, ref) < 5 * eps
    # forward and transposed applies interleave on one handle (shared barrier epochs)
    f = inputs.random_complex((n, n), 3)
    q1 = host(ls.ls_apply(H, dev(f), zeros(n, n)))
    q2 = host(ls.ls_apply(H, dev(f), zeros(n, n), transpose=True))
    q3 = host(ls.ls_apply(H, dev(f), zeros(n, n)))
    np.testing.assert_array_equal(q1, q3)
    assert rel(q2, nystrom.solve_dense(A.T, f.ravel()).reshape(n, n)) < 5 * eps


@pytest.mark.parametrize("precision", [ls.LS_FP32, ls.LS_TF32X3])
def test_solve_transpose_vs_lu(precision):
    n, kappa = 64, 40.0
    b = inputs.gaussian_family(n, 1)
    H = build(n, kappa, b, 1e-4, precision=precision)
    f = inputs.random_complex((2, n, n), 9)
    sig = zeros(2, n, n)
    infos = ls.ls_solve_transpose(H, dev(f), sig)
    A = nystrom.dense_operator(kappa, 1.0 / n, b, 10)
    s = host(sig)
    for r in range(2):
        assert infos[r]["converged"] and infos[r]["resid_true"] < 2e-10
        assert infos[r]["iterations"] < 30
        assert rel(s[r].ravel(), nystrom.solve_dense(A.T, f[r].ravel())) < 1e-9


def test_receiver_field_and_adjoint_vs_oracle():
    n, kappa, nrec, nrhs = 32, 20.0, 12, 3
    b = inputs.gaussian_bump(n)
    H = build(n, kappa, b, 1e-4)
    rec = inputs.receivers_circle(nrec)
    ls.ls_set_receivers(H, rec)
    R = oadj.receiver_matrix(kappa, 1.0 / n, n, n, rec)
    sig = inputs.random_complex((nrhs, n, n), 4)
    u = host(ls.ls_receiver_field(H, dev(sig), zeros(nrhs, nrec)))
    assert rel(u, sig.reshape(nrhs, -1) @ R.T) < 1e-12
    v = inputs.random_complex((nrhs, nrec), 5)
    g = host(ls.ls_receiver_adjoint(H, dev(v), zeros(nrhs, n, n)))
    assert rel(g.reshape(nrhs, -1), v @ R) < 1e-12
    # host buffers
    uh = ls.ls_receiver_field(H, sig, np.zeros((nrhs, nrec), np.complex128))
    np.testing.assert_array_equal(uh, u)


def test_misfit_gradient_vs_oracle_adjoint():
    """J and dJ/db of the receiver misfit against the oracle's dense adjoint
    gradient (itself pinned by finite differences)."""
    n, kappa, ndir, nrec = 32, 20.0, 3, 16
    h = 1.0 / n
    b = inputs.gaussian_family(n, 5)
    thetas = inputs.plane_wave_angles(ndir)
    rec = inputs.receivers_circle(nrec)
    data = 0.02 * inputs.random_complex((ndir, nrec), 12)
    J0, g0 = oadj.misfit_gradient(kappa, h, b, 10, thetas, rec, data)
    H = build(n, kappa, b, 1e-4, precision=ls.LS_FP32)
    ls.ls_set_receivers(H, rec)
    grad = torch.zeros(n, n, dtype=torch.float64, device=DEV)
    J, infos = ls.ls_misfit_gradient(H, thetas, dev(data), grad)
    assert all(i["converged"] for i in infos) and len(infos) == 2 * ndir
    assert abs(J - J0) < 1e-8 * J0
    assert rel(host(grad), g0) < 1e-8
    # host data and gradient buffers
    gh = np.zeros((n, n))
    Jh, _ = ls.ls_misfit_gradient(H, thetas, data, gh)
    assert Jh == J
    np.testing.assert_array_equal(gh, host(grad))


def test_lsmisfit_autograd_and_finite_differences():
    """LSMisfit.backward returns dJ/db, and J(b +- t db) on the GPU agrees with it
    (central differences; the solves stop at 1e-10, so t = 1e-4 gives ~1e-6)."""
    n, kappa, ndir, nrec = 64, 30.0, 4, 24
    h = 1.0 / n
    b = dev(inputs.gaussian_family(n, 6))
    thetas = inputs.plane_wave_angles(ndir)
    rec = inputs.receivers_circle(nrec)
    data = dev(0.02 * inputs.random_complex((ndir, nrec), 13))
    kw = {"tol": 1e-4, "precision": ls.LS_FP32}
    bb = b.clone().requires_grad_(True)
    J = ls.LSMisfit.apply(bb, h, kappa, thetas, rec, data, kw)
    J.backward()
    g = bb.grad.detach()
    db = dev(np.random.default_rng(3).standard_normal((n, n)) * inputs.cutoff(*inputs.grid_nodes(n)))
    t = 1e-4
    Jp = ls.LSMisfit.apply(b + t * db, h, kappa, thetas, rec, data, kw).item()
    Jm = ls.LSMisfit.apply(b - t * db, h, kappa, thetas, rec, data, kw).item()
    fd = (Jp - Jm) / (2 * t)
    an = float(torch.sum(g * db))
    assert abs(fd - an) < 1e-5 * abs(an), (fd, an)


@pytest.mark.slow
def test_misfit_gradient_full_size_n512_finite_differences():
    """The differentiation workload (512 x 512, kappa = 300, 32 directions, 256
    receivers on the circle r = 1.5): no dense oracle at this size, so the
    gradient is checked by central differences along a smooth direction, and
    every solve must converge."""
    n, kappa, ndir, nrec = 512, 300.0, 32, 256
    h = 1.0 / n
    b = inputs.gaussian_family(n, 0)
    thetas = inputs.plane_wave_angles(ndir)
    rec = inputs.receivers_circle(nrec)
    # data: the receiver field of the seed-1 potential
    Href = build(n, kappa, inputs.gaussian_family(n, 1), 1e-4, precision=ls.LS_FP32)
    f = zeros(ndir, n, n)
    ls.ls_rhs_plane_wave(Href, thetas, f)
    sig = zeros(ndir, n, n)
    assert all(i["converged"] for i in ls.ls_solve(Href, f, sig))
    ls.ls_set_receivers(Href, rec)
    data = ls.ls_receiver_field(Href, sig, zeros(ndir, nrec))
    ls.ls_free(Href)

    def misfit(bv, grad=None):
        H = build(n, kappa, bv, 1e-4, precision=ls.LS_FP32)
        ls.ls_set_receivers(H, rec)
        g = grad if grad is not None else torch.zeros(n, n, dtype=torch.float64, device=DEV)
        J, infos = ls.ls_misfit_gradient(H, thetas, data, g)
        ls.ls_free(H)
        assert all(i["converged"] for i in infos)
        return J

    grad = torch.zeros(n, n, dtype=torch.float64, device=DEV)
    J0 = misfit(dev(b), grad)
    assert J0 > 0
    X, Y = inputs.grid_nodes(n)
    db = np.sin(3 * np.pi * X) * np.cos(2 * np.pi * Y) * inputs.cutoff(X, Y)
    t = 1e-5
    fd = (misfit(dev(b + t * db)) - misfit(dev(b - t * db))) / (2 * t)
    an = float(torch.sum(grad * dev(db)))
    assert abs(fd - an) < 1e-4 * abs(an), (fd, an)


def test_adjoint_invalid_arguments():
    n, kappa = 32, 20.0
    H = build(n, kappa, inputs.gaussian_bump(n), 1e-4)
    lib = ls.load_library()
    x = zeros(n, n)
    y = zeros(n, n)
    import ctypes
    assert lib.ls_apply(H.ptr, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), 1, 2, None) == ls.LS_EINVAL
    assert lib.ls_matvec(H.ptr, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), 1, -1,
                         None) == ls.LS_EINVAL
    # no receivers yet
    with pytest.raises(ls.LSError):
        ls.ls_receiver_field(H, x, zeros(1, 4))
    with pytest.raises(ls.LSError):
        ls.ls_misfit_gradient(H, [0.0], zeros(1, 4), torch.zeros(n, n, dtype=torch.float64, device=DEV))
    # a receiver on a grid node
    with pytest.raises(ls.LSError):
        ls.ls_set_receivers(H, np.array([[0.5 + 0.5 / n, 0.5 + 0.5 / n]]))
