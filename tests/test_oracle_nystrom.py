"""Pins for the oracle's Nystrom system, FFT matvec and GMRES (Eqs. (3), (9), (10); Sec. 5)."""
import numpy as np
import pytest

from oracle import disk, gmres, nystrom
from paper_2007_12718_gb300 import inputs


def _case(n=16, kappa=12.0, order=10):
    h = 1.0 / n
    b = inputs.gaussian_bump(n, 0.5, 0.03)
    return n, kappa, h, b, order


def test_dense_G_symmetric_and_toeplitz():
    n, kappa, h, b, order = _case()
    G = nystrom.dense_G(kappa, h, n, n, order)
    np.testing.assert_allclose(G, G.T, rtol=0, atol=0)  # complex symmetric, not Hermitian
    assert np.abs(G - G.conj().T).max() > 1e-6


def test_fft_matvec_equals_dense():
    for order in (2, 4, 10):
        n, kappa, h, b, _ = _case(order=order)
        A = nystrom.dense_operator(kappa, h, b, order)
        spec = nystrom.conv_kernel_spectrum(kappa, h, n, n, order)
        x = inputs.random_complex(n * n, 3)
        y = nystrom.matvec_fft(spec, kappa, b, x)
        np.testing.assert_allclose(y, A @ x, rtol=0, atol=1e-13 * np.abs(A @ x).max())


def test_b_zero_gives_zero_density():
    n, kappa, h, _, order = _case()
    b = np.zeros((n, n))
    A = nystrom.dense_operator(kappa, h, b, order)
    f = nystrom.rhs(kappa, b, n, n, h)
    assert np.all(f == 0)
    np.testing.assert_array_equal(A, np.eye(n * n))
    s, k, _ = gmres.gmres(lambda v: A @ v, f)
    assert k == 0 and np.all(s == 0)


def test_gmres_matches_lu():
    n, kappa, h, b, order = _case()
    A = nystrom.dense_operator(kappa, h, b, order)
    f = nystrom.rhs(kappa, b, n, n, h)
    ref = nystrom.solve_dense(A, f)
    s, k, hist = gmres.gmres(lambda v: A @ v, f, tol=1e-12, maxit=200)
    assert hist[-1] <= 1e-12
    assert np.linalg.norm(A @ s - f) / np.linalg.norm(f) < 1e-11
    assert np.linalg.norm(s - ref) / np.linalg.norm(ref) < 1e-10


def test_disk_closed_form():
    """Constant-b disk (b = 0.5, radius 0.3, kappa = 10): the discretised solve
    approaches the transmission-problem series; b is discontinuous, so only a
    low order is expected."""
    kappa, bval, rad = 10.0, 0.5, 0.3
    rec = inputs.receivers_circle(8, 1.5)
    ref = disk.scattered_field(kappa, bval, rad, (0.5, 0.5), rec)
    errs = []
    for n in (24, 48):
        h = 1.0 / n
        b = inputs.constant_disk(n, bval, rad)
        spec = nystrom.conv_kernel_spectrum(kappa, h, n, n, 4)
        f = nystrom.rhs(kappa, b, n, n, h)
        s, k, hist = gmres.gmres(lambda v: nystrom.matvec_fft(spec, kappa, b, v), f, tol=1e-12, maxit=300)
        u = nystrom.field_at(kappa, h, n, n, s, rec)
        errs.append(np.linalg.norm(u - ref) / np.linalg.norm(ref))
    assert errs[1] < errs[0] and errs[1] < 5e-2, errs


@pytest.mark.slow
def test_solve_convergence_orders():
    """Self-convergence of the receiver field for a smooth b: slopes ~ 2, 4, 6, 8, 10."""
    kappa = 10.0
    rec = inputs.receivers_circle(8, 1.5)

    def field(n, order):
        h = 1.0 / n
        b = inputs.gaussian_bump(n, 0.5, 2 * 0.08 ** 2)
        A = nystrom.dense_operator(kappa, h, b, order)
        s = nystrom.solve_dense(A, nystrom.rhs(kappa, b, n, n, h))
        return nystrom.field_at(kappa, h, n, n, s, rec)

    for order, lo in [(2, 1.8), (4, 3.8), (6, 5.6), (8, 7.4), (10, 9.0)]:
        uref = field(64, order)
        e = [np.linalg.norm(field(n, order) - uref) / np.linalg.norm(uref) for n in (24, 32)]
        slope = np.log(e[0] / e[1]) / np.log(32 / 24)
        assert slope > lo, (order, e, slope)
