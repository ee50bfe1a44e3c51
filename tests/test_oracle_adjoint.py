"""Pins for the oracle's transposed operators and the adjoint gradient of the
receiver misfit (built on Eqs. (1), (9)-(10) and Algorithm 2)."""
import numpy as np
import pytest

from oracle import adjoint, hbs, nystrom
from paper_2007_12718_gb300 import inputs


def test_transpose_matvec_vs_dense():
    """(I + B G_p)^T x by FFT equals the dense transpose (G_p complex symmetric)."""
    n, kappa, order = 24, 18.0, 10
    h = 1.0 / n
    b = inputs.gaussian_family(n, 3)
    A = nystrom.dense_operator(kappa, h, b, order)
    spec = nystrom.conv_kernel_spectrum(kappa, h, n, n, order)
    x = inputs.random_complex(n * n, 4)
    y = nystrom.matvec_fft_transpose(spec, kappa, b, x)
    assert np.linalg.norm(y - A.T @ x) < 1e-12 * np.linalg.norm(A.T @ x)
    # and it is not the forward operator (b varies, so A is not symmetric)
    assert np.linalg.norm(y - A @ x) > 1e-3 * np.linalg.norm(y)


@pytest.mark.parametrize("order,eps,ring", [(4, 1e-4, 2), (10, 1e-10, 4)])
def test_apply_transpose_is_the_transpose(order, eps, ring):
    """M^T from the reversed Algorithm 2 matches the dense transpose of M,
    assembled column by column from the forward apply, and the bilinear
    identity y^T (M x) = (M^T y)^T x holds for random vectors."""
    n, kappa = 16, 15.0
    h = 1.0 / n
    b = inputs.gaussian_bump(n)
    tree = hbs.Tree(n, n, 4)
    comp = hbs.Compression(kappa, h, tree, order, eps, ring)
    inv = hbs.Inverse(comp, b)
    N = n * n
    M = np.stack([inv.apply(e) for e in np.eye(N)], axis=1)
    MT = np.stack([inv.apply_transpose(e) for e in np.eye(N)], axis=1)
    assert np.linalg.norm(MT - M.T) < 1e-12 * np.linalg.norm(M)
    for s in range(3):
        x = inputs.random_complex(N, 20 + s)
        y = inputs.random_complex(N, 30 + s)
        lhs = y @ inv.apply(x)
        rhs = inv.apply_transpose(y) @ x
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # M^T approximates (A^-1)^T = (A^T)^-1 to about eps
    A = nystrom.dense_operator(kappa, h, b, order)
    f = inputs.random_complex(N, 5)
    ref = nystrom.solve_dense(A.T, f)
    assert np.linalg.norm(inv.apply_transpose(f) - ref) < 5 * eps * np.linalg.norm(ref)


def _problem(n=16, ndir=2, nrec=8, seed=3):
    kappa, order = 12.0, 4
    h = 1.0 / n
    b = inputs.gaussian_family(n, seed)
    thetas = inputs.plane_wave_angles(ndir)
    rec = inputs.receivers_circle(nrec)
    return kappa, h, b, order, thetas, rec


def test_gradient_matches_finite_differences():
    """dJ/db from the adjoint state equals central differences of J along random
    directions (a dropped term, sign or transpose in the gradient fails this)."""
    kappa, h, b, order, thetas, rec = _problem()
    data = 0.05 * inputs.random_complex((len(thetas), len(rec)), 8)
    J, g = adjoint.misfit_gradient(kappa, h, b, order, thetas, rec, data)
    assert np.isclose(J, adjoint.misfit(kappa, h, b, order, thetas, rec, data), rtol=1e-12)
    rng = np.random.default_rng(11)
    for _ in range(3):
        db = rng.standard_normal(b.shape) * inputs.cutoff(*inputs.grid_nodes(b.shape[0]))
        t = 1e-6
        Jp = adjoint.misfit(kappa, h, b + t * db, order, thetas, rec, data)
        Jm = adjoint.misfit(kappa, h, b - t * db, order, thetas, rec, data)
        fd = (Jp - Jm) / (2 * t)
        an = float(np.sum(g * db))
        assert abs(fd - an) < 1e-6 * abs(an), (fd, an)


def test_gradient_vanishes_at_exact_data():
    """With data equal to the receiver field of b itself, J = 0 and dJ/db = 0."""
    kappa, h, b, order, thetas, rec = _problem(nrec=6)
    _, u = adjoint.forward(kappa, h, b, order, thetas, rec)
    J, g = adjoint.misfit_gradient(kappa, h, b, order, thetas, rec, u)
    assert J < 1e-24 * np.sum(np.abs(u) ** 2)
    assert np.abs(g).max() < 1e-10


def test_receiver_matrix_is_field_at():
    """R sigma equals the oracle's receiver field of Eq. (1)."""
    n, kappa = 16, 12.0
    h = 1.0 / n
    rec = inputs.receivers_circle(5)
    sig = inputs.random_complex((2, n * n), 6)
    R = adjoint.receiver_matrix(kappa, h, n, n, rec)
    ref = nystrom.field_at(kappa, h, n, n, sig, rec)
    assert np.linalg.norm(sig @ R.T - ref.T) < 1e-13 * np.linalg.norm(ref)
