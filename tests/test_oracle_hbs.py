"""Pins for the oracle's HBS compression and inverse (Secs. 2.1, 3, 4.1, 5)."""
import json
import os

import numpy as np
import pytest
import scipy.special as sp

from oracle import gmres, hbs, nystrom
from paper_2007_12718_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_table1_proxy_accuracy():
    """Table 1 (Sec. 3.2), to within a factor 3 (2.5x floor for the last row)."""
    g = json.load(open(os.path.join(GOLD, "table1_proxy.json")))
    box = hbs.box_points(20, 20)
    lat = hbs.box_points(40, 40) - 10
    inside = (lat[:, 0] >= 0) & (lat[:, 0] < 20) & (lat[:, 1] >= 0) & (lat[:, 1] < 20)
    comp = lat[~inside]
    for j, c in enumerate(g["box_sizes_in_wavelengths"]):
        kappa, h = 1.0, 2 * np.pi * c / 20
        B = hbs.kernel_block(kappa, h, 4, box, comp)
        for i, w in enumerate(g["ring_widths"]):
            P = hbs.kernel_block(kappa, h, 4, box, hbs.proxy_ring(20, 20, w))
            Q, _ = np.linalg.qr(P)
            err = np.abs(B - Q @ (Q.conj().T @ B)).max() / np.abs(B).max()
            ref = g["errors"][i][j]
            if ref > 1e-13:
                assert ref / 3 < err < ref * 3, (c, w, err, ref)
            else:
                assert err < 1e-13


def test_row_id_properties():
    rng = np.random.default_rng(1)
    kappa, h = 20.0, 1 / 32
    rows = hbs.box_points(8, 8)
    A = hbs.kernel_block(kappa, h, 4, rows, hbs.proxy_ring(8, 8, 2))
    J, U = hbs.row_id(A, 1e-6)
    np.testing.assert_array_equal(U[J], np.eye(len(J)))  # U(J,:) = I  (Sec. 2.1)
    # accuracy on the full complement in a 32 x 32 lattice (proxy claim, Eq. (13))
    lat = hbs.box_points(32, 32) - 12
    inside = (lat[:, 0] >= 0) & (lat[:, 0] < 8) & (lat[:, 1] >= 0) & (lat[:, 1] < 8)
    B = hbs.kernel_block(kappa, h, 4, rows, lat[~inside])
    assert np.linalg.norm(B - U @ B[J]) <= 10 * 1e-6 * np.linalg.norm(B)


def _setup(n, kappa, order, eps, ring, leaf=8):
    h = 1.0 / n
    b = inputs.gaussian_bump(n)
    tree = hbs.Tree(n, n, leaf)
    comp = hbs.Compression(kappa, h, tree, order, eps, ring)
    return h, b, tree, comp


def test_lemma_4_1_incoming_expansions():
    """Eq. (18): the incoming expansion of each leaf, built from sibling blocks and
    the parent's expansion, reproduces the exact incoming field
    G(I_tau, I_tau^c) q(I_tau^c) (with V* read as U^T, Eq. (17))."""
    n, kappa = 16, 15.0
    h, b, tree, comp = _setup(n, kappa, 4, 1e-12, 3)
    assert tree.L == 2
    G = nystrom.dense_G(kappa, h, n, n, 4)
    q = inputs.random_complex(n * n, 5)
    ql = hbs.gather_leaves(tree, q)  # (4, 64)
    U2, U1 = comp.U[2], comp.U[1]
    qt2 = ql @ U2  # U^T q per leaf, as rows
    qt1 = np.stack([np.concatenate([qt2[0], qt2[1]]) @ U1, np.concatenate([qt2[2], qt2[3]]) @ U1])
    G1, G2 = comp.G_sib[1], comp.G_sib[2]
    wt1 = [G1 @ qt1[1], G1.T @ qt1[0]]
    for p in range(2):
        Uw = U1 @ wt1[p]
        k = len(qt2[0])
        wa = G2 @ qt2[2 * p + 1] + Uw[:k]
        wb = G2.T @ qt2[2 * p] + Uw[k:]
        for leaf, wtil in ((2 * p, wa), (2 * p + 1, wb)):
            idx = hbs.gather_leaves(tree, np.arange(n * n))[leaf]
            mask = np.ones(n * n, bool)
            mask[idx] = False
            exact = G[np.ix_(idx, np.where(mask)[0])] @ q[mask]
            assert np.linalg.norm(U2 @ wtil - exact) < 1e-9 * np.linalg.norm(exact)


@pytest.mark.parametrize("order,eps,ring", [(4, 1e-4, 2), (4, 1e-7, 2), (10, 1e-10, 4)])
def test_hbs_inverse_vs_dense(order, eps, ring):
    """The HBS inverse approximates (I + B G_p)^-1 to about eps (Secs. 3.2, 4.1)."""
    n, kappa = 32, 20.0
    h, b, tree, comp = _setup(n, kappa, order, eps, ring)
    inv = hbs.Inverse(comp, b)
    A = nystrom.dense_operator(kappa, h, b, order)
    for f in (nystrom.rhs(kappa, b, n, n, h), inputs.random_complex(n * n, 9)):
        ref = nystrom.solve_dense(A, f)
        err = np.linalg.norm(inv.apply(f) - ref) / np.linalg.norm(ref)
        assert err < 5 * eps, err


def test_hbs_error_shrinks_with_eps():
    n, kappa = 32, 20.0
    errs = []
    for eps in (1e-3, 1e-6, 1e-9):
        h, b, tree, comp = _setup(n, kappa, 4, eps, 2 if eps > 1e-9 else 3)
        inv = hbs.Inverse(comp, b)
        A = nystrom.dense_operator(kappa, h, b, 4)
        f = inputs.random_complex(n * n, 2)
        ref = nystrom.solve_dense(A, f)
        errs.append(np.linalg.norm(inv.apply(f) - ref) / np.linalg.norm(ref))
    assert errs[0] > 10 * errs[1] > 100 * errs[2]


def test_spectrum_example_soft_pin():
    """Sec. 5: N = 1600, kappa = 8 pi, lens potential, 10th-order operator.  The paper
    reports 80 unpreconditioned GMRES iterations to 1e-10, 6 with the eps = 1e-2
    4th-order preconditioner, and eigenvalues of the preconditioned operator within
    0.06 of 1.  The weights and the lens placement differ from the paper's code,
    so only the qualitative facts are pinned: many iterations unpreconditioned, a
    handful preconditioned, and a tightly clustered spectrum."""
    n, kappa = 40, 8 * np.pi
    h = 1.0 / n
    x = nystrom.nodes(n, n, h, -0.5, -0.5)
    r = np.hypot(x[:, 0], x[:, 1])
    b = (4 * (x[:, 1] - 0.1) * (1 - sp.erf(25 * (r - 0.3)))).reshape(n, n)
    A = nystrom.dense_operator(kappa, h, b, 10)
    f = -(kappa ** 2) * b.ravel() * np.exp(1j * kappa * x[:, 0])
    _, k_plain, _ = gmres.gmres(lambda v: A @ v, f, tol=1e-10, maxit=200)
    tree = hbs.Tree(n, n, 10)
    comp = hbs.Compression(kappa, h, tree, 4, 1e-2, 2)
    inv = hbs.Inverse(comp, b)
    _, k_prec, _ = gmres.gmres(lambda v: A @ v, f, apply_M=inv.apply, tol=1e-10, maxit=200)
    assert 50 <= k_plain <= 110 and k_prec <= 10
    M = np.stack([inv.apply(e) for e in np.eye(n * n)], axis=1)
    assert np.abs(np.linalg.eigvals(A @ M) - 1).max() < 0.15


def test_cavity_preconditioned_iterations_match_paper():
    """Sec. 6.3, cavity table: at N = 6400 (80 x 80, kappa = 50.27, 10 points per
    wavelength, 100-point leaves, eps = 1e-4, 4th-order corrections in the HBS,
    10th-order FFT operator) the preconditioned GMRES reaches 1e-10 in 4 iterations.
    The oracle's HBS + GMRES must land within one iteration of that."""
    from oracle import gmres as ogmres
    from oracle import nystrom
    from paper_2007_12718_gb300 import inputs
    w = inputs.WORKLOADS["cavity_n80"]
    n, kappa = w["n"], w["kappa"]
    h = 1.0 / n
    b = w["b"](n)
    comp = hbs.Compression(kappa, h, hbs.Tree(n, n, w["leaf"]), 4, w["eps"], 2)
    inv = hbs.Inverse(comp, b)
    spec = nystrom.conv_kernel_spectrum(kappa, h, n, n, 10)
    f = nystrom.rhs(kappa, b, n, n, h)
    s, k, hist = ogmres.gmres(lambda v: nystrom.matvec_fft(spec, kappa, b, v), f, apply_M=inv.apply, tol=1e-10)
    r = np.linalg.norm(f - nystrom.matvec_fft(spec, kappa, b, s)) / np.linalg.norm(f)
    assert r < 2e-10
    assert 3 <= k <= 5, k


def test_woodbury_local_solution_is_inverse_of_eq26():
    """Sec. 4.1, Eq. blockinv: with G_ab = L R^T of rank r the Woodbury form equals
    [[I, S_a G_ab], [S_b G_ab^T, I]]^-1; the printed middle block
    [[I, R_ba^T L_ba], [R_ab^T L_ab, I]] (no S) does not."""
    rng = np.random.default_rng(3)
    k, r = 40, 9
    cplx = lambda *sh: rng.standard_normal(sh) + 1j * rng.standard_normal(sh)  # noqa: E731
    S_a, S_b = 0.3 * cplx(k, k), 0.3 * cplx(k, k)
    L, R = cplx(k, r), cplx(k, r)
    G = L @ R.T
    Z = np.block([[np.eye(k), S_a @ G], [S_b @ G.T, np.eye(k)]])
    X = hbs.woodbury_local_solution(S_a, S_b, L, R, R, L)  # G_ba = G^T = R L^T
    assert np.linalg.norm(X - np.linalg.inv(Z)) <= 1e-10 * np.linalg.norm(X)
    # the block as printed (children's S left out) gives another matrix
    P = np.zeros((2 * k, 2 * r), dtype=complex)
    P[:k, :r] = S_a @ L
    P[k:, r:] = S_b @ R
    Q = np.zeros((2 * r, 2 * k), dtype=complex)
    Q[:r, k:] = R.T
    Q[r:, :k] = L.T
    printed = np.block([[np.eye(r), L.T @ R], [R.T @ L, np.eye(r)]])
    Xp = np.eye(2 * k) - P @ np.linalg.solve(printed, Q)
    assert np.linalg.norm(Xp - np.linalg.inv(Z)) > 1e-2 * np.linalg.norm(X)
