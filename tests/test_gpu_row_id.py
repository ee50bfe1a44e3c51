"""Device interpolative decomposition (Sec. 2.1) against the oracle's row_id
(scipy's column-pivoted QR).  Pivots are unique only where the residual norms
are separated: on a random matrix they must agree step for step; on the
symmetric proxy blocks of the compression (many exactly tied norms) the rank
must agree within the ID tolerance and the factorisation must be a valid ID."""
import numpy as np
import pytest

import paper_2007_12718_gb300 as ls
from oracle import hbs

pytestmark = pytest.mark.gpu


def id_error(A, J, U):
    return np.linalg.norm(A - U @ A[J, :]) / np.linalg.norm(A)


def random_decaying(m, p, seed):
    rng = np.random.default_rng(seed)
    r = min(m, p)
    Q1, _ = np.linalg.qr(rng.standard_normal((m, r)) + 1j * rng.standard_normal((m, r)))
    Q2, _ = np.linalg.qr(rng.standard_normal((p, r)) + 1j * rng.standard_normal((p, r)))
    s = 10.0 ** (-8.0 * np.arange(r) / r)
    return (Q1 * s) @ Q2.conj().T


@pytest.mark.parametrize("m,p,eps", [(60, 90, 1e-5), (300, 200, 1e-5), (700, 500, 1e-5), (700, 500, 1e-7),
                                     (300, 200, 1e-7)])
def test_random_matrix_pivots_match_oracle(m, p, eps):
    """Distinct residual norms: the greedy pivot sequence is unique, FP64 must
    reproduce scipy's CPQR pivots and rank exactly (sizes cover the one-block,
    cluster and grid kernels; the small tolerance pins the stopping rule far
    below the initial total)."""
    A = random_decaying(m, p, 3)
    J0, U0 = hbs.row_id(A, eps)
    k, J, U = ls.ls_row_id(A, eps, precision=ls.LS_FP64)
    assert k == len(J0)
    assert np.array_equal(J, J0)
    assert np.abs(U - U0).max() <= 1e-8 * max(1.0, np.abs(U0).max())
    assert np.allclose(U[J, :], np.eye(k), atol=0)


@pytest.mark.parametrize("w,h,ring,prec", [(8, 8, 2, ls.LS_FP64), (16, 16, 2, ls.LS_FP64), (8, 8, 2, ls.LS_FP32),
                                           (16, 32, 2, ls.LS_FP32)])
def test_proxy_block_id_is_valid(w, h, ring, prec):
    """Leaf-type proxy blocks G(box, ring) of the n = 256, kappa = 60 problem."""
    n, kappa, eps = 256, 60.0, 1e-4
    A = hbs.kernel_block(kappa, 1.0 / n, 4, hbs.box_points(w, h), hbs.proxy_ring(w, h, ring))
    J0, _ = hbs.row_id(A, eps)
    k, J, U = ls.ls_row_id(A, eps, precision=prec)
    assert abs(k - len(J0)) <= max(2, 0.02 * len(J0)), (k, len(J0))
    assert len(set(J.tolist())) == k
    assert np.allclose(U[J, :], np.eye(k), atol=1e-6 if prec == ls.LS_FP32 else 0)
    assert id_error(A, J, U) <= (3 if prec == ls.LS_FP64 else 10) * eps


def test_host_and_device_inputs_agree():
    import torch
    A = random_decaying(120, 80, 5)
    k1, J1, U1 = ls.ls_row_id(A, 1e-6)
    k2, J2, U2 = ls.ls_row_id(torch.from_numpy(A).cuda(), 1e-6)
    assert k1 == k2 and np.array_equal(J1, J2) and np.array_equal(U1, U2)


def test_invalid_arguments():
    A = np.zeros((4, 4), np.complex128)
    with pytest.raises(ls.LSError):
        ls.ls_row_id(A, 0.0)
    with pytest.raises(ls.LSError):
        ls.ls_row_id(A, 1e-3, precision=ls.LS_TF32)


# ------------------------------------------------------------------ blocked pivot selection
def level_rows(n, kappa, level, eps=1e-4, ring=2, order=4):
    """Rows (candidates) of the level-`level` proxy block of an n x n grid: the
    children's skeletons from the oracle's greedy IDs of the levels below."""
    t = hbs.Tree(n, n, 8)
    h = 1.0 / n
    skel = None
    for l in range(t.L, level - 1, -1):
        w, hh = t.dims[l]
        if l == t.L:
            rows = hbs.box_points(w, hh)
        else:
            oa, ob = t.offsets[l]
            rows = np.concatenate([skel + oa, skel + ob])
        A = hbs.kernel_block(kappa, h, order, rows, hbs.proxy_ring(w, hh, ring))
        if l == level:
            return A
        J, _ = hbs.row_id(A, eps)
        skel = rows[J]


@pytest.mark.parametrize("m,p,eps,prec", [(60, 90, 1e-5, ls.LS_FP64), (300, 200, 1e-5, ls.LS_FP64),
                                          (700, 500, 1e-7, ls.LS_FP64), (1500, 900, 1e-6, ls.LS_FP64),
                                          (700, 500, 1e-4, ls.LS_FP32), (1500, 900, 1e-4, ls.LS_FP32)])
def test_blocked_id_random_matrix(m, p, eps, prec):
    """Blocked pivots on matrices with distinct, geometrically decaying singular
    values: the rank is decided on the explicit residual, so the ID error is
    within the tolerance and the rank within 2 % of the greedy one."""
    A = random_decaying(m, p, 3)
    J0, _ = hbs.row_id(A, eps)
    k, J, U = ls.ls_row_id(A, eps, precision=prec, method=ls.LS_ID_BLOCKED)
    assert abs(k - len(J0)) <= max(2, 0.02 * len(J0)), (k, len(J0))
    assert len(set(J.tolist())) == k
    assert np.allclose(U[J, :], np.eye(k), atol=0)
    assert id_error(A, J, U) <= (1.5 if prec == ls.LS_FP64 else 10) * eps


@pytest.mark.parametrize("n,kappa,level,prec", [(64, 40.0, 3, ls.LS_FP64), (128, 78.5, 3, ls.LS_FP32),
                                                (128, 78.5, 2, ls.LS_FP64), (256, 157.0, 4, ls.LS_FP32)])
def test_blocked_id_proxy_blocks(n, kappa, level, prec):
    """Upper-level proxy blocks (rows: the children's skeletons) at ~10 points per
    wavelength, the regime of the 2048^2 workload: rank within 2 % of the
    oracle's CPQR, ID error <= 3 eps (FP64) / 10 eps (FP32)."""
    eps = 1e-4
    A = level_rows(n, kappa, level, eps)
    J0, _ = hbs.row_id(A, eps)
    for method in (ls.LS_ID_BLOCKED, ls.LS_ID_AUTO):
        k, J, U = ls.ls_row_id(A, eps, precision=prec, method=method)
        assert abs(k - len(J0)) <= max(2, 0.02 * len(J0)), (method, k, len(J0))
        assert len(set(J.tolist())) == k
        assert np.allclose(U[J, :], np.eye(k), atol=0)
        assert id_error(A, J, U) <= (3 if prec == ls.LS_FP64 else 10) * eps


def test_blocked_id_edge_cases():
    """One candidate, one proxy, fewer proxies than candidates (rank capped at p),
    exact low rank, a zero block, and fewer candidates than the pool."""
    rng = np.random.default_rng(11)
    for prec in (ls.LS_FP64, ls.LS_FP32):
        tol = 1e-10 if prec == ls.LS_FP64 else 1e-5
        A = rng.standard_normal((1, 7)) + 1j * rng.standard_normal((1, 7))
        k, J, U = ls.ls_row_id(A, 1e-6, precision=prec, method=ls.LS_ID_BLOCKED)
        assert k == 1 and J[0] == 0 and U[0, 0] == 1
        A = rng.standard_normal((9, 1)) + 1j * rng.standard_normal((9, 1))
        k, J, U = ls.ls_row_id(A, 1e-6, precision=prec, method=ls.LS_ID_BLOCKED)
        assert k == 1 and id_error(A, J, U) <= tol
        A = rng.standard_normal((300, 40)) + 1j * rng.standard_normal((300, 40))
        k, J, U = ls.ls_row_id(A, 1e-6, precision=prec, method=ls.LS_ID_BLOCKED)
        assert k <= 40 and id_error(A, J, U) <= 1e-6 + tol
        B = (rng.standard_normal((400, 17)) + 1j * rng.standard_normal((400, 17))) @ \
            (rng.standard_normal((17, 250)) + 1j * rng.standard_normal((17, 250)))
        k, J, U = ls.ls_row_id(B, 1e-6, precision=prec, method=ls.LS_ID_BLOCKED)
        assert k == 17 and id_error(B, J, U) <= 1e-6
        k, J, U = ls.ls_row_id(np.zeros((50, 30), np.complex128), 1e-6, precision=prec, method=ls.LS_ID_BLOCKED)
        assert k == 0
        A = random_decaying(40, 70, 2)
        J0, _ = hbs.row_id(A, 1e-4)
        k, J, U = ls.ls_row_id(A, 1e-4, precision=prec, method=ls.LS_ID_BLOCKED)
        assert abs(k - len(J0)) <= 2 and id_error(A, J, U) <= 1.5e-4


def test_blocked_id_does_not_modify_input_and_repeats():
    """The caller's device matrix is left as it was, and two calls give the same pivots."""
    import torch
    A = random_decaying(900, 600, 8)
    At = torch.from_numpy(A).cuda()
    k1, J1, U1 = ls.ls_row_id(At, 1e-6, method=ls.LS_ID_BLOCKED)
    k2, J2, U2 = ls.ls_row_id(At, 1e-6, method=ls.LS_ID_BLOCKED)
    assert np.array_equal(At.cpu().numpy(), A)
    assert k1 == k2 and np.array_equal(J1, J2) and np.array_equal(U1, U2)
