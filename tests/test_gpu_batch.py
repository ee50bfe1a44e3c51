"""Blocks of right-hand sides: the apply with every product a GEMM over the block,
and block GMRES (one Krylov space per right-hand side, preconditioner and
operator applied to the block together).

* The block apply equals the one-at-a-time apply (which the parity tests hold to
  5 eps of the dense inverse) to the rounding of the working precision, forward and
  transposed.
* Block GMRES: each density matches the oracle's dense LU of the 10th-order system
  to 1e-9 at 64^2, a zero right-hand side stays zero with no iteration, and the
  transposed block solve matches one-at-a-time solves.
* 512^2, kappa = 300, 256 plane waves in one block: every right-hand side converges;
  sampled densities have true residual <= 1e-10 by the oracle's FFT matvec and agree
  with one-at-a-time solves to 1e-9.
"""
import numpy as np
import pytest

import paper_2007_12718_gb300 as ls
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


@pytest.mark.parametrize("precision", [ls.LS_FP64, ls.LS_FP32, ls.LS_TF32X3])
@pytest.mark.parametrize("transpose", [False, True])
def test_block_apply_matches_one_at_a_time(precision, transpose):
    n, kappa, nr = 64, 40.0, 37  # a ragged block: one full 32-column tile and a tail
    b = inputs.gaussian_family(n, 0)
    H1 = ls.ls_build(n, 1.0 / n, kappa, b, 1e-4, precision=precision, rhs_block=1)
    Hb = ls.ls_build(n, 1.0 / n, kappa, b, 1e-4, precision=precision)
    assert H1.info()["ranks"] == Hb.info()["ranks"]
    f = dev(inputs.random_complex((nr, n, n), 11))
    q1 = host(ls.ls_apply(H1, f, zeros(nr, n, n), transpose=transpose))
    qb = host(ls.ls_apply(Hb, f, zeros(nr, n, n), transpose=transpose))
    tol = 1e-12 if precision == ls.LS_FP64 else 2e-5
    for r in range(nr):
        assert rel(qb[r], q1[r]) <= tol, (r, rel(qb[r], q1[r]))
    ls.ls_free(H1)
    ls.ls_free(Hb)


@pytest.mark.parametrize("precision", [ls.LS_FP64, ls.LS_FP32, ls.LS_TF32X3, ls.LS_FP16SPLIT])
def test_block_solve_vs_dense_lu(precision):
    n, kappa = 64, 40.0
    h = 1.0 / n
    b = inputs.gaussian_family(n, 0)
    th = inputs.plane_wave_angles(6)
    F = np.stack([nystrom.rhs(kappa, b, n, n, h, t).reshape(n, n) for t in th])
    F[3] = 0.0  # a zero right-hand side inside the block
    H = ls.ls_build(n, h, kappa, b, 1e-4, precision=precision)
    sig = zeros(len(th), n, n)
    infos = ls.ls_solve(H, dev(F), sig)
    S = host(sig)
    A = nystrom.dense_operator(kappa, h, b, 10)
    for r in range(len(th)):
        if r == 3:
            assert infos[r]["iterations"] == 0 and infos[r]["converged"] and not S[r].any()
            continue
        assert infos[r]["converged"] and infos[r]["resid_true"] < 2e-10, infos[r]
        assert rel(S[r].ravel(), nystrom.solve_dense(A, F[r].ravel())) < 1e-9
    ls.ls_free(H)


def test_block_transpose_solve_matches_one_at_a_time():
    n, kappa, nr = 64, 40.0, 5
    b = inputs.gaussian_family(n, 1)
    f = dev(inputs.random_complex((nr, n, n), 4))
    out = []
    for blk in (1, 0):
        H = ls.ls_build(n, 1.0 / n, kappa, b, 1e-4, rhs_block=blk)
        sig = zeros(nr, n, n)
        infos = ls.ls_solve_transpose(H, f, sig)
        assert all(i["converged"] for i in infos)
        out.append(host(sig))
        ls.ls_free(H)
    for r in range(nr):
        assert rel(out[1][r], out[0][r]) < 1e-9


@pytest.mark.slow
def test_multirhs_n512_256_plane_waves():
    w = inputs.WORKLOADS["multirhs_n512"]
    n, kappa, nr = w["n"], w["kappa"], w["nrhs"]
    h = 1.0 / n
    b = w["b"](n)
    th = inputs.plane_wave_angles(nr)
    H = ls.ls_build(n, h, kappa, dev(b), w["eps"], precision=ls.LS_TF32X3)
    F = ls.ls_rhs_plane_wave(H, th, zeros(nr, n, n))
    sig = zeros(nr, n, n)
    infos = ls.ls_solve(H, F, sig)
    assert all(i["converged"] and i["resid_true"] <= 1e-10 for i in infos)
    sample = [0, 37, 64, 128, 201, 255]
    S = host(sig)
    spec = nystrom.conv_kernel_spectrum(kappa, h, n, n, 10)
    for r in sample:
        f = nystrom.rhs(kappa, b, n, n, h, th[r])
        assert np.linalg.norm(f - nystrom.matvec_fft(spec, kappa, b, S[r].ravel())) / np.linalg.norm(f) <= 1e-10
    H1 = ls.ls_build(n, h, kappa, dev(b), w["eps"], precision=ls.LS_TF32X3, rhs_block=1)
    sig1 = zeros(len(sample), n, n)
    ls.ls_solve(H1, F[sample].contiguous(), sig1)
    S1 = host(sig1)
    for i, r in enumerate(sample):
        assert rel(S[r], S1[i]) <= 1e-9
    ls.ls_free(H)
    ls.ls_free(H1)
