"""Several problems in one handle (ls_build_many): a forest of trees of the same
geometry sharing one compression, every level's nodes of every problem in the
same batched launches.

* Each problem's apply (forward, transposed) equals that of a handle built for
  it alone, to the rounding of the working precision.
* The matvec uses each problem's own potential: it equals the oracle's dense
  order-10 operator of that problem to 1e-12.
* Each problem's GMRES density matches the oracle's dense LU of its own system
  to 1e-9, with its own iteration count.
* 32 problems of sides 64/96/128/192 at 10 points per wavelength (grouped by
  side into four handles): every problem converges to 1e-10; sampled densities
  have true residual <= 1e-10 by the oracle's FFT matvec.
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
def test_forest_apply_matches_single_problems(precision):
    n, kappa, G = 64, 40.0, 3
    bs = np.stack([inputs.gaussian_family(n, s) for s in range(G)])
    F = ls.ls_build(n, 1.0 / n, kappa, bs, 1e-4, precision=precision)
    assert F.info()["nprob"] == G
    singles = [ls.ls_build(n, 1.0 / n, kappa, bs[g], 1e-4, precision=precision) for g in range(G)]
    assert all(F.info()["ranks"] == H.info()["ranks"] for H in singles)
    f = inputs.random_complex((2, G, n, n), 5)  # two sets of G right-hand sides
    # FP64 / FP32: the same kernels on the same numbers; tf32x3: the forest's
    # batched merge products cross the tensor cores' size threshold where the
    # single problems' do not, so two engines (each ~1e-5 per product, see the
    # GEMM tests' error model) meet: their difference is bounded here
    tol = {ls.LS_FP64: 1e-13, ls.LS_FP32: 1e-6, ls.LS_TF32X3: 2e-5}[precision]
    for tr in (False, True):
        qf = host(ls.ls_apply(F, dev(f), zeros(2, G, n, n), transpose=tr))
        for g, H in enumerate(singles):
            qs = host(ls.ls_apply(H, dev(f[:, g]), zeros(2, n, n), transpose=tr))
            assert rel(qf[:, g], qs) <= tol, (tr, g, rel(qf[:, g], qs))
    for H in singles + [F]:
        ls.ls_free(H)


def test_forest_matvec_and_solve_vs_oracle():
    n, kappa, G = 32, 20.0, 3
    h = 1.0 / n
    bs = np.stack([inputs.gaussian_family(n, 10 + s) for s in range(G)])
    F = ls.ls_build(n, h, kappa, bs, 1e-4, precision=ls.LS_FP32)
    x = inputs.random_complex((G, n, n), 8)
    y = host(ls.ls_matvec(F, dev(x), zeros(G, n, n)))
    rhs = host(ls.ls_rhs_plane_wave(F, [0.3], zeros(G, n, n)))
    sig = zeros(G, n, n)
    infos = ls.ls_solve(F, dev(rhs), sig)
    S = host(sig)
    assert len(infos) == G
    for g in range(G):
        A = nystrom.dense_operator(kappa, h, bs[g], 10)
        assert rel(y[g].ravel(), A @ x[g].ravel()) <= 1e-12
        fg = nystrom.rhs(kappa, bs[g], n, n, h, 0.3)
        assert np.abs(rhs[g].ravel() - fg).max() <= 1e-12 * np.abs(fg).max()
        assert infos[g]["converged"] and infos[g]["resid_true"] < 2e-10
        assert rel(S[g].ravel(), nystrom.solve_dense(A, fg)) < 1e-9
    ls.ls_free(F)


@pytest.mark.slow
def test_multiproblem_32_uneven_sizes():
    probs = inputs.multiproblem_set()
    by_side = {}
    for i, p in enumerate(probs):
        by_side.setdefault(p["n"], []).append((i, p))
    checked = 0
    for n, group in sorted(by_side.items()):
        kappa, leaf = group[0][1]["kappa"], group[0][1]["leaf"]
        h = 1.0 / n
        bs = np.stack([inputs.gaussian_family(n, p["b_seed"]) for _, p in group])
        F = ls.ls_build(n, h, kappa, dev(bs), 1e-4, leaf_side=leaf, precision=ls.LS_TF32X3)
        rhs = ls.ls_rhs_plane_wave(F, [0.0], zeros(len(group), n, n))
        sig = zeros(len(group), n, n)
        infos = ls.ls_solve(F, rhs, sig)
        assert all(i["converged"] and i["resid_true"] <= 1e-10 for i in infos), infos
        S = host(sig)
        spec = nystrom.conv_kernel_spectrum(kappa, h, n, n, 10)
        g = 0
        f = nystrom.rhs(kappa, bs[g], n, n, h)
        r = np.linalg.norm(f - nystrom.matvec_fft(spec, kappa, bs[g], S[g].ravel())) / np.linalg.norm(f)
        assert r <= 1e-10, (n, r)
        checked += len(group)
        ls.ls_free(F)
    assert checked == 32
