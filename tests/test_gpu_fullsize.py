"""GPU parity at the measured sizes, against references the CPU oracle computes
without the GPU path.

* The preconditioner alone (256^2, kappa = 60, eps = 1e-4): the exact
  q = (I + B G_4)^-1 f is too large for a dense solve; the oracle's GMRES on
  its own FFT operator A_4, preconditioned by its own HBS inverse, gives it to
  1e-13.  The method itself does not reach 5 eps at this size (the oracle's HBS
  inverse, FP64 with the greedy CPQR, is ~9 eps off on a random f and ~80 eps
  on the plane-wave right-hand side): the GPU inverse must be within 5 eps or
  within 1.5x the oracle's own error on the same f, whichever is larger.
* Mixed (tf32x3, FP16 split, FP32 HBS) vs FP64 paths: the scattered fields u = (G+T) sigma
  of the two GMRES solutions agree to 1e-9 (both are solves to 1e-10 of the
  same FP64 system; the preconditioner only changes the iterates).
* The 2048^2 workload of the benchmark (kappa = 400 pi): the true residual of
  the mixed solve, measured with the oracle's numpy FFT matvec, is <= 1e-10.
"""
import numpy as np
import pytest

import paper_2007_12718_gb300 as ls
from oracle import gmres as ogmres
from oracle import hbs as ohbs
from oracle import nystrom
from paper_2007_12718_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]
DEV = "cuda:0"


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def n256():
    n, kappa, eps = 256, 60.0, 1e-4
    h = 1.0 / n
    b = inputs.gaussian_family(n, 0)
    comp = ohbs.Compression(kappa, h, ohbs.Tree(n, n, 8), 4, eps, 2)
    inv = ohbs.Inverse(comp, b)
    spec4 = nystrom.conv_kernel_spectrum(kappa, h, n, n, 4)
    cases = {}
    for name, f in (("random", inputs.random_complex(n * n, 5)), ("plane", nystrom.rhs(kappa, b, n, n, h))):
        qref, k, _ = ogmres.gmres(lambda v: nystrom.matvec_fft(spec4, kappa, b, v), f, apply_M=inv.apply, tol=1e-13)
        cases[name] = (f, qref, rel(inv.apply(f), qref))
    return dict(n=n, kappa=kappa, eps=eps, b=b, cases=cases)


@pytest.mark.parametrize("precision,kw", [(ls.LS_FP64, {}), (ls.LS_FP32, {}), (ls.LS_TF32X3, {}),
                                          (ls.LS_TF32X3, {"top_uncompressed": 1}),
                                          (ls.LS_FP32, {"id_method": ls.LS_ID_GREEDY}),
                                          (ls.LS_TF32X3, {"woodbury": 0}), (ls.LS_FP64, {"woodbury": 0}),
                                          (ls.LS_FP16SPLIT, {}), (ls.LS_FP16SPLIT, {"top_uncompressed": 1})])
def test_preconditioner_forward_error_n256(n256, precision, kw):
    n, eps = n256["n"], n256["eps"]
    H = ls.ls_build(n, 1.0 / n, n256["kappa"], n256["b"], eps, precision=precision, **kw)
    info = H.info()
    assert info["pivot_fallbacks"] == 0
    unit = 1.11e-16 if precision == ls.LS_FP64 else 5.96e-8
    assert info["probe_resid_max"] <= max(eps, 10 * unit * max(info["ranks"])), info["probe_resid_max"]
    for name, (f, qref, err_oracle) in n256["cases"].items():
        q = host(ls.ls_apply(H, dev(f.reshape(n, n)), torch.zeros(n, n, dtype=torch.complex128, device=DEV)))
        err = rel(q.ravel(), qref)
        assert err <= max(5 * eps, 1.5 * err_oracle), (name, err, err_oracle)
    ls.ls_free(H)


def test_mixed_vs_fp64_fields_agree_n256():
    n, kappa = 256, 60.0
    b = inputs.gaussian_family(n, 0)
    f = dev(nystrom.rhs(kappa, b, n, n, 1.0 / n).reshape(n, n))
    u = {}
    for precision in (ls.LS_FP64, ls.LS_FP32, ls.LS_TF32X3, ls.LS_FP16SPLIT):
        H = ls.ls_build(n, 1.0 / n, kappa, b, 1e-4, precision=precision)
        sig = torch.zeros(n, n, dtype=torch.complex128, device=DEV)
        info = ls.ls_solve(H, f, sig)[0]
        assert info["converged"]
        u[precision] = host(ls.ls_field(H, sig, torch.zeros(n, n, dtype=torch.complex128, device=DEV)))
        ls.ls_free(H)
    assert rel(u[ls.LS_FP32], u[ls.LS_FP64]) <= 1e-9
    assert rel(u[ls.LS_TF32X3], u[ls.LS_FP64]) <= 1e-9
    assert rel(u[ls.LS_FP16SPLIT], u[ls.LS_FP64]) <= 1e-9


def test_precond_n2048_true_residual():
    """The benchmark's headline workload and configuration (tf32x3 merges, every
    level compressed): 7-8 GMRES iterations, true residual <= 1e-10 by the oracle's
    FFT matvec, and no merge inverse needed the row-pivoted fallback."""
    w = inputs.WORKLOADS["precond_n2048"]
    n, kappa = w["n"], w["kappa"]
    h = 1.0 / n
    b = w["b"](n)
    H = ls.ls_build(n, h, kappa, dev(b), w["eps"], precision=ls.LS_TF32X3)
    f = nystrom.rhs(kappa, b, n, n, h)
    sig = torch.zeros(n, n, dtype=torch.complex128, device=DEV)
    info = ls.ls_solve(H, dev(f.reshape(n, n)), sig)[0]
    bi = H.info()
    ls.ls_free(H)
    s = host(sig).ravel()
    del sig
    spec = nystrom.conv_kernel_spectrum(kappa, h, n, n, w["order_matvec"])
    r = np.linalg.norm(f - nystrom.matvec_fft(spec, kappa, b, s)) / np.linalg.norm(f)
    assert info["converged"] and r <= 1e-10, (info, r)
    assert info["iterations"] <= 12
    assert bi["pivot_fallbacks"] == 0
    assert bi["levels"] == 16 and bi["ranks"][16] > 0


@pytest.mark.parametrize("n", [80, 160])
def test_cavity_sweep_members(n):
    """The cavity of Sec. 6.2-6.3 at 10 points per wavelength with 100-point leaves
    (the paper's sweep, Table of Sec. 6.3): at 80^2 sigma matches the oracle's dense
    LU of the 10th-order system; at 160^2 the true residual by the oracle's FFT
    matvec is <= 1e-10; GMRES iterations within one of the paper's (4, 5)."""
    w = inputs.WORKLOADS[f"cavity_n{n}"]
    kappa = w["kappa"]
    h = 1.0 / n
    b = w["b"](n)
    f = nystrom.rhs(kappa, b, n, n, h)
    for precision in (ls.LS_TF32X3, ls.LS_FP64):
        H = ls.ls_build(n, h, kappa, b, w["eps"], leaf_side=w["leaf"], precision=precision)
        sig = torch.zeros(n, n, dtype=torch.complex128, device=DEV)
        info = ls.ls_solve(H, dev(f.reshape(n, n)), sig)[0]
        ls.ls_free(H)
        s = host(sig).ravel()
        assert info["converged"] and abs(info["iterations"] - {80: 4, 160: 5}[n]) <= 1, info
        if n == 80:
            A = nystrom.dense_operator(kappa, h, b, 10)
            assert rel(s, nystrom.solve_dense(A, f)) <= 1e-9
        else:
            spec = nystrom.conv_kernel_spectrum(kappa, h, n, n, 10)
            assert np.linalg.norm(f - nystrom.matvec_fft(spec, kappa, b, s)) / np.linalg.norm(f) <= 1e-10
