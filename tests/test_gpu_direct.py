"""The HBS inverse as a direct solver (Sec. 6.1): b = 1.5 exp(-160 |x|^2), kappa = 25,
10th-order corrections inside the HBS and in the operator, 100-point leaves.

* eps = 1e-12 (FP64) at 80^2: M f equals the oracle's solution of the 10th-order
  system (its GMRES on its FFT operator to 1e-13) to 1e-10, and the direct residual
  ||f - A M f|| / ||f|| is below 1e-10 (the paper's table: 1.9e-15).
* eps = 1e-9 (FP64) at 160^2 and eps = 1e-6 (tf32x3) at 160^2: direct residuals below
  100 eps (the paper's: 3.4e-12 and 7.1e-8).
"""
import numpy as np
import pytest

import paper_2007_12718_gb300 as ls
from oracle import gmres as ogmres
from oracle import nystrom
from paper_2007_12718_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def zeros(n):
    return torch.zeros(n, n, dtype=torch.complex128, device=DEV)


def direct(n, eps, precision):
    h, kappa = 1.0 / n, 25.0
    b = inputs.gaussian_direct(n)
    H = ls.ls_build(n, h, kappa, b, eps, leaf_side=10, order_precond=10, order_matvec=10, precision=precision)
    f = ls.ls_rhs_plane_wave(H, [0.0], zeros(n))
    q = ls.ls_apply(H, f, zeros(n))
    y = ls.ls_matvec(H, q, zeros(n))
    res = float(torch.linalg.norm(f - y) / torch.linalg.norm(f))
    torch.cuda.synchronize()
    out = q.cpu().numpy().ravel(), f.cpu().numpy().ravel(), res
    ls.ls_free(H)
    return out


def test_direct_eps_1e12_vs_oracle_80():
    n, kappa = 80, 25.0
    h = 1.0 / n
    q, f, res = direct(n, 1e-12, ls.LS_FP64)
    assert res < 1e-10, res
    b = inputs.gaussian_direct(n)
    spec = nystrom.conv_kernel_spectrum(kappa, h, n, n, 10)
    ref, _, _ = ogmres.gmres(lambda v: nystrom.matvec_fft(spec, kappa, b, v), f, tol=1e-13)
    assert np.linalg.norm(q - ref) / np.linalg.norm(ref) < 1e-10


@pytest.mark.parametrize("eps,precision", [(1e-9, ls.LS_FP64), (1e-6, ls.LS_TF32X3)])
def test_direct_residual_160(eps, precision):
    _, _, res = direct(160, eps, precision)
    assert res < 100 * eps, res
