"""Error paths on the GPU, none of which faults or hangs the device.

* A bounded device-side wait that runs out: the handle's poll limit
  (ls_opts.wait_limit) set to one poll makes the grid barriers of the greedy ID
  kernel (during ls_build) or of the persistent apply kernel (ls_apply,
  ls_solve) give up; the call returns LS_ETIMEOUT, the kernels unwind, and the
  context stays usable for the next handle.
* GMRES that reaches its iteration limit: LS_ENOCONV, sigma and info written.
* Host-side injection (ls_fault_inject): a failing device allocation at several
  points of ls_build (LS_ENOMEM, everything allocated so far released), and a
  NaN in b (LS_EINVAL from the finiteness check).
* The misfit without a gradient runs no adjoint solve and gives the same J.
"""
import numpy as np
import pytest

import paper_2007_12718_gb300 as ls
from paper_2007_12718_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def good_solve(n=64, kappa=40.0):
    b = inputs.gaussian_family(n, 0)
    H = ls.ls_build(n, 1.0 / n, kappa, b, 1e-4)
    f = torch.zeros(n, n, dtype=torch.complex128, device=DEV)
    ls.ls_rhs_plane_wave(H, [0.0], f)
    sig = torch.zeros_like(f)
    info = ls.ls_solve(H, f, sig)[0]
    ls.ls_free(H)
    assert info["converged"] and info["resid_true"] < 2e-10


def test_wait_limit_times_out_grid_id_in_build():
    """256^2 with the greedy ID: the level-3 proxy block (504 candidates) runs on
    the cooperative grid kernel, whose per-pivot barrier gives up after one poll."""
    n = 256
    with pytest.raises(ls.LSError) as e:
        ls.ls_build(n, 1.0 / n, 60.0, inputs.gaussian_family(n, 0), 1e-4, id_method=ls.LS_ID_GREEDY, wait_limit=1)
    assert e.value.code == ls.LS_ETIMEOUT
    good_solve()


def test_wait_limit_times_out_apply_and_solve():
    """The blocked ID and the merges wait on no grid barrier, so the build succeeds;
    the persistent apply kernel's phase barriers then give up."""
    n = 64
    b = inputs.gaussian_family(n, 0)
    H = ls.ls_build(n, 1.0 / n, 40.0, b, 1e-4, id_method=ls.LS_ID_BLOCKED, wait_limit=1)
    f = torch.from_numpy(inputs.random_complex((n, n), 1)).to(DEV)
    ls.ls_apply(H, f, torch.zeros_like(f))  # asynchronous: the status shows at the next synchronising call
    with pytest.raises(ls.LSError) as e:
        ls.ls_sync(H)
    assert e.value.code == ls.LS_ETIMEOUT
    ls.ls_free(H)
    H = ls.ls_build(n, 1.0 / n, 40.0, b, 1e-4, id_method=ls.LS_ID_BLOCKED, wait_limit=1)
    with pytest.raises(ls.LSError) as e:
        ls.ls_solve(H, f, torch.zeros_like(f))
    assert e.value.code == ls.LS_ETIMEOUT
    ls.ls_free(H)
    good_solve()


def test_gmres_iteration_limit_returns_noconv():
    n, kappa = 64, 40.0
    b = inputs.gaussian_family(n, 0)
    H = ls.ls_build(n, 1.0 / n, kappa, b, 1e-4, gmres_maxit=1)
    f = torch.zeros(n, n, dtype=torch.complex128, device=DEV)
    ls.ls_rhs_plane_wave(H, [0.0], f)
    sig = torch.zeros_like(f)
    with pytest.raises(ls.LSError) as e:
        ls.ls_solve(H, f, sig)
    assert e.value.code == ls.LS_ENOCONV
    info = ls.ls_solve(H, f, sig, allow_noconv=True)[0]
    assert not info["converged"] and info["iterations"] == 1 and info["resid_est"] > 1e-10
    assert torch.count_nonzero(sig).item() > 0  # the one-step iterate is written
    ls.ls_free(H)


@pytest.mark.parametrize("nth", [1, 2, 5, 12, 40])
def test_injected_allocation_failure(nth):
    n = 64
    b = inputs.gaussian_family(n, 0)
    ls.ls_fault_inject(f"alloc:{nth}")
    try:
        with pytest.raises(ls.LSError) as e:
            ls.ls_build(n, 1.0 / n, 40.0, b, 1e-4)
        assert e.value.code == ls.LS_ENOMEM
    finally:
        ls.ls_fault_inject("")
    good_solve()


def test_injected_nan_in_b():
    n = 32
    ls.ls_fault_inject("nan_b")
    try:
        with pytest.raises(ls.LSError) as e:
            ls.ls_build(n, 1.0 / n, 20.0, inputs.gaussian_bump(n), 1e-4)
        assert e.value.code == ls.LS_EINVAL
    finally:
        ls.ls_fault_inject("")
    good_solve(32, 20.0)


def test_misfit_without_gradient():
    n, kappa, ndir = 64, 30.0, 2
    thetas = inputs.plane_wave_angles(ndir)
    rec = inputs.receivers_circle(16)
    b = torch.from_numpy(inputs.gaussian_family(n, 0)).to(DEV)
    H = ls.ls_build(n, 1.0 / n, kappa, b, 1e-4)
    ls.ls_set_receivers(H, rec)
    data = torch.zeros(ndir, 16, dtype=torch.complex128, device=DEV)
    grad = torch.zeros(n, n, dtype=torch.float64, device=DEV)
    k0 = ls.ls_kernel_launches()
    J1, inf1 = ls.ls_misfit_gradient(H, thetas, data, grad)
    k1 = ls.ls_kernel_launches()
    J2, inf2 = ls.ls_misfit_gradient(H, thetas, data, None)
    k2 = ls.ls_kernel_launches()
    ls.ls_free(H)
    assert abs(J1 - J2) <= 1e-12 * abs(J1)
    assert inf2[ndir]["iterations"] == 0 and k2 - k1 < k1 - k0
