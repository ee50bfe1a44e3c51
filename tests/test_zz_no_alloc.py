"""The allocation-free matvec (ls_matvec_noalloc) against the regular one.

ls_matvec_noalloc serves callers that must not allocate device memory while
they apply the operator (a framework pool holding the free memory, loops that
cannot take cudaMalloc's implicit synchronisation, fixed memory budgets).  It
runs the same FFT convolution with its scratch in a fixed device array inside
the library.  This file is collected last on purpose; it must pass both alone
in a fresh process and after the other tests.
"""
import numpy as np
import pytest

import paper_2007_12718_gb300 as ls
from paper_2007_12718_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def test_noalloc_matvec_matches_matvec_twice():
    n, kappa = 64, 25.0
    b = inputs.gaussian_family(n, 3)
    H = ls.ls_build(n, 1.0 / n, kappa, b, 1e-4)
    for seed, nrhs in ((5, 1), (6, 2)):  # two calls in a row; the second reuses the array
        x = torch.from_numpy(inputs.random_complex((nrhs, n, n), seed)).to(DEV)
        y_ref = ls.ls_matvec(H, x, torch.zeros_like(x))
        y0 = torch.full_like(x, 7.0)
        allocs = ls.ls_allocations()  # the library's own count of its device and pinned allocations
        y = ls.ls_matvec_noalloc(H, x, y0)
        torch.cuda.synchronize()
        assert ls.ls_allocations() == allocs
        a, r = y.cpu().numpy(), y_ref.cpu().numpy()
        for k in range(nrhs):
            assert np.linalg.norm(a[k] - r[k]) / np.linalg.norm(r[k]) < 1e-12


def test_noalloc_rejects_oversize_and_host_buffers():
    n = 256
    H = ls.ls_build(n, 1.0 / n, 30.0, inputs.gaussian_family(n, 1), 1e-4)
    cap = ls.load_library().ls_matvec_noalloc_max_elems()
    nrhs = cap // (n * 2 * n) + 1  # one right-hand side more than the array holds
    x = torch.zeros(nrhs, n, n, dtype=torch.complex128, device=DEV)
    with pytest.raises(ls.LSError) as e:
        ls.ls_matvec_noalloc(H, x, torch.zeros_like(x))
    assert e.value.code == ls.LS_EINVAL
    xh = np.zeros((n, n), np.complex128)
    with pytest.raises(ls.LSError):
        ls.ls_matvec_noalloc(H, xh, np.zeros_like(xh))
