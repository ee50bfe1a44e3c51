"""Reuse and persistence of built data (the compression does not depend on b,
Sec. 3.2).

* reuse_compression: a second build with the same grid, kappa and tolerance but
  another potential takes the compression from the cache (same ranks and
  skeleton sizes), its apply agrees with a fresh build's to rounding, and it is
  within 5 eps of the dense inverse for the new b.
* ls_save / ls_load: the restored handle applies (forward and transposed) and
  solves bit for bit as the saved one; a truncated file is refused.
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


@pytest.mark.parametrize("precision", [ls.LS_FP64, ls.LS_FP32])
def test_reused_compression(precision):
    n, kappa, eps = 64, 40.0, 1e-4
    b0, b1 = inputs.gaussian_family(n, 0), inputs.gaussian_family(n, 1)
    ls.ls_compression_cache_clear()
    H0 = ls.ls_build(n, 1.0 / n, kappa, b0, eps, precision=precision, reuse_compression=1, woodbury=2)
    assert not H0.info()["compression_reused"]
    H1 = ls.ls_build(n, 1.0 / n, kappa, b1, eps, precision=precision, reuse_compression=1, woodbury=2)
    Hf = ls.ls_build(n, 1.0 / n, kappa, b1, eps, precision=precision, woodbury=2)
    i1, iff = H1.info(), Hf.info()
    assert i1["compression_reused"] and not iff["compression_reused"]
    assert i1["ranks"] == iff["ranks"] and i1["sibling_ranks"] == iff["sibling_ranks"]
    f = inputs.random_complex((n, n), 7)
    q1 = host(ls.ls_apply(H1, dev(f), zeros(n, n)))
    qf = host(ls.ls_apply(Hf, dev(f), zeros(n, n)))
    assert rel(q1, qf) <= (1e-12 if precision == ls.LS_FP64 else 1e-5)
    A = nystrom.dense_operator(kappa, 1.0 / n, b1, 4)
    assert rel(q1.ravel(), nystrom.solve_dense(A, f.ravel())) < 5 * eps
    # another kappa is another key
    H2 = ls.ls_build(n, 1.0 / n, kappa * 1.01, b1, eps, precision=precision, reuse_compression=1)
    assert not H2.info()["compression_reused"]
    for H in (H0, H1, Hf, H2):
        ls.ls_free(H)
    ls.ls_compression_cache_clear()


@pytest.mark.parametrize("precision", [ls.LS_FP64, ls.LS_TF32X3])
def test_save_load_roundtrip(tmp_path, precision):
    n, kappa, eps = 64, 40.0, 1e-4
    h = 1.0 / n
    b = inputs.gaussian_family(n, 0)
    H = ls.ls_build(n, h, kappa, b, eps, precision=precision, top_uncompressed=1)
    path = tmp_path / "h.lshbs"
    ls.ls_save(H, path)
    G = ls.ls_load(path)
    ia, ib = H.info(), G.info()
    assert ib["compression_reused"] and ia["ranks"] == ib["ranks"] and ia["sibling_ranks"] == ib["sibling_ranks"]
    assert ia["factor_bytes"] == ib["factor_bytes"]
    f = dev(inputs.random_complex((2, n, n), 9))
    for tr in (False, True):
        qa = host(ls.ls_apply(H, f, zeros(2, n, n), transpose=tr))
        qb = host(ls.ls_apply(G, f, zeros(2, n, n), transpose=tr))
        np.testing.assert_array_equal(qa, qb)
    rhs = dev(nystrom.rhs(kappa, b, n, n, h).reshape(n, n))
    sa, sb = zeros(n, n), zeros(n, n)
    ia = ls.ls_solve(H, rhs, sa)[0]
    ib = ls.ls_solve(G, rhs, sb)[0]
    assert ia["iterations"] == ib["iterations"] and ib["converged"]
    np.testing.assert_array_equal(host(sa), host(sb))
    ls.ls_free(H)
    ls.ls_free(G)
    data = path.read_bytes()
    bad = tmp_path / "cut.lshbs"
    bad.write_bytes(data[: len(data) // 2])
    with pytest.raises(ls.LSError):
        ls.ls_load(bad)
