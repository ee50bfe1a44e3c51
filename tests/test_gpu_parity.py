"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances (all relative, 2-norm unless stated):
* matvec (FP64 FFT convolution vs the oracle's dense matrix): 1e-12.  An FFT of
  length L in FP64 has error ~ log2(L) * 1e-16 relative to ||K|| ||x||.
* kernel values through the matvec impulse response: 1e-12 of max |K|.
* HBS inverse at tolerance eps vs the dense inverse of I + B G_p: 5 eps
  (the scheme's target, Sec. 3.2 Eq. (11) and Sec. 5); FP32 storage adds
  ~1e-6, so FP32 runs use eps >= 1e-4.
* preconditioned GMRES to 1e-10 vs dense LU: 1e-9 on sigma (cond(A) ~ 10 here)
  and the true residual, measured with the oracle's own FFT matvec, <= 2e-10.
"""
import numpy as np
import pytest

import paper_2007_12718_gb300 as ls
from oracle import hbs as ohbs
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


def build(n, kappa, b, eps, order_precond=4, order_matvec=10, precision=ls.LS_FP64, ny=None, **kw):
    return ls.ls_build(n, 1.0 / n, kappa, b, eps, order_matvec=order_matvec, order_precond=order_precond,
                       precision=precision, ny=ny, **kw)


@pytest.mark.parametrize("order", [2, 4, 6, 8, 10])
def test_matvec_impulse_response_is_kernel(order):
    """y = x + kappa^2 b (K * x) with b = 1 and x = e_c gives kappa^2 K(m) + delta:
    every kernel value h^2 (G + tau) compared with the oracle."""
    n, kappa = 32, 20.0
    b = np.ones((n, n))
    H = build(n, kappa, b, 1e-4, order_matvec=order)
    x = np.zeros((n, n), np.complex128)
    x[12, 9] = 1.0
    y = host(ls.ls_matvec(H, dev(x), torch.zeros(n, n, dtype=torch.complex128, device=DEV)))
    K = nystrom.kernel_offsets(kappa, 1.0 / n, order, n - 1, n - 1)
    ref = np.zeros((n, n), np.complex128)
    for j in range(n):
        for i in range(n):
            ref[j, i] = kappa ** 2 * K[j - 12 + n - 1, i - 9 + n - 1]
    ref[12, 9] += 1.0
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("n,ny,order,nrhs", [(32, 32, 10, 1), (64, 64, 4, 3), (32, 16, 10, 2), (128, 128, 10, 1)])
def test_matvec_vs_dense(n, ny, order, nrhs):
    kappa = 25.0
    X, Y = inputs.grid_nodes(n)
    b = inputs.gaussian_family(n, 3)[:ny, :]
    H = build(n, kappa, b, 1e-4, order_matvec=order, ny=ny)
    x = inputs.random_complex((nrhs, ny, n), 11)
    y = host(ls.ls_matvec(H, dev(x), torch.zeros(nrhs, ny, n, dtype=torch.complex128, device=DEV)))
    h = 1.0 / n
    if n * ny <= 4096:
        A = nystrom.dense_operator(kappa, h, b, order)
        ref = (A @ x.reshape(nrhs, -1).T).T.reshape(x.shape)
    else:
        spec = nystrom.conv_kernel_spectrum(kappa, h, n, ny, order)
        ref = nystrom.matvec_fft(spec, kappa, b, x.reshape(nrhs, -1)).reshape(x.shape)
    for r in range(nrhs):
        assert rel(y[r], ref[r]) < 1e-12


@pytest.mark.parametrize("n,ny,leaf", [(40, 40, 5), (80, 40, 10), (48, 24, 6)])
def test_matvec_non_power_of_two_grid(n, ny, leaf):
    """Grids whose padded FFT length is not 2n (the circulant embedded at the next
    power of two, zeros between the positive and negative offsets): the matvec
    still equals the oracle's dense 10th-order operator."""
    kappa = 25.0
    b = inputs.gaussian_family(n, 5)[:ny, :]
    H = build(n, kappa, b, 1e-4, order_matvec=10, ny=ny, leaf_side=leaf)
    x = inputs.random_complex((2, ny, n), 12)
    y = host(ls.ls_matvec(H, dev(x), torch.zeros(2, ny, n, dtype=torch.complex128, device=DEV)))
    A = nystrom.dense_operator(kappa, 1.0 / n, b, 10)
    ref = (A @ x.reshape(2, -1).T).T.reshape(x.shape)
    for r in range(2):
        assert rel(y[r], ref[r]) < 1e-12


def test_matvec_host_buffers_match_device():
    n, kappa = 32, 15.0
    b = inputs.gaussian_bump(n)
    H = build(n, kappa, b, 1e-4)
    x = inputs.random_complex((n, n), 4)
    yd = host(ls.ls_matvec(H, dev(x), torch.zeros(n, n, dtype=torch.complex128, device=DEV)))
    yh = ls.ls_matvec(H, x, np.zeros((n, n), np.complex128))
    np.testing.assert_array_equal(yd, yh)


@pytest.mark.parametrize("precision,eps", [(ls.LS_FP64, 1e-4), (ls.LS_FP32, 1e-4), (ls.LS_FP64, 1e-7)])
def test_hbs_apply_vs_dense_inverse(precision, eps):
    n, kappa = 32, 20.0
    b = inputs.gaussian_bump(n)
    H = build(n, kappa, b, eps, precision=precision)
    assert H.info()["pivot_fallbacks"] == 0
    A = nystrom.dense_operator(kappa, 1.0 / n, b, 4)
    for seed in (1, 2):
        f = inputs.random_complex((n, n), seed)
        q = host(ls.ls_apply(H, dev(f), torch.zeros(n, n, dtype=torch.complex128, device=DEV)))
        ref = nystrom.solve_dense(A, f.ravel()).reshape(n, n)
        assert rel(q, ref) < 5 * eps


def test_hbs_direct_solver_order10_vs_lu():
    """Plain method at the oracle size: 32 x 32, kappa = 20, Gaussian b, 10th order,
    eps = 1e-10, FP64: the HBS inverse applied to f is the direct solve (Sec. 4.1)."""
    n, kappa, eps = 32, 20.0, 1e-10
    b = inputs.gaussian_bump(n)
    H = build(n, kappa, b, eps, order_precond=10, order_matvec=10, precision=ls.LS_FP64)
    f = nystrom.rhs(kappa, b, n, n, 1.0 / n).reshape(n, n)
    q = host(ls.ls_apply(H, dev(f), torch.zeros(n, n, dtype=torch.complex128, device=DEV)))
    A = nystrom.dense_operator(kappa, 1.0 / n, b, 10)
    ref = nystrom.solve_dense(A, f.ravel()).reshape(n, n)
    assert rel(q, ref) < 5 * eps


@pytest.mark.parametrize("precision,pivoting", [(ls.LS_FP64, 0), (ls.LS_FP32, 0), (ls.LS_FP32, 1), (ls.LS_FP64, 1)])
def test_gmres_solve_vs_lu(precision, pivoting):
    """n = 64 has merge matrices of size ~190 (kc), large enough for the blocked
    inverses: pivoting 0 = blocks without interchanges (checked), 1 = row-pivoted."""
    n, kappa = 64, 40.0
    b = inputs.gaussian_family(n, 0)
    H = build(n, kappa, b, 1e-4, precision=precision, merge_pivoting=pivoting)
    f = nystrom.rhs(kappa, b, n, n, 1.0 / n).reshape(n, n)
    sig = torch.zeros(n, n, dtype=torch.complex128, device=DEV)
    info = ls.ls_solve(H, dev(f), sig)[0]
    s = host(sig)
    assert info["converged"] and info["resid_true"] < 2e-10
    A = nystrom.dense_operator(kappa, 1.0 / n, b, 10)
    ref = nystrom.solve_dense(A, f.ravel()).reshape(n, n)
    assert rel(s, ref) < 1e-9
    assert info["iterations"] < 30
    assert H.info()["pivot_fallbacks"] == 0


def test_rhs_plane_wave_matches_oracle():
    n, kappa = 32, 20.0
    b = inputs.gaussian_family(n, 2)
    H = build(n, kappa, b, 1e-4)
    th = np.array([0.0, 0.7])
    f = host(ls.ls_rhs_plane_wave(H, th, torch.zeros(2, n, n, dtype=torch.complex128, device=DEV)))
    for r in range(2):
        ref = nystrom.rhs(kappa, b, n, n, 1.0 / n, th[r]).reshape(n, n)
        assert np.abs(f[r] - ref).max() < 1e-12 * np.abs(ref).max()


def test_zero_potential_gives_zero_density():
    n = 32
    b = np.zeros((n, n))
    H = build(n, 20.0, b, 1e-4)
    f = torch.zeros(n, n, dtype=torch.complex128, device=DEV)
    sig = torch.ones(n, n, dtype=torch.complex128, device=DEV)
    info = ls.ls_solve(H, f, sig)[0]
    assert info["iterations"] == 0 and torch.count_nonzero(sig).item() == 0
    x = inputs.random_complex((n, n), 3)
    y = host(ls.ls_matvec(H, dev(x), torch.zeros(n, n, dtype=torch.complex128, device=DEV)))
    np.testing.assert_array_equal(y, x)  # A = I when b = 0


def test_invalid_arguments_rejected():
    n = 32
    with pytest.raises(ls.LSError) as e:
        build(n, 20.0, np.full((n, n), np.nan), 1e-4)
    assert e.value.code == ls.LS_EINVAL
    with pytest.raises(ls.LSError):
        ls.ls_build(24, 1 / 24, 20.0, np.zeros((24, 24)), 1e-4, leaf_side=8)  # 24 = 8 * 3
    with pytest.raises(ls.LSError):
        build(n, 20.0, np.zeros((n, n)), 1e-4, order_matvec=7)


def test_ranks_match_oracle_compression():
    """Skeleton sets are not unique, but the ranks chosen by the same rule on the
    same proxy blocks agree to within rounding near the threshold (CPQR by
    projections on the GPU, Householder in LAPACK): 2% or 2, whichever is larger."""
    n, kappa, eps = 64, 30.0, 1e-6
    b = inputs.gaussian_bump(n)
    H = build(n, kappa, b, eps, precision=ls.LS_FP64, proxy_width=2)
    got = H.info()["ranks"]
    comp = ohbs.Compression(kappa, 1.0 / n, ohbs.Tree(n, n, 8), 4, eps, 2)
    for l in range(1, len(got)):
        assert abs(got[l] - comp.rank[l]) <= max(2, 0.02 * comp.rank[l]), (got, comp.rank)


@pytest.mark.slow
def test_precond_solve_full_size_n256():
    """The measured workload (256 x 256, kappa = 60, 20-Gaussian b, eps = 1e-4), also
    in the measured configuration (tf32x3 merges, level 1 uncompressed): the true
    residual is checked with the oracle's own FFT matvec."""
    n, kappa = 256, 60.0
    b = inputs.gaussian_family(n, 0)
    spec = nystrom.conv_kernel_spectrum(kappa, 1.0 / n, n, n, 10)
    f = nystrom.rhs(kappa, b, n, n, 1.0 / n).reshape(n, n)
    for precision, kw in ((ls.LS_FP32, {}), (ls.LS_FP64, {}), (ls.LS_TF32X3, {"top_uncompressed": 1})):
        H = build(n, kappa, b, 1e-4, precision=precision, **kw)
        sig = torch.zeros(n, n, dtype=torch.complex128, device=DEV)
        info = ls.ls_solve(H, dev(f), sig)[0]
        s = host(sig).ravel()
        r = f.ravel() - nystrom.matvec_fft(spec, kappa, b, s)
        assert info["converged"]
        assert np.linalg.norm(r) / np.linalg.norm(f) < 2e-10
        # the merge inverses of orders up to 1014 (16 panels, a ragged last one) pass
        # their probe check without the row-pivoted fallback
        assert H.info()["pivot_fallbacks"] == 0, (precision, kw)
        ls.ls_free(H)


@pytest.mark.parametrize("precision", [ls.LS_TF32X3, ls.LS_FP16SPLIT])
def test_tensor_core_build(precision):
    """The tensor-core precision modes (tf32x3, FP16 split) at the oracle size: the
    HBS inverse stays within 5 eps of the dense inverse, and GMRES (FP64, FP64
    matvec) reaches the dense solution.  (At 64^2 the products are below the
    tensor cores' size threshold; the 256^2 tests of test_gpu_fullsize.py are
    where they run.)"""
    n, kappa = 64, 40.0
    b = inputs.gaussian_family(n, 0)
    H = build(n, kappa, b, 1e-4, precision=precision)
    A4 = nystrom.dense_operator(kappa, 1.0 / n, b, 4)
    f = inputs.random_complex((n, n), 1)
    q = host(ls.ls_apply(H, dev(f), torch.zeros(n, n, dtype=torch.complex128, device=DEV)))
    err = rel(q, nystrom.solve_dense(A4, f.ravel()).reshape(n, n))
    assert err < 5e-4, err
    fr = nystrom.rhs(kappa, b, n, n, 1.0 / n).reshape(n, n)
    sig = torch.zeros(n, n, dtype=torch.complex128, device=DEV)
    info = ls.ls_solve(H, dev(fr), sig)[0]
    A10 = nystrom.dense_operator(kappa, 1.0 / n, b, 10)
    assert info["converged"] and info["resid_true"] < 2e-10
    assert rel(host(sig), nystrom.solve_dense(A10, fr.ravel()).reshape(n, n)) < 1e-9


def test_plain_tf32_preconditioner_rejected():
    """One tf32 product per merge GEMM (~1e-3 relative error) cannot keep the HBS
    inverse within its tolerance: ls_build refuses the mode."""
    n = 32
    with pytest.raises(ls.LSError) as e:
        build(n, 20.0, inputs.gaussian_bump(n), 1e-4, precision=ls.LS_TF32)
    assert e.value.code == ls.LS_EINVAL


@pytest.mark.parametrize("precision", [ls.LS_FP32, ls.LS_FP64])
def test_top_level_uncompressed(precision):
    """top_uncompressed = 1 keeps every row of level 1 (U = I): still an HBS inverse
    of I + B G within 5 eps, with rank k_1 = m_1."""
    n, kappa = 64, 30.0
    b = inputs.gaussian_family(n, 4)
    H = build(n, kappa, b, 1e-4, precision=precision, top_uncompressed=1)
    info = H.info()
    assert info["ranks"][1] == 2 * info["ranks"][2]
    A4 = nystrom.dense_operator(kappa, 1.0 / n, b, 4)
    f = inputs.random_complex((n, n), 6)
    q = host(ls.ls_apply(H, dev(f), torch.zeros(n, n, dtype=torch.complex128, device=DEV)))
    assert rel(q, nystrom.solve_dense(A4, f.ravel()).reshape(n, n)) < 5e-4


@pytest.mark.parametrize("precision", [ls.LS_FP32, ls.LS_FP64])
def test_apply_graph_path_matches_persistent(precision, monkeypatch):
    """The CUDA-graph apply (used when the persistent grid cannot be co-resident,
    forced here with LS_APPLY_GRAPH) computes the same Algorithm 2: forward and
    transposed applies agree with the persistent kernel's to rounding."""
    n, kappa = 64, 40.0
    b = inputs.gaussian_family(n, 3)
    f = inputs.random_complex((n, n), 8)
    out = {}
    for mode in ("persistent", "graph"):
        if mode == "graph":
            monkeypatch.setenv("LS_APPLY_GRAPH", "1")
        H = build(n, kappa, b, 1e-4, precision=precision, top_uncompressed=1)
        out[mode] = (host(ls.ls_apply(H, dev(f), torch.zeros(n, n, dtype=torch.complex128, device=DEV))),
                     host(ls.ls_apply(H, dev(f), torch.zeros(n, n, dtype=torch.complex128, device=DEV), transpose=True)))
        ls.ls_free(H)
    tol = 1e-5 if precision == ls.LS_FP32 else 1e-12
    assert rel(out["graph"][0], out["persistent"][0]) < tol
    assert rel(out["graph"][1], out["persistent"][1]) < tol


@pytest.mark.parametrize("precision", [ls.LS_FP64, ls.LS_TF32X3])
def test_lens_potential_above_one(precision):
    """The lens of Sec. 6.2 (b from about -2.69 to 1.18, beyond the b <= 1 of the
    existence theorem) at 80^2 with 100-point leaves and kappa = 40: the density
    matches the oracle's dense LU of the 10th-order system to 1e-9."""
    n, kappa = 80, 40.0
    h = 1.0 / n
    b = inputs.lens(n)
    assert b.max() > 1.1 and b.min() < -2.5
    H = ls.ls_build(n, h, kappa, b, 1e-4, leaf_side=10, precision=precision)
    f = nystrom.rhs(kappa, b, n, n, h)
    sig = torch.zeros(n, n, dtype=torch.complex128, device=DEV)
    info = ls.ls_solve(H, dev(f.reshape(n, n)), sig)[0]
    assert info["converged"] and info["resid_true"] < 2e-10
    A = nystrom.dense_operator(kappa, h, b, 10)
    assert rel(host(sig).ravel(), nystrom.solve_dense(A, f)) < 1e-9
    ls.ls_free(H)
