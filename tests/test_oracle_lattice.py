"""Pins for the oracle's corrected-quadrature weights (Sec. 2.2, Eq. (8), Fig. 1).

The weights are not printed in the paper; these tests pin the oracle's
derivation to facts outside itself:
* the closed forms of Z'(-k) against a numerical derivative of 4 zeta(s) beta(s)
  (mpmath, only where it is installed);
* the H4 theta-split constants against Gaussian-regularised lattice sums;
* the stencils of Fig. 1 (1, 5, 13, 25 points);
* the observed order 4/6/8/10 of the corrected rule on a singular integral whose
  exact value comes from adaptive quadrature with a logarithmic weight.
"""
import math

import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as sp

from oracle import kernel, lattice, nystrom


def test_stencil_sizes_fig1():
    assert [len(lattice.stencil(p)) for p in (4, 6, 8, 10)] == [1, 5, 13, 25]
    assert len(lattice.stencil(2)) == 0


def test_zeta_closed_forms_against_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    Z = lambda s: 4 * mp.zeta(s) * mp.dirichlet(s, [0, 1, 0, -1])
    ref = [float(mp.diff(Z, -k)) for k in range(4)]
    np.testing.assert_allclose(lattice.zeta_square_lattice_derivs(), ref, rtol=1e-13, atol=1e-15)


def _gauss_regularised(P, eps):
    # E(eps) = int log|u| P e^{-eps|u|^2} - sum' log|m| P(m) e^{-eps|m|^2};
    # for harmonic P (and |u|^2 times harmonic) the integral vanishes.
    R = int(40 / math.sqrt(eps)) + 2
    a = np.arange(-R, R + 1, dtype=np.float64)
    A, B = np.meshgrid(a, a)
    A, B = A.ravel(), B.ravel()
    rr = A * A + B * B
    k = rr > 0
    A, B, rr = A[k], B[k], rr[k]
    return -np.sum(0.5 * np.log(rr) * P(A, B) * np.exp(-eps * rr))


def test_h4_constants_against_gaussian_regularisation():
    h4 = lambda a, b: a ** 4 - 6 * a * a * b * b + b ** 4
    eps = np.linspace(0.04, 0.2, 14)
    targets = 0.5 * lattice.zeta_h4_derivs()
    for P, ref, tol in [(h4, targets[0], 1e-7), (lambda a, b: (a * a + b * b) * h4(a, b), targets[1], 5e-6)]:
        v = np.array([_gauss_regularised(P, e) for e in eps])
        c = np.polynomial.polynomial.polyfit(eps, v, 9)
        assert abs(c[0] - ref) < tol * max(1.0, abs(ref))


def test_moments_reproduced_and_d4_symmetric():
    C = lattice.moment_targets()
    for order, neq in [(4, 1), (6, 2), (8, 4), (10, 6)]:
        c = lattice.lattice_constants(order)
        pts = lattice.stencil(order).astype(np.float64)
        w = np.array([c[lattice.orbit_id(*p)] for p in pts.astype(int)])
        m1, m2 = pts[:, 0], pts[:, 1]
        r2 = m1 ** 2 + m2 ** 2
        h4 = m1 ** 4 - 6 * m1 ** 2 * m2 ** 2 + m2 ** 4
        basis = [np.ones_like(r2), r2, r2 ** 2, h4, r2 ** 3, r2 * h4][:neq]
        got = [np.sum(w * P) for P in basis]
        np.testing.assert_allclose(got, C[:neq], rtol=1e-12, atol=1e-13)
        # odd moments vanish by symmetry
        assert abs(np.sum(w * m1)) < 1e-13 and abs(np.sum(w * m1 * m2 ** 2)) < 1e-13


def test_weights_depend_only_on_kappa_h():
    K1 = nystrom.kernel_offsets(10.0, 0.05, 10, 3, 3) / 0.05 ** 2
    K2 = nystrom.kernel_offsets(20.0, 0.025, 10, 3, 3) / 0.025 ** 2
    np.testing.assert_allclose(K1, K2, rtol=1e-13)


def _singular_integral(kappa, target, phi, R=1.0):
    """int G(|x_t - y|) phi(y) dy by polar quadrature about the target: the
    -1/(2pi) J0 log r part with QUADPACK's r log r weight, the smooth rest
    plainly; the angular integral is a periodic trapezoidal rule."""
    th = np.linspace(0, 2 * np.pi, 256, endpoint=False)

    def Phi(r):
        return np.sum(phi(target[0] + r * np.cos(th), target[1] + r * np.sin(th))) * (2 * np.pi / 256)

    g = np.euler_gamma
    logpart = si.quad(lambda r: -sp.j0(kappa * r) * Phi(r) / (2 * np.pi), 0, R,
                      weight="alg-loga", wvar=(1, 0), limit=400, epsabs=1e-15, epsrel=1e-14)[0]

    def S(r):
        if r == 0:
            return 0.25j - (np.log(kappa / 2) + g) / (2 * np.pi)
        return kernel.green(kappa, r) + np.log(r) * sp.j0(kappa * r) / (2 * np.pi)

    re = si.quad(lambda r: (S(r) * Phi(r) * r).real, 0, R, limit=400, epsabs=1e-15, epsrel=1e-14)[0]
    im = si.quad(lambda r: (S(r) * Phi(r) * r).imag, 0, R, limit=400, epsabs=1e-15, epsrel=1e-14)[0]
    return logpart + re + 1j * im


@pytest.mark.parametrize("order,lo", [(4, 3.8), (6, 5.8), (8, 7.6), (10, 9.4)])
def test_corrected_rule_order_on_singular_integral(order, lo):
    kappa, s0 = 10.0, 0.08
    xt = np.array([0.013, -0.021])
    # non-radial about the target, so the H4 moments matter
    phi = lambda y1, y2: np.exp(-(y1 ** 2 + y2 ** 2) / (2 * s0 ** 2)) * (1 + 3 * y1 + 20 * y2 ** 2)
    I = _singular_integral(kappa, xt, phi)
    errs, hs = [], []
    for n in (28, 40, 56, 80):
        h = 1.0 / n
        M = int(np.ceil(1.0 / h)) + 2
        K = nystrom.kernel_offsets(kappa, h, order, M, M)
        a = np.arange(-M, M + 1) * h
        Y1, Y2 = np.meshgrid(a + xt[0], a + xt[1])
        errs.append(abs(np.sum(K * phi(Y1, Y2)) - I) / abs(I))
        hs.append(h)
    slope = np.log(errs[-2] / errs[-1]) / np.log(hs[-2] / hs[-1])
    assert slope > lo, (order, errs)
