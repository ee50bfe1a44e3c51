"""Corrected-trapezoidal weights for the 2D Helmholtz kernel on a square lattice.

Test infrastructure only (see ``oracle/__init__``).

Paper: Sec. 2.2, Eq. (8) and Fig. 1.  The paper states that (i) the corrections
tau_ij live on stencils of 1, 5, 13, 25 points giving orders 4, 6, 8, 10,
(ii) they exploit the form of the kernel's singularity and the smoothness of
sigma, and (iii) they depend only on kappa*h and the order.  It does not print
the weights (they came from Duan & Rokhlin's code).  The reading used here:

  G(r) = -(1/2pi) J0(kappa r) log r + S(r),   S smooth,
  S(0) = i/4 - (1/2pi) (log(kappa/2) + gamma).

The smooth part S is integrated spectrally by the full trapezoidal rule, so
only the j = i term h^2 S(0) sigma_i must be added.  For the logarithmic part
phi(y) log|y|, phi(y) = -(1/2pi) J0(kappa|y|) sigma(x_i + y), the punctured
rule misses

  h^2 log(h) phi(0) + h^2 sum_alpha h^|alpha| d^alpha phi(0)/alpha! C_alpha,
  C_alpha = (1/2) Z'_{u^alpha}(0),   Z_P(s) = sum_{m != 0} P(m) |m|^{-2s}

(the zeta-regularised finite part of  int u^alpha log|u| - sum' m^alpha log|m|).
A D4-symmetric set of constants c_m on the L1 diamond |m1|+|m2| <= r
(r = 0..3 for orders 4..10) matching these moments for every D4-invariant
polynomial of degree <= 2r removes every term below h^(2r+4).  Hence

  tau_0 = i/4 - (1/2pi) (log(kappa h / 2) + gamma + c_0),
  tau_m = -(1/2pi) c_m J0(kappa h |m|)    (m != 0 in the stencil),

which depend on kappa*h only, as the paper states.  The D4-invariant
polynomials of degree <= 6 are spanned by 1, |u|^2, |u|^4, H4, |u|^6, |u|^2 H4
with H4 = u1^4 - 6 u1^2 u2^2 + u2^4 (harmonic), and

  Z_{|u|^2j}(s) = Z(s - j),      Z_{|u|^2j H4}(s) = Z_{H4}(s - j),
  Z(s) = 4 zeta(s) beta(s)       (sum of two squares).

Z'(0), Z'(-1), Z'(-2), Z'(-3) are taken from the closed forms of zeta and
Dirichlet beta at non-positive integers; Z_H4'(0), Z_H4'(-1) from the Mellin
split of the theta series (exponentially convergent).

Parity pins (tests/test_oracle_lattice.py; the solve orders in tests/test_oracle_nystrom.py):
closed forms vs an independent numerical derivative of 4 zeta beta; the H4
constants vs Gaussian-regularised lattice sums; the observed convergence
orders 2/4/6/8/10 of the full discretisation.  Agreement with Duan-Rokhlin's own
weights is unpinned (they are not in the paper).
"""
import math

import numpy as np
import scipy.special as sp

EULER_GAMMA = float(np.euler_gamma)

# Stencil radius per order: the L1 diamond |m1|+|m2| <= r (Fig. 1).
STENCIL_RADIUS = {4: 0, 6: 1, 8: 2, 10: 3}


def _dirichlet_beta(s):
    """beta(s) = sum_k (-1)^k (2k+1)^-s via Hurwitz zeta (s > 1)."""
    return 4.0 ** (-s) * (sp.zeta(s, 0.25) - sp.zeta(s, 0.75))


def zeta_square_lattice_derivs():
    """Z'(0), Z'(-1), Z'(-2), Z'(-3) for Z(s) = sum' |m|^{-2s} = 4 zeta(s) beta(s).

    Closed forms from the values of zeta and beta at 0, -1, -2, -3:
      Z'(0)  = log(4 pi) - 4 log Gamma(1/4)
      Z'(-1) = 4 zeta(-1) beta'(-1)   = -2 G / (3 pi)         (G = beta(2))
      Z'(-2) = 4 zeta'(-2) beta(-2)   =  zeta(3) / (2 pi^2)
      Z'(-3) = 4 zeta(-3) beta'(-3)   = -8 beta(4) / (5 pi^3)
    """
    catalan = _dirichlet_beta(2.0)
    zeta3 = float(sp.zeta(3.0))
    beta4 = _dirichlet_beta(4.0)
    return np.array([
        math.log(4.0 * math.pi) - 4.0 * math.log(sp.gamma(0.25)),
        -2.0 * catalan / (3.0 * math.pi),
        zeta3 / (2.0 * math.pi ** 2),
        -8.0 * beta4 / (5.0 * math.pi ** 3),
    ])


def _upper_gamma_int(n, x):
    """int_1^inf t^n e^{-x t} dt = Gamma(n+1, x) / x^(n+1) for integer n >= 0."""
    s = sum(x ** j / math.factorial(j) for j in range(n + 1))
    return math.factorial(n) * np.exp(-x) * s / x ** (n + 1)


def zeta_h4_derivs(rmax=9):
    """Z_H4'(0) and Z_H4'(-1) with H4(m) = m1^4 - 6 m1^2 m2^2 + m2^4.

    theta_H4(t) = sum' H4(m) exp(-pi t |m|^2) obeys theta(t) = t^-5 theta(1/t)
    (Hecke), so pi^-s Gamma(s) Z_H4(s) = int_1^inf (t^(s-1) + t^(4-s)) theta(t) dt,
    an entire function; with 1/Gamma(s) ~ (-1)^k k! (s+k) near s = -k:
      Z_H4'(0)  =        int_1^inf (t^-1 + t^4) theta(t) dt
      Z_H4'(-1) = -1/pi  int_1^inf (t^-2 + t^5) theta(t) dt
    The t-integrals of exp(-pi t |m|^2) are exponential integrals E_n and
    incomplete gamma functions; terms with |m| > rmax are below 1e-80.
    """
    a = np.arange(-rmax, rmax + 1, dtype=np.float64)
    m1, m2 = np.meshgrid(a, a)
    m1, m2 = m1.ravel(), m2.ravel()
    r2 = m1 * m1 + m2 * m2
    keep = r2 > 0
    m1, m2, r2 = m1[keep], m2[keep], r2[keep]
    h4 = m1 ** 4 - 6.0 * m1 ** 2 * m2 ** 2 + m2 ** 4
    x = math.pi * r2
    d0 = np.sum(h4 * (sp.expn(1, x) + _upper_gamma_int(4, x)))
    d1 = -np.sum(h4 * (sp.expn(2, x) + _upper_gamma_int(5, x))) / math.pi
    return np.array([d0, d1])


def moment_targets():
    """C_P = (1/2) Z_P'(0) for P in (1, |u|^2, |u|^4, H4, |u|^6, |u|^2 H4)."""
    z = zeta_square_lattice_derivs()
    zh = zeta_h4_derivs()
    return 0.5 * np.array([z[0], z[1], z[2], zh[0], z[3], zh[1]])


def _basis(m1, m2):
    r2 = m1 * m1 + m2 * m2
    h4 = m1 ** 4 - 6.0 * m1 ** 2 * m2 ** 2 + m2 ** 4
    return np.array([np.ones_like(r2), r2, r2 ** 2, h4, r2 ** 3, r2 * h4])


def stencil(order):
    """Offsets m of the order-p stencil (Fig. 1): the diamond |m1|+|m2| <= r."""
    if order == 2:
        return np.zeros((0, 2), dtype=np.int64)
    r = STENCIL_RADIUS[order]
    pts = [(i, j) for j in range(-r, r + 1) for i in range(-r, r + 1)
           if abs(i) + abs(j) <= r]
    return np.array(pts, dtype=np.int64)


def orbit_id(m1, m2):
    """D4 orbit key of an offset: the sorted pair (min|m|, max|m|)."""
    a, b = abs(int(m1)), abs(int(m2))
    return (min(a, b), max(a, b))


def lattice_constants(order):
    """Universal constants c_m on the order-p stencil (dict orbit -> c).

    Solves sum_{m in stencil} c_m P(m) = C_P for the D4-invariant basis
    polynomials of degree <= 2r (1, 2, 4, 6 equations for r = 0..3).
    """
    if order == 2:
        return {}
    pts = stencil(order)
    orbits = sorted({orbit_id(*p) for p in pts})
    neq = {4: 1, 6: 2, 8: 4, 10: 6}[order]
    A = np.zeros((neq, len(orbits)))
    for col, ob in enumerate(orbits):
        members = np.array([p for p in pts if orbit_id(*p) == ob], dtype=np.float64)
        A[:, col] = _basis(members[:, 0], members[:, 1])[:neq].sum(axis=1)
    c = np.linalg.solve(A, moment_targets()[:neq])
    return dict(zip(orbits, c))


def correction_weights(order, kh):
    """tau_m for every m in the order-p stencil, as an (npts, 2) offset array and
    a complex weight array.  The matrix entry for offset m is
    h^2 (G(h|m|) + tau_m) for m != 0 and h^2 tau_0 on the diagonal (Eq. (10))."""
    pts = stencil(order)
    if order == 2:
        return pts, np.zeros(0, dtype=np.complex128)
    c = lattice_constants(order)
    w = np.empty(len(pts), dtype=np.complex128)
    for i, (a, b) in enumerate(pts):
        cm = c[orbit_id(a, b)]
        if a == 0 and b == 0:
            w[i] = 0.25j - (math.log(kh / 2.0) + EULER_GAMMA + cm) / (2.0 * math.pi)
        else:
            w[i] = -cm * sp.j0(kh * math.hypot(a, b)) / (2.0 * math.pi)
    return pts, w
