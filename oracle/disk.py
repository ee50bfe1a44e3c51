"""Closed-form scattering of a plane wave by a disk of constant potential b.

Test infrastructure only (see ``oracle/__init__``).

Paper: Eq. (3) is equivalent to the Helmholtz problem Eq. (4),
-Delta u_tot - kappa^2 (1 - b) u_tot = 0, so inside a disk with constant b the
total field solves Helmholtz with wavenumber kappa_1 = kappa sqrt(1 - b), and
outside with kappa; u_tot and its normal derivative are continuous at the
interface.  With u_inc = exp(i kappa x1) = e^{i kappa c1} sum_n i^n J_n(kappa r) e^{i n theta}
about the disk centre c, the scattered field outside is
  u(r, theta) = e^{i kappa c1} sum_n B_n H_n^(1)(kappa r) e^{i n theta},
where for each n
  A_n J_n(k1 a)        = i^n J_n(k a)        + B_n H_n(k a)
  A_n k1 J_n'(k1 a)    = i^n k J_n'(k a)     + B_n k H_n'(k a).
This is the textbook transmission problem; it pins the kernel's kind, sign and
scale through the discretised solve (discontinuous b: low observed order).
"""
import numpy as np
import scipy.special as sp


def scattered_field(kappa, bval, radius, centre, points, nmax=None):
    """Scattered field u at points outside the disk (array (P, 2))."""
    k1 = kappa * np.sqrt(1.0 - bval)
    a = radius
    if nmax is None:
        nmax = int(kappa * a + 30)
    d = points - np.asarray(centre)[None, :]
    r = np.hypot(d[:, 0], d[:, 1])
    th = np.arctan2(d[:, 1], d[:, 0])
    u = np.zeros(len(points), dtype=np.complex128)
    for n in range(-nmax, nmax + 1):
        jn_k, djn_k = sp.jv(n, kappa * a), sp.jvp(n, kappa * a)
        hn_k, dhn_k = sp.hankel1(n, kappa * a), sp.h1vp(n, kappa * a)
        jn_1, djn_1 = sp.jv(n, k1 * a), sp.jvp(n, k1 * a)
        inc = 1j ** n
        M = np.array([[jn_1, -hn_k], [k1 * djn_1, -kappa * dhn_k]], dtype=np.complex128)
        rhs = np.array([inc * jn_k, inc * kappa * djn_k], dtype=np.complex128)
        _, Bn = np.linalg.solve(M, rhs)
        u += Bn * sp.hankel1(n, kappa * r) * np.exp(1j * n * th)
    return np.exp(1j * kappa * centre[0]) * u
