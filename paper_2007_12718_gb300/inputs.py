"""Seeded synthetic inputs (scattering potentials, incident directions, receivers).

This module holds only input generation: none of the solver's arithmetic.
It is shared by the tests, the benchmark and the CPU oracle's callers.

The paper's own potentials are analytic (Sec. 6: Gaussian bump, cavity, lens);
the workloads here use the family below, with the shapes and smoothness of
those experiments:

* ``gaussian_bump``   -- b = a exp(-|x - c|^2 / s2) (the plain oracle-size case).
* ``gaussian_family`` -- b = psi(x) * sum_{g<20} a_g exp(-|x - c_g|^2 / (2 w_g^2))
  with a ~ U[-0.5, 0.5], w ~ U[0.05, 0.15], c ~ U[0.15, 0.85]^2 drawn in that
  order from numpy.random.default_rng(seed); psi is a C-infinity cutoff that
  vanishes with all derivatives on the boundary of the unit square (ramp over
  a distance 0.1).  If max b >= 0.95 the field is scaled to max 0.95
  (b <= 1 guarantees existence and uniqueness, Sec. 1).
* ``constant_disk``   -- b = value inside a disk (closed-form pin).
* ``plane_wave_angles`` / ``receivers_circle``.
"""
import numpy as np


def grid_nodes(n, h=None, x0=0.0, y0=0.0):
    """Cell-centred nodes of an n x n grid on [x0, x0+1] x [y0, y0+1]; returns
    (X, Y) arrays [n][n] (row = y index, column = x index)."""
    h = 1.0 / n if h is None else h
    c = (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(x0 + c, y0 + c)
    return X, Y


def _smooth_step(t):
    """C-infinity step: 0 for t <= 0, 1 for t >= 1."""
    t = np.clip(t, 0.0, 1.0)
    with np.errstate(divide="ignore", over="ignore"):
        a = np.where(t > 0, np.exp(-1.0 / np.where(t > 0, t, 1.0)), 0.0)
        b = np.where(t < 1, np.exp(-1.0 / np.where(t < 1, 1.0 - t, 1.0)), 0.0)
    return a / (a + b)


def cutoff(X, Y, ramp=0.1):
    return (_smooth_step(X / ramp) * _smooth_step((1 - X) / ramp)
            * _smooth_step(Y / ramp) * _smooth_step((1 - Y) / ramp))


def gaussian_bump(n, amp=0.5, s2=0.04, centre=(0.5, 0.5)):
    X, Y = grid_nodes(n)
    return amp * np.exp(-((X - centre[0]) ** 2 + (Y - centre[1]) ** 2) / s2)


def gaussian_family(n, seed, count=20):
    rng = np.random.default_rng(seed)
    a = rng.uniform(-0.5, 0.5, count)
    w = rng.uniform(0.05, 0.15, count)
    c = rng.uniform(0.15, 0.85, (count, 2))
    X, Y = grid_nodes(n)
    b = np.zeros_like(X)
    for g in range(count):
        b += a[g] * np.exp(-((X - c[g, 0]) ** 2 + (Y - c[g, 1]) ** 2) / (2 * w[g] ** 2))
    b *= cutoff(X, Y)
    mx = b.max()
    if mx >= 0.95:
        b *= 0.95 / mx
    return b


def cavity(n, centre=(0.5, 0.5)):
    """The cavity of the paper's numerical experiments (Sec. 6.2): in polar
    coordinates (r, theta) about the domain centre,
    b = (1 - sin(theta / 2)^500) exp(-2000 (0.1 - r^2)^2), in [0, 1]; a ring of
    radius ~0.32 open towards -x1 (theta = pi)."""
    X, Y = grid_nodes(n)
    dx, dy = X - centre[0], Y - centre[1]
    r2 = dx * dx + dy * dy
    th = np.arctan2(dy, dx)
    return (1.0 - np.sin(0.5 * th) ** 500) * np.exp(-2000.0 * (0.1 - r2) ** 2)


def gaussian_direct(n, centre=(0.5, 0.5)):
    """The potential of the paper's direct-solver experiments (Sec. 6.1),
    b = 1.5 exp(-160 |x|^2), x measured from the domain centre."""
    X, Y = grid_nodes(n)
    return 1.5 * np.exp(-160.0 * ((X - centre[0]) ** 2 + (Y - centre[1]) ** 2))


def lens(n, centre=(0.5, 0.5)):
    """The vertically graded lens of the paper's Sec. 6.2 test problems,
    b = 4 (x2 - 0.1) (1 - erf(25 (|x| - 0.3))), with x measured from the
    domain centre (a disk of radius ~0.3 in the middle of the unit square);
    b ranges over about [-2.69, 1.18], above the b <= 1 of the existence theorem."""
    from scipy.special import erf
    X, Y = grid_nodes(n)
    dx, dy = X - centre[0], Y - centre[1]
    return 4.0 * (dy - 0.1) * (1.0 - erf(25.0 * (np.sqrt(dx * dx + dy * dy) - 0.3)))


def constant_disk(n, value, radius, centre=(0.5, 0.5)):
    X, Y = grid_nodes(n)
    return np.where((X - centre[0]) ** 2 + (Y - centre[1]) ** 2 < radius ** 2, value, 0.0)


def plane_wave_angles(count):
    return 2 * np.pi * np.arange(count) / count


def receivers_circle(count, radius=1.5, centre=(0.5, 0.5)):
    phi = 2 * np.pi * np.arange(count) / count
    return np.stack([centre[0] + radius * np.cos(phi), centre[1] + radius * np.sin(phi)], axis=1)


def random_complex(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# Workloads (grid side, kappa, potential, tolerances) of the measured cases.
WORKLOADS = {
    "direct_n32": dict(n=32, kappa=20.0, b=lambda n: gaussian_bump(n), order_precond=10,
                       order_matvec=10, eps=1e-10, leaf=8),
    "precond_n256": dict(n=256, kappa=60.0, b=lambda n: gaussian_family(n, 0), order_precond=4,
                         order_matvec=10, eps=1e-4, leaf=8),
    "precond_n2048": dict(n=2048, kappa=400 * np.pi, b=lambda n: gaussian_family(n, 0),
                          order_precond=4, order_matvec=10, eps=1e-4, leaf=8),
    # the 2048^2 workload's regime (kappa h = 0.614, 10.24 points per wavelength) at
    # smaller sizes: the CPU oracle's bounded samples and intermediate checks
    "precond_n256_10ppw": dict(n=256, kappa=50 * np.pi, b=lambda n: gaussian_family(n, 0), order_precond=4,
                               order_matvec=10, eps=1e-4, leaf=8),
    "precond_n512_10ppw": dict(n=512, kappa=100 * np.pi, b=lambda n: gaussian_family(n, 0), order_precond=4,
                               order_matvec=10, eps=1e-4, leaf=8),
    "precond_n1024_10ppw": dict(n=1024, kappa=200 * np.pi, b=lambda n: gaussian_family(n, 0), order_precond=4,
                                order_matvec=10, eps=1e-4, leaf=8),
    # the largest grid of the family the FFT matvec takes (padded rows of 8192):
    # N = 16,777,216, 400 wavelengths across
    "precond_n4096": dict(n=4096, kappa=800 * np.pi, b=lambda n: gaussian_family(n, 0), order_precond=4,
                          order_matvec=10, eps=1e-4, leaf=8),
    # many incident fields on one factorisation: 256 plane waves, angles 2 pi j / 256
    "multirhs_n512": dict(n=512, kappa=300.0, b=lambda n: gaussian_family(n, 0), order_precond=4,
                          order_matvec=10, eps=1e-4, leaf=8, nrhs=256),
}
# The lens of Sec. 6.2 at kappa = 300 (47.7 wavelengths across) on the grids of the
# paper's lens table, 100-point leaves, eps 1e-4, order 4 / 10.
for _j in range(4):
    _n = 320 << _j
    WORKLOADS[f"lens_n{_n}"] = dict(n=_n, kappa=300.0, b=lambda n: lens(n), order_precond=4,
                                    order_matvec=10, eps=1e-4, leaf=10)
# The cavity sweep of Sec. 6.3 (preconditioned solver, 10 points per wavelength,
# 100-point leaves): n = 80 2^j, kappa = 2 pi n / 10 (the domain is n / 10
# wavelengths across; kappa = 50.27 at n = 80), eps 1e-4, order 4 / 10.
for _j in range(7):
    _n = 80 << _j
    WORKLOADS[f"cavity_n{_n}"] = dict(n=_n, kappa=2 * np.pi * _n / 10, b=lambda n: cavity(n), order_precond=4,
                                      order_matvec=10, eps=1e-4, leaf=10)


def multiproblem_set(count=32, seed=7, sides=(64, 96, 128, 192), first_b_seed=100):
    """Many independent problems of uneven sizes at 10 points per wavelength:
    side n drawn from `sides` by default_rng(seed), kappa = 2 pi n / 10 (kappa h =
    0.628 for all), potential gaussian_family(n, first_b_seed + i), leaf side 8
    where n / 8 is a power of two times 8 and 12 otherwise (96 = 12 * 8, 192 = 12 * 16).
    Returns a list of dicts (n, kappa, b_seed, leaf) in draw order."""
    rng = np.random.default_rng(seed)
    out = []
    for i, n in enumerate(rng.choice(np.array(sides), size=count)):
        n = int(n)
        leaf = 12 if n % 3 == 0 else 8
        out.append(dict(n=n, kappa=2 * np.pi * n / 10, b_seed=first_b_seed + i, leaf=leaf))
    return out
