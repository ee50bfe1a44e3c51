"""Free-space Helmholtz kernel, Eq. (2): G(x, y) = (i/4) H0^(1)(kappa |x - y|).

Test infrastructure only (see ``oracle/__init__``).

H0^(1) (outgoing) is the reading that satisfies the radiation condition the
paper relies on (Sec. 1).  Evaluated with scipy's Hankel function.
Parity pins: the constant-b disk closed form (tests/test_oracle_nystrom.py, test_disk_closed_form) fixes
the kind, sign and scale of the kernel through the scattered field.
"""
import numpy as np
import scipy.special as sp


def green(kappa, r):
    """G(r) = (i/4) H0^(1)(kappa r) for r > 0 (array or scalar)."""
    return 0.25j * sp.hankel1(0, kappa * np.asarray(r, dtype=np.float64))
