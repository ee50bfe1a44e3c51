"""Corrected Nystrom discretisation of the Lippmann-Schwinger equation.

Test infrastructure only (see ``oracle/__init__``).

Paper: Eq. (3) (the equation), Eq. (7) (punctured trapezoidal rule, order 2),
Eq. (8) (corrected rule), Eqs. (9)-(10) (the linear system (I + B G) q = f with
B = diag(kappa^2 b), f = -kappa^2 b u_inc), and Sec. 5 (the 10th-order operator
applied by FFT as a convolution).

Grid: n_x * n_y cell-centred nodes x_ij = (x0 + (i + 1/2) h, y0 + (j + 1/2) h);
vectors are stored row-major as [n_y][n_x] (x fastest) and flattened.

Functions:
* ``kernel_offsets``  -- K(m) = h^2 (G(h|m|) + tau_m), K(0) = h^2 tau_0.
* ``dense_G``         -- the N x N matrix G_p of Eq. (10) (plus higher-order
                         corrections), assembled entry by entry from K.
* ``dense_operator``  -- I + B G_p.
* ``solve_dense``     -- LU solve (scipy).
* ``matvec_fft``      -- (I + B G_p) x by zero-padded 2D FFT convolution.
* ``matvec_fft_transpose`` -- (I + B G_p)^T x = x + G_p (B x).
* ``field_at``        -- u(r) = h^2 sum_j G(|r - x_j|) sigma_j (Eq. (1)) for
                         receivers outside the domain.
* ``rhs``             -- f = -kappa^2 b u_inc for a plane wave.
Parity pins: tests/test_oracle_nystrom.py (FFT vs dense, symmetry, b = 0),
tests/test_oracle_nystrom.py (test_solve_convergence_orders: observed orders; test_disk_closed_form).
"""
import numpy as np
import scipy.linalg as sla

from . import kernel, lattice


def nodes(nx, ny, h, x0=0.0, y0=0.0):
    """Node coordinates (N, 2), row-major [ny][nx]."""
    xs = x0 + (np.arange(nx) + 0.5) * h
    ys = y0 + (np.arange(ny) + 0.5) * h
    X, Y = np.meshgrid(xs, ys)
    return np.stack([X.ravel(), Y.ravel()], axis=1)


def kernel_offsets(kappa, h, order, mx, my):
    """K(m) for m1 in [-mx, mx], m2 in [-my, my]; array [2my+1][2mx+1]."""
    a1 = np.arange(-mx, mx + 1)
    a2 = np.arange(-my, my + 1)
    M1, M2 = np.meshgrid(a1, a2)
    r = h * np.hypot(M1, M2)
    K = np.zeros(M1.shape, dtype=np.complex128)
    nz = r > 0
    K[nz] = kernel.green(kappa, r[nz])
    pts, w = lattice.correction_weights(order, kappa * h)
    for (p1, p2), wt in zip(pts, w):
        if abs(p1) <= mx and abs(p2) <= my:
            K[p2 + my, p1 + mx] += wt
    return h * h * K


def dense_G(kappa, h, nx, ny, order):
    """G_p(i, j) = K(x_j - x_i) over all node pairs (Eq. (10) plus corrections)."""
    K = kernel_offsets(kappa, h, order, nx - 1, ny - 1)
    ix = np.tile(np.arange(nx), ny)
    iy = np.repeat(np.arange(ny), nx)
    d1 = ix[None, :] - ix[:, None]
    d2 = iy[None, :] - iy[:, None]
    return K[d2 + ny - 1, d1 + nx - 1]


def dense_operator(kappa, h, b, order):
    """A = I + B G_p with B = diag(kappa^2 b) (Eq. (9)); b has shape [ny][nx]."""
    ny, nx = b.shape
    G = dense_G(kappa, h, nx, ny, order)
    A = (kappa * kappa) * b.ravel()[:, None] * G
    A[np.diag_indices_from(A)] += 1.0
    return A


def solve_dense(A, f):
    """q = A^{-1} f by LU with partial pivoting (f may hold several columns)."""
    lu = sla.lu_factor(A)
    return sla.lu_solve(lu, f)


def rhs(kappa, b, nx, ny, h, theta=0.0, x0=0.0, y0=0.0):
    """f = -kappa^2 b u_inc, u_inc = exp(i kappa (x1 cos theta + x2 sin theta))
    (Eq. (3), right-hand side of Eq. (9))."""
    x = nodes(nx, ny, h, x0, y0)
    uinc = np.exp(1j * kappa * (x[:, 0] * np.cos(theta) + x[:, 1] * np.sin(theta)))
    return -(kappa * kappa) * b.ravel() * uinc


def conv_kernel_spectrum(kappa, h, nx, ny, order):
    """FFT of K embedded in a (2ny) x (2nx) circulant (offset m at index m mod 2n)."""
    K = kernel_offsets(kappa, h, order, nx - 1, ny - 1)
    C = np.zeros((2 * ny, 2 * nx), dtype=np.complex128)
    a1 = np.arange(-(nx - 1), nx) % (2 * nx)
    a2 = np.arange(-(ny - 1), ny) % (2 * ny)
    C[np.ix_(a2, a1)] = K
    return np.fft.fft2(C)


def apply_conv(spec, x, nx, ny):
    """(K * x) restricted to the grid, via the zero-padded circulant."""
    xs = np.asarray(x).reshape(-1, ny, nx)
    P = np.zeros((xs.shape[0], 2 * ny, 2 * nx), dtype=np.complex128)
    P[:, :ny, :nx] = xs
    Y = np.fft.ifft2(np.fft.fft2(P) * spec[None])
    return Y[:, :ny, :nx].reshape(np.asarray(x).shape)


def matvec_fft(spec, kappa, b, x):
    """(I + B G_p) x by FFT (Sec. 5); x is [N] or [nrhs, N]."""
    ny, nx = b.shape
    conv = apply_conv(spec, x, nx, ny)
    return np.asarray(x) + (kappa * kappa) * b.ravel() * conv


def matvec_fft_transpose(spec, kappa, b, x):
    """(I + B G_p)^T x = x + G_p (B x) by FFT: G_p is complex symmetric
    (Eq. (10): its entries depend on |x_i - x_j| and the corrections are
    symmetric in the offset), so only the diagonal scaling moves."""
    ny, nx = b.shape
    bx = (kappa * kappa) * b.ravel() * np.asarray(x)
    return np.asarray(x) + apply_conv(spec, bx, nx, ny)


def field_at(kappa, h, nx, ny, sigma, receivers, x0=0.0, y0=0.0):
    """u(r_k) = h^2 sum_j G(|r_k - x_j|) sigma_j, Eq. (1) with the trapezoidal
    rule (spectrally accurate for compactly supported sigma, r_k outside)."""
    x = nodes(nx, ny, h, x0, y0)
    d = np.hypot(receivers[:, None, 0] - x[None, :, 0], receivers[:, None, 1] - x[None, :, 1])
    return (h * h) * (kernel.green(kappa, d) @ np.asarray(sigma).T)
