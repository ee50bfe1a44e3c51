"""Receiver misfit and its gradient with respect to b (dense, FP64).

Test infrastructure only (see ``oracle/__init__``).

The paper solves the forward problem only; the misfit and its gradient are
built on its discretisation (Eqs. (1), (3), (9)-(10)):

* For each incident direction theta_d: sigma_d solves (I + B G_p) sigma_d = f_d
  with B = diag(kappa^2 b), f_d = -kappa^2 b u_inc,d (Eq. (9)).
* Receiver data u_d(r_k) = h^2 sum_j G(|r_k - x_j|) sigma_d,j (Eq. (1) with the
  trapezoidal rule; receivers outside the domain), i.e. u_d = R sigma_d.
* Misfit  J(b) = sum_d sum_k |u_d(r_k) - d_dk|^2.

Gradient (real b, complex fields).  Differentiating the system gives
A d(sigma) = -kappa^2 db .* (G_p sigma + u_inc) (both B and f depend on b), so
with r_d = u_d - d_d and the adjoint state lambda_d solving
A^T lambda_d = R^T conj(r_d):

    dJ/db_j = -2 kappa^2 sum_d Re(lambda_d,j (G_p sigma_d + u_inc,d)_j).

A^T uses the plain transpose (G_p is complex symmetric).  Pins
(tests/test_oracle_adjoint.py): central finite differences of ``misfit``
along random directions, and a zero gradient when the data are the
receiver field of b itself.
"""
import numpy as np

from . import kernel, nystrom


def plane_wave(kappa, nx, ny, h, theta, x0=0.0, y0=0.0):
    """u_inc = exp(i kappa (x1 cos theta + x2 sin theta)) at the grid nodes."""
    x = nystrom.nodes(nx, ny, h, x0, y0)
    return np.exp(1j * kappa * (x[:, 0] * np.cos(theta) + x[:, 1] * np.sin(theta)))


def receiver_matrix(kappa, h, nx, ny, receivers, x0=0.0, y0=0.0):
    """R[k, j] = h^2 G(|r_k - x_j|), the trapezoidal rule of Eq. (1)."""
    x = nystrom.nodes(nx, ny, h, x0, y0)
    d = np.hypot(receivers[:, None, 0] - x[None, :, 0], receivers[:, None, 1] - x[None, :, 1])
    return (h * h) * kernel.green(kappa, d)


def forward(kappa, h, b, order, thetas, receivers):
    """Densities sigma [ndir][N] and receiver data u [ndir][nr] for each theta."""
    ny, nx = b.shape
    A = nystrom.dense_operator(kappa, h, b, order)
    F = np.stack([nystrom.rhs(kappa, b, nx, ny, h, th) for th in thetas], axis=1)
    sigma = nystrom.solve_dense(A, F).T
    R = receiver_matrix(kappa, h, nx, ny, receivers)
    return sigma, sigma @ R.T


def misfit(kappa, h, b, order, thetas, receivers, data):
    """J(b) = sum over directions and receivers of |u - data|^2."""
    _, u = forward(kappa, h, b, order, thetas, receivers)
    return float(np.sum(np.abs(u - data) ** 2))


def misfit_gradient(kappa, h, b, order, thetas, receivers, data):
    """(J, dJ/db) by the adjoint method; dJ/db has the shape of b."""
    ny, nx = b.shape
    A = nystrom.dense_operator(kappa, h, b, order)
    G = nystrom.dense_G(kappa, h, nx, ny, order)
    R = receiver_matrix(kappa, h, nx, ny, receivers)
    F = np.stack([nystrom.rhs(kappa, b, nx, ny, h, th) for th in thetas], axis=1)
    sigma = nystrom.solve_dense(A, F)              # N x ndir
    r = (R @ sigma).T - data                       # ndir x nr
    lam = nystrom.solve_dense(A.T, R.T @ np.conj(r).T)   # N x ndir
    grad = np.zeros(nx * ny)
    for d, th in enumerate(thetas):
        v = G @ sigma[:, d] + plane_wave(kappa, nx, ny, h, th)
        grad += -2.0 * kappa * kappa * np.real(lam[:, d] * v)
    return float(np.sum(np.abs(r) ** 2)), grad.reshape(ny, nx)
