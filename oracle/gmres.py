"""Right-preconditioned GMRES (Sec. 5), plain numpy.

Test infrastructure only (see ``oracle/__init__``).

Solves A sigma = f as A M y = f, sigma = M y, from sigma_0 = 0 without restart,
stopping when the Arnoldi residual estimate |g_{j+1}| / ||f|| <= tol or after
maxit steps (the paper stops at relative residual 1e-10 or 100 iterations,
Sec. 6.3).  Arnoldi uses classical Gram-Schmidt applied twice; the small least
squares problem is reduced with complex Givens rotations
Q = [[conj(c), conj(s)], [-s, c]], c = a/rho, s = b/rho.
Parity pin: tests compare the result with a dense LU solve.
"""
import numpy as np


def gmres(apply_A, f, apply_M=None, tol=1e-10, maxit=100):
    """Return (sigma, iterations, relative residual estimate history)."""
    f = np.asarray(f, dtype=np.complex128)
    if apply_M is None:
        apply_M = lambda v: v
    nf = np.linalg.norm(f)
    if nf == 0.0:
        return np.zeros_like(f), 0, [0.0]
    V = np.zeros((maxit + 1, f.size), dtype=np.complex128)
    H = np.zeros((maxit + 1, maxit), dtype=np.complex128)
    c = np.zeros(maxit, dtype=np.complex128)
    s = np.zeros(maxit, dtype=np.complex128)
    g = np.zeros(maxit + 1, dtype=np.complex128)
    V[0] = f / nf
    g[0] = nf
    hist = [1.0]
    k = 0
    for j in range(maxit):
        w = apply_A(apply_M(V[j]))
        for _ in range(2):  # classical Gram-Schmidt, twice
            proj = V[: j + 1].conj() @ w
            w = w - proj @ V[: j + 1]
            H[: j + 1, j] += proj
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] != 0:
            V[j + 1] = w / H[j + 1, j]
        for i in range(j):  # rotations from earlier steps
            top = np.conj(c[i]) * H[i, j] + np.conj(s[i]) * H[i + 1, j]
            bot = -s[i] * H[i, j] + c[i] * H[i + 1, j]
            H[i, j], H[i + 1, j] = top, bot
        a, b = H[j, j], H[j + 1, j]
        rho = np.sqrt(abs(a) ** 2 + abs(b) ** 2)
        c[j], s[j] = a / rho, b / rho
        H[j, j], H[j + 1, j] = rho, 0.0
        g[j + 1] = -s[j] * g[j]
        g[j] = np.conj(c[j]) * g[j]
        k = j + 1
        hist.append(abs(g[j + 1]) / nf)
        if hist[-1] <= tol:
            break
    y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
    sigma = apply_M(y @ V[:k])
    return sigma, k, hist
