"""Complex FP32 GEMM engines of the HBS build (merge products, Eqs. 26-27),
through the C ABI (ls_cgemm_c64), against a plain numpy complex128 matmul of
the same complex64 inputs.

Tolerances (relative Frobenius norm of the error of C = op(A) op(B), random
operands, u = 2^-24 the FP32 unit roundoff):
* FP32 SIMT: every entry sums 4K rounded real products; the rounding errors of
  a sum of n terms of random sign grow like sqrt(n) u (a random walk), so the
  bound is 4 u sqrt(4K) with a floor of 1e-6.
* tf32x3 and f16x3: each operand carries 22 significant bits (hi + lo), so
  each real product loses ~2^-22 relative (the dropped lo lo term and the
  rounding of lo); the three partial products of every entry accumulate 6K
  terms in the tensor cores' FP32 adders, which measure like ~4 u per addition
  in a random walk (1.1e-5 at K = 1024, 4.5e-5 at K = 4096 observed for
  tf32x3): bound 8 u sqrt(6K) + 8 * 2^-22.
* plain tf32 (one product): inputs rounded to 11 bits, ~2^-11 relative per
  operand, so 3e-3.
The f16x3 engine scales each operand by one power of two from its largest
entry: entries of 1e-7 (the size of h^2 G at 2048^2) or 1e5 lose nothing.
"""
import numpy as np
import pytest

import paper_2007_12718_gb300 as ls
from paper_2007_12718_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
U32 = 2.0 ** -24


def tol(engine, K):
    if engine == 0:
        return max(1e-6, 4 * U32 * np.sqrt(4 * K))
    if engine == 1:
        return 3e-3
    return 8 * U32 * np.sqrt(6 * K) + 8 * 2.0 ** -22


def _rand(shape, seed):
    return inputs.random_complex(shape, seed).astype(np.complex64)


@pytest.mark.parametrize("engine", [0, 1, 2, 3])
@pytest.mark.parametrize("M,N,K,ta,tb,batch", [
    (128, 64, 16, False, False, 1), (200, 100, 50, False, True, 2), (1, 1, 1, False, False, 1),
    (130, 70, 33, True, False, 3), (300, 64, 764, False, False, 1), (64, 200, 96, True, True, 2),
    (764, 130, 40, False, False, 1), (97, 50, 37, False, True, 2)])
def test_cgemm_engines(engine, M, N, K, ta, tb, batch):
    A = _rand((batch, K, M) if ta else (batch, M, K), 1)
    B = _rand((batch, N, K) if tb else (batch, K, N), 2)
    C0 = _rand((batch, M, N), 3)
    alpha, beta = 1 - 0.5j, 0.3 + 0.2j
    C = torch.from_numpy(C0.copy()).to(DEV)
    ls.ls_cgemm_c64(engine, torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV), C, ta=ta, tb=tb,
                    alpha=alpha, beta=beta)
    got = C.cpu().numpy().astype(np.complex128)
    for b in range(batch):
        opA = A[b].T if ta else A[b]
        opB = B[b].T if tb else B[b]
        ref = alpha * (opA.astype(np.complex128) @ opB.astype(np.complex128)) + beta * C0[b]
        assert np.linalg.norm(got[b] - ref) <= tol(engine, K) * np.linalg.norm(ref), (engine, M, N, K, b)


@pytest.mark.parametrize("engine", [2, 3])
@pytest.mark.parametrize("scale_a,scale_b", [(1e-7, 1.0), (1e5, 3e-6), (1.0, 1.0)])
def test_cgemm_operand_scales(engine, scale_a, scale_b):
    """Operands far from 1 (the sibling blocks are ~h^2 at 2048^2) and rows of
    different sizes: the error bound holds relative to the product."""
    M, N, K = 256, 192, 1024
    A = _rand((M, K), 4) * scale_a
    A[: M // 2] *= 1e-3  # half the rows a thousand times smaller
    B = _rand((K, N), 5) * scale_b
    C = torch.zeros(1, M, N, dtype=torch.complex64, device=DEV)
    ls.ls_cgemm_c64(engine, torch.from_numpy(A.astype(np.complex64)[None]).to(DEV),
                    torch.from_numpy(B.astype(np.complex64)[None]).to(DEV), C)
    got = C[0].cpu().numpy().astype(np.complex128)
    ref = A.astype(np.complex64).astype(np.complex128) @ B.astype(np.complex64).astype(np.complex128)
    for rows in (slice(0, M // 2), slice(M // 2, M)):
        err = np.linalg.norm(got[rows] - ref[rows]) / np.linalg.norm(ref[rows])
        assert err <= tol(engine, K), (engine, scale_a, scale_b, err)


@pytest.mark.slow
@pytest.mark.parametrize("engine", [2, 3])
def test_cgemm_large_k(engine):
    """K = 4096 (the 2048^2 root's order is ~8000): within the random-walk bound."""
    M, N, K = 256, 256, 4096
    A = _rand((M, K), 6)
    B = _rand((K, N), 7)
    C = torch.zeros(1, M, N, dtype=torch.complex64, device=DEV)
    ls.ls_cgemm_c64(engine, torch.from_numpy(A[None]).to(DEV), torch.from_numpy(B[None]).to(DEV), C)
    ref = A.astype(np.complex128) @ B.astype(np.complex128)
    got = C[0].cpu().numpy()
    assert np.linalg.norm(got - ref) <= tol(engine, K) * np.linalg.norm(ref)
