"""Complex FP32 GEMM engines of the HBS build (merge products, Eqs. 26-27),
through the C ABI (ls_cgemm_c64), against a plain numpy complex128 matmul of
the same complex64 inputs.

Tolerances (relative Frobenius, K <= 1024 complex): FP32 SIMT accumulates 4K
rounded products per entry (2e-5); tensor-core tf32x3 accumulates three
partial products of 2K real terms each in FP32 (5e-5; 1.6e-5 seen at K = 764);
plain tf32 inputs carry a 2^-11 relative rounding each, so ~1e-3 (3e-3 allowed)."""
import numpy as np
import pytest

import paper_2007_12718_gb300 as ls
from paper_2007_12718_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = {0: 2e-5, 1: 3e-3, 2: 5e-5}


def _rand(shape, seed):
    return inputs.random_complex(shape, seed).astype(np.complex64)


@pytest.mark.parametrize("engine", [0, 1, 2])
@pytest.mark.parametrize("M,N,K,ta,tb,batch", [
    (128, 64, 16, False, False, 1), (200, 100, 50, False, True, 2), (1, 1, 1, False, False, 1),
    (130, 70, 33, True, False, 3), (300, 64, 764, False, False, 1), (64, 200, 96, True, True, 2),
    (764, 130, 40, False, False, 1)])
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
        assert np.linalg.norm(got[b] - ref) <= TOL[engine] * np.linalg.norm(ref), (engine, M, N, K, b)
