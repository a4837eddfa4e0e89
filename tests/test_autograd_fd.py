"""The gradient formulas the backward pass implements, pinned on the CPU
against FP64 central finite differences of the oracle's forward GEMM.

loss(X, W) = sum(Y * G) with Y = X W.  The loss is linear in X and in W,
so dL/dX = G W^T and dL/dW = X^T G exactly, and central differences agree
with them up to FP64 rounding.  Instance: X 64x48, W 48x32, G 64x32
(M = 64, K = 48, N = 32), entries normal(0, 1/sqrt(48))."""
import numpy as np

import oracle
from paper_2305_18236_gb300 import inputs

M, K, N = 64, 48, 32


def _loss(X, W, G):
    Y, _, _ = oracle.gemm(X, W)
    return float(np.sum(Y * G.astype(np.float64)))


def test_gradient_closed_forms_match_finite_differences():
    X = inputs.normal((M, K), 201, 1 / np.sqrt(K))
    W = inputs.normal((K, N), 202, 1 / np.sqrt(K))
    G = inputs.normal((M, N), 203, 1 / np.sqrt(K))
    dX, _, _ = oracle.gemm(G, W, transB=True)   # G W^T
    dW, _, _ = oracle.gemm(X, G, transA=True)   # X^T G
    h = 2.0 ** -8  # exact in FP32, so X +- h e_ij is representable without rounding
    rng = np.random.default_rng(7)
    for (i, j) in zip(rng.integers(0, M, 40), rng.integers(0, K, 40)):
        Xp, Xm = X.copy(), X.copy()
        Xp[i, j] += np.float32(h)
        Xm[i, j] -= np.float32(h)
        step = float(Xp[i, j]) - float(Xm[i, j])
        fd = (_loss(Xp, W, G) - _loss(Xm, W, G)) / step
        assert abs(fd - dX[i, j]) <= 1e-10 * (1 + abs(dX[i, j]))
    for (i, j) in zip(rng.integers(0, K, 40), rng.integers(0, N, 40)):
        Wp, Wm = W.copy(), W.copy()
        Wp[i, j] += np.float32(h)
        Wm[i, j] -= np.float32(h)
        step = float(Wp[i, j]) - float(Wm[i, j])
        fd = (_loss(X, Wp, G) - _loss(X, Wm, G)) / step
        assert abs(fd - dW[i, j]) <= 1e-10 * (1 + abs(dW[i, j]))
