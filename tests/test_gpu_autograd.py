"""Differentiable GEMM (GemmFn, torch.autograd.Function) on the GPU: the
forward and the hand-written backward (dX = dY W^T, dW = X^T dY through
gemm_backward) against the oracle's FP64 closed-form gradients of
loss = sum((X W) * G)."""
import numpy as np
import pytest

import oracle
from paper_2305_18236_gb300 import inputs
from tests.gpu_util import tol_exact

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2305_18236_gb300 import build

    build.build()


def _run(X, W, G, mode):
    import torch

    from paper_2305_18236_gb300 import gemm as g

    tX = torch.from_numpy(X).cuda().requires_grad_(True)
    tW = torch.from_numpy(W).cuda().requires_grad_(True)
    tG = torch.from_numpy(G).cuda()
    Y = g.GemmFn.apply(tX, tW, mode)
    loss = (Y * tG).sum()
    loss.backward()
    torch.cuda.synchronize()
    return Y.detach().cpu().numpy(), tX.grad.cpu().numpy(), tW.grad.cpu().numpy()


@pytest.mark.parametrize("mode", ["f32_simt", "bf16x3"])
def test_small_instance_gradients(mode):
    """X 64x48, W 48x32, G 64x32: forward and both gradients."""
    M, K, N = 64, 48, 32
    X = inputs.normal((M, K), 201, 1 / np.sqrt(K))
    W = inputs.normal((K, N), 202, 1 / np.sqrt(K))
    G = inputs.normal((M, N), 203, 1 / np.sqrt(K))
    Y, dX, dW = _run(X, W, G, mode)
    Y64, DY, _ = oracle.gemm(X, W)
    dX64, DX, _ = oracle.gemm(G, W, transB=True)
    dW64, DW, _ = oracle.gemm(X, G, transA=True)
    assert oracle.normwise_error(Y, Y64, DY) <= tol_exact(mode, K)
    assert oracle.normwise_error(dX, dX64, DX) <= tol_exact(mode, N)
    assert oracle.normwise_error(dW, dW64, DW) <= tol_exact(mode, M)


def test_chain_shape_sampled():
    """X 8192x4096, W 4096x4096, G 8192x4096, normal(0, 1/sqrt(4096)), 3xBF16:
    sampled rows of Y, dX and dW against the oracle."""
    M, K, N = 8192, 4096, 4096
    X = inputs.normal((M, K), 301, 1 / np.sqrt(4096))
    W = inputs.normal((K, N), 302, 1 / np.sqrt(4096))
    G = inputs.normal((M, N), 303, 1 / np.sqrt(4096))
    Y, dX, dW = _run(X, W, G, "bf16x3")
    rm = np.linspace(0, M - 1, 8).astype(np.int64)
    rk = np.linspace(0, K - 1, 8).astype(np.int64)
    Y64, DY, _ = oracle.gemm(X, W, rows=rm)
    dX64, DX, _ = oracle.gemm(G, W, transB=True, rows=rm)
    dW64, DW, _ = oracle.gemm(X, G, transA=True, rows=rk)
    assert oracle.normwise_error(Y[rm], Y64, DY) <= 1e-6
    assert oracle.normwise_error(dX[rm], dX64, DX) <= 1e-6
    assert oracle.normwise_error(dW[rk], dW64, DW) <= 1e-6
