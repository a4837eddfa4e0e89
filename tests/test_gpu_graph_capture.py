"""gemm() and gemm_bf16 captured in a CUDA graph and replayed on new data
(GB300 only): the split launch, the GEMM launched as its programmatic
dependent, split-K slices summed in clusters, and the in-kernel split all
replay exactly (integer data, so the exact product is the only right
answer)."""
import numpy as np
import pytest

import oracle
from paper_2305_18236_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2305_18236_gb300 import build

    build.build()


@pytest.mark.parametrize("mode,M,N,K", [
    ("bf16x3", 1024, 1024, 1024),   # both splits in one launch, split-K 4 in clusters
    ("bf16x3", 128, 8192, 2048),    # A split by the pass, B in the kernel, split-K
    ("bf16x3", 2048, 2048, 512),    # split launch, then the GEMM (no split-K)
    ("bf16", 1024, 768, 4096),      # plain BF16 on FP32 inputs
])
def test_captured_gemm_replays_exactly(mode, M, N, K):
    import torch

    from paper_2305_18236_gb300 import gemm as g

    h = g.Gemm()
    dA = torch.zeros((M, K), device="cuda")
    dB = torch.zeros((K, N), device="cuda")
    dC = torch.zeros((M, N), device="cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        g.matmul(dA, dB, C=dC, alpha=1.5, beta=0.5, mode=mode, h=h)  # workspace before capture
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        g.matmul(dA, dB, C=dC, alpha=1.5, beta=0.5, mode=mode, h=h)
    for seed in (80, 81):
        A = inputs.integers((M, K), seed)
        B = inputs.integers((K, N), seed + 10)
        C0 = inputs.integers((M, N), seed + 20)
        dA.copy_(torch.from_numpy(A))
        dB.copy_(torch.from_numpy(B))
        dC.copy_(torch.from_numpy(C0))
        graph.replay()
        torch.cuda.synchronize()
        assert h.sync() == 0
        C64, _, _ = oracle.gemm(A, B, 1.5, 0.5, C0)
        assert np.array_equal(dC.cpu().numpy().astype(np.float64), C64)


def test_captured_gemm_bf16_replays_exactly():
    import torch

    from paper_2305_18236_gb300 import gemm as g

    M, N, K = 128, 8192, 4096  # B read in place, split-K summed in clusters
    h = g.Gemm()
    dA = torch.zeros((M, K), device="cuda", dtype=torch.bfloat16)
    dB = torch.zeros((K, N), device="cuda", dtype=torch.bfloat16)
    dC = torch.zeros((M, N), device="cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        g.matmul_bf16(dA, dB, C=dC, h=h)
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        g.matmul_bf16(dA, dB, C=dC, h=h)
    A = inputs.integers((M, K), 90)
    B = inputs.integers((K, N), 91)
    dA.copy_(torch.from_numpy(A).to(torch.bfloat16))
    dB.copy_(torch.from_numpy(B).to(torch.bfloat16))
    graph.replay()
    torch.cuda.synchronize()
    assert h.sync() == 0
    C64, _, _ = oracle.gemm(A, B)
    assert np.array_equal(dC.cpu().numpy().astype(np.float64), C64)
