"""Split-K slices summed inside the GEMM kernel (the slices of a tile run as
one cluster of CTAs and add their partial tiles after a cluster barrier)
against the separate reduce launch and the FP64 oracle (GB300 only).

Both sum the slices in slice order with the same arithmetic, so they must
give the same bits; on integer data both must equal the exact product."""
import numpy as np
import pytest

import oracle
from paper_2305_18236_gb300 import inputs
from tests.gpu_util import make_problem, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2305_18236_gb300 import build

    build.build()


def _pair(**cfg):
    """A handle that sums split-K slices in the kernel and one that uses the
    reduce launch, with the same configuration otherwise."""
    from paper_2305_18236_gb300 import gemm as g

    hk = g.Gemm()
    hk.set_config(splitk_reduce="auto", **cfg)
    hl = g.Gemm()
    hl.set_config(splitk_reduce="launch", **cfg)
    return hk, hl


def _bf16_padded(x):
    """BF16 device view of x whose rows start 16 bytes apart (gemm_bf16 reads
    its operands in place)."""
    import torch

    rows, cols = x.shape
    buf = torch.zeros((rows, (cols + 7) // 8 * 8), dtype=torch.bfloat16, device="cuda")
    buf[:, :cols] = to_dev(x).to(torch.bfloat16)
    return buf[:, :cols]


def _run(h, A, B, C0, alpha, beta, tA, tB, mode):
    import torch

    from paper_2305_18236_gb300 import gemm as g

    M = A.shape[1] if tA else A.shape[0]
    N = B.shape[0] if tB else B.shape[1]
    C = to_dev(C0) if C0 is not None else torch.zeros((M, N), device="cuda")
    if mode == "bf16":
        g.matmul_bf16(_bf16_padded(A), _bf16_padded(B), C=C, alpha=alpha, beta=beta, transA=tA,
                      transB=tB, h=h)
    else:
        g.matmul(to_dev(A), to_dev(B), C=C, alpha=alpha, beta=beta, transA=tA, transB=tB,
                 mode=mode, h=h)
    assert h.sync() == 0
    return C.cpu().numpy(), h.last_launch_count()


@pytest.mark.parametrize("mode,place", [("bf16", "auto"), ("bf16x3", "prepass"),
                                        ("bf16x3", "in_kernel"), ("bf16x3", "in_kernel_b")])
@pytest.mark.parametrize("split", [2, 3, 4, 5, 8])
@pytest.mark.parametrize("M,N,K", [(200, 300, 3000), (130, 516, 2100), (77, 123, 4096)])
def test_integer_data_exact_and_equal_to_reduce_launch(mode, place, split, M, N, K):
    """Integer data (every partial sum exact): the in-kernel sum equals the
    exact product and the reduce launch bit for bit; ragged M and N (N % 4
    != 0 takes the scalar sum), one launch fewer where the slices form a
    cluster (2, 4 or 8)."""
    kw = dict(split_k=split, cta_group=1)
    if mode == "bf16x3":
        kw["split_place"] = place
    hk, hl = _pair(**kw)
    A, B, _ = make_problem(M, N, K, dist="integers", seed=60 + split)
    C0 = inputs.integers((M, N), 61)
    if mode == "bf16":  # integers in [-8, 8] are exact in BF16
        A, B = np.clip(A, -8, 8), np.clip(B, -8, 8)
    got, nk = _run(hk, A, B, C0, 1.5, 0.5, False, False, mode)
    ref, nl = _run(hl, A, B, C0, 1.5, 0.5, False, False, mode)
    # the slices the launch makes (every one non-empty): K blocks of 64
    # (plain BF16) or 32 (3xBF16, one CTA per tile), ceil(kb / split) a slice
    kb = -(-K // (64 if mode == "bf16" else 32))
    per = -(-kb // split)
    slices = -(-kb // per)
    # 2, 4 or 8 slices: no reduce launch; others keep it (same bits either way)
    assert nk == nl - (1 if slices in (2, 4, 8) else 0)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    C64, _, _ = oracle.gemm(A, B, 1.5, 0.5, C0)
    assert np.array_equal(got.astype(np.float64), C64)


@pytest.mark.parametrize("tA,tB", [(False, False), (False, True), (True, False), (True, True)])
@pytest.mark.parametrize("beta", [0.0, 0.5])
def test_float_data_equals_reduce_launch(tA, tB, beta):
    """Float data, every transpose, beta zero or not: the same bits as the
    reduce launch (the library's own split-K choice for this skinny shape)."""
    hk, hl = _pair()
    M, N, K = 128, 8192, 4096  # 32 tiles: split-K 4
    A, B, C0 = make_problem(M, N, K, tA, tB, seed=62, beta=beta)
    for mode in ("bf16x3", "bf16"):
        got, _ = _run(hk, A, B, C0 if beta else None, 1.25, beta, tA, tB, mode)
        ref, _ = _run(hl, A, B, C0 if beta else None, 1.25, beta, tA, tB, mode)
        assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_more_tile_slices_than_sms_use_the_reduce_launch():
    """Split-K 8 on 128 tiles (1024 tile slices, more than the SMs): the
    persistent kernel and the reduce launch run, with the same bits as the
    handle that asks for the launch."""
    hk, hl = _pair(split_k=8, cta_group=1)
    A, B, _ = make_problem(2048, 2048, 1024, dist="integers", seed=66)
    got, nk = _run(hk, A, B, None, 1.0, 0.0, False, False, "bf16x3")
    ref, nl = _run(hl, A, B, None, 1.0, 0.0, False, False, "bf16x3")
    assert nk == nl
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    C64, _, _ = oracle.gemm(A, B)
    assert np.array_equal(got.astype(np.float64), C64)


def test_skinny_library_path_has_no_reduce_launch():
    """(128, 8192, 8192) BF16 inputs: split-K 4 summed in the kernel, one
    launch; sampled rows against the oracle."""
    import torch

    from paper_2305_18236_gb300 import gemm as g

    M, N, K = 128, 8192, 8192
    A32, _ = inputs.bf16_values(inputs.normal((M, K), 63, 1 / np.sqrt(K)))
    B32, _ = inputs.bf16_values(inputs.normal((K, N), 64, 1 / np.sqrt(K)))
    h = g.Gemm()
    C = g.matmul_bf16(to_dev(A32).to(torch.bfloat16), to_dev(B32).to(torch.bfloat16), h=h)
    assert h.sync() == 0
    assert h.last_launch_count() == 1
    rows = np.linspace(0, M - 1, 8).astype(np.int64)
    C64, D, _ = oracle.gemm(A32, B32, rows=rows)
    # BF16 values: products exact, only FP32 accumulation rounding remains
    assert oracle.normwise_error(C.cpu().numpy()[rows], C64, D) <= 1e-6


def test_timeout_path_with_cluster_sum():
    """A one-poll wait limit makes the CTAs of each cluster abandon their
    waits; all still meet at the cluster barrier, the error reaches
    gemm_sync and the next call is correct."""
    import torch

    from paper_2305_18236_gb300 import _lib
    from paper_2305_18236_gb300 import gemm as g

    h = g.Gemm()
    h.set_config(split_k=4, cta_group=1, wait_poll_limit=1)
    A, B, _ = make_problem(256, 512, 4096, dist="integers", seed=65)
    dA, dB = to_dev(A), to_dev(B)
    C = torch.zeros((256, 512), device="cuda")
    g.matmul(dA, dB, C=C, mode="bf16x3", h=h)
    assert h.sync() == _lib.GEMM_ERR_TIMEOUT
    assert h.sync() == _lib.GEMM_OK
    h.set_config(split_k=4, cta_group=1)
    g.matmul(dA, dB, C=C, mode="bf16x3", h=h)
    assert h.sync() == _lib.GEMM_OK
    C64, _, _ = oracle.gemm(A, B)
    assert np.array_equal(C.cpu().numpy().astype(np.float64), C64)


def test_rejects_unknown_splitk_reduce():
    from paper_2305_18236_gb300 import _lib
    from paper_2305_18236_gb300 import gemm as g

    h = g.Gemm()
    with pytest.raises(_lib.GemmError) as e:
        h.set_config(splitk_reduce=2)
    assert e.value.status == _lib.GEMM_ERR_ARG
