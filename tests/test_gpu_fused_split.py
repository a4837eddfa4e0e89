"""The in-kernel split (the paper's packing step moved on chip, Section 3.1:
packed tiles are produced as the micro kernel's operands are loaded) against
the FP64 oracle and against the split-pass path (GB300 only).

The tensor-core kernel reads the caller's FP32 A and B through TMA and its
converter warps split each staged tile in shared memory into the hi/lo BF16
atoms the MMA reads.  The split is the pass's own (bit for bit), so with the
same tile shape both paths must give identical bits; integer data must match
the exact product bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2305_18236_gb300 import inputs
from tests.gpu_util import TERMS, make_problem, tol_exact, tol_terms, to_dev

pytestmark = pytest.mark.gpu

TRANS = [(False, False), (False, True), (True, False), (True, True)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2305_18236_gb300 import build

    build.build()


def _handles(**extra):
    """A handle forced to the in-kernel split and one forced to the split
    pass with the same tile shape (one CTA per 128 x 256 tile, BK 32)."""
    from paper_2305_18236_gb300 import gemm as g

    extra.setdefault("split_k", 1)
    hf = g.Gemm()
    hf.set_config(split_place="in_kernel", **extra)
    hp = g.Gemm()
    hp.set_config(split_place="prepass", cta_group=1, bn=256, bk=32, operand_layout="as_stored",
                  **extra)
    return hf, hp


def padded(x):
    """Device copy of a 2-D array whose row stride is a multiple of 4 floats
    (16 bytes, as TMA needs to read it in place): a view of a wider buffer."""
    import torch

    rows, cols = x.shape
    ld = (cols + 3) // 4 * 4
    buf = torch.full((rows, ld), float("nan"), device="cuda")
    buf[:, :cols] = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    return buf[:, :cols]


def _run(h, A, B, C0, alpha, beta, tA, tB):
    import torch

    from paper_2305_18236_gb300 import gemm as g

    M = A.shape[1] if tA else A.shape[0]
    N = B.shape[0] if tB else B.shape[1]
    C = to_dev(C0) if C0 is not None else torch.zeros((M, N), device="cuda")
    g.matmul(padded(A), padded(B), C=C, alpha=alpha, beta=beta, transA=tA, transB=tB,
             mode="bf16x3", h=h)
    assert h.sync() == 0
    return C.cpu().numpy(), h.last_launch_count()


@pytest.mark.parametrize("tA,tB", TRANS)
@pytest.mark.parametrize("M,N,K", [(300, 520, 333), (128, 256, 32), (1, 7, 1), (257, 129, 1000)])
def test_integer_data_bit_exact(M, N, K, tA, tB):
    """Integer data: every partial sum is exact, so the in-kernel split must
    give the exact product bit for bit (ragged tiles in every dimension, a
    K tail shorter than one stage; stored rows padded to 16 bytes with NaN,
    which must never be read)."""
    hf, _ = _handles()
    A, B, _ = make_problem(M, N, K, tA, tB, dist="integers", seed=40)
    C0 = inputs.integers((M, N), 39)  # 1.5 A B + 0.5 C0 is then exact in FP32
    got, launches = _run(hf, A, B, C0, 1.5, 0.5, tA, tB)
    if min(M, N, K) > 1:  # (a one-row operand passes ld = its width, read by the pass)
        assert launches == 1  # no split pass
    C64, _, _ = oracle.gemm(A, B, 1.5, 0.5, C0, transA=tA, transB=tB)
    assert np.array_equal(got.astype(np.float64), C64)


@pytest.mark.parametrize("dist", ["uniform", "log_uniform"])
@pytest.mark.parametrize("tA,tB", TRANS)
def test_float_data_equals_split_pass(tA, tB, dist):
    """Float data: the in-kernel split and the split pass give the same bits
    with the same tile shape; both meet the oracle's bounds."""
    hf, hp = _handles()
    M, N, K = 700, 600, 1300
    A, B, C0 = make_problem(M, N, K, tA, tB, dist=dist, seed=41, beta=0.5)
    got, _ = _run(hf, A, B, C0, 1.5, 0.5, tA, tB)
    ref, _ = _run(hp, A, B, C0, 1.5, 0.5, tA, tB)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    C64, D, _ = oracle.gemm(A, B, 1.5, 0.5, C0, transA=tA, transB=tB)
    assert oracle.normwise_error(got, C64, D) <= tol_exact("bf16x3", K)
    T64 = oracle.gemm_split_terms(A, B, TERMS["bf16x3"], 1.5, 0.5, C0, transA=tA, transB=tB)
    assert oracle.normwise_error(got, T64, D) <= tol_terms("bf16x3", K)


def test_non_finite_operands_equal_split_pass():
    """Inf and NaN in A and B travel through the in-kernel split exactly as
    through the pass (lo = 0 where hi is not finite)."""
    hf, hp = _handles()
    A, B, C0 = make_problem(256, 256, 256, seed=42, beta=0.0)
    A[3, 7] = np.inf
    A[10, 200] = -np.inf
    B[5, 9] = np.nan
    got, _ = _run(hf, A, B, None, 1.0, 0.0, False, False)
    ref, _ = _run(hp, A, B, None, 1.0, 0.0, False, False)
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    fin = ~np.isnan(ref)
    assert np.array_equal(got[fin].view(np.uint32), ref[fin].view(np.uint32))


def test_split_k_with_in_kernel_split():
    """Split-K slices of an in-kernel-split launch, reduced in fixed order:
    integer data exact."""
    for split, want in ((3, 2), (4, 1)):  # 4 slices: summed in the kernel, a cluster per tile
        hf, _ = _handles(split_k=split)
        A, B, _ = make_problem(200, 300, 3000, dist="integers", seed=43)
        C0 = inputs.integers((200, 300), 42)
        got, launches = _run(hf, A, B, C0, 1.5, 0.5, False, False)
        assert launches == want  # the kernel (and the reduce launch for 3 slices)
        C64, _, _ = oracle.gemm(A, B, 1.5, 0.5, C0)
        assert np.array_equal(got.astype(np.float64), C64)


@pytest.mark.parametrize("place", ["in_kernel_a", "in_kernel_b"])
@pytest.mark.parametrize("tA,tB", TRANS)
def test_one_operand_split_in_kernel(place, tA, tB):
    """Only A (only B) split in the kernel, the other by the pass, in one
    launch of the same kernel: integer data exact (ragged tiles, a K tail),
    float data equal bit for bit to both operands split either way."""
    from paper_2305_18236_gb300 import gemm as g

    h1 = g.Gemm()
    h1.set_config(split_place=place, split_k=1)
    A, B, _ = make_problem(300, 520, 333, tA, tB, dist="integers", seed=48)
    C0 = inputs.integers((300, 520), 49)
    got, launches = _run(h1, A, B, C0, 1.5, 0.5, tA, tB)
    assert launches == 2  # one split launch and the kernel
    C64, _, _ = oracle.gemm(A, B, 1.5, 0.5, C0, transA=tA, transB=tB)
    assert np.array_equal(got.astype(np.float64), C64)

    hf, hp = _handles()
    A, B, C0 = make_problem(700, 600, 1300, tA, tB, dist="log_uniform", seed=50, beta=0.5)
    got, _ = _run(h1, A, B, C0, 1.5, 0.5, tA, tB)
    both, _ = _run(hf, A, B, C0, 1.5, 0.5, tA, tB)
    ref, _ = _run(hp, A, B, C0, 1.5, 0.5, tA, tB)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    assert np.array_equal(both.view(np.uint32), ref.view(np.uint32))


def test_in_kernel_split_of_the_aligned_operand_only():
    """split_place in_kernel with one operand TMA cannot read in place (row
    stride not a multiple of 4 floats): the kernel splits the other, the pass
    this one; integer data exact."""
    import torch

    from paper_2305_18236_gb300 import gemm as g

    hf, _ = _handles()
    M, N, K = 130, 152, 97  # lda = K = 97; ldb = N = 152
    A, B, C0 = make_problem(M, N, K, dist="integers", seed=51, beta=0.0)
    C = torch.zeros((M, N), device="cuda")
    g.matmul(to_dev(A), to_dev(B), C=C, mode="bf16x3", h=hf)
    assert hf.sync() == 0
    assert hf.last_launch_count() == 2  # the split of A and the kernel
    C64, _, _ = oracle.gemm(A, B)
    assert np.array_equal(C.cpu().numpy().astype(np.float64), C64)


def test_grouped_rejects_one_operand_placement():
    """Grouped plans have one placement for both operands: in_kernel_a is an
    argument error there (the handle, position 1)."""
    from paper_2305_18236_gb300 import _lib
    from paper_2305_18236_gb300 import gemm as g
    from tests.test_gpu_grouped import make_problems, to_device

    h = g.Gemm()
    h.set_config(split_place="in_kernel_a")
    dev = to_device(make_problems(2, 52))
    with pytest.raises(_lib.GemmError) as e:
        g.GroupedPlan(dev, mode="bf16x3", h=h)
    assert e.value.status == _lib.GEMM_ERR_ARG


def test_unaligned_operand_falls_back_to_the_pass():
    """An operand TMA cannot read in place (row stride not a multiple of 4
    floats) is split by the pass instead; the result is unchanged."""
    import torch

    from paper_2305_18236_gb300 import gemm as g

    hf, _ = _handles()
    M, N, K = 130, 150, 97  # lda = K = 97
    A, B, C0 = make_problem(M, N, K, dist="integers", seed=44, beta=0.0)
    C = torch.zeros((M, N), device="cuda")
    g.matmul(to_dev(A), to_dev(B), C=C, mode="bf16x3", h=hf)
    assert hf.sync() == 0
    assert hf.last_launch_count() == 2  # one split launch for both operands, the kernel
    C64, _, _ = oracle.gemm(A, B)
    assert np.array_equal(C.cpu().numpy().astype(np.float64), C64)


def test_headline_size_sampled_in_kernel_split():
    """M = N = K = 8192, alpha = 1.5, beta = 0.5 with the in-kernel split:
    16 sampled rows reach the 1e-6 normwise bar."""
    import torch

    from paper_2305_18236_gb300 import gemm as g

    hf, _ = _handles()
    n = 8192
    A, B, C0 = make_problem(n, n, n, seed=0x5EED, beta=0.5)
    C = to_dev(C0)
    g.matmul(to_dev(A), to_dev(B), C=C, alpha=1.5, beta=0.5, mode="bf16x3", h=hf)
    assert hf.sync() == 0
    rows = np.linspace(0, n - 1, 16).astype(np.int64)
    C64, D, _ = oracle.gemm(A, B, 1.5, 0.5, C0, rows=rows)
    assert oracle.normwise_error(C.cpu().numpy()[rows], C64, D) <= 1e-6
    del C
    torch.cuda.empty_cache()


def test_skinny_shape_library_choice():
    """(128, 8192, 8192) on FP32 operands: the library splits the small A
    (which every one of the 32 N tiles stages) with the pass and B (staged by
    the one row of tiles) in the kernel: no split pass over B; sampled rows
    against the oracle."""
    from paper_2305_18236_gb300 import gemm as g

    M, N, K = 128, 8192, 8192
    A32, _ = inputs.bf16_values(inputs.normal((M, K), 121, 1 / np.sqrt(K)))
    B32, _ = inputs.bf16_values(inputs.normal((K, N), 122, 1 / np.sqrt(K)))
    h = g.Gemm()
    C = g.matmul(to_dev(A32), to_dev(B32), mode="bf16x3", h=h)
    assert h.sync() == 0
    assert h.last_launch_count() == 2  # the split of A, the kernel (split-K summed in it)
    rows = np.linspace(0, M - 1, 12).astype(np.int64)
    C64, D, _ = oracle.gemm(A32, B32, rows=rows)
    assert oracle.normwise_error(C.cpu().numpy()[rows], C64, D) <= tol_exact("bf16x3", K)


def test_timeout_path_in_kernel_split():
    """A one-poll wait limit makes the fused kernel abandon its waits; the
    error reaches gemm_sync and the next call is correct."""
    import torch

    from paper_2305_18236_gb300 import _lib
    from paper_2305_18236_gb300 import gemm as g

    h = g.Gemm()
    h.set_config(split_place="in_kernel", wait_poll_limit=1)
    A, B, _ = make_problem(1024, 1024, 4096, seed=45)
    dA, dB = to_dev(A), to_dev(B)
    C = torch.zeros((1024, 1024), device="cuda")
    g.matmul(dA, dB, C=C, mode="bf16x3", h=h)
    assert h.sync() == _lib.GEMM_ERR_TIMEOUT
    assert h.sync() == _lib.GEMM_OK
    h.set_config(split_place="in_kernel")
    g.matmul(dA, dB, C=C, mode="bf16x3", h=h)
    assert h.sync() == _lib.GEMM_OK
    rows = np.arange(0, 1024, 97)
    C64, D, _ = oracle.gemm(A, B, rows=rows)
    assert oracle.normwise_error(C.cpu().numpy()[rows], C64, D) <= tol_exact("bf16x3", 4096)


@pytest.mark.parametrize("autotune", [False, True])
def test_grouped_in_kernel_split(autotune):
    """Grouped plans with the in-kernel split: integer problems exact, and
    float problems equal to the split-pass plan with the same tile shape."""
    import torch

    from paper_2305_18236_gb300 import gemm as g
    from tests.test_gpu_grouped import make_problems, to_device

    hf, hp = _handles()
    probs = make_problems(20, 46, dist="integers")
    # the in-kernel split needs 16-byte rows: keep K multiples of 4 and
    # stored widths multiples of 4 (ragged problems use the pass)
    for p in probs:
        p["ok"] = all(x % 4 == 0 for x in p["A"].shape[1:] + p["B"].shape[1:])
    probs = [p for p in probs if p["ok"]]
    for i, p in enumerate(probs):
        p["C0"] = inputs.integers((p["M"], p["N"]), 300 + i)  # exact results
    dev = to_device(probs)
    plan = g.GroupedPlan(dev, mode="bf16x3", h=hf, autotune=autotune)
    assert plan.config()["split_place"] == "in_kernel"
    plan.run()
    torch.cuda.synchronize()
    for p, d in zip(probs, dev):
        C64, _, _ = oracle.gemm(p["A"], p["B"], p["alpha"], p["beta"], p["C0"],
                                transA=p["transA"], transB=p["transB"])
        assert np.array_equal(d["C"].cpu().numpy().astype(np.float64), C64)
    plan.close()
    fprobs = [p for p in make_problems(12, 47) if all(
        x % 4 == 0 for x in p["A"].shape[1:] + p["B"].shape[1:])]
    d1, d2 = to_device(fprobs), to_device(fprobs)
    pf = g.GroupedPlan(d1, mode="bf16x3", h=hf)
    pp = g.GroupedPlan(d2, mode="bf16x3", h=hp)
    assert pp.config()["split_place"] == "prepass"
    pf.run()
    pp.run()
    torch.cuda.synchronize()
    for a, b in zip(d1, d2):
        assert np.array_equal(a["C"].cpu().numpy().view(np.uint32),
                              b["C"].cpu().numpy().view(np.uint32))
    pf.close()
    pp.close()
