"""Operand layouts of the tensor-core kernel (GB300 only).

An operand stored K x rows (A with transA, B without transB) reaches the
tensor cores MN-major: it is split without transposing (or, for BF16 input,
read in place) and staged as 64-wide row groups with a 128-byte swizzle.
The K-major layout (every operand made K-contiguous first) is the other
path.  Both must give the oracle's answer: bit for bit on integer data,
within the accumulation bound otherwise, for every compiled tile shape,
with split-K, grouped, and through the host-buffer pipeline.
"""
import numpy as np
import pytest

import oracle
from paper_2305_18236_gb300 import inputs
from tests.gpu_util import check_mode, make_problem, run_mode, tol_exact, tol_terms

pytestmark = pytest.mark.gpu
TRANS = [(False, False), (False, True), (True, False), (True, True)]
LAYOUTS = ["as_stored", "k_major"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2305_18236_gb300 import build

    build.build()


def _handle(**cfg):
    from paper_2305_18236_gb300 import gemm as g

    h = g.Gemm()
    h.set_config(**cfg)
    return h


def _integer_problem(M, N, K, tA, tB, seed):
    A = inputs.integers((K, M) if tA else (M, K), seed)
    B = inputs.integers((N, K) if tB else (K, N), seed + 1)
    C0 = inputs.integers((M, N), seed + 2)
    return A, B, C0


@pytest.mark.parametrize("tA,tB", TRANS)
@pytest.mark.parametrize("bn,bk", [(128, 32), (128, 64), (256, 32), (256, 64)])
@pytest.mark.parametrize("mode", ["bf16", "bf16x3"])
def test_as_stored_integer_bit_exact(mode, bn, bk, tA, tB):
    """Every tile shape and transpose with MN-major operands: ragged M, N
    (not multiples of 64) and K (not a multiple of BK), exact."""
    h = _handle(bn=bn, bk=bk, operand_layout="as_stored")
    M, N, K = 333, 390, 1001
    A, B, C0 = _integer_problem(M, N, K, tA, tB, 100 + bn + bk)
    C = run_mode(mode, A, B, 1.5, 0.5, C0, tA, tB, h=h)
    ref, _, _ = oracle.gemm(A, B, 1.5, 0.5, C0, transA=tA, transB=tB)
    assert np.array_equal(C.astype(np.float64), ref)
    h.close()


@pytest.mark.parametrize("tA,tB", TRANS)
@pytest.mark.parametrize("bk", [32, 64])
@pytest.mark.parametrize("mode", ["bf16", "bf16x3"])
def test_cta_pair_as_stored_integer_bit_exact(mode, bk, tA, tB):
    """The CTA-pair kernel with MN-major operands (each CTA stages 128 rows of
    A and half of B as 64-row groups), ragged in every dimension, exact."""
    h = _handle(cta_group=2, bn=256, bk=bk, operand_layout="as_stored")
    M, N, K = 600, 530, 777
    A, B, C0 = _integer_problem(M, N, K, tA, tB, 190 + bk)
    C = run_mode(mode, A, B, 1.5, 0.5, C0, tA, tB, h=h)
    ref, _, _ = oracle.gemm(A, B, 1.5, 0.5, C0, transA=tA, transB=tB)
    assert np.array_equal(C.astype(np.float64), ref)
    h.close()


@pytest.mark.parametrize("tA,tB", TRANS)
@pytest.mark.parametrize("mode", ["bf16", "bf16x3"])
def test_k_major_integer_bit_exact(mode, tA, tB):
    h = _handle(operand_layout="k_major")
    A, B, C0 = _integer_problem(270, 300, 700, tA, tB, 140)
    C = run_mode(mode, A, B, 1.5, 0.5, C0, tA, tB, h=h)
    ref, _, _ = oracle.gemm(A, B, 1.5, 0.5, C0, transA=tA, transB=tB)
    assert np.array_equal(C.astype(np.float64), ref)
    h.close()


@pytest.mark.parametrize("tA,tB", TRANS)
@pytest.mark.parametrize("mode", ["bf16", "bf16x3"])
def test_layouts_agree_on_float_data(mode, tA, tB):
    """U[-1, 1] data: each layout within the bounds against the oracle, and
    the two layouts within twice the accumulation bound of each other."""
    M, N, K = 300, 520, 900
    A, B, C0 = make_problem(M, N, K, tA, tB, seed=150, beta=0.5)
    outs = []
    for layout in LAYOUTS:
        h = _handle(operand_layout=layout)
        check_mode(mode, A, B, 1.5, 0.5, C0, tA, tB, h=h)
        outs.append(run_mode(mode, A, B, 1.5, 0.5, C0, tA, tB, h=h))
        h.close()
    _, D, _ = oracle.gemm(A, B, 1.5, 0.5, C0, transA=tA, transB=tB)
    diff = float(np.max(np.abs(outs[0].astype(np.float64) - outs[1]))) / float(np.max(D))
    assert diff <= 2 * tol_terms(mode, K)


@pytest.mark.parametrize("split", [2, 5])
@pytest.mark.parametrize("tA,tB", [(True, False), (False, False)])
def test_as_stored_split_k_exact(tA, tB, split):
    """Split-K slices of MN-major operands start at K offsets inside the
    stored rows: exact on integer data."""
    h = _handle(split_k=split, operand_layout="as_stored")
    A, B, C0 = _integer_problem(200, 260, 1200, tA, tB, 160)
    C = run_mode("bf16x3", A, B, 1.5, 0.5, C0, tA, tB, h=h)
    ref, _, _ = oracle.gemm(A, B, 1.5, 0.5, C0, transA=tA, transB=tB)
    assert np.array_equal(C.astype(np.float64), ref)
    h.close()


def test_bf16_in_place_mn_major_alignment():
    """gemm_bf16 reads a K x N B in place (MN-major): with the stored layout
    forced, ldb % 8 != 0 is GEMM_ERR_ALIGN; with the K-major layout, or the
    library's choice, the same call packs B first and succeeds with the
    oracle's answer."""
    import torch

    from paper_2305_18236_gb300 import _lib
    from paper_2305_18236_gb300 import gemm as g

    M, N, K = 96, 61, 80
    A32, _ = inputs.bf16_values(inputs.integers((M, K), 170).astype(np.float32))
    B32, _ = inputs.bf16_values(inputs.integers((K, N), 171).astype(np.float32))
    A = torch.from_numpy(A32).cuda().to(torch.bfloat16)
    Bb = torch.zeros((K, 64), dtype=torch.bfloat16, device="cuda")
    Bb[:, :N] = torch.from_numpy(B32).cuda().to(torch.bfloat16)
    Bv = Bb[:, :N]  # ldb = 64: readable in place
    Bt = torch.from_numpy(B32).cuda().to(torch.bfloat16)  # contiguous: ldb = 61
    h = _handle(operand_layout="as_stored")
    C = g.matmul_bf16(A, Bv, h=h)  # ldb = 64: in place
    torch.cuda.synchronize()
    ref, _, _ = oracle.gemm(A32, B32)
    assert np.array_equal(C.cpu().numpy().astype(np.float64), ref)
    with pytest.raises(_lib.GemmError) as e:
        g.matmul_bf16(A, Bt, h=h)
    assert e.value.status == _lib.GEMM_ERR_ALIGN
    h.close()
    for layout in ("k_major", "auto"):
        h = _handle(operand_layout=layout)
        C = g.matmul_bf16(A, Bt, h=h)
        torch.cuda.synchronize()
        assert np.array_equal(C.cpu().numpy().astype(np.float64), ref)
        assert h.last_launch_count() == 2  # pack + GEMM
        h.close()


@pytest.mark.parametrize("layout", LAYOUTS)
def test_grouped_layouts_integer_exact(layout):
    """A grouped launch whose problems mix K-major and MN-major operands
    (all four transposes) per problem: exact on integer data."""
    import torch

    from paper_2305_18236_gb300 import gemm as g

    rng = np.random.default_rng(7)
    h = _handle(operand_layout=layout)
    probs, dev = [], []
    for i in range(12):
        M, N, K = (int(x) for x in rng.integers(40, 420, size=3))
        tA, tB = bool(i & 1), bool(i & 2)
        A, B, C0 = _integer_problem(M, N, K, tA, tB, 200 + 3 * i)
        probs.append((A, B, C0, tA, tB))
        dev.append(dict(A=torch.from_numpy(A).cuda(), B=torch.from_numpy(B).cuda(),
                        C=torch.from_numpy(C0.copy()).cuda(), transA=tA, transB=tB, alpha=1.5,
                        beta=0.5))
    plan = g.GroupedPlan(dev, mode="bf16x3", h=h)
    assert plan.config()["operand_layout"] == layout
    plan.run()
    torch.cuda.synchronize()
    for (A, B, C0, tA, tB), d in zip(probs, dev):
        ref, _, _ = oracle.gemm(A, B, 1.5, 0.5, C0, transA=tA, transB=tB)
        assert np.array_equal(d["C"].cpu().numpy().astype(np.float64), ref)
    plan.close()
    h.close()


@pytest.mark.parametrize("layout", LAYOUTS)
def test_from_host_transposed_a_blocks(layout):
    """gemm_from_host with A stored K x M: each row block of op(A) is a
    column block of A, split in place into the MN-major plane."""
    import torch

    from paper_2305_18236_gb300 import gemm as g

    M, N, K = 4200, 520, 400
    A, B, C0 = make_problem(M, N, K, True, False, seed=180, beta=0.5)
    h = _handle(operand_layout=layout)
    tC = torch.from_numpy(C0.copy()).pin_memory()
    g.gemm_from_host(torch.from_numpy(A).pin_memory(), torch.from_numpy(B).pin_memory(), C=tC,
                     alpha=1.5, beta=0.5, transA=True, mode="bf16x3", h=h)
    rows = np.linspace(0, M - 1, 48).astype(np.int64)
    C64, D, _ = oracle.gemm(A, B, 1.5, 0.5, C0, transA=True, rows=rows)
    assert oracle.normwise_error(tC.numpy()[rows], C64, D) <= tol_exact("bf16x3", K)
    h.close()


def test_auto_layout_choice():
    """Library choice: split operands K-major (workspace of K-major planes);
    gemm_bf16 packs an MN-contiguous B only when the pass is cheap next to
    the GEMM: a small NN problem reads B in place (one launch), a large one
    packs it first (two launches)."""
    import torch

    from paper_2305_18236_gb300 import gemm as g

    h = _handle()
    M, N, K = 1000, 3, 200

    def r256(x):
        return (x + 255) // 256 * 256

    assert h.workspace_size("bf16x3", False, False, M, N, K) == \
        r256(2 * M * K * 2) + r256(2 * N * K * 2)
    for (m, n, k), launches in [((256, 512, 64), 1), ((8192, 8192, 8192), 2)]:
        A = torch.ones((m, k), dtype=torch.bfloat16, device="cuda")
        B = torch.ones((k, n), dtype=torch.bfloat16, device="cuda")
        C = g.matmul_bf16(A, B, h=h)
        torch.cuda.synchronize()
        assert h.last_launch_count() == launches
        assert bool((C == float(k)).all())
    h.close()


def test_workspace_size_follows_layout():
    """The workspace query sizes the packed planes of the layout in use."""
    h = _handle(operand_layout="as_stored")
    M, N, K = 1000, 3, 200  # B MN-major: K x round8(N) = 200 x 8; K-major: N x K = 3 x 200
    as_stored = h.workspace_size("bf16x3", False, False, M, N, K)
    h.set_config(operand_layout="k_major")
    k_major = h.workspace_size("bf16x3", False, False, M, N, K)
    h.close()
    a = 2 * M * K * 2  # hi + lo planes of A (M x K, K-major) in BF16

    def r256(x):
        return (x + 255) // 256 * 256

    assert as_stored == r256(a) + r256(2 * K * 8 * 2)
    assert k_major == r256(a) + r256(2 * N * K * 2)
