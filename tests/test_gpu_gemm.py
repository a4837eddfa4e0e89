"""GPU parity: every mode of gemm() through the C ABI against the FP64
oracle, element by element, on seeded inputs (GB300 only)."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2305_18236_gb300 import inputs
from tests.gpu_util import MODES, check_mode, make_problem, run_mode, tol_exact, tol_terms

pytestmark = pytest.mark.gpu
TRANS = [(False, False), (False, True), (True, False), (True, True)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2305_18236_gb300 import build

    build.build()


@pytest.mark.parametrize("mode", MODES)
def test_golden_listing1_exact(mode):
    """The 8x5 . 5x16 tile of Listing 1 with integer data: bit-exact."""
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "listing1_8x5x16.json")))
    A = np.array(g["A"], np.float32)
    B = np.array(g["B"], np.float32)
    C0 = np.array(g["C0"], np.float32)
    C = run_mode(mode, A, B, g["alpha"], g["beta"], C0, False, False)
    assert np.array_equal(C.astype(np.float64), np.array(g["C"]))


def test_config1_simt_256():
    """Plain SGEMM C = A B, M = N = K = 256, U[-1, 1], FP32 SIMT."""
    A, B, _ = make_problem(256, 256, 256, dist="uniform", seed=0x5EED)
    check_mode("f32_simt", A, B, 1.0, 0.0, None, False, False)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("tA,tB", TRANS)
def test_transposes_ragged(mode, tA, tB):
    """All op(A)/op(B) combinations on a shape that spans several tiles in
    every dimension and ends in a ragged tail."""
    M, N, K = 300, 530, 200
    A, B, C0 = make_problem(M, N, K, tA, tB, seed=3, beta=0.5)
    check_mode(mode, A, B, 1.5, 0.5, C0, tA, tB)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("dist", ["uniform", "log_uniform"])
def test_distributions(mode, dist):
    M, N, K = 384, 512, 320
    A, B, C0 = make_problem(M, N, K, seed=5, dist=dist, beta=0.5)
    check_mode(mode, A, B, 1.5, 0.5, C0, False, False)


EDGE = [1, 7, 33, 127, 129, 255]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("M,N,K", [(m, n, k) for m in EDGE for n in (1, 129, 255) for k in (1, 33, 255)][::3])
def test_edge_sizes(mode, M, N, K):
    """Remainder handling (Section 3.1: zero-filled partial tiles, partial
    stores) around the tile sizes."""
    A, B, C0 = make_problem(M, N, K, seed=M * 7 + N * 3 + K, beta=0.5)
    check_mode(mode, A, B, 1.5, 0.5, C0, False, False)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("tA,tB", TRANS)
def test_integer_inputs_bit_exact(mode, tA, tB):
    """Integer data in [-8, 8], K <= 4096: every partial sum is an integer
    below 2**24, so any summation order is exact and the result must match
    the oracle bit for bit (BF16 holds these integers exactly, so lo = 0)."""
    M, N, K = 272, 400, 1000
    A = inputs.integers((K, M) if tA else (M, K), 11)
    B = inputs.integers((N, K) if tB else (K, N), 12)
    C0 = inputs.integers((M, N), 13)
    C = run_mode(mode, A, B, 1.5, 0.5, C0, tA, tB)
    ref, _, _ = oracle.gemm(A, B, 1.5, 0.5, C0, transA=tA, transB=tB)
    assert np.array_equal(C.astype(np.float64), ref)


@pytest.mark.parametrize("mode", MODES)
def test_identity_and_permutation(mode):
    """A I = A and P A = row permutation of A, exactly (A BF16-representable
    for the BF16 mode)."""
    X, _ = inputs.bf16_values(inputs.uniform((150, 96), 21))
    I = np.eye(96, dtype=np.float32)
    C = run_mode(mode, X, I, 1.0, 0.0, None, False, False)
    assert np.array_equal(C, X)
    perm = np.random.default_rng(3).permutation(150)
    P = np.eye(150, dtype=np.float32)[perm]
    C = run_mode(mode, P, X, 1.0, 0.0, None, False, False)
    assert np.array_equal(C, X[perm])


@pytest.mark.parametrize("mode", MODES)
def test_all_ones_closed_form(mode):
    M, N, K = 200, 300, 777
    C0 = inputs.integers((M, N), 4)
    C = run_mode(mode, np.ones((M, K), np.float32), np.ones((K, N), np.float32), 1.5, 0.5, C0,
                 False, False)
    assert np.array_equal(C.astype(np.float64), 1.5 * K + 0.5 * C0.astype(np.float64))


@pytest.mark.parametrize("mode", MODES)
def test_alpha_beta_special(mode):
    """beta == 0 with NaN in C (C never read); alpha == 0 (C = beta C);
    K == 0 (C = beta C)."""
    import torch

    from paper_2305_18236_gb300 import gemm as g

    A, B, _ = make_problem(130, 140, 150, seed=8)
    C = torch.full((130, 140), float("nan"), device="cuda")
    g.matmul(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), C=C, beta=0.0, mode=mode)
    assert torch.isfinite(C).all()
    C0 = inputs.uniform((130, 140), 9)
    Cd = torch.from_numpy(C0).cuda()
    nanA = torch.full((130, 150), float("nan"), device="cuda")
    g.matmul(nanA, torch.from_numpy(B).cuda(), C=Cd, alpha=0.0, beta=0.5, mode=mode)
    assert np.array_equal(Cd.cpu().numpy(), (np.float32(0.5) * C0))
    Cd = torch.from_numpy(C0).cuda()
    g.matmul(torch.empty((130, 0), device="cuda"), torch.empty((0, 140), device="cuda"), C=Cd,
             alpha=1.0, beta=0.25, mode=mode)
    assert np.array_equal(Cd.cpu().numpy(), (np.float32(0.25) * C0))


@pytest.mark.parametrize("mode", ["bf16", "bf16x3"])
def test_strided_ld(mode):
    """Row strides larger than the row length, unaligned for 16-byte
    vectors (ld = cols + 3), on A, B and C."""
    import torch

    from paper_2305_18236_gb300 import gemm as g

    M, N, K = 190, 210, 170
    A, B, C0 = make_problem(M, N, K, seed=31, beta=0.5)
    Ab = torch.zeros((M, K + 3)); Ab[:, :K] = torch.from_numpy(A)
    Bb = torch.zeros((K, N + 5)); Bb[:, :N] = torch.from_numpy(B)
    Cb = torch.zeros((M, N + 3)); Cb[:, :N] = torch.from_numpy(C0)
    Ab, Bb, Cb = Ab.cuda(), Bb.cuda(), Cb.cuda()
    g.matmul(Ab[:, :K], Bb[:, :N], C=Cb[:, :N], alpha=1.5, beta=0.5, mode=mode)
    torch.cuda.synchronize()
    C64, D, _ = oracle.gemm(A, B, 1.5, 0.5, C0)
    T64 = oracle.gemm_split_terms(A, B, 1 if mode == "bf16" else 7, 1.5, 0.5, C0)
    out = Cb[:, :N].cpu().numpy()
    assert oracle.normwise_error(out, T64, D) <= tol_terms(mode, K)
    assert np.all(Cb[:, N:].cpu().numpy() == 0)  # padding untouched


@pytest.mark.parametrize("split", [2, 3, 7])
@pytest.mark.parametrize("mode", ["bf16", "bf16x3"])
def test_forced_split_k_exact(mode, split):
    """Split-K (partial sums reduced in a fixed order, beta applied once --
    Algorithm 1) is exact on integer data."""
    from paper_2305_18236_gb300 import gemm as g

    h = g.Gemm()
    h.set_config(split_k=split)
    M, N, K = 200, 260, 1200
    A = inputs.integers((M, K), 41)
    B = inputs.integers((K, N), 42)
    C0 = inputs.integers((M, N), 43)
    C = run_mode(mode, A, B, 1.5, 0.5, C0, False, False, h=h)
    ref, _, _ = oracle.gemm(A, B, 1.5, 0.5, C0)
    assert np.array_equal(C.astype(np.float64), ref)
    h.close()


@pytest.mark.parametrize("bn,bk", [(128, 32), (128, 64), (256, 32), (256, 64)])
@pytest.mark.parametrize("mode", ["bf16", "bf16x3"])
def test_tile_configs(mode, bn, bk):
    """Every compiled tile shape gives the oracle's answer."""
    from paper_2305_18236_gb300 import gemm as g

    h = g.Gemm()
    h.set_config(bn=bn, bk=bk)
    A, B, C0 = make_problem(333, 600, 416, seed=51, beta=0.5)
    check_mode(mode, A, B, 1.5, 0.5, C0, False, False, h=h)
    h.close()


def test_persistent_small_grid():
    """Few persistent CTAs walking many tiles (accumulator double-buffer
    and ring phases wrap many times)."""
    from paper_2305_18236_gb300 import gemm as g

    h = g.Gemm()
    h.set_config(max_ctas=3, stages=2)
    A, B, C0 = make_problem(640, 1100, 300, seed=61, beta=0.5)
    check_mode("bf16x3", A, B, 1.5, 0.5, C0, False, False, h=h)
    h.close()


@pytest.mark.parametrize("promote_k", [-1, 64, 512])
def test_promotion_chunk_lengths(promote_k):
    """The split-precision mode with other TMEM chain lengths (including no
    promotion at all) stays within the accumulation bound of its chain."""
    from paper_2305_18236_gb300 import gemm as g

    h = g.Gemm()
    h.set_config(promote_k=promote_k)
    M, N, K = 256, 384, 1500
    A, B, C0 = make_problem(M, N, K, seed=71, beta=0.5)
    C = run_mode("bf16x3", A, B, 1.5, 0.5, C0, False, False, h=h)
    _, D, _ = oracle.gemm(A, B, 1.5, 0.5, C0)
    T64 = oracle.gemm_split_terms(A, B, 7, 1.5, 0.5, C0)
    chain = 3 * (K if promote_k < 0 else min(K, promote_k)) // 16 + 1
    bound = (chain + 2) * 2.0 ** -23 + (K // max(promote_k, 1) + 2) * 2.0 ** -24
    assert oracle.normwise_error(C, T64, D) <= bound
    h.close()


@pytest.mark.parametrize("mode,bk,split", [("bf16", 64, 1), ("bf16", 32, 1), ("bf16x3", 32, 1),
                                           ("bf16x3", 64, 1), ("bf16x3", 32, 3), ("bf16", 64, 2)])
def test_cta_pair_kernel(mode, bk, split):
    """The CTA-pair kernel (cluster of two, 256 x 256 tiles, each CTA staging
    half of B) on ragged shapes, with and without split-K."""
    from paper_2305_18236_gb300 import gemm as g

    h = g.Gemm()
    h.set_config(bn=256, bk=bk, cta_group=2, split_k=split)
    A, B, C0 = make_problem(700, 530, 1100, seed=81, beta=0.5)
    check_mode(mode, A, B, 1.5, 0.5, C0, False, False, h=h)
    Ai = inputs.integers((333, 999), 82)
    Bi = inputs.integers((999, 777), 83)
    Ci = inputs.integers((333, 777), 84)
    C = run_mode(mode, Ai, Bi, 1.5, 0.5, Ci, False, False, h=h)
    ref, _, _ = oracle.gemm(Ai, Bi, 1.5, 0.5, Ci)
    assert np.array_equal(C.astype(np.float64), ref)
    h.close()


@pytest.mark.parametrize("beta", [0.0, 0.5])
@pytest.mark.parametrize("layout", ["k_major", "as_stored"])
@pytest.mark.parametrize("tB", [False, True])
def test_wide_pair_tiles_exact(tB, layout, beta):
    """256 x 512 pair tiles (plain BF16, two MMAs per slice into two
    accumulators, one accumulator buffer): ragged M, N, K (none a multiple
    of its tile size), both B orientations and operand layouts, beta 0 (TMA
    store epilogue) and not, exact on integer data, through gemm() in BF16
    mode and through gemm_bf16; split-K partial tiles too."""
    import torch

    from paper_2305_18236_gb300 import gemm as g

    M, N, K = 600, 1096, 776  # ld % 8 == 0 (gemm_bf16 reads operands in place); ragged tiles
    A = inputs.integers((M, K), 86)
    B = inputs.integers((N, K) if tB else (K, N), 87)
    C0 = inputs.integers((M, N), 88)
    ref, _, _ = oracle.gemm(A, B, 1.5, beta, C0, transB=tB)
    for split in (1, 3):
        h = g.Gemm()
        h.set_config(bn=512, cta_group=2, operand_layout=layout, split_k=split)
        C = run_mode("bf16", A, B, 1.5, beta, C0, False, tB, h=h)
        assert np.array_equal(C.astype(np.float64), ref), split
        h.close()
    h = g.Gemm()
    h.set_config(bn=512, cta_group=2, operand_layout=layout)
    dC = torch.from_numpy(C0.copy()).cuda()
    g.matmul_bf16(torch.from_numpy(A).cuda().to(torch.bfloat16),
                  torch.from_numpy(B).cuda().to(torch.bfloat16), C=dC, alpha=1.5, beta=beta,
                  transB=tB, h=h)
    torch.cuda.synchronize()
    assert np.array_equal(dC.cpu().numpy().astype(np.float64), ref)
    h.close()


def test_wide_pair_tile_config_validation():
    """bn 512 exists only on CTA pairs with BK 64: other combinations are
    rejected at gemm_set_config (argument 2); with 3xBF16 the handle's bn 512
    runs 256-wide tiles."""
    from paper_2305_18236_gb300 import _lib
    from paper_2305_18236_gb300 import gemm as g

    h = g.Gemm()
    for bad in (dict(bn=512, cta_group=1), dict(bn=512, bk=32), dict(bn=384)):
        with pytest.raises(_lib.GemmError) as e:
            h.set_config(**bad)
        assert e.value.status == _lib.GEMM_ERR_ARG and h.last_error_arg() == 2
    h.set_config(bn=512)
    Ai = inputs.integers((300, 500), 89)
    Bi = inputs.integers((500, 700), 90)
    C = run_mode("bf16x3", Ai, Bi, 1.0, 0.0, None, False, False, h=h)
    ref, _, _ = oracle.gemm(Ai, Bi)
    assert np.array_equal(C.astype(np.float64), ref)
    h.close()


@pytest.mark.parametrize("mode,bn", [("bf16", 256), ("bf16x3", 256), ("bf16", 512)])
@pytest.mark.parametrize("layout", ["k_major", "as_stored"])
def test_cta_pair_timeout_path(layout, mode, bn):
    """The pair kernel's bounded waits expire cleanly too (one-poll limit):
    the even producer settles the stages each CTA filled, every copy lands
    before either CTA leaves, and the next call on the context is correct."""
    import torch

    from paper_2305_18236_gb300 import _lib
    from paper_2305_18236_gb300 import gemm as g

    h = g.Gemm()
    h.set_config(bn=bn, cta_group=2, wait_poll_limit=1, operand_layout=layout)
    A, B, _ = make_problem(1024, 1024, 2048, seed=85)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    C = torch.zeros((1024, 1024), device="cuda")
    g.matmul(dA, dB, C=C, mode=mode, h=h)
    assert h.sync() == _lib.GEMM_ERR_TIMEOUT
    h.set_config(bn=bn, cta_group=2, operand_layout=layout)
    g.matmul(dA, dB, C=C, mode=mode, h=h)
    assert h.sync() == _lib.GEMM_OK
    rows = np.arange(0, 1024, 101)
    C64, D, _ = oracle.gemm(A, B, rows=rows)
    assert oracle.normwise_error(C.cpu().numpy()[rows], C64, D) <= tol_exact(mode, 2048)
    h.close()


@pytest.mark.parametrize("mode", ["bf16", "bf16x3"])
@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (129, 33, 70), (300, 516, 200), (257, 1000, 64),
                                   (640, 260, 2048)])
def test_beta_zero_tma_store(mode, M, N, K):
    """beta == 0: the epilogue stores C tiles with TMA (clipped at ragged
    edges); C padding columns beyond N stay untouched."""
    import torch

    from paper_2305_18236_gb300 import gemm as g

    A = inputs.integers((M, K), 91)
    B = inputs.integers((K, N), 92)
    Cb = torch.full((M, N + 4), -7.0, device="cuda")  # ldc = N + 4 keeps 16-byte rows
    g.matmul(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), C=Cb[:, :N], alpha=1.5,
             mode=mode)
    torch.cuda.synchronize()
    ref, _, _ = oracle.gemm(A, B, 1.5, 0.0)
    out = Cb.cpu().numpy()
    assert np.array_equal(out[:, :N].astype(np.float64), ref)
    assert np.all(out[:, N:] == -7.0)


def test_beta_zero_unaligned_c_falls_back():
    """An ld that breaks 16-byte row alignment takes the ordinary store path."""
    import torch

    from paper_2305_18236_gb300 import gemm as g

    M, N, K = 200, 300, 96
    A = inputs.integers((M, K), 93)
    B = inputs.integers((K, N), 94)
    Cb = torch.zeros((M, N + 1), device="cuda")
    g.matmul(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), C=Cb[:, :N], mode="bf16x3")
    torch.cuda.synchronize()
    ref, _, _ = oracle.gemm(A, B)
    assert np.array_equal(Cb[:, :N].cpu().numpy().astype(np.float64), ref)
