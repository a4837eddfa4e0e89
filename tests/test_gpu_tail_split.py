"""Tail split of CTA-pair launches (GB300 only): when the output tiles leave
a last wave with at most half the CTA pairs busy, those tiles are computed
in two K halves on twice as many pairs, each half's raw partial tile goes
to workspace, and a reduce launch adds the halves into C.  Algorithm 1's
result is unchanged (only the order of each such tile's FP32 accumulation
differs): integer data must match the exact product bit for bit, float data
the oracle's bounds."""
import numpy as np
import pytest

import oracle
from paper_2305_18236_gb300 import inputs
from tests.gpu_util import check_mode, make_problem, run_mode, to_dev

pytestmark = pytest.mark.gpu

# forced CTA pairs, 10 of them: 12 x 7 = 84 pair tiles of 256 x 256 leave a
# last wave of 4 tiles (tile rows 8-11 of the last tile column), split into 8
# half-tile units.  The split is taken when products x K >= 3 x 4096.
CFG = dict(cta_group=2, max_ctas=20)
M, N, K = 12 * 256 - 40, 7 * 256 - 20, 12288 + 40  # ragged rows, columns and K
# sampled rows: some in the tail tiles (rows 2048 ..), some not
ROWS = np.array([0, 700, 2047, 2048, 2300, 2600, 2900, M - 1])


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2305_18236_gb300 import build

    build.build()


def _handle(**cfg):
    from paper_2305_18236_gb300 import gemm as g

    h = g.Gemm()
    h.set_config(**cfg)
    return h


@pytest.mark.parametrize("mode", ["bf16x3", "bf16"])
@pytest.mark.parametrize("tA,tB", [(False, False), (True, True)])
def test_integer_data_exact(mode, tA, tB):
    A, B, _ = make_problem(M, N, K, tA, tB, dist="integers", seed=90)
    C0 = inputs.integers((M, N), 91)
    h = _handle(**CFG)
    got = run_mode(mode, A, B, 1.5, 0.5, C0, tA, tB, h=h)
    # the operand split pass, the pair kernel and the tail reduce
    assert h.last_launch_count() == 3
    ref, _, _ = oracle.gemm(A, B, 1.5, 0.5, C0, transA=tA, transB=tB, rows=ROWS)
    assert np.array_equal(got[ROWS].astype(np.float64), ref)
    h.close()


def test_no_tail_split_when_the_last_wave_is_more_than_half_full():
    """12 pairs: 84 tiles leave a last wave of 12 tiles, all pairs busy."""
    A, B, _ = make_problem(M, N, K, dist="integers", seed=92)
    h = _handle(cta_group=2, max_ctas=24)
    got = run_mode("bf16x3", A, B, 1.0, 0.0, None, False, False, h=h)
    assert h.last_launch_count() == 2
    ref, _, _ = oracle.gemm(A, B, rows=ROWS)
    assert np.array_equal(got[ROWS].astype(np.float64), ref)
    h.close()


def test_no_tail_split_for_short_k():
    """3xBF16 at K = 2048: half a tile's K loop is worth less than the reduce
    launch, so the last wave runs whole."""
    A, B, _ = make_problem(M, N, 2048, dist="integers", seed=98)
    h = _handle(**CFG)
    got = run_mode("bf16x3", A, B, 1.0, 0.0, None, False, False, h=h)
    assert h.last_launch_count() == 2
    ref, _, _ = oracle.gemm(A, B, rows=ROWS)
    assert np.array_equal(got[ROWS].astype(np.float64), ref)
    h.close()


@pytest.mark.parametrize("dist", ["uniform", "log_uniform"])
def test_float_data_within_bounds(dist):
    A, B, C0 = make_problem(M, N, K, dist=dist, seed=93, beta=0.5)
    h = _handle(**CFG)
    check_mode("bf16x3", A, B, 1.5, 0.5, C0, False, False, rows=ROWS, h=h)
    h.close()


def test_beta_zero_ignores_nan_c():
    """beta = 0: TMA-stored C tiles outside the tail and the reduce launch's
    tail tiles both leave NaN in C unread."""
    import torch

    from paper_2305_18236_gb300 import gemm as g

    A, B, _ = make_problem(M, N, K, dist="integers", seed=94)
    h = _handle(**CFG)
    C = torch.full((M, N), float("nan"), device="cuda")
    g.matmul(to_dev(A), to_dev(B), C=C, alpha=2.0, beta=0.0, mode="bf16x3", h=h)
    torch.cuda.synchronize()
    assert h.last_launch_count() == 3
    ref, _, _ = oracle.gemm(A, B, 2.0, 0.0, rows=ROWS)
    assert np.array_equal(C.cpu().numpy()[ROWS].astype(np.float64), ref)
    assert not torch.isnan(C).any()
    h.close()


def test_workspace_covers_the_halves():
    """gemm_workspace_size counts the four tail tiles' two halves (256 x 256
    FP32 each) besides the split planes."""
    h = _handle(**CFG)
    plain = _handle(cta_group=2, max_ctas=24)
    extra = h.workspace_size("bf16x3", False, False, M, N, K) - \
        plain.workspace_size("bf16x3", False, False, M, N, K)
    assert extra >= 4 * 2 * 256 * 256 * 4
    h.close()
    plain.close()


def test_library_plan_at_8192_has_the_tail_split():
    """The library's own plan for the 8192^3 3xBF16 GEMM: 1024 pair tiles on
    (SMs / 2) pairs; a last wave at most half full is split, one more launch.
    Sampled rows against the oracle (the tail tiles' rows among them)."""
    import torch

    from paper_2305_18236_gb300 import gemm as g

    n = 8192
    pairs = torch.cuda.get_device_properties(0).multi_processor_count // 2
    tail = 1024 % pairs
    split = 0 < tail and 2 * tail <= pairs
    A = inputs.uniform((n, n), 95)
    B = inputs.uniform((n, n), 96)
    h = g.Gemm()
    C = g.matmul(to_dev(A), to_dev(B), mode="bf16x3", h=h)
    torch.cuda.synchronize()
    assert h.last_launch_count() == (3 if split else 2)
    rows = np.array([0, 4095, 6000, 7937, 8191])  # the last raster group holds the tail
    C64, D, _ = oracle.gemm(A, B, rows=rows)
    got = C.cpu().numpy()[rows]
    assert oracle.normwise_error(got, C64, D) <= 1e-6
    h.close()


def test_graph_replay_equals_eager():
    import torch

    from paper_2305_18236_gb300 import gemm as g

    A, B, C0 = make_problem(M, N, K, dist="uniform", seed=97, beta=0.5)
    h = _handle(**CFG)
    dA, dB = to_dev(A), to_dev(B)
    eager = to_dev(C0)
    g.matmul(dA, dB, C=eager, alpha=1.5, beta=0.5, mode="bf16x3", h=h)
    torch.cuda.synchronize()
    C = to_dev(C0)
    h.ensure_workspace(h.workspace_size("bf16x3", False, False, M, N, K))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s):
            g.matmul(dA, dB, C=C, alpha=1.5, beta=0.5, mode="bf16x3", h=h)
    C.copy_(to_dev(C0))
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(C, eager)
    h.close()


def test_wide_tiles_bf16_inputs_exact():
    """gemm_bf16 on 256 x 512 pair tiles (beta 0: TMA-stored C outside the
    tail): 12 x 7 = 84 tiles on 10 pairs, the last wave's 4 tiles split;
    integer data exact on sampled rows, NaN in C never read."""
    import torch

    from paper_2305_18236_gb300 import gemm as g

    Mw, Nw, Kw = 12 * 256 - 40, 7 * 512 - 24, 12288 + 64  # B rows 16-byte multiples
    A = inputs.integers((Mw, Kw), 99)
    B = inputs.integers((Kw, Nw), 100)
    h = _handle(cta_group=2, bn=512, max_ctas=20, operand_layout="as_stored")
    dA = torch.from_numpy(A).cuda().to(torch.bfloat16)
    dB = torch.from_numpy(B).cuda().to(torch.bfloat16)
    C = torch.full((Mw, Nw), float("nan"), device="cuda")
    g.matmul_bf16(dA, dB, C=C, alpha=1.5, beta=0.0, h=h)
    torch.cuda.synchronize()
    assert h.last_launch_count() == 2  # the pair kernel (B read in place) and the tail reduce
    rows = np.array([0, 2047, 2048, 2500, 3000, Mw - 1])
    ref, _, _ = oracle.gemm(A, B, 1.5, 0.0, rows=rows)
    assert np.array_equal(C.cpu().numpy()[rows].astype(np.float64), ref)
    assert not torch.isnan(C).any()
    h.close()
