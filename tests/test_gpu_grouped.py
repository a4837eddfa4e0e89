"""Grouped GEMM (gemm_grouped and the plan API) against the FP64 oracle:
uneven problems in one persistent launch, autotuned vs fixed configuration,
CUDA-graph replay vs eager (GB300 only)."""
import numpy as np
import pytest

import oracle
from paper_2305_18236_gb300 import inputs
from tests.gpu_util import tol_exact, tol_terms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2305_18236_gb300 import build

    build.build()


def make_problems(count, seed, lo=64, hi=512, dist="uniform", ragged=True, mixed=True):
    """Uneven problems: M, N, K multiples of 32 in [lo, hi] (plus a ragged
    offset on some), all transpose combinations, per-problem alpha/beta."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        M, N, K = (int(x) * 32 for x in rng.integers(lo // 32, hi // 32 + 1, size=3))
        if ragged and i % 3 == 1:
            M, N, K = M - 5, N - 11, K - 3
        tA = bool(i % 2) if mixed else False
        tB = bool((i // 2) % 2) if mixed else False
        alpha, beta = (1.5, 0.5) if mixed and i % 4 == 3 else (1.0, 0.0)
        A = inputs.make(dist, (K, M) if tA else (M, K), seed * 1000 + 3 * i, k=K)
        B = inputs.make(dist, (N, K) if tB else (K, N), seed * 1000 + 3 * i + 1, k=K)
        C0 = inputs.uniform((M, N), seed * 1000 + 3 * i + 2)
        out.append(dict(A=A, B=B, C0=C0, transA=tA, transB=tB, alpha=alpha, beta=beta, M=M, N=N,
                        K=K))
    return out


def to_device(problems):
    import torch

    dev = []
    for p in problems:
        dev.append(dict(A=torch.from_numpy(p["A"]).cuda(), B=torch.from_numpy(p["B"]).cuda(),
                        C=torch.from_numpy(p["C0"].copy()).cuda(), transA=p["transA"],
                        transB=p["transB"], alpha=p["alpha"], beta=p["beta"]))
    return dev


def check_against_oracle(problems, dev, mode, rows_per=None):
    import torch

    torch.cuda.synchronize()
    for p, d in zip(problems, dev):
        rows = None if rows_per is None else np.linspace(0, p["M"] - 1, rows_per).astype(np.int64)
        C64, D, _ = oracle.gemm(p["A"], p["B"], p["alpha"], p["beta"], p["C0"],
                                transA=p["transA"], transB=p["transB"], rows=rows)
        out = d["C"].cpu().numpy()
        out = out if rows is None else out[rows]
        assert oracle.normwise_error(out, C64, D) <= tol_exact(mode, p["K"])
        terms = 1 if mode == "bf16" else 7
        T64 = oracle.gemm_split_terms(p["A"], p["B"], terms, p["alpha"], p["beta"], p["C0"],
                                      transA=p["transA"], transB=p["transB"], rows=rows)
        assert oracle.normwise_error(out, T64, D) <= tol_terms(mode, p["K"])


@pytest.mark.parametrize("mode", ["bf16", "bf16x3"])
def test_grouped_uneven_problems(mode):
    from paper_2305_18236_gb300 import gemm as g

    probs = make_problems(24, 11)
    dev = to_device(probs)
    g.gemm_grouped(dev, mode=mode)
    check_against_oracle(probs, dev, mode)


def test_grouped_integer_bit_exact_autotuned_and_fixed():
    """Integer data: every configuration the autotuner may pick gives the
    oracle's result bit for bit; the tuned and the fixed plan agree."""
    import torch

    from paper_2305_18236_gb300 import gemm as g

    rng = np.random.default_rng(5)
    probs = []
    for i in range(16):
        M, N, K = (int(x) * 32 for x in rng.integers(2, 17, size=3))
        probs.append(dict(A=inputs.integers((M, K), 40 + i), B=inputs.integers((K, N), 80 + i),
                          C0=inputs.integers((M, N), 120 + i), transA=False, transB=False,
                          alpha=1.5, beta=0.5, M=M, N=N, K=K))
    results = []
    for autotune in (False, True):
        dev = to_device(probs)
        plan = g.GroupedPlan(dev, mode="bf16x3", autotune=autotune)
        plan.run()
        torch.cuda.synchronize()
        results.append([d["C"].cpu().numpy() for d in dev])
        cfg = plan.config()
        assert cfg["bn"] in (128, 256) and cfg["bk"] in (32, 64)
        plan.close()
    for p, a, b in zip(probs, results[0], results[1]):
        ref, _, _ = oracle.gemm(p["A"], p["B"], 1.5, 0.5, p["C0"])
        assert np.array_equal(a.astype(np.float64), ref)
        assert np.array_equal(b.astype(np.float64), ref)


@pytest.mark.parametrize("layout", ["as_stored", "k_major"])
def test_grouped_cta_pairs_integer_exact(layout):
    """The grouped launch on CTA pairs (256-row tiles, each CTA staging half
    of B, per-problem tensor maps): uneven problems with every transpose and
    ragged edges, exact on integer data, and within bounds on U[-1, 1]."""
    import torch

    from paper_2305_18236_gb300 import gemm as g

    h = g.Gemm()
    h.set_config(cta_group=2, operand_layout=layout)
    rng = np.random.default_rng(17)
    probs, dev = [], []
    for i in range(14):
        M, N, K = (int(x) for x in rng.integers(40, 700, size=3))
        tA, tB = bool(i & 1), bool(i & 2)
        A = inputs.integers((K, M) if tA else (M, K), 900 + 3 * i)
        B = inputs.integers((N, K) if tB else (K, N), 901 + 3 * i)
        C0 = inputs.integers((M, N), 902 + 3 * i)
        probs.append((A, B, C0, tA, tB))
        dev.append(dict(A=torch.from_numpy(A).cuda(), B=torch.from_numpy(B).cuda(),
                        C=torch.from_numpy(C0.copy()).cuda(), transA=tA, transB=tB, alpha=1.5,
                        beta=0.5))
    plan = g.GroupedPlan(dev, mode="bf16x3", h=h)
    assert plan.config()["cta_group"] == 2
    plan.run()
    torch.cuda.synchronize()
    for (A, B, C0, tA, tB), d in zip(probs, dev):
        ref, _, _ = oracle.gemm(A, B, 1.5, 0.5, C0, transA=tA, transB=tB)
        assert np.array_equal(d["C"].cpu().numpy().astype(np.float64), ref)
    plan.close()
    fl = make_problems(10, 23)
    dv = to_device(fl)
    plan = g.GroupedPlan(dv, mode="bf16x3", h=h)
    plan.run()
    check_against_oracle(fl, dv, "bf16x3")
    plan.close()
    h.close()


def test_grouped_default_configuration_follows_cost_model():
    """Untuned plans on a handle without tile settings take the cost model's
    first choice: CTA pairs for many large uneven problems, one CTA per
    tile when every problem is at most 128 rows tall (a 256-row pair tile
    would double the padded work); a handle that forces one CTA keeps it."""
    import torch

    from paper_2305_18236_gb300 import gemm as g

    def plan_cfg(shapes, h=None):
        dev = [dict(A=torch.zeros((M, K), device="cuda"), B=torch.zeros((K, N), device="cuda"),
                    C=torch.zeros((M, N), device="cuda")) for (M, N, K) in shapes]
        plan = g.GroupedPlan(dev, mode="bf16x3", h=h)
        cfg = plan.config()
        plan.close()
        return cfg

    rng = np.random.default_rng(31)
    large = [tuple(int(x) * 32 for x in rng.integers(24, 65, size=3)) for _ in range(200)]
    assert plan_cfg(large)["cta_group"] == 2
    short = [(int(m), 1024, 1024) for m in rng.integers(16, 129, size=200)]
    assert plan_cfg(short)["cta_group"] == 1
    h = g.Gemm()
    h.set_config(cta_group=1)
    cfg = plan_cfg(large, h)
    assert cfg["cta_group"] == 1 and cfg["bk"] == 32
    h.close()


def test_grouped_graph_replay_equals_eager():
    """A graph-captured plan replayed twice on beta = 0 problems equals an
    eager run, bit for bit; with beta != 0 each replay applies the update
    again (C <- alpha AB + beta C), as an eager run would."""
    import torch

    from paper_2305_18236_gb300 import gemm as g

    probs = make_problems(12, 21, mixed=False)
    dev_e = to_device(probs)
    dev_g = to_device(probs)
    eager = g.GroupedPlan(dev_e, mode="bf16x3")
    graph = g.GroupedPlan(dev_g, mode="bf16x3", graph=True)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        eager.run()
        graph.run()  # captures, then replays
        graph.run()  # replays again: beta = 0, same result
    stream.synchronize()
    for a, b in zip(dev_e, dev_g):
        assert torch.equal(a["C"], b["C"])
    check_against_oracle(probs, dev_g, "bf16x3")
    eager.close()
    graph.close()


def test_grouped_degenerate_problems():
    """Problems with M = 0, K = 0 or alpha = 0 mixed with ordinary ones."""
    import torch

    from paper_2305_18236_gb300 import gemm as g

    probs = make_problems(6, 31, mixed=False)
    dev = to_device(probs)
    z = dict(A=torch.zeros((0, 16), device="cuda"), B=torch.zeros((16, 8), device="cuda"),
             C=torch.zeros((0, 8), device="cuda"))
    C_k0 = torch.from_numpy(inputs.uniform((40, 24), 7)).cuda()
    k0 = dict(A=torch.zeros((40, 0), device="cuda"), B=torch.zeros((0, 24), device="cuda"),
              C=C_k0, beta=0.25)
    C_a0 = torch.from_numpy(inputs.uniform((33, 17), 8)).cuda()
    a0 = dict(A=torch.full((33, 9), float("nan"), device="cuda"),
              B=torch.full((9, 17), float("nan"), device="cuda"), C=C_a0, alpha=0.0, beta=2.0)
    ref_k0 = 0.25 * C_k0.clone()
    ref_a0 = 2.0 * C_a0.clone()
    g.gemm_grouped([z] + dev[:3] + [k0, a0] + dev[3:], mode="bf16x3")
    torch.cuda.synchronize()
    assert torch.equal(C_k0, ref_k0)
    assert torch.equal(C_a0, ref_a0)
    check_against_oracle(probs, dev, "bf16x3")


def test_grouped_bad_problem_position():
    import ctypes

    from paper_2305_18236_gb300 import _lib
    from paper_2305_18236_gb300 import gemm as g

    probs = make_problems(4, 41, mixed=False)
    dev = to_device(probs)
    arr, keep = g._problem_array(dev)
    arr[2].ldc = 1  # smaller than N
    h = g.handle()
    plan = ctypes.c_void_p()
    st = h.lib.gemm_grouped_plan_create(h.h, 2, arr, 4, 0, None, ctypes.byref(plan))
    assert st == _lib.GEMM_ERR_ARG
    assert h.last_error_arg() == 102


def test_grouped_config4_shapes_sampled():
    """512 problems with M, N, K uniform multiples of 32 in [64, 2048]
    (FP32, 3xBF16, alpha = 1, beta = 0), autotuned and graph-captured;
    eight problems checked against the oracle on sampled rows."""
    import torch

    from paper_2305_18236_gb300 import gemm as g

    rng = np.random.default_rng(0x5EED)
    shapes = [tuple(int(x) * 32 for x in rng.integers(2, 65, size=3)) for _ in range(512)]
    dev = []
    for i, (M, N, K) in enumerate(shapes):
        gen = torch.Generator(device="cuda").manual_seed(1000 + i)
        A = torch.rand((M, K), device="cuda", generator=gen) * 2 - 1
        B = torch.rand((K, N), device="cuda", generator=gen) * 2 - 1
        dev.append(dict(A=A, B=B, C=torch.empty((M, N), device="cuda")))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        plan = g.GroupedPlan(dev, mode="bf16x3", autotune=True, graph=True)
        plan.run()
    stream.synchronize()
    for i in np.linspace(0, 511, 8).astype(int):
        M, N, K = shapes[i]
        A = dev[i]["A"].cpu().numpy()
        B = dev[i]["B"].cpu().numpy()
        rows = np.linspace(0, M - 1, 6).astype(np.int64)
        C64, D, _ = oracle.gemm(A, B, rows=rows)
        out = dev[i]["C"].cpu().numpy()[rows]
        assert oracle.normwise_error(out, C64, D) <= tol_exact("bf16x3", K)
    plan.close()


def _straggler_problems(dist, seed):
    """A few long-K problems with one or a few tiles each (they would finish
    last in one persistent launch) among small ones."""
    shapes = [(128, 512, 8192), (64, 256, 4096), (256, 768, 6144), (96, 96, 64), (64, 160, 96)]
    out = []
    for i, (M, N, K) in enumerate(shapes):
        tA, tB = bool(i % 2), bool((i // 2) % 2)
        alpha, beta = (1.5, 0.5) if i % 2 else (1.0, 0.0)
        A = inputs.make(dist, (K, M) if tA else (M, K), seed + 3 * i, k=K)
        B = inputs.make(dist, (N, K) if tB else (K, N), seed + 3 * i + 1, k=K)
        C0 = inputs.integers((M, N), seed + 3 * i + 2) if dist == "integers" else \
            inputs.uniform((M, N), seed + 3 * i + 2)
        out.append(dict(A=A, B=B, C0=C0, transA=tA, transB=tB, alpha=alpha, beta=beta, M=M, N=N,
                        K=K))
    return out


@pytest.mark.parametrize("autotune", [False, True])
def test_grouped_straggler_split_k(autotune):
    """Problems whose one tile carries more K blocks than a CTA's share of the
    launch are split along K (slices in the launch, a reduce per split
    problem, alpha and beta applied once): integer data exact, float data
    within the oracle's bounds; graph replays equal eager runs."""
    import torch

    from paper_2305_18236_gb300 import gemm as g

    probs = _straggler_problems("integers", 900)
    dev = to_device(probs)
    plan = g.GroupedPlan(dev, mode="bf16x3", autotune=autotune)
    if not autotune:
        assert plan.config()["split_k"] > 1  # the cost model splits the long-K problems
    plan.run()
    torch.cuda.synchronize()
    for p, d in zip(probs, dev):
        C64, _, _ = oracle.gemm(p["A"], p["B"], p["alpha"], p["beta"], p["C0"],
                                transA=p["transA"], transB=p["transB"])
        assert np.array_equal(d["C"].cpu().numpy().astype(np.float64), C64)
    plan.close()

    fprobs = _straggler_problems("uniform", 950)
    d1, d2 = to_device(fprobs), to_device(fprobs)
    eager = g.GroupedPlan(d1, mode="bf16x3")
    graph = g.GroupedPlan(d2, mode="bf16x3", graph=True)
    stream = torch.cuda.Stream()  # graph capture needs a non-default stream
    with torch.cuda.stream(stream):
        eager.run()
        graph.run()
    stream.synchronize()
    check_against_oracle(fprobs, d1, "bf16x3")
    for a, b in zip(d1, d2):
        assert np.array_equal(a["C"].cpu().numpy().view(np.uint32),
                              b["C"].cpu().numpy().view(np.uint32))
    eager.close()
    graph.close()


def test_grouped_config4_set_has_no_straggler_split():
    """On the uneven configuration-4 style set every tile is short against a
    CTA's share of the launch: no problem is split."""
    from paper_2305_18236_gb300 import gemm as g

    probs = make_problems(64, 961, lo=64, hi=2048, ragged=False)
    plan = g.GroupedPlan(to_device(probs), mode="bf16x3")
    assert plan.config()["split_k"] == 1
    plan.close()


def test_grouped_straggler_split_off_by_handle():
    """A handle with split_k 1 keeps every problem whole: the same straggler
    set in one launch without reduces, integer data exact."""
    import torch

    from paper_2305_18236_gb300 import gemm as g

    probs = _straggler_problems("integers", 970)
    dev = to_device(probs)
    h = g.Gemm()
    h.set_config(split_k=1)
    plan = g.GroupedPlan(dev, mode="bf16x3", h=h)
    assert plan.config()["split_k"] == 1
    plan.run()
    torch.cuda.synchronize()
    for p, d in zip(probs, dev):
        C64, _, _ = oracle.gemm(p["A"], p["B"], p["alpha"], p["beta"], p["C0"],
                                transA=p["transA"], transB=p["transB"])
        assert np.array_equal(d["C"].cpu().numpy().astype(np.float64), C64)
    plan.close()
