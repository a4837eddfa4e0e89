"""Seeded randomized parity sweep (GB300 only): random modes, transposes,
ragged sizes, alpha/beta and launch configurations through gemm() and
gemm_bf16(), on integer data, where every partial sum is exact and the
oracle's result is the only correct one."""
import numpy as np
import pytest

import oracle
from paper_2305_18236_gb300 import inputs

pytestmark = pytest.mark.gpu

CONFIGS = [
    {},
    {"cta_group": 2},
    {"cta_group": 1, "bn": 128},
    {"cta_group": 1, "bk": 64},
    {"cta_group": 1, "bk": 32, "stages": 2},
    {"split_k": 3},
    {"operand_layout": "as_stored"},
    {"operand_layout": "k_major", "cta_group": 2},
    {"operand_layout": "as_stored", "cta_group": 2, "bk": 32},
    {"raster_group": 1, "max_ctas": 5},
    {"cta_group": 2, "bn": 512},
]
ALPHAS = [1.0, 1.5, -0.5, 0.0]
BETAS = [0.0, 1.0, 0.5]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2305_18236_gb300 import build

    build.build()


def _size(rng):
    # log-uniform in [1, 700], so tiny and multi-tile sizes both appear
    return int(np.exp(rng.uniform(0.0, np.log(700.0))))


@pytest.mark.parametrize("case", range(48))
def test_random_gemm_exact(case):
    import torch

    from paper_2305_18236_gb300 import gemm as g

    rng = np.random.default_rng(1000 + case)
    mode = ["f32_simt", "bf16", "bf16x3"][case % 3]
    tA, tB = bool(rng.integers(2)), bool(rng.integers(2))
    M, N, K = _size(rng), _size(rng), _size(rng)
    alpha = ALPHAS[int(rng.integers(len(ALPHAS)))]
    beta = BETAS[int(rng.integers(len(BETAS)))]
    cfg = CONFIGS[int(rng.integers(len(CONFIGS)))]
    A = inputs.integers((K, M) if tA else (M, K), 2000 + case)
    B = inputs.integers((N, K) if tB else (K, N), 3000 + case)
    C0 = inputs.integers((M, N), 4000 + case)
    h = g.Gemm()
    h.set_config(**cfg)
    out = g.matmul(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(),
                   C=torch.from_numpy(C0.copy()).cuda(), alpha=alpha, beta=beta, transA=tA,
                   transB=tB, mode=mode, h=h)
    torch.cuda.synchronize()
    assert h.sync() == 0
    ref, _, _ = oracle.gemm(A, B, alpha, beta, C0, transA=tA, transB=tB)
    got = out.cpu().numpy().astype(np.float64)
    assert np.array_equal(got, ref), (mode, tA, tB, M, N, K, alpha, beta, cfg)
    h.close()


@pytest.mark.parametrize("case", range(24))
def test_random_gemm_bf16_inputs_exact(case):
    import torch

    from paper_2305_18236_gb300 import gemm as g

    rng = np.random.default_rng(5000 + case)
    tA, tB = bool(rng.integers(2)), bool(rng.integers(2))
    # multiples of 8 keep every stored operand readable in place (ld % 8 == 0)
    M, N, K = (8 * max(1, _size(rng) // 8) for _ in range(3))
    alpha = ALPHAS[int(rng.integers(len(ALPHAS)))]
    beta = BETAS[int(rng.integers(len(BETAS)))]
    cfg = CONFIGS[int(rng.integers(len(CONFIGS)))]
    A = inputs.integers((K, M) if tA else (M, K), 6000 + case).astype(np.float32)
    B = inputs.integers((N, K) if tB else (K, N), 7000 + case).astype(np.float32)
    C0 = inputs.integers((M, N), 8000 + case)
    h = g.Gemm()
    h.set_config(**cfg)
    out = g.matmul_bf16(torch.from_numpy(A).cuda().to(torch.bfloat16),
                        torch.from_numpy(B).cuda().to(torch.bfloat16),
                        C=torch.from_numpy(C0.copy()).cuda(), alpha=alpha, beta=beta, transA=tA,
                        transB=tB, h=h)
    torch.cuda.synchronize()
    assert h.sync() == 0
    ref, _, _ = oracle.gemm(A, B, alpha, beta, C0, transA=tA, transB=tB)
    got = out.cpu().numpy().astype(np.float64)
    assert np.array_equal(got, ref), (tA, tB, M, N, K, alpha, beta, cfg)
    h.close()


@pytest.mark.parametrize("case", range(16))
def test_random_syr2k_exact(case):
    """Random triangle, orientation, mode, sizes, alpha/beta and tile
    configuration; elements outside the triangle start as NaN and must come
    back unchanged."""
    import torch

    from paper_2305_18236_gb300 import gemm as g

    rng = np.random.default_rng(9000 + case)
    mode = ["f32_simt", "bf16", "bf16x3"][case % 3]
    uplo = ["lower", "upper"][int(rng.integers(2))]
    trans = bool(rng.integers(2))
    N, K = _size(rng), _size(rng)
    alpha = ALPHAS[int(rng.integers(len(ALPHAS)))]
    beta = BETAS[int(rng.integers(len(BETAS)))]
    cfg = [{}, {"bn": 128}, {"bk": 64}, {"operand_layout": "as_stored"},
           {"operand_layout": "k_major", "max_ctas": 3}][int(rng.integers(5))]
    A = inputs.integers((K, N) if trans else (N, K), 9100 + case)
    B = inputs.integers((K, N) if trans else (N, K), 9200 + case)
    C0 = inputs.integers((N, N), 9300 + case)
    mask = np.tril(np.ones((N, N), bool)) if uplo == "lower" else np.triu(np.ones((N, N), bool))
    Cin = C0.copy()
    Cin[~mask] = np.nan
    h = g.Gemm()
    h.set_config(**cfg)
    dC = torch.from_numpy(Cin.copy()).cuda()
    g.syr2k(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), C=dC, alpha=alpha, beta=beta,
            uplo=uplo, trans=trans, mode=mode, h=h)
    torch.cuda.synchronize()
    assert h.sync() == 0
    out = dC.cpu().numpy()
    ref, _, _ = oracle.syr2k(A, B, alpha, beta, C0, uplo=uplo, trans=trans)
    assert np.array_equal(out[mask].astype(np.float64), ref[mask]), (mode, uplo, trans, N, K, cfg)
    assert np.all(np.isnan(out[~mask]))
    h.close()


@pytest.mark.parametrize("case", range(8))
def test_random_grouped_exact(case):
    """Random sets of problems (mixed transposes, ragged sizes, alpha/beta
    per problem, some empty) under random grouped configurations."""
    import torch

    from paper_2305_18236_gb300 import gemm as g

    rng = np.random.default_rng(9500 + case)
    mode = ["bf16", "bf16x3"][case % 2]
    cfg = [{}, {"cta_group": 2}, {"cta_group": 1, "bn": 128, "bk": 64},
           {"operand_layout": "k_major"}, {"operand_layout": "as_stored", "cta_group": 2}][
        int(rng.integers(5))]
    if mode == "bf16" and cfg.get("cta_group") == 2:
        cfg = dict(cfg, cta_group=1)  # grouped CTA pairs exist for 3xBF16
    probs, dev = [], []
    for i in range(int(rng.integers(3, 12))):
        M, N, K = _size(rng), _size(rng), _size(rng)
        tA, tB = bool(rng.integers(2)), bool(rng.integers(2))
        if i == 1:
            M, tA = 0, False  # an empty problem (stored 0 x K, so its ld stays valid)
        alpha = ALPHAS[int(rng.integers(len(ALPHAS)))]
        beta = BETAS[int(rng.integers(len(BETAS)))]
        A = inputs.integers((K, M) if tA else (M, K), 9600 + 40 * case + 3 * i)
        B = inputs.integers((N, K) if tB else (K, N), 9601 + 40 * case + 3 * i)
        C0 = inputs.integers((M, N), 9602 + 40 * case + 3 * i)
        probs.append((A, B, C0, tA, tB, alpha, beta))
        dev.append(dict(A=torch.from_numpy(A).cuda(), B=torch.from_numpy(B).cuda(),
                        C=torch.from_numpy(C0.copy()).cuda(), transA=tA, transB=tB,
                        alpha=alpha, beta=beta))
    h = g.Gemm()
    h.set_config(**cfg)
    plan = g.GroupedPlan(dev, mode=mode, h=h, autotune=bool(case % 4 == 3))
    plan.run()
    torch.cuda.synchronize()
    assert h.sync() == 0
    for (A, B, C0, tA, tB, alpha, beta), d in zip(probs, dev):
        ref, _, _ = oracle.gemm(A, B, alpha, beta, C0, transA=tA, transB=tB)
        assert np.array_equal(d["C"].cpu().numpy().astype(np.float64), ref), (mode, cfg)
    plan.close()
    h.close()


@pytest.mark.parametrize("case", range(24))
def test_random_float_within_bounds(case):
    """U[-1, 1] or log-uniform data under random configurations that keep the
    accumulation structure (no split-K, default promotion): normwise error
    against the exact oracle within the mode's bound, and against the
    oracle's GEMM of the same BF16 products within the accumulation bound."""
    from tests.gpu_util import TERMS, make_problem, oracle_ref, run_mode, tol_exact, tol_terms

    from paper_2305_18236_gb300 import gemm as g

    rng = np.random.default_rng(9900 + case)
    mode = ["f32_simt", "bf16", "bf16x3"][case % 3]
    tA, tB = bool(rng.integers(2)), bool(rng.integers(2))
    M, N, K = _size(rng), _size(rng), _size(rng)
    dist = ["uniform", "log_uniform"][int(rng.integers(2))]
    cfg = [{}, {"cta_group": 2}, {"cta_group": 1, "bn": 128}, {"cta_group": 1, "bk": 64},
           {"operand_layout": "as_stored"}, {"max_ctas": 7}][int(rng.integers(6))]
    A, B, C0 = make_problem(M, N, K, tA, tB, dist=dist, seed=9900 + 5 * case, beta=0.5)
    h = g.Gemm()
    h.set_config(**cfg)
    C = run_mode(mode, A, B, 1.5, 0.5, C0, tA, tB, h=h)
    assert h.sync() == 0
    C64, D = oracle_ref(A, B, 1.5, 0.5, C0, tA, tB)
    assert oracle.normwise_error(C, C64, D) <= tol_exact(mode, K), (mode, M, N, K, dist, cfg)
    if mode in TERMS:
        T64 = oracle.gemm_split_terms(A, B, TERMS[mode], 1.5, 0.5, C0, transA=tA, transB=tB)
        assert oracle.normwise_error(C, T64, D) <= tol_terms(mode, K), (mode, M, N, K, dist, cfg)
    h.close()
