"""SYR2K (Section 5.1) through the C ABI against the FP64 oracle (GB300 only).

C <- alpha (A B^T + B A^T) + beta C on one triangle (or alpha (A^T B + B^T A)
+ beta C with trans), every mode.  Elements outside the triangle must come
back bit for bit as they went in: they are set to NaN, so a stray read turns
a result NaN and a stray write replaces a NaN.
"""
import numpy as np
import pytest

import oracle
from paper_2305_18236_gb300 import inputs
from tests.gpu_util import TERMS, tol_exact, tol_terms

pytestmark = pytest.mark.gpu
MODES = ["f32_simt", "bf16", "bf16x3"]
UPLOS = ["lower", "upper"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2305_18236_gb300 import build

    build.build()


def _mask(N, uplo):
    return np.tril(np.ones((N, N), bool)) if uplo == "lower" else np.triu(np.ones((N, N), bool))


def _c_with_nan_outside(C0, uplo):
    C = C0.copy()
    C[~_mask(C0.shape[0], uplo)] = np.nan
    return C


def _run(A, B, C, alpha, beta, uplo, trans, mode, h=None):
    import torch

    from paper_2305_18236_gb300 import gemm as g

    dC = torch.from_numpy(C.copy()).cuda()
    g.syr2k(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), C=dC, alpha=alpha, beta=beta,
            uplo=uplo, trans=trans, mode=mode, h=h)
    torch.cuda.synchronize()
    return dC.cpu().numpy()


def _check_outside(out, Cin, uplo):
    m = ~_mask(out.shape[0], uplo)
    assert np.array_equal(out[m], Cin[m], equal_nan=True), "outside the triangle changed"


def _kpad(K, mode):
    # the tensor-core K loop runs over both products, each padded to BK = 64
    return 2 * (-(-K // 64) * 64) if mode != "f32_simt" else 2 * K


@pytest.mark.parametrize("trans", [False, True])
@pytest.mark.parametrize("uplo", UPLOS)
@pytest.mark.parametrize("mode", MODES)
def test_syr2k_integer_bit_exact(mode, uplo, trans):
    """Integer data in [-8, 8]: every partial sum exact, so the triangle is
    the oracle's bit for bit; ragged N spans several 128 x 256 tiles."""
    N, K = 333, 700
    A = inputs.integers((K, N) if trans else (N, K), 301)
    B = inputs.integers((K, N) if trans else (N, K), 302)
    C0 = inputs.integers((N, N), 303)
    Cin = _c_with_nan_outside(C0, uplo)
    out = _run(A, B, Cin, 1.5, 0.5, uplo, trans, mode)
    ref, _, _ = oracle.syr2k(A, B, 1.5, 0.5, C0, uplo=uplo, trans=trans)
    m = _mask(N, uplo)
    assert np.array_equal(out[m].astype(np.float64), ref[m])
    _check_outside(out, Cin, uplo)


@pytest.mark.parametrize("trans", [False, True])
@pytest.mark.parametrize("uplo", UPLOS)
@pytest.mark.parametrize("mode", MODES)
def test_syr2k_float_within_bounds(mode, uplo, trans):
    """U[-1, 1] data: normwise error against the exact oracle within the
    mode's bound, and against the oracle's split-product SYR2K within the
    accumulation bound of a 2K-long chain."""
    N, K = 300, 450
    A = inputs.uniform((K, N) if trans else (N, K), 311)
    B = inputs.uniform((K, N) if trans else (N, K), 312)
    C0 = inputs.uniform((N, N), 313)
    Cin = _c_with_nan_outside(C0, uplo)
    out = _run(A, B, Cin, 1.5, 0.5, uplo, trans, mode)
    _check_outside(out, Cin, uplo)
    m = _mask(N, uplo)
    C64, D, _ = oracle.syr2k(A, B, 1.5, 0.5, C0, uplo=uplo, trans=trans)
    sel = np.where(m, out, C0)
    assert oracle.normwise_error(sel, C64, D) <= tol_exact(mode, 2 * K)
    if mode in TERMS:
        T64, _, _ = oracle.syr2k(A, B, 1.5, 0.5, C0, uplo=uplo, trans=trans, terms=TERMS[mode],
                                 want_denominator=False)
        assert oracle.normwise_error(sel, T64, D) <= tol_terms(mode, _kpad(K, mode))


@pytest.mark.parametrize("bn,bk", [(128, 32), (128, 64), (256, 32), (256, 64)])
@pytest.mark.parametrize("uplo", UPLOS)
def test_syr2k_tile_configs_exact(bn, bk, uplo):
    """Every tile shape (the triangle walk depends on BN / 128) with a K
    that is not a multiple of BK in either product."""
    from paper_2305_18236_gb300 import gemm as g

    h = g.Gemm()
    h.set_config(bn=bn, bk=bk)
    N, K = 700, 333
    A = inputs.integers((N, K), 321)
    B = inputs.integers((N, K), 322)
    C0 = inputs.integers((N, N), 323)
    Cin = _c_with_nan_outside(C0, uplo)
    out = _run(A, B, Cin, 1.0, 1.0, uplo, False, "bf16x3", h=h)
    ref, _, _ = oracle.syr2k(A, B, 1.0, 1.0, C0, uplo=uplo)
    m = _mask(N, uplo)
    assert np.array_equal(out[m].astype(np.float64), ref[m])
    _check_outside(out, Cin, uplo)
    h.close()


@pytest.mark.parametrize("layout", ["as_stored", "k_major"])
@pytest.mark.parametrize("uplo", UPLOS)
def test_syr2k_layouts_and_small_grid(layout, uplo):
    """K x N operands (trans) staged MN-major or transposed K-major, with
    three persistent CTAs walking the triangle's tiles many times over."""
    from paper_2305_18236_gb300 import gemm as g

    h = g.Gemm()
    h.set_config(operand_layout=layout, max_ctas=3, stages=2)
    N, K = 900, 200
    A = inputs.integers((K, N), 331)
    B = inputs.integers((K, N), 332)
    C0 = inputs.integers((N, N), 333)
    Cin = _c_with_nan_outside(C0, uplo)
    out = _run(A, B, Cin, 1.5, 0.5, uplo, True, "bf16x3", h=h)
    ref, _, _ = oracle.syr2k(A, B, 1.5, 0.5, C0, uplo=uplo, trans=True)
    m = _mask(N, uplo)
    assert np.array_equal(out[m].astype(np.float64), ref[m])
    _check_outside(out, Cin, uplo)
    h.close()


@pytest.mark.parametrize("trans,launches", [(False, 3), (True, 1)])
@pytest.mark.parametrize("uplo", UPLOS)
def test_syr2k_simt_pack_exact(uplo, trans, launches):
    """FP32 SIMT SYR2K with N*N*K >= 2^30: operands stored N x K are first
    transposed into workspace (K x N copies, strides rounded up to 4) and
    the kernel runs its trans == T form; exact on integer data, nothing
    outside the triangle touched."""
    from paper_2305_18236_gb300 import gemm as g

    N, K = 1030, 1025
    A = inputs.integers((K, N) if trans else (N, K), 361)
    B = inputs.integers((K, N) if trans else (N, K), 362)
    C0 = inputs.integers((N, N), 363)
    Cin = _c_with_nan_outside(C0, uplo)
    h = g.Gemm()
    out = _run(A, B, Cin, 1.5, 0.5, uplo, trans, "f32_simt", h=h)
    assert h.last_launch_count() == launches
    ref, _, _ = oracle.syr2k(A, B, 1.5, 0.5, C0, uplo=uplo, trans=trans)
    m = _mask(N, uplo)
    assert np.array_equal(out[m].astype(np.float64), ref[m])
    _check_outside(out, Cin, uplo)
    h.close()


@pytest.mark.parametrize("mode", MODES)
def test_syr2k_special_cases(mode):
    """beta == 0 never reads C inside the triangle; alpha == 0 and K == 0
    scale the triangle only; N = 1 and tiny sizes."""
    import torch

    from paper_2305_18236_gb300 import gemm as g

    N, K = 150, 40
    A = inputs.uniform((N, K), 341)
    B = inputs.uniform((N, K), 342)
    C0 = inputs.uniform((N, N), 343)
    nan_in = np.full((N, N), np.nan, np.float32)
    nan_in[~_mask(N, "upper")] = 5.0
    out = _run(A, B, nan_in, 1.0, 0.0, "upper", False, mode)
    assert np.all(np.isfinite(out[_mask(N, "upper")]))
    _check_outside(out, nan_in, "upper")
    for uplo in UPLOS:
        m = _mask(N, uplo)
        Cin = _c_with_nan_outside(C0, uplo)
        nanA = np.full((N, K), np.nan, np.float32)
        out = _run(nanA, nanA, Cin, 0.0, 0.5, uplo, False, mode)
        assert np.array_equal(out[m], (np.float32(0.5) * C0)[m])
        _check_outside(out, Cin, uplo)
        dC = torch.from_numpy(Cin.copy()).cuda()
        g.syr2k(torch.zeros((N, 0), device="cuda"), torch.zeros((N, 0), device="cuda"), C=dC,
                alpha=1.0, beta=0.25, uplo=uplo, mode=mode)
        out = dC.cpu().numpy()
        assert np.array_equal(out[m], (np.float32(0.25) * C0)[m])
        _check_outside(out, Cin, uplo)
    for n, k in [(1, 1), (1, 7), (5, 3), (129, 17)]:
        A = inputs.integers((n, k), 344)
        B = inputs.integers((n, k), 345)
        C0 = inputs.integers((n, n), 346)
        Cin = _c_with_nan_outside(C0, "lower")
        out = _run(A, B, Cin, 1.5, 0.5, "lower", False, mode)
        ref, _, _ = oracle.syr2k(A, B, 1.5, 0.5, C0, uplo="lower")
        m = _mask(n, "lower")
        assert np.array_equal(out[m].astype(np.float64), ref[m])
        _check_outside(out, Cin, "lower")


def test_syr2k_large_sampled_rows():
    """N = K = 4096, 3xBF16, U[-1, 1]: sampled rows of the triangle against
    the exact oracle."""
    import torch

    from paper_2305_18236_gb300 import gemm as g

    N = K = 4096
    gen = torch.Generator(device="cuda").manual_seed(351)
    A = torch.rand((N, K), device="cuda", generator=gen) * 2 - 1
    B = torch.rand((N, K), device="cuda", generator=gen) * 2 - 1
    C = torch.zeros((N, N), device="cuda")
    g.syr2k(A, B, C=C, uplo="lower", mode="bf16x3")
    torch.cuda.synchronize()
    rows = np.linspace(0, N - 1, 10).astype(np.int64)
    C64, D, _ = oracle.syr2k(A.cpu().numpy(), B.cpu().numpy(), rows=rows, uplo="lower")
    out = C.cpu().numpy()[rows]
    out = np.where(np.tril(np.ones((N, N), bool))[rows], out, 0.0)
    assert oracle.normwise_error(out, C64, D) <= tol_exact("bf16x3", 2 * K)


def test_syr2k_argument_positions():
    import ctypes

    import torch

    from paper_2305_18236_gb300 import _lib
    from paper_2305_18236_gb300 import gemm as g

    h = g.Gemm()
    A = torch.zeros((64, 32), device="cuda")
    C = torch.zeros((64, 64), device="cuda")
    p = ctypes.c_void_p
    args = [h.h, 0, 0, 64, 32, 1.0, p(A.data_ptr()), 32, p(A.data_ptr()), 32, 0.0,
            p(C.data_ptr()), 64, 2, None]
    assert h.lib.gemm_syr2k(*args) == _lib.GEMM_OK
    for pos, value in [(2, 5), (3, 7), (4, -1), (5, -2), (8, 31), (10, 16), (13, 63), (14, 9)]:
        bad = list(args)
        bad[pos - 1] = value
        assert h.lib.gemm_syr2k(*bad) == _lib.GEMM_ERR_ARG
        assert h.last_error_arg() == pos
    bad = list(args)
    bad[6] = None  # A
    assert h.lib.gemm_syr2k(*bad) == _lib.GEMM_ERR_ARG and h.last_error_arg() == 7
    assert h.sync() == _lib.GEMM_OK
    h.close()
