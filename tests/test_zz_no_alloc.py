"""gemm_bf16x3_noalloc: the split-precision GEMM for callers that cannot
allocate device memory (a custom allocator's own hooks, plugins whose host
application owns all device memory, loops that must never enter the driver's
allocator).  It uses a fixed scratch array inside the library instead of a
handle and workspace.

Its results are checked against the FP64 oracle (the exact GEMM and the GEMM
of the same BF16 split products), bit for bit on integer data, and against
the ordinary gemm() entry point in GEMM_MODE_BF16X3, call after call; a call
must leave the device's free memory unchanged.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2305_18236_gb300 import inputs
from tests.gpu_util import TERMS, tol_exact, tol_terms

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2305_18236_gb300 import _lib, build

    build.build()
    return _lib.load()


def _stream():
    import torch

    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _noalloc(lib, A, B, C, alpha, beta, transA=0, transB=0, K=None):
    M, N = C.shape
    if K is None:
        K = A.shape[0] if transA else A.shape[1]
    return lib.gemm_bf16x3_noalloc(transA, transB, M, N, K, alpha,
                                   ctypes.c_void_p(A.data_ptr()), A.stride(0),
                                   ctypes.c_void_p(B.data_ptr()), B.stride(0), beta,
                                   ctypes.c_void_p(C.data_ptr()), C.stride(0), _stream())


def _check(lib):
    from paper_2305_18236_gb300 import _lib as L

    st = lib.gemm_bf16x3_noalloc_check(_stream())
    assert st == L.GEMM_OK, L.status_string(st)


def test_noalloc_matches_oracle_and_gemm_two_calls_in_a_row():
    import torch

    from paper_2305_18236_gb300 import _lib as L
    from paper_2305_18236_gb300 import gemm as g

    lib = _lib()
    # two different problems back to back: the second must not see the
    # first one's leftovers in the shared scratch array
    for call, (M, N, K, tA, tB) in enumerate([(520, 700, 1000, 0, 0), (300, 260, 1500, 1, 1)]):
        A = inputs.uniform((K, M) if tA else (M, K), 500 + call)
        B = inputs.uniform((N, K) if tB else (K, N), 600 + call)
        C0 = inputs.uniform((M, N), 700 + call)
        dA, dB, dC0 = (torch.from_numpy(x).cuda() for x in (A, B, C0))
        C_noalloc = dC0.clone()
        st = _noalloc(lib, dA, dB, C_noalloc, 1.5, 0.5, tA, tB)
        assert st == L.GEMM_OK, L.status_string(st)
        _check(lib)
        got = C_noalloc.cpu().numpy()
        assert np.all(np.isfinite(got))
        C64, D, _ = oracle.gemm(A, B, 1.5, 0.5, C0, transA=bool(tA), transB=bool(tB))
        assert oracle.normwise_error(got, C64, D) <= tol_exact("bf16x3", K)
        T64 = oracle.gemm_split_terms(A, B, TERMS["bf16x3"], 1.5, 0.5, C0, transA=bool(tA),
                                      transB=bool(tB))
        assert oracle.normwise_error(got, T64, D) <= tol_terms("bf16x3", K)
        # the ordinary entry point on the same problem (no split-K, so the
        # same kernels and configuration)
        C_ref = dC0.clone()
        h = g.Gemm()
        h.set_config(split_k=1)
        g.matmul(dA, dB, C=C_ref, alpha=1.5, beta=0.5, transA=bool(tA), transB=bool(tB),
                 mode="bf16x3", h=h)
        torch.cuda.synchronize()
        assert oracle.normwise_error(got, C_ref.cpu().numpy().astype(np.float64), D) \
            <= tol_terms("bf16x3", K)
        h.close()


def test_noalloc_integer_data_bit_exact_with_padded_strides():
    """Integer data (every partial sum exact in FP32) with lda > K and
    ldc > N: the result equals the exact product bit for bit, and the
    padding columns of C are untouched."""
    import torch

    from paper_2305_18236_gb300 import _lib as L

    lib = _lib()
    M, N, K = 300, 200, 777
    A = inputs.integers((M, K), 11)
    B = inputs.integers((K, N), 12)
    C0 = inputs.integers((M, N), 13)
    dA = torch.zeros((M, K + 9), device="cuda")
    dA[:, :K] = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    dC = torch.full((M, N + 5), -3.0, device="cuda")
    dC[:, :N] = torch.from_numpy(C0).cuda()
    st = lib.gemm_bf16x3_noalloc(0, 0, M, N, K, 1.5, ctypes.c_void_p(dA.data_ptr()), K + 9,
                                 ctypes.c_void_p(dB.data_ptr()), N, 0.5,
                                 ctypes.c_void_p(dC.data_ptr()), N + 5, _stream())
    assert st == L.GEMM_OK, L.status_string(st)
    _check(lib)
    got = dC.cpu().numpy()
    C64, _, _ = oracle.gemm(A, B, 1.5, 0.5, C0)
    assert np.array_equal(got[:, :N].astype(np.float64), C64)
    assert np.all(got[:, N:] == -3.0)


def test_noalloc_quick_returns():
    """alpha == 0 never reads A or B (NaN there stays out); K == 0 gives
    C <- beta C; beta == 0 never reads C."""
    import torch

    lib = _lib()
    M, N, K = 70, 90, 50
    nanA = torch.full((M, K), float("nan"), device="cuda")
    nanB = torch.full((K, N), float("nan"), device="cuda")
    C0 = torch.from_numpy(inputs.uniform((M, N), 21)).cuda()
    C = C0.clone()
    assert _noalloc(lib, nanA, nanB, C, 0.0, 0.5) == 0
    torch.cuda.synchronize()
    assert torch.equal(C, 0.5 * C0)
    C = C0.clone()
    assert _noalloc(lib, nanA, nanB, C, 1.0, 2.0, K=0) == 0
    torch.cuda.synchronize()
    assert torch.equal(C, 2.0 * C0)
    A = torch.from_numpy(inputs.integers((M, K), 22)).cuda()
    B = torch.from_numpy(inputs.integers((K, N), 23)).cuda()
    C = torch.full((M, N), float("nan"), device="cuda")
    assert _noalloc(lib, A, B, C, 1.0, 0.0) == 0
    _check(lib)
    exact, _, _ = oracle.gemm(A.cpu().numpy(), B.cpu().numpy())
    assert np.array_equal(C.cpu().numpy().astype(np.float64), exact)


def test_noalloc_allocates_nothing():
    """After one call on the device (which loads the module and reserves its
    scratch), further calls leave the device's free memory unchanged."""
    import torch

    lib = _lib()
    M, N, K = 512, 384, 640
    A = torch.from_numpy(inputs.uniform((M, K), 31)).cuda()
    B = torch.from_numpy(inputs.uniform((K, N), 32)).cuda()
    C = torch.zeros((M, N), device="cuda")
    assert _noalloc(lib, A, B, C, 1.0, 0.0) == 0
    _check(lib)
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert _noalloc(lib, A, B, C, 1.0, 0.0) == 0
    _check(lib)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_problems_beyond_its_scratch():
    import torch

    from paper_2305_18236_gb300 import _lib as L

    lib = _lib()
    # 4 * (M + N) * K = 4 * 8192 * 4096 bytes = 128 MiB > 64 MiB: refused, nothing launched
    A = torch.zeros((4096, 4096), device="cuda")
    B = torch.zeros((4096, 4096), device="cuda")
    C = torch.full((4096, 4096), 7.0, device="cuda")
    st = _noalloc(lib, A, B, C, 1.0, 0.0)
    assert st == L.GEMM_ERR_WORKSPACE
    torch.cuda.synchronize()
    assert bool((C == 7.0).all())
