"""gemm_bf16x3_noalloc: the split-precision GEMM for callers that cannot
allocate device memory (it uses a fixed scratch array inside the library
instead of a handle and workspace).  Its results must equal those of the
ordinary gemm() entry point in GEMM_MODE_BF16X3, call after call.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from paper_2305_18236_gb300 import inputs
from tests.gpu_util import tol_terms

pytestmark = pytest.mark.gpu


def _noalloc(lib, A, B, C, alpha, beta, transA=0, transB=0):
    import torch

    M, N = C.shape
    K = A.shape[0] if transA else A.shape[1]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.gemm_bf16x3_noalloc(transA, transB, M, N, K, alpha,
                                   ctypes.c_void_p(A.data_ptr()), A.stride(0),
                                   ctypes.c_void_p(B.data_ptr()), B.stride(0), beta,
                                   ctypes.c_void_p(C.data_ptr()), C.stride(0), stream)


def test_noalloc_matches_gemm_two_calls_in_a_row():
    import torch

    from paper_2305_18236_gb300 import _lib, build
    from paper_2305_18236_gb300 import gemm as g

    build.build()
    lib = _lib.load()
    # two different problems back to back: the second must not see the
    # first one's leftovers in the shared scratch array
    for call, (M, N, K, tA, tB) in enumerate([(520, 700, 1000, 0, 0), (300, 260, 1500, 1, 1)]):
        A = torch.from_numpy(inputs.uniform((K, M) if tA else (M, K), 500 + call)).cuda()
        B = torch.from_numpy(inputs.uniform((N, K) if tB else (K, N), 600 + call)).cuda()
        C0 = torch.from_numpy(inputs.uniform((M, N), 700 + call)).cuda()
        C_noalloc = C0.clone()
        st = _noalloc(lib, A, B, C_noalloc, 1.5, 0.5, tA, tB)
        assert st == _lib.GEMM_OK, _lib.status_string(st)
        C_ref = C0.clone()
        h = g.Gemm()
        h.set_config(split_k=1)
        g.matmul(A, B, C=C_ref, alpha=1.5, beta=0.5, transA=bool(tA), transB=bool(tB),
                 mode="bf16x3", h=h)
        torch.cuda.synchronize()
        got, ref = C_noalloc.cpu().numpy(), C_ref.cpu().numpy()
        assert np.all(np.isfinite(got))
        # same kernels and configuration: identical up to the accumulation bound
        scale = float(np.max(np.abs(ref))) or 1.0
        assert float(np.max(np.abs(got - ref))) / scale <= tol_terms("bf16x3", K)
        h.close()


def test_noalloc_rejects_problems_beyond_its_scratch():
    import torch

    from paper_2305_18236_gb300 import _lib, build

    build.build()
    lib = _lib.load()
    # 4 * (M + N) * K = 4 * 8192 * 4096 bytes = 128 MiB > 64 MiB: refused, nothing launched
    A = torch.zeros((4096, 4096), device="cuda")
    B = torch.zeros((4096, 4096), device="cuda")
    C = torch.full((4096, 4096), 7.0, device="cuda")
    st = _noalloc(lib, A, B, C, 1.0, 0.0)
    assert st == _lib.GEMM_ERR_WORKSPACE
    torch.cuda.synchronize()
    assert bool((C == 7.0).all())
