"""Shared helpers of the GPU parity tests: seeded inputs on the device,
oracle references on the host, and the tolerances of each mode.

Tolerances (normwise error max|C - C64| / max D, D = |alpha||A||B| + |beta||C0|):
  * f32_simt: 1e-6 (FP32 accumulation).
  * bf16 vs the exact FP64 GEMM: 1e-2 (operands rounded to 8 bits).
  * bf16 vs the FP64 GEMM of the BF16-rounded operands: 1e-6.
  * bf16x3 vs the FP64 GEMM of the three split products: 1e-6.
  * bf16x3 vs the exact FP64 GEMM: 5e-5 = 3 * 2**-16 (each product keeps
    hi*hi + hi*lo + lo*hi; the dropped lo*lo and the split residuals are each
    below 2**-16 |a b|) plus FP32 accumulation; the headline size
    (K = 8192) is additionally held to 1e-6.
"""
import numpy as np
import torch

import oracle
from paper_2305_18236_gb300 import inputs

TOL_EXACT = {"f32_simt": 1e-6, "bf16": 1e-2, "bf16x3": 5e-5}
TOL_TERMS = 1e-6
TERMS = {"bf16": oracle.TERM_HH, "bf16x3": oracle.TERM_HH | oracle.TERM_HL | oracle.TERM_LH}
MODES = ["f32_simt", "bf16", "bf16x3"]


def stored_shape(rows, cols, trans):
    return (cols, rows) if trans else (rows, cols)


def make_problem(M, N, K, transA=False, transB=False, dist="uniform", seed=1, beta=0.0):
    A = inputs.make(dist, stored_shape(M, K, transA), seed, k=K)
    B = inputs.make(dist, stored_shape(K, N, transB), seed + 1, k=K)
    C0 = inputs.uniform((M, N), seed + 2) if beta != 0.0 else None
    return A, B, C0


def to_dev(x):
    return None if x is None else torch.from_numpy(np.ascontiguousarray(x)).cuda()


def oracle_ref(A, B, alpha, beta, C0, transA, transB, rows=None):
    C64, D, _ = oracle.gemm(A, B, alpha, beta, C0, transA=transA, transB=transB, rows=rows)
    return C64, D


def run_mode(mode, A, B, alpha, beta, C0, transA, transB, h=None):
    from paper_2305_18236_gb300 import gemm as g

    dA, dB = to_dev(A), to_dev(B)
    M = A.shape[1] if transA else A.shape[0]
    N = B.shape[0] if transB else B.shape[1]
    C = to_dev(C0) if C0 is not None else None
    out = g.matmul(dA, dB, C=C, alpha=alpha, beta=beta, transA=transA, transB=transB, mode=mode,
                   h=h)
    torch.cuda.synchronize()
    assert tuple(out.shape) == (M, N)
    return out.cpu().numpy()


def check_mode(mode, A, B, alpha, beta, C0, transA, transB, rows=None, tol_exact=None, h=None):
    """Run one GEMM on the GPU and compare it to the oracle; returns the
    normwise error against the exact FP64 GEMM."""
    C = run_mode(mode, A, B, alpha, beta, C0, transA, transB, h=h)
    sel = C if rows is None else C[rows]
    C64, D = oracle_ref(A, B, alpha, beta, C0, transA, transB, rows)
    err = oracle.normwise_error(sel, C64, D)
    tol = TOL_EXACT[mode] if tol_exact is None else tol_exact
    assert np.all(np.isfinite(sel)), "non-finite output"
    assert err <= tol, "%s: normwise error %.3e > %.1e" % (mode, err, tol)
    if mode in TERMS:
        T64 = oracle.gemm_split_terms(A, B, TERMS[mode], alpha, beta, C0, transA=transA,
                                      transB=transB, rows=rows)
        terr = oracle.normwise_error(sel, T64, D)
        assert terr <= TOL_TERMS, "%s vs split-term oracle: %.3e" % (mode, terr)
    return err
