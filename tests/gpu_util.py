"""Shared helpers of the GPU parity tests: seeded inputs on the device,
oracle references on the host, and the tolerances of each mode.

Error measure: normwise error max|C - C64| / max D with
D = |alpha| |op(A)| |op(B)| + |beta| |C0| (the oracle's denominator).

Tolerances, derived from the arithmetic of each path:
  * f32_simt: 1e-6 (FP32 fused multiply-adds in increasing k).
  * bf16 vs the exact FP64 GEMM: 1e-2 (operands rounded to 8 bits).
  * bf16 / bf16x3 vs the oracle's FP64 GEMM of the same BF16 products
    (``oracle.gemm_split_terms``): only accumulation error remains.  The
    tensor core adds each 16-deep MMA into its FP32 accumulator rounding
    toward zero, losing less than one ulp of the running sum (<= D) per
    MMA: at most (number of MMAs summed in one TMEM chain + 2) * 2**-23.
    bf16 sums all ceil(K/16) MMAs in one chain; bf16x3 sums chains of
    3 * 512/16 = 96 MMAs and adds the chains in FP32 with round-to-nearest
    (at most 2**-24 each).
  * bf16x3 vs the exact FP64 GEMM: the three kept products miss lo*lo and
    the split residuals, each below 2**-16 |a b|: 3 * 2**-16 plus the
    accumulation bound.  The benchmark size (K = 8192, uniform data) is
    additionally held to the 1e-6 bar.
"""
import numpy as np
import torch

import oracle
from paper_2305_18236_gb300 import inputs

PROMOTE_K = 512  # K elements per TMEM chain in the bf16x3 mode (library default)


def tol_terms(mode, K):
    """Accumulation-error bound of a tensor-core mode (see module doc)."""
    ulp = 2.0 ** -23
    if mode == "bf16":
        return (-(-K // 16) + 2) * ulp
    chain = 3 * min(K, PROMOTE_K) // 16 + 1
    return (chain + 2) * ulp + (-(-K // PROMOTE_K) + 1) * 2.0 ** -24


def tol_exact(mode, K):
    if mode == "f32_simt":
        return 1e-6
    if mode == "bf16":
        return 1e-2
    return 3 * 2.0 ** -16 + tol_terms(mode, K)


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


def check_mode(mode, A, B, alpha, beta, C0, transA, transB, rows=None, tol=None, h=None):
    """Run one GEMM on the GPU and compare it to the oracle; returns the
    normwise error against the exact FP64 GEMM."""
    C = run_mode(mode, A, B, alpha, beta, C0, transA, transB, h=h)
    sel = C if rows is None else C[rows]
    C64, D = oracle_ref(A, B, alpha, beta, C0, transA, transB, rows)
    err = oracle.normwise_error(sel, C64, D)
    K = A.shape[0] if transA else A.shape[1]
    tol = tol_exact(mode, K) if tol is None else tol
    assert np.all(np.isfinite(sel)), "non-finite output"
    assert err <= tol, "%s: normwise error %.3e > %.1e" % (mode, err, tol)
    if mode in TERMS:
        T64 = oracle.gemm_split_terms(A, B, TERMS[mode], alpha, beta, C0, transA=transA,
                                      transB=transB, rows=rows)
        terr = oracle.normwise_error(sel, T64, D)
        assert terr <= tol_terms(mode, K), "%s vs split-term oracle: %.3e > %.3e" % (
            mode, terr, tol_terms(mode, K))
    return err
