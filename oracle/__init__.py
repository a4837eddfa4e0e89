"""FP64 CPU oracle for C = alpha*op(A)*op(B) + beta*C -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library shares no code with
it: the arithmetic lives in ``gemm_ref.c`` (compiled with gcc by
``oracle/build.py``) and this module only marshals numpy arrays.

Functions (each follows Kuzma et al., Section 3, Algorithm 1, whose blocked
loop nest computes alpha * op(A) op(B) + beta * C with beta applied once):

* ``gemm`` -- the FP64 result C64 and the error denominator D.
* ``gemm_split_terms`` -- the same with op(A), op(B) replaced by sums of
  their BF16 split parts (not in the paper; the definition is stated in
  ``gemm_ref.c``).
* ``split_bf16`` / ``bf16_bits_to_f32`` -- the hi/lo BF16 split.
* ``syr2k`` -- one triangle of C = alpha (opA opB^T + opB opA^T) + beta C,
  the rank-2k update of Section 5.1 (exact or with split products).
* ``normwise_error`` -- max |C - C64| / max D, the error measure.

Every function is pinned by ``tests/test_oracle_pins.py`` (the checks in
``tests/oracle_pins.py``), ``normwise_error`` included (hand-computed cases);
``tests/test_oracle_mutants.py`` plants mistakes in ``gemm_ref.c`` and in
``normwise_error`` and each one fails a pin.
"""
import ctypes
import os

import numpy as np

from .build import build_oracle

_lib = None


def _declare(lib):
    """Declare the C signatures on a loaded oracle library."""
    i64, f64p, f32p = ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float)
    i64p, u16p = ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_uint16)
    lib.oracle_gemm.restype = ctypes.c_int
    lib.oracle_gemm.argtypes = [ctypes.c_int, ctypes.c_int, i64, i64, i64,
                                ctypes.c_double, f32p, i64, f32p, i64,
                                ctypes.c_double, f32p, i64, i64p, i64,
                                f64p, f64p, ctypes.c_int]
    lib.oracle_gemm_split_terms.restype = ctypes.c_int
    lib.oracle_gemm_split_terms.argtypes = [ctypes.c_int, ctypes.c_int, i64, i64, i64,
                                            ctypes.c_double, f32p, i64, f32p, i64,
                                            ctypes.c_double, f32p, i64, ctypes.c_int,
                                            i64p, i64, f64p, ctypes.c_int]
    lib.oracle_syr2k.restype = ctypes.c_int
    lib.oracle_syr2k.argtypes = [ctypes.c_int, ctypes.c_int, i64, i64, ctypes.c_double,
                                 f32p, i64, f32p, i64, ctypes.c_double, f32p, i64,
                                 ctypes.c_int, i64p, i64, f64p, f64p, ctypes.c_int]
    lib.oracle_split.restype = None
    lib.oracle_split.argtypes = [f32p, i64, u16p, u16p]
    lib.oracle_bf16_rne.restype = ctypes.c_uint16
    lib.oracle_bf16_rne.argtypes = [ctypes.c_float]
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _declare(ctypes.CDLL(build_oracle()))
    return _lib


def load_variant(path):
    """Load another build of the oracle source (mutation tests) and return an
    object with this module's functions bound to it."""
    lib = _declare(ctypes.CDLL(path))

    class _Bound:
        pass

    b = _Bound()
    for name in ("gemm", "gemm_split_terms", "split_bf16", "syr2k"):
        fn = globals()[name]
        setattr(b, name, (lambda f: lambda *a, **k: f(*a, _library=lib, **k))(fn))
    b.normwise_error = normwise_error
    b.bf16_bits_to_f32 = bf16_bits_to_f32
    return b


def lib():
    """The loaded ctypes library (for tests that call a symbol directly)."""
    return _load()


def _f32_view(x):
    """(pointer, ld, keepalive) for a 2-D float32 array whose last axis is
    contiguous; a strided row view passes its row stride as ld."""
    x = np.asarray(x)
    if x.dtype != np.float32:
        raise TypeError("oracle inputs are float32")
    if x.ndim != 2:
        raise ValueError("oracle inputs are 2-D")
    if x.strides[1] != 4 or x.strides[0] % 4 != 0 or x.strides[0] < 0:
        x = np.ascontiguousarray(x)
    ld = x.strides[0] // 4 if x.shape[0] > 1 else max(1, x.shape[1])
    return x.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ld, x


def _dims(transA, transB, A, B):
    A = np.asarray(A)
    B = np.asarray(B)
    M, K = (A.shape[1], A.shape[0]) if transA else A.shape
    Kb, N = (B.shape[1], B.shape[0]) if transB else B.shape
    if K != Kb:
        raise ValueError("inner dimensions differ: %d vs %d" % (K, Kb))
    return M, N, K


def gemm(A, B, alpha=1.0, beta=0.0, C0=None, transA=False, transB=False,
         rows=None, threads=0, want_denominator=True, _library=None):
    """C64 = alpha*op(A)@op(B) + beta*C0 in FP64 (rows: optional row subset).

    Returns (C64, D, threads_used).  A, B, C0 are float32 2-D arrays in
    row-major storage; op(X) = X.T when trans is set.
    """
    l = _library or _load()
    M, N, K = _dims(transA, transB, A, B)
    pa, lda, ka = _f32_view(A)
    pb, ldb, kb = _f32_view(B)
    if beta != 0.0:
        if C0 is None:
            raise ValueError("beta != 0 needs C0")
        pc, ldc, kc = _f32_view(C0)
        if C0.shape != (M, N):
            raise ValueError("C0 shape")
    else:
        pc, ldc, kc = None, max(1, N), None
    if rows is None:
        nrows, prow, krow = M, None, None
    else:
        krow = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
        if krow.size and (krow.min() < 0 or krow.max() >= M):
            raise ValueError("row index out of range")
        nrows = krow.size
        prow = krow.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    C64 = np.zeros((nrows, N), dtype=np.float64)
    D = np.zeros((nrows, N), dtype=np.float64) if want_denominator else None
    used = l.oracle_gemm(int(bool(transA)), int(bool(transB)), M, N, K,
                         float(alpha), pa, lda, pb, ldb, float(beta), pc, ldc,
                         prow, nrows,
                         C64.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                         D.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if D is not None else None,
                         int(threads))
    return C64, D, used


TERM_HH, TERM_HL, TERM_LH, TERM_LL = 1, 2, 4, 8


def gemm_split_terms(A, B, terms, alpha=1.0, beta=0.0, C0=None, transA=False,
                     transB=False, rows=None, threads=0, _library=None):
    """FP64 GEMM of the selected BF16 split cross products (see gemm_ref.c)."""
    l = _library or _load()
    M, N, K = _dims(transA, transB, A, B)
    pa, lda, ka = _f32_view(A)
    pb, ldb, kb = _f32_view(B)
    if beta != 0.0:
        pc, ldc, kc = _f32_view(C0)
    else:
        pc, ldc, kc = None, max(1, N), None
    if rows is None:
        nrows, prow, krow = M, None, None
    else:
        krow = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
        nrows = krow.size
        prow = krow.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    C64 = np.zeros((nrows, N), dtype=np.float64)
    l.oracle_gemm_split_terms(int(bool(transA)), int(bool(transB)), M, N, K,
                              float(alpha), pa, lda, pb, ldb, float(beta), pc, ldc,
                              int(terms), prow, nrows,
                              C64.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                              int(threads))
    return C64


def syr2k(A, B, alpha=1.0, beta=0.0, C0=None, uplo="lower", trans=False, terms=0, rows=None,
          threads=0, want_denominator=True, _library=None):
    """One triangle of alpha (opA opB^T + opB opA^T) + beta C0 in FP64.

    opX = X (stored N x K) or X.T (X stored K x N, ``trans``).  Entries outside
    the ``uplo`` triangle ("lower": j <= i, "upper": j >= i) hold C0 (0 when
    C0 is None) and a zero denominator.  ``terms`` != 0 replaces every product
    by the selected BF16 split cross products (bits as in gemm_split_terms).
    Returns (C64, D, threads_used) for the requested rows.
    """
    l = _library or _load()
    A = np.asarray(A)
    B = np.asarray(B)
    if A.shape != B.shape:
        raise ValueError("A and B must have the same shape")
    N, K = (A.shape[1], A.shape[0]) if trans else A.shape
    if uplo not in ("lower", "upper"):
        raise ValueError("uplo is 'lower' or 'upper'")
    pa, lda, ka = _f32_view(A)
    pb, ldb, kb = _f32_view(B)
    if C0 is not None:
        if C0.shape != (N, N):
            raise ValueError("C0 shape")
        pc, ldc, kc = _f32_view(C0)
    elif beta != 0.0:
        raise ValueError("beta != 0 needs C0")
    else:
        pc, ldc, kc = None, max(1, N), None
    if rows is None:
        nrows, prow, krow = N, None, None
    else:
        krow = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
        if krow.size and (krow.min() < 0 or krow.max() >= N):
            raise ValueError("row index out of range")
        nrows = krow.size
        prow = krow.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    C64 = np.zeros((nrows, N), dtype=np.float64)
    D = np.zeros((nrows, N), dtype=np.float64) if want_denominator else None
    used = l.oracle_syr2k(0 if uplo == "lower" else 1, int(bool(trans)), N, K, float(alpha),
                          pa, lda, pb, ldb, float(beta), pc, ldc, int(terms), prow, nrows,
                          C64.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                          D.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if D is not None else None,
                          int(threads))
    return C64, D, used


def split_bf16(x, _library=None):
    """(hi, lo) BF16 bit patterns (uint16) of a float32 array."""
    l = _library or _load()
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    hi = np.empty(x.shape, dtype=np.uint16)
    lo = np.empty(x.shape, dtype=np.uint16)
    l.oracle_split(x.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), x.size,
                   hi.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16)),
                   lo.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16)))
    return hi, lo


def bf16_bits_to_f32(h):
    """BF16 bit patterns -> the float32 values they denote (exact)."""
    h = np.asarray(h, dtype=np.uint16)
    return (h.astype(np.uint32) << 16).view(np.float32)


def normwise_error(C, C64, D):
    """max_ij |C - C64| / max_ij D (0 when both numerator and D vanish)."""
    C = np.asarray(C, dtype=np.float64)
    num = float(np.max(np.abs(C - C64))) if C.size else 0.0
    den = float(np.max(D)) if D is not None and D.size else 0.0
    if num == 0.0:
        return 0.0
    if den == 0.0:
        return float("inf")
    return num / den


def host_cores():
    """Number of host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1
