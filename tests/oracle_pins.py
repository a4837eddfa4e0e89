"""Pins for the FP64 oracle: checks against facts that do not come from the
oracle itself (exact rational brute force, closed forms, integer matmul,
library conversions, invariants of the GEMM definition).

Each ``check_*`` takes an oracle-like object (the ``oracle`` package or a
mutant build bound with ``oracle.load_variant``) and raises AssertionError
on a mismatch, so the mutation tests can run the same checks against
planted mistakes.

GEMM definition: Kuzma et al., Section 3, Algorithm 1 -- the blocked loop
nest leaves C = alpha * op(A) op(B) + beta * C0, beta applied once (on the
first K block), alpha applied to every block's product.
"""
from fractions import Fraction
from itertools import product

import numpy as np

from paper_2305_18236_gb300 import inputs

TRANS = list(product([False, True], [False, True]))


def _stored(x, trans):
    """Storage that makes op(stored) == x."""
    return np.ascontiguousarray(x.T) if trans else np.ascontiguousarray(x)


def _exact(opA, opB, alpha, beta, C0):
    M, K = opA.shape
    N = opB.shape[1]
    C = [[None] * N for _ in range(M)]
    D = [[None] * N for _ in range(M)]
    fa, fb = Fraction(float(alpha)), Fraction(float(beta))
    for i in range(M):
        for j in range(N):
            s = Fraction(0)
            m = Fraction(0)
            for k in range(K):
                a, b = Fraction(float(opA[i, k])), Fraction(float(opB[k, j]))
                s += a * b
                m += abs(a) * abs(b)
            c = fa * s
            d = abs(fa) * m
            if beta != 0.0:
                c0 = Fraction(float(C0[i, j]))
                c += fb * c0
                d += abs(fb) * abs(c0)
            C[i][j] = c
            D[i][j] = d
    return C, D


def check_brute_force(orc, seed=1):
    """FP64 result within the FP64 summation bound of the exact rational
    result, for tiny shapes including the 8x5 . 5x16 tile of Listing 1,
    all four transpose combinations and several alpha/beta."""
    shapes = [(8, 16, 5), (1, 1, 1), (3, 4, 2), (7, 3, 6), (2, 9, 1)]
    for (M, N, K), (tA, tB), (alpha, beta) in product(
            shapes, TRANS, [(1.0, 0.0), (1.5, 0.5), (-0.75, 2.0)]):
        opA = inputs.uniform((M, K), seed)
        opB = inputs.uniform((K, N), seed + 1)
        C0 = inputs.uniform((M, N), seed + 2)
        C64, D, _ = orc.gemm(_stored(opA, tA), _stored(opB, tB), alpha, beta,
                             C0, transA=tA, transB=tB)
        Cx, Dx = _exact(opA, opB, alpha, beta, C0)
        u = 2.0 ** -53
        for i in range(M):
            for j in range(N):
                bound = 2.0 * (K + 3) * u * float(Dx[i][j])
                assert abs(Fraction(float(C64[i, j])) - Cx[i][j]) <= Fraction(bound), \
                    ("C", M, N, K, tA, tB, alpha, beta, i, j)
                assert abs(Fraction(float(D[i, j])) - Dx[i][j]) <= Fraction(bound), \
                    ("D", M, N, K, tA, tB, alpha, beta, i, j)


def check_identity(orc):
    """op(A) I = op(A) and I op(B) = op(B) exactly."""
    for tA, tB in TRANS:
        X = inputs.log_uniform((9, 6), 3)
        I6 = np.eye(6, dtype=np.float32)
        I9 = np.eye(9, dtype=np.float32)
        C, _, _ = orc.gemm(_stored(X, tA), _stored(I6, tB), transA=tA, transB=tB)
        assert np.array_equal(C, X.astype(np.float64))
        C, _, _ = orc.gemm(_stored(I9, tA), _stored(X, tB), transA=tA, transB=tB)
        assert np.array_equal(C, X.astype(np.float64))


def check_permutation(orc):
    """P A permutes rows and A Q permutes columns, exactly."""
    X = inputs.uniform((7, 5), 4)
    rp = np.array([3, 0, 6, 1, 5, 2, 4])
    cp = np.array([4, 2, 0, 3, 1])
    P = np.eye(7, dtype=np.float32)[rp]
    Q = np.eye(5, dtype=np.float32)[:, cp]
    for tA, tB in TRANS:
        C, _, _ = orc.gemm(_stored(P, tA), _stored(X, tB), transA=tA, transB=tB)
        assert np.array_equal(C, X[rp].astype(np.float64))
        C, _, _ = orc.gemm(_stored(X, tA), _stored(Q, tB), transA=tA, transB=tB)
        assert np.array_equal(C, X[:, cp].astype(np.float64))


def check_all_ones(orc):
    """All-ones operands: C_ij = alpha*K + beta*C0_ij exactly."""
    for (M, N, K), (tA, tB) in product([(5, 7, 33), (1, 3, 1), (4, 4, 1000)], TRANS):
        C0 = inputs.integers((M, N), 5).astype(np.float32) / 4
        C, _, _ = orc.gemm(np.ones((K, M) if tA else (M, K), np.float32),
                           np.ones((N, K) if tB else (K, N), np.float32),
                           1.5, 0.5, C0, transA=tA, transB=tB)
        assert np.array_equal(C, 1.5 * K + 0.5 * C0.astype(np.float64))


def check_integers(orc):
    """Integer-valued inputs equal numpy's int64 matmul exactly."""
    for (M, N, K), (tA, tB) in product([(13, 11, 17), (64, 3, 130)], TRANS):
        opA = inputs.integers((M, K), 6)
        opB = inputs.integers((K, N), 7)
        C0 = inputs.integers((M, N), 8)
        ref = 2 * (opA.astype(np.int64) @ opB.astype(np.int64)) - 3 * C0.astype(np.int64)
        C, _, _ = orc.gemm(_stored(opA, tA), _stored(opB, tB), 2.0, -3.0, C0,
                           transA=tA, transB=tB)
        assert np.array_equal(C, ref.astype(np.float64))


def check_transpose_identity(orc):
    """(op(A) op(B))^T = op(B)^T op(A)^T: the column-major call is the
    row-major call with operands swapped."""
    opA = inputs.integers((6, 9), 9)
    opB = inputs.integers((9, 4), 10)
    C, _, _ = orc.gemm(opA, opB)
    Ct, _, _ = orc.gemm(opB, opA, transA=True, transB=True)
    # op(B)^T is passed as the first operand: stored opB with trans -> opB^T
    assert np.array_equal(Ct, C.T)


def check_blocked_k(orc):
    """Algorithm 1's blocking: beta on the first K block only, alpha on every
    block, equals the unblocked result (exact on dyadic inputs)."""
    opA = inputs.integers((10, 24), 11) / 8
    opB = inputs.integers((24, 7), 12) / 4
    C0 = inputs.integers((10, 7), 13).astype(np.float32)
    full, _, _ = orc.gemm(opA, opB, 1.5, 0.5, C0)
    cur = C0
    for k0, k1 in [(0, 5), (5, 16), (16, 24)]:
        beta = 0.5 if k0 == 0 else 1.0
        part, _, _ = orc.gemm(np.ascontiguousarray(opA[:, k0:k1]),
                              np.ascontiguousarray(opB[k0:k1]), 1.5, beta, cur)
        cur = part.astype(np.float32)
        assert np.array_equal(part, cur.astype(np.float64))
    assert np.array_equal(full, cur.astype(np.float64))


def check_alpha_beta_special(orc):
    """beta == 0 never reads C0 (NaN there stays out of the result);
    alpha == 0 never reads A, B (C = beta * C0)."""
    opA = inputs.uniform((5, 4), 14)
    opB = inputs.uniform((4, 3), 15)
    nan_c = np.full((5, 3), np.nan, np.float32)
    C, _, _ = orc.gemm(opA, opB, 1.0, 0.0, nan_c)
    assert np.all(np.isfinite(C))
    C0 = inputs.uniform((5, 3), 16)
    C, D, _ = orc.gemm(np.full((5, 4), np.nan, np.float32),
                       np.full((4, 3), np.nan, np.float32), 0.0, 0.5, C0)
    assert np.array_equal(C, 0.5 * C0.astype(np.float64))
    assert np.array_equal(D, 0.5 * np.abs(C0.astype(np.float64)))


def check_rows_subset(orc):
    """A row subset equals the same rows of the full result."""
    opA = inputs.uniform((12, 7), 17)
    opB = inputs.uniform((7, 5), 18)
    C0 = inputs.uniform((12, 5), 19)
    full, Dfull, _ = orc.gemm(opA, opB, 1.5, 0.5, C0)
    rows = [11, 0, 5, 5, 3]
    sub, Dsub, _ = orc.gemm(opA, opB, 1.5, 0.5, C0, rows=rows)
    assert np.array_equal(sub, full[rows])
    assert np.array_equal(Dsub, Dfull[rows])


def check_denominator(orc):
    """D = |alpha| |op(A)| |op(B)| + |beta| |C0| (numpy FP64 on exact
    dyadic values)."""
    opA = inputs.integers((6, 5), 20) / 2
    opB = inputs.integers((5, 4), 21) / 2
    C0 = inputs.integers((6, 4), 22)
    _, D, _ = orc.gemm(opA, opB, -1.5, -0.5, C0)
    ref = 1.5 * (np.abs(opA.astype(np.float64)) @ np.abs(opB.astype(np.float64))) \
        + 0.5 * np.abs(C0.astype(np.float64))
    assert np.array_equal(D, ref)



def check_normwise_error(orc):
    """The error measure max_ij |C - C64| / max_ij D on hand-computed cases.

    Case 1 (2 x 3): |C - C64| = [[0, 1.5, 0], [0, 0, 1]] (the larger
    deviation is negative), max D = 8, so the error is 1.5 / 8 = 0.1875;
    a mean in place of a max, an element-wise ratio (0.5), a signed
    difference (1/8), D at the worst element (1.5/4) or no denominator all
    give other values.  Row subsets take the max over their own rows only.
    The difference is formed in FP64 (a 2**-30 gap survives), a NaN in C
    gives NaN (it is within no tolerance), a zero numerator gives 0 even
    when D vanishes, and a nonzero numerator over D = 0 gives inf."""
    C = np.array([[1.0, 2.0, 3.0], [4.0, 5.0, 6.0]], np.float32)
    C64 = np.array([[1.0, 3.5, 3.0], [4.0, 5.0, 5.0]], np.float64)
    D = np.array([[2.0, 4.0, 1.0], [8.0, 3.0, 2.0]], np.float64)
    assert orc.normwise_error(C, C64, D) == 0.1875
    assert orc.normwise_error(C[[1]], C64[[1]], D[[1]]) == 1.0 / 8.0
    assert orc.normwise_error(C[[0]], C64[[0]], D[[0]]) == 1.5 / 4.0
    assert orc.normwise_error(C[:, [0, 2]], C64[:, [0, 2]], D[:, [0, 2]]) == 1.0 / 8.0
    one = np.ones((1, 1), np.float32)
    gap = np.array([[1.0 + 2.0 ** -30]])
    assert orc.normwise_error(one, gap, np.ones((1, 1))) == 2.0 ** -30
    nan_c = C.copy()
    nan_c[0, 0] = np.nan
    assert np.isnan(orc.normwise_error(nan_c, C64, D))
    assert orc.normwise_error(C, C.astype(np.float64), np.zeros((2, 3))) == 0.0
    assert orc.normwise_error(C, C64, np.zeros((2, 3))) == float("inf")
    empty = np.zeros((0, 3))
    assert orc.normwise_error(empty.astype(np.float32), empty, empty) == 0.0


def _edge_values():
    bits = np.array([
        0x00000000, 0x80000000, 0x3f800000, 0xbf800000,   # +-0, +-1
        0x3f808000, 0x3f818000, 0x3f808001, 0x3f817fff,   # ties (even/odd), above/below
        0x7f7fffff, 0xff7fffff, 0x7f7f7fff, 0x7f7f8000,   # near the top of the range
        0x00000001, 0x00400000, 0x80008000, 0x00018000,   # denormals, denormal ties
        0x7f800000, 0xff800000,                           # infinities
        0x3eaaaaab, 0x40490fdb, 0xc2c80000, 0x33800000,
    ], dtype=np.uint32)
    return bits.view(np.float32)


def check_split_vs_library(orc):
    """hi matches torch's CPU float->bfloat16 conversion (round to nearest
    even), and lo matches the same conversion applied to x - hi."""
    import torch

    x = np.concatenate([_edge_values(), inputs.uniform((4096,), 23),
                        inputs.log_uniform((4096,), 24, -130.0, 127.0),
                        inputs.normal((4096,), 25, 1e-3)]).astype(np.float32)
    hi, lo = orc.split_bf16(x)
    t_hi = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(hi, t_hi)
    hv = orc.bf16_bits_to_f32(hi).astype(np.float64)
    fin = np.isfinite(hv)
    r = (x.astype(np.float64)[fin] - hv[fin]).astype(np.float32)
    t_lo = torch.from_numpy(r).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(lo[fin], t_lo)
    assert np.all(lo[~fin] == 0)


def check_split_invariants(orc):
    """|x - (hi + lo)| <= 2**-16 |x|; x - hi is exact in FP32; integers
    below 2**16 split exactly; NaN stays NaN."""
    x = np.concatenate([inputs.uniform((20000,), 26),
                        inputs.log_uniform((20000,), 27, -100.0, 100.0)]).astype(np.float32)
    hi, lo = orc.split_bf16(x)
    h = orc.bf16_bits_to_f32(hi).astype(np.float64)
    l = orc.bf16_bits_to_f32(lo).astype(np.float64)
    xd = x.astype(np.float64)
    assert np.all(np.abs(xd - (h + l)) <= 2.0 ** -16 * np.abs(xd))
    assert np.all(np.abs(xd - h) <= 2.0 ** -8 * np.abs(xd))
    r = xd - h
    assert np.array_equal(r.astype(np.float32).astype(np.float64), r)
    ints = np.arange(-65535, 65536, 7, dtype=np.float32)
    hi, lo = orc.split_bf16(ints)
    assert np.array_equal(orc.bf16_bits_to_f32(hi).astype(np.float64)
                          + orc.bf16_bits_to_f32(lo), ints.astype(np.float64))
    hi, lo = orc.split_bf16(np.array([np.nan], np.float32))
    assert np.isnan(orc.bf16_bits_to_f32(hi)[0])


def _torch_split(x):
    import torch

    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32))
    h = t.to(torch.bfloat16).to(torch.float64)
    l = (t.to(torch.float64) - h).to(torch.float32).to(torch.bfloat16).to(torch.float64)
    return h.numpy(), l.numpy()


def check_split_terms_brute_force(orc):
    """Each selected cross product of the split parts, against exact
    rational sums of torch-split operands, for every transpose combination."""
    M, N, K = 4, 6, 5
    opA = inputs.uniform((M, K), 28)
    opB = inputs.log_uniform((K, N), 29, -4.0, 4.0)
    C0 = inputs.uniform((M, N), 30)
    ah, al = _torch_split(opA)
    bh, bl = _torch_split(opB)
    parts = {1: (ah, bh), 2: (ah, bl), 4: (al, bh), 8: (al, bl)}
    for terms, (tA, tB) in product([1, 2, 4, 8, 7, 15], TRANS):
        C = orc.gemm_split_terms(_stored(opA, tA), _stored(opB, tB), terms, 1.5, 0.5, C0,
                                 transA=tA, transB=tB)
        for i, j in product(range(M), range(N)):
            s = Fraction(0)
            mag = Fraction(0)
            for bit, (pa, pb) in parts.items():
                if terms & bit:
                    for k in range(K):
                        v = Fraction(float(pa[i, k])) * Fraction(float(pb[k, j]))
                        s += v
                        mag += abs(v)
            ex = Fraction(1.5) * s + Fraction(0.5) * Fraction(float(C0[i, j]))
            bound = Fraction(2.0 * (4 * K + 3) * 2.0 ** -53) * (Fraction(1.5) * mag
                                                                 + abs(Fraction(float(C0[i, j]))))
            assert abs(Fraction(float(C[i, j])) - ex) <= bound, (terms, tA, tB, i, j)


def check_split_terms_reduce(orc):
    """Special cases: on BF16-representable operands the hi.hi term alone is
    the plain GEMM; when hi + lo == x exactly (integers below 2**16) all four
    terms together are the plain GEMM."""
    opA, _ = inputs.bf16_values(inputs.uniform((9, 20), 31))
    opB, _ = inputs.bf16_values(inputs.uniform((20, 7), 32))
    plain, _, _ = orc.gemm(opA, opB)
    assert np.array_equal(orc.gemm_split_terms(opA, opB, 1), plain)
    iA = inputs.integers((9, 20), 33, -3000, 3000)
    iB = inputs.integers((20, 7), 34, -3000, 3000)
    plain, _, _ = orc.gemm(iA, iB)
    assert np.array_equal(orc.gemm_split_terms(iA, iB, 15), plain)


# ------------------------------------------------------------------ SYR2K
# Section 5.1: one triangle of C <- alpha (opA opB^T + opB opA^T) + beta C,
# opX = X (stored N x K) or X^T (stored K x N); the other triangle is not
# part of the update.

UPLOS = ["lower", "upper"]


def _inside(i, j, uplo):
    return j <= i if uplo == "lower" else j >= i


def _syr2k_exact(opA, opB, alpha, beta, C0, uplo, parts=None):
    """Exact rational triangle (dict (i, j) -> (C, D)); with ``parts`` the
    products are sums over (x-part of row i, y-part of row j) pairs."""
    N, K = opA.shape
    fa, fb = Fraction(float(alpha)), Fraction(float(beta))
    out = {}
    for i, j in product(range(N), range(N)):
        if not _inside(i, j, uplo):
            continue
        s = Fraction(0)
        m = Fraction(0)
        for x, y in ((opA, opB), (opB, opA)):
            for p in range(K):
                xv, yv = Fraction(float(x[i, p])), Fraction(float(y[j, p]))
                m += abs(xv) * abs(yv)
                if parts is None:
                    s += xv * yv
                else:
                    for px, py in parts(x is opA):
                        s += Fraction(float(px[i, p])) * Fraction(float(py[j, p]))
        c = fa * s
        d = abs(fa) * m
        if beta != 0.0:
            c0 = Fraction(float(C0[i, j]))
            c += fb * c0
            d += abs(fb) * abs(c0)
        out[i, j] = (c, d)
    return out


def _check_outside(C64, D, C0, uplo):
    N = C64.shape[0]
    for i, j in product(range(N), range(N)):
        if not _inside(i, j, uplo):
            assert C64[i, j] == C0[i, j] and D[i, j] == 0.0, ("outside", i, j)


def check_syr2k_brute_force(orc):
    """Exact rational sums on tiny shapes, both triangles, both trans, several
    alpha/beta; entries outside the triangle are C0 with zero denominator."""
    for (N, K), uplo, trans, (alpha, beta) in product(
            [(1, 1), (4, 3), (6, 5), (9, 2)], UPLOS, [False, True],
            [(1.0, 0.0), (1.5, 0.5), (-0.75, 2.0)]):
        opA = inputs.uniform((N, K), 61)
        opB = inputs.log_uniform((N, K), 62, -3.0, 3.0)
        C0 = inputs.uniform((N, N), 63)
        C64, D, _ = orc.syr2k(_stored(opA, trans), _stored(opB, trans), alpha, beta, C0,
                              uplo=uplo, trans=trans)
        u = 2.0 ** -53
        for (i, j), (c, d) in _syr2k_exact(opA, opB, alpha, beta, C0, uplo).items():
            bound = Fraction(2.0 * (2 * K + 3) * u * float(d))
            assert abs(Fraction(float(C64[i, j])) - c) <= bound, ("C", N, K, uplo, trans, i, j)
            assert abs(Fraction(float(D[i, j])) - d) <= bound, ("D", N, K, uplo, trans, i, j)
        _check_outside(C64, D, C0, uplo)


def check_syr2k_vs_library(orc):
    """The triangle of numpy's FP64 alpha (A B^T + B A^T) + beta C0."""
    N, K = 37, 23
    opA = inputs.uniform((N, K), 64)
    opB = inputs.uniform((N, K), 65)
    C0 = inputs.uniform((N, N), 66)
    a, b = opA.astype(np.float64), opB.astype(np.float64)
    ref = 1.5 * (a @ b.T + b @ a.T) + 0.5 * C0.astype(np.float64)
    den = 1.5 * (np.abs(a) @ np.abs(b).T + np.abs(b) @ np.abs(a).T) + 0.5 * np.abs(C0)
    for uplo, trans in product(UPLOS, [False, True]):
        C64, D, _ = orc.syr2k(_stored(opA, trans), _stored(opB, trans), 1.5, 0.5, C0,
                              uplo=uplo, trans=trans)
        mask = np.tril(np.ones((N, N), bool)) if uplo == "lower" else np.triu(np.ones((N, N), bool))
        assert np.max(np.abs(C64 - ref)[mask] / den[mask]) <= 1e-14
        assert np.max(np.abs(D - den)[mask] / den[mask]) <= 1e-14
        _check_outside(C64, D, C0, uplo)


def check_syr2k_integers(orc):
    """Integer data (every FP64 sum exact): A B^T + B A^T against numpy int64,
    and B = A giving the rank-k closed form 2 A A^T."""
    N, K = 20, 30
    iA = inputs.integers((N, K), 67)
    iB = inputs.integers((N, K), 68)
    C0 = inputs.integers((N, N), 69)
    a, b, c0 = iA.astype(np.int64), iB.astype(np.int64), C0.astype(np.int64)
    for uplo, trans in product(UPLOS, [False, True]):
        mask = np.tril(np.ones((N, N), bool)) if uplo == "lower" else np.triu(np.ones((N, N), bool))
        C64, _, _ = orc.syr2k(_stored(iA, trans), _stored(iB, trans), 1.0, 1.0, C0, uplo=uplo,
                              trans=trans)
        assert np.array_equal(C64[mask], (a @ b.T + b @ a.T + c0)[mask].astype(np.float64))
        C64, _, _ = orc.syr2k(_stored(iA, trans), _stored(iA, trans), 1.0, 0.0, uplo=uplo,
                              trans=trans)
        assert np.array_equal(C64[mask], (2 * (a @ a.T))[mask].astype(np.float64))


def check_syr2k_symmetry(orc):
    """With symmetric C0, the upper triangle is the transpose of the lower
    one, bit for bit (each entry sums the same pairs in the same order)."""
    N, K = 15, 40
    opA = inputs.uniform((N, K), 70)
    opB = inputs.log_uniform((N, K), 71)
    S = inputs.uniform((N, N), 72)
    C0 = np.ascontiguousarray(np.tril(S) + np.tril(S, -1).T)
    for trans in (False, True):
        lo, _, _ = orc.syr2k(_stored(opA, trans), _stored(opB, trans), 1.5, 0.5, C0,
                             uplo="lower", trans=trans)
        up, _, _ = orc.syr2k(_stored(opA, trans), _stored(opB, trans), 1.5, 0.5, C0,
                             uplo="upper", trans=trans)
        assert np.array_equal(np.tril(lo), np.tril(up.T))


def check_syr2k_special(orc):
    """beta == 0 never reads C0 inside the triangle (NaN there stays out);
    alpha == 0 and K == 0 give beta C0 exactly; row subsets are rows."""
    N, K = 11, 7
    opA = inputs.uniform((N, K), 73)
    opB = inputs.uniform((N, K), 74)
    C0 = inputs.uniform((N, N), 75)
    nanC = C0.copy()
    nanC[np.tril_indices(N)] = np.nan
    C64, _, _ = orc.syr2k(opA, opB, 1.0, 0.0, nanC, uplo="lower")
    assert np.all(np.isfinite(np.tril(C64)))
    assert np.array_equal(np.triu(C64, 1), np.triu(C0, 1).astype(np.float64))
    nanA = np.full((N, K), np.nan, np.float32)
    for uplo in UPLOS:
        mask = np.tril(np.ones((N, N), bool)) if uplo == "lower" else np.triu(np.ones((N, N), bool))
        C64, _, _ = orc.syr2k(nanA, nanA, 0.0, 0.5, C0, uplo=uplo)
        assert np.array_equal(C64[mask], (0.5 * C0.astype(np.float64))[mask])
        C64, _, _ = orc.syr2k(np.zeros((N, 0), np.float32), np.zeros((N, 0), np.float32), 1.0,
                              0.25, C0, uplo=uplo)
        assert np.array_equal(C64[mask], (0.25 * C0.astype(np.float64))[mask])
        full, Df, _ = orc.syr2k(opA, opB, 1.5, 0.5, C0, uplo=uplo)
        rows = np.array([10, 0, 4, 4])
        sub, Ds, _ = orc.syr2k(opA, opB, 1.5, 0.5, C0, uplo=uplo, rows=rows)
        assert np.array_equal(sub, full[rows]) and np.array_equal(Ds, Df[rows])


def check_syr2k_split_terms(orc):
    """Split products: each selection of cross products against exact rational
    sums of torch-split operands (x in the A role: opA in the first product,
    opB in the second)."""
    N, K = 5, 4
    opA = inputs.uniform((N, K), 76)
    opB = inputs.log_uniform((N, K), 77, -4.0, 4.0)
    C0 = inputs.uniform((N, N), 78)
    ah, al = _torch_split(opA)
    bh, bl = _torch_split(opB)
    for terms, uplo, trans in product([1, 2, 4, 7, 15], UPLOS, [False, True]):
        def parts(first, terms=terms):
            xh, xl, yh, yl = (ah, al, bh, bl) if first else (bh, bl, ah, al)
            sel = {1: (xh, yh), 2: (xh, yl), 4: (xl, yh), 8: (xl, yl)}
            return [v for bit, v in sel.items() if terms & bit]
        C64, _, _ = orc.syr2k(_stored(opA, trans), _stored(opB, trans), 1.5, 0.5, C0,
                              uplo=uplo, trans=trans, terms=terms)
        for (i, j), (c, d) in _syr2k_exact(opA, opB, 1.5, 0.5, C0, uplo, parts).items():
            bound = Fraction(2.0 * (8 * K + 3) * 2.0 ** -53) * d
            assert abs(Fraction(float(C64[i, j])) - c) <= bound, (terms, uplo, trans, i, j)


ALL_CHECKS = [check_brute_force, check_identity, check_permutation, check_all_ones,
              check_integers, check_transpose_identity, check_blocked_k,
              check_alpha_beta_special, check_rows_subset, check_denominator,
              check_normwise_error,
              check_split_vs_library, check_split_invariants,
              check_split_terms_brute_force, check_split_terms_reduce,
              check_syr2k_brute_force, check_syr2k_vs_library, check_syr2k_integers,
              check_syr2k_symmetry, check_syr2k_special, check_syr2k_split_terms]
