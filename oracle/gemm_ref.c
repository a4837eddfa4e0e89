/*
 * FP64 reference GEMM and BF16 split -- TEST INFRASTRUCTURE ONLY.
 *
 * This file is the correctness oracle for the GPU library.  It is plain,
 * slow and meant to be read against the paper, not to be fast.  Only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark may
 * load it; the GPU library never links, includes or calls anything here, and
 * nothing here includes a header of the GPU library.
 *
 * What is computed (Kuzma et al., "Fast Matrix Multiplication via
 * Compiler-only Layered Data Reorganization and Intrinsic Lowering",
 * Section 3, Algorithm 1):
 *
 *     C <- alpha * op(A) * op(B) + beta * C0
 *
 * Algorithm 1 computes exactly this: the K dimension is walked in blocks,
 * beta scales the C tile once (on the first K block) and alpha scales every
 * block's accumulated product before it is added.  By distributivity that
 * equals alpha times the full sum plus beta times C0, so the oracle is the
 * definition written as a triple loop, accumulating in FP64 in increasing k.
 *
 * Storage is row-major.  op(X) = X when trans == 0 and X^T when trans == 1;
 * "ld" is the distance in elements between consecutive stored rows.
 * Readings where the paper is silent:
 *   - beta == 0: C0 is not read (so NaN/Inf in C0 does not reach the result);
 *   - alpha == 0: A and B are not read; the result is beta * C0.
 *
 * The split used by the split-precision tensor-core mode is not in the
 * paper.  Its definition here: hi = bf16_rne(x), lo = bf16_rne(x - hi),
 * where bf16_rne keeps the top 16 bits of the IEEE binary32 pattern,
 * rounding the dropped 16 bits to nearest with ties to even; for
 * non-finite hi, lo = 0.
 *
 * The file also holds the SYR2K update of Section 5.1 (oracle_syr2k, at
 * the end), written out from its definition in the same way.
 *
 * Parity of every function here is pinned by the CPU tests against brute
 * force in exact rational arithmetic, closed forms and library routines.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Element (r, c) of op(X), X stored row-major with row stride ld. */
static double op_at(const float *X, int64_t ld, int trans, int64_t r, int64_t c)
{
    return trans ? (double)X[c * ld + r] : (double)X[r * ld + c];
}

/*
 * oracle_gemm: C64 = alpha * sum_k op(A)[i][k] * op(B)[k][j] + beta * C0[i][j]
 * and the error denominator D = |alpha| * sum_k |op(A)[i][k]| |op(B)[k][j]|
 * + |beta| |C0[i][j]|, both in FP64, for the requested rows.
 *
 * rows/nrows: the output rows to evaluate (rows == NULL: all M rows, in
 * order).  C64 and D (D may be NULL) are nrows x N, row-major, dense.
 * C0 may be NULL when beta == 0.  nthreads <= 0 uses the OpenMP default.
 * Returns the number of threads used.
 */
int oracle_gemm(int transA, int transB, int64_t M, int64_t N, int64_t K,
                double alpha, const float *A, int64_t lda,
                const float *B, int64_t ldb,
                double beta, const float *C0, int64_t ldc0,
                const int64_t *rows, int64_t nrows,
                double *C64, double *D, int nthreads)
{
    int used = 1;
    if (rows == NULL)
        nrows = M;
#ifdef _OPENMP
    if (nthreads <= 0)
        nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
    {
#pragma omp single
        used = omp_get_num_threads();
#else
    (void)nthreads;
    {
#endif
        double *acc = (double *)calloc((size_t)(N > 0 ? N : 1), sizeof(double));
        double *mag = (double *)calloc((size_t)(N > 0 ? N : 1), sizeof(double));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t r = 0; r < nrows; ++r) {
            int64_t i = rows ? rows[r] : r;
            for (int64_t j = 0; j < N; ++j) {
                acc[j] = 0.0;
                mag[j] = 0.0;
            }
            if (alpha != 0.0) {
                for (int64_t k = 0; k < K; ++k) {
                    double a = op_at(A, lda, transA, i, k);
                    for (int64_t j = 0; j < N; ++j) {
                        double b = op_at(B, ldb, transB, k, j);
                        acc[j] += a * b;
                        mag[j] += fabs(a) * fabs(b);
                    }
                }
            }
            for (int64_t j = 0; j < N; ++j) {
                double c = alpha * acc[j];
                double d = fabs(alpha) * mag[j];
                if (beta != 0.0) {
                    double c0 = (double)C0[i * ldc0 + j];
                    c += beta * c0;
                    d += fabs(beta) * fabs(c0);
                }
                C64[r * N + j] = c;
                if (D)
                    D[r * N + j] = d;
            }
        }
        free(acc);
        free(mag);
    }
    return used;
}

/* IEEE binary32 -> bfloat16 bit pattern, round to nearest, ties to even. */
uint16_t oracle_bf16_rne(float x)
{
    uint32_t u;
    memcpy(&u, &x, sizeof u);
    if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x007fffffu) != 0u)
        return (uint16_t)((u >> 16) | 0x0040u); /* NaN stays a (quiet) NaN */
    uint32_t upper = u >> 16;
    uint32_t dropped = u & 0xffffu;
    if (dropped > 0x8000u || (dropped == 0x8000u && (upper & 1u)))
        upper += 1u; /* a carry into the exponent is the correct rounding */
    return (uint16_t)upper;
}

float oracle_bf16_to_float(uint16_t h)
{
    uint32_t u = (uint32_t)h << 16;
    float f;
    memcpy(&f, &u, sizeof f);
    return f;
}

/* hi = bf16(x), lo = bf16(x - hi); lo = 0 when hi is not finite. */
void oracle_split(const float *x, int64_t n, uint16_t *hi, uint16_t *lo)
{
    for (int64_t t = 0; t < n; ++t) {
        uint16_t h = oracle_bf16_rne(x[t]);
        double hv = (double)oracle_bf16_to_float(h);
        uint16_t l = 0;
        if (isfinite(hv))
            l = oracle_bf16_rne((float)((double)x[t] - hv));
        hi[t] = h;
        lo[t] = l;
    }
}

/*
 * The split-product GEMM in FP64: the product op(A) op(B) replaced by the
 * sum of the selected cross products of the split parts,
 *   terms bit 0: Ahi*Bhi, bit 1: Ahi*Blo, bit 2: Alo*Bhi, bit 3: Alo*Blo,
 * then alpha and beta as in oracle_gemm.  terms == 1 is the plain BF16 mode
 * applied to FP32 inputs; terms == 7 is the three-product compensated mode.
 * The difference to the tensor-core result is then only FP32 accumulation.
 */
int oracle_gemm_split_terms(int transA, int transB, int64_t M, int64_t N, int64_t K,
                            double alpha, const float *A, int64_t lda,
                            const float *B, int64_t ldb,
                            double beta, const float *C0, int64_t ldc0,
                            int terms, const int64_t *rows, int64_t nrows,
                            double *C64, int nthreads)
{
    int used = 1;
    if (rows == NULL)
        nrows = M;
    /* split op(B) once: K x N of (hi, lo) in double */
    double *bh = (double *)malloc((size_t)(K * N > 0 ? K * N : 1) * sizeof(double));
    double *bl = (double *)malloc((size_t)(K * N > 0 ? K * N : 1) * sizeof(double));
    for (int64_t k = 0; k < K; ++k)
        for (int64_t j = 0; j < N; ++j) {
            float x = (float)op_at(B, ldb, transB, k, j);
            uint16_t h, l;
            oracle_split(&x, 1, &h, &l);
            bh[k * N + j] = (double)oracle_bf16_to_float(h);
            bl[k * N + j] = (double)oracle_bf16_to_float(l);
        }
#ifdef _OPENMP
    if (nthreads <= 0)
        nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
    {
#pragma omp single
        used = omp_get_num_threads();
#else
    (void)nthreads;
    {
#endif
        double *acc = (double *)calloc((size_t)(N > 0 ? N : 1), sizeof(double));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t r = 0; r < nrows; ++r) {
            int64_t i = rows ? rows[r] : r;
            for (int64_t j = 0; j < N; ++j)
                acc[j] = 0.0;
            if (alpha != 0.0) {
                for (int64_t k = 0; k < K; ++k) {
                    float x = (float)op_at(A, lda, transA, i, k);
                    uint16_t h, l;
                    oracle_split(&x, 1, &h, &l);
                    double ah = (double)oracle_bf16_to_float(h);
                    double al = (double)oracle_bf16_to_float(l);
                    for (int64_t j = 0; j < N; ++j) {
                        double s = 0.0;
                        if (terms & 1) s += ah * bh[k * N + j];
                        if (terms & 2) s += ah * bl[k * N + j];
                        if (terms & 4) s += al * bh[k * N + j];
                        if (terms & 8) s += al * bl[k * N + j];
                        acc[j] += s;
                    }
                }
            }
            for (int64_t j = 0; j < N; ++j) {
                double c = alpha * acc[j];
                if (beta != 0.0)
                    c += beta * (double)C0[i * ldc0 + j];
                C64[r * N + j] = c;
            }
        }
        free(acc);
    }
    free(bh);
    free(bl);
    return used;
}

/*
 * SYR2K, the rank-2k update used as the example of Section 5.1 (macro-level
 * strategy for other BLAS kernels): one triangle of the symmetric C,
 *
 *   C64[i][j] = alpha * sum_p ( opA[i][p] opB[j][p] + opB[i][p] opA[j][p] )
 *             + beta * C0[i][j]
 *
 * for (i, j) in the triangle -- uplo 0: j <= i (lower), uplo 1: j >= i
 * (upper), diagonal included -- where opX is X (stored N x K, trans == 0)
 * or X^T (X stored K x N, trans == 1).  That is C <- alpha (A B^T + B A^T)
 * + beta C, or alpha (A^T B + B^T A) + beta C, the two GEMM updates of each
 * block that Section 5.1 describes.  Both products of one p are summed
 * first and then accumulated in increasing p, so C64[i][j] of the lower
 * triangle equals C64[j][i] of the upper one bit for bit.
 *
 * Entries outside the triangle are not part of the update: C64 holds C0
 * there (0 when C0 is NULL) and D holds 0.  Same readings as oracle_gemm:
 * beta == 0 does not read C0 inside the triangle, alpha == 0 does not read
 * A or B.
 *
 * terms == 0: exact FP64 products; otherwise every product x*y is replaced
 * by the selected cross products of the BF16 split parts of x and y, with
 * the bits of oracle_gemm_split_terms (x plays the A role: opA[i] in the
 * first product, opB[i] in the second).  D is the error denominator
 * |alpha| sum_p (|opA[i][p] opB[j][p]| + |opB[i][p] opA[j][p]|) + |beta||C0|
 * from the unsplit values.  rows/nrows as in oracle_gemm; C64 and D are
 * nrows x N.
 */
static double split_product(float x, float y, int terms)
{
    uint16_t xh, xl, yh, yl;
    oracle_split(&x, 1, &xh, &xl);
    oracle_split(&y, 1, &yh, &yl);
    double ah = (double)oracle_bf16_to_float(xh), al = (double)oracle_bf16_to_float(xl);
    double bh = (double)oracle_bf16_to_float(yh), bl = (double)oracle_bf16_to_float(yl);
    double s = 0.0;
    if (terms & 1) s += ah * bh;
    if (terms & 2) s += ah * bl;
    if (terms & 4) s += al * bh;
    if (terms & 8) s += al * bl;
    return s;
}

int oracle_syr2k(int uplo, int trans, int64_t N, int64_t K, double alpha,
                 const float *A, int64_t lda, const float *B, int64_t ldb,
                 double beta, const float *C0, int64_t ldc0, int terms,
                 const int64_t *rows, int64_t nrows, double *C64, double *D,
                 int nthreads)
{
    int used = 1;
    if (rows == NULL)
        nrows = N;
#ifdef _OPENMP
    if (nthreads <= 0)
        nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#else
    (void)nthreads;
#endif
    for (int64_t r = 0; r < nrows; ++r) {
#ifdef _OPENMP
        if (r == 0)
            used = omp_get_num_threads();
#endif
        int64_t i = rows ? rows[r] : r;
        for (int64_t j = 0; j < N; ++j) {
            int inside = uplo == 0 ? (j <= i) : (j >= i);
            if (!inside) {
                C64[r * N + j] = C0 ? (double)C0[i * ldc0 + j] : 0.0;
                if (D)
                    D[r * N + j] = 0.0;
                continue;
            }
            double acc = 0.0, mag = 0.0;
            if (alpha != 0.0) {
                for (int64_t p = 0; p < K; ++p) {
                    double aip = op_at(A, lda, trans, i, p), bjp = op_at(B, ldb, trans, j, p);
                    double bip = op_at(B, ldb, trans, i, p), ajp = op_at(A, lda, trans, j, p);
                    if (terms == 0)
                        acc += aip * bjp + bip * ajp;
                    else
                        acc += split_product((float)aip, (float)bjp, terms) +
                               split_product((float)bip, (float)ajp, terms);
                    mag += fabs(aip) * fabs(bjp) + fabs(bip) * fabs(ajp);
                }
            }
            double c = alpha * acc;
            double d = fabs(alpha) * mag;
            if (beta != 0.0) {
                double c0 = (double)C0[i * ldc0 + j];
                c += beta * c0;
                d += fabs(beta) * fabs(c0);
            }
            C64[r * N + j] = c;
            if (D)
                D[r * N + j] = d;
        }
    }
    return used;
}
