// FP32 SIMT GEMM: C <- alpha * op(A) op(B) + beta * C on the CUDA cores.
//
// The "generic lowering" of Kuzma et al. (Section 3.2: llvm.matrix.multiply
// lowered to plain vector fused multiply-adds when no matrix engine is
// used), laid out for an SM instead of a CPU core:
//  * a 128 x 128 C block per CTA plays the mc x nc block of Algorithm 1 and
//    a BK = 16 slice of K plays kc;
//  * the shared-memory tiles As[k][m], Bs[k][n] are the packed ATile/BTile
//    buffers (Section 3.1: tiles stored in the order the micro kernel reads
//    them).  When both operands are stored K x rows (the form the library
//    packs large problems into) a three-stage ring filled by cp.async
//    copies stages them with no registers in flight; the other orientations
//    double-buffer them with a register prefetch of the next K slice;
//  * each thread's 8 x 8 register accumulator is the mr x nr micro tile of
//    Algorithm 2, updated by rank-1 outer products (Blackwell's packed FP32
//    FMA, two fused multiply-adds per instruction) and never spilled;
//  * remainder tiles are zero-filled on load and stored element by element
//    (Section 3.1, last paragraph), full tiles with 16-byte accesses.
// All four op(A)/op(B) combinations are handled by the load index math.
//
// SYR2K (Section 5.1, UPLO 1 = lower / 2 = upper triangle): the same kernel
// over the two GEMM updates of each C block.  The K loop runs over both
// products, A-side rows of X with B-side rows of Y and then the reverse, each
// half zero-padded to whole BK slices; blocks wholly outside the triangle
// return at once and the epilogue stores only triangle elements.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace gb300 {

namespace {

constexpr int BM = 128, BN = 128, BK = 16, PAD = 4, THREADS = 256;

struct Frag {
    float v[8];
};

// Load this thread's 8 elements of the K slice [k0, k0+BK) of op(X), where
// op(X) is R x K (R = M for A, N for B).  TRANS_K: X is stored R x K (K
// contiguous, "K-major"); otherwise X is stored K x R (R contiguous).
template <bool K_CONTIG, bool VEC>
__device__ __forceinline__ void load_slice(const float* __restrict__ X, int64_t ldx, int R, int K,
                                           int r0, int k0, bool full, Frag& f) {
    const int t = threadIdx.x;
    if (K_CONTIG) {
        // thread -> row r0 + (t & 127), k0 + (t >> 7) * 8 .. +7
        const int r = r0 + (t & 127);
        const int k = k0 + (t >> 7) * 8;
        const float* p = X + int64_t(r) * ldx + k;
        if (VEC && full) {
            const float4 a = __ldg(reinterpret_cast<const float4*>(p));
            const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
            f.v[0] = a.x; f.v[1] = a.y; f.v[2] = a.z; f.v[3] = a.w;
            f.v[4] = b.x; f.v[5] = b.y; f.v[6] = b.z; f.v[7] = b.w;
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) f.v[q] = (r < R && k + q < K) ? __ldg(p + q) : 0.0f;
        }
    } else {
        // thread -> k0 + (t >> 5) and k0 + (t >> 5) + 8, rows r0 + (t & 31) * 4 .. +3:
        // a warp reads one 512-byte row segment per instruction
        const int k = k0 + (t >> 5);
        const int r = r0 + (t & 31) * 4;
        const float* p = X + int64_t(k) * ldx + r;
        const float* p8 = p + 8 * ldx;
        if (VEC && full) {
            const float4 a = __ldg(reinterpret_cast<const float4*>(p));
            const float4 b = __ldg(reinterpret_cast<const float4*>(p8));
            f.v[0] = a.x; f.v[1] = a.y; f.v[2] = a.z; f.v[3] = a.w;
            f.v[4] = b.x; f.v[5] = b.y; f.v[6] = b.z; f.v[7] = b.w;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                f.v[q] = (k < K && r + q < R) ? __ldg(p + q) : 0.0f;
                f.v[4 + q] = (k + 8 < K && r + q < R) ? __ldg(p8 + q) : 0.0f;
            }
        }
    }
}

// 16-byte asynchronous copy global -> shared memory (no registers); bytes
// beyond `src_bytes` (0..16) are zero-filled and not read.
__device__ __forceinline__ void cp_async_16(void* smem_dst, const float* src, int src_bytes) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// The K slice [k0, k0+BK) of op(X) (R x K) for X stored K x R with 16-byte
// aligned rows, copied asynchronously into an unpadded [BK][BM] tile: thread
// t copies rows k0 + (t >> 5) and +8, elements r0 + (t & 31) * 4 .. +3, so a
// warp moves one 512-byte row segment per copy; ragged edges zero-filled.
__device__ __forceinline__ void copy_slice_async(const float* __restrict__ X, int64_t ldx, int R,
                                                 int K, int r0, int k0, float (*S)[BM]) {
    const int t = threadIdx.x;
    const int c = (t & 31) * 4;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int kk = (t >> 5) + 8 * h;
        const int gk = k0 + kk, gr = r0 + c;
        const int bytes = (gk < K && gr < R) ? min(4, R - gr) * 4 : 0;
        cp_async_16(&S[kk][c], bytes ? X + int64_t(gk) * ldx + gr : X, bytes);
    }
}

// Store the thread's 8 elements into the [BK][BM + PAD] tile (k-major rows).
template <bool K_CONTIG>
__device__ __forceinline__ void store_slice(float (*S)[BM + PAD], const Frag& f) {
    const int t = threadIdx.x;
    if (K_CONTIG) {
        const int r = t & 127, k = (t >> 7) * 8;
#pragma unroll
        for (int q = 0; q < 8; ++q) S[k + q][r] = f.v[q];
    } else {
        const int k = t >> 5, r = (t & 31) * 4;
        *reinterpret_cast<float4*>(&S[k][r]) = make_float4(f.v[0], f.v[1], f.v[2], f.v[3]);
        *reinterpret_cast<float4*>(&S[k + 8][r]) = make_float4(f.v[4], f.v[5], f.v[6], f.v[7]);
    }
}

template <bool TA, bool TB, bool VEC, int UPLO>
__global__ void __launch_bounds__(THREADS, 2)
    simt_f32_kernel(int M, int N, int K, float alpha, const float* __restrict__ A, int64_t lda,
                    const float* __restrict__ B, int64_t ldb, float beta, float* __restrict__ C,
                    int64_t ldc, int c_vec) {
    // op(A) rows are K-contiguous when A is stored M x K (no transpose);
    // op(B)^T rows (N x K) are K-contiguous when B is stored N x K (transposed).
    constexpr bool A_KC = !TA;
    constexpr bool B_KC = TB;
    // Both operands stored K x R with aligned rows (the form large problems
    // get after the pack pass): a three-stage ring filled by asynchronous
    // copies, which hold no registers.  Otherwise: two stages filled through
    // a register prefetch, transposing K-contiguous rows on the way.
    constexpr bool ASYNC = !A_KC && !B_KC && VEC;
    constexpr int STAGES = ASYNC ? 3 : 2;
    constexpr int SP = ASYNC ? 0 : PAD;  // cp.async rows need no padding
    __shared__ __align__(16) float As[STAGES][BK][BM + SP];
    __shared__ __align__(16) float Bs[STAGES][BK][BN + SP];

    const int m0 = blockIdx.y * BM;
    const int n0 = blockIdx.x * BN;
    if (UPLO == 1 && n0 > m0 + BM - 1) return;  // every column right of every row
    if (UPLO == 2 && n0 + BN - 1 < m0) return;  // every column left of every row
    const int tid = threadIdx.x;
    const int ty = tid >> 4, tx = tid & 15;
    const bool mn_full = (m0 + BM <= M) && (n0 + BN <= N);

    // acc2[i][j] holds columns 2j and 2j+1 of accumulator row i: Blackwell's
    // packed FP32 FMA (two round-to-nearest fused multiply-adds per lane and
    // instruction) halves the issue slots the rank-1 updates take, so the
    // fragment loads and loop overhead no longer compete with them.  Each
    // element sees exactly the FMA chain of the scalar form.
    float2 acc2[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc2[i][j] = make_float2(0.0f, 0.0f);

    const int nk1 = (K + BK - 1) / BK;  // slices of one product
    const int nk = UPLO ? 2 * nk1 : nk1;
    // slice kt: its K offset and the matrices feeding the A and B sides
    auto slice = [&](int kt, const float*& xa, int64_t& lxa, const float*& xb, int64_t& lxb) {
        const bool second = UPLO && kt >= nk1;
        xa = second ? B : A;
        lxa = second ? ldb : lda;
        xb = second ? A : B;
        lxb = second ? lda : ldb;
        return (second ? kt - nk1 : kt) * BK;
    };
    // one BK slice of rank-1 updates from ring stage `cur`
    auto compute = [&](int cur) {
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][k][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[cur][k][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[cur][k][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[cur][k][64 + tx * 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float2 b2[4] = {make_float2(b0.x, b0.y), make_float2(b0.z, b0.w),
                                  make_float2(b1.x, b1.y), make_float2(b1.z, b1.w)};
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float2 ai = make_float2(a[i], a[i]);
#pragma unroll
                for (int j = 0; j < 4; ++j) acc2[i][j] = __ffma2_rn(ai, b2[j], acc2[i][j]);
            }
        }
    };

    if constexpr (ASYNC) {
        auto issue = [&](int kt) {
            const float *xa, *xb;
            int64_t lxa, lxb;
            const int k0 = slice(kt, xa, lxa, xb, lxb);
            copy_slice_async(xa, lxa, M, K, m0, k0, As[kt % STAGES]);
            copy_slice_async(xb, lxb, N, K, n0, k0, Bs[kt % STAGES]);
        };
#pragma unroll
        for (int st = 0; st < STAGES - 1; ++st) {
            if (st < nk) issue(st);
            cp_async_commit();  // one group per slice, empty past the end
        }
        for (int kt = 0; kt < nk; ++kt) {
            cp_async_wait<STAGES - 2>();  // this thread's copies of slice kt landed
            __syncthreads();  // everyone's copies landed; stage of slice kt-1 is free
            if (kt + STAGES - 1 < nk) issue(kt + STAGES - 1);
            cp_async_commit();
            compute(kt % STAGES);
        }
    } else {
        Frag fa, fb;
        {
            const float *xa, *xb;
            int64_t lxa, lxb;
            const int k0 = slice(0, xa, lxa, xb, lxb);
            load_slice<A_KC, VEC>(xa, lxa, M, K, m0, k0, mn_full && BK <= K, fa);
            load_slice<B_KC, VEC>(xb, lxb, N, K, n0, k0, mn_full && BK <= K, fb);
        }
        store_slice<A_KC>(As[0], fa);
        store_slice<B_KC>(Bs[0], fb);
        __syncthreads();

        for (int kt = 0; kt < nk; ++kt) {
            const int cur = kt & 1;
            if (kt + 1 < nk) {
                const float *xa, *xb;
                int64_t lxa, lxb;
                const int k0 = slice(kt + 1, xa, lxa, xb, lxb);
                const bool full = mn_full && (k0 + BK <= K);
                load_slice<A_KC, VEC>(xa, lxa, M, K, m0, k0, full, fa);
                load_slice<B_KC, VEC>(xb, lxb, N, K, n0, k0, full, fb);
            }
            compute(cur);
            if (kt + 1 < nk) {
                store_slice<A_KC>(As[cur ^ 1], fa);
                store_slice<B_KC>(Bs[cur ^ 1], fb);
            }
            __syncthreads();
        }
    }

    // epilogue: C = alpha * acc + beta * C (C not read when beta == 0)
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int row = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        if (row >= M) continue;
        float* crow = C + int64_t(row) * ldc;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int col = n0 + (h == 0 ? tx * 4 : 64 + tx * 4);
            float o[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 pr = acc2[i][(h * 4 + j) >> 1];
                o[j] = alpha * (((h * 4 + j) & 1) ? pr.y : pr.x);
            }
            // SYR2K: the 4-wide group is wholly inside the triangle, or is
            // stored element by element
            const bool whole = UPLO == 0 || (UPLO == 1 ? col + 3 <= row : col >= row);
            if (c_vec && col + 4 <= N && whole) {
                float4* p = reinterpret_cast<float4*>(crow + col);
                if (beta != 0.0f) {
                    const float4 old = *p;
                    o[0] = fmaf(beta, old.x, o[0]);
                    o[1] = fmaf(beta, old.y, o[1]);
                    o[2] = fmaf(beta, old.z, o[2]);
                    o[3] = fmaf(beta, old.w, o[3]);
                }
                *p = make_float4(o[0], o[1], o[2], o[3]);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const bool in = UPLO == 0 || (UPLO == 1 ? col + j <= row : col + j >= row);
                    if (col + j < N && in) {
                        float v = o[j];
                        if (beta != 0.0f) v = fmaf(beta, crow[col + j], v);
                        crow[col + j] = v;
                    }
                }
            }
        }
    }
}

template <bool TA, bool TB, int UPLO = 0>
cudaError_t launch_tt(int M, int N, int K, float alpha, const float* A, int64_t lda,
                      const float* B, int64_t ldb, float beta, float* C, int64_t ldc,
                      cudaStream_t stream) {
    const bool vec = ((reinterpret_cast<uintptr_t>(A) & 15) == 0) && (lda % 4 == 0) &&
                     ((reinterpret_cast<uintptr_t>(B) & 15) == 0) && (ldb % 4 == 0);
    const int c_vec = ((reinterpret_cast<uintptr_t>(C) & 15) == 0) && (ldc % 4 == 0);
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
    if (vec)
        simt_f32_kernel<TA, TB, true, UPLO><<<grid, THREADS, 0, stream>>>(M, N, K, alpha, A, lda,
                                                                          B, ldb, beta, C, ldc,
                                                                          c_vec);
    else
        simt_f32_kernel<TA, TB, false, UPLO><<<grid, THREADS, 0, stream>>>(M, N, K, alpha, A, lda,
                                                                           B, ldb, beta, C, ldc,
                                                                           c_vec);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_simt_syr2k(int uplo, int trans, int64_t N, int64_t K, float alpha,
                              const float* X, int64_t ldx, const float* Y, int64_t ldy, float beta,
                              float* C, int64_t ldc, cudaStream_t stream) {
    if ((N + BM - 1) / BM > 65535 || N > (1ll << 31) - BM || K > (1ll << 30) - BK)
        return cudaErrorInvalidValue;
    const int n = int(N), k = int(K);
    // trans 0: X, Y stored N x K; the A side reads rows of X (K-contiguous)
    // and the B side needs X^T, i.e. rows of the stored N x K matrix again
    // (the "transposed B" load).  trans 1: X, Y stored K x N, the other way.
    if (uplo == 1)
        return trans ? launch_tt<true, false, 1>(n, n, k, alpha, X, ldx, Y, ldy, beta, C, ldc, stream)
                     : launch_tt<false, true, 1>(n, n, k, alpha, X, ldx, Y, ldy, beta, C, ldc, stream);
    return trans ? launch_tt<true, false, 2>(n, n, k, alpha, X, ldx, Y, ldy, beta, C, ldc, stream)
                 : launch_tt<false, true, 2>(n, n, k, alpha, X, ldx, Y, ldy, beta, C, ldc, stream);
}

cudaError_t launch_simt_f32(int transA, int transB, int64_t M, int64_t N, int64_t K, float alpha,
                            const float* A, int64_t lda, const float* B, int64_t ldb, float beta,
                            float* C, int64_t ldc, cudaStream_t stream) {
    if ((M + BM - 1) / BM > 65535 || M > (1ll << 31) - BM || N > (1ll << 31) - BN ||
        K > (1ll << 31) - BK)
        return cudaErrorInvalidValue;
    const int m = int(M), n = int(N), k = int(K);
    if (transA) {
        return transB ? launch_tt<true, true>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, stream)
                      : launch_tt<true, false>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, stream);
    }
    return transB ? launch_tt<false, true>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, stream)
                  : launch_tt<false, false>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, stream);
}

}  // namespace gb300
