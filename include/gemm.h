/*
 * gb300 GEMM -- C ABI of a one-GPU GEMM library for NVIDIA GB300 (sm_103a).
 *
 * Every entry point computes (a piece of) the BLAS SGEMM contract that
 * Kuzma et al., "Fast Matrix Multiplication via Compiler-only Layered Data
 * Reorganization and Intrinsic Lowering" (SPE 2023) generate code for:
 *
 *     C <- alpha * op(A) * op(B) + beta * C                     (Algorithm 1)
 *
 * Section 3 and Algorithm 1 define the operation: beta scales C once, alpha
 * scales the accumulated product, op(X) is X or X^T ("access order",
 * Section 3.2 end), ld* are the leading dimensions of the stored matrices.
 *
 * Conventions shared by all entry points
 * --------------------------------------
 * Storage is ROW-MAJOR (the paper's matrices are column-major; a column-major
 * caller computes C^T = op(B)^T op(A)^T, i.e. swaps A/B and M/N).
 *   op(A) is M x K: A is stored M x K (transA == GEMM_OP_N) or K x M (GEMM_OP_T);
 *   op(B) is K x N: B is stored K x N (transB == GEMM_OP_N) or N x K (GEMM_OP_T);
 *   C is M x N.  ld* = distance in elements between consecutive stored rows,
 *   and must be >= max(1, number of stored columns).
 * Pointers named A, B, C, X, hi, lo, ws are DEVICE pointers unless the
 * function says otherwise; the caller owns them.  `stream` is a cudaStream_t
 * passed as void* (NULL = legacy default stream); all work is enqueued on
 * it and nothing synchronises with the host unless stated.
 * Errors are BLAS-style: an invalid argument returns GEMM_ERR_ARG, records
 * its 1-based position (see gemm_last_error_arg) and launches nothing.
 * Quick returns: M == 0 or N == 0 does nothing; K == 0 or alpha == 0 gives
 * C <- beta * C without reading A or B; beta == 0 never reads C, so NaN or
 * Inf already in C does not reach the result.
 * A handle may be used by one host thread at a time.
 * Stream order: the tensor-core GEMM kernels are launched with programmatic
 * stream serialisation.  They may start setting up while the kernel before
 * them on the stream finishes, but touch no global memory until it has
 * completed.  Once a GEMM kernel has issued its operand loads it lets a
 * following kernel that was launched with the same attribute start early.
 * Such a kernel, like any dependent kernel, must wait for its prerequisite
 * (cudaGridDependencySynchronize) before it reads C; kernels launched
 * without the attribute are ordered as usual.
 */
#ifndef GB300_GEMM_H
#define GB300_GEMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { GEMM_OP_N = 0, GEMM_OP_T = 1 } gemm_op_t;

/* How op(A) op(B) is multiplied.
 *  GEMM_MODE_F32_SIMT: FP32 fused multiply-adds on the CUDA cores (the
 *    "generic lowering" of Section 3.2: plain vector FMA, no matrix engine).
 *  GEMM_MODE_BF16: A and B rounded to BF16 (round to nearest even), products
 *    on the tensor cores (tcgen05), FP32 accumulation.  The matrix-engine
 *    lowering of Section 3.2 / Algorithm 2 with 16-bit inputs (rank-2
 *    updates per element pair, Section 3.3).
 *  GEMM_MODE_BF16X3: split-precision -- x = hi + lo with hi = bf16(x),
 *    lo = bf16(x - hi); op(A) op(B) ~ Ahi Bhi + Ahi Blo + Alo Bhi on the
 *    tensor cores with FP32 accumulation, recovering FP32-level accuracy.
 *    Not in the paper. */
typedef enum {
    GEMM_MODE_F32_SIMT = 0,
    GEMM_MODE_BF16 = 1,
    GEMM_MODE_BF16X3 = 2
} gemm_mode_t;

typedef enum {
    GEMM_OK = 0,
    GEMM_ERR_ARG = -1,         /* invalid argument; position in gemm_last_error_arg */
    GEMM_ERR_ALIGN = -2,       /* a tensor-core operand is not 16-byte aligned */
    GEMM_ERR_WORKSPACE = -3,   /* caller workspace too small / allocation failed */
    GEMM_ERR_CUDA = -4,        /* a CUDA runtime or driver call failed */
    GEMM_ERR_TIMEOUT = -5,     /* a kernel's bounded wait expired (reported by gemm_sync) */
    GEMM_ERR_UNSUPPORTED = -6, /* valid request this build cannot serve */
    GEMM_ERR_DEVICE = -7       /* current device is not an sm_103 GPU */
} gemm_status_t;

typedef struct gemm_context *gemm_handle_t;

/* Launch configuration overrides (all 0 = library choice).
 *  bn:        tensor-core tile width in N (128 or 256; the tile height is 128,
 *             256 on CTA pairs), or 512: 256 x 512 pair tiles for plain BF16
 *             (gemm_bf16, GEMM_MODE_BF16 in gemm()) with BK 64 -- other calls
 *             use 256 -- which the library also picks for those calls when
 *             beta == 0 and the problem has a 256 x 512 tile per SM pair and
 *             K >= 8192, or K >= 2048 with B read in place as MN-major tiles;
 *             bn 512 with cta_group 1 or bk 32 is GEMM_ERR_ARG.
 *  bk:        K depth of one pipeline stage (32 or 64 BF16 elements).
 *  stages:    shared-memory ring depth (2..8; clamped to what fits).
 *  split_k:   number of K slices (1 = none), each a partial sum; the partial
 *             sums are added in slice order, then C = alpha * sum + beta * C,
 *             as splitk_reduce says.  Grouped plans choose per problem
 *             instead: a problem whose one tile carries more K blocks than a
 *             CTA's even share of the launch is cut into up to 8 slices
 *             (problems of their own, then one reduce launch for all
 *             of them), by the cost model, or by the autotuner when it times
 *             faster; split_k 1 on the handle turns this off.
 *  raster_group: number of M tiles walked together before moving along N.
 *  max_ctas:  upper bound on persistent CTAs (0 = one per SM).
 *  promote_k: GEMM_MODE_BF16X3 only: K elements summed in tensor memory
 *    before the partial sum is added into FP32 registers with round-to-
 *    nearest (0 = default 512, -1 = never; the tensor core's own FP32
 *    accumulation rounds toward zero, so long chains lose accuracy).
 *  cta_group: 1 = one CTA per 128-row tile; 2 = CTA pairs (a cluster of two
 *    SMs shares a 256-row tile, each staging half of B; bn must be 256);
 *    0 = library choice: pairs when the problem has at least as many
 *    256 x 256 tiles as the GPU has SM pairs, for GEMM_MODE_BF16X3 in
 *    gemm(), gemm_from_host and gemm_backward, and for plain BF16 (gemm_bf16,
 *    GEMM_MODE_BF16 in gemm()) when K >= 512; else one CTA per tile;
 *    gemm_syr2k always uses one CTA per tile; grouped plans and
 *    gemm_grouped on a handle that sets none of bn, bk, stages and
 *    cta_group take the tile shape, depth and grouping that an analytic cost
 *    model (padded tensor work, wave quantisation, measured per-clock
 *    efficiency) ranks first.  bk 0 = 64, or 32 for GEMM_MODE_BF16X3 with
 *    one CTA per tile.
 *  wait_poll_limit: mbarrier polls before a kernel abandons a wait, sets
 *    the device error word and exits cleanly (0 = default, about seconds).
 *  operand_layout: GEMM_LAYOUT_K_MAJOR (1): every operand is made
 *    K-contiguous first (a transposing split, or a pack pass in gemm_bf16);
 *    GEMM_LAYOUT_AS_STORED (2): each operand reaches the tensor cores in its
 *    stored orientation -- A stored K x M (transA == T) and B stored K x N
 *    (transB == N) are split without transposing and read as MN-major tiles,
 *    and gemm_bf16 reads every operand in place; GEMM_LAYOUT_AUTO (0,
 *    default): K-major in gemm(), gemm_from_host and gemm_backward (the
 *    K-major kernel is a few percent faster and the split transposes at
 *    nearly the copy rate), as stored in grouped plans and gemm_syr2k, and
 *    in gemm_bf16 K-major only when the pack pass costs under a tenth of the
 *    GEMM (large, compute-bound shapes) -- as stored otherwise.
 *  splitk_reduce: GEMM_SPLITK_AUTO (0): with one CTA per tile, 2, 4 or 8
 *    slices, no more (tile, slice) pairs than SMs and every such cluster
 *    resident at once, the slices of a tile run as one cluster of CTAs and
 *    the GEMM kernel itself adds them after a cluster barrier (no second
 *    launch); otherwise a second kernel adds them.  GEMM_SPLITK_LAUNCH (1): always
 *    the second kernel.  Both give the same bits. */
typedef enum {
    GEMM_LAYOUT_AUTO = 0,
    GEMM_LAYOUT_K_MAJOR = 1,
    GEMM_LAYOUT_AS_STORED = 2
} gemm_layout_t;

/* split_place: where GEMM_MODE_BF16X3 splits FP32 operands into hi/lo BF16
 * (the paper's packing step, Algorithm 1 / Section 3.1, with the split
 * added).
 *  GEMM_SPLIT_PREPASS (1): a bandwidth-bound pass writes the hi/lo planes to
 *    workspace before the tensor-core kernel (8 bytes of HBM traffic per
 *    element of A and B, one launch per operand).
 *  GEMM_SPLIT_IN_KERNEL (2): the tensor-core kernel reads the caller's FP32
 *    A and B through TMA and splits each staged tile in shared memory
 *    (converter warps), bit-identical to the pass; no split workspace.  It
 *    runs one CTA per 128 x 256 tile with BK 32 (bn 0 or 256, bk 0 or 32,
 *    cta_group 0 or 1, else GEMM_ERR_ARG).  An operand TMA cannot read in
 *    place (base not 16-byte aligned, or ld not a multiple of 4) is split by
 *    the pass instead.  gemm() and grouped plans only (gemm_from_host,
 *    gemm_syr2k use the pass).
 *  GEMM_SPLIT_IN_KERNEL_A (3), GEMM_SPLIT_IN_KERNEL_B (4): the same kernel,
 *    but only A (only B) is split in the kernel; the pass splits the other.
 *    The same tile-shape rules; gemm() only (grouped plans: GEMM_ERR_ARG).
 *    The results equal those of the other placements bit for bit.
 *  GEMM_SPLIT_AUTO (0): when the handle forces no tile shape or layout,
 *    gemm() picks per operand by a cost model: an operand the kernel would
 *    re-split in many tiles (A when N spans many 256-wide tiles, B when M
 *    spans many 128-high tiles) goes to the pass, a large one staged by few
 *    tiles to the kernel, and nothing to the kernel when the pass plus the
 *    CTA-pair kernel is faster (large problems).  Grouped plans take the
 *    faster of the split pass and the in-kernel split of both operands by
 *    the cost model or the autotuner. */
typedef enum {
    GEMM_SPLIT_AUTO = 0,
    GEMM_SPLIT_PREPASS = 1,
    GEMM_SPLIT_IN_KERNEL = 2,
    GEMM_SPLIT_IN_KERNEL_A = 3,
    GEMM_SPLIT_IN_KERNEL_B = 4
} gemm_split_place_t;

typedef enum {
    GEMM_SPLITK_AUTO = 0,
    GEMM_SPLITK_LAUNCH = 1
} gemm_splitk_reduce_t;

typedef struct {
    int32_t bn;
    int32_t bk;
    int32_t stages;
    int32_t split_k;
    int32_t raster_group;
    int32_t max_ctas;
    int32_t promote_k;
    int32_t cta_group;
    int64_t wait_poll_limit;
    int32_t operand_layout;
    int32_t split_place;   /* gemm_split_place_t */
    int32_t splitk_reduce; /* gemm_splitk_reduce_t */
} gemm_config_t;

/* Create a handle bound to the CURRENT CUDA device.  Allocates a 256-byte
 * device error word.  Returns GEMM_ERR_DEVICE if the device is not sm_103,
 * GEMM_ERR_ARG (arg 1) if handle is NULL. */
gemm_status_t gemm_create(gemm_handle_t *handle);

/* Free the handle, its error word and any workspace it allocated itself.
 * Synchronises the device first.  NULL is accepted. */
gemm_status_t gemm_destroy(gemm_handle_t handle);

/* Override (cfg != NULL) or reset (cfg == NULL) the launch configuration.
 * Invalid fields give GEMM_ERR_ARG with position 2. */
gemm_status_t gemm_set_config(gemm_handle_t handle, const gemm_config_t *cfg);

/* Bytes of device workspace gemm() needs for this problem and mode with the
 * handle's current configuration.  Workspace holds the BF16 split/packed
 * operands (Algorithm 1's APack/BPack buffers) and split-K partial sums; for
 * GEMM_MODE_F32_SIMT, the FP32 operands packed for the SIMT kernel when
 * M*N*K >= 2^30 (room for both operands whatever the transposes; 0 below
 * that size).  Returns 0 for invalid arguments. */
size_t gemm_workspace_size(gemm_handle_t handle, gemm_mode_t mode, gemm_op_t transA,
                           gemm_op_t transB, int64_t M, int64_t N, int64_t K);

/* Give the handle caller-owned device workspace (256-byte aligned, or
 * GEMM_ERR_ALIGN).  The caller keeps ownership and must keep it alive until
 * the work using it has finished on the stream.  ws == NULL returns to the
 * handle's own workspace, which it grows with cudaMalloc on demand. */
gemm_status_t gemm_set_workspace(gemm_handle_t handle, void *ws, size_t bytes);

/* C <- alpha * op(A) op(B) + beta * C, FP32 in and out, device pointers,
 * computed as `mode` says.  Argument positions for GEMM_ERR_ARG:
 * 1 handle, 2 transA, 3 transB, 4 M, 5 N, 6 K, 7 alpha, 8 A, 9 lda, 10 B,
 * 11 ldb, 12 beta, 13 C, 14 ldc, 15 mode, 16 stream.
 * A, B, C may have any 4-byte alignment and any valid ld.
 * With a tensor-core mode and no caller workspace, the first call of a new
 * largest size allocates (cudaMalloc) and is therefore not graph-capturable.
 * GEMM_MODE_F32_SIMT with M*N*K >= 2^30 first transposes each operand stored
 * K-contiguous (A with transA == N, B with transB == T) into workspace, the
 * layout its kernel reads fastest; with a caller workspace smaller than
 * gemm_workspace_size, or no memory for one, it reads them as stored. */
gemm_status_t gemm(gemm_handle_t handle, gemm_op_t transA, gemm_op_t transB,
                   int64_t M, int64_t N, int64_t K,
                   float alpha, const float *A, int64_t lda,
                   const float *B, int64_t ldb,
                   float beta, float *C, int64_t ldc,
                   gemm_mode_t mode, void *stream);

/* C <- alpha * op(A) op(B) + beta * C with BF16 A and B (uint16_t bit
 * patterns), FP32 C, tensor cores with FP32 accumulation.  K-contiguous
 * operands (A stored M x K, B stored N x K) are always read in place by TMA
 * and need a 16-byte aligned base and ld % 8 == 0 (else GEMM_ERR_ALIGN).
 * MN-contiguous ones (A stored K x M, B stored K x N) are either read in
 * place as MN-major tiles (same alignment rule) or first packed K-contiguous
 * into workspace (Algorithm 1's pack step; any ld), as operand_layout says
 * (library choice: packed when the pass costs under a tenth of the GEMM or
 * when the operand cannot be read in place).  Argument positions as for gemm() (no mode; 15 is stream). */
gemm_status_t gemm_bf16(gemm_handle_t handle, gemm_op_t transA, gemm_op_t transB,
                        int64_t M, int64_t N, int64_t K,
                        float alpha, const uint16_t *A, int64_t lda,
                        const uint16_t *B, int64_t ldb,
                        float beta, float *C, int64_t ldc, void *stream);

/* The split step on its own: Y = op(X) (rows x cols, X stored row-major
 * with row stride ldx, op as `trans`), written as hi = bf16_rne(Y) and
 * lo = bf16_rne(Y - hi) (lo = 0 where hi is not finite) with row stride
 * ldo elements.  lo may be NULL (hi only).  hi and lo must be 16-byte
 * aligned and ldo % 8 == 0 (GEMM_ERR_ALIGN).  Positions: 1 handle,
 * 2 trans, 3 rows, 4 cols, 5 X, 6 ldx, 7 hi, 8 lo, 9 ldo, 10 stream. */
gemm_status_t gemm_split_bf16(gemm_handle_t handle, gemm_op_t trans, int64_t rows, int64_t cols,
                              const float *X, int64_t ldx, uint16_t *hi, uint16_t *lo,
                              int64_t ldo, void *stream);

/* gemm() on HOST buffers: copies A, B (and C when beta != 0) to device
 * buffers the handle owns (grown with cudaMalloc on demand), computes, copies
 * C back and synchronises `stream`.  A three-stream pipeline the handle owns
 * runs over up to sixteen row blocks of op(A) and C (of at least 512 rows):
 * one stream copies B and then every block's A and C rows in back to back,
 * one splits and multiplies each block as its rows arrive, one copies each
 * block's C out as soon as it is done, so the host link stays busy in both
 * directions.  Pinned host memory gives asynchronous, overlapped copies;
 * pageable memory works but is slower.  Also reports a kernel's
 * bounded-wait expiry (GEMM_ERR_TIMEOUT).  Positions as for gemm(). */
gemm_status_t gemm_from_host(gemm_handle_t handle, gemm_op_t transA, gemm_op_t transB,
                             int64_t M, int64_t N, int64_t K,
                             float alpha, const float *A, int64_t lda,
                             const float *B, int64_t ldb,
                             float beta, float *C, int64_t ldc,
                             gemm_mode_t mode, void *stream);

/* One problem of a grouped call: C_g <- alpha_g op(A_g) op(B_g) + beta_g C_g. */
typedef struct {
    int64_t M, N, K;
    int64_t lda, ldb, ldc;
    const float *A;
    const float *B;
    float *C;
    float alpha, beta;
    int32_t transA, transB; /* gemm_op_t values */
} gemm_problem_t;

/* Many independent FP32 GEMMs in one call: one split launch for all
 * operands plus one persistent tensor-core launch over the concatenated
 * output tiles of all problems.  host_problems (HOST memory, `count`
 * entries) describe the problems; their pointers are device pointers.
 * GEMM_MODE_BF16 and GEMM_MODE_BF16X3 only.  Not in the paper; the launch's
 * tile parameters play the role of its per-target mc/kc/nc blocking
 * (Section 3.1, Eqs. 1-7).  This convenience call builds a plan, runs it and
 * frees it, so it allocates and synchronises the device; use the plan API
 * below for repeated calls.  Positions: 1 handle, 2 mode, 3 host_problems
 * (a bad problem i is reported as 100 + i), 4 count, 5 stream. */
gemm_status_t gemm_grouped(gemm_handle_t handle, gemm_mode_t mode,
                           const gemm_problem_t *host_problems, int32_t count, void *stream);

typedef struct gemm_grouped_plan_s *gemm_grouped_plan_t;

/* Flags of gemm_grouped_plan_create. */
enum {
    GEMM_GROUPED_AUTOTUNE = 1, /* choose tile shape, stage depth and raster by timing */
    GEMM_GROUPED_GRAPH = 2     /* capture the launches in a CUDA graph and replay it */
};

/* Prepare a grouped GEMM: validate the problems, allocate the plan's device
 * tables and BF16 split workspace (cudaMalloc; the plan owns them) and fix
 * the launch configuration.  With GEMM_GROUPED_AUTOTUNE the configurations a
 * shared-memory / tensor-memory feasibility model admits are ranked by a cost
 * model (padded tile work x wave quantisation), the best few are timed on the
 * problems themselves -- all of them when their outputs fit in scratch of
 * up to 4 GB and a quarter of the free device memory, else the leading ones
 * that do; writing only to that plan-owned scratch, never to any C -- and
 * the fastest is kept; results are cached per process (and in the
 * file named by the GEMM_AUTOTUNE_CACHE environment variable, if set) keyed
 * by SM count, mode and problem shapes.  Tuning runs on `stream` and
 * synchronises it.  Without it, a handle that sets none of bn, bk, stages
 * and cta_group gets the cost model's first choice, untimed; otherwise the
 * handle's configuration is used.  The
 * problems' pointers and sizes are fixed at creation.  Positions: 1 handle,
 * 2 mode, 3 host_problems (100 + i for problem i), 4 count, 5 flags,
 * 6 stream, 7 plan. */
gemm_status_t gemm_grouped_plan_create(gemm_handle_t handle, gemm_mode_t mode,
                                       const gemm_problem_t *host_problems, int32_t count,
                                       uint32_t flags, void *stream, gemm_grouped_plan_t *plan);

/* Enqueue the plan on `stream`: the split launch, the tensor-core launch and
 * one scaling launch per problem with K == 0 or alpha == 0.  With
 * GEMM_GROUPED_GRAPH and a non-NULL stream, the first run captures these
 * launches in a CUDA graph and every run replays that graph.  Runs of one
 * plan share its workspace: do not let them overlap on different streams. */
gemm_status_t gemm_grouped_plan_run(gemm_grouped_plan_t plan, void *stream);

/* The configuration the plan launches with, and the tuned time of one
 * tensor-core launch on the tuning set in ms (0 if not tuned). */
gemm_status_t gemm_grouped_plan_config(gemm_grouped_plan_t plan, gemm_config_t *cfg,
                                       double *tuned_ms);

/* Synchronise the device and free the plan.  NULL is accepted. */
gemm_status_t gemm_grouped_plan_destroy(gemm_grouped_plan_t plan);

/* Triangle selector of gemm_syr2k (diagonal included in both). */
typedef enum { GEMM_LOWER = 0, GEMM_UPPER = 1 } gemm_uplo_t;

/* SYR2K, the rank-2k update of Section 5.1 ("macro-level strategy for other
 * BLAS kernels"): on the `uplo` triangle of the N x N matrix C,
 *   trans == GEMM_OP_N: C <- alpha (A B^T + B A^T) + beta C, A and B N x K;
 *   trans == GEMM_OP_T: C <- alpha (A^T B + B^T A) + beta C, A and B K x N;
 * row-major FP32, device pointers, asynchronous on `stream`.  Elements of C
 * outside the triangle are neither read nor written; inside it C is not read
 * when beta == 0, and K == 0 or alpha == 0 give C <- beta C without reading A
 * or B.  Each C block is updated by the pair of GEMM products the section
 * describes, computed as one K loop of twice the length: the tensor-core
 * modes split A and B once into one workspace buffer and stage A-side rows of
 * A with B-side rows of B, then the reverse; only tiles that meet the
 * triangle are computed.  Modes as in gemm() (GEMM_MODE_F32_SIMT runs the
 * SIMT kernel's SYR2K variant).  Positions for GEMM_ERR_ARG: 1 handle,
 * 2 uplo, 3 trans, 4 N, 5 K, 6 alpha, 7 A, 8 lda, 9 B, 10 ldb, 11 beta, 12 C,
 * 13 ldc, 14 mode, 15 stream.  Workspace: gemm_syr2k_workspace_size. */
gemm_status_t gemm_syr2k(gemm_handle_t handle, gemm_uplo_t uplo, gemm_op_t trans,
                         int64_t N, int64_t K, float alpha,
                         const float *A, int64_t lda, const float *B, int64_t ldb,
                         float beta, float *C, int64_t ldc, gemm_mode_t mode, void *stream);

/* Bytes of workspace gemm_syr2k needs: the split planes of A and B; for
 * GEMM_MODE_F32_SIMT with N*N*K >= 2^30, FP32 K x N copies of A and B (used
 * with trans == N; the kernel reads A and B as stored when there is no room
 * for them, and below that size the result is 0); 0 for invalid arguments. */
size_t gemm_syr2k_workspace_size(gemm_handle_t handle, gemm_mode_t mode, gemm_op_t trans,
                                 int64_t N, int64_t K);

/* Gradients of C = op(A) op(B) (alpha = 1, beta = 0) for a given dC:
 *   dA = dC op(B)^T  (stored like A: M x K, or K x M when transA == T),
 *   dB = op(A)^T dC  (stored like B).
 * dA or dB may be NULL to skip it.  Not in the paper.  Positions:
 * 1 handle, 2 transA, 3 transB, 4 M, 5 N, 6 K, 7 dC, 8 lddc, 9 A, 10 lda,
 * 11 B, 12 ldb, 13 dA, 14 ldda, 15 dB, 16 lddb, 17 mode, 18 stream. */
gemm_status_t gemm_backward(gemm_handle_t handle, gemm_op_t transA, gemm_op_t transB,
                            int64_t M, int64_t N, int64_t K,
                            const float *dC, int64_t lddc,
                            const float *A, int64_t lda, const float *B, int64_t ldb,
                            float *dA, int64_t ldda, float *dB, int64_t lddb,
                            gemm_mode_t mode, void *stream);

/* Benchmark hook.  While enabled, every call records a pair of CUDA events
 * around its main GEMM kernel (the tensor-core or SIMT kernel, not the
 * split/pack or reduce kernels) on the call's stream.  Not in the paper. */
gemm_status_t gemm_profile_enable(gemm_handle_t handle, int enable);

/* Synchronise on the recorded events and return the summed duration of the
 * main kernels recorded since enabling or the last read (milliseconds) and
 * their number; then forget them. */
gemm_status_t gemm_profile_read(gemm_handle_t handle, double *main_ms, int *main_launches);

/* The same events one launch at a time: writes the duration (milliseconds)
 * of each recorded main kernel, in launch order, to ms[0 .. capacity-1],
 * sets *count to the number recorded (which may exceed capacity; the rest
 * are dropped), then forgets them.  Positions: 1 handle, 2 ms (NULL with
 * capacity > 0), 3 capacity (< 0), 4 count.  Not in the paper. */
gemm_status_t gemm_profile_read_each(gemm_handle_t handle, float *ms, int capacity, int *count);

/* gemm() in GEMM_MODE_BF16X3 for callers that cannot allocate device
 * memory: code running where cudaMalloc is forbidden or would stall, such as
 * a custom allocator's own hooks, a plugin whose host application owns all
 * device memory, or a loop that must never enter the driver's allocator.
 * No handle: it calls no cudaMalloc, cudaFree or other allocating routine.
 * The paper has no counterpart.
 * Scratch is one 64 MiB device array inside the library.  The runtime
 * reserves it on a GPU when it loads the library's module there -- with
 * lazy module loading (the CUDA default) during the FIRST call on that
 * device, which is also when the call looks up the array's device address
 * (cudaGetSymbolAddress) with that device current.  That first call may
 * therefore synchronise or fail for lack of memory: make it once at
 * start-up, before any stream capture.  The array is kept until the process
 * exits.  A problem must fit: 4 * (M + N) * round_up(K, 8) bytes <= 64 MiB,
 * else GEMM_ERR_WORKSPACE and nothing is launched.  All calls share the
 * array (it keeps the last call's contents; each call overwrites what it
 * reads): calls whose GPU work overlaps, on different streams or threads,
 * race -- serialise them.  Invalid arguments give GEMM_ERR_ARG (no position
 * is recorded: there is no handle).  A kernel that abandons a bounded wait
 * leaves C undefined and sets a device error word that
 * gemm_bf16x3_noalloc_check reports.  Same arguments and results as gemm()
 * in GEMM_MODE_BF16X3 without split-K. */
gemm_status_t gemm_bf16x3_noalloc(gemm_op_t transA, gemm_op_t transB,
                                  int64_t M, int64_t N, int64_t K,
                                  float alpha, const float *A, int64_t lda,
                                  const float *B, int64_t ldb,
                                  float beta, float *C, int64_t ldc, void *stream);

/* Synchronise `stream`, then read and clear gemm_bf16x3_noalloc's device
 * error word on the current device: GEMM_ERR_TIMEOUT if a call since the
 * last check abandoned a bounded wait (its C is undefined), GEMM_ERR_CUDA if
 * the stream reported an error, GEMM_ERR_DEVICE if the current device is
 * not an sm_103 GPU, else GEMM_OK.  Allocates nothing.  The paper has no
 * counterpart. */
gemm_status_t gemm_bf16x3_noalloc_check(void *stream);

/* Synchronise `stream`, then read and clear the handle's device error word:
 * GEMM_ERR_TIMEOUT if a kernel abandoned a bounded wait since the last
 * check, GEMM_ERR_CUDA if the stream reported an error, else GEMM_OK. */
gemm_status_t gemm_sync(gemm_handle_t handle, void *stream);

/* 1-based position of the invalid argument of the handle's last call
 * (0 if the last call succeeded or failed for another reason). */
int gemm_last_error_arg(gemm_handle_t handle);

/* The same as a status-returning call (the BLAS xerbla convention): *pos
 * receives the position; GEMM_ERR_ARG (position 1 or 2) for a NULL handle
 * or pos. */
gemm_status_t gemm_get_last_error_arg(gemm_handle_t handle, int *pos);

/* Number of kernels the handle's last successful call enqueued. */
int gemm_last_launch_count(gemm_handle_t handle);

/* Static text for a status code. */
const char *gemm_status_string(gemm_status_t status);

#ifdef __cplusplus
}
#endif

#endif /* GB300_GEMM_H */
