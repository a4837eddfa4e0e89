// Host-side interfaces between the C-ABI layer (api.cu) and the kernel
// launchers (simt_f32.cu, split.cu, tc_gemm.cu).  Not part of the public ABI.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace gb300 {

// Tensor-core GEMM launch parameters chosen by the host.
struct TcLaunch {
    int bn = 256;            // tile width (tile height is 128)
    int bk = 32;             // K depth per pipeline stage
    int stages = 0;          // 0 = deepest ring that fits
    int raster_group = 16;   // M tiles walked together
    int max_ctas = 0;        // 0 = one per SM
    int split_k = 1;         // K slices (>1: partial sums, summed by a reduce kernel or in the GEMM)
    int splitk_reduce = 0;   // split-K sum: 0 in the GEMM kernel when possible, 1 reduce launch
    long long poll_limit = 0;  // 0 = default
    int promote_k = 512;     // split-precision: K elements per TMEM chunk (0 = no promotion)
    int cta_group = 1;       // 2: CTA-pair kernel (256-row tiles, BN = 256 only)
    int kmajor = 0;          // 1: every operand K-major (transposing split / pack)
    int fuse = 0;            // in-kernel split: bit 0 A, bit 1 B is FP32 (TcOperand::f32),
                             // split inside the kernel; the other operand is BF16 planes
};

// One operand of the tensor-core kernel: BF16, `planes` stacked planes
// (1: hi only; 2: hi then lo) `plane_ld` elements apart, each holding the
// operand's `rows` (M for A, N for B) x `k` elements.  K-major (mn_major 0):
// one stored row per operand row, K contiguous, row stride `ld`.  MN-major
// (mn_major 1): one stored row per K index, the operand rows contiguous,
// row stride `ld` (the layout of A stored K x M, or of B stored K x N).
struct TcOperand {
    const uint16_t* base;
    int64_t rows;
    int64_t k;
    int64_t ld;
    int64_t plane_ld;
    int planes;
    int mn_major = 0;
    int box_planes = 0;  // planes one TMA box copies (0 = all); SYR2K buffers hold two matrices
    // In-kernel split: the caller's FP32 matrix (base unused), `ld` in FP32
    // elements, 16-byte aligned with ld % 4 == 0 (TMA); the kernel splits it
    // into hi/lo planes in shared memory.
    const float* f32 = nullptr;
};

// Row stride and plane size (elements) of an operand written by the split
// or pack pass: K-major rows x round8(k), or MN-major k x round8(rows), so
// that every stored row starts on a 16-byte boundary.
struct PackedLayout {
    int64_t ld;
    int64_t plane;
};
inline PackedLayout packed_layout(int64_t rows, int64_t k, bool mn_major) {
    const int64_t ld = ((mn_major ? rows : k) + 7) / 8 * 8;
    return PackedLayout{ld, (mn_major ? k : rows) * ld};
}

// One problem of a grouped tensor-core launch, as the kernel reads it from
// device memory.  tile_start is the index of the problem's first output
// tile in the launch's concatenated tile space (a prefix sum).
struct GroupedProblem {
    float* C;
    long long ldc;
    int M, N, K;
    int num_m, num_n, k_blocks;
    int tile_start;
    float alpha, beta;
    int major;  // bit 0: A MN-major, bit 1: B MN-major (TcOperand::mn_major)
};

// Encode the 3-D TMA map of a BF16 operand with the box and swizzle the
// UMMA descriptor expects: K-major (k, row, plane) with a (bk, box_rows,
// planes) box; MN-major (row, k, plane) with a (64, bk, planes) box, loaded
// box_rows / 64 times per stage.
bool encode_operand(CUtensorMap* map, const TcOperand& op, int bk, int box_rows);

// Grouped launch: `count` problems described by dev_problems (device) with
// two tensor maps each in dev_maps (device, encoded with cfg.bk and a box of
// 128 rows for A and cfg.bn / cfg.cta_group rows for B); total_tiles = sum of
// num_m * num_n, with num_m counting tiles of 128 * cfg.cta_group rows;
// dev_tile_prob[t] = index of the problem that owns tile t.  cta_group 2
// runs the CTA-pair kernel (split precision, bn 256 only).
int launch_tc_grouped(int nterms, const TcLaunch& cfg, const GroupedProblem* dev_problems,
                      const CUtensorMap* dev_maps, const int* dev_tile_prob, int count,
                      int total_tiles, int* err_word, int num_sms, cudaStream_t stream);

// Dynamic shared memory the tensor-core kernel (one CTA per tile, or CTA
// pairs with cta_group 2) asks for with this config (0 if the configuration
// does not exist).
int tc_smem_bytes(int nterms, int bn, int bk, int stages, int cta_group = 1);

// Floats of workspace a CTA-pair launch with one K slice uses to split the
// tiles of a mostly idle last wave in two K halves (0: no tail split).
int64_t tc_tail_floats(const TcLaunch& cfg, int nterms, int64_t M, int64_t N, int64_t K, int split,
                       int num_sms);

// C <- alpha * A_op B_op^T + beta * C where A_op is M x K and B_op is N x K
// (both K-contiguous BF16); nterms = 1 (hi.hi) or 3 (lo.hi + hi.lo + hi.hi).
// `partial`: split_k * M * N floats of workspace when split_k > 1; with one
// K slice, null or the tc_tail_floats floats for a tail split (which then
// adds a reduce launch).  Returns 0 or a negative gemm_status_t value.
int launch_tc_gemm(const TcOperand& a, const TcOperand& b, int nterms, int64_t M, int64_t N,
                   int64_t K, float alpha, float beta, float* C, int64_t ldc, float* partial,
                   const TcLaunch& cfg, int* err_word, int num_sms, cudaStream_t stream,
                   int* launches);

// SYR2K (Section 5.1) on the tensor cores: the `uplo` (1 lower, 2 upper)
// triangle of C (N x N) <- alpha (X Y^T + Y X^T) + beta C, X and Y the two
// N x K operands stored in one buffer `xy`: planes [0, P) hold X, planes
// [P, 2P) hold Y (P = 1 for nterms 1: hi; 2 for nterms 3: hi, lo), with
// xy.planes = 2P and xy.box_planes = P.  Only tiles that meet the triangle
// are computed and only triangle elements are stored.
int launch_tc_syr2k(const TcOperand& xy, int nterms, int uplo, int64_t N, int64_t K, float alpha,
                    float beta, float* C, int64_t ldc, const TcLaunch& cfg, int* err_word,
                    int num_sms, cudaStream_t stream, int* launches);

// FP32 SIMT GEMM (row-major, op by trans flags).
cudaError_t launch_simt_f32(int transA, int transB, int64_t M, int64_t N, int64_t K, float alpha,
                            const float* A, int64_t lda, const float* B, int64_t ldb, float beta,
                            float* C, int64_t ldc, cudaStream_t stream);

// Y = op(X) split into hi/lo BF16 (lo may be null), rows x cols, row stride ldo.
cudaError_t launch_split_bf16(int trans, int64_t rows, int64_t cols, const float* X, int64_t ldx,
                              uint16_t* hi, uint16_t* lo, int64_t ldo, cudaStream_t stream);

// One matrix of a two-matrix split launch: Y = op(X) (trans 1: X stored
// cols x rows), rows x cols, hi/lo BF16 with row stride ldo (lo may be null).
// x_vec and blocks are filled in by the launcher.
struct SplitArg {
    int trans;
    int64_t rows, cols;
    const float* X;
    int64_t ldx;
    uint16_t* hi;
    uint16_t* lo;
    int64_t ldo;
    int x_vec = 0;
    int blocks = 0;
};

// Both operands' split in one launch, each as launch_split_bf16 would do it
// (same results, one launch fewer).
cudaError_t launch_split_bf16_pair(SplitArg a, SplitArg b, cudaStream_t stream);

// One matrix of a grouped split launch (device table entry): Y = op(X),
// rows x cols, written as hi/lo BF16 with row stride ldo; tile_start is the
// prefix sum of 64 x 64 output tiles over the preceding jobs.
struct SplitJob {
    const float* src;
    long long ldx;
    uint16_t* hi;
    uint16_t* lo;
    long long ldo;
    int rows, cols;
    int trans;
    int x_vec;  // src 16-byte aligned and ldx % 4 == 0
    int tile_start;
    int tiles_r;  // (rows + 63) / 64
};

// Split every job of the table in one launch (total_tiles 64 x 64 tiles;
// dev_tile_job[t] = index of the job that owns tile t).
cudaError_t launch_split_grouped(const SplitJob* dev_jobs, const int* dev_tile_job, int njobs,
                                 int total_tiles, int num_sms, cudaStream_t stream);

// The same for a table whose tile map lists only transposed jobs, with a
// double-buffered shared tile (asynchronous copies of the next tile in flight).
cudaError_t launch_split_grouped_t(const SplitJob* dev_jobs, const int* dev_tile_job, int njobs,
                                   int total_tiles, int num_sms, cudaStream_t stream);

// Y = op(X) for BF16 X (a pure re-layout), rows x cols, row stride ldo.
cudaError_t launch_pack_bf16(int trans, int64_t rows, int64_t cols, const uint16_t* X,
                             int64_t ldx, uint16_t* out, int64_t ldo, cudaStream_t stream);

// Y = X^T in FP32: Y is rows x cols (row stride ldy), X is stored cols x rows.
cudaError_t launch_transpose_f32(int64_t rows, int64_t cols, const float* X, int64_t ldx,
                                 float* Y, int64_t ldy, cudaStream_t stream);

// C <- beta * C (C <- 0 when beta == 0, without reading C); uplo 1 / 2
// restricts it to the lower / upper triangle (diagonal included).
cudaError_t launch_scale_c(int64_t M, int64_t N, float beta, float* C, int64_t ldc,
                           cudaStream_t stream, int uplo = 0);

// SYR2K on the CUDA cores: the `uplo` (1 lower, 2 upper) triangle of C
// (N x N) <- alpha (op(X) op(Y)^T + op(Y) op(X)^T) + beta C, op(X) = X
// (stored N x K, trans 0) or X^T (stored K x N, trans 1).
cudaError_t launch_simt_syr2k(int uplo, int trans, int64_t N, int64_t K, float alpha,
                              const float* X, int64_t ldx, const float* Y, int64_t ldy, float beta,
                              float* C, int64_t ldc, cudaStream_t stream);

// C <- alpha * sum_s P[s] + beta * C over split_k dense M x N slabs.
cudaError_t launch_splitk_reduce(int64_t M, int64_t N, int split_k, const float* P, float alpha,
                                 float beta, float* C, int64_t ldc, cudaStream_t stream);

// One problem of a grouped split-K sum (device table entry): the same
// C <- alpha * sum_s P[s] + beta * C over its `split` dense M x N slabs.
// unit_start: the prefix sum of units (4 elements when vec, else 1) over the
// preceding jobs; vec: N, ldc multiples of 4 and P, C 16-byte aligned.
struct ReduceJob {
    const float* P;
    float* C;
    long long M, N, ldc;
    long long unit_start;
    int split;
    int vec;
    float alpha, beta;
};

// Every job's sum in one launch (total_units units), with the arithmetic of
// launch_splitk_reduce, so the two give the same bits.
cudaError_t launch_splitk_reduce_grouped(const ReduceJob* dev_jobs, int njobs,
                                         long long total_units, int num_sms, cudaStream_t stream);

}  // namespace gb300
