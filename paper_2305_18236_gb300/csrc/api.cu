// C ABI of the GEMM library (declarations and contracts in include/gemm.h).
//
// Host-side work only: argument checks (BLAS xerbla style), quick returns,
// workspace planning, the launch plan, and dispatch to the kernels.  Every
// arithmetic step of C = alpha op(A) op(B) + beta C runs in a CUDA kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/gemm.h"
#include "internal.h"

// Row blocks of the gemm_from_host pipeline (at most; blocks of >= 512 rows).
constexpr int kPipeBlocks = 16;

struct gemm_context {
    int device = 0;
    int num_sms = 0;
    int* err_word = nullptr;  // device, 256 bytes
    void* own_ws = nullptr;
    size_t own_ws_bytes = 0;
    void* user_ws = nullptr;
    size_t user_ws_bytes = 0;
    gemm_config_t cfg{};
    int last_err_arg = 0;
    int last_launches = 0;
    // device staging for gemm_from_host
    float* hA = nullptr;
    float* hB = nullptr;
    float* hC = nullptr;
    size_t hA_bytes = 0, hB_bytes = 0, hC_bytes = 0;
    // gemm_from_host pipeline: copy-in, compute and copy-out streams; events
    // start, B ready, end, then per block "inputs in" and "product done"
    cudaStream_t pipe[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t pipe_ev[3 + 2 * kPipeBlocks] = {};
    // benchmark hook: event pairs around main kernels
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;  // 2 per recorded launch
    size_t ev_used = 0;
};

namespace {

using gb300::TcLaunch;
using gb300::TcOperand;

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

gemm_status_t fail_arg(gemm_context* h, int pos) {
    if (h) h->last_err_arg = pos;
    return GEMM_ERR_ARG;
}

// Stored-matrix geometry check: rows x cols stored with row stride ld.
bool ld_ok(int64_t ld, int64_t cols) { return ld >= std::max<int64_t>(1, cols); }

// What a tensor-core launch serves (its library-choice defaults differ).
enum class Call {
    Split,    // gemm(), gemm_from_host, gemm_backward: FP32 operands split first
    Bf16,     // gemm_bf16: BF16 operands, read in place or packed
    Grouped,  // grouped plans (one CTA per tile)
    Syr2k,    // gemm_syr2k (one CTA per tile)
};

// True when packing the MN-contiguous BF16 operands K-contiguous (a launch
// of about 5 us plus 4 bytes of traffic per element) costs less than a
// tenth of the GEMM itself (time estimates at rough GB300 rates): the
// K-major kernel, ~15 % faster on the tensor cores, then wins overall;
// otherwise the operands are read in place.
bool pack_pays(int64_t M, int64_t N, int64_t K, bool pack_a, bool pack_b) {
    const double m = double(M), n = double(N), k = double(K);
    const double t_mma = 2.0 * m * n * k / 1.2e15;
    const double t_mem = (2.0 * (m * k + n * k) + 4.0 * m * n) / 6.0e12;
    const double packed = (pack_a ? m * k : 0.0) + (pack_b ? n * k : 0.0);
    if (packed == 0.0) return false;
    return 5e-6 + 4.0 * packed / 6.0e12 < 0.1 * std::max(t_mma, t_mem);
}

// Tile plan of one tensor-core launch.  Library choice (configuration 0):
//  * CTA pairs (256 x 256 tiles, cta_group::2, BK 64) when there are at
//    least as many pair tiles as SM pairs, for split precision on split
//    operands (each SM then stages half of B and runs ~12 % fewer cycles per
//    GEMM) and for plain BF16 with K >= 512 (7-14 % faster than one CTA per
//    tile from K = 1024 up, with a second producer warp for the B copies);
//    one CTA per 128 x 256 tile otherwise (BK 32 for split precision, 64
//    for plain BF16);
//  * operands K-major for split operands (the split transposes at nearly the
//    copy rate and the K-major kernel runs a few % faster) and for gemm_bf16
//    when packing pays (pack_pays); in their stored orientation otherwise,
//    and always in grouped plans and SYR2K, whose transposing passes cost
//    more than the kernel gains.
// K slices of a launch with `tiles` output tiles and `kblocks` K blocks when
// the handle leaves split-K to the library: few tiles and a long K are
// sliced so that every SM gets work, at least 4 K blocks a slice and at most
// 8 slices, so that the GEMM kernel can sum them itself (a cluster of CTAs
// per tile).  Measured at 1024^3 plain BF16 (16 K blocks of 64): 4 slices
// 0.021 ms a call against 0.023 ms with 2.
int auto_split_k(int64_t tiles, int64_t kblocks, int num_sms) {
    int64_t split = 1;
    if (tiles * 2 <= num_sms && kblocks >= 8)
        split = std::min<int64_t>({num_sms / std::max<int64_t>(tiles, 1), kblocks / 4, 8});
    return int(std::max<int64_t>(split, 1));
}

// Split placement of a split-precision call: which operands the kernel
// splits itself (bit 0 A, bit 1 B; `allowed` = those TMA can read in place)
// and which the pass splits first, by expected seconds (rough GB300 rates).
//  * The pass moves 8 bytes per element (FP32 read, hi and lo written) at
//    HBM speed for each operand it splits, plus one launch (one for both).
//  * The in-kernel split (one CTA per 128 x 256 tile, BK 32) re-splits every
//    staged element of a fused operand in every tile that stages it: A once
//    per N tile, B once per M tile.  A CTA splits about 9e9 elements/s; the
//    tiles run in waves of one per SM.  Its MMAs run at about 3/5 of the
//    pair kernel's rate; the kernel takes the longer of the two.
//  * Mask 0 is the CTA-pair kernel on pre-split operands, bounded by its
//    MMAs or by the C traffic (short K); with too few tiles for pairs, the
//    one-CTA kernel, whose MMAs run at about 4/5 of the pair rate.
// So a small operand staged by many tiles (A of a skinny M) goes to the pass
// and a large one staged by few tiles (its B) to the kernel.  Fit to per-call
// times of all four placements on eight shapes from (128, 8192, 8192) to
// 2048^3; on each it picks the placement measured fastest.
int fuse_mask(int64_t M, int64_t N, int64_t K, int num_sms, bool beta_zero, int allowed) {
    const double m = double(M), n = double(N), k = double(K);
    const double hbm = 6.5e12, sm_rate = 1.8e15 / std::max(num_sms, 1);
    const double t_c = (beta_zero ? 4.0 : 8.0) * m * n / hbm;
    const double launch = 3e-6;
    auto pass = [&](double rows) { return 8.0 * rows * k / hbm; };
    // one CTA per 128 x 256 tile, split-K as the plan would slice it
    const int64_t tiles = ((M + 127) / 128) * ((N + 255) / 256);
    const int split = auto_split_k(tiles, (K + 31) / 32, num_sms);
    const double waves = double((tiles * split + num_sms - 1) / num_sms);
    const double k_tile = k / split;
    auto tile_mma = [&](double eff) { return waves * 6.0 * 128.0 * 256.0 * k_tile / (eff * sm_rate); };
    const bool pairs = ((M + 255) / 256) * ((N + 255) / 256) >= num_sms / 2;
    double best = pass(m) + pass(n) + launch +
                  std::max(pairs ? 6.0 * m * n * k / 1.8e15 : tile_mma(0.8), t_c);
    int best_mask = 0;
    for (int mask = 1; mask <= 3; ++mask) {
        if ((mask & allowed) != mask) continue;
        const double per_tile = ((mask & 1) ? 128.0 : 0.0) + ((mask & 2) ? 256.0 : 0.0);
        const double t_conv = waves * per_tile * k_tile / 9e9;
        const double t_mma = tile_mma(0.6);
        const double t = ((mask & 1) ? 0.0 : pass(m)) + ((mask & 2) ? 0.0 : pass(n)) +
                         (mask == 3 ? 0.0 : launch) + std::max(t_conv, t_mma);
        if (t < best) {
            best = t;
            best_mask = mask;
        }
    }
    return best_mask;
}

TcLaunch plan_tc(const gemm_context* h, int nterms, int64_t M, int64_t N, int64_t K, Call call,
                 bool pack_a = false, bool pack_b = false, bool beta_zero = false,
                 int f32_ops = 0) {
    TcLaunch c;
    c.bn = h->cfg.bn ? h->cfg.bn : 256;
    if (call == Call::Syr2k) {
        c.cta_group = 1;  // the triangle walk exists in the one-CTA kernel only
    } else if (h->cfg.cta_group != 0) {
        c.cta_group = h->cfg.cta_group;
    } else {
        // CTA pairs when the problem has a 256 x 256 tile for every SM pair:
        // split precision always; plain BF16 when K >= 512 (measured: pairs
        // 7-14 % faster from K = 1024 up, 11 % slower at K = 64, where the C
        // write bounds the call).
        const int64_t pair_tiles = ((M + 255) / 256) * ((N + 255) / 256);
        const bool pair_kind = (nterms == 3 && call == Call::Split) ||
                               (nterms == 1 && (call == Call::Split || call == Call::Bf16) &&
                                K >= 512);
        c.cta_group = (pair_kind && c.bn >= 256 && h->cfg.split_k <= 1 &&
                       pair_tiles >= h->num_sms / 2)
                          ? 2
                          : 1;
    }
    c.bk = h->cfg.bk ? h->cfg.bk : (nterms == 3 && c.cta_group == 1 ? 32 : 64);
    switch (h->cfg.operand_layout) {
        case GEMM_LAYOUT_K_MAJOR: c.kmajor = 1; break;
        case GEMM_LAYOUT_AS_STORED: c.kmajor = 0; break;
        default:
            c.kmajor = call == Call::Split ? 1
                       : call == Call::Bf16 ? (pack_pays(M, N, K, pack_a, pack_b) ? 1 : 0)
                                            : 0;
    }
    // 256 x 512 pair tiles (plain BF16): two MMAs share each staged A tile, so
    // a stage moves a third fewer bytes per flop through shared memory, but
    // their two accumulators fill the tensor memory and the epilogue no longer
    // overlaps the next tile's MMAs.  Measured against 256-wide pair tiles
    // with beta == 0 (TMA-store epilogue): 5-6 % faster at K = 8192, 10-12 %
    // faster at K = 4096 with B read MN-major in place, up to 5 % slower at
    // K = 4096 with K-major B and 11-18 % slower at K = 1024; with beta != 0
    // the drain waits on reads of C and 8192^3 is 15 % slower, so the
    // library takes them only for beta == 0.
    const bool wide_ok = c.cta_group == 2 && nterms == 1 && c.bk == 64 &&
                         (call == Call::Split || call == Call::Bf16);
    const bool b_in_place_mn = call == Call::Bf16 && !c.kmajor && pack_b;
    if (h->cfg.bn == 0 && wide_ok && beta_zero &&
        (K >= 8192 || (K >= 2048 && b_in_place_mn)) &&
        ((M + 255) / 256) * ((N + 511) / 512) >= h->num_sms / 2)
        c.bn = 512;
    if (c.bn == 512 && !wide_ok) c.bn = 256;
    // In-kernel split (split precision; f32_ops: bit 0 A, bit 1 B is an FP32
    // matrix TMA can read in place): one CTA per 128 x 256 tile with BK 32,
    // operands as stored; an operand the kernel does not split is split by
    // the pass.
    int fuse = 0;
    if (nterms == 3 && call == Call::Split) {
        switch (h->cfg.split_place) {
            case GEMM_SPLIT_IN_KERNEL: fuse = 3; break;
            case GEMM_SPLIT_IN_KERNEL_A: fuse = 1; break;
            case GEMM_SPLIT_IN_KERNEL_B: fuse = 2; break;
            case GEMM_SPLIT_AUTO:
                if (h->cfg.bn == 0 && h->cfg.bk == 0 && h->cfg.cta_group == 0 &&
                    h->cfg.operand_layout == GEMM_LAYOUT_AUTO)
                    fuse = fuse_mask(M, N, K, h->num_sms, beta_zero, f32_ops);
                break;
            default: break;
        }
        fuse &= f32_ops;
    }
    if (fuse) {
        c.fuse = fuse;
        c.cta_group = 1;
        c.bn = 256;
        c.bk = 32;
        c.kmajor = 0;
    }
    c.stages = h->cfg.stages;
    c.raster_group = h->cfg.raster_group ? h->cfg.raster_group : 16;
    c.max_ctas = h->cfg.max_ctas;
    c.poll_limit = h->cfg.wait_poll_limit;
    c.promote_k = h->cfg.promote_k == 0 ? 512 : (h->cfg.promote_k < 0 ? 0 : h->cfg.promote_k);
    if (h->cfg.split_k > 0) {
        c.split_k = h->cfg.split_k;
    } else {
        c.split_k = auto_split_k(((M + 127) / 128) * ((N + c.bn - 1) / c.bn),
                                 (K + c.bk - 1) / c.bk, h->num_sms);
    }
    c.splitk_reduce = h->cfg.splitk_reduce;
    return c;
}

struct WsPlan {
    size_t a_off = 0, b_off = 0, p_off = 0, total = 0;
    int planes = 1;
    int split = 1;
    bool tail = false;  // p_off holds a CTA-pair launch's tail-split halves
};

// How one operand reaches the tensor cores after the split / pack pass.  An
// operand stored K x rows (A with transA == T, B with transB == N) keeps
// that orientation (MN-major tiles, a plain non-transposing pass) unless the
// launch wants every operand K-major; the others become op(X) as rows x K.
struct OpPlan {
    bool stored_k_rows;  // stored K x rows
    bool mn;             // packed MN-major
    gb300::PackedLayout lay;
};

OpPlan plan_op(int64_t rows, int64_t K, bool stored_k_rows, const TcLaunch& c) {
    OpPlan o;
    o.stored_k_rows = stored_k_rows;
    o.mn = stored_k_rows && !c.kmajor;
    o.lay = gb300::packed_layout(rows, K, o.mn);
    return o;
}

// Split op(X) (rows x K) into hi (and lo, `planes` == 2) planes at `hi` in the
// operand's packed layout.
cudaError_t split_op(const OpPlan& o, int64_t rows, int64_t K, const float* X, int64_t ldx,
                     uint16_t* hi, int planes, cudaStream_t s) {
    uint16_t* lo = planes > 1 ? hi + o.lay.plane : nullptr;
    if (o.mn) return gb300::launch_split_bf16(0, K, rows, X, ldx, hi, lo, o.lay.ld, s);
    return gb300::launch_split_bf16(o.stored_k_rows ? 1 : 0, rows, K, X, ldx, hi, lo, o.lay.ld, s);
}

// The same for two operands in one launch (the pass over A and B together).
gb300::SplitArg split_arg(const OpPlan& o, int64_t rows, int64_t K, const float* X, int64_t ldx,
                          uint16_t* hi, int planes) {
    gb300::SplitArg a;
    a.trans = o.mn ? 0 : (o.stored_k_rows ? 1 : 0);
    a.rows = o.mn ? K : rows;
    a.cols = o.mn ? rows : K;
    a.X = X;
    a.ldx = ldx;
    a.hi = hi;
    a.lo = planes > 1 ? hi + o.lay.plane : nullptr;
    a.ldo = o.lay.ld;
    return a;
}

cudaError_t split_ops(const OpPlan& pa, int64_t M, const float* A, int64_t lda, uint16_t* a_hi,
                      const OpPlan& pb, int64_t N, const float* B, int64_t ldb, uint16_t* b_hi,
                      int64_t K, int planes, cudaStream_t s) {
    return gb300::launch_split_bf16_pair(split_arg(pa, M, K, A, lda, a_hi, planes),
                                         split_arg(pb, N, K, B, ldb, b_hi, planes), s);
}

TcOperand operand_of(const OpPlan& o, const uint16_t* hi, int64_t rows, int64_t K, int planes) {
    TcOperand t{hi, rows, K, o.lay.ld, o.lay.plane, planes};
    t.mn_major = o.mn ? 1 : 0;
    return t;
}

// An FP32 matrix TMA can read in place: 16-byte aligned base and row stride.
bool f32_tma_ok(const float* X, int64_t ld) {
    return (reinterpret_cast<uintptr_t>(X) & 15) == 0 && ld % 4 == 0;
}

// The caller's FP32 op(X) (rows x K) for the in-kernel split: stored K x rows
// (MN-major tiles) or rows x K (K-major tiles).
TcOperand f32_operand(const float* X, int64_t ld, int64_t rows, int64_t K, bool stored_k_rows) {
    TcOperand t{nullptr, rows, K, ld, 0, 2};
    t.mn_major = stored_k_rows ? 1 : 0;
    t.f32 = X;
    return t;
}

// Workspace of a tensor-core call: packed A and packed B (planes x the
// operand's packed plane, BF16; plane size 0 = not packed), split-K partials
// (split x M x N FP32) or, with one K slice and num_sms > 0, the tail split's
// half tiles of a CTA-pair launch.
WsPlan plan_ws(int planes, int64_t a_plane, int64_t b_plane, int64_t M, int64_t N, int64_t K,
               const TcLaunch& c, int num_sms = 0) {
    WsPlan w;
    w.planes = planes;
    size_t off = 0;
    if (a_plane > 0) {
        w.a_off = off;
        off += align_up(size_t(planes) * a_plane * 2);
    }
    if (b_plane > 0) {
        w.b_off = off;
        off += align_up(size_t(planes) * b_plane * 2);
    }
    const int64_t kblocks = (K + c.bk - 1) / c.bk;
    int split = std::max(1, std::min<int>(c.split_k, int(std::max<int64_t>(kblocks, 1))));
    if (split > 1) {
        const int64_t per = (kblocks + split - 1) / split;
        split = int((kblocks + per - 1) / per);
    }
    w.split = split;
    if (split > 1) {
        w.p_off = off;
        off += align_up(size_t(split) * M * N * 4);
    } else if (num_sms > 0) {
        const int64_t tail = gb300::tc_tail_floats(c, planes == 2 ? 3 : 1, M, N, K, 1, num_sms);
        if (tail > 0) {
            w.p_off = off;
            off += align_up(size_t(tail) * 4);
            w.tail = true;
        }
    }
    w.total = off;
    return w;
}

// Workspace pointer of at least `bytes`, from the caller or the handle.
gemm_status_t get_ws(gemm_context* h, size_t bytes, uint8_t** out) {
    *out = nullptr;
    if (bytes == 0) return GEMM_OK;
    if (h->user_ws) {
        if (h->user_ws_bytes < bytes) return GEMM_ERR_WORKSPACE;
        *out = static_cast<uint8_t*>(h->user_ws);
        return GEMM_OK;
    }
    if (h->own_ws_bytes < bytes) {
        if (h->own_ws) {
            cudaDeviceSynchronize();  // earlier work may still use the old buffer
            cudaFree(h->own_ws);
            h->own_ws = nullptr;
            h->own_ws_bytes = 0;
        }
        if (cudaMalloc(&h->own_ws, bytes) != cudaSuccess) {
            cudaGetLastError();
            return GEMM_ERR_WORKSPACE;
        }
        h->own_ws_bytes = bytes;
    }
    *out = static_cast<uint8_t*>(h->own_ws);
    return GEMM_OK;
}

// Event pair bracketing the next main-kernel launch (profiling only).
cudaEvent_t* prof_slot(gemm_context* h) {
    if (!h->profiling) return nullptr;
    if (h->ev_used + 2 > h->ev_pool.size()) {
        for (int i = 0; i < 2; ++i) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            h->ev_pool.push_back(e);
        }
    }
    cudaEvent_t* p = &h->ev_pool[h->ev_used];
    h->ev_used += 2;
    return p;
}

struct ProfScope {
    cudaEvent_t* ev;
    cudaStream_t s;
    ProfScope(gemm_context* h, cudaStream_t st) : ev(prof_slot(h)), s(st) {
        if (ev) cudaEventRecord(ev[0], s);
    }
    ~ProfScope() {
        if (ev) cudaEventRecord(ev[1], s);
    }
};

gemm_status_t status_of(cudaError_t e) { return e == cudaSuccess ? GEMM_OK : GEMM_ERR_CUDA; }

gemm_status_t check_common(gemm_context* h, int transA, int transB, int64_t M, int64_t N,
                           int64_t K, float alpha, const void* A, int64_t lda, const void* B,
                           int64_t ldb, const void* C, int64_t ldc) {
    if (!h) return fail_arg(h, 1);
    h->last_err_arg = 0;
    if (transA != GEMM_OP_N && transA != GEMM_OP_T) return fail_arg(h, 2);
    if (transB != GEMM_OP_N && transB != GEMM_OP_T) return fail_arg(h, 3);
    if (M < 0) return fail_arg(h, 4);
    if (N < 0) return fail_arg(h, 5);
    if (K < 0) return fail_arg(h, 6);
    const bool reads_ab = M > 0 && N > 0 && K > 0 && alpha != 0.0f;
    if (reads_ab && !A) return fail_arg(h, 8);
    if (!ld_ok(lda, transA ? M : K)) return fail_arg(h, 9);
    if (reads_ab && !B) return fail_arg(h, 10);
    if (!ld_ok(ldb, transB ? K : N)) return fail_arg(h, 11);
    if (M > 0 && N > 0 && !C) return fail_arg(h, 13);
    if (!ld_ok(ldc, N)) return fail_arg(h, 14);
    return GEMM_OK;
}

bool too_large(int64_t M, int64_t N, int64_t K) {
    const int64_t lim = (int64_t(1) << 31) - 1024;
    return M > lim || N > lim || K > lim;
}

// FP32 SIMT pack (Algorithm 1's pack step for the SIMT kernel): an operand
// stored K-contiguous (A with transA == N, B with transB == T) is first
// transposed into workspace, so the kernel reads both operands with rows
// along M and N (its fastest form, 74 % of the FP32 peak at 8192^3 against
// 56-61 % when it transposes K-contiguous rows itself).  Only for problems of
// at least 2^30 multiply-adds, where the pass costs under 1 % of the GEMM.
// The workspace size does not depend on the transposes (room for both
// operands), so one query covers every orientation of a problem.
struct SimtPack {
    bool on = false;
    int64_t lda_p = 0, ldb_p = 0;  // packed strides: K x round4(M), K x round4(N)
    size_t a_bytes = 0, total = 0;
};

SimtPack plan_simt_pack(int64_t M, int64_t N, int64_t K) {
    SimtPack p;
    if (double(M) * double(N) * double(K) < double(int64_t(1) << 30)) return p;
    p.on = true;
    p.lda_p = (M + 3) / 4 * 4;
    p.ldb_p = (N + 3) / 4 * 4;
    p.a_bytes = align_up(size_t(K) * size_t(p.lda_p) * 4);
    p.total = p.a_bytes + align_up(size_t(K) * size_t(p.ldb_p) * 4);
    return p;
}

// The pack is an optimisation: without room for it (caller workspace too
// small, or no memory) the kernel reads the operands as stored.
bool simt_pack_ws(gemm_context* h, const SimtPack& pk, uint8_t** ws) {
    *ws = nullptr;
    if (!pk.on || (h->user_ws && h->user_ws_bytes < pk.total)) return false;
    return get_ws(h, pk.total, ws) == GEMM_OK && *ws;
}

gemm_status_t run_simt(gemm_context* h, int transA, int transB, int64_t M, int64_t N, int64_t K,
                       float alpha, const float* A, int64_t lda, const float* B, int64_t ldb,
                       float beta, float* C, int64_t ldc, cudaStream_t s) {
    const SimtPack pk = plan_simt_pack(M, N, K);
    uint8_t* ws = nullptr;
    const bool pack = (!transA || transB) && simt_pack_ws(h, pk, &ws);
    int launches = 1;
    if (pack) {
        float* ap = reinterpret_cast<float*>(ws);
        float* bp = reinterpret_cast<float*>(ws + pk.a_bytes);
        if (!transA) {
            if (gb300::launch_transpose_f32(K, M, A, lda, ap, pk.lda_p, s) != cudaSuccess)
                return GEMM_ERR_CUDA;
            A = ap;
            lda = pk.lda_p;
            transA = GEMM_OP_T;
            ++launches;
        }
        if (transB) {
            if (gb300::launch_transpose_f32(K, N, B, ldb, bp, pk.ldb_p, s) != cudaSuccess)
                return GEMM_ERR_CUDA;
            B = bp;
            ldb = pk.ldb_p;
            transB = GEMM_OP_N;
            ++launches;
        }
    }
    h->last_launches = launches;
    ProfScope prof(h, s);
    return status_of(
        gb300::launch_simt_f32(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s));
}

gemm_status_t run_gemm(gemm_context* h, int transA, int transB, int64_t M, int64_t N, int64_t K,
                       float alpha, const float* A, int64_t lda, const float* B, int64_t ldb,
                       float beta, float* C, int64_t ldc, int mode, cudaStream_t s) {
    h->last_launches = 0;
    if (M == 0 || N == 0) return GEMM_OK;
    if (K == 0 || alpha == 0.0f) {
        h->last_launches = 1;
        return status_of(gb300::launch_scale_c(M, N, beta, C, ldc, s));
    }
    if (too_large(M, N, K)) return GEMM_ERR_UNSUPPORTED;
    if (mode == GEMM_MODE_F32_SIMT)
        return run_simt(h, transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s);
    const int nterms = mode == GEMM_MODE_BF16X3 ? 3 : 1;
    const int planes = nterms == 3 ? 2 : 1;
    const TcLaunch cfg = plan_tc(h, nterms, M, N, K, Call::Split, false, false, beta == 0.0f,
                                 (f32_tma_ok(A, lda) ? 1 : 0) | (f32_tma_ok(B, ldb) ? 2 : 0));
    // op(A) is M x K and op(B)^T is N x K, split K-major or as stored -- or,
    // with the in-kernel split (cfg.fuse bit 0 A, bit 1 B), read as stored in
    // FP32 and split on chip
    const bool fa = cfg.fuse & 1, fb = cfg.fuse & 2;
    const OpPlan pa = plan_op(M, K, transA == GEMM_OP_T, cfg);
    const OpPlan pb = plan_op(N, K, transB == GEMM_OP_N, cfg);
    const WsPlan w = plan_ws(planes, fa ? 0 : pa.lay.plane, fb ? 0 : pb.lay.plane, M, N, K, cfg,
                             h->num_sms);
    uint8_t* ws;
    gemm_status_t st = get_ws(h, w.total, &ws);
    if (st != GEMM_OK) return st;
    TcOperand oa, ob;
    int launches = 0;
    uint16_t* a_hi = reinterpret_cast<uint16_t*>(ws + w.a_off);
    uint16_t* b_hi = reinterpret_cast<uint16_t*>(ws + w.b_off);
    if (!fa && !fb) {  // both by the pass: one launch
        if (split_ops(pa, M, A, lda, a_hi, pb, N, B, ldb, b_hi, K, planes, s) != cudaSuccess)
            return GEMM_ERR_CUDA;
        launches = 1;
    } else if (!fa || !fb) {
        const bool a_pass = !fa;
        if ((a_pass ? split_op(pa, M, K, A, lda, a_hi, planes, s)
                    : split_op(pb, N, K, B, ldb, b_hi, planes, s)) != cudaSuccess)
            return GEMM_ERR_CUDA;
        launches = 1;
    }
    oa = fa ? f32_operand(A, lda, M, K, transA == GEMM_OP_T) : operand_of(pa, a_hi, M, K, planes);
    ob = fb ? f32_operand(B, ldb, N, K, transB == GEMM_OP_N) : operand_of(pb, b_hi, N, K, planes);
    TcLaunch c2 = cfg;
    c2.split_k = w.split;
    float* partial = w.split > 1 || w.tail ? reinterpret_cast<float*>(ws + w.p_off) : nullptr;
    int rc;
    {
        ProfScope prof(h, s);
        rc = gb300::launch_tc_gemm(oa, ob, nterms, M, N, K, alpha, beta, C, ldc, partial, c2,
                                   h->err_word, h->num_sms, s, &launches);
    }
    if (rc != 0) return static_cast<gemm_status_t>(rc);
    h->last_launches = launches;
    return GEMM_OK;
}

gemm_status_t grow(float** p, size_t* have, size_t want) {
    if (*have >= want) return GEMM_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *have = 0;
    if (cudaMalloc(reinterpret_cast<void**>(p), want) != cudaSuccess) {
        cudaGetLastError();
        return GEMM_ERR_WORKSPACE;
    }
    *have = want;
    return GEMM_OK;
}

}  // namespace

// Accessors for the grouped-plan translation unit (grouped.cu).
namespace gb300 {
int handle_device(gemm_handle_t h) { return h->device; }
int handle_num_sms(gemm_handle_t h) { return h->num_sms; }
int* handle_err_word(gemm_handle_t h) { return h->err_word; }
void handle_set_err_arg(gemm_handle_t h, int pos) { h->last_err_arg = pos; }
void handle_set_launches(gemm_handle_t h, int n) { h->last_launches = n; }
bool handle_tile_auto(gemm_handle_t h) {
    // no tile shape, ring depth or CTA grouping forced by the handle
    return h->cfg.bn == 0 && h->cfg.bk == 0 && h->cfg.stages == 0 && h->cfg.cta_group == 0;
}
int handle_split_place(gemm_handle_t h) { return h->cfg.split_place; }
int handle_split_k(gemm_handle_t h) { return h->cfg.split_k; }
TcLaunch handle_tc_config(gemm_handle_t h, int nterms) {
    // tile choice of the handle's configuration (problem-size independent
    // parts) for grouped launches
    TcLaunch c = plan_tc(h, nterms, 1 << 20, 1 << 20, 1, Call::Grouped);
    return c;
}
}  // namespace gb300

namespace {

// SYR2K workspace: the split planes of both operands in one buffer (X then Y,
// each P planes of the same packed layout) so that one tensor map reaches
// both matrices by plane index.
struct Syr2kPlan {
    OpPlan op;
    int planes;  // P per operand
    size_t bytes;
};

Syr2kPlan plan_syr2k(const gemm_context* h, int nterms, int trans, int64_t N, int64_t K,
                     TcLaunch* cfg) {
    *cfg = plan_tc(h, nterms, N, N, K, Call::Syr2k);
    cfg->split_k = 1;
    Syr2kPlan sp;
    sp.planes = nterms == 3 ? 2 : 1;
    // an operand stored K x N (trans) stays MN-major unless K-major is asked for
    sp.op = plan_op(N, K, trans == GEMM_OP_T, *cfg);
    sp.bytes = align_up(size_t(2 * sp.planes) * size_t(sp.op.lay.plane) * 2);
    return sp;
}

}  // namespace

extern "C" {

gemm_status_t gemm_create(gemm_handle_t* handle) {
    if (!handle) return GEMM_ERR_ARG;
    *handle = nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return GEMM_ERR_DEVICE;
    }
    int major = 0, minor = 0, sms = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (major != 10 || minor != 3) return GEMM_ERR_DEVICE;
    gemm_context* h = new (std::nothrow) gemm_context();
    if (!h) return GEMM_ERR_WORKSPACE;
    h->device = dev;
    h->num_sms = sms;
    if (cudaMalloc(reinterpret_cast<void**>(&h->err_word), 256) != cudaSuccess ||
        cudaMemset(h->err_word, 0, 256) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return GEMM_ERR_CUDA;
    }
    *handle = h;
    return GEMM_OK;
}

gemm_status_t gemm_destroy(gemm_handle_t h) {
    if (!h) return GEMM_OK;
    cudaDeviceSynchronize();
    cudaFree(h->err_word);
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    if (h->own_ws) cudaFree(h->own_ws);
    if (h->hA) cudaFree(h->hA);
    if (h->hB) cudaFree(h->hB);
    if (h->hC) cudaFree(h->hC);
    for (cudaStream_t st : h->pipe)
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t e : h->pipe_ev)
        if (e) cudaEventDestroy(e);
    delete h;
    return GEMM_OK;
}

gemm_status_t gemm_set_config(gemm_handle_t h, const gemm_config_t* cfg) {
    if (!h) return fail_arg(h, 1);
    h->last_err_arg = 0;
    if (!cfg) {
        h->cfg = gemm_config_t{};
        return GEMM_OK;
    }
    const gemm_config_t& c = *cfg;
    if ((c.bn != 0 && c.bn != 128 && c.bn != 256 && c.bn != 512) ||
        (c.bk != 0 && c.bk != 32 && c.bk != 64) || (c.bn == 512 && (c.cta_group == 1 || c.bk == 32)) ||
        c.stages < 0 || c.stages > 8 || c.stages == 1 || c.split_k < 0 || c.split_k > 64 ||
        c.raster_group < 0 || c.max_ctas < 0 || c.promote_k < -1 || c.cta_group < 0 ||
        c.cta_group > 2 || (c.cta_group == 2 && c.bn == 128) ||
        c.wait_poll_limit < 0 ||
        (c.operand_layout != GEMM_LAYOUT_AUTO && c.operand_layout != GEMM_LAYOUT_K_MAJOR &&
         c.operand_layout != GEMM_LAYOUT_AS_STORED) ||
        c.split_place < GEMM_SPLIT_AUTO || c.split_place > GEMM_SPLIT_IN_KERNEL_B ||
        (c.splitk_reduce != GEMM_SPLITK_AUTO && c.splitk_reduce != GEMM_SPLITK_LAUNCH) ||
        (c.split_place >= GEMM_SPLIT_IN_KERNEL &&
         ((c.bn != 0 && c.bn != 256) || (c.bk != 0 && c.bk != 32) || c.cta_group == 2)))
        return fail_arg(h, 2);
    h->cfg = c;
    return GEMM_OK;
}

size_t gemm_workspace_size(gemm_handle_t h, gemm_mode_t mode, gemm_op_t transA, gemm_op_t transB,
                           int64_t M, int64_t N, int64_t K) {
    if (!h || M < 0 || N < 0 || K < 0) return 0;
    if (M == 0 || N == 0 || K == 0) return 0;
    if ((transA != GEMM_OP_N && transA != GEMM_OP_T) || (transB != GEMM_OP_N && transB != GEMM_OP_T))
        return 0;
    if (mode == GEMM_MODE_F32_SIMT) return plan_simt_pack(M, N, K).total;
    if (mode != GEMM_MODE_BF16 && mode != GEMM_MODE_BF16X3) return 0;
    const int nterms = mode == GEMM_MODE_BF16X3 ? 3 : 1;
    // gemm() splits the operands the kernel does not split itself; gemm_bf16
    // needs at most as much (packs only).  Which operands the in-kernel split
    // takes depends on their alignment, unknown here: the largest plan over
    // the four cases (neither, A, B or both readable in place), with beta zero
    // or not (the plan weighs the C traffic), covers any call.
    size_t bytes = 0;
    for (int v = 0; v < (nterms == 3 ? 8 : 2); ++v) {
        const int f32_ops = v >> 1;
        const TcLaunch c =
            plan_tc(h, nterms, M, N, K, Call::Split, false, false, (v & 1) != 0, f32_ops);
        const OpPlan pa = plan_op(M, K, transA == GEMM_OP_T, c);
        const OpPlan pb = plan_op(N, K, transB == GEMM_OP_N, c);
        bytes = std::max(bytes, plan_ws(nterms == 3 ? 2 : 1, (c.fuse & 1) ? 0 : pa.lay.plane,
                                        (c.fuse & 2) ? 0 : pb.lay.plane, M, N, K, c, h->num_sms)
                                    .total);
    }
    if (nterms == 1) {
        // gemm_bf16's own plan: its tiles (and so a tail split) may be wider;
        // every MN-contiguous operand packed, beta zero or not
        const bool a_kr = transA == GEMM_OP_T, b_kr = transB == GEMM_OP_N;
        const gb300::PackedLayout la = gb300::packed_layout(M, K, false);
        const gb300::PackedLayout lb = gb300::packed_layout(N, K, false);
        for (int bz = 0; bz < 2; ++bz) {
            const TcLaunch c = plan_tc(h, 1, M, N, K, Call::Bf16, a_kr, b_kr, bz != 0);
            bytes = std::max(bytes, plan_ws(1, a_kr ? la.plane : 0, b_kr ? lb.plane : 0, M, N, K, c,
                                            h->num_sms)
                                        .total);
        }
    }
    return bytes;
}

gemm_status_t gemm_set_workspace(gemm_handle_t h, void* ws, size_t bytes) {
    if (!h) return fail_arg(h, 1);
    h->last_err_arg = 0;
    if (ws && (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0) return GEMM_ERR_ALIGN;
    h->user_ws = ws;
    h->user_ws_bytes = ws ? bytes : 0;
    return GEMM_OK;
}

gemm_status_t gemm(gemm_handle_t h, gemm_op_t transA, gemm_op_t transB, int64_t M, int64_t N,
                   int64_t K, float alpha, const float* A, int64_t lda, const float* B, int64_t ldb,
                   float beta, float* C, int64_t ldc, gemm_mode_t mode, void* stream) {
    gemm_status_t st = check_common(h, transA, transB, M, N, K, alpha, A, lda, B, ldb, C, ldc);
    if (st != GEMM_OK) return st;
    if (mode != GEMM_MODE_F32_SIMT && mode != GEMM_MODE_BF16 && mode != GEMM_MODE_BF16X3)
        return fail_arg(h, 15);
    return run_gemm(h, transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, mode,
                    static_cast<cudaStream_t>(stream));
}

gemm_status_t gemm_bf16(gemm_handle_t h, gemm_op_t transA, gemm_op_t transB, int64_t M, int64_t N,
                        int64_t K, float alpha, const uint16_t* A, int64_t lda, const uint16_t* B,
                        int64_t ldb, float beta, float* C, int64_t ldc, void* stream) {
    gemm_status_t st = check_common(h, transA, transB, M, N, K, alpha, A, lda, B, ldb, C, ldc);
    if (st != GEMM_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    h->last_launches = 0;
    if (M == 0 || N == 0) return GEMM_OK;
    if (K == 0 || alpha == 0.0f) {
        h->last_launches = 1;
        return status_of(gb300::launch_scale_c(M, N, beta, C, ldc, s));
    }
    if (too_large(M, N, K)) return GEMM_ERR_UNSUPPORTED;
    // K-contiguous operands (A stored M x K, B stored N x K) are read in place
    // by TMA; MN-contiguous ones (A stored K x M, B stored K x N) are read in
    // place as MN-major tiles, or packed K-contiguous first when the plan
    // wants K-major operands.
    const bool a_kr = transA == GEMM_OP_T, b_kr = transB == GEMM_OP_N;  // stored K x rows
    const TcLaunch cfg = plan_tc(h, 1, M, N, K, Call::Bf16, a_kr, b_kr, beta == 0.0f);
    auto misaligned = [](const void* p, int64_t ld) {
        return (reinterpret_cast<uintptr_t>(p) & 15) != 0 || ld % 8 != 0;
    };
    // With the library's layout choice an MN-contiguous operand that TMA
    // cannot read in place is packed instead of rejected.
    const bool lib_choice = h->cfg.operand_layout == GEMM_LAYOUT_AUTO;
    const bool pack_a = a_kr && (cfg.kmajor || (lib_choice && misaligned(A, lda)));
    const bool pack_b = b_kr && (cfg.kmajor || (lib_choice && misaligned(B, ldb)));
    if (!pack_a && misaligned(A, lda)) return GEMM_ERR_ALIGN;
    if (!pack_b && misaligned(B, ldb)) return GEMM_ERR_ALIGN;
    const gb300::PackedLayout la = gb300::packed_layout(M, K, false);
    const gb300::PackedLayout lb = gb300::packed_layout(N, K, false);
    const WsPlan w =
        plan_ws(1, pack_a ? la.plane : 0, pack_b ? lb.plane : 0, M, N, K, cfg, h->num_sms);
    uint8_t* ws;
    st = get_ws(h, w.total, &ws);
    if (st != GEMM_OK) return st;
    int launches = 0;
    TcOperand oa{A, M, K, lda, 0, 1};
    oa.mn_major = a_kr ? 1 : 0;
    TcOperand ob{B, N, K, ldb, 0, 1};
    ob.mn_major = b_kr ? 1 : 0;
    if (pack_a) {
        uint16_t* pa = reinterpret_cast<uint16_t*>(ws + w.a_off);
        if (gb300::launch_pack_bf16(1, M, K, A, lda, pa, la.ld, s) != cudaSuccess) return GEMM_ERR_CUDA;
        oa = TcOperand{pa, M, K, la.ld, la.plane, 1};
        ++launches;
    }
    if (pack_b) {
        uint16_t* pb = reinterpret_cast<uint16_t*>(ws + w.b_off);
        if (gb300::launch_pack_bf16(1, N, K, B, ldb, pb, lb.ld, s) != cudaSuccess) return GEMM_ERR_CUDA;
        ob = TcOperand{pb, N, K, lb.ld, lb.plane, 1};
        ++launches;
    }
    TcLaunch c2 = cfg;
    c2.split_k = w.split;
    float* partial = w.split > 1 || w.tail ? reinterpret_cast<float*>(ws + w.p_off) : nullptr;
    int rc;
    {
        ProfScope prof(h, s);
        rc = gb300::launch_tc_gemm(oa, ob, 1, M, N, K, alpha, beta, C, ldc, partial, c2,
                                   h->err_word, h->num_sms, s, &launches);
    }
    if (rc != 0) return static_cast<gemm_status_t>(rc);
    h->last_launches = launches;
    return GEMM_OK;
}

gemm_status_t gemm_split_bf16(gemm_handle_t h, gemm_op_t trans, int64_t rows, int64_t cols,
                              const float* X, int64_t ldx, uint16_t* hi, uint16_t* lo, int64_t ldo,
                              void* stream) {
    if (!h) return fail_arg(h, 1);
    h->last_err_arg = 0;
    h->last_launches = 0;
    if (trans != GEMM_OP_N && trans != GEMM_OP_T) return fail_arg(h, 2);
    if (rows < 0) return fail_arg(h, 3);
    if (cols < 0) return fail_arg(h, 4);
    const bool any = rows > 0 && cols > 0;
    if (any && !X) return fail_arg(h, 5);
    if (!ld_ok(ldx, trans ? rows : cols)) return fail_arg(h, 6);
    if (any && !hi) return fail_arg(h, 7);
    if (!ld_ok(ldo, cols)) return fail_arg(h, 9);
    if ((reinterpret_cast<uintptr_t>(hi) & 15) || (reinterpret_cast<uintptr_t>(lo) & 15) ||
        (ldo % 8))
        return GEMM_ERR_ALIGN;
    if (!any) return GEMM_OK;
    h->last_launches = 1;
    return status_of(gb300::launch_split_bf16(trans, rows, cols, X, ldx, hi, lo, ldo,
                                              static_cast<cudaStream_t>(stream)));
}

gemm_status_t gemm_from_host(gemm_handle_t h, gemm_op_t transA, gemm_op_t transB, int64_t M,
                             int64_t N, int64_t K, float alpha, const float* A, int64_t lda,
                             const float* B, int64_t ldb, float beta, float* C, int64_t ldc,
                             gemm_mode_t mode, void* stream) {
    gemm_status_t st = check_common(h, transA, transB, M, N, K, alpha, A, lda, B, ldb, C, ldc);
    if (st != GEMM_OK) return st;
    if (mode != GEMM_MODE_F32_SIMT && mode != GEMM_MODE_BF16 && mode != GEMM_MODE_BF16X3)
        return fail_arg(h, 15);
    if (M == 0 || N == 0) return GEMM_OK;
    if (too_large(M, N, K)) return GEMM_ERR_UNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((st = grow(&h->hC, &h->hC_bytes, size_t(M) * ldc * 4)) != GEMM_OK) return st;
    if (K == 0 || alpha == 0.0f) {  // C <- beta C: no operand copies
        if (beta != 0.0f && cudaMemcpy2DAsync(h->hC, ldc * 4, C, ldc * 4, N * 4, M,
                                              cudaMemcpyHostToDevice, s) != cudaSuccess)
            return GEMM_ERR_CUDA;
        if (gb300::launch_scale_c(M, N, beta, h->hC, ldc, s) != cudaSuccess ||
            cudaMemcpy2DAsync(C, ldc * 4, h->hC, ldc * 4, N * 4, M, cudaMemcpyDeviceToHost, s) !=
                cudaSuccess)
            return GEMM_ERR_CUDA;
        st = gemm_sync(h, stream);
        h->last_launches = 1;
        return st;
    }
    const int64_t ar = transA ? K : M;
    const int64_t br = transB ? N : K, bc = transB ? K : N;
    if ((st = grow(&h->hA, &h->hA_bytes, size_t(ar) * lda * 4)) != GEMM_OK) return st;
    if ((st = grow(&h->hB, &h->hB_bytes, size_t(br) * ldb * 4)) != GEMM_OK) return st;
    for (cudaStream_t& q : h->pipe)
        if (!q && cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking) != cudaSuccess)
            return GEMM_ERR_CUDA;
    for (cudaEvent_t& e : h->pipe_ev)
        if (!e && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            return GEMM_ERR_CUDA;

    // Three-stage pipeline over row blocks of op(A) and C, one stream per
    // stage so that no stage waits behind another in stream order:
    //   copy-in  (pipe[0]): B, then A_i and C_i of every block back to back;
    //   compute  (pipe[1]): split B, then per block split A_i and multiply;
    //   copy-out (pipe[2]): C_i as soon as its product is done.
    // The host link then stays busy from the first byte, C_i travels back
    // while later blocks travel in, and only the last block's product and
    // copy-out follow the last input byte.
    const int nb = int(std::min<int64_t>(kPipeBlocks, std::max<int64_t>(1, M / 512)));
    const int64_t rb = ((M + nb - 1) / nb + 127) / 128 * 128;
    const bool tc = mode != GEMM_MODE_F32_SIMT;
    const int nterms = mode == GEMM_MODE_BF16X3 ? 3 : 1;
    const int planes = nterms == 3 ? 2 : 1;
    TcLaunch cfg = plan_tc(h, nterms, rb, N, K, Call::Split);  // split pass (no f32_ok)
    cfg.split_k = 1;
    const OpPlan pa = plan_op(M, K, transA == GEMM_OP_T, cfg);
    const OpPlan pb = plan_op(N, K, transB == GEMM_OP_N, cfg);
    WsPlan w{};
    uint8_t* ws = nullptr;
    if (tc) {
        w = plan_ws(planes, pa.lay.plane, pb.lay.plane, M, N, K, cfg);
        if ((st = get_ws(h, w.total, &ws)) != GEMM_OK) return st;
    }
    uint16_t* a_hi = reinterpret_cast<uint16_t*>(ws + w.a_off);
    uint16_t* b_hi = reinterpret_cast<uint16_t*>(ws + w.b_off);
    cudaStream_t s_in = h->pipe[0], s_mm = h->pipe[1], s_out = h->pipe[2];
    cudaEvent_t ev_start = h->pipe_ev[0], ev_b = h->pipe_ev[1], ev_end = h->pipe_ev[2];
    cudaEvent_t* ev_in = h->pipe_ev + 3;               // [kPipeBlocks]
    cudaEvent_t* ev_done = h->pipe_ev + 3 + kPipeBlocks;  // [kPipeBlocks]
    int launches = 0;
    // everything earlier on the caller's stream comes first
    if (cudaEventRecord(ev_start, s) != cudaSuccess ||
        cudaStreamWaitEvent(s_in, ev_start, 0) != cudaSuccess ||
        cudaStreamWaitEvent(s_mm, ev_start, 0) != cudaSuccess ||
        cudaStreamWaitEvent(s_out, ev_start, 0) != cudaSuccess)
        return GEMM_ERR_CUDA;
    if (cudaMemcpy2DAsync(h->hB, ldb * 4, B, ldb * 4, bc * 4, br, cudaMemcpyHostToDevice, s_in) !=
            cudaSuccess ||
        cudaEventRecord(ev_b, s_in) != cudaSuccess || cudaStreamWaitEvent(s_mm, ev_b, 0) != cudaSuccess)
        return GEMM_ERR_CUDA;
    if (tc) {
        if (split_op(pb, N, K, h->hB, ldb, b_hi, planes, s_mm) != cudaSuccess) return GEMM_ERR_CUDA;
        ++launches;
    }
    for (int i = 0; i < nb; ++i) {
        const int64_t r0 = i * rb;
        if (r0 >= M) break;
        const int64_t rows = std::min(rb, M - r0);
        // copy-in: rows r0.. of op(A) (stored rows of A, or stored columns
        // when transposed) and of C
        const size_t aoff = transA ? size_t(r0) : size_t(r0) * lda;
        const cudaError_t ce =
            transA ? cudaMemcpy2DAsync(h->hA + aoff, lda * 4, A + aoff, lda * 4, rows * 4, K,
                                       cudaMemcpyHostToDevice, s_in)
                   : cudaMemcpy2DAsync(h->hA + aoff, lda * 4, A + aoff, lda * 4, K * 4, rows,
                                       cudaMemcpyHostToDevice, s_in);
        if (ce != cudaSuccess) return GEMM_ERR_CUDA;
        float* cblk = h->hC + size_t(r0) * ldc;
        if (beta != 0.0f && cudaMemcpy2DAsync(cblk, ldc * 4, C + size_t(r0) * ldc, ldc * 4, N * 4,
                                              rows, cudaMemcpyHostToDevice, s_in) != cudaSuccess)
            return GEMM_ERR_CUDA;
        if (cudaEventRecord(ev_in[i], s_in) != cudaSuccess ||
            cudaStreamWaitEvent(s_mm, ev_in[i], 0) != cudaSuccess)
            return GEMM_ERR_CUDA;
        // compute
        if (tc) {
            // the block's rows inside the packed A: packed rows (K-major) or
            // columns (MN-major; r0 is a multiple of 128, so 16-byte aligned)
            uint16_t* ablk = a_hi + (pa.mn ? r0 : r0 * pa.lay.ld);
            if (split_op(pa, rows, K, h->hA + aoff, lda, ablk, planes, s_mm) != cudaSuccess)
                return GEMM_ERR_CUDA;
            const TcOperand oa = operand_of(pa, ablk, rows, K, planes);
            const TcOperand ob = operand_of(pb, b_hi, N, K, planes);
            int n = 0;
            const int rc = gb300::launch_tc_gemm(oa, ob, nterms, rows, N, K, alpha, beta, cblk, ldc,
                                                 nullptr, cfg, h->err_word, h->num_sms, s_mm, &n);
            if (rc != 0) return static_cast<gemm_status_t>(rc);
            launches += 1 + n;
        } else {
            if (gb300::launch_simt_f32(transA, transB, rows, N, K, alpha, h->hA + aoff, lda, h->hB,
                                       ldb, beta, cblk, ldc, s_mm) != cudaSuccess)
                return GEMM_ERR_CUDA;
            ++launches;
        }
        // copy-out
        if (cudaEventRecord(ev_done[i], s_mm) != cudaSuccess ||
            cudaStreamWaitEvent(s_out, ev_done[i], 0) != cudaSuccess ||
            cudaMemcpy2DAsync(C + size_t(r0) * ldc, ldc * 4, cblk, ldc * 4, N * 4, rows,
                              cudaMemcpyDeviceToHost, s_out) != cudaSuccess)
            return GEMM_ERR_CUDA;
    }
    // the copy-out stream ends after every product (it waited on each) and
    // every product after its inputs: joining it joins the whole pipeline
    if (cudaEventRecord(ev_end, s_out) != cudaSuccess ||
        cudaStreamWaitEvent(s, ev_end, 0) != cudaSuccess)
        return GEMM_ERR_CUDA;
    st = gemm_sync(h, stream);
    h->last_launches = launches;
    return st;
}

gemm_status_t gemm_backward(gemm_handle_t h, gemm_op_t transA, gemm_op_t transB, int64_t M,
                            int64_t N, int64_t K, const float* dC, int64_t lddc, const float* A,
                            int64_t lda, const float* B, int64_t ldb, float* dA, int64_t ldda,
                            float* dB, int64_t lddb, gemm_mode_t mode, void* stream) {
    if (!h) return fail_arg(h, 1);
    h->last_err_arg = 0;
    if (transA != GEMM_OP_N && transA != GEMM_OP_T) return fail_arg(h, 2);
    if (transB != GEMM_OP_N && transB != GEMM_OP_T) return fail_arg(h, 3);
    if (M < 0) return fail_arg(h, 4);
    if (N < 0) return fail_arg(h, 5);
    if (K < 0) return fail_arg(h, 6);
    const bool any = M > 0 && N > 0 && K > 0;
    if (any && !dC) return fail_arg(h, 7);
    if (!ld_ok(lddc, N)) return fail_arg(h, 8);
    if (any && dA == nullptr && dB == nullptr) return GEMM_OK;
    if (any && dB && !A) return fail_arg(h, 9);
    if (!ld_ok(lda, transA ? M : K)) return fail_arg(h, 10);
    if (any && dA && !B) return fail_arg(h, 11);
    if (!ld_ok(ldb, transB ? K : N)) return fail_arg(h, 12);
    if (dA && !ld_ok(ldda, transA ? M : K)) return fail_arg(h, 14);
    if (dB && !ld_ok(lddb, transB ? K : N)) return fail_arg(h, 16);
    if (mode != GEMM_MODE_F32_SIMT && mode != GEMM_MODE_BF16 && mode != GEMM_MODE_BF16X3)
        return fail_arg(h, 17);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int total = 0;
    gemm_status_t st = GEMM_OK;
    if (dA) {
        // dA = dC op(B)^T (M x K); stored transposed when transA == T.
        if (transA == GEMM_OP_N)
            st = run_gemm(h, GEMM_OP_N, !transB, M, K, N, 1.0f, dC, lddc, B, ldb, 0.0f, dA, ldda,
                          mode, s);
        else
            st = run_gemm(h, transB, GEMM_OP_T, K, M, N, 1.0f, B, ldb, dC, lddc, 0.0f, dA, ldda,
                          mode, s);
        if (st != GEMM_OK) return st;
        total += h->last_launches;
    }
    if (dB) {
        // dB = op(A)^T dC (K x N); stored transposed when transB == T.
        if (transB == GEMM_OP_N)
            st = run_gemm(h, !transA, GEMM_OP_N, K, N, M, 1.0f, A, lda, dC, lddc, 0.0f, dB, lddb,
                          mode, s);
        else
            st = run_gemm(h, GEMM_OP_T, transA, N, K, M, 1.0f, dC, lddc, A, lda, 0.0f, dB, lddb,
                          mode, s);
        if (st != GEMM_OK) return st;
        total += h->last_launches;
    }
    h->last_launches = total;
    return GEMM_OK;
}

size_t gemm_syr2k_workspace_size(gemm_handle_t h, gemm_mode_t mode, gemm_op_t trans, int64_t N,
                                 int64_t K) {
    if (!h || N <= 0 || K <= 0) return 0;
    if (trans != GEMM_OP_N && trans != GEMM_OP_T) return 0;
    if (mode == GEMM_MODE_F32_SIMT) return plan_simt_pack(N, N, K).total;
    if (mode != GEMM_MODE_BF16 && mode != GEMM_MODE_BF16X3) return 0;
    TcLaunch cfg;
    return plan_syr2k(h, mode == GEMM_MODE_BF16X3 ? 3 : 1, trans, N, K, &cfg).bytes;
}

gemm_status_t gemm_syr2k(gemm_handle_t h, gemm_uplo_t uplo, gemm_op_t trans, int64_t N, int64_t K,
                         float alpha, const float* A, int64_t lda, const float* B, int64_t ldb,
                         float beta, float* C, int64_t ldc, gemm_mode_t mode, void* stream) {
    if (!h) return fail_arg(h, 1);
    h->last_err_arg = 0;
    h->last_launches = 0;
    if (uplo != GEMM_LOWER && uplo != GEMM_UPPER) return fail_arg(h, 2);
    if (trans != GEMM_OP_N && trans != GEMM_OP_T) return fail_arg(h, 3);
    if (N < 0) return fail_arg(h, 4);
    if (K < 0) return fail_arg(h, 5);
    const bool reads_ab = N > 0 && K > 0 && alpha != 0.0f;
    if (reads_ab && !A) return fail_arg(h, 7);
    if (!ld_ok(lda, trans ? N : K)) return fail_arg(h, 8);
    if (reads_ab && !B) return fail_arg(h, 9);
    if (!ld_ok(ldb, trans ? N : K)) return fail_arg(h, 10);
    if (N > 0 && !C) return fail_arg(h, 12);
    if (!ld_ok(ldc, N)) return fail_arg(h, 13);
    if (mode != GEMM_MODE_F32_SIMT && mode != GEMM_MODE_BF16 && mode != GEMM_MODE_BF16X3)
        return fail_arg(h, 14);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int tri = uplo == GEMM_LOWER ? 1 : 2;
    if (N == 0) return GEMM_OK;
    if (!reads_ab) {  // C <- beta C on the triangle
        h->last_launches = 1;
        return status_of(gb300::launch_scale_c(N, N, beta, C, ldc, s, tri));
    }
    if (too_large(N, N, 2 * K)) return GEMM_ERR_UNSUPPORTED;
    if (mode == GEMM_MODE_F32_SIMT) {
        // X, Y stored N x K: packed into K x N copies first (as in gemm()),
        // and the kernel runs its trans == T form
        const SimtPack pk = plan_simt_pack(N, N, K);
        uint8_t* ws = nullptr;
        int launches = 1;
        if (trans == GEMM_OP_N && simt_pack_ws(h, pk, &ws)) {
            float* xp = reinterpret_cast<float*>(ws);
            float* yp = reinterpret_cast<float*>(ws + pk.a_bytes);
            if (gb300::launch_transpose_f32(K, N, A, lda, xp, pk.lda_p, s) != cudaSuccess ||
                gb300::launch_transpose_f32(K, N, B, ldb, yp, pk.ldb_p, s) != cudaSuccess)
                return GEMM_ERR_CUDA;
            A = xp;
            lda = pk.lda_p;
            B = yp;
            ldb = pk.ldb_p;
            trans = GEMM_OP_T;
            launches = 3;
        }
        h->last_launches = launches;
        ProfScope prof(h, s);
        return status_of(gb300::launch_simt_syr2k(tri, trans, N, K, alpha, A, lda, B, ldb, beta, C,
                                                  ldc, s));
    }
    const int nterms = mode == GEMM_MODE_BF16X3 ? 3 : 1;
    TcLaunch cfg;
    const Syr2kPlan sp = plan_syr2k(h, nterms, trans, N, K, &cfg);
    uint8_t* ws;
    gemm_status_t st = get_ws(h, sp.bytes, &ws);
    if (st != GEMM_OK) return st;
    uint16_t* x_hi = reinterpret_cast<uint16_t*>(ws);
    uint16_t* y_hi = x_hi + size_t(sp.planes) * size_t(sp.op.lay.plane);
    if (split_ops(sp.op, N, A, lda, x_hi, sp.op, N, B, ldb, y_hi, K, sp.planes, s) != cudaSuccess)
        return GEMM_ERR_CUDA;
    TcOperand xy = operand_of(sp.op, x_hi, N, K, 2 * sp.planes);
    xy.box_planes = sp.planes;
    int launches = 1;
    int rc;
    {
        ProfScope prof(h, s);
        rc = gb300::launch_tc_syr2k(xy, nterms, tri, N, K, alpha, beta, C, ldc, cfg, h->err_word,
                                    h->num_sms, s, &launches);
    }
    if (rc != 0) return static_cast<gemm_status_t>(rc);
    h->last_launches = launches;
    return GEMM_OK;
}

gemm_status_t gemm_profile_enable(gemm_handle_t h, int enable) {
    if (!h) return fail_arg(h, 1);
    h->profiling = enable != 0;
    h->ev_used = 0;
    return GEMM_OK;
}

gemm_status_t gemm_profile_read(gemm_handle_t h, double* main_ms, int* main_launches) {
    if (!h) return fail_arg(h, 1);
    if (!main_ms) return fail_arg(h, 2);
    if (!main_launches) return fail_arg(h, 3);
    double total = 0.0;
    int n = 0;
    for (size_t i = 0; i + 1 < h->ev_used; i += 2) {
        if (cudaEventSynchronize(h->ev_pool[i + 1]) != cudaSuccess) {
            cudaGetLastError();
            return GEMM_ERR_CUDA;
        }
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, h->ev_pool[i], h->ev_pool[i + 1]) != cudaSuccess) {
            cudaGetLastError();
            return GEMM_ERR_CUDA;
        }
        total += ms;
        ++n;
    }
    h->ev_used = 0;
    *main_ms = total;
    *main_launches = n;
    return GEMM_OK;
}

gemm_status_t gemm_profile_read_each(gemm_handle_t h, float* ms, int capacity, int* count) {
    if (!h) return fail_arg(h, 1);
    if (!ms && capacity > 0) return fail_arg(h, 2);
    if (capacity < 0) return fail_arg(h, 3);
    if (!count) return fail_arg(h, 4);
    int n = 0;
    for (size_t i = 0; i + 1 < h->ev_used; i += 2) {
        if (cudaEventSynchronize(h->ev_pool[i + 1]) != cudaSuccess) {
            cudaGetLastError();
            return GEMM_ERR_CUDA;
        }
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, h->ev_pool[i], h->ev_pool[i + 1]) != cudaSuccess) {
            cudaGetLastError();
            return GEMM_ERR_CUDA;
        }
        if (n < capacity) ms[n] = t;
        ++n;
    }
    h->ev_used = 0;
    *count = n;
    return GEMM_OK;
}

gemm_status_t gemm_sync(gemm_handle_t h, void* stream) {
    if (!h) return fail_arg(h, 1);
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GEMM_ERR_CUDA;
    }
    int word = 0;
    if (cudaMemcpy(&word, h->err_word, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return GEMM_ERR_CUDA;
    if (word != 0) {
        cudaMemset(h->err_word, 0, sizeof(int));
        return GEMM_ERR_TIMEOUT;
    }
    return GEMM_OK;
}

int gemm_last_error_arg(gemm_handle_t h) { return h ? h->last_err_arg : 1; }

gemm_status_t gemm_get_last_error_arg(gemm_handle_t h, int* pos) {
    if (!h) {
        if (pos) *pos = 1;
        return GEMM_ERR_ARG;
    }
    if (!pos) return GEMM_ERR_ARG;  // the handle keeps its recorded position
    *pos = h->last_err_arg;
    return GEMM_OK;
}

int gemm_last_launch_count(gemm_handle_t h) { return h ? h->last_launches : 0; }

const char* gemm_status_string(gemm_status_t s) {
    switch (s) {
        case GEMM_OK: return "GEMM_OK";
        case GEMM_ERR_ARG: return "GEMM_ERR_ARG: invalid argument";
        case GEMM_ERR_ALIGN: return "GEMM_ERR_ALIGN: operand not 16-byte aligned";
        case GEMM_ERR_WORKSPACE: return "GEMM_ERR_WORKSPACE: workspace too small or allocation failed";
        case GEMM_ERR_CUDA: return "GEMM_ERR_CUDA: CUDA call failed";
        case GEMM_ERR_TIMEOUT: return "GEMM_ERR_TIMEOUT: a kernel's bounded wait expired";
        case GEMM_ERR_UNSUPPORTED: return "GEMM_ERR_UNSUPPORTED: not supported by this build";
        case GEMM_ERR_DEVICE: return "GEMM_ERR_DEVICE: current device is not sm_103";
    }
    return "unknown gemm_status_t";
}

}  // extern "C"
