// Tensor-core GEMM for sm_103a: TMA -> shared-memory ring -> tcgen05.mma
// into tensor memory -> alpha/beta epilogue.
//
// This is the GPU form of Algorithm 1 (Kuzma et al., Section 3):
//  * the paper's pack() calls (Algorithm 1, packing of A and B blocks into
//    tile order, Section 3.1) become TMA tensor loads that drop swizzled
//    BM x BK and BN x BK tiles into a multi-stage shared-memory ring, either
//    K-major (operand rows K-contiguous) or MN-major (an operand stored
//    K x rows, read as 64-wide row groups without a transposing pass);
//  * the j/i block loops become a persistent tile scheduler: each CTA walks
//    output tiles t = blockIdx.x, blockIdx.x + gridDim.x, ... in an order
//    that keeps `raster_group` M tiles per B panel together (the paper's
//    "pack B once, reuse it over all i");
//  * the kk loop of llvm.matrix.multiply calls (Algorithm 2: outer-product
//    MACs into accumulators that never spill, hardware constraint 5) becomes
//    tcgen05.mma issued by one thread into a TMEM accumulator that lives for
//    the whole K loop;
//  * the alpha/beta update of the C tile (Algorithm 1, beta once, alpha on
//    the product) is the epilogue, which reads TMEM with tcgen05.ld.
//
// Split-precision (nterms == 3, not in the paper): every stage holds the hi
// and lo planes of both operands and each 16-deep K slice issues
// acc += Alo*Bhi; acc += Ahi*Blo; acc += Ahi*Bhi (small terms first).
//
// Warp roles (320 threads): warp 0 = TMA producer, warp 1 = TMEM owner and
// MMA issuer, warps 2-9 = epilogue (warp w reads TMEM lanes 32*(w%4)..+31
// and one half of the tile's columns); the plain-BF16 CTA-pair kernel adds
// warp 10, which issues the B copies (352 threads).  With the in-kernel
// split (FUSE, 640 threads) the epilogue is warps 4-11 and warps 2-3 and
// 12-19 split FP32 stages into hi/lo in shared memory.
// Two accumulators (2 x BN TMEM columns) let the epilogue of tile i overlap
// the MMAs of tile i+1.  Every wait is bounded (ptx.cuh); on expiry the
// kernel records the error, drains its own copies and MMAs, frees TMEM and
// returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <mutex>

#include "internal.h"
#include "ptx.cuh"
#include "split_bf16.cuh"

namespace gb300 {

namespace {

constexpr int kBM = 128;
constexpr int kEpiWarps = 8;               // warps 2..9
constexpr int kThreads = 64 + 32 * kEpiWarps;  // producer, MMA, epilogue
// In-kernel split (FUSE): 20 warps in five warpgroups -- warp 0 producer,
// warp 1 MMA, warps 2-3 and 12-19 split FP32 stages into hi/lo in place,
// warps 4-11 epilogue.  Registers are handed to a CTA per warpgroup: the
// block gets 96 a thread at launch (65536 / 640, in steps of 8), and
// setmaxnreg moves them to the epilogue warpgroups, 168 a thread (128
// running FP32 sums), from the others, 48: 256 x 168 + 384 x 48 = 640 x 96.
constexpr int kFusedThreads = 640;
constexpr int kConvWarps = 10;
constexpr int kFusedEpi0 = 4;  // first epilogue warp
constexpr int kFusedEpiRegs = 168;
constexpr int kFusedOtherRegs = 48;
static_assert(256 * kFusedEpiRegs + (kFusedThreads - 256) * kFusedOtherRegs <=
                  (65536 / kFusedThreads) / 8 * 8 * kFusedThreads,
              "register split must fit what the block is launched with");
constexpr int kMaxSmem = 232448;  // 227 KB opt-in dynamic shared memory per block

struct TcParams {
    int M, N, K;
    float alpha, beta;
    float* C;
    long long ldc;
    int num_m, num_n, num_tiles, k_blocks;
    int split_k, kb_per_split;
    int chunk_kb;    // k-blocks per accumulation chunk (PROMOTE)
    float* partial;  // split_k > 1: split_k slabs of M x N
    int stages;
    int raster_group;
    WaitLimit lim;
    int* err;
    // grouped launches: problem table (prefix-summed tile starts) and two
    // tensor maps per problem (A then B), all in device memory
    const GroupedProblem* problems;
    const CUtensorMap* maps;
    const int* tile_prob;  // problem index of every tile
    int count;
    int c_tma;  // epilogue writes through the C tensor map (beta == 0 or split-K partials)
    int fuse_ops;  // FUSE: bit 0 A, bit 1 B arrives as FP32 and is split in the kernel
    int cluster_k;  // > 1: split-K slices of a tile run as one cluster and sum in the kernel
    int sum_vec;    // cluster_k: the sum may use float4 (N, ldc % 4 == 0, C 16-byte aligned)
    int ring_epi;   // cluster_k with TMA partials: the ring holds every partial piece at once
    int own_local;  // ring_epi, sum_vec, cluster_k 2 or 4: a CTA's own rows of its slice stay
                    // in its ring (only it sums them) and are not stored
    int maj;    // single launches: bit 0 A MN-major, bit 1 B MN-major
    // SYR2K (single launches): uplo 1 = lower, 2 = upper triangle of C (0 =
    // plain GEMM); syr_kb = K blocks of one product (the K loop runs twice as
    // far: A-side rows then B-side rows); syr_plane = plane index where the
    // second matrix's planes start in the shared operand buffer
    int uplo;
    int syr_kb;
    int syr_plane;
    int tri_r;  // BN / 128
    // Tail split (CTA-pair launches with one K slice): when the tiles leave
    // a last wave with at most half the pairs busy, tiles tail_base ..
    // tail_base + tail_n - 1 are each computed in two halves of their K
    // blocks, the even ones by unit tail_base + i and the odd ones by unit
    // tail_base + tail_n + i, in parallel (both sweep the whole K range, so
    // both find the previous wave's operand blocks in L2); each half stores
    // its raw partial tile (2 kBM rows of BN floats) at tail_part +
    // (2 i + half) tiles, and tail_reduce_kernel adds the two into C.
    // tail_n 0: none.
    int tail_base;
    int tail_n;
    float* tail_part;
};

template <int BN, int BK, int NTERMS>
struct Shape {
    static constexpr int PLANES = NTERMS == 1 ? 1 : 2;
    static constexpr int A_PLANE = kBM * BK * 2;
    static constexpr int B_PLANE = BN * BK * 2;
    static constexpr int STAGE = PLANES * (A_PLANE + B_PLANE);
    static constexpr int TMEM_COLS = 2 * BN;  // two FP32 accumulators
    static constexpr int ROW_BYTES = BK * 2;  // 64 (SW64) or 128 (SW128)
    // MN-major operands: 64-element MN groups of all planes (each plane BK
    // rows of 128 bytes), one TMA box each, MN_GROUP bytes apart
    static constexpr int MN_GROUP = PLANES * BK * 128;
    static constexpr int BAR_BYTES = 1024;    // barriers + TMEM slot + abort flag
    static constexpr int STAGING = kEpiWarps * 32 * 33 * 4;  // epilogue store slabs
    static_assert(ROW_BYTES == 64 || ROW_BYTES == 128, "BK must be 32 or 64");
    static_assert(BN % 32 == 0 && BN >= 32 && BN <= 256, "BN");
    static_assert(TMEM_COLS == 256 || TMEM_COLS == 512, "TMEM allocation is a power of two");
    static int smem_bytes(int stages) { return 1024 + stages * STAGE + BAR_BYTES + STAGING; }
    static int max_stages() {
        int s = (kMaxSmem - 1024 - BAR_BYTES - STAGING) / STAGE;
        return s > 8 ? 8 : s;
    }
};

// Where output tile t sits: coordinates, K-block range, operand maps.
struct TileInfo {
    int mt, nt, ks, kb0, kb1;
    int kstep = 1, koff = 0;  // K block j of the tile is block koff + kstep * j of the operands
    int prob;  // problem index (grouped launches)
    int maj;   // bit 0: A MN-major, bit 1: B MN-major
    const CUtensorMap* ma;
    const CUtensorMap* mb;
};

// The output side of a tile's problem (looked up only where it is used, so
// that it does not occupy registers across the K loop).
struct EpiInfo {
    int M, N;
    float alpha, beta;
    float* C;
    long long ldc;
    int uplo;  // 1: store only col <= row, 2: only col >= row (SYR2K)
    int r_off = 0, c_off = 0;  // C holds the tile from row r_off, column c_off (tail partials)
};

// Local tile index -> (m tile, n tile): groups of `g` M tiles are walked
// N-tile by N-tile, so concurrently running CTAs share B panels in L2.
__device__ __forceinline__ void raster(int t, int num_m, int num_n, int g, int& mt, int& nt) {
    const int group = g * num_n;
    const int first_m = (t / group) * g;
    const int gm = min(num_m - first_m, g);
    const int r = t % group;
    mt = first_m + r % gm;
    nt = r / gm;
}

// SYR2K tile space: only the 128 x BN tiles that meet the stored triangle,
// row of tiles by row of tiles.  With r = BN / 128, tile row mt needs the
// column tiles nt <= mt / r (lower) or nt >= mt / r (upper), so the number
// of tiles in rows 0 .. m-1 is F(m) + m (lower) or m * num_n - F(m)
// (upper), F(m) = sum_{i<m} floor(i / r).
__device__ __forceinline__ int tri_floor_sum(int m, int r) {
    if (r == 1) return m * (m - 1) / 2;
    const int q = m >> 1;
    return q * (q - 1) + ((m & 1) ? q : 0);
}

__device__ __forceinline__ int tri_tiles_before(int m, int r, int uplo, int num_n) {
    return uplo == 1 ? tri_floor_sum(m, r) + m : m * num_n - tri_floor_sum(m, r);
}

__device__ __forceinline__ void tri_tile(int t, int num_m, int num_n, int r, int uplo, int& mt,
                                         int& nt) {
    int lo = 0, hi = num_m;  // tiles_before(lo) <= t < tiles_before(hi)
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (tri_tiles_before(mid, r, uplo, num_n) <= t)
            lo = mid;
        else
            hi = mid;
    }
    mt = lo;
    nt = t - tri_tiles_before(lo, r, uplo, num_n) + (uplo == 1 ? 0 : lo / r);
}

template <bool GROUPED>
__device__ __forceinline__ TileInfo get_tile(int t, const TcParams& p, const CUtensorMap* tmA,
                                             const CUtensorMap* tmB) {
    TileInfo ti;
    if (!GROUPED && p.uplo) {
        ti.ks = 0;
        tri_tile(t, p.num_m, p.num_n, p.tri_r, p.uplo, ti.mt, ti.nt);
        ti.kb0 = 0;
        ti.kb1 = p.k_blocks;
        ti.prob = 0;
        ti.maj = p.maj;
        ti.ma = tmA;
        ti.mb = tmB;
    } else if (!GROUPED) {
        int tt = t, half = -1;  // tail split: the tile of unit t and which K half
        if (p.tail_n > 0 && t >= p.tail_base) {
            const int u = t - p.tail_base;
            half = u / p.tail_n;
            tt = p.tail_base + u % p.tail_n;
        }
        const int per_split = p.num_m * p.num_n;
        ti.ks = tt / per_split;
        raster(tt - ti.ks * per_split, p.num_m, p.num_n, p.raster_group, ti.mt, ti.nt);
        ti.kb0 = ti.ks * p.kb_per_split;
        ti.kb1 = min(ti.kb0 + p.kb_per_split, p.k_blocks);
        ti.prob = 0;
        if (half >= 0) {  // prob: 1 + tail index, ks: the half (even or odd K blocks)
            ti.kb0 = 0;
            ti.kb1 = (p.k_blocks - half + 1) / 2;
            ti.kstep = 2;
            ti.koff = half;
            ti.ks = half;
            ti.prob = 1 + (tt - p.tail_base);
        }
        ti.maj = p.maj;
        ti.ma = tmA;
        ti.mb = tmB;
    } else {
        const int lo = __ldg(&p.tile_prob[t]);
        const GroupedProblem* q = p.problems + lo;
        ti.ks = 0;
        raster(t - __ldg(&q->tile_start), __ldg(&q->num_m), __ldg(&q->num_n), p.raster_group,
               ti.mt, ti.nt);
        ti.kb0 = 0;
        ti.kb1 = __ldg(&q->k_blocks);
        ti.prob = lo;
        ti.maj = __ldg(&q->major);
        ti.ma = p.maps + 2 * lo;
        ti.mb = p.maps + 2 * lo + 1;
    }
    return ti;
}

// Split-K launches write raw partial sums: their "C" is slab ks of the
// partial buffer with alpha = 1, beta = 0.
template <bool GROUPED>
__device__ __forceinline__ EpiInfo get_epi(int prob, int ks, const TcParams& p) {
    EpiInfo e;
    if (!GROUPED) {
        e.M = p.M;
        e.N = p.N;
        if (p.split_k > 1) {
            e.alpha = 1.0f;
            e.beta = 0.0f;
            e.C = p.partial + size_t(ks) * size_t(p.M) * size_t(p.N);
            e.ldc = p.N;
        } else {
            e.alpha = p.alpha;
            e.beta = p.beta;
            e.C = p.C;
            e.ldc = p.ldc;
        }
        e.uplo = p.uplo;
    } else {
        const GroupedProblem* q = p.problems + prob;
        e.M = __ldg(&q->M);
        e.N = __ldg(&q->N);
        e.alpha = __ldg(&q->alpha);
        e.beta = __ldg(&q->beta);
        e.C = q->C;
        e.ldc = __ldg(&q->ldc);
        e.uplo = 0;
    }
    return e;
}

// Store a 32 x 32 piece of the tile: lane l holds v[0..31] = row (row0 + l),
// columns col0 .. col0+31.  The piece goes through this warp's padded
// shared-memory slab so that the global accesses are coalesced: in step rr
// the warp writes row (row0 + rr), 32 consecutive columns, one per lane.
// Reads of C are issued eight at a time so that their latencies overlap.
// Split-K stores raw FP32 partial sums; otherwise C = alpha*v + beta*C
// (C not read when beta == 0).  SYR2K (e.uplo) stores only the elements of
// its triangle: lane `col` keeps the piece rows [rlo, rhi).
__device__ __forceinline__ void store_piece(const float* v, float* stg, int row0, int col0,
                                            const EpiInfo& e, int lane) {
#pragma unroll
    for (int j = 0; j < 32; ++j) stg[lane * 33 + j] = v[j];
    __syncwarp();
    const int col = col0 + lane;
    int rlo = 0, rhi = min(32, e.M - row0);
    if (e.uplo == 1) rlo = max(0, col - row0);           // col <= row
    if (e.uplo == 2) rhi = min(rhi, col - row0 + 1);      // col >= row
    if (col < e.N) {
        float* base = e.C + size_t(row0 - e.r_off) * size_t(e.ldc) + (col - e.c_off);
        const size_t ldc = size_t(e.ldc);
        if (e.beta != 0.0f) {
#pragma unroll
            for (int r0 = 0; r0 < 32; r0 += 8) {
                float old[8];
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    old[i] = (r0 + i >= rlo && r0 + i < rhi) ? base[(r0 + i) * ldc] : 0.0f;
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    if (r0 + i >= rlo && r0 + i < rhi)
                        base[(r0 + i) * ldc] =
                            fmaf(e.beta, old[i], e.alpha * stg[(r0 + i) * 33 + lane]);
            }
        } else {
#pragma unroll 8
            for (int rr = 0; rr < 32; ++rr)
                if (rr >= rlo && rr < rhi) base[rr * ldc] = e.alpha * stg[rr * 33 + lane];
        }
    }
    __syncwarp();
}

// Ask L2 to fetch this warp's part of the C tile (rows row0..row0+31,
// `cols` columns from col0) ahead of the beta * C reads.
__device__ __forceinline__ void prefetch_c(const EpiInfo& ti, int row0, int col0, int cols,
                                           int lane) {
    if (ti.beta == 0.0f) return;
    const int lines_per_row = cols / 32;  // 128-byte lines
    for (int l = lane; l < 32 * lines_per_row; l += 32) {
        const int rr = l / lines_per_row, c = col0 + (l % lines_per_row) * 32;
        if (row0 + rr < ti.M && c < ti.N) {
            const float* a = ti.C + size_t(row0 + rr) * size_t(ti.ldc) + c;
            asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
        }
    }
}

// The same 32 x 32 piece stored by TMA: the warp writes alpha * v into its
// 4 KB slab in the 128-byte-swizzled layout of the C tensor map (row l of the
// piece is lane l; its 16-byte chunk c sits at chunk c ^ (l % 8)), then one
// lane issues a bulk tensor store to (col0, row0, z).  TMA clips the parts
// of the box outside C.  Before rewriting the slab the lane waits until its
// previous store has finished reading it (`reuse`; a slab used once needs
// no wait).  `store` false leaves the piece in the slab only.
__device__ __forceinline__ void store_piece_tma(const float* v, float* slab, int row0, int col0,
                                                int z, float alpha, const CUtensorMap* map,
                                                int lane, bool reuse = true, bool store = true) {
    if (reuse) {
        if (lane == 0) bulk_wait_read_all();
        __syncwarp();
    }
    uint8_t* row = reinterpret_cast<uint8_t*>(slab) + lane * 128;
#pragma unroll
    for (int c = 0; c < 8; ++c)
        *reinterpret_cast<float4*>(row + ((c ^ (lane & 7)) << 4)) =
            make_float4(alpha * v[4 * c], alpha * v[4 * c + 1], alpha * v[4 * c + 2],
                        alpha * v[4 * c + 3]);
    fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0 && store) {
        tma_store_3d(map, slab, col0, row0, z);
        bulk_commit_group();
    }
}

// The one-CTA kernel.  GROUPED: tiles of many problems (per-tile problem
// lookup, tensor maps in device memory).  PROMOTE: the K range of a tile is
// cut into chunks of p.chunk_kb k-blocks; each chunk is accumulated in TMEM
// from zero and then added, in FP32 with round-to-nearest, into registers of
// the epilogue warps.  The tensor core's own FP32 accumulation rounds toward
// zero, so its error grows with the number of MMAs summed into one
// accumulator; short chunks bound that growth and the register sums carry
// the rest of K with ordinary FP32 rounding.  Without PROMOTE a tile is one
// chunk.
// Where one operand's hi/lo planes and 16-deep K slices sit inside a stage,
// and the descriptor fields that describe its tiles.  K-major: planes of
// `rows` rows x BK (one swizzled row per operand row); a K slice is 32 bytes
// along the rows.  MN-major: 64-element MN groups of [plane][BK rows of
// 128 bytes]; a K slice is 16 rows = 2048 bytes down the group.
struct OpLayout {
    uint64_t fields;
    uint32_t lo_off;  // hi plane -> lo plane
    uint32_t k_step;  // one 16-deep K slice
};

template <class S>
__device__ __forceinline__ OpLayout op_layout(int mn, int plane_bytes) {
    OpLayout l;
    if (mn) {
        l.fields = sdesc_fields(S::MN_GROUP, 1024, 2);
        l.lo_off = S::MN_GROUP / S::PLANES;
        l.k_step = 2048;
    } else {
        l.fields = sdesc_fields(16, 8 * S::ROW_BYTES, S::ROW_BYTES == 128 ? 2 : 4);
        l.lo_off = plane_bytes;
        l.k_step = 32;
    }
    return l;
}

// Layout of an operand whose FP32 tile was split in place (FUSE): each
// group of 8 rows (K-major: operand rows; MN-major: K indices) that TMA
// wrote as 8 x W FP32 values becomes [hi atom][lo atom] of 8 rows of 2W
// bytes, so consecutive 8-row groups of the hi plane are 32 W bytes apart
// and the lo plane is 16 W bytes further on.  K-major: W = BK (64-byte
// swizzle for BK 32, 128-byte for BK 64).  MN-major: W = 64 MN elements
// (128-byte swizzle), 64-element groups MN_GROUP apart, a 16-deep K slice
// two 8-row groups down.
template <class S>
__device__ __forceinline__ OpLayout op_layout_fused(int mn) {
    OpLayout l;
    if (mn) {
        l.fields = sdesc_fields(S::MN_GROUP, 2048, 2);
        l.lo_off = 1024;
        l.k_step = 4096;
    } else {
        l.fields = sdesc_fields(16, 16 * S::ROW_BYTES, S::ROW_BYTES == 128 ? 2 : 4);
        l.lo_off = 8 * S::ROW_BYTES;
        l.k_step = 32;
    }
    return l;
}

// The in-kernel split of one group (the packing step moved on chip): at
// shared address g, TMA left 8 rows of W FP32 values (row r at 4 W r bytes,
// no swizzle); they become, in place, the hi atom at g and the lo atom at
// g + 16 W: 8 rows of 2 W bytes in the swizzled layout the MMA reads, the
// 16-byte chunk c of row r stored at chunk c ^ (r mod 8) (128-byte swizzle,
// W = 64) or c ^ ((r / 2) mod 4) (64-byte swizzle, W = 32).  Lane l's i-th
// 16-byte load covers row (512 i + 16 l) / 4W, 4 consecutive columns; its
// two 8-byte stores go to group_store_offset<W>(i, l) and 16 W further on.
// The warp reads the whole group before any lane writes.  The split is
// split_bf16_2, bit-identical to the split pass.
template <int W>
__device__ __forceinline__ uint32_t group_store_offset(int i, int lane) {
    const int o = i * 512 + lane * 16;
    const int r = o / (W * 4);
    const int c0 = (o % (W * 4)) / 4;  // first of the lane's 4 columns
    const int sw = W == 64 ? (r & 7) : ((r >> 1) & 3);
    return uint32_t(r * (W * 2) + (((c0 >> 3) ^ sw) << 4) + (c0 & 7) * 2);
}

template <int W>
__device__ __forceinline__ void split_group_in_place(uint32_t g, int lane,
                                                     const uint32_t (&off)[8 * W * 4 / 512]) {
    static_assert(W == 32 || W == 64, "row width");
    constexpr int N4 = 8 * W * 4 / 512;  // 16-byte loads per lane
    float4 v[N4];
#pragma unroll
    for (int i = 0; i < N4; ++i) v[i] = ld_shared_f4(g + i * 512 + lane * 16);
    __syncwarp();
#pragma unroll
    for (int i = 0; i < N4; ++i) {
        uint32_t h01, h23, l01, l23;
        split_bf16_2(v[i].x, v[i].y, h01, l01);
        split_bf16_2(v[i].z, v[i].w, h23, l23);
        st_shared_v2(g + off[i], h01, h23);
        st_shared_v2(g + 16 * W + off[i], l01, l23);
    }
}

// The same in descriptor units: the descriptor of the operand's hi tile in
// ring slot 0, and what a lo plane and a 16-deep K slice add to it.  The
// start-address field holds address / 16 in 14 bits and shared memory ends
// below 2^18 bytes, so adding (offset / 16) to a descriptor never carries out
// of the field; the MMA issuer builds every descriptor of a stage with adds.
struct OpDesc {
    uint64_t d0;
    uint32_t lo16;
    uint32_t k16;
};

__device__ __forceinline__ OpDesc op_desc(uint32_t slot0_addr, const OpLayout& l) {
    OpDesc d;
    d.d0 = sdesc_at(slot0_addr, l.fields);
    d.lo16 = l.lo_off >> 4;
    d.k16 = l.k_step >> 4;
    return d;
}

// TMA copies of one operand's BK-deep slice into a stage: one box for a
// K-major operand, rows / 64 boxes for an MN-major one.  x coordinates are
// multiples of BK or of 64 elements (16-byte aligned) and never negative.
// `plane` is the first plane copied (0, or where the second matrix of a
// SYR2K operand buffer starts).
__device__ __forceinline__ void load_operand(uint8_t* dst, const CUtensorMap* map, uint64_t* bar,
                                             int mn, int rows, int group_bytes, int kcoord,
                                             int row0, int plane, uint64_t pol) {
    if (!mn) {
        tma_load_3d(dst, map, bar, kcoord, row0, plane, pol);
    } else {
        for (int g = 0; g < rows / 64; ++g)
            tma_load_3d(dst + g * group_bytes, map, bar, row0 + g * 64, kcoord, plane, pol);
    }
}

// The same boxes as load_operand, prefetched into L2.
__device__ __forceinline__ void prefetch_operand(const CUtensorMap* map, int mn, int rows,
                                                 int kcoord, int row0, uint64_t pol) {
    if (!mn) {
        tma_prefetch_3d(map, kcoord, row0, 0, pol);
    } else {
        for (int g = 0; g < rows / 64; ++g) tma_prefetch_3d(map, row0 + g * 64, kcoord, 0, pol);
    }
}

// Byte offset, in the ring, of tile row lr / columns lc..lc+3 (lc a multiple
// of 4) of a partial tile staged by the epilogue (ring_slab pieces: epilogue
// warp w holds rows 32 ((w + epi0) % 4) .. +31 and column half w / 4, in
// 4 KB pieces of 32 columns, 128-byte rows, 16-byte chunks swizzled by the
// row's low three bits).
template <int BN>
__device__ __forceinline__ uint32_t ring_offset(int lr, int lc, int epi0) {
    constexpr int COLS = BN / 2, PIECES = COLS / 32;
    const int w = (lc / COLS) * 4 + (((lr >> 5) - epi0) & 3);
    const int l = lr & 31, c = (lc & 31) >> 2;
    return uint32_t(w * PIECES * 4096 + ((lc % COLS) >> 5) * 4096 + l * 128 + ((c ^ (l & 7)) << 4));
}

// In-kernel split-K reduction (p.cluster_k = S > 1 CTAs per cluster, one
// K slice each, all slices' partial tiles stored in p.partial): CTA rank r
// sums tile rows [r R, r R + R), R = ceil(128 / S), over the slices in slice
// order and writes C = alpha * sum (+ beta * C), the arithmetic of the
// separate reduce kernel, so both give the same bits.  The partial tiles
// come from L2; each thread keeps U x S 16-byte loads in flight (U = 16 / S
// units of 4 columns) so the sum is not one L2 round trip per slice.  `ok`
// false (a wait of this CTA gave up) skips the sum: the error is reported,
// C is undefined.  `ring` (non-null with p.own_local): this CTA's own slice
// rows come from the epilogue's slabs in its ring instead (not stored).
template <int BN, int S>
__device__ __forceinline__ void cluster_sum_rows_s(const TcParams& p, int mt, int nt, int tid,
                                                   int nthreads, const uint8_t* ring, int epi0) {
    constexpr int R = (kBM + S - 1) / S;
    constexpr int U = S >= 16 ? 1 : 16 / S;
    const int rank = int(blockIdx.x % unsigned(S));
    const int r0 = mt * kBM + rank * R;
    const int r1 = min(min(r0 + R, mt * kBM + kBM), p.M);
    const int c0 = nt * BN;
    const int cols = min(BN, p.N - c0);
    if (r1 <= r0 || cols <= 0) return;
    const size_t slab = size_t(p.M) * size_t(p.N);
    const float alpha = p.alpha, beta = p.beta;
    if (p.sum_vec) {  // N, ldc multiples of 4 and C 16-byte aligned
        const int q4 = cols / 4;
        const int units = (r1 - r0) * q4;
        for (int i0 = tid; i0 < units; i0 += U * nthreads) {
            // every load of this batch (partials and C) before any store
            float4 v[U][S], old[U];
            float4* cp[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = min(i0 + u * nthreads, units - 1);  // clamped: loaded, not stored
                const int r = r0 + i / q4, c = c0 + (i % q4) * 4;
                const size_t e = size_t(r) * size_t(p.N) + size_t(c);
#pragma unroll
                for (int q = 0; q < S; ++q)
                    v[u][q] = ring && q == rank
                                  ? *reinterpret_cast<const float4*>(
                                        ring + ring_offset<BN>(r - mt * kBM, i % q4 * 4, epi0))
                                  : __ldcs(reinterpret_cast<const float4*>(p.partial + q * slab + e));
                cp[u] = reinterpret_cast<float4*>(p.C + size_t(r) * size_t(p.ldc) + size_t(c));
                old[u] = beta != 0.0f ? *cp[u] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (i0 + u * nthreads >= units) break;
                float4 acc = v[u][0];
#pragma unroll
                for (int q = 1; q < S; ++q) {
                    acc.x += v[u][q].x;
                    acc.y += v[u][q].y;
                    acc.z += v[u][q].z;
                    acc.w += v[u][q].w;
                }
                float4 o = make_float4(alpha * acc.x, alpha * acc.y, alpha * acc.z, alpha * acc.w);
                if (beta != 0.0f) {
                    o.x = fmaf(beta, old[u].x, o.x);
                    o.y = fmaf(beta, old[u].y, o.y);
                    o.z = fmaf(beta, old[u].z, o.z);
                    o.w = fmaf(beta, old[u].w, o.w);
                }
                *cp[u] = o;
            }
        }
    } else {
        for (int i = tid; i < (r1 - r0) * cols; i += nthreads) {
            const int r = r0 + i / cols, c = c0 + i % cols;
            const size_t e = size_t(r) * size_t(p.N) + size_t(c);
            float part[S];
#pragma unroll
            for (int q = 0; q < S; ++q) part[q] = p.partial[q * slab + e];
            float acc = part[0];
#pragma unroll
            for (int q = 1; q < S; ++q) acc += part[q];
            float* cp = p.C + size_t(r) * size_t(p.ldc) + size_t(c);
            float o = alpha * acc;
            if (beta != 0.0f) o = fmaf(beta, *cp, o);
            *cp = o;
        }
    }
}

// The C rows of cluster_sum_rows, fetched into L2 ahead of its beta * C
// reads (one prefetch per 128-byte line).
template <int BN>
__device__ __forceinline__ void cluster_sum_prefetch_c(const TcParams& p, int t, int tid,
                                                       int nthreads) {
    if (p.beta == 0.0f) return;
    const int S = p.cluster_k;
    const int rank = int(blockIdx.x % unsigned(S));
    int mt, nt;
    raster(t - rank * (p.num_m * p.num_n), p.num_m, p.num_n, p.raster_group, mt, nt);
    const int R = (kBM + S - 1) / S;
    const int r0 = mt * kBM + rank * R;
    const int r1 = min(min(r0 + R, mt * kBM + kBM), p.M);
    const int c0 = nt * BN;
    const int cols = min(BN, p.N - c0);
    if (r1 <= r0 || cols <= 0) return;
    const int lines = (cols + 31) / 32;  // 128-byte lines per row (from the row's first column)
    for (int i = tid; i < (r1 - r0) * lines; i += nthreads) {
        const float* a = p.C + size_t(r0 + i / lines) * size_t(p.ldc) + size_t(c0 + (i % lines) * 32);
        asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
    }
}

// `ring` (p.own_local): the CTA's shared-memory ring, where the epilogue
// (first warp epi0) left this slice's partial rows of the CTA's share.
template <int BN>
__device__ __noinline__ void cluster_sum_rows(const TcParams& p, int t, int tid, int nthreads,
                                              bool ok, const uint8_t* ring, int epi0) {
    if (!ok) return;
    const int rank = int(blockIdx.x % unsigned(p.cluster_k));
    int mt, nt;
    raster(t - rank * (p.num_m * p.num_n), p.num_m, p.num_n, p.raster_group, mt, nt);
    if (!p.own_local) ring = nullptr;
    switch (p.cluster_k) {
        case 2: cluster_sum_rows_s<BN, 2>(p, mt, nt, tid, nthreads, ring, epi0); break;
        case 3: cluster_sum_rows_s<BN, 3>(p, mt, nt, tid, nthreads, ring, epi0); break;
        case 4: cluster_sum_rows_s<BN, 4>(p, mt, nt, tid, nthreads, ring, epi0); break;
        case 5: cluster_sum_rows_s<BN, 5>(p, mt, nt, tid, nthreads, ring, epi0); break;
        case 6: cluster_sum_rows_s<BN, 6>(p, mt, nt, tid, nthreads, ring, epi0); break;
        case 7: cluster_sum_rows_s<BN, 7>(p, mt, nt, tid, nthreads, ring, epi0); break;
        default: cluster_sum_rows_s<BN, 8>(p, mt, nt, tid, nthreads, ring, epi0); break;
    }
}

// FUSE (split precision only): the operands marked in p.fuse_ops are the
// caller's FP32 matrices; TMA stages their FP32 tiles, converter warps split
// them in place into the hi/lo atoms the MMA reads (split_group_in_place) and
// arrive on conv[s], which the MMA issuer waits on instead of full[s].  An
// operand not marked arrives as BF16 hi/lo planes from the split pass, in the
// layout of the kernel without FUSE (a stage holds the same bytes either way).
template <int BN, int BK, int NTERMS, bool PROMOTE, bool GROUPED, bool FUSE = false>
__global__ void __launch_bounds__(FUSE ? kFusedThreads : kThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmC, const TcParams p) {
    using S = Shape<BN, BK, NTERMS>;
    static_assert(!FUSE || NTERMS == 3, "the in-kernel split feeds the split-precision MMAs");
    constexpr int EPI0 = FUSE ? kFusedEpi0 : 2;  // first epilogue warp
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                               ~uintptr_t(1023));
    const int stages = p.stages;
    uint8_t* bar_area = smem + stages * S::STAGE;
    uint64_t* full = reinterpret_cast<uint64_t*>(bar_area);
    uint64_t* empty = full + stages;
    uint64_t* acc_full = empty + stages;  // [2]
    uint64_t* acc_empty = acc_full + 2;   // [2]
    uint64_t* drain = acc_empty + 2;
    uint64_t* conv = drain + 1;  // FUSE: [stages], stage s split in place
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(FUSE ? conv + stages : drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    float* staging = reinterpret_cast<float*>(bar_area + S::BAR_BYTES);  // [kEpiWarps][32][33]

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
            if (FUSE) mbar_init(&conv[s], kConvWarps);  // one arrival per converter warp
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&acc_full[a], 1);
            mbar_init(&acc_empty[a], kEpiWarps);  // one arrival per epilogue warp
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        fence_mbar_init();
        if (!GROUPED) {
            tma_prefetch_desc(&tmA);
            tma_prefetch_desc(&tmB);
        }
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, S::TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    // In-kernel split-K reduction: the grid is exactly the tile space and the
    // cluster_k CTAs of a cluster take the K slices of one output tile (slice
    // = rank in the cluster); otherwise CTAs walk the tiles persistently.
    const bool cluster_sum = !GROUPED && p.cluster_k > 1;
    const int t_first = cluster_sum ? int(blockIdx.x % unsigned(p.cluster_k)) * (p.num_m * p.num_n) +
                                          int(blockIdx.x / unsigned(p.cluster_k))
                                    : int(blockIdx.x);
    // While the preceding kernel of the stream finishes, start pulling the
    // first ring's worth of this CTA's first tile into L2.  Prefetches read
    // nothing into the CTA, so they may come before pdl_wait: the loads that
    // use the data are issued after it.
    if (!GROUPED && p.uplo == 0 && threadIdx.x == 0 && t_first < p.num_tiles) {
        const TileInfo ti = get_tile<GROUPED>(t_first, p, &tmA, &tmB);
        const uint64_t keep = l2_policy_evict_last(), once = l2_policy_evict_first();
        const int kb_end = min(ti.kb1, ti.kb0 + stages);
        for (int kb = ti.kb0; kb < kb_end; ++kb) {
            prefetch_operand(ti.ma, ti.maj & 1, kBM, kb * BK, ti.mt * kBM, p.num_n == 1 ? once : keep);
            prefetch_operand(ti.mb, (ti.maj >> 1) & 1, BN, kb * BK, ti.nt * BN,
                             p.num_m == 1 ? once : keep);
        }
    }
    // launched as a dependent of a split pass or another GEMM: its writes
    // are complete and visible from here on (the set-up above overlapped its
    // tail)
    pdl_wait();

    // Role dispatch, epilogue first: with FUSE the epilogue warpgroups raise
    // their register budget and the others (producer, MMA issuer, converters)
    // lower theirs at the head of their branch, so that the raised budget
    // covers the epilogue code (warpgroups 0 and 3 execute the same lowering).
    if (FUSE ? (warp >= EPI0 && warp < EPI0 + kEpiWarps) : warp >= 2) {
        if constexpr (FUSE) regs_inc<kFusedEpiRegs>();
        // ------------------------------------------------ epilogue
        // Warp w reads TMEM lanes 32*(w%4)..+31 (tile rows) and one half of
        // the tile's columns.
        constexpr int COLS = BN / 2;     // columns per epilogue warp
        constexpr int PIECES = COLS / 32;
        const int ew = warp & 3;
        const int col_base = ((warp - EPI0) >> 2) * COLS;
        float* stg = staging + (warp - EPI0) * 32 * 33;
        float* slab = staging + (warp - EPI0) * 1024;  // 4 KB, 1024-byte aligned (TMA store)
        // A cluster CTA owns one tile, so once its last chunk is in TMEM the
        // ring is idle (every copy consumed by the MMAs): each partial piece
        // then gets a slab of its own there and the stores go out back to
        // back instead of waiting for one another
        const bool ring = cluster_sum && p.ring_epi;
        float* ring_slab = reinterpret_cast<float*>(smem) + (warp - EPI0) * PIECES * 1024;
        // rows of this CTA's own share of the sum: kept in the ring, not stored
        const bool keep = ring && p.own_local &&
                          ew * 32 / (kBM / p.cluster_k) == int(blockIdx.x % unsigned(p.cluster_k));
        float sum[PROMOTE ? COLS : 1];
        int g = 0;
        bool ok = true;
        // the C rows this CTA's split-K sum will read: into L2 while the
        // K loop runs
        if (cluster_sum) cluster_sum_prefetch_c<BN>(p, t_first, (warp - EPI0) * 32 + lane,
                                                    kEpiWarps * 32);
#pragma unroll 1
        for (int t = t_first; t < p.num_tiles && ok; t += gridDim.x) {
            const TileInfo ti = get_tile<GROUPED>(t, p, &tmA, &tmB);
            const int kb0 = ti.kb0, kb1 = ti.kb1;
            const int chunk = PROMOTE ? p.chunk_kb : kb1 - kb0;
            const int row0 = ti.mt * kBM + ew * 32;  // first tile row of this warp
            const int col0 = ti.nt * BN + col_base;
#pragma unroll 1
            for (int c0 = kb0; c0 < kb1; c0 += chunk, ++g) {
                const int buf = g & 1;
                const uint32_t acc_ph = (g >> 1) & 1;
                int got = 0;
                if (lane == 0)
                    got = FUSE ? mbar_wait_bounded_sleep(&acc_full[buf], acc_ph, p.lim, abort_flag,
                                                         p.err, 256)
                               : mbar_wait_bounded(&acc_full[buf], acc_ph, p.lim, abort_flag,
                                                   p.err);
                got = __shfl_sync(0xffffffffu, got, 0);
                if (!got) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t taddr = tmem_base + (uint32_t(ew * 32) << 16) + buf * BN + col_base;
                // one chunk before the final store, start pulling C into L2
                if (c0 + 2 * chunk >= kb1 && c0 + chunk < kb1)
                    prefetch_c(get_epi<GROUPED>(ti.prob, ti.ks, p), row0, col0, COLS, lane);
                if (PROMOTE) {
                    // 16 columns per TMEM load keeps the live registers at
                    // the running sums plus one 16-wide piece.
                    if (c0 == kb0) {
#pragma unroll
                        for (int q = 0; q < 2 * PIECES; ++q) {
                            uint32_t r[16];
                            tmem_ld_32x32b_x16(taddr + q * 16, r);
                            tmem_ld_wait();
#pragma unroll
                            for (int j = 0; j < 16; ++j) sum[q * 16 + j] = __uint_as_float(r[j]);
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 2 * PIECES; ++q) {
                            uint32_t r[16];
                            tmem_ld_32x32b_x16(taddr + q * 16, r);
                            tmem_ld_wait();
#pragma unroll
                            for (int j = 0; j < 16; ++j) sum[q * 16 + j] += __uint_as_float(r[j]);
                        }
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&acc_empty[buf]);  // TMEM free before the stores
                    if (c0 + chunk >= kb1) {
                        const EpiInfo e = get_epi<GROUPED>(ti.prob, ti.ks, p);
                        if (p.c_tma) {
#pragma unroll
                            for (int q = 0; q < PIECES; ++q)
                                store_piece_tma(&sum[q * 32], ring ? ring_slab + q * 1024 : slab,
                                                row0, col0 + q * 32, ti.ks, e.alpha, &tmC, lane,
                                                !ring, !keep);
                        } else {
#pragma unroll
                            for (int q = 0; q < PIECES; ++q)
                                store_piece(&sum[q * 32], stg, row0, col0 + q * 32, e, lane);
                        }
                    }
                } else {
#pragma unroll 1
                    for (int q = 0; q < PIECES; ++q) {
                        uint32_t r[32];
                        tmem_ld_32x32b_x32(taddr + q * 32, r);
                        tmem_ld_wait();
                        float v[32];
#pragma unroll
                        for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
                        const EpiInfo e = get_epi<GROUPED>(ti.prob, ti.ks, p);
                        if (p.c_tma)
                            store_piece_tma(v, ring ? ring_slab + q * 1024 : slab, row0,
                                            col0 + q * 32, ti.ks, e.alpha, &tmC, lane, !ring,
                                            !keep);
                        else
                            store_piece(v, stg, row0, col0 + q * 32, e, lane);
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&acc_empty[buf]);
                }
            }
        }
        if (cluster_sum) {
            // this warp's partial-tile stores have landed; then every CTA of
            // the cluster has stored its slice and the sum may read them all
            if (lane == 0) {
                bulk_wait_all();
                fence_proxy_async_global();
            }
            __syncwarp();
            cluster_sync();
            // without FUSE the producer and MMA warps (threads 0-63) join
            // the sum as threads 256-319
            cluster_sum_rows<BN>(p, t_first, (warp - EPI0) * 32 + lane,
                                 FUSE ? kEpiWarps * 32 : kThreads, *abort_flag == 0, smem, EPI0);
        }
    } else {
        if constexpr (FUSE) regs_dec<kFusedOtherRegs>();
        if (warp == 0) {
            // ------------------------------------------------ TMA producer
            if (lane == 0) {
                // L2 hints: an operand whose tiles only one tile row or
                // column reads (B with a single M tile, A with a single N
                // tile) streams through once and is evicted first; the
                // other is kept for the tiles that read it again
                const uint64_t keep = l2_policy_evict_last(), once = l2_policy_evict_first();
                const uint64_t pol_a = !GROUPED && p.num_n == 1 ? once : keep;
                const uint64_t pol_b = !GROUPED && p.num_m == 1 ? once : keep;
                uint32_t filled = 0;      // bit s: slot s received a fill
                uint32_t fill_par = 0;    // bit s: parity of slot s's latest fill
                int s = 0;                // ring slot of the next fill
                uint32_t ph = 0;          // and its parity
                bool ok = true;
                // Consecutive tiles of a CTA walk K in alternate directions:
                // the CTAs move through a wave of tiles together, and the
                // next wave of the raster reuses most of its operand panels,
                // so starting it at the K blocks loaded last finds them still
                // in L2.  (Only the order of a tile's K blocks changes, hence
                // the order of its FP32 accumulation; it is fixed for a given
                // grid.)
                bool rev = false;  // K blocks of this tile in descending order
                for (int t = t_first; t < p.num_tiles && ok; t += gridDim.x, rev = !rev) {
                    const TileInfo ti = get_tile<GROUPED>(t, p, &tmA, &tmB);
                    for (int kq = ti.kb0; kq < ti.kb1; ++kq) {
                        const int kb = ti.koff + ti.kstep * (rev ? ti.kb0 + ti.kb1 - 1 - kq : kq);
                        if (!mbar_wait_bounded(&empty[s], ph ^ 1, p.lim, abort_flag, p.err)) {
                            ok = false;
                            break;
                        }
                        // SYR2K: K blocks [0, syr_kb) pair A-side rows of the first
                        // matrix with B-side rows of the second, the next syr_kb
                        // blocks the other way round (the two GEMM updates of a block)
                        int kc = kb, za = 0, zb = 0;
                        if (!GROUPED && p.syr_kb > 0) {
                            const int second = kb >= p.syr_kb;
                            kc = kb - (second ? p.syr_kb : 0);
                            za = second ? p.syr_plane : 0;
                            zb = second ? 0 : p.syr_plane;
                        }
                        uint8_t* st = smem + s * S::STAGE;
                        mbar_arrive_expect_tx(&full[s], S::STAGE);
                        load_operand(st, ti.ma, &full[s], ti.maj & 1, kBM, S::MN_GROUP, kc * BK,
                                     ti.mt * kBM, za, pol_a);
                        load_operand(st + S::PLANES * S::A_PLANE, ti.mb, &full[s], (ti.maj >> 1) & 1,
                                     BN, S::MN_GROUP, kc * BK, ti.nt * BN, zb, pol_b);
                        filled |= 1u << s;
                        fill_par = (fill_par & ~(1u << s)) | (ph << s);
                        if (++s == stages) {
                            s = 0;
                            ph ^= 1;
                        }
                    }
                }
                // every operand load of this CTA is issued: the next GEMM
                // of the stream may start setting up on idle SMs
                pdl_launch_dependents();
                // Wait for every copy this thread started before the CTA may exit.
                for (int s = 0; s < stages; ++s)
                    if (filled & (1u << s)) mbar_wait_drain(&full[s], (fill_par >> s) & 1, p.err);
            }
        } else if (warp == 1) {
            // ------------------------------------------------ MMA issuer
            if (lane == 0) {
                // One thread issues every MMA, so its per-stage instruction path
                // is on the critical path of the tensor pipe: ring slot and parity
                // are running counters and descriptors are built with adds.
                int g = 0;        // accumulation chunks started by this CTA
                int s = 0;        // ring slot of the next stage to consume
                uint32_t ph = 0;  // and its fill parity
                bool ok = true;
                const uint32_t slot0 = smem_u32(smem);
                for (int t = t_first; t < p.num_tiles && ok; t += gridDim.x) {
                    const TileInfo ti = get_tile<GROUPED>(t, p, &tmA, &tmB);
                    const int kb0 = ti.kb0, kb1 = ti.kb1;
                    const int a_mn = ti.maj & 1, b_mn = (ti.maj >> 1) & 1;
                    const uint32_t idesc = make_idesc_bf16_f32(kBM, BN, a_mn, b_mn);
                    const OpDesc da = op_desc(slot0, FUSE && (p.fuse_ops & 1)
                                                          ? op_layout_fused<S>(a_mn)
                                                          : op_layout<S>(a_mn, S::A_PLANE));
                    const OpDesc db = op_desc(slot0 + S::PLANES * S::A_PLANE,
                                              FUSE && (p.fuse_ops & 2)
                                                  ? op_layout_fused<S>(b_mn)
                                                  : op_layout<S>(b_mn, S::B_PLANE));
                    const int chunk = PROMOTE ? p.chunk_kb : kb1 - kb0;
                    for (int c0 = kb0; c0 < kb1 && ok; c0 += chunk, ++g) {
                        const int buf = g & 1;
                        const uint32_t acc_ph = (g >> 1) & 1;
                        if (!mbar_wait_bounded(&acc_empty[buf], acc_ph ^ 1, p.lim, abort_flag, p.err)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t d_tmem = tmem_base + buf * BN;
                        const int c1 = min(c0 + chunk, kb1);
                        for (int kb = c0; kb < c1; ++kb) {
                            // FUSE: the stage is usable once it has been split in place
                            if (!mbar_wait_bounded(FUSE ? &conv[s] : &full[s], ph, p.lim, abort_flag,
                                                   p.err)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const uint32_t slot16 = uint32_t(s) * uint32_t(S::STAGE >> 4);
                            const uint64_t a_s = da.d0 + slot16, b_s = db.d0 + slot16;
    #pragma unroll
                            for (int kk = 0; kk < BK / 16; ++kk) {
                                const uint64_t ah = a_s + uint32_t(kk) * da.k16;
                                const uint64_t bh = b_s + uint32_t(kk) * db.k16;
                                const uint32_t acc = (kb > c0 || kk > 0) ? 1u : 0u;
                                if (NTERMS == 3) {
                                    umma_bf16(d_tmem, ah + da.lo16, bh, idesc, acc);
                                    umma_bf16(d_tmem, ah, bh + db.lo16, idesc, 1u);
                                    umma_bf16(d_tmem, ah, bh, idesc, 1u);
                                } else {
                                    umma_bf16(d_tmem, ah, bh, idesc, acc);
                                }
                            }
                            umma_commit(&empty[s]);  // slot free once these MMAs have read it
                            if (++s == stages) {
                                s = 0;
                                ph ^= 1;
                            }
                        }
                        if (!ok) break;
                        umma_commit(&acc_full[buf]);  // chunk ready for the epilogue
                    }
                }
                // All MMAs this thread issued must finish before TMEM is freed.
                umma_commit(drain);
                mbar_wait_drain(drain, 0, p.err);
            }
        } else if constexpr (FUSE) {
            // ------------------------------------------------ converters (FUSE)
            // Converter cw of 6 splits every 6th 8-row group of each stage: the A
            // groups first, then the B groups.  All lanes wait for the stage (the
            // copies' writes become visible to each waiting thread), split, make
            // their shared-memory writes visible to the tensor core (proxy
            // fence), and lane 0 arrives on conv[s] once the warp has finished.
            const int cw = warp < EPI0 ? warp - 2 : warp - (EPI0 + kEpiWarps) + 2;
            const uint32_t slot0 = smem_u32(smem);
            uint32_t off32[2], off64[4];  // this lane's store offsets in a group
#pragma unroll
            for (int i = 0; i < 2; ++i) off32[i] = group_store_offset<32>(i, lane);
#pragma unroll
            for (int i = 0; i < 4; ++i) off64[i] = group_store_offset<64>(i, lane);
            int s = 0;
            uint32_t ph = 0;
            bool ok = true;
    #pragma unroll 1
            for (int t = t_first; t < p.num_tiles && ok; t += gridDim.x) {
                const TileInfo ti = get_tile<GROUPED>(t, p, &tmA, &tmB);
                const int wa = (ti.maj & 1) ? 64 : BK;         // row width of an A group
                const int wb = ((ti.maj >> 1) & 1) ? 64 : BK;  // and of a B group
                // groups of 32 W bytes; an operand that arrives as BF16
                // planes (split by the pass) has none
                const int na = (p.fuse_ops & 1) ? kBM * BK * 4 / (32 * wa) : 0;
                const int nb = (p.fuse_ops & 2) ? BN * BK * 4 / (32 * wb) : 0;
    #pragma unroll 1
                for (int kb = ti.kb0; kb < ti.kb1; ++kb) {
                    // lane 0 polls; then every lane observes the completed
                    // phase itself (one try_wait that succeeds at once), so
                    // the copies' writes are visible to the whole warp
                    int got = 0;
                    if (lane == 0) got = mbar_wait_bounded(&full[s], ph, p.lim, abort_flag, p.err);
                    got = __shfl_sync(0xffffffffu, got, 0);
                    if (got) got = mbar_wait_bounded(&full[s], ph, p.lim, abort_flag, p.err);
                    if (!__all_sync(0xffffffffu, got)) {
                        ok = false;
                        break;
                    }
                    const uint32_t st = slot0 + uint32_t(s) * uint32_t(S::STAGE);
    #pragma unroll 1
                    for (int gi = cw; gi < na + nb; gi += kConvWarps) {
                        const bool in_a = gi < na;
                        const int w = in_a ? wa : wb;
                        const uint32_t g = in_a ? st + uint32_t(gi * 32 * wa)
                                                : st + uint32_t(S::PLANES * S::A_PLANE) +
                                                      uint32_t((gi - na) * 32 * wb);
                        if (w == 64)
                            split_group_in_place<64>(g, lane, off64);
                        else
                            split_group_in_place<32>(g, lane, off32);
                    }
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&conv[s]);
                    if (++s == stages) {
                        s = 0;
                        ph ^= 1;
                    }
                }
            }
        }
        if (cluster_sum) {  // the epilogue warps' barrier before their sum
            __syncwarp();
            cluster_sync();
            if constexpr (!FUSE)
                cluster_sum_rows<BN>(p, t_first, kEpiWarps * 32 + threadIdx.x, kThreads,
                                     *abort_flag == 0, smem, EPI0);
        }
    }

    // ------------------------------------------------ teardown
    if (warp >= 2 && lane == 0) bulk_wait_all();  // TMA stores of C finished
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, S::TMEM_COLS);
    }
}

// The output side of a CTA-pair tile: get_epi's, or for a tail-split unit
// its half's raw partial tile (alpha 1, beta 0) in the tail buffer.
template <bool GROUPED, int BN>
__device__ __forceinline__ EpiInfo pair_epi(const TileInfo& ti, const TcParams& p) {
    EpiInfo e = get_epi<GROUPED>(ti.prob, ti.ks, p);
    if (!GROUPED && ti.prob > 0) {
        e.C = p.tail_part + size_t((ti.prob - 1) * 2 + ti.ks) * size_t(2 * kBM * BN);
        e.ldc = BN;
        e.alpha = 1.0f;
        e.beta = 0.0f;
        e.uplo = 0;
        e.r_off = ti.mt * 2 * kBM;
        e.c_off = ti.nt * BN;
    }
    return e;
}

// C = alpha (P0 + P1) + beta C over the tiles of a tail split (TcParams
// tail_*): P0 the even K blocks' partial, P1 the odd ones', added in that
// order with the split-K reduce's arithmetic; block (i, y) takes every
// gridDim.y-th row chunk of tail tile i.
// Launched as a dependent of the pair kernel that wrote the halves.
template <int BN>
__global__ void __launch_bounds__(256) tail_reduce_kernel(const TcParams p, int vec) {
    pdl_wait();
    const int i = int(blockIdx.x);
    int mt, nt;
    raster(p.tail_base + i, p.num_m, p.num_n, p.raster_group, mt, nt);
    const int r0 = mt * 2 * kBM, c0 = nt * BN;
    const int rows = min(2 * kBM, p.M - r0), cols = min(BN, p.N - c0);
    const float* P0 = p.tail_part + size_t(2 * i) * size_t(2 * kBM * BN);
    const float* P1 = P0 + size_t(2 * kBM * BN);
    const float alpha = p.alpha, beta = p.beta;
    if (vec) {  // N, ldc multiples of 4, C 16-byte aligned
        const int q4 = cols / 4;
        for (int idx = int(blockIdx.y * blockDim.x + threadIdx.x); idx < rows * q4;
             idx += int(gridDim.y * blockDim.x)) {
            const int lr = idx / q4, lc = (idx % q4) * 4;
            const float4 a = __ldcs(reinterpret_cast<const float4*>(P0 + lr * BN + lc));
            const float4 b = __ldcs(reinterpret_cast<const float4*>(P1 + lr * BN + lc));
            float4* cp = reinterpret_cast<float4*>(p.C + size_t(r0 + lr) * size_t(p.ldc) + (c0 + lc));
            float4 o = make_float4(alpha * (a.x + b.x), alpha * (a.y + b.y), alpha * (a.z + b.z),
                                   alpha * (a.w + b.w));
            if (beta != 0.0f) {
                const float4 old = *cp;
                o.x = fmaf(beta, old.x, o.x);
                o.y = fmaf(beta, old.y, o.y);
                o.z = fmaf(beta, old.z, o.z);
                o.w = fmaf(beta, old.w, o.w);
            }
            *cp = o;
        }
    } else {
        for (int idx = int(blockIdx.y * blockDim.x + threadIdx.x); idx < rows * cols;
             idx += int(gridDim.y * blockDim.x)) {
            const int lr = idx / cols, lc = idx % cols;
            float* cp = p.C + size_t(r0 + lr) * size_t(p.ldc) + (c0 + lc);
            float o = alpha * (P0[lr * BN + lc] + P1[lr * BN + lc]);
            if (beta != 0.0f) o = fmaf(beta, *cp, o);
            *cp = o;
        }
    }
}

// ---------------------------------------------------------------- CTA pairs
// The same GEMM with CTA pairs (cluster of two, tcgen05 cta_group::2): a
// pair owns a 256 x BN output tile; each CTA stages its 128 rows of A and
// half (BN/2 rows) of B, so each SM moves half the B bytes of the one-CTA
// kernel through shared memory, and the even CTA issues 256 x BN MMAs that
// read both CTAs' tiles and write each CTA's 128 accumulator rows in its own
// tensor memory.
//
// Synchronisation: both CTAs' TMA copies of stage s count their bytes on the
// EVEN CTA's full[s] (the odd CTA uses the cta_group::2 form of the copy,
// which may signal the pair's even CTA); the even producer arms each phase
// for both halves (2 x STAGE bytes), so the MMA issuer's one wait covers the
// whole 256-row stage.  (A design that signalled each CTA's own barrier and
// forwarded the odd half with a remote mbarrier arrive ran at about one stage
// per microsecond whatever the ring depth: the remote arrive on the critical
// path of every stage, 2.6x slower.)  The even CTA's commits are multicast
// to both CTAs' empty[s] / acc_full[b] / drain barriers; both CTAs' epilogue
// warps arrive on the even CTA's acc_empty[b] (16 arrivals).
//
// Producers: one thread per CTA copies A and B; for plain BF16, whose stages
// hold only BK / 16 MMAs, the copy issue (about 200 cycles a copy on the
// issuing thread) was the limit, so A and B come from two warps (10 to 11 %
// faster at BK 64 on 8192^3).
//
// Teardown: the producers other than the even A copier cannot observe their
// own copies' barrier phases, so each reports how many stages it filled (a
// store and a release-arrive on the even CTA's odd_done); the even A copier
// settles every phase that some producer filled and another did not
// (complete_tx for the parts never issued when it armed the phase,
// arrive.expect_tx for the issued parts when it did not), then waits for the
// last phase of every slot, so all copies of both CTAs have landed before the
// cluster barrier that precedes the tensor-memory free lets either CTA leave.
template <int BN, int BK, int NTERMS>
struct Shape2 {
    static constexpr int PLANES = NTERMS == 1 ? 1 : 2;
    static constexpr int BNH = BN / 2;  // B rows staged by each CTA
    static constexpr int A_PLANE = kBM * BK * 2;
    static constexpr int B_PLANE = BNH * BK * 2;
    static constexpr int STAGE = PLANES * (A_PLANE + B_PLANE);
    // BN 512 (plain BF16): two N = 256 MMAs per 16-deep slice into two
    // accumulators that fill the tensor memory, so one buffer, not two
    static constexpr int MMA_N = BN > 256 ? 256 : BN;
    static constexpr int NSUB = BN / MMA_N;
    static constexpr int NBUF = BN > 256 ? 1 : 2;
    static constexpr int TMEM_COLS = NBUF * BN;
    static constexpr int ROW_BYTES = BK * 2;
    static constexpr int MN_GROUP = PLANES * BK * 128;  // as in Shape
    // offset of the second MMA's B rows inside a CTA's B box: 128 rows,
    // K-major (128 rows of ROW_BYTES) or MN-major (two 64-row groups)
    static constexpr int SUB_B = 128 * BK * 2 * PLANES;
    static_assert(NSUB == 1 || (PLANES == 1 && SUB_B == 2 * MN_GROUP),
                  "wide pair tiles are plain BF16 only");
    static constexpr int BAR_BYTES = 1024;
    static constexpr int STAGING = kEpiWarps * 32 * 33 * 4;
    static_assert(B_PLANE % 1024 == 0, "B plane must keep swizzle atoms aligned");
    static int smem_bytes(int stages) { return 1024 + stages * STAGE + BAR_BYTES + STAGING; }
    static int max_stages() {
        int s = (kMaxSmem - 1024 - BAR_BYTES - STAGING) / STAGE;
        return s > 8 ? 8 : s;
    }
};

// Tile column of accumulator column c in a 512-wide pair tile: MMA j takes
// rows 128j.. of each CTA's 256-row B box (the even CTA's box holds tile
// columns 0..255, the odd CTA's 256..511), so its accumulator holds tile
// columns 128j + [0, 128) and then 256 + 128j + [0, 128).
__device__ __forceinline__ int wide_tile_col(int c) {
    const int j = c >> 8, w = c & 255;
    return w < 128 ? j * 128 + w : 256 + j * 128 + (w - 128);
}

// The pair form of load_operand: the even CTA's copies count on its own full
// barrier, the odd CTA's on the even CTA's (`peer_bar`, cta_group::2 form).
__device__ __forceinline__ void load_operand_pair(uint8_t* dst, const CUtensorMap* map,
                                                  uint64_t* own_bar, uint32_t peer_bar, bool odd,
                                                  int mn, int rows, int group_bytes, int kcoord,
                                                  int row0, uint64_t pol) {
    const int groups = mn ? rows / 64 : 1;
    for (int g = 0; g < groups; ++g) {
        const int x = mn ? row0 + g * 64 : kcoord;
        const int y = mn ? kcoord : row0;
        if (odd)
            tma_load_3d_to_peer_bar(dst + g * group_bytes, map, peer_bar, x, y, 0, pol);
        else
            tma_load_3d(dst + g * group_bytes, map, own_bar, x, y, 0, pol);
    }
}

// Threads of a pair CTA: plain BF16 adds a warp that issues the B copies.
template <int NTERMS>
constexpr int pair_threads() {
    return NTERMS == 1 ? kThreads + 32 : kThreads;
}

template <int BN, int BK, int NTERMS, bool PROMOTE, bool GROUPED>
__global__ void __launch_bounds__(pair_threads<NTERMS>(), 1)
    tc_gemm_pair_kernel(const __grid_constant__ CUtensorMap tmA,
                        const __grid_constant__ CUtensorMap tmB,
                        const __grid_constant__ CUtensorMap tmC, const TcParams p) {
    using S = Shape2<BN, BK, NTERMS>;
    constexpr bool SPLIT = NTERMS == 1;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                               ~uintptr_t(1023));
    const int stages = p.stages;
    uint8_t* bar_area = smem + stages * S::STAGE;
    uint64_t* full = reinterpret_cast<uint64_t*>(bar_area);  // even CTA's count both halves
    uint64_t* empty = full + stages;
    uint64_t* acc_full = empty + stages;  // [2]
    uint64_t* acc_empty = acc_full + 2;   // [2]
    uint64_t* drain = acc_empty + 2;
    uint64_t* odd_done = drain + 1;       // even CTA: the other producers have finished
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(odd_done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    volatile uint32_t* fills = reinterpret_cast<volatile uint32_t*>(tmem_slot + 2);  // [3]
    float* staging = reinterpret_cast<float*>(bar_area + S::BAR_BYTES);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t rank = cluster_ctarank();  // 0: issues the MMAs
    const int pair = blockIdx.x >> 1;
    const int npairs = gridDim.x >> 1;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&acc_full[a], 1);
            mbar_init(&acc_empty[a], 2 * kEpiWarps);  // both CTAs' epilogue warps
        }
        mbar_init(drain, 1);
        mbar_init(odd_done, SPLIT ? 3 : 1);  // reporting producers
        *abort_flag = 0;
        fills[0] = fills[1] = fills[2] = 0;
        fence_mbar_init();
        if (!GROUPED) {
            tma_prefetch_desc(&tmA);
            tma_prefetch_desc(&tmB);
        }
    }
    __syncthreads();
    cluster_sync();  // barriers initialised in both CTAs before any remote arrive
    if (warp == 1) {
        tmem_alloc_pair(tmem_slot, S::TMEM_COLS);
        tmem_relinquish_pair();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    pdl_wait();  // as in the one-CTA kernel

    // One thread per producer role fills the ring; with SPLIT (plain BF16, whose
    // short stages make the copy issue the limit) warp 0 copies A and a second
    // warp copies B, otherwise warp 0 copies both.  Returns the stages filled.
    auto produce = [&](bool copy_a, bool copy_b) -> int {
        // L2 hints as in the one-CTA kernel (single pair-tile row: B once)
        const uint64_t keep = l2_policy_evict_last(), once = l2_policy_evict_first();
        const uint64_t pol_a = !GROUPED && p.num_n == 1 ? once : keep;
        const uint64_t pol_b = !GROUPED && p.num_m == 1 ? once : keep;
        const uint32_t leader_full = mapa_shared(smem_u32(full), 0);
        const bool arm = rank == 0 && copy_a;  // the even A copier arms every phase
        int it = 0;       // stages filled
        int s = 0;        // ring slot of the next fill
        uint32_t ph = 0;  // and its parity
        bool ok = true;
        // alternate K directions on consecutive tiles, as in the one-CTA kernel
        bool rev = false;  // K blocks of this tile in descending order
        for (int t = pair; t < p.num_tiles && ok; t += npairs, rev = !rev) {
            const TileInfo ti = get_tile<GROUPED>(t, p, &tmA, &tmB);
            for (int kq = ti.kb0; kq < ti.kb1; ++kq, ++it) {
                const int kb = ti.koff + ti.kstep * (rev ? ti.kb0 + ti.kb1 - 1 - kq : kq);
                if (!mbar_wait_bounded_cluster(&empty[s], ph ^ 1, p.lim, abort_flag, p.err)) {
                    ok = false;
                    break;
                }
                uint8_t* st = smem + s * S::STAGE;
                const uint32_t bar = leader_full + uint32_t(s) * 8u;
                if (arm) mbar_arrive_expect_tx(&full[s], 2 * S::STAGE);  // all four parts
                if (copy_a)
                    load_operand_pair(st, ti.ma, &full[s], bar, rank != 0, ti.maj & 1, kBM,
                                      S::MN_GROUP, kb * BK, ti.mt * 2 * kBM + int(rank) * kBM, pol_a);
                if (copy_b)
                    load_operand_pair(st + S::PLANES * S::A_PLANE, ti.mb, &full[s], bar,
                                      rank != 0, (ti.maj >> 1) & 1, S::BNH, S::MN_GROUP, kb * BK,
                                      ti.nt * BN + int(rank) * S::BNH, pol_b);
                if (++s == stages) {
                    s = 0;
                    ph ^= 1;
                }
            }
        }
        return it;
    };
    // A producer that does not arm reports its fill count to the even CTA:
    // fills[0] even B, fills[1] odd A (odd A and B without SPLIT), fills[2]
    // odd B; a store, then a release-arrive on odd_done.
    auto report = [&](int idx, int count) {
        if (rank == 0) {
            fills[idx] = uint32_t(count);
            mbar_arrive(odd_done);
        } else {
            st_shared_cluster_u32(mapa_shared(smem_u32(const_cast<uint32_t*>(fills + idx)), 0),
                                  uint32_t(count));
            mbar_arrive_remote(mapa_shared(smem_u32(odd_done), 0));
        }
    };

    if (warp == 0) {
        // ------------------------------------------------ TMA producer (both CTAs)
        if (lane == 0) {
            const int it = produce(true, !SPLIT);
            pdl_launch_dependents();  // as in the one-CTA kernel
            if (rank != 0) {
                report(1, it);
            } else {
                // Settle every phase that some producer filled and another did
                // not, then wait until every copy of both CTAs has landed.  A
                // producer fills phase j only after phase j - stages completed
                // (all four parts issued), so the counts differ by at most
                // `stages` and the phases settled here are the current phases
                // of distinct slots.
                int cnt[4] = {it, it, it, it};  // even A, even B, odd A, odd B
                if (mbar_wait_drain_cluster(odd_done, 0, p.err)) {
                    if (SPLIT) cnt[1] = int(fills[0]);
                    cnt[2] = int(fills[1]);
                    cnt[3] = SPLIT ? int(fills[2]) : cnt[2];
                }
                constexpr uint32_t part[4] = {S::PLANES * S::A_PLANE, S::PLANES * S::B_PLANE,
                                              S::PLANES * S::A_PLANE, S::PLANES * S::B_PLANE};
                const int lo = min(min(cnt[0], cnt[1]), min(cnt[2], cnt[3]));
                const int hi = max(max(cnt[0], cnt[1]), max(cnt[2], cnt[3]));
                for (int j = lo; j < hi; ++j) {
                    uint32_t issued = 0;
                    for (int r = 0; r < 4; ++r)
                        if (j < cnt[r]) issued += part[r];
                    if (j < cnt[0])
                        mbar_complete_tx(&full[j % stages], 2 * S::STAGE - issued);  // armed
                    else
                        mbar_arrive_expect_tx(&full[j % stages], issued);  // never armed
                }
                for (int s = 0; s < stages && s < hi; ++s) {
                    const int j = hi - 1 - ((hi - 1 - s) % stages);  // last fill of slot s
                    mbar_wait_drain(&full[s], uint32_t(j / stages) & 1, p.err);
                }
            }
        }
    } else if (SPLIT && warp == 2 + kEpiWarps) {
        // ------------------------------------------------ B producer (plain BF16)
        if (lane == 0) report(rank == 0 ? 0 : 2, produce(false, true));
    } else if (warp == 1) {
        if (lane == 0 && rank == 0) {
            // -------------------------------------------- pair MMA issuer (even CTA)
            // (per-stage path kept short as in the one-CTA issuer)
            int g = 0;
            int s = 0;        // ring slot of the next stage to consume
            uint32_t ph = 0;  // and its fill parity
            bool ok = true;
            const uint32_t slot0 = smem_u32(smem);
            for (int t = pair; t < p.num_tiles && ok; t += npairs) {
                const TileInfo ti = get_tile<GROUPED>(t, p, &tmA, &tmB);
                const int kb0 = ti.kb0, kb1 = ti.kb1;
                const int a_mn = ti.maj & 1, b_mn = (ti.maj >> 1) & 1;
                const uint32_t idesc = make_idesc_bf16_f32(2 * kBM, S::MMA_N, a_mn, b_mn);
                const OpDesc da = op_desc(slot0, op_layout<S>(a_mn, S::A_PLANE));
                const OpDesc db =
                    op_desc(slot0 + S::PLANES * S::A_PLANE, op_layout<S>(b_mn, S::B_PLANE));
                const int chunk = PROMOTE ? p.chunk_kb : kb1 - kb0;
                for (int c0 = kb0; c0 < kb1 && ok; c0 += chunk, ++g) {
                    const int buf = S::NBUF == 2 ? (g & 1) : 0;
                    const uint32_t acc_ph = (S::NBUF == 2 ? (g >> 1) : g) & 1;
                    if (!mbar_wait_bounded_cluster(&acc_empty[buf], acc_ph ^ 1, p.lim, abort_flag,
                                                   p.err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d_tmem = tmem_base + buf * BN;
                    const int c1 = min(c0 + chunk, kb1);
                    for (int kb = c0; kb < c1; ++kb) {
                        if (!mbar_wait_bounded(&full[s], ph, p.lim, abort_flag, p.err)) {
                            ok = false;  // both CTAs' halves of stage s are counted on full[s]
                            break;
                        }
                        tc_fence_after();
                        const uint32_t slot16 = uint32_t(s) * uint32_t(S::STAGE >> 4);
                        const uint64_t a_s = da.d0 + slot16, b_s = db.d0 + slot16;
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk) {
                            const uint64_t ah = a_s + uint32_t(kk) * da.k16;
                            const uint64_t bh = b_s + uint32_t(kk) * db.k16;
                            const uint32_t acc = (kb > c0 || kk > 0) ? 1u : 0u;
                            if (NTERMS == 3) {
                                umma_bf16_pair(d_tmem, ah + da.lo16, bh, idesc, acc);
                                umma_bf16_pair(d_tmem, ah, bh + db.lo16, idesc, 1u);
                                umma_bf16_pair(d_tmem, ah, bh, idesc, 1u);
                            } else {
#pragma unroll
                                for (int j = 0; j < S::NSUB; ++j)
                                    umma_bf16_pair(d_tmem + j * S::MMA_N, ah,
                                                   bh + uint32_t(j) * (S::SUB_B >> 4), idesc, acc);
                            }
                        }
                        umma_commit_pair(&empty[s], 0x3);  // both CTAs may refill slot s
                        if (++s == stages) {
                            s = 0;
                            ph ^= 1;
                        }
                    }
                    if (!ok) break;
                    umma_commit_pair(&acc_full[buf], 0x3);
                }
            }
            umma_commit_pair(drain, 0x3);  // both CTAs learn when every pair MMA is done
            mbar_wait_drain_cluster(drain, 0, p.err);
        } else if (lane == 0) {
            // -------------------------------------------- odd CTA
            // the even CTA's MMAs read this CTA's tiles and write its TMEM
            mbar_wait_drain_cluster(drain, 0, p.err);
        }
    } else {
        // ------------------------------------------------ epilogue (both CTAs)
        constexpr int COLS = BN / 2;
        constexpr int PIECES = COLS / 32;
        const int ew = warp & 3;
        const int col_base = ((warp - 2) >> 2) * COLS;
        float* stg = staging + (warp - 2) * 32 * 33;
        float* slab = staging + (warp - 2) * 1024;  // 4 KB, 1024-byte aligned (TMA store)
        float sum[PROMOTE ? COLS : 1];
        const uint32_t leader_acc_empty = mapa_shared(smem_u32(acc_empty), 0);
        int g = 0;
        bool ok = true;
#pragma unroll 1
        for (int t = pair; t < p.num_tiles && ok; t += npairs) {
            const TileInfo ti = get_tile<GROUPED>(t, p, &tmA, &tmB);
            const int kb0 = ti.kb0, kb1 = ti.kb1;
            const int chunk = PROMOTE ? p.chunk_kb : kb1 - kb0;
            const int row0 = ti.mt * 2 * kBM + int(rank) * kBM + ew * 32;
            const int col0 = ti.nt * BN + col_base;
#pragma unroll 1
            for (int c0 = kb0; c0 < kb1; c0 += chunk, ++g) {
                const int buf = S::NBUF == 2 ? (g & 1) : 0;
                const uint32_t acc_ph = (S::NBUF == 2 ? (g >> 1) : g) & 1;
                int got = 0;
                if (lane == 0)
                    got = mbar_wait_bounded_cluster(&acc_full[buf], acc_ph, p.lim, abort_flag,
                                                    p.err);
                got = __shfl_sync(0xffffffffu, got, 0);
                if (!got) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t taddr = tmem_base + (uint32_t(ew * 32) << 16) + buf * BN + col_base;
                if (c0 + 2 * chunk >= kb1 && c0 + chunk < kb1) {
                    if (S::NSUB == 1) {
                        prefetch_c(get_epi<GROUPED>(ti.prob, ti.ks, p), row0, col0, COLS, lane);
                    } else {
                        const int tc0 = ti.nt * BN;
                        prefetch_c(get_epi<GROUPED>(ti.prob, ti.ks, p), row0,
                                   tc0 + wide_tile_col(col_base), 128, lane);
                        prefetch_c(get_epi<GROUPED>(ti.prob, ti.ks, p), row0,
                                   tc0 + wide_tile_col(col_base + 128), 128, lane);
                    }
                }
                if (PROMOTE) {
                    if (c0 == kb0) {
#pragma unroll
                        for (int q = 0; q < 2 * PIECES; ++q) {
                            uint32_t r[16];
                            tmem_ld_32x32b_x16(taddr + q * 16, r);
                            tmem_ld_wait();
#pragma unroll
                            for (int j = 0; j < 16; ++j) sum[q * 16 + j] = __uint_as_float(r[j]);
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 2 * PIECES; ++q) {
                            uint32_t r[16];
                            tmem_ld_32x32b_x16(taddr + q * 16, r);
                            tmem_ld_wait();
#pragma unroll
                            for (int j = 0; j < 16; ++j) sum[q * 16 + j] += __uint_as_float(r[j]);
                        }
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) {
                        if (rank == 0)
                            mbar_arrive(&acc_empty[buf]);
                        else
                            mbar_arrive_remote(leader_acc_empty + uint32_t(buf) * 8u);
                    }
                    if (c0 + chunk >= kb1) {
                        const EpiInfo e = pair_epi<GROUPED, BN>(ti, p);
                        if (p.c_tma && ti.prob == 0) {  // (a tail half goes to its buffer)
#pragma unroll
                            for (int q = 0; q < PIECES; ++q)
                                store_piece_tma(&sum[q * 32], slab, row0, col0 + q * 32, ti.ks,
                                                e.alpha, &tmC, lane);
                        } else {
#pragma unroll
                            for (int q = 0; q < PIECES; ++q)
                                store_piece(&sum[q * 32], stg, row0, col0 + q * 32, e, lane);
                        }
                    }
                } else {
#pragma unroll 1
                    for (int q = 0; q < PIECES; ++q) {
                        uint32_t r[32];
                        tmem_ld_32x32b_x32(taddr + q * 32, r);
                        tmem_ld_wait();
                        float v[32];
#pragma unroll
                        for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
                        const EpiInfo e = pair_epi<GROUPED, BN>(ti, p);
                        // 32-column pieces never cross a 128-column block
                        const int col = S::NSUB == 1 ? col0 + q * 32
                                                     : ti.nt * BN + wide_tile_col(col_base + q * 32);
                        if (p.c_tma && ti.prob == 0)
                            store_piece_tma(v, slab, row0, col, ti.ks, e.alpha, &tmC, lane);
                        else
                            store_piece(v, stg, row0, col, e, lane);
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) {
                        if (rank == 0)
                            mbar_arrive(&acc_empty[buf]);
                        else
                            mbar_arrive_remote(leader_acc_empty + uint32_t(buf) * 8u);
                    }
                }
            }
        }
    }

    // ------------------------------------------------ teardown
    if (warp >= 2 && lane == 0) bulk_wait_all();  // TMA stores of C finished
    tc_fence_before();
    __syncthreads();
    cluster_sync();  // no remote arrive or pair MMA may target a CTA that has left
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc_pair(tmem_base, S::TMEM_COLS);
    }
}

// ---------------------------------------------------------------- host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    });
    return fn;
}

// Raise a kernel's dynamic shared-memory limit to the most any of its
// launches asks for (kMaxSmem), once per kernel and device: the attribute
// persists, and setting it on every call costs host time.  `done` is the
// calling kernel's own bit set (bit d: device d).
template <class Kernel>
bool allow_max_smem(Kernel kern, std::atomic<uint64_t>& done) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    const uint64_t bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return true;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem) !=
        cudaSuccess)
        return false;
    done.fetch_or(bit, std::memory_order_release);
    return true;
}

// Launch attribute that lets the kernel start while the preceding kernel of
// its stream finishes (a split pass allows that from its start, a GEMM
// kernel once its operand loads are issued); the kernel's pdl_wait, before
// its first global-memory access, orders it after that kernel's reads and
// writes.  Every GEMM kernel, and the tail reduce, is launched with it.
inline void set_pdl(cudaLaunchAttribute& a) {
    a.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    a.val.programmaticStreamSerializationAllowed = 1;
}

// launch_variant's answer when a split-K cluster cannot be resident (not a
// gemm_status_t: the caller falls back to the reduce launch)
constexpr int kNoClusterRoom = -100;

template <int BN, int BK, int NTERMS, bool PROMOTE, bool GROUPED, bool FUSE = false>
int launch_variant(const CUtensorMap& ta, const CUtensorMap& tb, const CUtensorMap& tc,
                   TcParams p, const TcLaunch& cfg, int num_sms, cudaStream_t stream) {
    using S = Shape<BN, BK, NTERMS>;
    int stages = cfg.stages > 0 ? std::min(cfg.stages, S::max_stages()) : S::max_stages();
    if (stages < 2) stages = 2;
    p.stages = stages;
    // split-K partial pieces of a cluster CTA: one 4 KB slab each in the ring
    p.ring_epi = !GROUPED && p.cluster_k > 1 && p.c_tma &&
                 stages * S::STAGE >= kEpiWarps * (BN / 64) * 4096;
    p.own_local = p.ring_epi && p.sum_vec && (p.cluster_k == 2 || p.cluster_k == 4);
    // Ask for enough shared memory that co-resident CTAs can never want more
    // tensor memory than an SM has (512 columns), so tcgen05.alloc never waits.
    const int min_smem = S::TMEM_COLS == 512 ? 120 * 1024 : 80 * 1024;
    const int smem = std::max(S::smem_bytes(stages), min_smem);
    auto kern = tc_gemm_kernel<BN, BK, NTERMS, PROMOTE, GROUPED, FUSE>;
    static std::atomic<uint64_t> smem_set{0};  // bit d: limit raised on device d
    if (!allow_max_smem(kern, smem_set)) return -4;
    const int threads = FUSE ? kFusedThreads : kThreads;
    if (!GROUPED && p.cluster_k > 1) {
        // split-K slices summed in the kernel: one CTA per (tile, slice), the
        // slices of a tile one cluster
        cudaLaunchConfig_t lc{};
        lc.gridDim = dim3(unsigned(p.num_tiles), 1, 1);
        lc.blockDim = dim3(unsigned(threads), 1, 1);
        lc.dynamicSmemBytes = size_t(smem);
        lc.stream = stream;
        cudaLaunchAttribute attr[2];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = unsigned(p.cluster_k);
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        set_pdl(attr[1]);
        lc.attrs = attr;
        lc.numAttrs = 2;
        // every cluster of the grid must be resident at once (a second wave
        // would wait for whole clusters of the first to drain): the number
        // of such clusters the GPU holds, asked once per device and size
        static std::atomic<int> resident[8][9];  // +1, 0 = not asked yet
        int dev = 0;
        cudaGetDevice(&dev);
        int fit = 0;
        if (dev >= 0 && dev < 8) fit = resident[dev][p.cluster_k].load(std::memory_order_relaxed) - 1;
        if (fit < 0) {
            if (cudaOccupancyMaxActiveClusters(&fit, kern, &lc) != cudaSuccess) {
                cudaGetLastError();
                fit = 0;
            }
            if (dev >= 0 && dev < 8) resident[dev][p.cluster_k].store(fit + 1, std::memory_order_relaxed);
        }
        if (p.num_tiles / p.cluster_k > fit) return kNoClusterRoom;
        if (cudaLaunchKernelEx(&lc, kern, ta, tb, tc, p) != cudaSuccess) return -4;
        return cudaGetLastError() == cudaSuccess ? 0 : -4;
    }
    int ctas = num_sms;
    if (cfg.max_ctas > 0) ctas = std::min(ctas, cfg.max_ctas);
    ctas = std::min(ctas, p.num_tiles);
    if (ctas < 1) ctas = 1;
    cudaLaunchConfig_t lc{};
    lc.gridDim = dim3(unsigned(ctas), 1, 1);
    lc.blockDim = dim3(unsigned(threads), 1, 1);
    lc.dynamicSmemBytes = size_t(smem);
    lc.stream = stream;
    cudaLaunchAttribute attr[1];
    set_pdl(attr[0]);
    lc.attrs = attr;
    lc.numAttrs = 1;
    if (cudaLaunchKernelEx(&lc, kern, ta, tb, tc, p) != cudaSuccess) return -4;
    return cudaGetLastError() == cudaSuccess ? 0 : -4;
}

template <int BN, int BK, int NTERMS, bool PROMOTE, bool GROUPED>
int launch_pair_variant(const CUtensorMap& ta, const CUtensorMap& tb, const CUtensorMap& tc,
                        TcParams p, const TcLaunch& cfg, int num_sms, cudaStream_t stream) {
    using S = Shape2<BN, BK, NTERMS>;
    int stages = cfg.stages > 0 ? std::min(cfg.stages, S::max_stages()) : S::max_stages();
    if (stages < 2) stages = 2;
    p.stages = stages;
    const int min_smem = S::TMEM_COLS == 512 ? 120 * 1024 : 80 * 1024;
    const int smem = std::max(S::smem_bytes(stages), min_smem);
    auto kern = tc_gemm_pair_kernel<BN, BK, NTERMS, PROMOTE, GROUPED>;
    static std::atomic<uint64_t> smem_set{0};
    if (!allow_max_smem(kern, smem_set)) return -4;
    int pairs = num_sms / 2;
    if (cfg.max_ctas > 0) pairs = std::min(pairs, std::max(1, cfg.max_ctas / 2));
    pairs = std::max(1, std::min(pairs, p.num_tiles));
    cudaLaunchConfig_t lc{};
    lc.gridDim = dim3(2 * pairs, 1, 1);
    lc.blockDim = dim3(pair_threads<NTERMS>(), 1, 1);
    lc.dynamicSmemBytes = smem;
    lc.stream = stream;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    set_pdl(attr[1]);
    lc.attrs = attr;
    lc.numAttrs = 2;
    if (cudaLaunchKernelEx(&lc, kern, ta, tb, tc, p) != cudaSuccess) return -4;
    return cudaGetLastError() == cudaSuccess ? 0 : -4;
}

template <bool GROUPED>
int dispatch_pair(int nterms, bool promote, int bn, int bk, const CUtensorMap& ta,
                  const CUtensorMap& tb, const CUtensorMap& tc, const TcParams& p,
                  const TcLaunch& cfg, int num_sms, cudaStream_t s) {
#define GB300_PAIR_CASE(BN_, BK_, NT_, PR_)                                                    \
    if (bn == BN_ && bk == BK_ && nterms == NT_ && promote == PR_)                             \
        return launch_pair_variant<BN_, BK_, NT_, PR_, GROUPED>(ta, tb, tc, p, cfg, num_sms, s);
    if (GROUPED) {  // grouped plans: the split-precision shapes the plan can pick
        GB300_PAIR_CASE(256, 32, 3, true)
        GB300_PAIR_CASE(256, 64, 3, true)
        return -6;
    }
    GB300_PAIR_CASE(256, 32, 3, true)
    GB300_PAIR_CASE(256, 64, 3, true)
    GB300_PAIR_CASE(256, 32, 3, false)
    GB300_PAIR_CASE(256, 64, 3, false)
    GB300_PAIR_CASE(256, 64, 1, false)
    GB300_PAIR_CASE(256, 32, 1, false)
    GB300_PAIR_CASE(512, 64, 1, false)
#undef GB300_PAIR_CASE
    return -6;
}

template <bool GROUPED>
int dispatch(int nterms, bool promote, int bn, int bk, const CUtensorMap& ta,
             const CUtensorMap& tb, const CUtensorMap& tc, const TcParams& p, const TcLaunch& cfg,
             int num_sms, cudaStream_t s) {
    if (cfg.fuse) {  // in-kernel split: split precision, 128 x 256 tiles, BK 32
        if (nterms != 3 || bn != 256 || bk != 32) return -6;
        return promote ? launch_variant<256, 32, 3, true, GROUPED, true>(ta, tb, tc, p, cfg,
                                                                          num_sms, s)
                       : launch_variant<256, 32, 3, false, GROUPED, true>(ta, tb, tc, p, cfg,
                                                                           num_sms, s);
    }
#define GB300_TC_CASE(BN_, BK_, NT_, PR_)                                                      \
    if (bn == BN_ && bk == BK_ && nterms == NT_ && promote == PR_)                             \
        return launch_variant<BN_, BK_, NT_, PR_, GROUPED>(ta, tb, tc, p, cfg, num_sms, s);
    GB300_TC_CASE(256, 32, 3, true)
    GB300_TC_CASE(256, 64, 3, true)
    GB300_TC_CASE(128, 32, 3, true)
    GB300_TC_CASE(128, 64, 3, true)
    GB300_TC_CASE(256, 32, 3, false)
    GB300_TC_CASE(256, 64, 3, false)
    GB300_TC_CASE(128, 32, 3, false)
    GB300_TC_CASE(128, 64, 3, false)
    GB300_TC_CASE(256, 32, 1, false)
    GB300_TC_CASE(256, 64, 1, false)
    GB300_TC_CASE(128, 32, 1, false)
    GB300_TC_CASE(128, 64, 1, false)
#undef GB300_TC_CASE
    return -6;
}

// 3-D (column, row, slab) FP32 map of C (or of the split-K partial slabs)
// with the 32 x 32 box and 128-byte swizzle the TMA-store epilogue writes.
bool encode_output(CUtensorMap* map, float* base, int64_t M, int64_t N, int64_t ld, int slabs) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {cuuint64_t(N), cuuint64_t(M), cuuint64_t(slabs)};
    cuuint64_t strides[2] = {cuuint64_t(ld) * 4, cuuint64_t(ld) * cuuint64_t(M) * 4};
    cuuint32_t box[3] = {32, 32, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void fill_common(TcParams& p, const TcLaunch& cfg, int bk, int nterms, int* err_word) {
    p.raster_group = cfg.raster_group > 0 ? cfg.raster_group : 16;
    p.lim.polls = cfg.poll_limit > 0 ? cfg.poll_limit : (1ll << 30);
    p.lim.ns = 4000000000ull;
    p.err = err_word;
    const bool promote = nterms == 3 && cfg.promote_k > 0;
    p.chunk_kb = promote ? std::max(1, cfg.promote_k / bk) : 1;
    p.fuse_ops = cfg.fuse & 3;
}

}  // namespace

bool encode_operand(CUtensorMap* map, const TcOperand& op, int bk, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    if (op.mn_major && box_rows % 64 != 0) return false;
    if (op.f32) {
        // FP32 operand for the in-kernel split: unswizzled boxes (bk, box_rows)
        // K-major or (64, bk) MN-major, a third extent of 1 so that the
        // kernel's 3-D copies address it like a one-plane buffer
        const int64_t stored_rows = op.mn_major ? op.k : op.rows;
        cuuint64_t dims[3] = {cuuint64_t(op.mn_major ? op.rows : op.k), cuuint64_t(stored_rows), 1};
        cuuint64_t strides[2] = {cuuint64_t(op.ld) * 4, cuuint64_t(op.ld) * stored_rows * 4};
        cuuint32_t box[3] = {cuuint32_t(op.mn_major ? 64 : bk),
                             cuuint32_t(op.mn_major ? bk : box_rows), 1};
        cuuint32_t estr[3] = {1, 1, 1};
        return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(op.f32), dims,
                  strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    // stored rows: operand rows (K-major) or K indices (MN-major)
    const int64_t stored_rows = op.mn_major ? op.k : op.rows;
    cuuint64_t dims[3] = {cuuint64_t(op.mn_major ? op.rows : op.k), cuuint64_t(stored_rows),
                          cuuint64_t(op.planes)};
    cuuint64_t strides[2] = {cuuint64_t(op.ld) * 2,
                             cuuint64_t(op.planes > 1 ? op.plane_ld : op.ld * stored_rows) * 2};
    cuuint32_t box[3] = {cuuint32_t(op.mn_major ? 64 : bk), cuuint32_t(op.mn_major ? bk : box_rows),
                         cuuint32_t(op.box_planes > 0 ? op.box_planes : op.planes)};
    cuuint32_t estr[3] = {1, 1, 1};
    const bool sw128 = op.mn_major || bk * 2 == 128;
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<uint16_t*>(op.base), dims,
                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    sw128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

int tc_smem_bytes(int nterms, int bn, int bk, int stages, int cta_group) {
    const int planes = nterms == 1 ? 1 : 2;
    if ((bn != 128 && bn != 256 && bn != 512) || (bk != 32 && bk != 64)) return 0;
    if (cta_group == 2 && bn == 128) return 0;
    if (bn == 512 && (cta_group != 2 || nterms != 1 || bk != 64)) return 0;
    const int b_rows = cta_group == 2 ? bn / 2 : bn;  // a pair stages half of B per CTA
    const int stage = planes * (kBM * bk * 2 + b_rows * bk * 2);
    return 1024 + stages * stage + 1024 + kEpiWarps * 32 * 33 * 4;
}

// Tail split of a CTA-pair launch with one K slice: the number of tiles in
// a last wave that would keep at most half the pairs busy (0: no split).
// The library then computes each of those tiles as two halves (its even and
// its odd K blocks) on twice as many pairs and adds the halves with
// tail_reduce_kernel, instead of leaving the other pairs idle for a whole
// tile.  The same answer for the planner
// (workspace) and the launch.
int64_t tail_split_tiles(const TcLaunch& cfg, int nterms, int64_t M, int64_t N, int64_t K,
                         int split, int num_sms) {
    const bool wide = cfg.bn == 512 && cfg.cta_group == 2 && nterms == 1 && cfg.bk != 32;
    const int bn = wide ? 512 : cfg.bn == 128 ? 128 : 256;
    const int bk = wide ? 64 : cfg.bk == 64 ? 64 : 32;
    if (!(cfg.cta_group == 2 && bn >= 256) || split > 1 || cfg.fuse) return 0;
    // Half a tile's K loop must outweigh the reduce launch and the halves'
    // partial-tile traffic.  Measured against no split on the same box:
    // 3xBF16 at K = 4096 0.8-5.5 % faster (8192^3: 6 %), at K = 2048 even,
    // at K = 1024 2 % slower; plain BF16 (a third of the work per K block)
    // at K = 1024 and 4096 10 and 3 % slower.
    if (int64_t(nterms) * K < 3 * 4096) return 0;
    const int64_t tiles = ((M + 2 * kBM - 1) / (2 * kBM)) * ((N + bn - 1) / bn);
    int pairs = num_sms / 2;
    if (cfg.max_ctas > 0) pairs = std::min(pairs, std::max(1, cfg.max_ctas / 2));
    if (pairs < 2 || tiles < pairs || tiles + pairs > (1ll << 31) - 1) return 0;
    const int64_t r = tiles % pairs;
    if (r == 0 || 2 * r > pairs || (K + bk - 1) / bk < 2) return 0;
    return r;
}

int64_t tc_tail_floats(const TcLaunch& cfg, int nterms, int64_t M, int64_t N, int64_t K, int split,
                       int num_sms) {
    const bool wide = cfg.bn == 512 && cfg.cta_group == 2 && nterms == 1 && cfg.bk != 32;
    const int bn = wide ? 512 : cfg.bn == 128 ? 128 : 256;
    return tail_split_tiles(cfg, nterms, M, N, K, split, num_sms) * 2 * (2 * kBM) * bn;
}

namespace {
template <int BN>
int launch_tail_reduce(const TcParams& p, cudaStream_t stream) {
    const int vec = p.N % 4 == 0 && p.ldc % 4 == 0 && (reinterpret_cast<uintptr_t>(p.C) & 15) == 0;
    cudaLaunchConfig_t lc{};
    lc.gridDim = dim3(unsigned(p.tail_n), 16, 1);
    lc.blockDim = dim3(256, 1, 1);
    lc.stream = stream;
    cudaLaunchAttribute attr[1];
    set_pdl(attr[0]);
    lc.attrs = attr;
    lc.numAttrs = 1;
    if (cudaLaunchKernelEx(&lc, tail_reduce_kernel<BN>, p, vec) != cudaSuccess) return -4;
    return cudaGetLastError() == cudaSuccess ? 0 : -4;
}
}  // namespace

int launch_tc_gemm(const TcOperand& a, const TcOperand& b, int nterms, int64_t M, int64_t N,
                   int64_t K, float alpha, float beta, float* C, int64_t ldc, float* partial,
                   const TcLaunch& cfg, int* err_word, int num_sms, cudaStream_t stream,
                   int* launches) {
    if (M > (1ll << 31) - 256 || N > (1ll << 31) - 256 || K > (1ll << 31) - 256) return -6;
    // 512-wide tiles exist for plain BF16 on CTA pairs with BK 64 only
    const bool wide = cfg.bn == 512 && cfg.cta_group == 2 && nterms == 1 && cfg.bk != 32;
    const int bn = wide ? 512 : cfg.bn == 128 ? 128 : 256;
    const int bk = wide ? 64 : cfg.bk == 64 ? 64 : 32;
    const bool pair = cfg.cta_group == 2 && bn >= 256;
    const int bm = pair ? 2 * kBM : kBM;  // output rows per tile (per CTA pair)
    TcParams p{};
    p.maj = (a.mn_major ? 1 : 0) | (b.mn_major ? 2 : 0);
    p.M = int(M);
    p.N = int(N);
    p.K = int(K);
    p.alpha = alpha;
    p.beta = beta;
    p.C = C;
    p.ldc = ldc;
    p.num_m = int((M + bm - 1) / bm);
    p.num_n = int((N + bn - 1) / bn);
    p.k_blocks = int((K + bk - 1) / bk);
    int split = std::max(1, cfg.split_k);
    split = std::min(split, p.k_blocks);
    p.kb_per_split = (p.k_blocks + split - 1) / split;
    split = (p.k_blocks + p.kb_per_split - 1) / p.kb_per_split;  // every slice non-empty
    p.split_k = split;
    p.partial = partial;
    if (split > 1 && partial == nullptr) return -3;
    p.num_tiles = p.num_m * p.num_n * split;
    fill_common(p, cfg, bk, nterms, err_word);
    CUtensorMap ta, tb, tc{};
    if (!encode_operand(&ta, a, bk, kBM) || !encode_operand(&tb, b, bk, pair ? bn / 2 : bn))
        return -4;
    // beta == 0 (or split-K partials): store C tiles with TMA when C allows it
    if (split > 1) {
        p.c_tma = (N % 4 == 0) && encode_output(&tc, partial, M, N, N, split);
    } else if (beta == 0.0f && (reinterpret_cast<uintptr_t>(C) & 15) == 0 && ldc % 4 == 0) {
        p.c_tma = encode_output(&tc, C, M, N, ldc, 1);
    }
    // A tile whose K range is one accumulation chunk has nothing to promote:
    // the kernel without promotion stores the same TMEM sums, bit for bit,
    // without holding them in registers first.
    const bool promote = nterms == 3 && cfg.promote_k > 0 && p.kb_per_split > p.chunk_kb;
    // Split-K slices summed inside the GEMM kernel (a cluster of `split` CTAs
    // per tile, at most 8 so the cluster size stays portable) instead of by
    // a reduce launch; the same bits either way.  Only when every (tile,
    // slice) has its own SM: with a second wave the clusters of the first
    // must drain before those of the second start, which measured slower
    // than persistent CTAs and the reduce launch (split-K 6 and 8 on
    // (128, 8192, 8192): 0.050 / 0.059 ms against 0.046 / 0.041 ms).
    // Cluster sizes 2, 4 and 8 only: with 5 slices (28 clusters, which the
    // occupancy query says fit) the in-kernel split form measured 0.110 ms
    // at (128, 7168, 8192) against 0.073 ms with persistent CTAs and the
    // reduce launch; 3 slices gained nothing.
    // `partial` with one K slice: the tail-split buffer the planner reserved
    const int64_t tail = partial && split == 1
                             ? tail_split_tiles(cfg, nterms, M, N, K, split, num_sms)
                             : 0;
    if (tail > 0) {
        p.tail_n = int(tail);
        p.tail_base = p.num_tiles - p.tail_n;
        p.tail_part = partial;
        p.num_tiles += p.tail_n;
    }
    if ((split == 2 || split == 4 || split == 8) && !pair && cfg.splitk_reduce != 1 &&
        p.num_tiles <= num_sms) {
        p.cluster_k = split;
        p.sum_vec = N % 4 == 0 && ldc % 4 == 0 && (reinterpret_cast<uintptr_t>(C) & 15) == 0;
    }
    int rc = pair ? dispatch_pair<false>(nterms, promote, bn, bk, ta, tb, tc, p, cfg, num_sms,
                                         stream)
                  : dispatch<false>(nterms, promote, bn, bk, ta, tb, tc, p, cfg, num_sms, stream);
    if (rc == kNoClusterRoom) {  // no room for such a cluster: persistent CTAs, reduce launch
        p.cluster_k = 0;
        rc = dispatch<false>(nterms, promote, bn, bk, ta, tb, tc, p, cfg, num_sms, stream);
    }
    if (rc != 0) return rc;
    int n = 1;
    if (p.tail_n > 0) {
        if ((bn == 512 ? launch_tail_reduce<512>(p, stream) : launch_tail_reduce<256>(p, stream)) != 0)
            return -4;
        ++n;
    }
    if (split > 1 && p.cluster_k == 0) {
        if (launch_splitk_reduce(M, N, split, partial, alpha, beta, C, ldc, stream) != cudaSuccess)
            return -4;
        ++n;
    }
    if (launches) *launches += n;
    return 0;
}

int launch_tc_syr2k(const TcOperand& xy, int nterms, int uplo, int64_t N, int64_t K, float alpha,
                    float beta, float* C, int64_t ldc, const TcLaunch& cfg, int* err_word,
                    int num_sms, cudaStream_t stream, int* launches) {
    const int P = nterms == 1 ? 1 : 2;
    if (uplo != 1 && uplo != 2) return -1;
    if (xy.planes != 2 * P || xy.box_planes != P) return -1;
    if (N > (1ll << 31) - 256 || K > (1ll << 30) - 256) return -6;
    const int bn = cfg.bn == 128 ? 128 : 256;
    const int bk = cfg.bk == 64 ? 64 : 32;
    TcParams p{};
    p.M = int(N);
    p.N = int(N);
    p.K = int(K);
    p.alpha = alpha;
    p.beta = beta;
    p.C = C;
    p.ldc = ldc;
    p.num_m = int((N + kBM - 1) / kBM);
    p.num_n = int((N + bn - 1) / bn);
    p.syr_kb = int((K + bk - 1) / bk);
    p.k_blocks = 2 * p.syr_kb;
    p.kb_per_split = p.k_blocks;
    p.split_k = 1;
    p.uplo = uplo;
    p.syr_plane = P;
    p.tri_r = bn / kBM;
    // tiles meeting the triangle (host copy of the kernel's tri_tiles_before(num_m))
    const int64_t r = p.tri_r, m = p.num_m;
    const int64_t q = m / 2;
    const int64_t fsum = r == 1 ? m * (m - 1) / 2 : q * (q - 1) + ((m & 1) ? q : 0);
    const int64_t tiles = uplo == 1 ? fsum + m : m * p.num_n - fsum;
    if (tiles > (1ll << 31) - 1) return -6;
    p.num_tiles = int(tiles);
    p.maj = xy.mn_major ? 3 : 0;
    fill_common(p, cfg, bk, nterms, err_word);
    CUtensorMap ta, tb, tc{};
    if (!encode_operand(&ta, xy, bk, kBM) || !encode_operand(&tb, xy, bk, bn)) return -4;
    p.c_tma = 0;  // diagonal tiles store only their triangle
    const bool promote = nterms == 3 && cfg.promote_k > 0 && p.k_blocks > p.chunk_kb;
    const int rc = dispatch<false>(nterms, promote, bn, bk, ta, tb, tc, p, cfg, num_sms, stream);
    if (rc != 0) return rc;
    if (launches) *launches += 1;
    return 0;
}

int launch_tc_grouped(int nterms, const TcLaunch& cfg, const GroupedProblem* dev_problems,
                      const CUtensorMap* dev_maps, const int* dev_tile_prob, int count,
                      int total_tiles, int* err_word, int num_sms, cudaStream_t stream) {
    if (count <= 0 || total_tiles <= 0) return 0;
    const int bn = cfg.bn == 128 ? 128 : 256;
    const int bk = cfg.bk == 64 ? 64 : 32;
    TcParams p{};
    p.num_tiles = total_tiles;
    p.split_k = 1;
    p.problems = dev_problems;
    p.maps = dev_maps;
    p.tile_prob = dev_tile_prob;
    p.count = count;
    fill_common(p, cfg, bk, nterms, err_word);
    CUtensorMap unused{};  // grouped kernels read their maps from dev_maps
    const bool promote = nterms == 3 && cfg.promote_k > 0;
    if (cfg.cta_group == 2 && bn == 256)
        return dispatch_pair<true>(nterms, promote, bn, bk, unused, unused, unused, p, cfg, num_sms,
                                   stream);
    return dispatch<true>(nterms, promote, bn, bk, unused, unused, unused, p, cfg, num_sms,
                          stream);
}

}  // namespace gb300
