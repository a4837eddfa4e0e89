// HBM-bound helper kernels of the GEMM path.
//
//  * split_bf16: the packing step (Algorithm 1's pack(), Section 3.1) for the
//    tensor-core modes: op(X) is re-laid out K-contiguous for the MMA and
//    each FP32 value x is written as hi = bf16_rne(x), lo = bf16_rne(x - hi)
//    (lo = 0 where hi is not finite).  x - hi is exact in FP32, so hi + lo
//    keeps x to within 2^-16 |x|.  The split is not in the paper.
//  * pack_bf16: the same re-layout for BF16 inputs (no arithmetic).
//  * scale_c: C <- beta * C, the K == 0 / alpha == 0 quick return (of a
//    whole matrix, or of one triangle for SYR2K).
//  * splitk_reduce: C <- alpha * sum_s P_s + beta * C over split-K partial
//    sums, in increasing s (beta applied once, as in Algorithm 1).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "internal.h"
#include "split_bf16.cuh"

namespace gb300 {

namespace {

__device__ __forceinline__ void split1(float x, uint16_t& h, uint16_t& l) {
    split_bf16_1(x, h, l);
}

__device__ __forceinline__ uint32_t pack2(uint16_t a, uint16_t b) { return pack_bf16x2(a, b); }

// Let a GEMM launched as this kernel's programmatic dependent start its set-up
// (barriers, tensor memory) once every block of this kernel has begun; the
// GEMM waits for this kernel's completion before reading what it wrote.
__device__ __forceinline__ void allow_dependent_launch() {
    asm volatile("griddepcontrol.launch_dependents;");
}

int grid_for(int64_t work, int per_block) {
    static int sms_of[64] = {};  // SM count per device, queried once
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && sms_of[dev] > 0) {
        sms = sms_of[dev];
    } else {
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (dev >= 0 && dev < 64) sms_of[dev] = sms;
    }
    const int64_t want = (work + per_block - 1) / per_block;
    return int(std::max<int64_t>(1, std::min<int64_t>(want, int64_t(sms) * 16)));
}

// Y = X (no transpose): each thread converts 8 consecutive elements of a row
// and writes 16 bytes of hi and 16 bytes of lo; block `bid` of `nblk`.
__device__ __forceinline__ void split_rows_body(int64_t rows, int64_t cols,
                                                const float* __restrict__ X, int64_t ldx,
                                                uint16_t* __restrict__ hi,
                                                uint16_t* __restrict__ lo, int64_t ldo, int x_vec,
                                                int bid, int nblk) {
    const int64_t chunks_per_row = (cols + 7) / 8;
    const int64_t total = rows * chunks_per_row;
    for (int64_t idx = bid * int64_t(blockDim.x) + threadIdx.x; idx < total;
         idx += int64_t(nblk) * blockDim.x) {
        const int64_t r = idx / chunks_per_row;
        const int64_t c0 = (idx - r * chunks_per_row) * 8;
        const float* src = X + r * ldx + c0;
        float v[8];
        if (x_vec && c0 + 8 <= cols) {
            const float4 a = __ldcs(reinterpret_cast<const float4*>(src));
            const float4 b = __ldcs(reinterpret_cast<const float4*>(src) + 1);
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
            v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = (c0 + q < cols) ? src[q] : 0.0f;
        }
        uint16_t h[8], l[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) split1(v[q], h[q], l[q]);
        uint16_t* dh = hi + r * ldo + c0;
        uint16_t* dl = lo ? lo + r * ldo + c0 : nullptr;
        if (c0 + 8 <= cols) {
            *reinterpret_cast<uint4*>(dh) =
                make_uint4(pack2(h[0], h[1]), pack2(h[2], h[3]), pack2(h[4], h[5]), pack2(h[6], h[7]));
            if (dl)
                *reinterpret_cast<uint4*>(dl) = make_uint4(pack2(l[0], l[1]), pack2(l[2], l[3]),
                                                           pack2(l[4], l[5]), pack2(l[6], l[7]));
        } else {
            for (int q = 0; q < 8 && c0 + q < cols; ++q) {
                dh[q] = h[q];
                if (dl) dl[q] = l[q];
            }
        }
    }
}

__global__ void __launch_bounds__(256) split_rows_kernel(int64_t rows, int64_t cols,
                                                         const float* __restrict__ X, int64_t ldx,
                                                         uint16_t* __restrict__ hi,
                                                         uint16_t* __restrict__ lo, int64_t ldo,
                                                         int x_vec) {
    allow_dependent_launch();
    split_rows_body(rows, cols, X, ldx, hi, lo, ldo, x_vec, blockIdx.x, gridDim.x);
}

// Y = X^T through a 64 x 64 shared-memory tile: reads along X's rows, writes
// along Y's rows, both coalesced.  T is float (split into hi/lo) or
// uint16_t (BF16 copy into `hi`); block `bid` of `nblk` (every thread of a
// block calls it: it synchronises the block).
template <typename T>
__device__ __forceinline__ void transpose_body(int64_t rows, int64_t cols,
                                               const T* __restrict__ X, int64_t ldx,
                                               uint16_t* __restrict__ hi,
                                               uint16_t* __restrict__ lo, int64_t ldo,
                                               T (*tile)[65], int bid, int nblk) {
    // Y is rows x cols; X is cols x rows.  Tile: Y rows [r0, r0+64), Y cols [c0, c0+64).
    const int64_t tiles_r = (rows + 63) / 64;
    const int64_t tiles_c = (cols + 63) / 64;
    const int tid = threadIdx.x;
    for (int64_t tIdx = bid; tIdx < tiles_r * tiles_c; tIdx += nblk) {
        const int64_t r0 = (tIdx % tiles_r) * 64;
        const int64_t c0 = (tIdx / tiles_r) * 64;
        // load: X row (c0 + i), columns r0 .. r0+63
#pragma unroll
        for (int pass = 0; pass < 16; ++pass) {
            const int i = pass * 4 + (tid >> 6);
            const int j = tid & 63;
            const int64_t xr = c0 + i, xc = r0 + j;
            tile[i][j] = (xr < cols && xc < rows) ? X[xr * ldx + xc] : T(0);
        }
        __syncthreads();
        // store: Y row (r0 + rr), 8 consecutive columns per thread
#pragma unroll
        for (int pass = 0; pass < 2; ++pass) {
            const int rr = pass * 32 + (tid >> 3);
            const int cc = (tid & 7) * 8;
            const int64_t yr = r0 + rr, yc = c0 + cc;
            if (yr < rows && yc < cols) {
                uint16_t h[8], l[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if constexpr (sizeof(T) == 4) {
                        split1(tile[cc + q][rr], h[q], l[q]);
                    } else {
                        h[q] = tile[cc + q][rr];
                        l[q] = 0;
                    }
                }
                uint16_t* dh = hi + yr * ldo + yc;
                uint16_t* dl = lo ? lo + yr * ldo + yc : nullptr;
                if (yc + 8 <= cols) {
                    *reinterpret_cast<uint4*>(dh) = make_uint4(pack2(h[0], h[1]), pack2(h[2], h[3]),
                                                               pack2(h[4], h[5]), pack2(h[6], h[7]));
                    if (dl)
                        *reinterpret_cast<uint4*>(dl) =
                            make_uint4(pack2(l[0], l[1]), pack2(l[2], l[3]), pack2(l[4], l[5]),
                                       pack2(l[6], l[7]));
                } else {
                    for (int q = 0; q < 8 && yc + q < cols; ++q) {
                        dh[q] = h[q];
                        if (dl) dl[q] = l[q];
                    }
                }
            }
        }
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(256) transpose_kernel(int64_t rows, int64_t cols,
                                                        const T* __restrict__ X, int64_t ldx,
                                                        uint16_t* __restrict__ hi,
                                                        uint16_t* __restrict__ lo, int64_t ldo) {
    __shared__ T tile[64][65];
    allow_dependent_launch();
    transpose_body<T>(rows, cols, X, ldx, hi, lo, ldo, tile, blockIdx.x, gridDim.x);
}

// Both operands of a GEMM split in one launch: blocks [0, a.blocks) work on
// a, the rest on b, each with the body of its single-matrix kernel (a block
// takes one branch, so the transposing body's barriers stay block-uniform).
__global__ void __launch_bounds__(256) split_pair_kernel(const SplitArg a, const SplitArg b) {
    __shared__ float tile[64][65];
    allow_dependent_launch();
    const bool second = int(blockIdx.x) >= a.blocks;
    const SplitArg& j = second ? b : a;
    const int bid = second ? int(blockIdx.x) - a.blocks : int(blockIdx.x);
    if (j.trans)
        transpose_body<float>(j.rows, j.cols, j.X, j.ldx, j.hi, j.lo, j.ldo, tile, bid, j.blocks);
    else
        split_rows_body(j.rows, j.cols, j.X, j.ldx, j.hi, j.lo, j.ldo, j.x_vec, bid, j.blocks);
}

// Y = X^T in FP32 (Y rows x cols, X stored cols x rows) through a 64 x 64
// shared-memory tile, both sides coalesced: the pack pass that hands the FP32
// SIMT kernel operands with rows along M and N.
__global__ void __launch_bounds__(256) transpose_f32_kernel(int64_t rows, int64_t cols,
                                                            const float* __restrict__ X,
                                                            int64_t ldx, float* __restrict__ Y,
                                                            int64_t ldy, int y_vec) {
    __shared__ float tile[64][65];
    const int64_t tiles_r = (rows + 63) / 64;
    const int64_t tiles_c = (cols + 63) / 64;
    const int tid = threadIdx.x;
    for (int64_t tIdx = blockIdx.x; tIdx < tiles_r * tiles_c; tIdx += gridDim.x) {
        const int64_t r0 = (tIdx % tiles_r) * 64;
        const int64_t c0 = (tIdx / tiles_r) * 64;
#pragma unroll
        for (int pass = 0; pass < 16; ++pass) {
            const int i = pass * 4 + (tid >> 6);
            const int j = tid & 63;
            const int64_t xr = c0 + i, xc = r0 + j;
            tile[i][j] = (xr < cols && xc < rows) ? X[xr * ldx + xc] : 0.0f;
        }
        __syncthreads();
        // Y row r0 + rr, 4 consecutive columns per thread
#pragma unroll
        for (int pass = 0; pass < 4; ++pass) {
            const int rr = pass * 16 + (tid >> 4);
            const int cc = (tid & 15) * 4;
            const int64_t yr = r0 + rr, yc = c0 + cc;
            if (yr < rows && yc < cols) {
                float* dy = Y + yr * ldy + yc;
                if (y_vec && yc + 4 <= cols) {
                    *reinterpret_cast<float4*>(dy) = make_float4(
                        tile[cc][rr], tile[cc + 1][rr], tile[cc + 2][rr], tile[cc + 3][rr]);
                } else {
                    for (int q = 0; q < 4 && yc + q < cols; ++q) dy[q] = tile[cc + q][rr];
                }
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) pack_rows_kernel(int64_t rows, int64_t cols,
                                                        const uint16_t* __restrict__ X, int64_t ldx,
                                                        uint16_t* __restrict__ out, int64_t ldo) {
    const int64_t total = rows * cols;
    for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < total;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int64_t r = idx / cols, c = idx - r * cols;
        out[r * ldo + c] = X[r * ldx + c];
    }
}

__global__ void __launch_bounds__(256) scale_c_kernel(int64_t M, int64_t N, float beta, float* C,
                                                      int64_t ldc, int uplo) {
    const int64_t total = M * N;
    for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < total;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int64_t i = idx / N, j = idx - i * N;
        if ((uplo == 1 && j > i) || (uplo == 2 && j < i)) continue;
        float* c = C + i * ldc + j;
        *c = beta == 0.0f ? 0.0f : beta * *c;
    }
}

__global__ void __launch_bounds__(256) splitk_reduce_kernel(int64_t M, int64_t N, int split,
                                                            const float* __restrict__ P,
                                                            float alpha, float beta, float* C,
                                                            int64_t ldc, int vec) {
    const int64_t slab = M * N;
    if (vec) {
        const int64_t total = slab / 4;
        for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < total;
             idx += int64_t(gridDim.x) * blockDim.x) {
            const int64_t e = idx * 4;
            const int64_t i = e / N, j = e - i * N;
            float4 s = __ldcs(reinterpret_cast<const float4*>(P + e));
            for (int q = 1; q < split; ++q) {
                const float4 t = __ldcs(reinterpret_cast<const float4*>(P + q * slab + e));
                s.x += t.x; s.y += t.y; s.z += t.z; s.w += t.w;
            }
            float4* c = reinterpret_cast<float4*>(C + i * ldc + j);
            float4 o = make_float4(alpha * s.x, alpha * s.y, alpha * s.z, alpha * s.w);
            if (beta != 0.0f) {
                const float4 old = *c;
                o.x = fmaf(beta, old.x, o.x);
                o.y = fmaf(beta, old.y, o.y);
                o.z = fmaf(beta, old.z, o.z);
                o.w = fmaf(beta, old.w, o.w);
            }
            *c = o;
        }
    } else {
        for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < slab;
             e += int64_t(gridDim.x) * blockDim.x) {
            const int64_t i = e / N, j = e - i * N;
            float s = P[e];
            for (int q = 1; q < split; ++q) s += P[q * slab + e];
            float* c = C + i * ldc + j;
            float o = alpha * s;
            if (beta != 0.0f) o = fmaf(beta, *c, o);
            *c = o;
        }
    }
}

// Grouped split: the concatenated 64 x 64 output tiles of all jobs; each
// tile finds its job in the host-built tile -> job map.  Transposed
// jobs go through a shared-memory tile; the others convert straight along
// the rows (each thread 16 consecutive elements of one row).
__global__ void __launch_bounds__(256, 8) split_grouped_kernel(const SplitJob* __restrict__ jobs,
                                                            const int* __restrict__ tile_job,
                                                            int total_tiles) {
    __shared__ float tile[64][65];
    const int tid = threadIdx.x;
    // grid-stride over tiles, so concurrently running blocks work on
    // neighbouring tiles of the same source rows (DRAM page locality)
    for (int t = blockIdx.x; t < total_tiles; t += gridDim.x) {
        const SplitJob& j = jobs[__ldg(&tile_job[t])];
        // neighbouring tiles are neighbours along the source's rows: along
        // Y's rows (r0) for a transposed job, along Y's columns (c0) otherwise
        const int local = t - j.tile_start;
        const int tiles_c = (j.cols + 63) / 64;
        const int64_t r0 = int64_t(j.trans ? local % j.tiles_r : local / tiles_c) * 64;
        const int64_t c0 = int64_t(j.trans ? local / j.tiles_r : local % tiles_c) * 64;
        if (j.trans) {
            // X is cols x rows: read X rows c0.., columns r0.. coalesced
#pragma unroll
            for (int pass = 0; pass < 16; ++pass) {
                const int i = pass * 4 + (tid >> 6);
                const int jj = tid & 63;
                const int64_t xr = c0 + i, xc = r0 + jj;
                tile[i][jj] = (xr < j.cols && xc < j.rows) ? j.src[xr * j.ldx + xc] : 0.0f;
            }
            __syncthreads();
#pragma unroll
            for (int pass = 0; pass < 2; ++pass) {
                const int rr = pass * 32 + (tid >> 3);
                const int cc = (tid & 7) * 8;
                const int64_t yr = r0 + rr, yc = c0 + cc;
                if (yr < j.rows && yc < j.cols) {
                    uint16_t h[8], l[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) split1(tile[cc + q][rr], h[q], l[q]);
                    uint16_t* dh = j.hi + yr * j.ldo + yc;
                    uint16_t* dl = j.lo ? j.lo + yr * j.ldo + yc : nullptr;
                    if (yc + 8 <= j.cols) {
                        *reinterpret_cast<uint4*>(dh) = make_uint4(
                            pack2(h[0], h[1]), pack2(h[2], h[3]), pack2(h[4], h[5]), pack2(h[6], h[7]));
                        if (dl)
                            *reinterpret_cast<uint4*>(dl) =
                                make_uint4(pack2(l[0], l[1]), pack2(l[2], l[3]), pack2(l[4], l[5]),
                                           pack2(l[6], l[7]));
                    } else {
                        for (int q = 0; q < 8 && yc + q < j.cols; ++q) {
                            dh[q] = h[q];
                            if (dl) dl[q] = l[q];
                        }
                    }
                }
            }
            __syncthreads();
        } else {
            // 64 rows x 16 float4 per tile; float4 f = q*256 + tid, so a warp
            // reads two whole 256-byte row segments per instruction
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int f = q * 256 + tid;
                const int64_t yr = r0 + (f >> 4);
                const int64_t yc = c0 + (f & 15) * 4;
                if (yr < j.rows && yc < j.cols) {
                    const float* src = j.src + yr * j.ldx + yc;
                    float v[4];
                    if (j.x_vec && yc + 4 <= j.cols) {
                        const float4 a = __ldcs(reinterpret_cast<const float4*>(src));
                        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e) v[e] = yc + e < j.cols ? src[e] : 0.0f;
                    }
                    uint16_t h[4], l[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) split1(v[e], h[e], l[e]);
                    uint16_t* dh = j.hi + yr * j.ldo + yc;
                    uint16_t* dl = j.lo ? j.lo + yr * j.ldo + yc : nullptr;
                    if (yc + 4 <= j.cols) {  // ldo % 8 == 0 and yc % 4 == 0: 8-byte aligned
                        *reinterpret_cast<uint2*>(dh) = make_uint2(pack2(h[0], h[1]), pack2(h[2], h[3]));
                        if (dl)
                            *reinterpret_cast<uint2*>(dl) = make_uint2(pack2(l[0], l[1]), pack2(l[2], l[3]));
                    } else {
                        for (int e = 0; e < 4 && yc + e < j.cols; ++e) {
                            dh[e] = h[e];
                            if (dl) dl[e] = l[e];
                        }
                    }
                }
            }
        }
    }
}

__device__ __forceinline__ void cp_async4(float* smem_dst, const float* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                     static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst))),
                 "l"(src)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Issue the 4-byte asynchronous copies of transposed tile t (X rows c0..+63,
// columns r0..+63) into `buf`; out-of-range elements are zero-filled.
__device__ __forceinline__ void load_transposed_tile(const SplitJob* __restrict__ jobs,
                                                     const int* __restrict__ tile_job, int t,
                                                     float (*buf)[65], int tid) {
    const SplitJob& j = jobs[__ldg(&tile_job[t])];
    const int local = t - j.tile_start;
    const int64_t r0 = int64_t(local % j.tiles_r) * 64;
    const int64_t c0 = int64_t(local / j.tiles_r) * 64;
#pragma unroll
    for (int pass = 0; pass < 16; ++pass) {
        const int i = pass * 4 + (tid >> 6);
        const int jj = tid & 63;
        const int64_t xr = c0 + i, xc = r0 + jj;
        if (xr < j.cols && xc < j.rows)
            cp_async4(&buf[i][jj], j.src + xr * j.ldx + xc);
        else
            buf[i][jj] = 0.0f;
    }
    cp_async_commit();
}

// Grouped split of transposed jobs only (Y = X^T): the shared tile is double
// buffered and the next tile's copies are in flight while the current tile
// is converted and stored, so each block keeps two tiles of reads pending.
__global__ void __launch_bounds__(256, 6) split_grouped_t_kernel(const SplitJob* __restrict__ jobs,
                                                              const int* __restrict__ tile_job,
                                                              int total_tiles) {
    __shared__ float tile[2][64][65];
    const int tid = threadIdx.x;
    int t = blockIdx.x;
    if (t < total_tiles) load_transposed_tile(jobs, tile_job, t, tile[0], tid);
    for (int k = 0; t < total_tiles; t += gridDim.x, ++k) {
        const int b = k & 1;
        const int tn = t + gridDim.x;
        if (tn < total_tiles) {
            load_transposed_tile(jobs, tile_job, tn, tile[b ^ 1], tid);
            cp_async_wait<1>();  // tile t has landed; tile tn may still be in flight
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const SplitJob& j = jobs[__ldg(&tile_job[t])];
        const int local = t - j.tile_start;
        const int64_t r0 = int64_t(local % j.tiles_r) * 64;
        const int64_t c0 = int64_t(local / j.tiles_r) * 64;
#pragma unroll
        for (int pass = 0; pass < 2; ++pass) {
            const int rr = pass * 32 + (tid >> 3);
            const int cc = (tid & 7) * 8;
            const int64_t yr = r0 + rr, yc = c0 + cc;
            if (yr < j.rows && yc < j.cols) {
                uint16_t h[8], l[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) split1(tile[b][cc + q][rr], h[q], l[q]);
                uint16_t* dh = j.hi + yr * j.ldo + yc;
                uint16_t* dl = j.lo ? j.lo + yr * j.ldo + yc : nullptr;
                if (yc + 8 <= j.cols) {
                    *reinterpret_cast<uint4*>(dh) = make_uint4(pack2(h[0], h[1]), pack2(h[2], h[3]),
                                                               pack2(h[4], h[5]), pack2(h[6], h[7]));
                    if (dl)
                        *reinterpret_cast<uint4*>(dl) = make_uint4(
                            pack2(l[0], l[1]), pack2(l[2], l[3]), pack2(l[4], l[5]), pack2(l[6], l[7]));
                } else {
                    for (int q = 0; q < 8 && yc + q < j.cols; ++q) {
                        dh[q] = h[q];
                        if (dl) dl[q] = l[q];
                    }
                }
            }
        }
        __syncthreads();  // tile[b] is refilled by the copies issued next iteration
    }
}

}  // namespace

cudaError_t launch_split_grouped_t(const SplitJob* dev_jobs, const int* dev_tile_job, int njobs,
                                   int total_tiles, int num_sms, cudaStream_t stream) {
    if (njobs <= 0 || total_tiles <= 0) return cudaSuccess;
    const int grid = std::max(1, std::min(total_tiles, num_sms * 12));
    split_grouped_t_kernel<<<grid, 256, 0, stream>>>(dev_jobs, dev_tile_job, total_tiles);
    return cudaGetLastError();
}

cudaError_t launch_split_grouped(const SplitJob* dev_jobs, const int* dev_tile_job, int njobs,
                                 int total_tiles, int num_sms, cudaStream_t stream) {
    if (njobs <= 0 || total_tiles <= 0) return cudaSuccess;
    const int grid = std::max(1, std::min(total_tiles, num_sms * 16));
    split_grouped_kernel<<<grid, 256, 0, stream>>>(dev_jobs, dev_tile_job, total_tiles);
    return cudaGetLastError();
}

cudaError_t launch_split_bf16(int trans, int64_t rows, int64_t cols, const float* X, int64_t ldx,
                              uint16_t* hi, uint16_t* lo, int64_t ldo, cudaStream_t stream) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    if (!trans) {
        const int x_vec = ((reinterpret_cast<uintptr_t>(X) & 15) == 0) && (ldx % 4 == 0);
        const int64_t work = rows * ((cols + 7) / 8);
        split_rows_kernel<<<grid_for(work, 256), 256, 0, stream>>>(rows, cols, X, ldx, hi, lo, ldo,
                                                                   x_vec);
    } else {
        const int64_t tiles = ((rows + 63) / 64) * ((cols + 63) / 64);
        transpose_kernel<float><<<grid_for(tiles, 1), 256, 0, stream>>>(rows, cols, X, ldx, hi, lo,
                                                                        ldo);
    }
    return cudaGetLastError();
}

cudaError_t launch_split_bf16_pair(SplitArg a, SplitArg b, cudaStream_t stream) {
    SplitArg* js[2] = {&a, &b};
    for (SplitArg* j : js) {
        j->x_vec = ((reinterpret_cast<uintptr_t>(j->X) & 15) == 0) && (j->ldx % 4 == 0);
        // the blocks each single-matrix launch would take (0 for an empty matrix)
        j->blocks = j->rows <= 0 || j->cols <= 0 ? 0
                    : j->trans ? grid_for(((j->rows + 63) / 64) * ((j->cols + 63) / 64), 1)
                               : grid_for(j->rows * ((j->cols + 7) / 8), 256);
    }
    if (a.blocks + b.blocks == 0) return cudaSuccess;
    split_pair_kernel<<<a.blocks + b.blocks, 256, 0, stream>>>(a, b);
    return cudaGetLastError();
}

cudaError_t launch_pack_bf16(int trans, int64_t rows, int64_t cols, const uint16_t* X,
                             int64_t ldx, uint16_t* out, int64_t ldo, cudaStream_t stream) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    if (!trans) {
        pack_rows_kernel<<<grid_for(rows * cols, 256), 256, 0, stream>>>(rows, cols, X, ldx, out,
                                                                          ldo);
    } else {
        const int64_t tiles = ((rows + 63) / 64) * ((cols + 63) / 64);
        transpose_kernel<uint16_t><<<grid_for(tiles, 1), 256, 0, stream>>>(rows, cols, X, ldx, out,
                                                                           nullptr, ldo);
    }
    return cudaGetLastError();
}

cudaError_t launch_transpose_f32(int64_t rows, int64_t cols, const float* X, int64_t ldx,
                                 float* Y, int64_t ldy, cudaStream_t stream) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    const int y_vec = ((reinterpret_cast<uintptr_t>(Y) & 15) == 0) && (ldy % 4 == 0);
    const int64_t tiles = ((rows + 63) / 64) * ((cols + 63) / 64);
    transpose_f32_kernel<<<grid_for(tiles, 1), 256, 0, stream>>>(rows, cols, X, ldx, Y, ldy,
                                                                  y_vec);
    return cudaGetLastError();
}

cudaError_t launch_scale_c(int64_t M, int64_t N, float beta, float* C, int64_t ldc,
                           cudaStream_t stream, int uplo) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    scale_c_kernel<<<grid_for(M * N, 256), 256, 0, stream>>>(M, N, beta, C, ldc, uplo);
    return cudaGetLastError();
}

namespace {

// The grouped form: unit u belongs to the last job whose unit_start <= u
// (binary search over the job table), then the per-element work of
// splitk_reduce_kernel.
__global__ void __launch_bounds__(256) splitk_reduce_grouped_kernel(
    const ReduceJob* __restrict__ jobs, int njobs, long long total) {
    for (long long u = blockIdx.x * 256ll + threadIdx.x; u < total; u += gridDim.x * 256ll) {
        int lo = 0, hi = njobs;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (jobs[mid].unit_start <= u)
                lo = mid;
            else
                hi = mid;
        }
        const ReduceJob& j = jobs[lo];
        const long long slab = j.M * j.N;
        const long long e0 = u - j.unit_start;
        if (j.vec) {
            const long long e = e0 * 4;
            const long long i = e / j.N, c = e - i * j.N;
            float4 s = __ldcs(reinterpret_cast<const float4*>(j.P + e));
            for (int q = 1; q < j.split; ++q) {
                const float4 t = __ldcs(reinterpret_cast<const float4*>(j.P + q * slab + e));
                s.x += t.x; s.y += t.y; s.z += t.z; s.w += t.w;
            }
            float4* cp = reinterpret_cast<float4*>(j.C + i * j.ldc + c);
            float4 o = make_float4(j.alpha * s.x, j.alpha * s.y, j.alpha * s.z, j.alpha * s.w);
            if (j.beta != 0.0f) {
                const float4 old = *cp;
                o.x = fmaf(j.beta, old.x, o.x);
                o.y = fmaf(j.beta, old.y, o.y);
                o.z = fmaf(j.beta, old.z, o.z);
                o.w = fmaf(j.beta, old.w, o.w);
            }
            *cp = o;
        } else {
            const long long i = e0 / j.N, c = e0 - i * j.N;
            float s = j.P[e0];
            for (int q = 1; q < j.split; ++q) s += j.P[q * slab + e0];
            float* cp = j.C + i * j.ldc + c;
            float o = j.alpha * s;
            if (j.beta != 0.0f) o = fmaf(j.beta, *cp, o);
            *cp = o;
        }
    }
}

}  // namespace

cudaError_t launch_splitk_reduce_grouped(const ReduceJob* dev_jobs, int njobs,
                                         long long total_units, int num_sms, cudaStream_t stream) {
    if (njobs <= 0 || total_units <= 0) return cudaSuccess;
    const long long want = (total_units + 255) / 256;
    const int grid = int(std::max<long long>(1, std::min<long long>(want, 16ll * num_sms)));
    splitk_reduce_grouped_kernel<<<grid, 256, 0, stream>>>(dev_jobs, njobs, total_units);
    return cudaGetLastError();
}

cudaError_t launch_splitk_reduce(int64_t M, int64_t N, int split_k, const float* P, float alpha,
                                 float beta, float* C, int64_t ldc, cudaStream_t stream) {
    const int vec = (N % 4 == 0) && (ldc % 4 == 0) && ((reinterpret_cast<uintptr_t>(C) & 15) == 0) &&
                    ((reinterpret_cast<uintptr_t>(P) & 15) == 0);
    splitk_reduce_kernel<<<grid_for(vec ? M * N / 4 : M * N, 256), 256, 0, stream>>>(
        M, N, split_k, P, alpha, beta, C, ldc, vec);
    return cudaGetLastError();
}

}  // namespace gb300
