// gemm_bf16x3_noalloc: the split-precision GEMM for callers that cannot
// allocate device memory.
//
// Who needs this: code that runs where cudaMalloc is off limits -- a custom
// allocator's own hooks (which must not re-enter the allocator), a plugin
// whose host application owns all device memory and forbids other
// allocations, or a latency-critical loop that must never hit the driver's
// allocator (which can synchronise the device).  gemm() needs a handle, and
// both the handle and its workspace come from cudaMalloc; this entry point
// needs neither.
//
// Its scratch (the BF16 hi/lo copies of op(A) and op(B), i.e. the packed
// operands the tensor-core kernel reads) lives in one file-scope device array
// of kScratchBytes = 64 MiB.  The CUDA runtime reserves it when it loads this
// file's module on a GPU and keeps it until the process exits.  With lazy
// module loading (the default since CUDA 12.2) that load happens during the
// first call on each device -- the address lookup below triggers it -- so
// that first call is the one that reserves the 64 MiB and may synchronise or
// fail for lack of memory: make it once at start-up, before any stream
// capture.  Nothing here calls cudaMalloc, cudaFree or any allocating
// library routine.
//
// Host code cannot use the array's name as a device address (on the host it
// names a stand-in object), so each device's first call -- with that device
// current -- asks the runtime for the array's device address with
// cudaGetSymbolAddress and caches it; a failed lookup is not cached and is
// retried by the next call.
//
// All calls share the one array and it keeps whatever the last call wrote:
// every call overwrites the parts it reads.  A separate device error word
// collects bounded-wait expiries of every call until
// gemm_bf16x3_noalloc_check reads and clears it.  Calls whose GPU work can
// overlap (different streams, or different host threads) race on the array;
// serialise them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "../../include/gemm.h"
#include "internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;

// The scratch array itself, and a separate error word for the kernels'
// bounded waits (zero at module load; cleared by gemm_bf16x3_noalloc_check).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];
static __device__ __align__(256) int g_noalloc_err[64];

struct DeviceAddrs {
    bool ready = false;  // set only after both lookups succeeded
    unsigned char* scratch = nullptr;
    int* err = nullptr;
};
DeviceAddrs g_addrs[kMaxDevices];
std::mutex g_addrs_mu;

// The device addresses of the scratch array and the error word on the
// current device `dev` (looked up once; a failure is retried next time).
cudaError_t device_addrs(int dev, DeviceAddrs** out) {
    std::lock_guard<std::mutex> lock(g_addrs_mu);
    DeviceAddrs& d = g_addrs[dev];
    if (!d.ready) {
        void* p = nullptr;
        void* e = nullptr;
        cudaError_t rc = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (rc == cudaSuccess) rc = cudaGetSymbolAddress(&e, g_noalloc_err);
        if (rc != cudaSuccess) {
            cudaGetLastError();
            return rc;
        }
        d.scratch = static_cast<unsigned char*>(p);
        d.err = static_cast<int*>(e);
        d.ready = true;
    }
    *out = &d;
    return cudaSuccess;
}

// Current device, checked to be an sm_103 GPU within the address table.
gemm_status_t current_device(int* dev, int* sms) {
    if (cudaGetDevice(dev) != cudaSuccess || *dev < 0 || *dev >= kMaxDevices) {
        cudaGetLastError();
        return GEMM_ERR_DEVICE;
    }
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, *dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, *dev);
    cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, *dev);
    if (major != 10 || minor != 3) return GEMM_ERR_DEVICE;
    return GEMM_OK;
}

size_t round256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" gemm_status_t gemm_bf16x3_noalloc(gemm_op_t transA, gemm_op_t transB, int64_t M,
                                             int64_t N, int64_t K, float alpha, const float* A,
                                             int64_t lda, const float* B, int64_t ldb, float beta,
                                             float* C, int64_t ldc, void* stream) {
    if (transA != GEMM_OP_N && transA != GEMM_OP_T) return GEMM_ERR_ARG;
    if (transB != GEMM_OP_N && transB != GEMM_OP_T) return GEMM_ERR_ARG;
    if (M < 0 || N < 0 || K < 0) return GEMM_ERR_ARG;
    const bool reads_ab = M > 0 && N > 0 && K > 0 && alpha != 0.0f;
    if (reads_ab && (!A || !B)) return GEMM_ERR_ARG;
    if (lda < std::max<int64_t>(1, transA ? M : K)) return GEMM_ERR_ARG;
    if (ldb < std::max<int64_t>(1, transB ? K : N)) return GEMM_ERR_ARG;
    if (M > 0 && N > 0 && !C) return GEMM_ERR_ARG;
    if (ldc < std::max<int64_t>(1, N)) return GEMM_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (M == 0 || N == 0) return GEMM_OK;
    if (!reads_ab)
        return gb300::launch_scale_c(M, N, beta, C, ldc, s) == cudaSuccess ? GEMM_OK
                                                                           : GEMM_ERR_CUDA;

    // Scratch needed: hi and lo planes of op(A) (M x Kp) and of op(B)^T
    // (N x Kp), Kp = K rounded up to 8 so that rows stay 16-byte aligned.
    const int64_t kp = (K + 7) / 8 * 8;
    const size_t a_bytes = round256(size_t(2) * M * kp * 2);
    const size_t b_bytes = round256(size_t(2) * N * kp * 2);
    if (M > (int64_t(1) << 30) || N > (int64_t(1) << 30) || K > (int64_t(1) << 30) ||
        a_bytes + b_bytes > kScratchBytes)
        return GEMM_ERR_WORKSPACE;  // 4 * (M + N) * round_up(K, 8) bytes must fit in 64 MiB

    int dev = 0, sms = 0;
    const gemm_status_t dst = current_device(&dev, &sms);
    if (dst != GEMM_OK) return dst;
    DeviceAddrs* dp = nullptr;
    if (device_addrs(dev, &dp) != cudaSuccess) return GEMM_ERR_CUDA;
    DeviceAddrs& d = *dp;

    uint16_t* a_hi = reinterpret_cast<uint16_t*>(d.scratch);
    uint16_t* b_hi = reinterpret_cast<uint16_t*>(d.scratch + a_bytes);
    const int64_t a_plane = M * kp, b_plane = N * kp;
    if (gb300::launch_split_bf16(transA, M, K, A, lda, a_hi, a_hi + a_plane, kp, s) != cudaSuccess)
        return GEMM_ERR_CUDA;
    if (gb300::launch_split_bf16(!transB, N, K, B, ldb, b_hi, b_hi + b_plane, kp, s) !=
        cudaSuccess)
        return GEMM_ERR_CUDA;
    gb300::TcOperand oa{a_hi, M, K, kp, a_plane, 2};
    gb300::TcOperand ob{b_hi, N, K, kp, b_plane, 2};
    gb300::TcLaunch cfg;  // library defaults, no split-K (no partial-sum scratch)
    cfg.split_k = 1;
    int launches = 0;
    const int rc = gb300::launch_tc_gemm(oa, ob, 3, M, N, K, alpha, beta, C, ldc, nullptr, cfg,
                                         d.err, sms, s, &launches);
    return rc == 0 ? GEMM_OK : static_cast<gemm_status_t>(rc);
}

extern "C" gemm_status_t gemm_bf16x3_noalloc_check(void* stream) {
    int dev = 0, sms = 0;
    const gemm_status_t dst = current_device(&dev, &sms);
    if (dst != GEMM_OK) return dst;
    DeviceAddrs* d = nullptr;
    if (device_addrs(dev, &d) != cudaSuccess) return GEMM_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return GEMM_ERR_CUDA;
    }
    int word = 0;
    if (cudaMemcpyAsync(&word, d->err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemsetAsync(d->err, 0, sizeof(int), s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return GEMM_ERR_CUDA;
    }
    return word != 0 ? GEMM_ERR_TIMEOUT : GEMM_OK;
}
