// The BF16 hi/lo split of one FP32 value, shared by the split pass
// (split.cu) and the tensor-core kernel's in-kernel split (tc_gemm.cu), so
// that both produce the same bits.  Not in the paper.
//
//   hi = bf16_rn(x);  lo = bf16_rn(x - hi), or 0 where hi is not finite.
//
// x - hi is exact in FP32 (hi keeps the top 8 significant bits of x), so
// hi + lo keeps x to within 2^-16 |x|; lo = 0 for non-finite hi keeps an
// Inf or NaN operand from turning into Inf - Inf = NaN in the lo products.
#pragma once
#include <cuda_bf16.h>

#include <cstdint>

namespace gb300 {

__device__ __forceinline__ void split_bf16_1(float x, uint16_t& h, uint16_t& l) {
    const __nv_bfloat16 hb = __float2bfloat16_rn(x);
    const float hv = __bfloat162float(hb);
    h = __bfloat16_as_ushort(hb);
    l = isfinite(hv) ? __bfloat16_as_ushort(__float2bfloat16_rn(x - hv)) : uint16_t(0);
}

// Two 16-bit halves into one 32-bit word, `a` at the lower address.
__device__ __forceinline__ uint32_t pack_bf16x2(uint16_t a, uint16_t b) {
    return uint32_t(a) | (uint32_t(b) << 16);
}

// The same split for two values at once, packed as stored (x0 in the low
// half): hi = both rounded in one conversion; lo = bf16_rn(x - hi), cleared
// in the half whose hi is Inf or NaN (exponent field all ones: adding 0x80
// to the masked exponent 0x7f80 carries into bit 15 of that half, and into
// nothing else).  A byte permute that replicates the top bit of bytes 1 and
// 3 across their halves turns those two bits into the 16-bit clear masks.
// Bit-identical to split_bf16_1 on each value.
__device__ __forceinline__ void split_bf16_2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    const float d0 = x0 - __uint_as_float(hi << 16);
    const float d1 = x1 - __uint_as_float(hi & 0xffff0000u);
    const __nv_bfloat162 l = __floats2bfloat162_rn(d0, d1);
    const uint32_t top = (hi & 0x7f807f80u) + 0x00800080u;  // bit 15 / 31: that half not finite
    uint32_t clear;
    asm("prmt.b32 %0, %1, 0, 0xBB99;" : "=r"(clear) : "r"(top));  // sign-replicate bytes 1, 3
    lo = *reinterpret_cast<const uint32_t*>(&l) & ~clear;
}

}  // namespace gb300
