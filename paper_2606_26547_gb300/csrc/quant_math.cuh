// Element conversions of the row quantisation (Sec. 4.2 "Element Type
// Representation"), shared by the quantiser kernels and the tensor-core
// kernel that quantises its own query tiles.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

namespace hdc {

// Smallest k with amax <= 448 * 2^k (k = 0 for amax == 0), from the bits of
// the FP32 amax = 2^e * (1 + frac/2^23): 448 = 2^8 * 1.75, so k = e - 8 when
// 1 + frac/2^23 <= 1.75 and e - 7 otherwise.  Integer-only (no FP64).
__device__ __forceinline__ int pow2_scale_exp(float amax)
{
    const uint32_t b = __float_as_uint(amax) & 0x7fffffffu;
    if (b == 0) return 0;
    int e;
    uint32_t frac;
    if (b >= 0x00800000u) {
        e = (int)(b >> 23) - 127;
        frac = b & 0x7fffffu;
    } else {  // subnormal: normalise the leading bit
        const int p = 31 - __clz(b);
        e = p - 149;
        frac = (b << (23 - p)) & 0x7fffffu;
    }
    return e - 8 + (frac > 0x600000u ? 1 : 0);
}

// x * 2^-k exactly (the result is at most 448 in magnitude, so scaling never
// rounds a value that survives the E4M3 conversion).
__device__ __forceinline__ float scale_pow2(float x, int k)
{
    if (k >= -126) return x * __int_as_float((127 - k) << 23);
    return (x * __int_as_float((127 + 64) << 23)) * __int_as_float((127 - k - 64) << 23);
}

__device__ __forceinline__ uint32_t to_e4m3x4(float a, float b, float c, float d)
{
    const __nv_fp8x2_storage_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
    const __nv_fp8x2_storage_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
    return (uint32_t)lo | ((uint32_t)hi << 16);
}

__device__ __forceinline__ uint2 to_bf16x4(float a, float b, float c, float d)
{
    __nv_bfloat162 x = __floats2bfloat162_rn(a, b), y = __floats2bfloat162_rn(c, d);
    return make_uint2(*reinterpret_cast<uint32_t *>(&x), *reinterpret_cast<uint32_t *>(&y));
}

}  // namespace hdc
