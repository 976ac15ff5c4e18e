// K1 (row quantisation) and class-hypervector preparation.
//
// Row quantisation (Sec. 4.2 "Element Type Representation"): BF16 by
// round-to-nearest-even; FP8 E4M3 by a per-row power-of-two scale
// s = smallest 2^k with amax <= 448*s, then round-to-nearest-even with
// saturation.  Scaling by a power of two is exact, so x/s is the same real
// number on every device and the positive scale leaves sign(x.B) unchanged.
//
// Class preparation: b-bit class hypervectors quantised per class with a
// symmetric rule (Q = 2^(b-1)-1, M = max|acc|, nearest integer of acc*Q/M,
// halves away from zero), restricted to the kept dimensions and stored as
// two's-complement bit planes for popcount arithmetic.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "hdc_internal.cuh"

namespace hdc {
namespace {

// Smallest k with amax <= 448 * 2^k (k = 0 for amax == 0).  Double
// comparisons are exact: 448 * 2^k and the FP32 amax are both representable.
__device__ int pow2_scale_exp(float amax)
{
    if (!(amax > 0.f)) return 0;
    double a = (double)amax;
    int k = ilogb(a) - 8;
    while (a > ldexp(448.0, k)) k++;
    while (a <= ldexp(448.0, k - 1)) k--;
    return k;
}

__device__ __forceinline__ float ldg_or0(const float *p, int f, int F) { return f < F ? __ldg(p + f) : 0.f; }

template <int ENC>
__global__ void __launch_bounds__(256) quant_rows_kernel(const float *__restrict__ src, int64_t lds,
                                                         int64_t row_off, int64_t row_step, int64_t nrows,
                                                         int F, void *__restrict__ dst, int ldd,
                                                         float *__restrict__ scale)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < nrows; r += nwarps) {
        const float *row = src + (row_off + r * row_step) * lds;
        float mul = 1.f;
        int k = 0;
        bool slow = false;
        if (ENC == HDC_ENC_FP8_E4M3) {
            float amax = 0.f;
            for (int f = lane; f < F; f += 32) amax = fmaxf(amax, fabsf(__ldg(row + f)));
#pragma unroll
            for (int o = 16; o; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
            k = pow2_scale_exp(amax);
            // 2^-k as an FP32 normal number when in range; else go through double
            if (k >= -126 && k <= 126) mul = __int_as_float((127 - k) << 23);
            else slow = true;
            if (lane == 0) scale[r] = (float)ldexp(1.0, k);
        }
        // each lane converts 4 consecutive elements per step
        for (int f0 = lane * 4; f0 < ldd; f0 += 128) {
            float v[4];
#pragma unroll
            for (int j = 0; j < 4; j++) v[j] = ldg_or0(row, f0 + j, F);
            if (ENC == HDC_ENC_FP32) {
                float *o = (float *)dst + r * (int64_t)ldd + f0;
#pragma unroll
                for (int j = 0; j < 4; j++)
                    if (f0 + j < ldd) o[j] = v[j];
            } else if (ENC == HDC_ENC_BF16) {
                __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]);
                __nv_bfloat162 b = __floats2bfloat162_rn(v[2], v[3]);
                uint2 pk;
                pk.x = *reinterpret_cast<uint32_t *>(&a);
                pk.y = *reinterpret_cast<uint32_t *>(&b);
                *reinterpret_cast<uint2 *>((__nv_bfloat16 *)dst + r * (int64_t)ldd + f0) = pk;
            } else {
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    if (slow) v[j] = (float)((double)v[j] * ldexp(1.0, -k));
                    else v[j] *= mul;
                }
                __nv_fp8x2_storage_t lo = __nv_cvt_float2_to_fp8x2(make_float2(v[0], v[1]), __NV_SATFINITE, __NV_E4M3);
                __nv_fp8x2_storage_t hi = __nv_cvt_float2_to_fp8x2(make_float2(v[2], v[3]), __NV_SATFINITE, __NV_E4M3);
                uint32_t pk = (uint32_t)lo | ((uint32_t)hi << 16);
                *reinterpret_cast<uint32_t *>((uint8_t *)dst + r * (int64_t)ldd + f0) = pk;
            }
        }
    }
}

// One block per class.  b == 1: plane 0 = sign bits.  b > 1: symmetric
// per-class quantisation, two's-complement planes, sums and norms over K.
__global__ void __launch_bounds__(256) class_prepare_kernel(const int32_t *__restrict__ acc, int D, int64_t s0,
                                                            int64_t stride, int64_t Dk, int b, int C,
                                                            uint32_t *__restrict__ planes, int W,
                                                            int32_t *__restrict__ csum, double *__restrict__ cnorm)
{
    __shared__ long long s_max;
    __shared__ long long s_sum, s_sq;
    const int c = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int32_t *a = acc + (int64_t)c * D;
    if (threadIdx.x == 0) { s_max = 0; s_sum = 0; s_sq = 0; }
    __syncthreads();
    long long M = 0;
    if (b > 1) {
        long long m = 0;
        for (int d = threadIdx.x; d < D; d += blockDim.x) {
            long long v = a[d];
            m = max(m, v < 0 ? -v : v);
        }
        atomicMax(&s_max, m);
        __syncthreads();
        M = s_max;
    }
    const long long Q = (1ll << (b - 1)) - 1;
    long long lsum = 0, lsq = 0;
    for (int w = warp; w < W; w += nw) {
        int64_t k = (int64_t)w * 32 + lane;
        long long val = 0;
        bool kept = k < Dk;
        if (kept) {
            long long x = a[s0 + k * stride];
            if (b == 1) {
                val = x < 0 ? -1 : 1;
            } else if (M > 0) {
                long long mag = x < 0 ? -x : x;
                long long r = (2 * mag * Q + M) / (2 * M);
                val = x < 0 ? -r : r;
            }
        }
        lsum += val;
        lsq += val * val;
        for (int j = 0; j < b; j++) {
            // b == 1: the single plane is the sign (set bit = element -1)
            bool bit = b == 1 ? val < 0 : ((val >> j) & 1) != 0;
            unsigned bal = __ballot_sync(0xffffffffu, kept && bit);
            if (lane == 0) planes[((int64_t)j * C + c) * W + w] = bal;
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
        lsq += __shfl_xor_sync(0xffffffffu, lsq, o);
    }
    if (lane == 0) {
        atomicAdd((unsigned long long *)&s_sum, (unsigned long long)lsum);
        atomicAdd((unsigned long long *)&s_sq, (unsigned long long)lsq);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        csum[c] = (int32_t)s_sum;
        cnorm[c] = sqrt((double)s_sq);
    }
}

}  // namespace

cudaError_t launch_quant_rows(const float *src, int64_t lds, int64_t row_off, int64_t row_step, int64_t nrows,
                              int F, int enc, void *dst, int ldd, float *scale, cudaStream_t st)
{
    if (nrows <= 0) return cudaSuccess;
    int64_t blocks = (nrows + 7) / 8;
    if (blocks > 152 * 16) blocks = 152 * 16;
    dim3 g((unsigned)blocks), b(256);
    switch (enc) {
    case HDC_ENC_FP32:
        quant_rows_kernel<HDC_ENC_FP32><<<g, b, 0, st>>>(src, lds, row_off, row_step, nrows, F, dst, ldd, scale);
        break;
    case HDC_ENC_BF16:
        quant_rows_kernel<HDC_ENC_BF16><<<g, b, 0, st>>>(src, lds, row_off, row_step, nrows, F, dst, ldd, scale);
        break;
    default:
        quant_rows_kernel<HDC_ENC_FP8_E4M3><<<g, b, 0, st>>>(src, lds, row_off, row_step, nrows, F, dst, ldd, scale);
    }
    return cudaGetLastError();
}

cudaError_t launch_class_prepare(const int32_t *acc, int C, int D, const Perf &p, int b, uint32_t *planes, int W,
                                 int32_t *csum, double *cnorm, cudaStream_t st)
{
    if (C <= 0) return cudaSuccess;
    class_prepare_kernel<<<C, 256, 0, st>>>(acc, D, p.s0, p.stride, p.Dk, b, C, planes, W, csum, cnorm);
    return cudaGetLastError();
}

}  // namespace hdc
