// K0: random-projection encoding on CUDA cores (FFMA), fused with
// sign binarisation and bit packing (Listing 1 __hetero_hdc_matmul followed
// by Automatic Binarization, Sec. 4.2).
//
// s[i][k] = sum_f X[i][f] * Bq[k][f] in FP32; bit = s < 0 (sign(0) = +1);
// 32 consecutive dims per word.  With FP32 inputs this is the plain exact
// form of the method; with BF16/FP8 inputs the products are exact in FP32,
// which gives a CUDA-core cross-check of the tensor-core encoder.
//
// Tiling: 128 queries x 128 dims per block, K slabs of 16, 256 threads with
// 8x8 outputs each (rows ty*4+{0..3} and 64+ty*4+{0..3}, the same for
// columns with tx), double-buffered shared memory with register prefetch.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "hdc_internal.cuh"

namespace hdc {
namespace {

constexpr int BM = 128, BN = 128, BK = 16, LDS = BM + 4;

__device__ __forceinline__ void cvt4(const float *p, float *v)
{
    float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void cvt4(const __nv_bfloat16 *p, float *v)
{
    uint2 t = *reinterpret_cast<const uint2 *>(p);
    __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162 *>(&t.x), b = *reinterpret_cast<__nv_bfloat162 *>(&t.y);
    float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
    v[0] = fa.x; v[1] = fa.y; v[2] = fb.x; v[3] = fb.y;
}
__device__ __forceinline__ float fp8_to_f(uint8_t b)
{
    __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)b, __NV_E4M3);
    return __half2float(__half(h));
}
__device__ __forceinline__ void cvt4(const uint8_t *p, float *v)
{
    uint32_t t = *reinterpret_cast<const uint32_t *>(p);
#pragma unroll
    for (int j = 0; j < 4; j++) v[j] = fp8_to_f((uint8_t)(t >> (8 * j)));
}
__device__ __forceinline__ float cvt1(const float *p) { return *p; }
__device__ __forceinline__ float cvt1(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
__device__ __forceinline__ float cvt1(const uint8_t *p) { return fp8_to_f(*p); }

// Four consecutive elements [f, f+4) of a row, zero outside [0, F) or for an
// invalid row; vector load when the four are in range and aligned.
template <typename T>
__device__ __forceinline__ void load4(const T *row, bool valid, int f, int F, float *v)
{
    if (valid && f + 3 < F && (reinterpret_cast<uintptr_t>(row + f) % (4 * sizeof(T))) == 0) {
        cvt4(row + f, v);
        return;
    }
#pragma unroll
    for (int j = 0; j < 4; j++) v[j] = (valid && f + j < F) ? cvt1(row + f + j) : 0.f;
}

template <typename T>
__global__ void __launch_bounds__(256) encode_simt_kernel(const T *__restrict__ X, int64_t ldx, int64_t N, int F,
                                                          const T *__restrict__ B, int ldb, int Dk,
                                                          const float *__restrict__ sx, const float *__restrict__ sb,
                                                          uint32_t *__restrict__ H, int W, float *__restrict__ scores)
{
    __shared__ __align__(16) float As[2][BK][LDS];
    __shared__ __align__(16) float Bs[2][BK][LDS];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t m0 = (int64_t)blockIdx.y * BM;
    const int n0 = blockIdx.x * BN;

    // loader mapping: rows lr and lr+64, k offset lk
    const int lr = tid >> 2, lk = (tid & 3) * 4;
    const T *arow0 = X + (m0 + lr) * ldx, *arow1 = X + (m0 + lr + 64) * ldx;
    const bool av0 = m0 + lr < N, av1 = m0 + lr + 64 < N;
    const T *brow0 = B + (int64_t)(n0 + lr) * ldb, *brow1 = B + (int64_t)(n0 + lr + 64) * ldb;
    const bool bv0 = n0 + lr < Dk, bv1 = n0 + lr + 64 < Dk;

    float ra[8], rb[8];
    auto gload = [&](int k0) {
        load4(arow0, av0, k0 + lk, F, ra);
        load4(arow1, av1, k0 + lk, F, ra + 4);
        load4(brow0, bv0, k0 + lk, F, rb);
        load4(brow1, bv1, k0 + lk, F, rb + 4);
    };
    auto sstore = [&](int buf) {
#pragma unroll
        for (int j = 0; j < 4; j++) {
            As[buf][lk + j][lr] = ra[j];
            As[buf][lk + j][lr + 64] = ra[4 + j];
            Bs[buf][lk + j][lr] = rb[j];
            Bs[buf][lk + j][lr + 64] = rb[4 + j];
        }
    };

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; i++)
#pragma unroll
        for (int j = 0; j < 8; j++) acc[i][j] = 0.f;

    const int nk = (F + BK - 1) / BK;
    gload(0);
    sstore(0);
    __syncthreads();
    for (int kt = 0; kt < nk; kt++) {
        const int cur = kt & 1;
        if (kt + 1 < nk) gload((kt + 1) * BK);
#pragma unroll
        for (int kk = 0; kk < BK; kk++) {
            float a[8], b[8];
            *reinterpret_cast<float4 *>(a) = *reinterpret_cast<const float4 *>(&As[cur][kk][ty * 4]);
            *reinterpret_cast<float4 *>(a + 4) = *reinterpret_cast<const float4 *>(&As[cur][kk][64 + ty * 4]);
            *reinterpret_cast<float4 *>(b) = *reinterpret_cast<const float4 *>(&Bs[cur][kk][tx * 4]);
            *reinterpret_cast<float4 *>(b + 4) = *reinterpret_cast<const float4 *>(&Bs[cur][kk][64 + tx * 4]);
#pragma unroll
            for (int i = 0; i < 8; i++)
#pragma unroll
                for (int j = 0; j < 8; j++) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (kt + 1 < nk) sstore(cur ^ 1);
        __syncthreads();
    }

    // ---- epilogue: optional projections, then sign -> pack ---------------
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const int64_t row = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
        if (scores != nullptr && row < N) {
            const float rs = sx ? sx[row] : 1.f;
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const int col = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4);
                if (col < Dk) scores[row * Dk + col] = acc[i][j] * rs * (sb ? sb[col] : 1.f);
            }
        }
#pragma unroll
        for (int h = 0; h < 2; h++) {
            uint32_t nib = 0;
#pragma unroll
            for (int j = 0; j < 4; j++) nib |= (acc[i][h * 4 + j] < 0.f ? 1u : 0u) << j;
            uint32_t v = nib << (4 * (tx & 7));
            v |= __shfl_xor_sync(0xffffffffu, v, 1);
            v |= __shfl_xor_sync(0xffffffffu, v, 2);
            v |= __shfl_xor_sync(0xffffffffu, v, 4);
            if ((tx & 7) == 0 && row < N) {
                const int word = n0 / 32 + h * 2 + (tx >> 3);
                if (word < W) H[row * W + word] = v;
            }
        }
    }
}

}  // namespace

cudaError_t launch_encode_simt(const void *X, int64_t ldx, int64_t N, int F, const void *Bq, int ldb, int Dk, int enc,
                               const float *sx, const float *sb, uint32_t *H, int W, float *scores, cudaStream_t st)
{
    const int64_t chunk = (int64_t)65535 * BM;  // grid.y limit per launch
    const int es = esize_for(enc);
    for (int64_t off = 0; off < N; off += chunk) {
        const int64_t n = N - off < chunk ? N - off : chunk;
        const char *Xc = (const char *)X + off * ldx * es;
        const float *sxc = sx ? sx + off : nullptr;
        uint32_t *Hc = H + off * W;
        float *sc = scores ? scores + off * Dk : nullptr;
        dim3 grid((Dk + BN - 1) / BN, (unsigned)((n + BM - 1) / BM)), block(256);
        switch (enc) {
        case HDC_ENC_FP32:
            encode_simt_kernel<float><<<grid, block, 0, st>>>((const float *)Xc, ldx, n, F, (const float *)Bq, ldb,
                                                              Dk, sxc, sb, Hc, W, sc);
            break;
        case HDC_ENC_BF16:
            encode_simt_kernel<__nv_bfloat16><<<grid, block, 0, st>>>((const __nv_bfloat16 *)Xc, ldx, n, F,
                                                                      (const __nv_bfloat16 *)Bq, ldb, Dk, sxc, sb,
                                                                      Hc, W, sc);
            break;
        default:
            encode_simt_kernel<uint8_t><<<grid, block, 0, st>>>((const uint8_t *)Xc, ldx, n, F, (const uint8_t *)Bq,
                                                                ldb, Dk, sxc, sb, Hc, W, sc);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace hdc
