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
#include "quant_math.cuh"

namespace hdc {
namespace {

// Four consecutive elements [f, f+4) of a row (zero past F); with GATHER,
// element f of the row is column c0 + f * cstep of the source.
template <bool VEC, bool GATHER = false>
__device__ __forceinline__ float4 load4(const float *row, int f, int F, int64_t c0 = 0, int64_t cstep = 1)
{
    if (GATHER) {
        float4 v;
        v.x = f < F ? __ldg(row + c0 + (int64_t)f * cstep) : 0.f;
        v.y = f + 1 < F ? __ldg(row + c0 + (int64_t)(f + 1) * cstep) : 0.f;
        v.z = f + 2 < F ? __ldg(row + c0 + (int64_t)(f + 2) * cstep) : 0.f;
        v.w = f + 3 < F ? __ldg(row + c0 + (int64_t)(f + 3) * cstep) : 0.f;
        return v;
    }
    if (VEC) {  // F % 4 == 0 and 16-byte aligned rows
        if (f < F) return __ldg(reinterpret_cast<const float4 *>(row + f));
        return make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float4 v;
    v.x = f < F ? __ldg(row + f) : 0.f;
    v.y = f + 1 < F ? __ldg(row + f + 1) : 0.f;
    v.z = f + 2 < F ? __ldg(row + f + 2) : 0.f;
    v.w = f + 3 < F ? __ldg(row + f + 3) : 0.f;
    return v;
}

// One warp per row; each lane owns 4 consecutive elements of every 128.
// Rows of up to 128*MAXIT elements stay in registers between the amax
// reduction and the conversion.
constexpr int MAXIT = 8;

// GATHER: the F elements of a row are the source columns c0 + f * cstep
// (the kept features of a perforated encoding reduction).
template <int ENC, bool VEC, bool GATHER = false>
__global__ void __launch_bounds__(256) quant_rows_kernel(const float *__restrict__ src, int64_t lds,
                                                         int64_t row_off, int64_t row_step, int64_t nrows,
                                                         int F, void *__restrict__ dst, int ldd,
                                                         float *__restrict__ scale, int64_t c0 = 0,
                                                         int64_t cstep = 1)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int nit = (ldd + 127) / 128;
    for (int64_t r = warp; r < nrows; r += nwarps) {
        const float *row = src + (row_off + r * row_step) * lds;
        float4 v[MAXIT];
        const bool in_regs = nit <= MAXIT;
        int k = 0;
        if (ENC == HDC_ENC_FP8_E4M3) {
            float amax = 0.f;
            if (in_regs) {
#pragma unroll
                for (int it = 0; it < MAXIT; it++)
                    if (it < nit) {
                        v[it] = load4<VEC, GATHER>(row, it * 128 + lane * 4, F, c0, cstep);
                        amax = fmaxf(amax, fmaxf(fmaxf(fabsf(v[it].x), fabsf(v[it].y)),
                                                 fmaxf(fabsf(v[it].z), fabsf(v[it].w))));
                    }
            } else {
                for (int f = lane; f < F; f += 32) amax = fmaxf(amax, fabsf(__ldg(row + c0 + (int64_t)f * cstep)));
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
            k = pow2_scale_exp(amax);
            if (lane == 0) scale[r] = k >= -126 ? __int_as_float((127 + k) << 23) : ldexpf(1.f, k);
        }
        auto emit = [&](int f0, float4 x) {
            if (ENC == HDC_ENC_FP32) {
                float *o = (float *)dst + r * (int64_t)ldd + f0;
                o[0] = x.x; o[1] = x.y; o[2] = x.z; o[3] = x.w;
            } else if (ENC == HDC_ENC_BF16) {
                *reinterpret_cast<uint2 *>((__nv_bfloat16 *)dst + r * (int64_t)ldd + f0) = to_bf16x4(x.x, x.y, x.z, x.w);
            } else {
                *reinterpret_cast<uint32_t *>((uint8_t *)dst + r * (int64_t)ldd + f0) =
                    to_e4m3x4(scale_pow2(x.x, k), scale_pow2(x.y, k), scale_pow2(x.z, k), scale_pow2(x.w, k));
            }
        };
        if (ENC == HDC_ENC_FP8_E4M3 && in_regs) {
#pragma unroll
            for (int it = 0; it < MAXIT; it++) {
                const int f0 = it * 128 + lane * 4;
                if (it < nit && f0 < ldd) emit(f0, v[it]);
            }
        } else {
            for (int f0 = lane * 4; f0 < ldd; f0 += 128) emit(f0, load4<VEC, GATHER>(row, f0, F, c0, cstep));
        }
    }
}

// ---------------------------------------------------------------------------
// Streaming variant for 16-byte aligned rows: every warp keeps a ring of
// QSLOTS rows in shared memory, filled by bulk asynchronous copies
// (cp.async.bulk, completion on one mbarrier per slot), so many rows are in
// flight per SM without holding them in registers.  The warp reduces the
// row maximum and converts straight from shared memory.  Waits are bounded
// by the global timer; on expiry the kernel records status 1 and stops.
constexpr int QSLOTS = 4, QWARPS = 4;
constexpr unsigned long long QTIMEOUT_NS = 2000000000ull;

static __device__ int g_quant_status;

__device__ __forceinline__ unsigned long long qtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool qbar_try(uint32_t a, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}

template <int ENC>
__global__ void __launch_bounds__(QWARPS * 32) quant_rows_bulk_kernel(const float *__restrict__ src, int64_t lds,
                                                                      int64_t row_off, int64_t row_step,
                                                                      int64_t nrows, int F, void *__restrict__ dst,
                                                                      int ldd, float *__restrict__ scale)
{
    extern __shared__ __align__(128) uint8_t qsm[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint32_t rowbytes = (uint32_t)F * 4u;  // multiple of 16 (F % 4 == 0)
    float *ring = reinterpret_cast<float *>(qsm + (size_t)wib * QSLOTS * rowbytes);
    uint64_t *bars = reinterpret_cast<uint64_t *>(qsm + (size_t)QWARPS * QSLOTS * rowbytes) + wib * QSLOTS;
    const int64_t gw = (int64_t)blockIdx.x * QWARPS + wib, nw = (int64_t)gridDim.x * QWARPS;
    const int64_t my_rows = gw < nrows ? (nrows - 1 - gw) / nw + 1 : 0;
    auto bar = [&](int s) { return (uint32_t)__cvta_generic_to_shared(bars + s); };
    auto issue = [&](int64_t i) {  // lane 0: fetch this warp's i-th row into slot i % QSLOTS
        const int s = (int)(i % QSLOTS);
        const float *g = src + (row_off + (gw + i * nw) * row_step) * lds;
        const uint32_t d = (uint32_t)__cvta_generic_to_shared(ring + (size_t)s * F);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar(s)), "r"(rowbytes) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d),
                     "l"(g), "r"(rowbytes), "r"(bar(s))
                     : "memory");
    };
    if (lane == 0) {
        for (int s = 0; s < QSLOTS; s++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar(s)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int64_t i = 0; i < my_rows && i < QSLOTS; i++) issue(i);
    }
    __syncwarp();
    for (int64_t i = 0; i < my_rows; i++) {
        const int s = (int)(i % QSLOTS);
        const uint32_t parity = (uint32_t)((i / QSLOTS) & 1);
        bool ok = qbar_try(bar(s), parity);
        if (!ok) {
            const unsigned long long t0 = qtimer();
            while (!(ok = qbar_try(bar(s), parity)) && qtimer() - t0 < QTIMEOUT_NS) {}
        }
        if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0) {
                atomicCAS(&g_quant_status, 0, 1);
                // let this warp's copies in flight land before the block exits
                const int64_t issued = i + QSLOTS < my_rows ? i + QSLOTS : my_rows;
                for (int64_t j = i; j < issued; j++) {
                    const unsigned long long t0 = qtimer();
                    while (!qbar_try(bar((int)(j % QSLOTS)), (uint32_t)((j / QSLOTS) & 1)) &&
                           qtimer() - t0 < 100000000ull) {}
                }
            }
            break;
        }
        const float *row = ring + (size_t)s * F;
        const int64_t r = gw + i * nw;
        int k = 0;
        if (ENC == HDC_ENC_FP8_E4M3) {
            float amax = 0.f;
            for (int f = lane * 4; f < F; f += 128) {
                const float4 x = *reinterpret_cast<const float4 *>(row + f);
                amax = fmaxf(amax, fmaxf(fmaxf(fabsf(x.x), fabsf(x.y)), fmaxf(fabsf(x.z), fabsf(x.w))));
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
            k = pow2_scale_exp(amax);
            if (lane == 0) scale[r] = k >= -126 ? __int_as_float((127 + k) << 23) : ldexpf(1.f, k);
        }
        for (int f0 = lane * 4; f0 < ldd; f0 += 128) {
            const float4 x = f0 < F ? *reinterpret_cast<const float4 *>(row + f0) : make_float4(0.f, 0.f, 0.f, 0.f);
            if (ENC == HDC_ENC_FP32) {
                *reinterpret_cast<float4 *>((float *)dst + r * (int64_t)ldd + f0) = x;
            } else if (ENC == HDC_ENC_BF16) {
                *reinterpret_cast<uint2 *>((__nv_bfloat16 *)dst + r * (int64_t)ldd + f0) = to_bf16x4(x.x, x.y, x.z, x.w);
            } else {
                *reinterpret_cast<uint32_t *>((uint8_t *)dst + r * (int64_t)ldd + f0) =
                    to_e4m3x4(scale_pow2(x.x, k), scale_pow2(x.y, k), scale_pow2(x.z, k), scale_pow2(x.w, k));
            }
        }
        // every lane is done reading the slot before the copy engine refills it
        __syncwarp();
        if (lane == 0 && i + QSLOTS < my_rows) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(i + QSLOTS);
        }
    }
}

// Streaming variant for rows that are not 16-byte aligned (F % 4 != 0, an
// odd row stride or base): the 16-byte aligned span around each row (at
// most 12 bytes before and after it, inside the same tensor) is copied by
// cp.async.bulk into the slot, and the row is read from its offset there.
// A row whose span would reach outside [first row, end of the last row) of
// this launch -- at most the first and the last -- is read from device
// memory directly (its slot's barrier gets a plain arrival).  The
// arithmetic per element is that of quant_rows_kernel.
__host__ __device__ inline uint32_t span_slot_bytes(int F) { return (((uint32_t)F * 4u + 15u) & ~15u) + 16u; }

template <int ENC>
__global__ void __launch_bounds__(QWARPS * 32) quant_rows_span_kernel(const float *__restrict__ src, int64_t lds,
                                                                      int64_t row_off, int64_t row_step,
                                                                      int64_t nrows, int F, void *__restrict__ dst,
                                                                      int ldd, float *__restrict__ scale)
{
    extern __shared__ __align__(128) uint8_t qsm[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint32_t slot_bytes = span_slot_bytes(F);
    uint8_t *ring = qsm + (size_t)wib * QSLOTS * slot_bytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(qsm + (size_t)QWARPS * QSLOTS * slot_bytes) + wib * QSLOTS;
    const int64_t gw = (int64_t)blockIdx.x * QWARPS + wib, nw = (int64_t)gridDim.x * QWARPS;
    const int64_t my_rows = gw < nrows ? (nrows - 1 - gw) / nw + 1 : 0;
    const uintptr_t lo = reinterpret_cast<uintptr_t>(src + row_off * lds);
    const uintptr_t hi = reinterpret_cast<uintptr_t>(src + (row_off + (nrows - 1) * row_step) * lds + F);
    auto bar = [&](int s) { return (uint32_t)__cvta_generic_to_shared(bars + s); };
    auto rowptr = [&](int64_t i) { return src + (row_off + (gw + i * nw) * row_step) * lds; };
    auto span_start = [&](const float *g) { return reinterpret_cast<uintptr_t>(g) & ~(uintptr_t)15; };
    auto span_bytes = [&](const float *g) {
        return (uint32_t)(((reinterpret_cast<uintptr_t>(g) & 15u) + (uint32_t)F * 4u + 15u) & ~15u);
    };
    auto direct = [&](const float *g) { return span_start(g) < lo || span_start(g) + span_bytes(g) > hi; };
    auto issue = [&](int64_t i) {  // lane 0: this warp's i-th row into slot i % QSLOTS
        const int s = (int)(i % QSLOTS);
        const float *g = rowptr(i);
        if (direct(g)) {
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar(s)) : "memory");
            return;
        }
        const uint32_t nb = span_bytes(g);
        const uint32_t d = (uint32_t)__cvta_generic_to_shared(ring + (size_t)s * slot_bytes);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar(s)), "r"(nb) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d),
                     "l"(span_start(g)), "r"(nb), "r"(bar(s))
                     : "memory");
    };
    if (lane == 0) {
        for (int s = 0; s < QSLOTS; s++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar(s)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int64_t i = 0; i < my_rows && i < QSLOTS; i++) issue(i);
    }
    __syncwarp();
    for (int64_t i = 0; i < my_rows; i++) {
        const int s = (int)(i % QSLOTS);
        const uint32_t parity = (uint32_t)((i / QSLOTS) & 1);
        bool ok = qbar_try(bar(s), parity);
        if (!ok) {
            const unsigned long long t0 = qtimer();
            while (!(ok = qbar_try(bar(s), parity)) && qtimer() - t0 < QTIMEOUT_NS) {}
        }
        if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0) {
                atomicCAS(&g_quant_status, 0, 1);
                // let this warp's copies in flight land before the block exits
                const int64_t issued = i + QSLOTS < my_rows ? i + QSLOTS : my_rows;
                for (int64_t j = i; j < issued; j++) {
                    const unsigned long long t0 = qtimer();
                    while (!qbar_try(bar((int)(j % QSLOTS)), (uint32_t)((j / QSLOTS) & 1)) &&
                           qtimer() - t0 < 100000000ull) {}
                }
            }
            break;
        }
        const float *g = rowptr(i);
        const float *row = direct(g) ? g
                                     : reinterpret_cast<const float *>(ring + (size_t)s * slot_bytes +
                                                                       (reinterpret_cast<uintptr_t>(g) & 15u));
        const int64_t r = gw + i * nw;
        int k = 0;
        if (ENC == HDC_ENC_FP8_E4M3) {
            float amax = 0.f;
            for (int f = lane; f < F; f += 32) amax = fmaxf(amax, fabsf(row[f]));
#pragma unroll
            for (int o = 16; o; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
            k = pow2_scale_exp(amax);
            if (lane == 0) scale[r] = k >= -126 ? __int_as_float((127 + k) << 23) : ldexpf(1.f, k);
        }
        for (int f0 = lane * 4; f0 < ldd; f0 += 128) {
            const float4 x = make_float4(f0 < F ? row[f0] : 0.f, f0 + 1 < F ? row[f0 + 1] : 0.f,
                                         f0 + 2 < F ? row[f0 + 2] : 0.f, f0 + 3 < F ? row[f0 + 3] : 0.f);
            if (ENC == HDC_ENC_FP32) {
                *reinterpret_cast<float4 *>((float *)dst + r * (int64_t)ldd + f0) = x;
            } else if (ENC == HDC_ENC_BF16) {
                *reinterpret_cast<uint2 *>((__nv_bfloat16 *)dst + r * (int64_t)ldd + f0) = to_bf16x4(x.x, x.y, x.z, x.w);
            } else {
                *reinterpret_cast<uint32_t *>((uint8_t *)dst + r * (int64_t)ldd + f0) =
                    to_e4m3x4(scale_pow2(x.x, k), scale_pow2(x.y, k), scale_pow2(x.z, k), scale_pow2(x.w, k));
            }
        }
        // every lane is done reading the slot before the copy engine refills it
        __syncwarp();
        if (lane == 0 && i + QSLOTS < my_rows) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(i + QSLOTS);
        }
    }
}

// One block per class.  b == 1: plane 0 = sign bits.  b > 1: symmetric
// per-class quantisation, two's-complement planes, sums and norms over K.
__global__ void __launch_bounds__(256) class_prepare_kernel(const int32_t *__restrict__ acc, int D, int64_t s0,
                                                            int64_t stride, int64_t Dk, int b, int C,
                                                            uint32_t *__restrict__ planes, int W,
                                                            int32_t *__restrict__ csum, double *__restrict__ cnorm,
                                                            uint16_t *__restrict__ vals, int ldv)
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
    // with vals: the row of ldv BF16 values (integers |v| <= 127: exact)
    const int nwords = vals ? (ldv + 31) / 32 : W;
    for (int w = warp; w < nwords; w += nw) {
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
        if (vals) {
            if (k < ldv) vals[(int64_t)c * ldv + k] = __bfloat16_as_ushort(__float2bfloat16_rn((float)val));
            continue;
        }
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
                              int F, int enc, void *dst, int ldd, float *scale, cudaStream_t st, int64_t c0,
                              int64_t cstep)
{
    if (nrows <= 0) return cudaSuccess;
    if (c0 != 0 || cstep != 1) {  // kept features of a perforated encoding: gathering row kernel
        const int64_t blocks = (nrows + 7) / 8 < 65535 * 8 ? (nrows + 7) / 8 : 65535 * 8;
#define HDC_QUANT_G(E) quant_rows_kernel<E, false, true><<<(unsigned)blocks, 256, 0, st>>>( \
        src, lds, row_off, row_step, nrows, F, dst, ldd, scale, c0, cstep)
        if (enc == HDC_ENC_FP32) HDC_QUANT_G(HDC_ENC_FP32);
        else if (enc == HDC_ENC_BF16) HDC_QUANT_G(HDC_ENC_BF16);
        else HDC_QUANT_G(HDC_ENC_FP8_E4M3);
#undef HDC_QUANT_G
        return cudaGetLastError();
    }
    const bool aligned_rows = F % 4 == 0 && lds % 4 == 0 && ((uintptr_t)src % 16) == 0;
    const size_t qsmem = (size_t)QWARPS * QSLOTS * F * 4 + (size_t)QWARPS * QSLOTS * 8;
    if (aligned_rows && qsmem <= 200 * 1024) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
        const int per_sm = (int)((220 * 1024) / qsmem) > 0 ? (int)((220 * 1024) / qsmem) : 1;
        int64_t qblocks = (nrows + QWARPS - 1) / QWARPS;
        if (qblocks > (int64_t)sms * per_sm) qblocks = (int64_t)sms * per_sm;
#define HDC_QBULK(E)                                                                                              \
    do {                                                                                                          \
        cudaError_t e = cudaFuncSetAttribute(quant_rows_bulk_kernel<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                             (int)qsmem);                                                         \
        if (e != cudaSuccess) return e;                                                                           \
        quant_rows_bulk_kernel<E><<<(unsigned)qblocks, QWARPS * 32, qsmem, st>>>(src, lds, row_off, row_step,     \
                                                                                 nrows, F, dst, ldd, scale);      \
    } while (0)
        switch (enc) {
        case HDC_ENC_FP32: HDC_QBULK(HDC_ENC_FP32); break;
        case HDC_ENC_BF16: HDC_QBULK(HDC_ENC_BF16); break;
        default: HDC_QBULK(HDC_ENC_FP8_E4M3);
        }
#undef HDC_QBULK
        return cudaGetLastError();
    }
    // rows not 16-byte aligned: their aligned spans streamed the same way
    const size_t ssmem = (size_t)QWARPS * QSLOTS * span_slot_bytes(F) + (size_t)QWARPS * QSLOTS * 8;
    if (ssmem <= 200 * 1024 && ldd % 4 == 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
        const int per_sm = (int)((220 * 1024) / ssmem) > 0 ? (int)((220 * 1024) / ssmem) : 1;
        int64_t qblocks = (nrows + QWARPS - 1) / QWARPS;
        if (qblocks > (int64_t)sms * per_sm) qblocks = (int64_t)sms * per_sm;
#define HDC_QSPAN(E)                                                                                              \
    do {                                                                                                          \
        cudaError_t e = cudaFuncSetAttribute(quant_rows_span_kernel<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                             (int)ssmem);                                                         \
        if (e != cudaSuccess) return e;                                                                           \
        quant_rows_span_kernel<E><<<(unsigned)qblocks, QWARPS * 32, ssmem, st>>>(src, lds, row_off, row_step,     \
                                                                                 nrows, F, dst, ldd, scale);      \
    } while (0)
        switch (enc) {
        case HDC_ENC_FP32: HDC_QSPAN(HDC_ENC_FP32); break;
        case HDC_ENC_BF16: HDC_QSPAN(HDC_ENC_BF16); break;
        default: HDC_QSPAN(HDC_ENC_FP8_E4M3);
        }
#undef HDC_QSPAN
        return cudaGetLastError();
    }
    // very long rows: one warp per row straight from global memory
    int64_t blocks = (nrows + 7) / 8;
    if (blocks > 152 * 8 * 4) blocks = 152 * 8 * 4;
    dim3 g((unsigned)blocks), b(256);
    const bool vec = F % 4 == 0 && lds % 4 == 0 && ((uintptr_t)src % 16) == 0;
#define HDC_QUANT(E, V) quant_rows_kernel<E, V><<<g, b, 0, st>>>(src, lds, row_off, row_step, nrows, F, dst, ldd, scale)
    switch (enc) {
    case HDC_ENC_FP32:
        if (vec) HDC_QUANT(HDC_ENC_FP32, true); else HDC_QUANT(HDC_ENC_FP32, false);
        break;
    case HDC_ENC_BF16:
        if (vec) HDC_QUANT(HDC_ENC_BF16, true); else HDC_QUANT(HDC_ENC_BF16, false);
        break;
    default:
        if (vec) HDC_QUANT(HDC_ENC_FP8_E4M3, true); else HDC_QUANT(HDC_ENC_FP8_E4M3, false);
    }
#undef HDC_QUANT
    return cudaGetLastError();
}

cudaError_t launch_class_prepare(const int32_t *acc, int C, int D, const Perf &p, int b, uint32_t *planes, int W,
                                 int32_t *csum, double *cnorm, uint16_t *vals, int ldv, cudaStream_t st)
{
    if (C <= 0) return cudaSuccess;
    class_prepare_kernel<<<C, 256, 0, st>>>(acc, D, p.s0, p.stride, p.Dk, b, C, planes, W, csum, cnorm, vals, ldv);
    return cudaGetLastError();
}

namespace {
__global__ void class_sign_kernel(const uint32_t *__restrict__ planes, int C, int W, int Dk, int Cp, int ldcs,
                                  uint8_t *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)Cp * ldcs) return;
    const int c = (int)(i / ldcs), k = (int)(i % ldcs);
    uint8_t v = 0;
    if (c < C && k < Dk) v = ((planes[(int64_t)c * W + (k >> 5)] >> (k & 31)) & 1u) ? 0xB8 : 0x38;  // -1.0 : +1.0
    out[i] = v;
}
}  // namespace

cudaError_t launch_class_sign(const uint32_t *planes, int C, int W, int Dk, int Cp, int ldcs, uint8_t *out,
                              cudaStream_t st)
{
    const int64_t n = (int64_t)Cp * ldcs;
    if (n <= 0) return cudaSuccess;
    class_sign_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(planes, C, W, Dk, Cp, ldcs, out);
    return cudaGetLastError();
}

namespace {
// One warp per row: BF16 of each projection (zero past Dk) and the FP32
// sum of the squared BF16 values, in column order per lane, lanes combined
// by a butterfly.
__global__ void proj_bf16_kernel(const float *__restrict__ s, int64_t N, int Dk, uint16_t *__restrict__ q, int ldS,
                                 float *__restrict__ qn)
{
    const int lane = threadIdx.x & 31;
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= N) return;
    float acc = 0.f;
    for (int k = lane; k < ldS; k += 32) {
        const __nv_bfloat16 b = __float2bfloat16_rn(k < Dk ? s[row * Dk + k] : 0.f);
        const float g = __bfloat162float(b);
        acc = fmaf(g, g, acc);
        q[row * ldS + k] = __bfloat16_as_ushort(b);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) qn[row] = acc;
}
}  // namespace

cudaError_t launch_proj_bf16(const float *s, int64_t N, int Dk, uint16_t *q, int ldS, float *qn, cudaStream_t st)
{
    if (N <= 0) return cudaSuccess;
    const int64_t blocks = (N * 32 + 255) / 256;
    proj_bf16_kernel<<<(unsigned)blocks, 256, 0, st>>>(s, N, Dk, q, ldS, qn);
    return cudaGetLastError();
}

}  // namespace hdc

namespace hdc {

// Read and clear the streaming quantiser's device status word.
cudaError_t quant_read_status(cudaStream_t st, int *status)
{
    int h = 0;
    cudaError_t e = cudaMemcpyFromSymbolAsync(&h, g_quant_status, sizeof(int), 0, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    *status = h;
    if (h != 0) {
        const int zero = 0;
        e = cudaMemcpyToSymbolAsync(g_quant_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    return e;
}

}  // namespace hdc
