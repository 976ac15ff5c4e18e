// Cosine similarity of float (non-binarised) query hypervectors on the
// tensor cores (Sec. 4.2 Algorithmic Choice: cosine; the float + cosine
// form of Sec. 5.2):
//   dot[i][c]   = sum_k q[i][k] * cv[c][k]     BF16 x BF16, FP32 in TMEM
//   score[i][c] = dot / (sqrt(qn[i]) * cnorm[c])   in FP64, 0 for a zero norm
//   label[i]    = arg-max_c score (lowest index on ties)
// q: N x ldS BF16 projections (written by the encoder's projection mode),
// qn: their squared row norms; cv: Cp x ldS BF16 class values (Cp = C
// rounded up to 16, rows past C zero), cnorm: their norms over the kept dims.
//
// Structure as the encoder: one CTA per SM, persistent over 128-query tiles;
// warp 4 lane 0 streams A (128 queries x 64 dims) and B (Cp classes x 64
// dims) through a 4-stage ring of 128-byte-swizzled TMA tiles, warp 5 lane 0
// issues tcgen05.mma (M = 128, N = Cp, K = 16 per instruction) into one of
// two accumulators, warps 0-3 read their TMEM lane (one query) and take the
// arg-max.  Waits are bounded; on expiry the status word is set and the CTA
// drains its own copies and MMAs, frees TMEM and returns.
#include <cudaTypedefs.h>

#include <mutex>

#include "tc_kernel.cuh"

namespace hdc {
namespace tc {
namespace {

constexpr int CBN = 256;                          // TMEM columns per accumulator
constexpr int CSTAGES = 4;
constexpr int CA_BYTES = BM * BKB;                // 16 KB
constexpr int CB_MAX = 256 * BKB;                 // 32 KB (Cp <= 256)
constexpr int CSTAGE_BYTES = CA_BYTES + CB_MAX;
constexpr int CNUM_BARS = 2 * CSTAGES + 5;        // full, empty, tfull[2], tempty[2], done
constexpr size_t CSMEM = 1024 + (size_t)CSTAGES * CSTAGE_BYTES + CNUM_BARS * 8 + 16;

struct CosParams {
    int64_t N;
    int C, Cp, num_kb;
    const float *qn;
    const double *cnorm;
    int32_t *labels;
    double *scores;
};

__global__ void __launch_bounds__(192, 1)
    tc_cosine_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     const CosParams p)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = smem;
    uint8_t *sB = smem + CSTAGES * CA_BYTES;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + CSTAGES * CSTAGE_BYTES);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + CNUM_BARS);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    auto full = [&](int s) { return su32(bars + s); };
    auto empty = [&](int s) { return su32(bars + CSTAGES + s); };
    auto tfull = [&](int a) { return su32(bars + 2 * CSTAGES + a); };
    auto tempty = [&](int a) { return su32(bars + 2 * CSTAGES + 2 + a); };
    const uint32_t done_bar = su32(bars + 2 * CSTAGES + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t num_m_tiles = (p.N + BM - 1) / BM;
    const uint32_t b_bytes = (uint32_t)p.Cp * BKB;

    if (threadIdx.x == 0) {
        for (int s = 0; s < CSTAGES; s++) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        for (int a = 0; a < 2; a++) {
            mbar_init(tfull(a), 1);
            mbar_init(tempty(a), BM);
        }
        mbar_init(done_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(2 * CBN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 4) {
        if (lane == 0) {  // ---------------------------------- TMA producer
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
            int stage = 0;
            uint32_t phase = 0;
            bool issued[CSTAGES];
            uint32_t ipar[CSTAGES];
            for (int s = 0; s < CSTAGES; s++) { issued[s] = false; ipar[s] = 0; }
            bool ab = false;
            for (int64_t mt = blockIdx.x; mt < num_m_tiles && !ab; mt += gridDim.x)
                for (int kb = 0; kb < p.num_kb; kb++) {
                    if (!mbar_wait(empty(stage), phase ^ 1, abort_flag)) { ab = true; break; }
                    mbar_expect_tx(full(stage), CA_BYTES + b_bytes);
                    tma_load_2d(su32(sA + stage * CA_BYTES), &tmA, kb * (BKB / 2), (int)(mt * BM), full(stage));
                    tma_load_2d(su32(sB + stage * CB_MAX), &tmB, kb * (BKB / 2), 0, full(stage));
                    issued[stage] = true;
                    ipar[stage] = phase;
                    if (++stage == CSTAGES) { stage = 0; phase ^= 1; }
                }
            if (ab) {  // let our own copies land before the CTA exits
                for (int s = 0; s < CSTAGES; s++)
                    if (issued[s]) {
                        const unsigned long long t0 = gtimer();
                        while (!mbar_try(full(s), ipar[s]) && gtimer() - t0 < 100000000ull) {}
                    }
            }
        }
    } else if (warp == 5) {
        if (lane == 0) {  // ---------------------------------- MMA issuer
            // BF16 x BF16 -> FP32, K-major A and B, M = 128, N = Cp
            const uint32_t id = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(p.Cp >> 3) << 17) |
                                ((uint32_t)(BM >> 4) << 24);
            const uint64_t da0 = sdesc(su32(sA)), db0 = sdesc(su32(sB));
            const uint32_t full0 = full(0), empty0 = empty(0);   // stage s: + 8 * s
            int stage = 0, acc = 0;
            uint32_t phase = 0, aphase = 0;
            bool ab = false;
            for (int64_t mt = blockIdx.x; mt < num_m_tiles && !ab; mt += gridDim.x) {
                if (!mbar_wait_fast(tempty(acc), aphase ^ 1, abort_flag)) { ab = true; break; }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(acc * CBN);
                for (int kb = 0; kb < p.num_kb; kb++) {
                    if (!mbar_wait_fast(full0 + 8u * stage, phase, abort_flag)) { ab = true; break; }
                    tc_fence_after();
                    const uint64_t da = da0 + (uint64_t)(stage * (CA_BYTES >> 4));
                    const uint64_t db = db0 + (uint64_t)(stage * (CB_MAX >> 4));
#pragma unroll
                    for (int k = 0; k < BKB / 32; k++) mma<HDC_ENC_BF16>(d, da + 2 * k, db + 2 * k, id, (kb | k) != 0);
                    mma_commit(empty0 + 8u * stage);
                    if (++stage == CSTAGES) { stage = 0; phase ^= 1; }
                }
                if (ab) break;
                mma_commit(tfull(acc));
                if (++acc == 2) { acc = 0; aphase ^= 1; }
            }
            mma_commit(done_bar);
            const unsigned long long t0 = gtimer();
            while (!mbar_try(done_bar, 0) && gtimer() - t0 < 100000000ull) {}
        }
    } else {  // ------------------------------------------ epilogue warps 0-3
        const int q = warp;
        int acc = 0;
        uint32_t aphase = 0;
        for (int64_t mt = blockIdx.x; mt < num_m_tiles; mt += gridDim.x) {
            const int64_t row = mt * BM + q * 32 + lane;
            const bool valid = row < p.N;
            const bool ok = mbar_wait(tfull(acc), aphase, abort_flag);
            if (!__all_sync(0xffffffffu, ok)) break;
            tc_fence_after();
            const double qnorm = valid ? sqrt((double)p.qn[row]) : 0.0;
            int best = 0;
            double bs = 0.0;
            for (int j0 = 0; j0 < p.Cp; j0 += 32) {
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * CBN + j0), v);
#pragma unroll
                for (int i = 0; i < 32; i++) {
                    const int c = j0 + i;
                    if (c < p.C) {
                        const double den = qnorm * p.cnorm[c];
                        const double sc = den == 0.0 ? 0.0 : (double)__uint_as_float(v[i]) / den;
                        if (valid && p.scores) p.scores[row * p.C + c] = sc;
                        if (c == 0 || sc > bs) { bs = sc; best = c; }
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(tempty(acc));
            if (++acc == 2) { acc = 0; aphase ^= 1; }
            if (valid) p.labels[row] = best;
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * CBN) : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    });
    return fn;
}

// BF16 rows of ld elements (a multiple of 64), box = 64 elements x box_rows.
bool make_bf16_map(CUtensorMap *m, const void *base, int ld, int64_t rows, int box_rows)
{
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)(BKB / 2), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace
}  // namespace tc

cudaError_t launch_tc_cosine(const CosArgs &a, cudaStream_t st)
{
    if (a.N <= 0) return cudaSuccess;
    if (a.C <= 0 || a.C > 256 || a.Cp != (a.C + 15) / 16 * 16 || a.ldS <= 0 || a.ldS % 64 != 0 ||
        a.N > 0x7fffffffLL - tc::BM || !a.q || !a.qn || !a.cv || !a.cnorm || !a.labels)
        return cudaErrorInvalidValue;
    CUtensorMap ma, mb;
    if (!tc::make_bf16_map(&ma, a.q, a.ldS, a.N, tc::BM) || !tc::make_bf16_map(&mb, a.cv, a.ldS, a.Cp, a.Cp))
        return cudaErrorInvalidValue;
    tc::CosParams p;
    p.N = a.N;
    p.C = a.C;
    p.Cp = a.Cp;
    p.num_kb = a.ldS / 64;
    p.qn = a.qn;
    p.cnorm = a.cnorm;
    p.labels = a.labels;
    p.scores = a.scores;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess)
        return cudaErrorNoDevice;
    const int64_t m_tiles = (a.N + tc::BM - 1) / tc::BM;
    const unsigned grid = (unsigned)(m_tiles < sms ? m_tiles : sms);
    cudaError_t e = cudaFuncSetAttribute(tc::tc_cosine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tc::CSMEM);
    if (e != cudaSuccess) return e;
    tc::tc_cosine_kernel<<<grid, 192, tc::CSMEM, st>>>(ma, mb, p);
    return cudaGetLastError();
}

cudaError_t tc_cosine_read_status(cudaStream_t st, int *status) { return tc::read_status(st, status); }

}  // namespace hdc
