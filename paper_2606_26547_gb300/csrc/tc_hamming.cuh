// Fused classify with the Hamming distances on the tensor cores (binary
// classes, up to 112; the library routes 33 <= C <= 112 here).
//
// For +-1 vectors over the kept dims, Hamming(q, c) = (Dk - q.c) / 2, and
// q.c is a sum of Dk products +-1 (0 for padding): an exact integer in FP32
// for Dk < 2^24.  So after the encode GEMM of a 192-dim tile
//   S = Xq . Bq^T          (MMA1: M 128, N 192, K = F, BF16 or E4M3)
// the epilogue writes sign(S) as E4M3 +-1 bytes back into the accumulator:
// the 64 bytes of a thread's 64 read columns into the first 16 of them (four
// per column, lowest dim in the lowest byte), and a second GEMM with its A
// operand in tensor memory accumulates
//   D2 += sign(S) . Csign^T  (MMA2: M 128, N = Cp, K = 192, E4M3)
// over all tiles of the query block, Csign being the class hypervectors as
// E4M3 +-1 bytes (zero past Dk and for the pad classes up to Cp = C rounded
// to 16).  The final epilogue reads D2 and takes the arg-min of
// (Dk - dot) / 2 (lowest class on ties).
//
// Tensor memory (512 columns): two 192-column encode accumulators (the
// encode stays double buffered; each also holds its tile's sign bytes until
// MMA2 has read them, MMA2's commit releasing it to MMA1) and the Cp <= 128
// columns of D2.
//
// Roles (16 warps): warps 0-11 epilogue (three warpgroups, 64 columns of a
// tile each), warp 12 TMA producer of the A / B stages (4 x 40 KB), warp 13
// MMA1 issuer, warp 14 TMA producer of the class-sign tiles, warp 15 MMA2
// issuer.  The two issuers keep separate commit chains, so the MMA2 of tile t
// enters the tensor pipe as soon as its sign tile is ready, without holding
// back the issue of the next tile's MMA1 (a single issuer measured ~2,400
// cycles of issue and commit latency at each tile boundary).  With QIN,
// warps 16-19 quantise the query tiles from FP32 rows one tile ahead into the
// CTA's two staged tiles, as in the encoder (tc_kernel.cuh).  Every wait
// is bounded as in the encoder.
#pragma once
#include "tc_kernel.cuh"

namespace hdc {
namespace tc {

constexpr int HBN = 192;                      // dims per tile
constexpr int H_STAGES = 4;
constexpr int HA_BYTES = BM * BKB;            // 16 KB
constexpr int HB_BYTES = HBN * BKB;           // 24 KB
constexpr int H_STAGE_BYTES = HA_BYTES + HB_BYTES;
constexpr int HEWG = 3;                       // epilogue warpgroups
constexpr int H_THREADS = (4 * HEWG + 4) * 32;   // + the MMA2 issuer
constexpr int H_QW = 4;                          // quantiser warps (QIN): 20 warps at up to 96 registers
__host__ __device__ constexpr int h_threads(bool qin) { return H_THREADS + (qin ? H_QW * 32 : 0); }
constexpr int H_CMAX = 112;
// full[S], empty[S], sfull[2], sempty[2], a2full[2], b2full, b2empty,
// d2full, d2empty, done, merge_full, merge_empty, done2, a0_ready, a_ready[2], a_free[2].
// a2full is per accumulator: epilogue warps that run ahead to the next tile
// arrive on the other barrier, and tile t + 2's arrivals wait (through
// sempty and MMA1) for MMA2 of tile t.
constexpr int H_NUM_BARS = 2 * H_STAGES + 4 + 6 + 3 + 1 + 5;

__host__ __device__ constexpr size_t h_smem_bytes(int Cp)
{
    return 1024 + (size_t)H_STAGES * H_STAGE_BYTES + (size_t)2 * Cp * 128 + H_NUM_BARS * 8 + 16 +
           (size_t)2 * BM * 4 * (HEWG - 1);
}
static_assert(h_smem_bytes(H_CMAX) <= 232448, "shared memory of the tensor-core Hamming kernel");

// Sixteen 32-bit TMEM columns of this thread's lane (the warp's own 32-lane
// quarter), and the wait for this thread's stores to land.
__device__ __forceinline__ void h_tmem_st16(uint32_t taddr, const uint32_t (&r)[16])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
                 ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]),
                 "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
                 "r"(r[15])
                 : "memory");
}
__device__ __forceinline__ void h_tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// D += A . B^T, E4M3, A (128 rows x 32 bytes) in tensor memory at column a.
__device__ __forceinline__ void h_mma_ts_fp8(uint32_t d, uint32_t a, uint64_t b, uint32_t id, uint32_t accum)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
        "r"(a), "l"(b), "r"(id), "r"(accum));
}

struct HParams {
    int64_t N;
    int Dk, num_kb, nt;     // nt: 192-dim tiles
    int C, Cp;
    int32_t *labels, *dists;
    // QIN: FP32 query rows and the staged tiles (2 per CTA), as in Params
    const float *X = nullptr;
    int64_t ldX = 0;
    int F = 0, ld = 0;
    uint8_t *stage = nullptr;
};

template <int ENC>
__device__ __forceinline__ uint32_t idesc_n(int n)
{
    const uint32_t fmt = ENC == HDC_ENC_BF16 ? 1u : 0u;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

template <int ENC, bool QIN = false>
__global__ void __launch_bounds__(h_threads(QIN), 1)
    tc_hamming_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                      const __grid_constant__ CUtensorMap tmS, const HParams p)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = smem;
    uint8_t *sB = smem + H_STAGES * HA_BYTES;
    uint8_t *sB2 = smem + H_STAGES * H_STAGE_BYTES;                 // 2 atoms x Cp rows x 128 B
    uint64_t *bars = reinterpret_cast<uint64_t *>(sB2 + 2 * p.Cp * 128);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + H_NUM_BARS);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    int32_t *s_val = reinterpret_cast<int32_t *>(tmem_slot + 4);    // warpgroups 1.. : per-row minimum
    int32_t *s_idx = s_val + (HEWG - 1) * BM;                        // and its class
    auto full = [&](int s) { return su32(bars + s); };
    auto empty = [&](int s) { return su32(bars + H_STAGES + s); };
    auto sfull = [&](int a) { return su32(bars + 2 * H_STAGES + a); };
    auto sempty = [&](int a) { return su32(bars + 2 * H_STAGES + 2 + a); };
    auto a2full = [&](int a) { return su32(bars + 2 * H_STAGES + 4 + a); };
    const uint32_t b2full = su32(bars + 2 * H_STAGES + 6), b2empty = su32(bars + 2 * H_STAGES + 7);
    const uint32_t d2full = su32(bars + 2 * H_STAGES + 8), d2empty = su32(bars + 2 * H_STAGES + 9);
    const uint32_t done_bar = su32(bars + 2 * H_STAGES + 10);
    const uint32_t merge_full = su32(bars + 2 * H_STAGES + 11), merge_empty = su32(bars + 2 * H_STAGES + 12);
    const uint32_t done2_bar = su32(bars + 2 * H_STAGES + 13);
    const uint32_t a0_ready = su32(bars + 2 * H_STAGES + 14);
    auto a_ready = [&](int b) { return su32(bars + 2 * H_STAGES + 15 + b); };
    auto a_free = [&](int b) { return su32(bars + 2 * H_STAGES + 17 + b); };
    constexpr int QW0 = 4 * HEWG + 4;                  // first quantiser warp
    constexpr int QES = ENC == HDC_ENC_BF16 ? 2 : 1;
    const QinRows qr = {p.X, p.ldX, p.N, p.F, p.ld};
    constexpr int PRODUCER = 4 * HEWG, ISSUER = 4 * HEWG + 1, CPRODUCER = 4 * HEWG + 2, ISSUER2 = 4 * HEWG + 3;
    constexpr int KELEMS = ENC == HDC_ENC_BF16 ? BKB / 2 : BKB;
    constexpr uint32_t D2_COL = 2 * HBN;     // D2 after the two encode accumulators

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t num_m_tiles = (p.N + BM - 1) / BM;

    if (threadIdx.x == 0) {
        for (int s = 0; s < H_STAGES; s++) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        for (int a = 0; a < 2; a++) {
            mbar_init(sfull(a), 1);
            mbar_init(sempty(a), 1);   // the commit of the tile's MMA2
            mbar_init(a2full(a), BM * HEWG);
        }
        mbar_init(b2full, 1);
        mbar_init(b2empty, 1);
        mbar_init(d2full, 1);
        mbar_init(d2empty, BM * HEWG);
        mbar_init(done_bar, 1);
        mbar_init(done2_bar, 1);
        mbar_init(merge_full, BM * (HEWG - 1));
        mbar_init(merge_empty, BM);
        mbar_init(a0_ready, (4 * HEWG + H_QW) * 32);
        for (int b = 0; b < 2; b++) {
            mbar_init(a_ready(b), H_QW * 32);
            mbar_init(a_free(b), 1);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == PRODUCER) {
        if (lane == 0) {  // ------------------------------ A / B stage producer
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
            int stage = 0;
            uint32_t phase = 0;
            bool issued[H_STAGES];
            uint32_t ipar[H_STAGES];
            for (int s = 0; s < H_STAGES; s++) { issued[s] = false; ipar[s] = 0; }
            bool ab = false;
            int64_t it = 0;
            for (int64_t mt = blockIdx.x; mt < num_m_tiles && !ab; mt += gridDim.x, it++)
                for (int t = 0; t < p.nt && !ab; t++)
                    for (int kb = 0; kb < p.num_kb; kb++) {
                        if (QIN && t == 0 && kb == 0) {  // the tile's staged query rows have been written
                            const bool okq = it == 0 ? mbar_wait(a0_ready, 0, abort_flag)
                                                     : mbar_wait(a_ready((int)(it & 1)),
                                                                 (uint32_t)(((it - 1) >> 1) & 1), abort_flag);
                            if (!okq) { ab = true; break; }
                        }
                        if (!mbar_wait(empty(stage), phase ^ 1, abort_flag)) { ab = true; break; }
                        mbar_expect_tx(full(stage), H_STAGE_BYTES);
                        const int ay = QIN ? (int)((blockIdx.x * 2 + (it & 1)) * BM) : (int)(mt * BM);
                        tma_load_2d(su32(sA + stage * HA_BYTES), &tmA, kb * KELEMS, ay, full(stage));
                        tma_load_2d(su32(sB + stage * HB_BYTES), &tmB, kb * KELEMS, t * HBN, full(stage));
                        issued[stage] = true;
                        ipar[stage] = phase;
                        if (++stage == H_STAGES) { stage = 0; phase ^= 1; }
                    }
            if (ab) {
                for (int s = 0; s < H_STAGES; s++)
                    if (issued[s]) {
                        const unsigned long long t0 = gtimer();
                        while (!mbar_try(full(s), ipar[s]) && gtimer() - t0 < 100000000ull) {}
                    }
            }
        }
    } else if (warp == CPRODUCER) {
        if (lane == 0) {  // ------------------------------ class-sign producer
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmS)) : "memory");
            uint32_t ph = 0, last = 0;
            bool any = false, ab = false;
            const uint32_t bytes = 2u * (uint32_t)p.Cp * 128u;
            for (int64_t mt = blockIdx.x; mt < num_m_tiles && !ab; mt += gridDim.x)
                for (int t = 0; t < p.nt; t++) {
                    if (!mbar_wait(b2empty, ph ^ 1, abort_flag)) { ab = true; break; }
                    mbar_expect_tx(b2full, bytes);
                    tma_load_2d(su32(sB2), &tmS, t * HBN, 0, b2full);
                    tma_load_2d(su32(sB2 + p.Cp * 128), &tmS, t * HBN + 128, 0, b2full);
                    any = true;
                    last = ph;
                    ph ^= 1;
                }
            if (ab && any) {
                const unsigned long long t0 = gtimer();
                while (!mbar_try(b2full, last) && gtimer() - t0 < 100000000ull) {}
            }
        }
    } else if (warp == ISSUER) {
        if (lane == 0) {  // ------------------------------ MMA1 issuer (encode)
            const uint32_t id1 = idesc_n<ENC>(HBN);
            const uint64_t da0 = sdesc(su32(sA)), db0 = sdesc(su32(sB));
            const uint32_t full0 = full(0), empty0 = empty(0);   // stage s: + 8 * s
            int stage = 0, acc = 0;
            uint32_t phase = 0, aphase = 0;
            bool ab = false;
            int64_t it = 0;
            for (int64_t mt = blockIdx.x; mt < num_m_tiles && !ab; mt += gridDim.x, it++) {
                for (int t = 0; t < p.nt && !ab; t++) {
                    if (!mbar_wait_fast(sempty(acc), aphase ^ 1, abort_flag)) { ab = true; break; }
                    tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)(acc * HBN);
                    for (int kb = 0; kb < p.num_kb; kb++) {
                        if (!mbar_wait_fast(full0 + 8u * stage, phase, abort_flag)) { ab = true; break; }
                        tc_fence_after();
                        // the last copy of the staged query tile has landed
                        if (QIN && t == p.nt - 1 && kb == p.num_kb - 1) mbar_arrive(a_free((int)(it & 1)));
                        const uint64_t da = da0 + (uint64_t)(stage * (HA_BYTES >> 4));
                        const uint64_t db = db0 + (uint64_t)(stage * (HB_BYTES >> 4));
#pragma unroll
                        for (int k = 0; k < BKB / 32; k++) mma<ENC>(d, da + 2 * k, db + 2 * k, id1, (kb | k) != 0);
                        mma_commit(empty0 + 8u * stage);
                        if (++stage == H_STAGES) { stage = 0; phase ^= 1; }
                    }
                    if (ab) break;
                    mma_commit(sfull(acc));
                    if (++acc == 2) { acc = 0; aphase ^= 1; }
                }
            }
            mma_commit(done_bar);
            const unsigned long long t0 = gtimer();
            while (!mbar_try(done_bar, 0) && gtimer() - t0 < 100000000ull) {}
        }
    } else if (warp == ISSUER2) {
        if (lane == 0) {  // ------------------------------ MMA2 issuer: D2 (+)= signs . class signs, K = 192
            const uint32_t id2 = idesc_n<HDC_ENC_FP8_E4M3>(p.Cp);
            uint32_t a2ph = 0, b2ph = 0, d2ph = 0;   // a2ph: both accumulators' parity, flipped per pair
            int acc = 0;
            bool ab = false;
            for (int64_t mt = blockIdx.x; mt < num_m_tiles && !ab; mt += gridDim.x) {
                for (int t = 0; t < p.nt; t++) {
                    const bool first = t == 0;
                    if (first && !mbar_wait(d2empty, d2ph ^ 1, abort_flag)) { ab = true; break; }
                    if (!mbar_wait(a2full(acc), a2ph, abort_flag)) { ab = true; break; }
                    if (!mbar_wait(b2full, b2ph, abort_flag)) { ab = true; break; }
                    tc_fence_after();
                    const uint32_t b0 = su32(sB2), tacc = tmem + (uint32_t)(acc * HBN);
#pragma unroll
                    for (int k = 0; k < 6; k++) {   // class atom 0: K bytes 0..127, atom 1: 128..191
                        // dims 32k..32k+31: warpgroup k / 2's first 16 columns, eight in for odd k
                        const uint32_t col = (uint32_t)((k >> 1) * 64 + (k & 1) * 8);
                        const uint32_t off_b = (k < 4 ? 0u : (uint32_t)(p.Cp * 128)) + 32u * (k & 3);
                        h_mma_ts_fp8(tmem + D2_COL, tacc + col, sdesc(b0 + off_b), id2, (first && k == 0) ? 0u : 1u);
                    }
                    mma_commit(sempty(acc));   // the accumulator (and its sign bytes) is free for MMA1
                    mma_commit(b2empty);
                    if (++acc == 2) { acc = 0; a2ph ^= 1; }
                    b2ph ^= 1;
                }
                if (ab) break;
                mma_commit(d2full);
                d2ph ^= 1;
            }
            mma_commit(done2_bar);
            const unsigned long long t0 = gtimer();
            while (!mbar_try(done2_bar, 0) && gtimer() - t0 < 100000000ull) {}
        }
    } else if (QIN && warp >= QW0) {  // ----------------------------- query quantisers
        const int qw = warp - QW0;
        uint32_t fph = 0;
        int64_t it = 0;
        for (int64_t mt = blockIdx.x; mt < num_m_tiles && !*abort_flag; mt += gridDim.x, it++) {
            const int b = (int)(it & 1);
            uint8_t *tile = p.stage + (size_t)(blockIdx.x * 2 + b) * BM * p.ld * QES;
            if (it >= 2) {
                const bool okf = mbar_wait(a_free(b), (fph >> b) & 1u, abort_flag);
                fph ^= 1u << b;
                if (!__all_sync(0xffffffffu, okf)) break;
            }
            if (it == 0)
                quant_tile<ENC, 2>(qr, mt * BM, tile, 4 * HEWG + qw, 4 * HEWG + H_QW, lane);
            else
                quant_tile<ENC, 2>(qr, mt * BM, tile, qw, H_QW, lane);
            fence_to_async_global();
            mbar_arrive(it == 0 ? a0_ready : a_ready(b));
        }
    } else {  // ------------------------------------------ epilogue warps 0 .. 11
        if (QIN) {  // the first staged tile, with the quantiser warps
            quant_tile<ENC, 2>(qr, (int64_t)blockIdx.x * BM, p.stage + (size_t)blockIdx.x * 2 * BM * p.ld * QES, warp,
                               4 * HEWG + H_QW, lane);
            fence_to_async_global();
            mbar_arrive(a0_ready);
        }
        const int q = warp & 3, g = warp >> 2;
        const int r = q * 32 + lane;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        int acc = 0;
        uint32_t aphase = 0, d2ph = 0;
        bool ab = false;
        int64_t it = 0;
        for (int64_t mt = blockIdx.x; mt < num_m_tiles && !ab; mt += gridDim.x, it++) {
            const int64_t row = mt * BM + r;
            const bool valid = row < p.N;
            for (int t = 0; t < p.nt; t++) {
                const bool ok = mbar_wait(sfull(acc), aphase, abort_flag);
                if (!__all_sync(0xffffffffu, ok)) { ab = true; break; }
                tc_fence_after();
                const uint32_t tcol = tmem + lane_base + (uint32_t)(acc * HBN + g * 64);
                uint32_t v0[32], v1[32];
                tmem_ld32(tcol, v0);
                tmem_ld32(tcol + 32, v1);
                // E4M3 +1.0 = 0x38, -1.0 = 0xB8 (sign(0) = +1); byte i of word j is dim 4j + i
                // of this warpgroup's 64
                uint32_t w[16];
#pragma unroll
                for (int i = 0; i < 8; i++) {
                    uint32_t x = 0;
#pragma unroll
                    for (int b = 0; b < 4; b++)
                        x |= (__uint_as_float(v0[4 * i + b]) < 0.f ? 0xB8u : 0x38u) << (8 * b);
                    w[i] = x;
                    uint32_t y = 0;
#pragma unroll
                    for (int b = 0; b < 4; b++)
                        y |= (__uint_as_float(v1[4 * i + b]) < 0.f ? 0xB8u : 0x38u) << (8 * b);
                    w[8 + i] = y;
                }
                h_tmem_st16(tcol, w);   // into the first 16 of the 64 columns read above
                h_tmem_st_wait();
                tc_fence_before();
                mbar_arrive(a2full(acc));
                if (++acc == 2) { acc = 0; aphase ^= 1; }
            }
            if (ab) break;
            // distances of this warpgroup's 32-class chunks (chunk j to warpgroup j % 3)
            const bool okd = mbar_wait(d2full, d2ph, abort_flag);
            if (!__all_sync(0xffffffffu, okd)) { ab = true; break; }
            tc_fence_after();
            int best = 0x7fffffff, bv = 0x7fffffff;
            for (int j = g; j * 32 < p.Cp; j += HEWG) {
                uint32_t v[32];
                tmem_ld32(tmem + lane_base + D2_COL + (uint32_t)(j * 32), v);
#pragma unroll
                for (int i = 0; i < 32; i++) {
                    const int c = j * 32 + i;
                    if (c < p.C) {
                        const int dist = (p.Dk - (int)__uint_as_float(v[i])) / 2;
                        if (p.dists && valid) p.dists[row * p.C + c] = dist;
                        if (dist < bv) { bv = dist; best = c; }   // ascending c: lowest on ties
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(d2empty);
            d2ph ^= 1;
            const uint32_t par = (uint32_t)(it & 1);
            if (g > 0) {
                if (!mbar_wait(merge_empty, par ^ 1, abort_flag)) { ab = true; break; }
                s_val[(g - 1) * BM + r] = bv;
                s_idx[(g - 1) * BM + r] = best;
                mbar_arrive(merge_full);
            } else {
                if (!mbar_wait(merge_full, par, abort_flag)) { ab = true; break; }
#pragma unroll
                for (int h = 0; h < HEWG - 1; h++) {   // (distance, class) order: lowest class on ties
                    const int v1 = s_val[h * BM + r], i1 = s_idx[h * BM + r];
                    if (v1 < bv || (v1 == bv && i1 < best)) { bv = v1; best = i1; }
                }
                mbar_arrive(merge_empty);
                if (valid) p.labels[row] = best;
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

template <int ENC, bool QIN>
static cudaError_t launch_hamming_q(const CUtensorMap &ma, const CUtensorMap &mb, const CUtensorMap &ms,
                                    const HParams &p, unsigned grid, cudaStream_t st)
{
    auto k = tc_hamming_kernel<ENC, QIN>;
    const size_t smem = h_smem_bytes(p.Cp);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, h_threads(QIN), smem, st>>>(ma, mb, ms, p);
    return cudaGetLastError();
}

template <int ENC>
static cudaError_t launch_hamming_enc(const CUtensorMap &ma, const CUtensorMap &mb, const CUtensorMap &ms,
                                      const HParams &p, unsigned grid, cudaStream_t st)
{
    return p.X ? launch_hamming_q<ENC, true>(ma, mb, ms, p, grid, st)
               : launch_hamming_q<ENC, false>(ma, mb, ms, p, grid, st);
}

cudaError_t launch_hamming_bf16(const CUtensorMap &ma, const CUtensorMap &mb, const CUtensorMap &ms,
                                const HParams &p, unsigned grid, cudaStream_t st);
cudaError_t launch_hamming_fp8(const CUtensorMap &ma, const CUtensorMap &mb, const CUtensorMap &ms,
                               const HParams &p, unsigned grid, cudaStream_t st);

}  // namespace tc
}  // namespace hdc
