// Fused classify of float (non-binarised) query hypervectors: encode and
// cosine in one kernel (Sec. 4.2 Algorithmic Choice; the float + cosine form
// of Sec. 5.2), C <= 128 classes.
//
// For each 192-dim tile t of a 128-query block:
//   S = Xq . Bq^T                (MMA1: M 128, N 192, K = F, BF16 or E4M3)
//   q = bf16(S * sb_k)           (the epilogue: 64 columns per warpgroup;
//                                 sum of q^2 kept per row).  Each thread
//                                 writes the 32 BF16 of every 32-column
//                                 half it has read back into the first 16
//                                 of those columns (two per column, lower
//                                 dim in the low half)
//   D2 += q . Cv^T               (MMA2: M 128, N = Cp, K = 192, BF16, A from
//                                 tensor memory; its commit releases the
//                                 accumulator to MMA1)
// with Cv the model's BF16 class values (Cp x ldS; TMA zero fill past ldS).
// After the last tile: score_c = D2_c / (||q|| ||c||) in FP64 (0 for a zero
// norm), arg-max with the lowest class on ties.  The projections never
// reach device memory.
//
// Tensor memory: two 192-column encode accumulators (each also holding its
// tile's BF16 values) and D2 (Cp <= 128).  Shared memory: three or four A/B
// stages (40 KB each) and one or two Cp x 384-byte class tiles: with two, the
// next tile's class values load while the current tile's cosine MMAs run.
// Roles as the tensor-core Hamming kernel:
// warps 0-11 epilogue (three warpgroups), 12 stage producer, 13 MMA1 issuer,
// 14 class-tile producer, 15 MMA2 issuer (its own commit chain: 4.65 vs
// 5.47 ms per 2^20 queries at C = 10 with one issuer); every wait bounded.
#pragma once
#include "tc_hamming.cuh"

namespace hdc {
namespace tc {

// A/B stages: four when the class tile leaves room (C <= 16), else three.
// At N = 192 a stage feeds about 0.2 us of MMA work, so the stages in
// flight are what covers the L2 latency (36 % tensor activity measured with
// three stages at C = 10).
constexpr int FC_THREADS = (4 * HEWG + 4) * 32;     // + the cosine MMA issuer
constexpr int FC_CMAX = 128;   // TMEM: 2 x 192 + 128 columns
// full[S], empty[S], sfull[2], sempty[2], a2full[2], b2full[0], b2empty[0],
// d2full, d2empty, done, merge_full, merge_empty, qfull[2], done2, b2full[1], b2empty[1].
// a2full is per accumulator: epilogue warps that run ahead to the next tile
// arrive on the other barrier, and tile t + 2's arrivals wait (through
// sempty and MMA1) for MMA2 of tile t.
__host__ __device__ constexpr int fc_num_bars(int stages) { return 2 * stages + 4 + 6 + 3 + 2 + 1 + 2; }

__host__ __device__ constexpr size_t fc_smem_bytes(int stages, int Cp, int b2bufs)
{
    return 1024 + (size_t)stages * H_STAGE_BYTES + (size_t)b2bufs * 3 * Cp * 128 +
           fc_num_bars(stages) * 8 + 16 + (size_t)2 * BM * 8 * (HEWG - 1) + (size_t)2 * HEWG * BM * 4;
}
static_assert(fc_smem_bytes(3, FC_CMAX, 1) <= 232448, "shared memory of the fused float-query kernel");
static_assert(fc_smem_bytes(3, 32, 2) <= 232448, "shared memory of the double-buffered class tile");

struct FCParams {
    int64_t N;
    int Dk, num_kb, nt;
    int C, Cp;
    const float *sb;         // base-row scales (FP8) or NULL
    const double *cnorm;     // C norms of the class values over the kept dims
    int32_t *labels;
    double *scores;          // optional N x C
};

// Sixteen 32-bit TMEM columns of this thread's lane (the warp's own 32-lane
// quarter), and the wait for this thread's stores to land.
__device__ __forceinline__ void fc_tmem_st16(uint32_t taddr, const uint32_t (&r)[16])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
                 ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]),
                 "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
                 "r"(r[15])
                 : "memory");
}
__device__ __forceinline__ void fc_tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// D += A . B^T, BF16, A (128 rows x 16 BF16) in tensor memory at column a.
__device__ __forceinline__ void fc_mma_ts(uint32_t d, uint32_t a, uint64_t b, uint32_t id, uint32_t accum)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
        "r"(a), "l"(b), "r"(id), "r"(accum));
}

template <int ENC, int FC_STAGES, int B2BUF>
__global__ void __launch_bounds__(FC_THREADS, 1)
    tc_fcos_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmV, const FCParams p)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = smem;
    uint8_t *sB = smem + FC_STAGES * HA_BYTES;
    uint8_t *sB2 = smem + FC_STAGES * H_STAGE_BYTES;                // B2BUF x 3 atoms x Cp rows x 128 B
    const int b2_bytes = 3 * p.Cp * 128;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sB2 + B2BUF * b2_bytes);
    constexpr int FC_NUM_BARS = fc_num_bars(FC_STAGES);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + FC_NUM_BARS);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    double *s_val = reinterpret_cast<double *>(tmem_slot + 4);       // warpgroups 1.. : per-row best score
    int32_t *s_idx = reinterpret_cast<int32_t *>(s_val + (HEWG - 1) * BM);   // and its class
    float *s_q = reinterpret_cast<float *>(s_idx + (HEWG - 1) * BM);  // 2 x [HEWG][BM] partial squared norms
    auto full = [&](int s) { return su32(bars + s); };
    auto empty = [&](int s) { return su32(bars + FC_STAGES + s); };
    auto sfull = [&](int a) { return su32(bars + 2 * FC_STAGES + a); };
    auto sempty = [&](int a) { return su32(bars + 2 * FC_STAGES + 2 + a); };
    auto a2full = [&](int a) { return su32(bars + 2 * FC_STAGES + 4 + a); };
    auto b2full = [&](int b) { return su32(bars + 2 * FC_STAGES + (b ? 16 : 6)); };
    auto b2empty = [&](int b) { return su32(bars + 2 * FC_STAGES + (b ? 17 : 7)); };
    const uint32_t d2full = su32(bars + 2 * FC_STAGES + 8), d2empty = su32(bars + 2 * FC_STAGES + 9);
    const uint32_t done_bar = su32(bars + 2 * FC_STAGES + 10);
    const uint32_t merge_full = su32(bars + 2 * FC_STAGES + 11), merge_empty = su32(bars + 2 * FC_STAGES + 12);
    auto qfull = [&](int b) { return su32(bars + 2 * FC_STAGES + 13 + b); };
    const uint32_t done2_bar = su32(bars + 2 * FC_STAGES + 15);
    constexpr int PRODUCER = 4 * HEWG, ISSUER = 4 * HEWG + 1, CPRODUCER = 4 * HEWG + 2, ISSUER2 = 4 * HEWG + 3;
    constexpr int KELEMS = ENC == HDC_ENC_BF16 ? BKB / 2 : BKB;
    constexpr uint32_t D2_COL = 2 * HBN;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t num_m_tiles = (p.N + BM - 1) / BM;

    if (threadIdx.x == 0) {
        for (int s = 0; s < FC_STAGES; s++) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        for (int a = 0; a < 2; a++) {
            mbar_init(sfull(a), 1);
            mbar_init(sempty(a), 1);   // the commit of the tile's MMA2
            mbar_init(qfull(a), BM * HEWG);
            mbar_init(a2full(a), BM * HEWG);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(b2full(b), 1);
            mbar_init(b2empty(b), 1);
        }
        mbar_init(d2full, 1);
        mbar_init(d2empty, BM * HEWG);
        mbar_init(done_bar, 1);
        mbar_init(done2_bar, 1);
        mbar_init(merge_full, BM * (HEWG - 1));
        mbar_init(merge_empty, BM);
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
            bool issued[FC_STAGES];
            uint32_t ipar[FC_STAGES];
            for (int s = 0; s < FC_STAGES; s++) { issued[s] = false; ipar[s] = 0; }
            bool ab = false;
            for (int64_t mt = blockIdx.x; mt < num_m_tiles && !ab; mt += gridDim.x)
                for (int t = 0; t < p.nt && !ab; t++)
                    for (int kb = 0; kb < p.num_kb; kb++) {
                        if (!mbar_wait(empty(stage), phase ^ 1, abort_flag)) { ab = true; break; }
                        mbar_expect_tx(full(stage), H_STAGE_BYTES);
                        tma_load_2d(su32(sA + stage * HA_BYTES), &tmA, kb * KELEMS, (int)(mt * BM), full(stage));
                        tma_load_2d(su32(sB + stage * HB_BYTES), &tmB, kb * KELEMS, t * HBN, full(stage));
                        issued[stage] = true;
                        ipar[stage] = phase;
                        if (++stage == FC_STAGES) { stage = 0; phase ^= 1; }
                    }
            if (ab) {
                for (int s = 0; s < FC_STAGES; s++)
                    if (issued[s]) {
                        const unsigned long long t0 = gtimer();
                        while (!mbar_try(full(s), ipar[s]) && gtimer() - t0 < 100000000ull) {}
                    }
            }
        }
    } else if (warp == CPRODUCER) {
        if (lane == 0) {  // ------------------------------ class-value tile producer
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmV)) : "memory");
            uint32_t ph[2] = {0, 0}, last[2] = {0, 0};
            bool any[2] = {false, false}, ab = false;
            int bi = 0;
            const uint32_t bytes = 3u * (uint32_t)p.Cp * 128u;
            for (int64_t mt = blockIdx.x; mt < num_m_tiles && !ab; mt += gridDim.x)
                for (int t = 0; t < p.nt; t++) {
                    if (!mbar_wait(b2empty(bi), ph[bi] ^ 1, abort_flag)) { ab = true; break; }
                    mbar_expect_tx(b2full(bi), bytes);
#pragma unroll
                    for (int a = 0; a < 3; a++)   // 64 BF16 of K per atom
                        tma_load_2d(su32(sB2 + bi * b2_bytes + a * p.Cp * 128), &tmV, t * HBN + a * 64, 0,
                                    b2full(bi));
                    any[bi] = true;
                    last[bi] = ph[bi];
                    ph[bi] ^= 1;
                    if (++bi == B2BUF) bi = 0;
                }
            if (ab)
                for (int b = 0; b < B2BUF; b++)
                    if (any[b]) {
                        const unsigned long long t0 = gtimer();
                        while (!mbar_try(b2full(b), last[b]) && gtimer() - t0 < 100000000ull) {}
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
            for (int64_t mt = blockIdx.x; mt < num_m_tiles && !ab; mt += gridDim.x) {
                for (int t = 0; t < p.nt && !ab; t++) {
                    if (!mbar_wait_fast(sempty(acc), aphase ^ 1, abort_flag)) { ab = true; break; }
                    tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)(acc * HBN);
                    for (int kb = 0; kb < p.num_kb; kb++) {
                        if (!mbar_wait_fast(full0 + 8u * stage, phase, abort_flag)) { ab = true; break; }
                        tc_fence_after();
                        const uint64_t da = da0 + (uint64_t)(stage * (HA_BYTES >> 4));
                        const uint64_t db = db0 + (uint64_t)(stage * (HB_BYTES >> 4));
#pragma unroll
                        for (int k = 0; k < BKB / 32; k++) mma<ENC>(d, da + 2 * k, db + 2 * k, id1, (kb | k) != 0);
                        mma_commit(empty0 + 8u * stage);
                        if (++stage == FC_STAGES) { stage = 0; phase ^= 1; }
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
        if (lane == 0) {  // ------------------------------ MMA2 issuer (cosine), its own commit chain
            const uint32_t id2 = idesc_n<HDC_ENC_BF16>(p.Cp);
            uint32_t a2ph = 0, b2ph[2] = {0, 0}, d2ph = 0;   // a2ph: both accumulators' parity, flipped per pair
            int bi = 0, acc = 0;
            bool ab = false;
            for (int64_t mt = blockIdx.x; mt < num_m_tiles && !ab; mt += gridDim.x) {
                for (int t = 0; t < p.nt; t++) {
                    const bool first = t == 0;
                    if (first && !mbar_wait(d2empty, d2ph ^ 1, abort_flag)) { ab = true; break; }
                    if (!mbar_wait(a2full(acc), a2ph, abort_flag)) { ab = true; break; }
                    if (!mbar_wait(b2full(bi), b2ph[bi], abort_flag)) { ab = true; break; }
                    tc_fence_after();
                    const uint32_t b0 = su32(sB2 + bi * b2_bytes), tacc = tmem + (uint32_t)(acc * HBN);
#pragma unroll
                    for (int k = 0; k < 12; k++) {   // three atoms of four 16-element K steps
                        // dims 16k..16k+15: warpgroup k / 4's columns, half (k % 4) / 2, eight columns in
                        const uint32_t col = (uint32_t)((k >> 2) * 64 + ((k & 3) >> 1) * 32 + (k & 1) * 8);
                        const uint32_t off_b = (uint32_t)((k >> 2) * p.Cp * 128) + 32u * (k & 3);
                        fc_mma_ts(tmem + D2_COL, tacc + col, sdesc(b0 + off_b), id2, (first && k == 0) ? 0u : 1u);
                    }
                    mma_commit(sempty(acc));   // the accumulator (and its BF16 values) is free for MMA1
                    mma_commit(b2empty(bi));
                    if (++acc == 2) { acc = 0; a2ph ^= 1; }
                    b2ph[bi] ^= 1;
                    if (++bi == B2BUF) bi = 0;
                }
                if (ab) break;
                mma_commit(d2full);
                d2ph ^= 1;
            }
            mma_commit(done2_bar);
            const unsigned long long t0 = gtimer();
            while (!mbar_try(done2_bar, 0) && gtimer() - t0 < 100000000ull) {}
        }
    } else {  // ------------------------------------------ epilogue warps 0 .. 11
        const int q = warp & 3, g = warp >> 2;
        const int r = q * 32 + lane;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        int acc = 0, qb = 0;
        uint32_t aphase = 0, d2ph = 0, qph = 0;
        bool ab = false;
        int64_t it = 0;
        for (int64_t mt = blockIdx.x; mt < num_m_tiles && !ab; mt += gridDim.x, it++) {
            const int64_t row = mt * BM + r;
            const bool valid = row < p.N;
            float qsum = 0.f;
            for (int t = 0; t < p.nt; t++) {
                const bool ok = mbar_wait(sfull(acc), aphase, abort_flag);
                if (!__all_sync(0xffffffffu, ok)) { ab = true; break; }
                tc_fence_after();
                // two halves of the warpgroup's 64 columns: BF16 of s * sb (zero
                // past Dk) into the half's first 16 columns; squared norm of the BF16 values
                const int col0 = t * HBN + g * 64;
#pragma unroll 1
                for (int h = 0; h < 2; h++) {
                    const uint32_t tcol = tmem + lane_base + (uint32_t)(acc * HBN + g * 64 + 32 * h);
                    uint32_t v[32];
                    tmem_ld32(tcol, v);
                    const int c0 = col0 + 32 * h;
                    float sbv[32];
                    if (c0 + 32 <= p.Dk) {
                        if (p.sb) {
                            const float4 *s4 = reinterpret_cast<const float4 *>(p.sb + c0);
#pragma unroll
                            for (int i = 0; i < 8; i++) {
                                const float4 x = s4[i];
                                sbv[4 * i] = x.x; sbv[4 * i + 1] = x.y; sbv[4 * i + 2] = x.z; sbv[4 * i + 3] = x.w;
                            }
                        } else {
#pragma unroll
                            for (int i = 0; i < 32; i++) sbv[i] = 1.f;
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < 32; i++) sbv[i] = c0 + i < p.Dk ? (p.sb ? p.sb[c0 + i] : 1.f) : 0.f;
                    }
                    uint32_t w[16];
                    float qa = 0.f, qb2 = 0.f;   // two chains
#pragma unroll
                    for (int i = 0; i < 16; i++) {
                        const __nv_bfloat16 b0 = __float2bfloat16_rn(__uint_as_float(v[2 * i]) * sbv[2 * i]);
                        const __nv_bfloat16 b1 = __float2bfloat16_rn(__uint_as_float(v[2 * i + 1]) * sbv[2 * i + 1]);
                        const float g0 = __bfloat162float(b0), g1 = __bfloat162float(b1);
                        qa = fmaf(g0, g0, qa);
                        qb2 = fmaf(g1, g1, qb2);
                        w[i] = (uint32_t)__bfloat16_as_ushort(b0) | ((uint32_t)__bfloat16_as_ushort(b1) << 16);
                    }
                    qsum += qa + qb2;
                    fc_tmem_st16(tcol, w);   // the half's 32 BF16 into its first 16 columns (read above)
                }
                fc_tmem_st_wait();
                tc_fence_before();
                mbar_arrive(a2full(acc));
                if (++acc == 2) { acc = 0; aphase ^= 1; }
            }
            if (ab) break;
            // the row's squared norm: the warpgroups' partial sums in order g = 0, 1, 2
            float *sq = s_q + (size_t)qb * HEWG * BM;
            sq[g * BM + r] = qsum;
            mbar_arrive(qfull(qb));
            const bool okq = mbar_wait(qfull(qb), qph, abort_flag);
            if (!__all_sync(0xffffffffu, okq)) { ab = true; break; }
            float qn = 0.f;
#pragma unroll
            for (int h = 0; h < HEWG; h++) qn += sq[h * BM + r];
            if (++qb == 2) { qb = 0; qph ^= 1; }
            const double qnorm = sqrt((double)qn);
            const bool okd = mbar_wait(d2full, d2ph, abort_flag);
            if (!__all_sync(0xffffffffu, okd)) { ab = true; break; }
            tc_fence_after();
            // warpgroup g scores classes [c0, c1), a third of them (FP64
            // arithmetic is slow on this part: spread it over all warpgroups)
            const int cper = (p.C + HEWG - 1) / HEWG;
            const int c0 = g * cper, c1 = min(c0 + cper, p.C);
            int best = -1;
            double bs = 0.0;
            for (int j = c0 / 32; j * 32 < c1; j++) {   // the 32-class chunks that hold [c0, c1)
                uint32_t v[32];
                tmem_ld32(tmem + lane_base + D2_COL + (uint32_t)(j * 32), v);
#pragma unroll
                for (int i = 0; i < 32; i++) {
                    const int c = j * 32 + i;
                    if (c >= c0 && c < c1) {
                        const double den = qnorm * p.cnorm[c];
                        const double sc = den == 0.0 ? 0.0 : (double)__uint_as_float(v[i]) / den;
                        if (p.scores && valid) p.scores[row * p.C + c] = sc;
                        if (best < 0 || sc > bs) { bs = sc; best = c; }   // ascending c: lowest on ties
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(d2empty);
            d2ph ^= 1;
            const uint32_t par = (uint32_t)(it & 1);
            if (g > 0) {
                if (!mbar_wait(merge_empty, par ^ 1, abort_flag)) { ab = true; break; }
                s_val[(g - 1) * BM + r] = bs;
                s_idx[(g - 1) * BM + r] = best;
                mbar_arrive(merge_full);
            } else {
                if (!mbar_wait(merge_full, par, abort_flag)) { ab = true; break; }
#pragma unroll
                for (int h = 0; h < HEWG - 1; h++) {   // (score desc, class asc)
                    const double v1 = s_val[h * BM + r];
                    const int i1 = s_idx[h * BM + r];
                    if (i1 >= 0 && (best < 0 || v1 > bs || (v1 == bs && i1 < best))) { bs = v1; best = i1; }
                }
                mbar_arrive(merge_empty);
                if (valid) p.labels[row] = best < 0 ? 0 : best;
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

template <int ENC, int STAGES, int B2BUF>
static cudaError_t launch_fcos_stages(const CUtensorMap &ma, const CUtensorMap &mb, const CUtensorMap &mv,
                                      const FCParams &p, unsigned grid, cudaStream_t st)
{
    auto k = tc_fcos_kernel<ENC, STAGES, B2BUF>;
    const size_t smem = fc_smem_bytes(STAGES, p.Cp, B2BUF);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, FC_THREADS, smem, st>>>(ma, mb, mv, p);
    return cudaGetLastError();
}

template <int ENC>
static cudaError_t launch_fcos_enc(const CUtensorMap &ma, const CUtensorMap &mb, const CUtensorMap &mv,
                                   const FCParams &p, unsigned grid, cudaStream_t st)
{
    // a second class tile where it fits (small C), else a fourth A/B stage
    // where that fits, else three stages and one class tile
    if (fc_smem_bytes(3, p.Cp, 2) <= 232448) return launch_fcos_stages<ENC, 3, 2>(ma, mb, mv, p, grid, st);
    if (fc_smem_bytes(4, p.Cp, 1) <= 232448) return launch_fcos_stages<ENC, 4, 1>(ma, mb, mv, p, grid, st);
    return launch_fcos_stages<ENC, 3, 1>(ma, mb, mv, p, grid, st);
}

cudaError_t launch_fcos_bf16(const CUtensorMap &ma, const CUtensorMap &mb, const CUtensorMap &mv,
                             const FCParams &p, unsigned grid, cudaStream_t st);
cudaError_t launch_fcos_fp8(const CUtensorMap &ma, const CUtensorMap &mb, const CUtensorMap &mv,
                            const FCParams &p, unsigned grid, cudaStream_t st);

}  // namespace tc
}  // namespace hdc
