// Fused classify of float (non-binarised) query hypervectors for at most 16
// classes, on the binary classify's 256-dim encode tiles (Sec. 4.2
// Algorithmic Choice; the float + cosine form of Sec. 5.2).
//
// For each 256-dim tile t of a 128-query block:
//   S = Xq . Bq^T          (MMA1: M 128, N 256, K = F, BF16 or E4M3) into one
//                          of two 256-column TMEM accumulators
//   q = bf16(S * sb_k)     (epilogue: four warpgroups, 64 columns each; sum of
//                          q^2 kept per row; the tile's 256 base-row scales
//                          arrive in shared memory with its class values, zero
//                          past D').  Each thread writes the 32 BF16 of every
//                          32-column half it has read back into the first 16
//                          of those columns (two per column, lower dim in the
//                          low half), so the operand never touches shared
//                          memory
//   P_t = q . Cv_t^T       (MMA2: M 128, N 16, K 256, BF16, A from tensor
//                          memory) written into columns 16..31 of tile t's own
//                          accumulator, S values the epilogue has read and no
//                          BF16 pair occupies
//   dot += P_t             (warpgroup 0, FP32 registers)
// After the last tile: score_c = dot_c / (||q|| ||c||) in FP64 (0 for a zero
// norm), arg-max with the lowest class on ties.  The projections never reach
// device memory.  Reusing the encode accumulator for the cosine partials is
// what lets the encode keep 256-dim tiles with both TMEM accumulators: 20
// tiles of 7 stages per block at D' = 5,000 instead of 27 with 192-dim tiles.
//
// Roles: warps 0-15 epilogue, 16 stage producer, 17 MMA1 issuer, 18 class
// tile producer, 19 MMA2 issuer.  Every wait is bounded as in the encoder.
#pragma once
#include "tc_fcos.cuh"

namespace hdc {
namespace tc {

constexpr int F16_EWG = 4;                             // epilogue warpgroups, 64 columns of a tile each
// encode stages: three for E4M3, four for BF16 (the shared memory the value
// tile no longer takes; FP8 measured 1 % slower with four, BF16 5 % faster)
template <int ENC>
__host__ __device__ constexpr int f16_stages() { return ENC == HDC_ENC_BF16 ? 4 : 3; }
constexpr int F16_CP = 16;                             // class rows of MMA2
constexpr int F16_THREADS = (4 * F16_EWG + 4) * 32;
constexpr int F16_B2_BYTES = 4 * F16_CP * 128;         // 16 class rows x 256 BF16: four atoms
constexpr int F16_SB_BYTES = BN * 4;                   // the tile's base-row scales (FP8)
// full[S], empty[S], tfull[2], tempty[2], d2full[2], a2full[2], b2full,
// b2empty, qfull[2], done, done2.  a2full is per accumulator: epilogue
// warps that run ahead to the next tile arrive on the other barrier, and
// tile t + 2's arrivals wait (through tempty) for MMA2 of tile t.
template <int ENC>
__host__ __device__ constexpr int f16_num_bars() { return 2 * f16_stages<ENC>() + 14; }

template <int ENC>
__host__ __device__ constexpr size_t f16_smem_bytes()
{
    return 1024 + (size_t)f16_stages<ENC>() * STAGE_BYTES + F16_B2_BYTES + F16_SB_BYTES + f16_num_bars<ENC>() * 8 +
           16 + (size_t)2 * F16_EWG * BM * 4;
}

// Sixteen 32-bit TMEM columns of this thread's lane (the warp's own 32-lane
// quarter), and the wait for this thread's stores to land.
__device__ __forceinline__ void f16_tmem_st16(uint32_t taddr, const uint32_t (&r)[16])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
                 ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]),
                 "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
                 "r"(r[15])
                 : "memory");
}
__device__ __forceinline__ void f16_tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// D += A . B^T, BF16, A (128 rows x 16 BF16) in tensor memory at column a.
__device__ __forceinline__ void f16_mma_ts(uint32_t d, uint32_t a, uint64_t b, uint32_t id, uint32_t accum)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
        "r"(a), "l"(b), "r"(id), "r"(accum));
}
static_assert(f16_smem_bytes<HDC_ENC_BF16>() <= 232448 && f16_smem_bytes<HDC_ENC_FP8_E4M3>() <= 232448,
              "shared memory of the 16-class fused float-query kernel");

template <int ENC>
__global__ void __launch_bounds__(F16_THREADS, 1)
    tc_fcos16_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     const __grid_constant__ CUtensorMap tmV, const __grid_constant__ CUtensorMap tmS,
                     const FCParams p)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = smem;
    constexpr int S = f16_stages<ENC>();
    uint8_t *sB = smem + S * A_BYTES;
    uint8_t *sB2 = smem + S * STAGE_BYTES;
    float *s_sb = reinterpret_cast<float *>(sB2 + F16_B2_BYTES);   // BN scales of the tile (FP8)
    uint64_t *bars = reinterpret_cast<uint64_t *>(sB2 + F16_B2_BYTES + F16_SB_BYTES);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + f16_num_bars<ENC>());
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    float *s_q = reinterpret_cast<float *>(tmem_slot + 4);   // 2 x [F16_EWG][BM] partial squared norms
    auto full = [&](int s) { return su32(bars + s); };
    auto empty = [&](int s) { return su32(bars + S + s); };
    auto tfull = [&](int a) { return su32(bars + 2 * S + a); };
    auto tempty = [&](int a) { return su32(bars + 2 * S + 2 + a); };
    auto d2full = [&](int a) { return su32(bars + 2 * S + 4 + a); };
    auto a2full = [&](int a) { return su32(bars + 2 * S + 6 + a); };
    const uint32_t b2full = su32(bars + 2 * S + 8), b2empty = su32(bars + 2 * S + 9);
    auto qfull = [&](int b) { return su32(bars + 2 * S + 10 + b); };
    const uint32_t done_bar = su32(bars + 2 * S + 12), done2_bar = su32(bars + 2 * S + 13);
    constexpr int PRODUCER = 4 * F16_EWG, ISSUER = PRODUCER + 1, CPRODUCER = PRODUCER + 2, ISSUER2 = PRODUCER + 3;
    constexpr int KELEMS = ENC == HDC_ENC_BF16 ? BKB / 2 : BKB;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t num_m_tiles = (p.N + BM - 1) / BM;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; s++) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        for (int a = 0; a < 2; a++) {
            mbar_init(tfull(a), 1);
            mbar_init(tempty(a), BM * F16_EWG);
            mbar_init(d2full(a), 1);
            mbar_init(qfull(a), BM * F16_EWG);
        }
        for (int a = 0; a < 2; a++) mbar_init(a2full(a), BM * F16_EWG);
        mbar_init(b2full, 1);
        mbar_init(b2empty, 1);
        mbar_init(done_bar, 1);
        mbar_init(done2_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(TMEM_COLS)
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
            bool issued[S];
            uint32_t ipar[S];
            for (int s = 0; s < S; s++) { issued[s] = false; ipar[s] = 0; }
            bool ab = false;
            for (int64_t mt = blockIdx.x; mt < num_m_tiles && !ab; mt += gridDim.x)
                for (int t = 0; t < p.nt && !ab; t++)
                    for (int kb = 0; kb < p.num_kb; kb++) {
                        if (!mbar_wait(empty(stage), phase ^ 1, abort_flag)) { ab = true; break; }
                        mbar_expect_tx(full(stage), STAGE_BYTES);
                        tma_load_2d(su32(sA + stage * A_BYTES), &tmA, kb * KELEMS, (int)(mt * BM), full(stage));
                        tma_load_2d(su32(sB + stage * B_BYTES), &tmB, kb * KELEMS, t * BN, full(stage));
                        issued[stage] = true;
                        ipar[stage] = phase;
                        if (++stage == S) { stage = 0; phase ^= 1; }
                    }
            if (ab) {  // let our own copies land before the CTA exits
                for (int s = 0; s < S; s++)
                    if (issued[s]) {
                        const unsigned long long t0 = gtimer();
                        while (!mbar_try(full(s), ipar[s]) && gtimer() - t0 < 100000000ull) {}
                    }
            }
        }
    } else if (warp == CPRODUCER) {
        if (lane == 0) {  // ------------------------------ class-value tile producer
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmV)) : "memory");
            const bool has_sb = p.sb != nullptr;
            uint32_t ph = 0, last = 0;
            bool any = false, ab = false;
            for (int64_t mt = blockIdx.x; mt < num_m_tiles && !ab; mt += gridDim.x)
                for (int t = 0; t < p.nt; t++) {
                    if (!mbar_wait(b2empty, ph ^ 1, abort_flag)) { ab = true; break; }
                    mbar_expect_tx(b2full, (uint32_t)(F16_B2_BYTES + (has_sb ? F16_SB_BYTES : 0)));
#pragma unroll
                    for (int a = 0; a < 4; a++)   // 64 BF16 of K per atom
                        tma_load_2d(su32(sB2 + a * F16_CP * 128), &tmV, t * BN + a * 64, 0, b2full);
                    if (has_sb) tma_load_2d(su32(s_sb), &tmS, t * BN, 0, b2full);
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
            const uint32_t id1 = idesc_n<ENC>(BN);
            const uint64_t da0 = sdesc(su32(sA)), db0 = sdesc(su32(sB));
            const uint32_t full0 = full(0), empty0 = empty(0);   // stage s: + 8 * s
            int stage = 0, acc = 0;
            uint32_t phase = 0, aphase = 0;
            bool ab = false;
            for (int64_t mt = blockIdx.x; mt < num_m_tiles && !ab; mt += gridDim.x) {
                for (int t = 0; t < p.nt && !ab; t++) {
                    if (!mbar_wait_fast(tempty(acc), aphase ^ 1, abort_flag)) { ab = true; break; }
                    tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)(acc * BN);
                    for (int kb = 0; kb < p.num_kb; kb++) {
                        if (!mbar_wait_fast(full0 + 8u * stage, phase, abort_flag)) { ab = true; break; }
                        tc_fence_after();
                        const uint64_t da = da0 + (uint64_t)(stage * (A_BYTES >> 4));
                        const uint64_t db = db0 + (uint64_t)(stage * (B_BYTES >> 4));
#pragma unroll
                        for (int k = 0; k < BKB / 32; k++) mma<ENC>(d, da + 2 * k, db + 2 * k, id1, (kb | k) != 0);
                        mma_commit(empty0 + 8u * stage);
                        if (++stage == S) { stage = 0; phase ^= 1; }
                    }
                    if (ab) break;
                    mma_commit(tfull(acc));
                    if (++acc == 2) { acc = 0; aphase ^= 1; }
                }
            }
            mma_commit(done_bar);
            const unsigned long long t0 = gtimer();
            while (!mbar_try(done_bar, 0) && gtimer() - t0 < 100000000ull) {}
        }
    } else if (warp == ISSUER2) {
        if (lane == 0) {  // ------------------------------ MMA2 issuer (the tile's cosine partials)
            const uint32_t id2 = idesc_n<HDC_ENC_BF16>(F16_CP);
            uint32_t a2ph = 0, b2ph = 0;   // a2ph: the parity of both accumulators' a2full, flipped per pair
            int acc = 0;
            bool ab = false;
            for (int64_t mt = blockIdx.x; mt < num_m_tiles && !ab; mt += gridDim.x)
                for (int t = 0; t < p.nt; t++) {
                    if (!mbar_wait(a2full(acc), a2ph, abort_flag)) { ab = true; break; }
                    if (!mbar_wait(b2full, b2ph, abort_flag)) { ab = true; break; }
                    tc_fence_after();
                    const uint32_t b0 = su32(sB2);
                    // into columns 16..31 of tile t's accumulator; K step k (dims
                    // 16k..16k+15): warpgroup k / 4's columns, half (k % 4) / 2,
                    // eight columns in
                    const uint32_t tacc = tmem + (uint32_t)(acc * BN), d2 = tacc + 16;
#pragma unroll
                    for (int k = 0; k < 16; k++) {   // four atoms of four 16-element K steps
                        const uint32_t col = (uint32_t)((k >> 2) * 64 + ((k & 3) >> 1) * 32 + (k & 1) * 8);
                        const uint32_t off_b = (uint32_t)((k >> 2) * F16_CP * 128) + 32u * (k & 3);
                        f16_mma_ts(d2, tacc + col, sdesc(b0 + off_b), id2, k == 0 ? 0u : 1u);
                    }
                    mma_commit(b2empty);
                    mma_commit(d2full(acc));
                    b2ph ^= 1;
                    if (++acc == 2) { acc = 0; a2ph ^= 1; }
                }
            mma_commit(done2_bar);
            const unsigned long long t0 = gtimer();
            while (!mbar_try(done2_bar, 0) && gtimer() - t0 < 100000000ull) {}
        }
    } else {  // ------------------------------------------ epilogue warps 0 .. 15
        const int q = warp & 3, g = warp >> 2;
        const int r = q * 32 + lane;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        int acc = 0, qb = 0;
        uint32_t aphase = 0, qph = 0, b2ph = 0;
        bool ab = false;
        const bool has_sb = p.sb != nullptr;
        for (int64_t mt = blockIdx.x; mt < num_m_tiles && !ab; mt += gridDim.x) {
            const int64_t row = mt * BM + r;
            const bool valid = row < p.N;
            float qsum = 0.f;
            float dot[F16_CP];
#pragma unroll
            for (int c = 0; c < F16_CP; c++) dot[c] = 0.f;
            for (int t = 0; t < p.nt; t++) {
                const bool ok = mbar_wait(tfull(acc), aphase, abort_flag);
                if (!__all_sync(0xffffffffu, ok)) { ab = true; break; }
                tc_fence_after();
                if (has_sb) {   // the tile's scales (read before MMA2 of this tile frees the buffer)
                    const bool oks = mbar_wait(b2full, b2ph, abort_flag);
                    if (!__all_sync(0xffffffffu, oks)) { ab = true; break; }
                }
                b2ph ^= 1;
#pragma unroll 1
                for (int h = 0; h < 2; h++) {
                    const uint32_t col = tmem + lane_base + (uint32_t)(acc * BN + g * 64 + 32 * h);
                    uint32_t v[32];
                    tmem_ld32(col, v);
                    // BF16 of s * sb; past D' the projections are zero (zero base rows)
                    const float4 *s4 = reinterpret_cast<const float4 *>(s_sb + g * 64 + 32 * h);
                    uint32_t w[16];
                    float qa = 0.f, qc = 0.f;   // two chains
#pragma unroll
                    for (int i4 = 0; i4 < 8; i4++) {
                        const float4 sv = has_sb ? s4[i4] : make_float4(1.f, 1.f, 1.f, 1.f);
                        const __nv_bfloat162 b01 = __floats2bfloat162_rn(__uint_as_float(v[4 * i4]) * sv.x,
                                                                         __uint_as_float(v[4 * i4 + 1]) * sv.y);
                        const __nv_bfloat162 b23 = __floats2bfloat162_rn(__uint_as_float(v[4 * i4 + 2]) * sv.z,
                                                                         __uint_as_float(v[4 * i4 + 3]) * sv.w);
                        const uint32_t u01 = *reinterpret_cast<const uint32_t *>(&b01);
                        const uint32_t u23 = *reinterpret_cast<const uint32_t *>(&b23);
                        const float g0 = __uint_as_float(u01 << 16), g1 = __uint_as_float(u01 & 0xffff0000u);
                        const float g2 = __uint_as_float(u23 << 16), g3 = __uint_as_float(u23 & 0xffff0000u);
                        qa = fmaf(g0, g0, qa);
                        qc = fmaf(g1, g1, qc);
                        qa = fmaf(g2, g2, qa);
                        qc = fmaf(g3, g3, qc);
                        w[2 * i4] = u01;
                        w[2 * i4 + 1] = u23;
                    }
                    qsum += qa + qc;
                    f16_tmem_st16(col, w);   // the half's 32 BF16 into its first 16 columns (read above)
                }
                f16_tmem_st_wait();
                tc_fence_before();
                mbar_arrive(a2full(acc));
                if (g == 0) {
                    // this tile's cosine partials, in columns 0..15 of its accumulator
                    const bool okd = mbar_wait(d2full(acc), aphase, abort_flag);
                    if (!__all_sync(0xffffffffu, okd)) { ab = true; break; }
                    tc_fence_after();
                    uint32_t v[32];
                    tmem_ld32(tmem + lane_base + (uint32_t)(acc * BN + 16), v);
#pragma unroll
                    for (int c = 0; c < F16_CP; c++) dot[c] += __uint_as_float(v[c]);
                    tc_fence_before();
                }
                mbar_arrive(tempty(acc));
                if (++acc == 2) { acc = 0; aphase ^= 1; }
            }
            if (ab) break;
            // the row's squared norm: the warpgroups' partial sums in order g = 0 .. 3
            float *sq = s_q + (size_t)qb * F16_EWG * BM;
            sq[g * BM + r] = qsum;
            mbar_arrive(qfull(qb));
            if (g == 0) {
                const bool okq = mbar_wait(qfull(qb), qph, abort_flag);
                if (!__all_sync(0xffffffffu, okq)) { ab = true; break; }
                float qn = 0.f;
#pragma unroll
                for (int h = 0; h < F16_EWG; h++) qn += sq[h * BM + r];
                const double qnorm = sqrt((double)qn);
                int best = 0;
                double bs = 0.0;
#pragma unroll
                for (int c = 0; c < F16_CP; c++)
                    if (c < p.C) {
                        const double den = qnorm * p.cnorm[c];
                        const double sc = den == 0.0 ? 0.0 : (double)dot[c] / den;
                        if (p.scores && valid) p.scores[row * p.C + c] = sc;
                        if (c == 0 || sc > bs) { bs = sc; best = c; }   // ascending c: lowest on ties
                    }
                if (valid) p.labels[row] = best;
            }
            if (++qb == 2) { qb = 0; qph ^= 1; }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// ms: map of the Dk base-row scales as one row (box BN, zero fill past Dk); any
// map when p.sb is NULL (BF16), then it is not read.
template <int ENC>
static cudaError_t launch_fcos16_enc(const CUtensorMap &ma, const CUtensorMap &mb, const CUtensorMap &mv,
                                     const CUtensorMap &ms, const FCParams &p, unsigned grid, cudaStream_t st)
{
    auto k = tc_fcos16_kernel<ENC>;
    constexpr size_t smem = f16_smem_bytes<ENC>();
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, F16_THREADS, smem, st>>>(ma, mb, mv, ms, p);
    return cudaGetLastError();
}

cudaError_t launch_fcos16_bf16(const CUtensorMap &ma, const CUtensorMap &mb, const CUtensorMap &mv,
                               const CUtensorMap &ms, const FCParams &p, unsigned grid, cudaStream_t st);
cudaError_t launch_fcos16_fp8(const CUtensorMap &ma, const CUtensorMap &mb, const CUtensorMap &mv,
                              const CUtensorMap &ms, const FCParams &p, unsigned grid, cudaStream_t st);

}  // namespace tc
}  // namespace hdc
