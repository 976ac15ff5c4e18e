// Hamming arg-min of packed binary hypervectors on the tensor cores
// (Sec. 4.1 Hamming distance and arg-min primitives; 17 <= C <= 256 binary
// classes).
//
// For +-1 vectors over the kept dims K, Hamming(q, c) = (|K| - q.c) / 2 and
// q.c is an exact integer in FP32.  The packed words of a 256-dim tile are
// expanded in shared memory into E4M3 bytes: +1.0 (0x38) for bit 0, -1.0
// (0xB8) for bit 1, 0 for a dim outside K (perforated away, or past D).  A
// nibble of four dims becomes four bytes through one multiply that moves
// its bits to the byte sign bits:
//   ((nib * 0x10204080) & 0x80808080) | 0x38383838
// (the four shifted copies of the nibble occupy disjoint bits, so there are
// no carries).  Then
//   D2 += Qtile . Ctile^T     (M 128 queries, N = Cp, K = 256 bytes)
// accumulates over all tiles in tensor memory, and the epilogue takes the
// arg-min of (|K| - dot) / 2 with the lowest class on ties.
//
// Roles (9 warps): warps 0-7 expand the query tile (thread = row x 128-dim
// half; its words loaded three tiles ahead) and the class tile, double
// buffered, and afterwards read D2 (two
// warpgroups, alternate 32-class chunks, merged by (distance, class));
// warp 8 issues the MMAs.  Every wait is bounded as in the encoder.
//
// TA: the query tile goes to tensor memory instead: each expanding thread
// writes its row's E4M3 bytes into its own TMEM lane (tcgen05.st, four bytes
// per column, dims in ascending byte order) and the MMAs take A from there
// (K-major, row i in lane i), so that shared memory carries only the class
// operand.  TMEM: with two CTAs per SM (Cp <= 128) D2 in columns 0..127 and
// the two query buffers of 64 columns (256 dims) each in columns 128..255 of
// 256; with one (Cp <= 256) D2 in columns 0..255 and the buffers in
// 256..383 of 512.
//
// PRE: the class hypervectors come already expanded (E4M3 +-1 bytes, Cp rows
// of ldcs bytes, from launch_class_sign into the caller's workspace), and
// thread 0 streams each tile's two class atoms by TMA on a barrier of their
// own; the expanders then expand only the query rows.  Classes outside the
// kept dims need no zeros there: the query bytes are zero outside K.
#pragma once
#include "tc_hamming.cuh"

namespace hdc {
namespace tc {

// 256-dim tiles: eight packed words per row, two 128-byte K atoms
constexpr int HP_EXP = 256;                    // expanding threads (warps 0-7)
constexpr int HP_THREADS = HP_EXP + 32;
constexpr int HP_CMAX = 256;
constexpr int HP_A_BYTES = 2 * BM * 128;       // query tile: two atoms of 128 rows x 128 bytes
constexpr int HP_MAX_W = 4096;                 // words of a packed row (D <= 131072)
// full[2], empty[2], d2full, d2empty, merge_full, merge_empty, done, cfull[2]
constexpr int HP_NUM_BARS = 11;

constexpr int HP_TA_CMAX = 128;                // TA: largest padded class count with two CTAs per SM

// bbuf: class-tile buffers (2, or 1 so that two CTAs fit per SM); ta: the
// query tile in tensor memory (no shared-memory query buffers)
__host__ __device__ constexpr size_t hp_smem_bytes(int Cp, int W, int bbuf = 2, bool ta = false)
{
    return 1024 + (ta ? (size_t)0 : (size_t)2 * HP_A_BYTES) + (size_t)bbuf * 2 * Cp * 128 + (size_t)(W + 2) * 4 +
           HP_NUM_BARS * 8 + 16 + (size_t)2 * BM * 4;
}
static_assert(hp_smem_bytes(HP_CMAX, HP_MAX_W) <= 232448, "shared memory of the packed tensor-core Hamming kernel");
static_assert(2 * (hp_smem_bytes(HP_TA_CMAX, HP_MAX_W, 2, true) + 1024) <= 228 * 1024, "two TA CTAs per SM");
static_assert(hp_smem_bytes(HP_CMAX, HP_MAX_W, 2, true) <= 232448, "one TA CTA per SM");

struct HPParams {
    const uint32_t *Q;       // N x W packed rows
    const uint32_t *cls;     // C x W packed class hypervectors
    int64_t N;
    int W, C, Cp, nt;        // nt: 256-dim tiles = ceil(W / 8)
    int64_t D, s0, e0, stride;   // dims of the rows; kept dims s0 + k*stride < e0 (stride 1, [0, D) if none)
    int32_t *labels, *dists;
};

// Four dims as four E4M3 bytes.  t holds the four bits at bits 0..3 (lo) or
// 4..7 (hi), nothing else: the multiply moves bit i to bit 7 of byte i (its
// four shifted copies occupy disjoint bits, so no carry reaches a sign
// bit), the AND keeps the four sign bits and the OR adds 1.0 = 0x38.
__device__ __forceinline__ uint32_t signs_lo(uint32_t t) { return ((t * 0x10204080u) & 0x80808080u) | 0x38383838u; }
__device__ __forceinline__ uint32_t signs_hi(uint32_t t) { return ((t * 0x01020408u) & 0x80808080u) | 0x38383838u; }

// The eight words of E4M3 bytes of one packed word (dims 4k..4k+3 in b[k]).
__device__ __forceinline__ void expand_word(uint32_t w, uint32_t b[8])
{
    const uint32_t w8 = w >> 8, w16 = w >> 16, w24 = w >> 24;
    b[0] = signs_lo(w & 0xFu);
    b[1] = signs_hi(w & 0xF0u);
    b[2] = signs_lo(w8 & 0xFu);
    b[3] = signs_hi(w8 & 0xF0u);
    b[4] = signs_lo(w16 & 0xFu);
    b[5] = signs_hi(w16 & 0xF0u);
    b[6] = signs_lo(w24 & 0xFu);
    b[7] = signs_lo(w >> 28);
}

// Byte masks of the kept dims: 0xFF where kept, 0 elsewhere.
__device__ __forceinline__ void expand_mask(uint32_t m, uint32_t b[8])
{
    expand_word(m, b);
#pragma unroll
    for (int k = 0; k < 8; k++) b[k] = ((b[k] >> 7) & 0x01010101u) * 0xFFu;
}

// 128 dims (four words) of one row into its 128-byte row of a K atom
// (128-byte swizzle: 16-byte chunk ch of row r at ((ch ^ (r & 7)) * 16)).
// Four all-ones mask words (no perforation, not the tail) skip the mask.
__device__ __forceinline__ void expand_row(uint8_t *atom, int r, const uint4 w, const uint4 m)
{
    uint8_t *row = atom + (r >> 3) * 1024 + (r & 7) * 128;
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w}, ms[4] = {m.x, m.y, m.z, m.w};
    const bool all = (m.x & m.y & m.z & m.w) == 0xffffffffu;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        uint32_t b[8];
        expand_word(ws[i], b);
        if (!all) {
            uint32_t mb[8];
            expand_mask(ms[i], mb);
#pragma unroll
            for (int k = 0; k < 8; k++) b[k] &= mb[k];
        }
        *reinterpret_cast<uint4 *>(row + (((2 * i) ^ (r & 7)) * 16)) = make_uint4(b[0], b[1], b[2], b[3]);
        *reinterpret_cast<uint4 *>(row + (((2 * i + 1) ^ (r & 7)) * 16)) = make_uint4(b[4], b[5], b[6], b[7]);
    }
}

// Eight 32-bit TMEM columns of this thread's lane (a warp writes its own
// 32-lane quarter), and the wait for this thread's stores to land.
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(r[0]),
                 "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// 128 dims (four words) of one row into 32 TMEM columns of its lane: dims
// 4j..4j+3 of the four words in column taddr + j, lowest dim in the lowest
// byte.  The mask words are the same for the whole warp (one 128-dim half).
__device__ __forceinline__ void expand_row_tmem(uint32_t taddr, const uint4 w, const uint4 m)
{
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w}, ms[4] = {m.x, m.y, m.z, m.w};
    const bool all = (m.x & m.y & m.z & m.w) == 0xffffffffu;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        uint32_t b[8];
        expand_word(ws[i], b);
        if (!all) {
            uint32_t mb[8];
            expand_mask(ms[i], mb);
#pragma unroll
            for (int k = 0; k < 8; k++) b[k] &= mb[k];
        }
        tmem_st8(taddr + 8 * i, b);
    }
}

// D += A . B^T with A (128 rows x 32 E4M3 bytes) in tensor memory at column a.
__device__ __forceinline__ void mma_ts_fp8(uint32_t d, uint32_t a, uint64_t b, uint32_t id, uint32_t accum)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
        "r"(a), "l"(b), "r"(id), "r"(accum));
}

// MINB = 2: two CTAs per SM, registers capped to fit.  BBUF = 1: one
// class-tile buffer (so two CTAs fit with larger class tiles): the class rows
// of tile t are written once the MMAs of tile t - 1 have read them.
template <int MINB, int BBUF, bool PRE, bool TA = false>
__global__ void __launch_bounds__(HP_THREADS, MINB)
    tc_hamming_packed_kernel(const HPParams p, const __grid_constant__ CUtensorMap tmC)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = smem;                                          // 2 buffers x HP_A_BYTES (none with TA)
    uint8_t *sB = sA + (TA ? 0 : 2 * HP_A_BYTES);                // 2 buffers x two atoms of Cp x 128 bytes
    const int b_bytes = 2 * p.Cp * 128;
    uint32_t *smask = reinterpret_cast<uint32_t *>(sB + BBUF * b_bytes);   // W mask words
    uint64_t *bars = reinterpret_cast<uint64_t *>(smask + ((p.W + 1) & ~1));
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + HP_NUM_BARS);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    int *s_kept = reinterpret_cast<int *>(tmem_slot + 2);
    int32_t *s_val = reinterpret_cast<int32_t *>(tmem_slot + 4);   // warpgroup 1: per-row minimum
    int32_t *s_idx = s_val + BM;                                   // and its class
    auto full = [&](int b) { return su32(bars + b); };
    auto empty = [&](int b) { return su32(bars + 2 + b); };
    const uint32_t d2full = su32(bars + 4), d2empty = su32(bars + 5);
    const uint32_t merge_full = su32(bars + 6), merge_empty = su32(bars + 7), done_bar = su32(bars + 8);
    auto cfull = [&](int b) { return su32(bars + 9 + b); };   // PRE: the class atoms of buffer b landed
    constexpr int ISSUER = HP_EXP / 32;
    // TMEM columns of the CTA and the first column of its TA query buffers
    constexpr int TCOLS = TA && MINB == 1 ? 512 : 256;
    constexpr uint32_t TA_COL = MINB == 1 ? 256 : 128;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t num_m_tiles = (p.N + BM - 1) / BM;

    if (tid == 0) {
        for (int b = 0; b < 2; b++) {
            mbar_init(full(b), HP_EXP);
            mbar_init(empty(b), 1);
        }
        mbar_init(d2full, 1);
        mbar_init(d2empty, HP_EXP);
        mbar_init(merge_full, BM);
        mbar_init(merge_empty, BM);
        mbar_init(done_bar, 1);
        for (int b = 0; b < 2; b++) mbar_init(cfull(b), 1);
        *abort_flag = 0;
        *s_kept = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // kept-dim mask of every word (dims past D are never kept), and |K|
    for (int w = tid; w < p.W; w += blockDim.x) {
        uint32_t m = 0;
        const int64_t base = (int64_t)w * 32;
        const int64_t lo = max(p.s0, base), hi = min(min(p.e0, p.D), base + 32);
        if (lo < hi) {
            if (p.stride == 1) {
                const int a = (int)(lo - base), b = (int)(hi - base);
                m = (b == 32 ? 0xffffffffu : ((1u << b) - 1u)) & ~((1u << a) - 1u);
            } else {
                const int64_t r0 = (lo - p.s0) % p.stride;
                for (int64_t d = r0 ? lo + (p.stride - r0) : lo; d < hi; d += p.stride) m |= 1u << (d - base);
            }
        }
        smask[w] = m;
        if (m) atomicAdd(s_kept, __popc(m));
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int kept = *s_kept;

    if (warp == ISSUER) {
        if (lane == 0) {  // ------------------------------ MMA issuer
            const uint32_t id = idesc_n<HDC_ENC_FP8_E4M3>(p.Cp);
            int buf = 0;
            uint32_t ph = 0, d2ph = 0, cph[2] = {0, 0};
            bool ab = false;
            for (int64_t mt = blockIdx.x; mt < num_m_tiles && !ab; mt += gridDim.x) {
                if (!mbar_wait_fast(d2empty, d2ph ^ 1, abort_flag)) { ab = true; break; }
                for (int t = 0; t < p.nt; t++) {
                    if (!mbar_wait_fast(full(buf), ph, abort_flag)) { ab = true; break; }
                    if (PRE) {
                        const int cb = BBUF == 2 ? buf : 0;
                        if (!mbar_wait_fast(cfull(cb), cph[cb], abort_flag)) { ab = true; break; }
                        cph[cb] ^= 1;
                    }
                    tc_fence_after();
                    const uint64_t da = sdesc(su32(sA + buf * HP_A_BYTES));
                    const uint64_t db = sdesc(su32(sB + (BBUF == 2 ? buf : 0) * b_bytes));
                    const uint32_t atom_b = (uint32_t)(p.Cp * 128) >> 4;   // second K atom of the class tile
                    const uint32_t ta = tmem + TA_COL + (uint32_t)(buf * 64);   // TA: this buffer's columns
#pragma unroll
                    for (int k = 0; k < 8; k++) {   // two atoms of four 32-byte K steps
                        const uint64_t ob = (uint64_t)((k >> 2) * atom_b + 2 * (k & 3));
                        if (TA) {
                            mma_ts_fp8(tmem, ta + (uint32_t)(8 * k), db + ob, id, (t | k) != 0);
                        } else {
                            const uint64_t oa = (uint64_t)((k >> 2) * ((BM * 128) >> 4) + 2 * (k & 3));
                            mma<HDC_ENC_FP8_E4M3>(tmem, da + oa, db + ob, id, (t | k) != 0);
                        }
                    }
                    mma_commit(empty(buf));
                    if (++buf == 2) { buf = 0; ph ^= 1; }
                }
                if (ab) break;
                mma_commit(d2full);
                d2ph ^= 1;
            }
            mma_commit(done_bar);
            const unsigned long long t0 = gtimer();
            while (!mbar_try(done_bar, 0) && gtimer() - t0 < 100000000ull) {}
        }
    } else if (warp < ISSUER) {  // ------------------------ expansion and epilogue warps 0 .. 7
        const int r = tid & (BM - 1), half = tid >> 7;   // query row of the tile, 128-dim half (atom)
        const int g = half;                               // epilogue warpgroup
        const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
        int buf = 0;
        uint32_t ph = 0, d2ph = 0;
        bool ab = false;
        int64_t it = 0, gt = 0;   // gt: tiles expanded by this CTA
        uint32_t c_issued = 0, c_par = 0, c_ph[2] = {0, 0};   // PRE (thread 0): class copies in flight
        for (int64_t mt = blockIdx.x; mt < num_m_tiles && !ab; mt += gridDim.x, it++) {
            const int64_t row = mt * BM + r;
            const bool valid = row < p.N;
            const uint32_t *qrow = p.Q + (valid ? row : 0) * (int64_t)p.W;
            // query and class words of the next tile, loaded one tile ahead;
            // class items i = tid and tid + HP_EXP: half h = i / Cp, class
            // c = i % Cp (consecutive lanes on consecutive rows of one atom:
            // no shared-memory bank conflicts on the expanded stores)
            auto class_words = [&](int i, int t) {
                const int c = i % p.Cp, wc = t * 8 + (i / p.Cp) * 4;
                return (i < 2 * p.Cp && c < p.C && wc < p.W)
                           ? *reinterpret_cast<const uint4 *>(p.cls + (int64_t)c * p.W + wc)
                           : make_uint4(0, 0, 0, 0);
            };
            // this thread's four words of tile t, loaded three tiles ahead
            auto query_words = [&](int t) {
                const int w = t * 8 + half * 4;
                return (valid && w < p.W) ? __ldg(reinterpret_cast<const uint4 *>(qrow + w)) : make_uint4(0, 0, 0, 0);
            };
            uint4 q0 = query_words(0), q1 = query_words(1), q2 = query_words(2);
            uint4 cn0 = make_uint4(0, 0, 0, 0), cn1 = cn0;
            if (!PRE) {
                cn0 = class_words(tid, 0);
                cn1 = class_words(tid + HP_EXP, 0);
            }
            for (int t = 0; t < p.nt; t++) {
                const uint4 qw = q0, cw0 = cn0, cw1 = cn1;
                const int w0 = t * 8 + half * 4;                  // this thread's four words
                q0 = q1;
                q1 = q2;
                q2 = query_words(t + 3);
                if (!PRE && t + 1 < p.nt) {
                    cn0 = class_words(tid, t + 1);
                    cn1 = class_words(tid + HP_EXP, t + 1);
                }
                const bool oke = mbar_wait(empty(buf), ph ^ 1, abort_flag);   // the MMAs of this buffer's last use
                if (!__all_sync(0xffffffffu, oke)) { ab = true; break; }
                if (TA) tc_fence_after();   // this thread's TMEM stores after those MMAs
                if (BBUF == 1 && gt > 0) {   // the single class tile: the previous tile's MMAs have read it
                    const bool okp = mbar_wait(empty(buf ^ 1), buf ? ph : ph ^ 1, abort_flag);
                    if (!__all_sync(0xffffffffu, okp)) { ab = true; break; }
                }
                gt++;
                uint8_t *bt = sB + (BBUF == 2 ? buf : 0) * b_bytes;
                if (PRE && tid == 0) {   // the tile's two class atoms, on their own barrier
                    const int cb = BBUF == 2 ? buf : 0;
                    mbar_expect_tx(cfull(cb), (uint32_t)b_bytes);
                    tma_load_2d(su32(bt), &tmC, t * 256, 0, cfull(cb));
                    tma_load_2d(su32(bt + p.Cp * 128), &tmC, t * 256 + 128, 0, cfull(cb));
                    c_issued |= 1u << cb;
                    c_par = (c_par & ~(1u << cb)) | (c_ph[cb] << cb);
                    c_ph[cb] ^= 1;
                }
                const uint4 mq = w0 < p.W ? *reinterpret_cast<const uint4 *>(smask + w0) : make_uint4(0, 0, 0, 0);
                if (TA) {   // converged for the warp-wide TMEM stores (thread 0 may have issued the class copy)
                    __syncwarp();
                    expand_row_tmem(tmem + lane_base + TA_COL + (uint32_t)(buf * 64 + half * 32), qw, mq);
                } else {
                    expand_row(sA + buf * HP_A_BYTES + half * (BM * 128), r, qw, mq);
                }
                // class rows: items (class c, half h) i = tid, tid + HP_EXP (2 * Cp <= 512)
#pragma unroll
                for (int ii = 0; ii < (PRE ? 0 : 2); ii++) {
                    const int i = tid + ii * HP_EXP;
                    if (i < 2 * p.Cp) {
                        const int c = i % p.Cp, h = i / p.Cp;
                        const int wc = t * 8 + h * 4;
                        const uint4 mc = (c < p.C && wc < p.W) ? *reinterpret_cast<const uint4 *>(smask + wc)
                                                               : make_uint4(0, 0, 0, 0);
                        expand_row(bt + h * (p.Cp * 128), c, ii ? cw1 : cw0, mc);
                    }
                }
                if (TA) {   // the query columns landed before the MMAs read them
                    tmem_st_wait();
                    tc_fence_before();
                }
                fence_async_smem();
                mbar_arrive(full(buf));
                if (++buf == 2) { buf = 0; ph ^= 1; }
            }
            if (ab) break;
            // distances: warpgroup g reads the 32-class chunks j = g, g + 2, ...
            const bool okd = mbar_wait(d2full, d2ph, abort_flag);
            if (!__all_sync(0xffffffffu, okd)) { ab = true; break; }
            tc_fence_after();
            int best = 0x7fffffff, bv = 0x7fffffff;
            for (int j = g; j * 32 < p.Cp; j += 2) {
                uint32_t v[32];
                tmem_ld32(tmem + lane_base + (uint32_t)(j * 32), v);
#pragma unroll
                for (int i = 0; i < 32; i++) {
                    const int c = j * 32 + i;
                    if (c < p.C) {
                        const int dist = (kept - (int)__uint_as_float(v[i])) / 2;
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
                s_val[r] = bv;
                s_idx[r] = best;
                mbar_arrive(merge_full);
            } else {
                if (!mbar_wait(merge_full, par, abort_flag)) { ab = true; break; }
                const int v1 = s_val[r], i1 = s_idx[r];
                if (v1 < bv || (v1 == bv && i1 < best)) { bv = v1; best = i1; }   // (distance, class)
                mbar_arrive(merge_empty);
                if (valid) p.labels[row] = best;
            }
        }
        if (PRE && ab && tid == 0)   // let this thread's class copies land before the CTA exits
            for (int b = 0; b < 2; b++)
                if (c_issued >> b & 1) {
                    const unsigned long long t0 = gtimer();
                    while (!mbar_try(cfull(b), c_par >> b & 1) && gtimer() - t0 < 100000000ull) {}
                }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS) : "memory");
    }
}

}  // namespace tc
}  // namespace hdc
