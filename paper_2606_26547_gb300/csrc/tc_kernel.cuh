// Tensor-core encoder for sm_103a (tcgen05 + TMA + TMEM), fused with sign
// binarisation, bit packing and -- in classify mode -- Hamming distance to
// binary class hypervectors and arg-min, so encoded hypervectors never reach
// device memory.
//
// What it computes (Listing 1 end to end, Sec. 4.2 knobs):
//   s[i][k] = sum_f xq[i][f] * bq[k][f]   (BF16 or E4M3 operands, FP32
//                                          accumulation in tensor memory)
//   bit[i][k] = s < 0                      (sign(0) = +1)
//   classify: dist[i][c] = sum_w popc(q_w ^ cls_c,w)      -> arg-min
//   encode:   H[i] = packed bits (and optionally the de-scaled s).
// The per-row power-of-two scales of FP8 are positive, so they do not change
// any bit; they are applied only to the optional projection output.
//
// Structure (one CTA per SM, persistent over 128-query tiles, or over
// (tile, dim-tile range) units for batches of fewer tiles than SMs):
//   warp 4 lane 0  TMA producer: A tile (128 queries x 128 B of K) and B tile
//                  (256 dims x 128 B of K) per stage into a 4-stage ring,
//                  128-byte swizzle, completion on an mbarrier;
//   warp 5 lane 0  MMA issuer: 4 tcgen05.mma (K = 32 bytes each) per stage
//                  into one of two 128 x 256 FP32 accumulators in TMEM,
//                  tcgen05.commit frees the stage / publishes the tile;
//   warps 4*EWG+2, 4*EWG+3 (QIN only)  query quantisers: FP32 rows of the
//                  CTA's next 128-query tile -> BF16 / E4M3 (the row
//                  quantisation of Sec. 4.2) into one of two staged tiles
//                  the CTA owns in global memory, read back by the TMA
//                  producer; the first tile is quantised by the epilogue
//                  warps too, before their first accumulator arrives;
//   warps 0-3      epilogue: tcgen05.ld of the thread's row (TMEM lane),
//                  32 columns at a time -> one packed word, releases the
//                  accumulator, then popcounts against the class words
//                  (CMAX register counters per query).  With EWG = 2 or 4
//                  epilogue warpgroups (classify, C > 16) each warpgroup
//                  packs 8/EWG of the tile's 8 words, the words are
//                  exchanged through shared memory, and warpgroup g counts
//                  the g-th of EWG equal class ranges.
// Every wait is bounded by the global timer; on expiry the kernel records
// status 1 in g_tc_status, stops its loops, drains its own copies and MMAs
// (again with a bound), frees TMEM and returns.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>

#include "hdc_internal.cuh"
#include "quant_math.cuh"

namespace hdc {
namespace tc {

// Device status of the kernels of the including translation unit:
// 0 ok, 1 a bounded wait timed out.
static __device__ int g_tc_status;

constexpr int BM = 128;                      // queries per tile (TMEM lanes)
constexpr int BN = 256;                      // dims per tile (TMEM columns)
constexpr int BKB = 128;                     // K bytes per stage row
constexpr int STAGES = 4;
constexpr int A_BYTES = BM * BKB;            // 16 KB
constexpr int B_BYTES = BN * BKB;            // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
// threads: 4*EWG epilogue warps (EWG = 1, 2 or 4 warpgroups), a TMA warp, an
// MMA warp and, when the kernel quantises its own query tiles, two quantiser
// warps.  Their loads are latency-bound, so the rows each keeps in flight
// (quant_tile's RQ) set how fast a tile's FP32 rows arrive: four beside one
// epilogue warpgroup (eight warps, two per scheduler, up to 255 registers),
// two beside two (twelve warps, three per scheduler: at most 168 registers).
constexpr int QWARPS = 2;
__host__ __device__ constexpr int num_threads(int ewg, bool qin = false)
{
    return (4 * ewg + 2 + (qin ? QWARPS : 0)) * 32;
}
// elements of a staged query row the quantisers hold in registers (8 x 128)
constexpr int QIN_MAX_LD = 1024;
constexpr int TMEM_COLS = 2 * BN;            // two accumulators
// class-word ring (classify): the 8 words of every class for one 256-dim tile
constexpr int CBUF = 4, CLS_BYTES = 128 * 32;
// sign words exchanged between epilogue warpgroups: WXB buffers of [8 words][BM rows]
constexpr int WXB = 2;
// full, empty, tfull[2], tempty[2], done, merge_full, merge_empty, cfull[CBUF], cempty[CBUF], wfull[WXB],
// a0_ready, a_ready[2], a_free[2] (staged query tiles)
constexpr int NUM_BARS = 2 * STAGES + 7 + 2 * CBUF + WXB + 5;
// dynamic shared memory: 1 KB alignment slack, stages, class ring, barriers,
// TMEM slot + abort flag, per-row minimum and class of warpgroups 1..EWG-1,
// exchanged words
__host__ __device__ constexpr size_t smem_bytes(int ewg)
{
    return 1024 + (size_t)STAGES * STAGE_BYTES + CBUF * CLS_BYTES + NUM_BARS * 8 + 16 +
           (size_t)2 * BM * 4 * (ewg > 1 ? ewg - 1 : 1) + (ewg > 1 ? (size_t)WXB * 8 * BM * 4 : 0);
}
static_assert(smem_bytes(4) <= 232448, "shared memory of the four-warpgroup kernel");
constexpr unsigned long long TIMEOUT_NS = 2000000000ull;

struct Params {
    int64_t N;
    int Dk, num_kb, W;
    int last_k = BKB / 32;   // MMA K steps of the last K block that reach into [0, F) (1..4)
    const float *sx, *sb;
    uint32_t *H;
    float *scores;
    const uint32_t *planes;  // binary class hypervectors, C x W
    int C;
    int32_t *labels, *dists;
    uint16_t *sproj;         // encode-only: BF16 projections s_k * sb_k (N x ldS) or NULL
    int ldS;
    float *qn;               // and the squared norm of each BF16 row
    // QIN: the FP32 query rows (N x ldX, 16-byte aligned, F % 4 == 0) and the
    // staged tiles, 2 per CTA of BM rows x ld elements (zeros past F)
    const float *X = nullptr;
    int64_t ldX = 0;
    int F = 0, ld = 0;
    uint8_t *stage = nullptr;
    // classify of few query tiles: each tile's dim tiles split over nsplit
    // CTAs, which add their partial distances into dacc (N x C, zeroed) and
    // count themselves in tile_done (one word per query tile, zeroed); the
    // last contribution takes the arg-min
    int nsplit = 1;
    int32_t *dacc = nullptr;
    unsigned *tile_done = nullptr;
};

// ------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t n)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(n) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity.  Returns false (and
// raises the CTA's abort flag and the device status) after `limit` ns, or
// as soon as another role of the CTA has aborted.
static __device__ __noinline__ bool mbar_wait(uint32_t a, uint32_t parity, volatile int *abort_flag,
                                       unsigned long long limit = TIMEOUT_NS)
{
    if (mbar_try(a, parity)) return true;
    const unsigned long long t0 = gtimer();
    while (true) {
        for (int i = 0; i < 32; i++)
            if (mbar_try(a, parity)) return true;
        if (*abort_flag) return false;
        if (gtimer() - t0 > limit) {
            *abort_flag = 1;
            atomicCAS(&g_tc_status, 0, 1);
            return false;
        }
    }
}

// The bounded wait with its common case inline: an MMA or TMA issuing thread
// that finds the phase already complete spends one try_wait on it.  (Issue
// overhead in the single MMA-issuing thread sits on the tensor pipe's
// critical path: a non-inlined wait and descriptor arithmetic per stage held
// the pipe ~20 % idle in a TMA + MMA pipeline with no epilogue.)
__device__ __forceinline__ bool mbar_wait_fast(uint32_t a, uint32_t parity, volatile int *abort_flag)
{
    return mbar_try(a, parity) || mbar_wait(a, parity, abort_flag);
}

__device__ __forceinline__ void mbar_arrive(uint32_t a)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows
// of 128 bytes, 8-row core groups 1024 bytes apart (SBO), version 1.  The
// start address sits in bits 0-13 in 16-byte units, so the descriptor of an
// operand `bytes` further on is sdesc(addr) + bytes / 16 (shared addresses
// stay below 256 KB: no carry out of the field).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr)
{
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;           // LBO (ignored for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32; // SBO
    d |= (uint64_t)1 << 46;           // descriptor version
    d |= (uint64_t)2 << 61;           // SWIZZLE_128B
    return d;
}

// Instruction descriptor: FP32 accumulator, K-major A and B, M = 128, N = 256;
// operand format BF16 (kind::f16, code 1) or E4M3 (kind::f8f6f4, code 0).
template <int ENC>
__device__ __forceinline__ uint32_t idesc()
{
    const uint32_t fmt = ENC == HDC_ENC_BF16 ? 1u : 0u;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

template <int ENC>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t accum)
{
    if (ENC == HDC_ENC_BF16)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
            "l"(a), "l"(b), "r"(id), "r"(accum));
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
            "l"(a), "l"(b), "r"(id), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane; the wait names the
// registers so no use of them is scheduled before the load has landed.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

// One 32-byte store (a whole sector); p must be 32-byte aligned.
__device__ __forceinline__ void st_global_v8(void *p, const uint32_t *w)
{
    asm volatile("st.global.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "r"(w[0]), "r"(w[1]), "r"(w[2]),
                 "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
                 : "memory");
}

// sign(0) = +1: -0.0 and +0.0 both give bit 0.
__device__ __forceinline__ uint32_t pack_signs(const uint32_t (&r)[32])
{
    uint32_t w = 0;
#pragma unroll
    for (int j = 0; j < 32; j++) w |= (__uint_as_float(r[j]) < 0.f ? 1u : 0u) << j;
    return w;
}

// Quantise rows of one 128-query tile into a staged tile in global memory
// (BM rows x p.ld elements; zeros past F and for rows past N).  This warp
// takes the tile rows w, w + nw, w + 2*nw, ... RQ at a time, issuing all of
// their loads (streaming, evict-first) before converting the first.  The
// arithmetic is the row quantiser's: BF16 by round-to-nearest-even, E4M3
// after the row's power-of-two scale.  The scale itself is not kept: it is
// positive, and the classify epilogue uses only the signs.
// Source and layout of the rows a kernel quantises itself.
struct QinRows {
    const float *X;   // N x ldX FP32 rows (16-byte aligned, F % 4 == 0)
    int64_t ldX, N;
    int F, ld;        // features, elements per staged row (<= QIN_MAX_LD)
};

template <int ENC, int RQ>
__device__ __forceinline__ void quant_tile(const QinRows &p, int64_t row0, uint8_t *tile, int w, int nw, int lane)
{
    constexpr int ES = ENC == HDC_ENC_BF16 ? 2 : 1;
    constexpr int MAXIT = QIN_MAX_LD / 128;
    const int nit = (p.ld + 127) / 128;
    for (int r = w; r < BM; r += nw * RQ) {
        float4 v[RQ][MAXIT];
#pragma unroll
        for (int q = 0; q < RQ; q++) {
            const int rr = r + q * nw;
            const int64_t grow = row0 + rr;
            const bool live = rr < BM && grow < p.N;
            const float *src = p.X + (live ? grow : 0) * p.ldX;
#pragma unroll
            for (int it = 0; it < MAXIT; it++) {
                const int f = it * 128 + lane * 4;
                v[q][it] = live && it < nit && f < p.F ? __ldcs(reinterpret_cast<const float4 *>(src + f))
                                                       : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
#pragma unroll
        for (int q = 0; q < RQ; q++) {
            const int rr = r + q * nw;
            if (rr >= BM) break;   // the same for every lane
            int k = 0;
            if (ENC == HDC_ENC_FP8_E4M3) {
                float amax = 0.f;
#pragma unroll
                for (int it = 0; it < MAXIT; it++)
                    amax = fmaxf(amax, fmaxf(fmaxf(fabsf(v[q][it].x), fabsf(v[q][it].y)),
                                             fmaxf(fabsf(v[q][it].z), fabsf(v[q][it].w))));
#pragma unroll
                for (int o = 16; o; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
                k = pow2_scale_exp(amax);
            }
            uint8_t *dst = tile + (size_t)rr * p.ld * ES;
#pragma unroll
            for (int it = 0; it < MAXIT; it++) {
                const int f0 = it * 128 + lane * 4;
                if (it < nit && f0 < p.ld) {
                    const float4 x = v[q][it];
                    if (ENC == HDC_ENC_BF16)
                        *reinterpret_cast<uint2 *>(dst + (size_t)f0 * 2) = to_bf16x4(x.x, x.y, x.z, x.w);
                    else
                        *reinterpret_cast<uint32_t *>(dst + f0) =
                            to_e4m3x4(scale_pow2(x.x, k), scale_pow2(x.y, k), scale_pow2(x.z, k), scale_pow2(x.w, k));
                }
            }
        }
    }
}

// The staged-tile writes of this thread become visible to the TMA (async
// proxy) reads that follow the barrier it arrives on next.
__device__ __forceinline__ void fence_to_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// ------------------------------------------------------------------ kernel
// QIN (classify, EWG = 1 or 2): the query operand is quantised inside the
// kernel from FP32 rows (quant_tile), one tile ahead of the MMAs, into the
// CTA's two staged tiles; the TMA producer waits for a tile's a_ready (tile
// 0: a0_ready, written by the epilogue and quantiser warps together) and
// the MMA issuer frees it (a_free) once the last stage that reads it has
// landed.
// Work units: every role walks the same units, a query tile and a range of
// its dim tiles (the whole tile unless p.nsplit > 1, a classify of fewer
// tiles than SMs).  A split range's epilogue warps add their partial
// distances into p.dacc and count themselves in p.tile_done; the warp whose
// count completes the tile reads the totals and takes the arg-min.
// EWG = 2 or 4 (classify only): the epilogue warpgroups read the same TMEM
// lanes, warpgroup g the columns of words [g*8/EWG, (g+1)*8/EWG); every
// thread publishes its words to shared memory and, after an mbarrier that
// all epilogue threads arrive on (bounded wait), reads the row's 8 words.
// Warpgroup g counts classes [g*CP, (g+1)*CP), CP = ceil(C/EWG) <= CMAX,
// and warpgroups 1..EWG-1 hand their per-row minimum to warpgroup 0 through
// shared memory (an mbarrier pair with bounded waits), which keeps the lower class
// index on ties.
template <int ENC, int CMAX, bool CLASSIFY, int EWG, bool QIN = false>
__global__ void __launch_bounds__(num_threads(EWG, QIN), 1)
    tc_encode_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     const __grid_constant__ CUtensorMap tmC, const Params p)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = smem;
    uint8_t *sB = smem + STAGES * A_BYTES;
    uint8_t *sCls = smem + STAGES * STAGE_BYTES;  // CBUF x [128 classes][8 words]
    uint64_t *bars = reinterpret_cast<uint64_t *>(sCls + CBUF * CLS_BYTES);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + NUM_BARS);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    auto full = [&](int s) { return su32(bars + s); };
    auto empty = [&](int s) { return su32(bars + STAGES + s); };
    auto tfull = [&](int a) { return su32(bars + 2 * STAGES + a); };
    auto tempty = [&](int a) { return su32(bars + 2 * STAGES + 2 + a); };
    const uint32_t done_bar = su32(bars + 2 * STAGES + 4);
    const uint32_t merge_full = su32(bars + 2 * STAGES + 5), merge_empty = su32(bars + 2 * STAGES + 6);
    auto cfull = [&](int b) { return su32(bars + 2 * STAGES + 7 + b); };
    auto cempty = [&](int b) { return su32(bars + 2 * STAGES + 7 + CBUF + b); };
    auto wfull = [&](int b) { return su32(bars + 2 * STAGES + 7 + 2 * CBUF + b); };
    constexpr int QB = 2 * STAGES + 7 + 2 * CBUF + WXB;   // staged query tile barriers
    const uint32_t a0_ready = su32(bars + QB);
    auto a_ready = [&](int b) { return su32(bars + QB + 1 + b); };
    auto a_free = [&](int b) { return su32(bars + QB + 3 + b); };
    constexpr int QW0 = 4 * EWG + 2;                   // first quantiser warp
    constexpr int QW = QWARPS;                         // quantiser warps
    constexpr int RQ = EWG == 1 ? 4 : 2;               // rows in flight per quantising warp
    constexpr int QES = ENC == HDC_ENC_BF16 ? 2 : 1;
    static_assert(!QIN || (CLASSIFY && EWG <= 2), "in-kernel quantisation: classify with one or two warpgroups");
    const QinRows qr = {p.X, p.ldX, p.N, p.F, p.ld};
    constexpr int NMRG = EWG > 1 ? EWG - 1 : 1;
    int32_t *s_val = reinterpret_cast<int32_t *>(tmem_slot + 4);  // per-row minimum of warpgroups 1..EWG-1
    int32_t *s_idx = s_val + NMRG * BM;                             // and its class
    uint32_t *s_words = reinterpret_cast<uint32_t *>(s_idx + NMRG * BM);  // WXB x [8][BM]
    constexpr int PRODUCER = 4 * EWG, ISSUER = 4 * EWG + 1;
    constexpr int WPG = (BN / 32) / EWG;  // words packed by each epilogue warpgroup
    static_assert(EWG == 1 || EWG == 2 || EWG == 4, "one, two or four epilogue warpgroups");

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t num_m_tiles = (p.N + BM - 1) / BM;
    const int num_n_tiles = (p.Dk + BN - 1) / BN;
    constexpr int KELEMS = ENC == HDC_ENC_BF16 ? BKB / 2 : BKB;
    // work units: (query tile, range of its dim tiles); one range per tile
    // unless the tile's dim tiles are split over several CTAs (nsplit)
    const int NS = (CLASSIFY && !QIN) ? p.nsplit : 1;
    const int ntps = (num_n_tiles + NS - 1) / NS;   // dim tiles per range
    const int64_t num_units = num_m_tiles * NS;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        for (int a = 0; a < 2; a++) {
            mbar_init(tfull(a), 1);
            mbar_init(tempty(a), BM * EWG);
        }
        mbar_init(done_bar, 1);
        mbar_init(merge_full, BM * NMRG);
        mbar_init(merge_empty, BM);
        for (int b = 0; b < CBUF; b++) {
            mbar_init(cfull(b), 1);
            mbar_init(cempty(b), BM * EWG);
        }
        for (int b = 0; b < WXB; b++) mbar_init(wfull(b), BM * EWG);
        mbar_init(a0_ready, (4 * EWG + QW) * 32);
        for (int b = 0; b < 2; b++) {
            mbar_init(a_ready(b), QW * 32);
            mbar_init(a_free(b), 1);
        }
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
        if (lane == 0) {  // ---------------------------------- TMA producer
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
            if (CLASSIFY) asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmC)) : "memory");
            int stage = 0, cb = 0;
            uint32_t phase = 0, cph = 0;
            bool issued[STAGES];
            uint32_t ipar[STAGES];
            for (int s = 0; s < STAGES; s++) { issued[s] = false; ipar[s] = 0; }
            uint32_t c_issued = 0, c_par = 0;
            bool ab = false;
            int64_t it = 0;
            for (int64_t u = blockIdx.x; u < num_units && !ab; u += gridDim.x, it++) {
                const int64_t mt = u / NS;
                const int nt0 = (int)(u % NS) * ntps, nt1 = min(num_n_tiles, nt0 + ntps);
                for (int nt = nt0; nt < nt1 && !ab; nt++) {
                    if (QIN && nt == 0) {  // the tile's staged query rows have been written
                        const bool okq = it == 0 ? mbar_wait(a0_ready, 0, abort_flag)
                                                 : mbar_wait(a_ready((int)(it & 1)), (uint32_t)(((it - 1) >> 1) & 1),
                                                             abort_flag);
                        if (!okq) { ab = true; break; }
                    }
                    if (CLASSIFY) {  // this dim tile's class words: C rows x 8 words (zeros past W)
                        if (!mbar_wait(cempty(cb), cph ^ 1, abort_flag)) { ab = true; break; }
                        mbar_expect_tx(cfull(cb), (uint32_t)p.C * 32u);
                        tma_load_2d(su32(sCls + cb * CLS_BYTES), &tmC, nt * 8, 0, cfull(cb));
                        c_issued |= 1u << cb;
                        c_par = (c_par & ~(1u << cb)) | (cph << cb);
                        if (++cb == CBUF) { cb = 0; cph ^= 1; }
                    }
                    for (int kb = 0; kb < p.num_kb; kb++) {
                        if (!mbar_wait(empty(stage), phase ^ 1, abort_flag)) { ab = true; break; }
                        mbar_expect_tx(full(stage), STAGE_BYTES);
                        const int ay = QIN ? (int)((blockIdx.x * 2 + (it & 1)) * BM) : (int)(mt * BM);
                        tma_load_2d(su32(sA + stage * A_BYTES), &tmA, kb * KELEMS, ay, full(stage));
                        tma_load_2d(su32(sB + stage * B_BYTES), &tmB, kb * KELEMS, nt * BN, full(stage));
                        issued[stage] = true;
                        ipar[stage] = phase;
                        if (++stage == STAGES) { stage = 0; phase ^= 1; }
                    }
                }
            }
            if (ab) {  // let our own copies land before the CTA exits
                for (int s = 0; s < STAGES; s++)
                    if (issued[s]) {
                        const unsigned long long t0 = gtimer();
                        while (!mbar_try(full(s), ipar[s]) && gtimer() - t0 < 100000000ull) {}
                    }
                for (int b = 0; b < CBUF; b++)
                    if (c_issued >> b & 1) {
                        const unsigned long long t0 = gtimer();
                        while (!mbar_try(cfull(b), c_par >> b & 1) && gtimer() - t0 < 100000000ull) {}
                    }
            }
        }
    } else if (warp == ISSUER) {
        if (lane == 0) {  // ---------------------------------- MMA issuer
            const uint32_t id = idesc<ENC>();
            const uint64_t da0 = sdesc(su32(sA)), db0 = sdesc(su32(sB));
            const uint32_t full0 = full(0), empty0 = empty(0);   // stage s: + 8 * s
            int stage = 0, acc = 0;
            uint32_t phase = 0, aphase = 0;
            bool ab = false;
            int64_t it = 0;
            for (int64_t u = blockIdx.x; u < num_units && !ab; u += gridDim.x, it++) {
                const int nt0 = (int)(u % NS) * ntps, nt1 = min(num_n_tiles, nt0 + ntps);
                for (int nt = nt0; nt < nt1 && !ab; nt++) {
                    if (!mbar_wait_fast(tempty(acc), aphase ^ 1, abort_flag)) { ab = true; break; }
                    tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)(acc * BN);
                    for (int kb = 0; kb < p.num_kb; kb++) {
                        if (!mbar_wait_fast(full0 + 8u * stage, phase, abort_flag)) { ab = true; break; }
                        tc_fence_after();
                        // the last copy of the staged query tile has landed:
                        // its quantisers may overwrite it
                        if (QIN && nt == num_n_tiles - 1 && kb == p.num_kb - 1) mbar_arrive(a_free((int)(it & 1)));
                        const uint64_t da = da0 + (uint64_t)(stage * (A_BYTES >> 4));
                        const uint64_t db = db0 + (uint64_t)(stage * (B_BYTES >> 4));
                        // K steps wholly in the zero padding past F add nothing: skipped
                        const int nk = kb == p.num_kb - 1 ? p.last_k : BKB / 32;
#pragma unroll
                        for (int k = 0; k < BKB / 32; k++)
                            if (k < nk) mma<ENC>(d, da + 2 * k, db + 2 * k, id, (kb | k) != 0);
                        mma_commit(empty0 + 8u * stage);
                        if (++stage == STAGES) { stage = 0; phase ^= 1; }
                    }
                    if (ab) break;
                    mma_commit(tfull(acc));
                    if (++acc == 2) { acc = 0; aphase ^= 1; }
                }
            }
            // all MMAs of this thread complete before TMEM is released
            mma_commit(done_bar);
            const unsigned long long t0 = gtimer();
            while (!mbar_try(done_bar, 0) && gtimer() - t0 < 100000000ull) {}
        }
    } else if (QIN && warp >= QW0) {  // --------------------- query quantisers
        const int qw = warp - QW0;
        uint32_t fph = 0;   // parities of the next completions of a_free[0], a_free[1] (bits 0, 1)
        int64_t it = 0;
        for (int64_t mt = blockIdx.x; mt < num_m_tiles && !*abort_flag; mt += gridDim.x, it++) {
            const int b = (int)(it & 1);
            uint8_t *tile = p.stage + (size_t)(blockIdx.x * 2 + b) * BM * p.ld * QES;
            if (it >= 2) {   // tile it - 2 has been read out of this buffer
                const bool okf = mbar_wait(a_free(b), (fph >> b) & 1u, abort_flag);
                fph ^= 1u << b;
                if (!__all_sync(0xffffffffu, okf)) break;
            }
            if (it == 0)
                quant_tile<ENC, RQ>(qr, mt * BM, tile, 4 * EWG + qw, 4 * EWG + QW, lane);
            else
                quant_tile<ENC, RQ>(qr, mt * BM, tile, qw, QW, lane);
            fence_to_async_global();
            mbar_arrive(it == 0 ? a0_ready : a_ready(b));
        }
    } else {  // ------------------------------------ epilogue warps 0 .. 4*EWG-1
        if (QIN) {  // the first staged tile, with the quantiser warps
            quant_tile<ENC, RQ>(qr, (int64_t)blockIdx.x * BM, p.stage + (size_t)blockIdx.x * 2 * BM * p.ld * QES, warp,
                                4 * EWG + QW, lane);
            fence_to_async_global();
            mbar_arrive(a0_ready);
        }
        const int q = warp & 3;             // TMEM lane quarter of this warp
        const int g = warp >> 2;            // epilogue warpgroup
        const int r = q * 32 + lane;        // row of the tile (TMEM lane)
        const int cper = (p.C + EWG - 1) / EWG;
        const int c0 = g * cper;            // classes [c0, c1) counted by this warpgroup
        const int c1 = min(c0 + cper, p.C);
        int acc = 0, cb = 0, wb = 0;
        uint32_t aphase = 0, cph = 0, wph = 0;
        bool ab = false;
        int64_t it = 0;
        for (int64_t u = blockIdx.x; u < num_units && !ab; u += gridDim.x, it++) {
            const int64_t mt = u / NS;
            const int nt0 = (int)(u % NS) * ntps, nt1 = min(num_n_tiles, nt0 + ntps);
            const int64_t row = mt * BM + r;
            const bool valid = row < p.N;
            float qsum = 0.f;   // squared norm of the BF16 projections of this row
            int dist[CLASSIFY ? CMAX : 1];
#pragma unroll
            for (int c = 0; c < (CLASSIFY ? CMAX : 1); c++) dist[c] = 0;
            for (int nt = nt0; nt < nt1; nt++) {
                // warp-uniform outcome: the TMEM loads below are .sync.aligned
                const bool ok = mbar_wait(tfull(acc), aphase, abort_flag);
                if (!__all_sync(0xffffffffu, ok)) { ab = true; break; }
                tc_fence_after();
                uint32_t words[BN / 32];
#pragma unroll
                for (int j = 0; j < WPG; j++) {
                    uint32_t v[32];
                    const int jw = g * WPG + j;   // word of the tile
                    tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN + jw * 32), v);
                    if (!CLASSIFY && p.scores && valid) {
                        const float rs = p.sx ? p.sx[row] : 1.f;
#pragma unroll
                        for (int i = 0; i < 32; i++) {
                            const int col = nt * BN + jw * 32 + i;
                            if (col < p.Dk)
                                p.scores[row * p.Dk + col] = __uint_as_float(v[i]) * rs * (p.sb ? p.sb[col] : 1.f);
                        }
                    }
                    const int col0 = nt * BN + jw * 32;
                    if (!CLASSIFY && p.sproj && valid && col0 < p.ldS) {
                        // 32 BF16 projections (zeros past Dk: the base rows
                        // there are TMA zero fill), two whole 32-byte sectors
                        float sbv[32];
                        if (p.sb && col0 + 32 <= p.Dk) {
                            const float4 *s4 = reinterpret_cast<const float4 *>(p.sb + col0);
#pragma unroll
                            for (int i = 0; i < 8; i++) {
                                const float4 t = s4[i];
                                sbv[4 * i] = t.x; sbv[4 * i + 1] = t.y; sbv[4 * i + 2] = t.z; sbv[4 * i + 3] = t.w;
                            }
                        } else {
#pragma unroll
                            for (int i = 0; i < 32; i++) sbv[i] = col0 + i < p.Dk ? (p.sb ? p.sb[col0 + i] : 1.f) : 0.f;
                        }
                        uint32_t pk[16];
#pragma unroll
                        for (int i = 0; i < 32; i += 2) {
                            const float f0 = __uint_as_float(v[i]) * sbv[i];
                            const float f1 = __uint_as_float(v[i + 1]) * sbv[i + 1];
                            const __nv_bfloat16 b0 = __float2bfloat16_rn(f0), b1 = __float2bfloat16_rn(f1);
                            const float g0 = __bfloat162float(b0), g1 = __bfloat162float(b1);
                            qsum = fmaf(g0, g0, qsum);
                            qsum = fmaf(g1, g1, qsum);
                            pk[i / 2] = (uint32_t)__bfloat16_as_ushort(b0) | ((uint32_t)__bfloat16_as_ushort(b1) << 16);
                        }
                        uint16_t *dst = p.sproj + row * (int64_t)p.ldS + col0;   // 64-byte aligned
                        st_global_v8(dst, pk);
                        st_global_v8(dst + 16, pk + 8);
                    }
                    words[j] = pack_signs(v);
                }
                tc_fence_before();
                mbar_arrive(tempty(acc));
                if (++acc == 2) { acc = 0; aphase ^= 1; }
                if (CLASSIFY && EWG > 1) {
                    // publish this warpgroup's words, then read the row's 8
                    uint32_t *sw = s_words + (size_t)wb * 8 * BM;
#pragma unroll
                    for (int j = 0; j < WPG; j++) sw[(g * WPG + j) * BM + r] = words[j];
                    mbar_arrive(wfull(wb));
                    const bool okw = mbar_wait(wfull(wb), wph, abort_flag);
                    if (!__all_sync(0xffffffffu, okw)) { ab = true; break; }
#pragma unroll
                    for (int j = 0; j < BN / 32; j++) words[j] = sw[j * BM + r];
                    if (++wb == WXB) { wb = 0; wph ^= 1; }
                }
                const int gw0 = nt * (BN / 32);
                if (CLASSIFY) {
                    // this tile's 8 words of every class, staged by the TMA
                    // producer (words past W are zero, as in the query);
                    // every lane reads the same address: broadcast
                    const bool okc = mbar_wait(cfull(cb), cph, abort_flag);
                    if (!__all_sync(0xffffffffu, okc)) { ab = true; break; }
                    const uint4 *sc = reinterpret_cast<const uint4 *>(sCls + cb * CLS_BYTES);
#pragma unroll
                    for (int c = 0; c < CMAX; c++)
                        if (c0 + c < c1) {
                            const uint4 ca = sc[2 * (c0 + c)], cc = sc[2 * (c0 + c) + 1];
                            dist[c] += __popc(words[0] ^ ca.x) + __popc(words[1] ^ ca.y) + __popc(words[2] ^ ca.z) +
                                       __popc(words[3] ^ ca.w) + __popc(words[4] ^ cc.x) + __popc(words[5] ^ cc.y) +
                                       __popc(words[6] ^ cc.z) + __popc(words[7] ^ cc.w);
                        }
                    mbar_arrive(cempty(cb));
                    if (++cb == CBUF) { cb = 0; cph ^= 1; }
                } else if (valid && p.H) {
                    uint32_t *h = p.H + row * (int64_t)p.W + gw0;
                    if (EWG == 1) {
                        if (gw0 + 4 <= p.W) *reinterpret_cast<uint4 *>(h) = make_uint4(words[0], words[1], words[2], words[3]);
                        if (gw0 + 8 <= p.W) *reinterpret_cast<uint4 *>(h + 4) = make_uint4(words[4], words[5], words[6], words[7]);
                    } else {  // this warpgroup's words only (W is a multiple of 4)
                        const int w0 = gw0 + g * WPG;
                        if (w0 + WPG <= p.W) {
#pragma unroll
                            for (int j = 0; j < WPG; j++) h[g * WPG + j] = words[j];
                        }
                    }
                }
            }
            if (!CLASSIFY && !ab && p.qn) {
                if (EWG == 1) {
                    if (valid) p.qn[row] = qsum;
                } else {  // partial norms of the warpgroups' columns, summed in order g = 0, 1, ...
                    const uint32_t par = (uint32_t)(it & 1);
                    if (g > 0) {
                        if (!mbar_wait(merge_empty, par ^ 1, abort_flag)) { ab = true; break; }
                        s_val[(g - 1) * BM + r] = __float_as_int(qsum);
                        mbar_arrive(merge_full);
                    } else {
                        if (!mbar_wait(merge_full, par, abort_flag)) { ab = true; break; }
                        float t = qsum;
#pragma unroll
                        for (int h = 0; h < EWG - 1; h++) t += __int_as_float(s_val[h * BM + r]);
                        mbar_arrive(merge_empty);
                        if (valid) p.qn[row] = t;
                    }
                }
            }
            if (CLASSIFY && !ab && NS > 1) {
                // this range's partial distances go into the tile's totals;
                // the warp whose contribution completes them (all NS ranges x
                // 4 * EWG warps) takes the arg-min of the whole tile
                if (valid) {
#pragma unroll
                    for (int c = 0; c < CMAX; c++)
                        if (c0 + c < c1) atomicAdd(p.dacc + row * p.C + c0 + c, dist[c]);
                }
                __threadfence();
                __syncwarp();
                unsigned prev = 0;
                if (lane == 0) prev = atomicAdd(p.tile_done + mt, 1u);
                prev = __shfl_sync(0xffffffffu, prev, 0);
                if (prev == (unsigned)(NS * 4 * EWG - 1)) {
                    __threadfence();
                    for (int rr = lane; rr < BM; rr += 32) {
                        const int64_t rw = mt * BM + rr;
                        if (rw >= p.N) break;
                        const volatile int32_t *dr = p.dacc + rw * p.C;
                        int best = 0, bv = 0x7fffffff;
                        for (int c = 0; c < p.C; c++) {   // ascending: ties keep the lowest class
                            const int v = dr[c];
                            if (p.dists) p.dists[rw * p.C + c] = v;
                            if (v < bv) { bv = v; best = c; }
                        }
                        p.labels[rw] = best;
                    }
                }
            } else if (CLASSIFY && !ab) {  // arg-min over this warpgroup's classes, lowest index on ties
                int best = c0, bv = 0x7fffffff;
#pragma unroll
                for (int c = 0; c < CMAX; c++)
                    if (c0 + c < c1) {
                        if (p.dists && valid) p.dists[row * p.C + c0 + c] = dist[c];
                        if (dist[c] < bv) { bv = dist[c]; best = c0 + c; }
                    }
                if (EWG > 1) {
                    const uint32_t par = (uint32_t)(it & 1);
                    if (g > 0) {
                        if (!mbar_wait(merge_empty, par ^ 1, abort_flag)) { ab = true; break; }
                        s_val[(g - 1) * BM + r] = bv;
                        s_idx[(g - 1) * BM + r] = best;
                        mbar_arrive(merge_full);
                    } else {
                        if (!mbar_wait(merge_full, par, abort_flag)) { ab = true; break; }
#pragma unroll
                        for (int h = 0; h < EWG - 1; h++) {  // ascending class ranges: ties keep the lower
                            const int v1 = s_val[h * BM + r], i1 = s_idx[h * BM + r];
                            if (v1 < bv) { bv = v1; best = i1; }
                        }
                        mbar_arrive(merge_empty);
                    }
                }
                if (g == 0 && valid) p.labels[row] = best;
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// Launch helpers, instantiated by each encoding's translation unit.
template <int ENC, int CMAX, bool CLASSIFY, int EWG, bool QIN = false>
static cudaError_t launch_one(const CUtensorMap &ma, const CUtensorMap &mb, const CUtensorMap &mc, const Params &p,
                              unsigned grid, cudaStream_t st)
{
    auto k = tc_encode_kernel<ENC, CMAX, CLASSIFY, EWG, QIN>;
    constexpr size_t smem = smem_bytes(EWG);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, num_threads(EWG, QIN), smem, st>>>(ma, mb, mc, p);
    return cudaGetLastError();
}

template <int ENC>
static cudaError_t launch_enc(const CUtensorMap &ma, const CUtensorMap &mb, const CUtensorMap &mc, const Params &p,
                              unsigned grid, bool classify, cudaStream_t st)
{
    // encode-only: packed words with one warpgroup; BF16 projections (heavier
    // epilogue) with four, each converting and storing its 64 columns
    if (!classify)
        return p.sproj ? launch_one<ENC, 1, false, 4>(ma, mb, mc, p, grid, st)
                       : launch_one<ENC, 1, false, 1>(ma, mb, mc, p, grid, st);
    if (p.X) {  // query tiles quantised in the kernel (classify, up to 32 classes)
        if (p.C <= 16) return launch_one<ENC, 16, true, 1, true>(ma, mb, mc, p, grid, st);
        if (p.C <= 32) return launch_one<ENC, 16, true, 2, true>(ma, mb, mc, p, grid, st);
        return cudaErrorNotSupported;
    }
    // up to 16 classes: one epilogue warpgroup; up to 32: two; more: four,
    // each counting ceil(C / EWG) <= CMAX classes
    if (p.C <= 16) return launch_one<ENC, 16, true, 1>(ma, mb, mc, p, grid, st);
    if (p.C <= 32) return launch_one<ENC, 16, true, 2>(ma, mb, mc, p, grid, st);
    if (p.C <= 64) return launch_one<ENC, 16, true, 4>(ma, mb, mc, p, grid, st);
    return launch_one<ENC, 32, true, 4>(ma, mb, mc, p, grid, st);
}

// Read and clear this translation unit's device status word.
static cudaError_t read_status(cudaStream_t st, int *status)
{
    int h = 0;
    cudaError_t e = cudaMemcpyFromSymbolAsync(&h, g_tc_status, sizeof(int), 0, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    *status = h;
    if (h != 0) {
        const int zero = 0;
        e = cudaMemcpyToSymbolAsync(g_tc_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    return e;
}

// Entry points of the two encoding translation units.
cudaError_t launch_bf16(const CUtensorMap &ma, const CUtensorMap &mb, const CUtensorMap &mc, const Params &p,
                        unsigned grid, bool classify, cudaStream_t st);
cudaError_t launch_fp8(const CUtensorMap &ma, const CUtensorMap &mb, const CUtensorMap &mc, const Params &p,
                       unsigned grid, bool classify, cudaStream_t st);
cudaError_t status_bf16(cudaStream_t st, int *status);
cudaError_t status_fp8(cudaStream_t st, int *status);

}  // namespace tc
}  // namespace hdc
