// Level-ID encoding (Sec. 4.2 Algorithmic Choice: ID-based encoding as the
// alternative to random projection; Sec. 5.3: Micro-HD-Classification's
// Level-ID encoder and its N_LEVELS knob).
//
//   level(x_f) = clamp(floor((x_f - lo) * scale), 0, L-1)     FP32, as written
//   s_d        = sum_f ID_f[d] * LEVEL_{level(x_f)}[d]          (+-1 elements)
//   bit_d      = s_d < 0                                        (sign(0) = +1)
// With bit 1 = element -1, the product of two elements is -1 exactly when
// their bits differ, so s_d = F - 2 cnt_d with cnt_d = #{f : id_f,d != lv_f,d}
// and bit_d = cnt_d > floor(F/2): a per-dimension majority of XORs.
//
// Level hypervectors: level l has the bit of `hi_hv` at dim d when
// l >= flip[d], else the bit of `lo_hv` (flip[d] in 1..L-1: level 0 is lo_hv,
// level L-1 is hi_hv, neighbouring levels differ in the dims that switch
// between them).  ID and level rows are compacted to the kept dims at
// model preparation, like the base rows of the random projection.
//
// Encode kernel: one block per (32 queries, 32 words); the block stages its
// word slice of every ID row and every level row in shared memory.  A warp
// takes four queries at a time (four independent counter chains, each ID
// word loaded once for the four), a lane one word (32 dims): lane j
// quantises feature f0 + j of each query, the warp broadcasts the levels by
// shuffle, and each lane adds id ^ level rows into a bit-sliced counter per
// query (carry-save adders over groups of 16 rows with the planes of weight
// 1, 2, 4 and 8 as carry-save state, then a ripple-carry add of the
// weight-16 row into planes sized for F), then compares the counter against
// floor(F/2) bit-sliced.  The next 32 features of each query are loaded
// while the current ones are counted.
#include <cmath>
#include <cstring>

#include "bitslice.cuh"
#include "hdc_internal.cuh"

namespace hdc {
namespace {

constexpr int LQ = 32;       // queries per block
constexpr int LWC = 32;      // words per block (one per lane)
constexpr int LWARPS = 8;
// counter planes of weight 16, 32, ...: HP of them hold floor(F / 16) < 2^HP
__host__ __device__ constexpr int hp_for(int F) { return F < 1024 ? 6 : 9; }

__device__ __forceinline__ int quant_level(float x, float lo, float scale, int L)
{
    // separate FP32 rounding of the difference and the product (no FMA), as the oracle
    const float t = __fmul_rn(__fsub_rn(x, lo), scale);
    if (t >= (float)L) return L - 1;
    if (t > 0.f) return (int)t;  // floor of a positive value
    return 0;                    // t <= 0, or NaN
}

// The counter of one query and lane: planes c1, c2, c4, c8 (weights 1, 2,
// 4, 8) and hp[k] (weight 16 * 2^k); bit position i of the planes spells
// the count of dim i in binary.
template <int HP>
struct Counter {
    uint32_t c1, c2, c4, c8, hp[HP];
};

// Add 16 rows of weight 1: a carry-save tree (15 full adders) to one row of
// weight 16, then a ripple-carry add of it into hp.
template <int HP>
__device__ __forceinline__ void add16(Counter<HP> &k, const uint32_t (&r)[16])
{
    uint32_t c = csa16(k.c1, k.c2, k.c4, k.c8, r);
#pragma unroll
    for (int i = 0; i < HP; i++) {
        const uint32_t t = k.hp[i] & c;
        k.hp[i] ^= c;
        c = t;
    }
}

// Add one row of weight 1 (ripple carry through every plane).
template <int HP>
__device__ __forceinline__ void add1(Counter<HP> &k, uint32_t c)
{
    uint32_t t = k.c1 & c; k.c1 ^= c; c = t;
    t = k.c2 & c; k.c2 ^= c; c = t;
    t = k.c4 & c; k.c4 ^= c; c = t;
    t = k.c8 & c; k.c8 ^= c; c = t;
#pragma unroll
    for (int i = 0; i < HP; i++) {
        const uint32_t u = k.hp[i] & c;
        k.hp[i] ^= c;
        c = u;
    }
}

// count > T per bit position, from the most significant plane down.
template <int HP>
__device__ __forceinline__ uint32_t greater(const Counter<HP> &k, uint32_t T)
{
    uint32_t gt = 0, eq = 0xffffffffu;
#pragma unroll
    for (int i = HP - 1; i >= 0; i--) {
        const uint32_t cp = k.hp[i];
        if ((T >> (i + 4)) & 1u) eq &= cp;
        else { gt |= eq & cp; eq &= ~cp; }
    }
    const uint32_t pl[4] = {k.c8, k.c4, k.c2, k.c1};
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const uint32_t cp = pl[i];
        if ((T >> (3 - i)) & 1u) eq &= cp;
        else { gt |= eq & cp; eq &= ~cp; }
    }
    return gt;
}

// A warp encodes QW queries at once (independent counter chains; each ID
// word loaded once for all of them).
constexpr int QW = 4;
// per warp: the level-row offsets (level x LWC words) of its QW queries'
// current 32 features, read back 16 at a time as broadcasts
constexpr size_t LOFF_BYTES = (size_t)LWARPS * QW * 32 * 4;

template <int HP>
__global__ void __launch_bounds__(LWARPS * 32) levelid_encode_kernel(const float *__restrict__ X, int64_t N, int F,
                                                                   int L, int W, float lo, float scale,
                                                                   const uint32_t *__restrict__ id,
                                                                   const uint32_t *__restrict__ lv,
                                                                   uint32_t *__restrict__ H)
{
    extern __shared__ uint32_t lsm[];
    uint32_t *sid = lsm;                          // F x LWC
    uint32_t *slv = lsm + (size_t)F * LWC;        // L x LWC
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int *soff = reinterpret_cast<int *>(lsm + (size_t)(F + L) * LWC) + warp * (QW * 32);   // [QW][32]
    const int w0 = blockIdx.y * LWC;
    const int nw = min(LWC, W - w0);
    for (int i = threadIdx.x; i < F * LWC; i += blockDim.x) {
        const int f = i / LWC, j = i % LWC;
        sid[i] = j < nw ? id[(int64_t)f * W + w0 + j] : 0u;
    }
    for (int i = threadIdx.x; i < L * LWC; i += blockDim.x) {
        const int l = i / LWC, j = i % LWC;
        slv[i] = j < nw ? lv[(int64_t)l * W + w0 + j] : 0u;
    }
    __syncthreads();
    const uint32_t T = (uint32_t)F >> 1;
    for (int qb = warp * QW; qb < LQ; qb += LWARPS * QW) {
        const int64_t q0 = (int64_t)blockIdx.x * LQ + qb;
        if (q0 >= N) break;                       // warp-uniform
        Counter<HP> cnt[QW];
#pragma unroll
        for (int a = 0; a < QW; a++) {
            cnt[a].c1 = cnt[a].c2 = cnt[a].c4 = cnt[a].c8 = 0;
#pragma unroll
            for (int k = 0; k < HP; k++) cnt[a].hp[k] = 0;
        }
        // feature f0 + lane of each query, loaded one 32-feature batch ahead
        // so the quantisation does not wait on device memory
        float xn[QW];
#pragma unroll
        for (int a = 0; a < QW; a++) xn[a] = (lane < F && q0 + a < N) ? X[(q0 + a) * (int64_t)F + lane] : 0.f;
        for (int f0 = 0; f0 < F; f0 += 32) {
            const int f = f0 + lane;
            // level-row offset of feature f of each query (rows past N: level 0, not stored)
#pragma unroll
            for (int a = 0; a < QW; a++) {
                soff[a * 32 + lane] = (f < F && q0 + a < N) ? quant_level(xn[a], lo, scale, L) * LWC : 0;
                const int fn = f + 32;
                xn[a] = (fn < F && q0 + a < N) ? X[(q0 + a) * (int64_t)F + fn] : 0.f;
            }
            __syncwarp();
            const int nf = min(32, F - f0);
            int j = 0;
            for (; j + 16 <= nf; j += 16) {
                uint32_t idw[16];
#pragma unroll
                for (int u = 0; u < 16; u++) idw[u] = sid[(f0 + j + u) * LWC + lane];
#pragma unroll
                for (int a = 0; a < QW; a++) {
                    int o[16];   // four 16-byte broadcasts (j is a multiple of 16)
                    const int4 *o4 = reinterpret_cast<const int4 *>(soff + a * 32 + j);
#pragma unroll
                    for (int v = 0; v < 4; v++) {
                        const int4 t = o4[v];
                        o[4 * v] = t.x; o[4 * v + 1] = t.y; o[4 * v + 2] = t.z; o[4 * v + 3] = t.w;
                    }
                    uint32_t r[16];
#pragma unroll
                    for (int u = 0; u < 16; u++) r[u] = idw[u] ^ slv[o[u] + lane];
                    add16(cnt[a], r);
                }
            }
            for (; j < nf; j++) {
                const uint32_t idw = sid[(f0 + j) * LWC + lane];
#pragma unroll
                for (int a = 0; a < QW; a++) add1(cnt[a], idw ^ slv[soff[a * 32 + j] + lane]);
            }
            __syncwarp();   // the batch's offsets are read before the next batch writes them
        }
#pragma unroll
        for (int a = 0; a < QW; a++)
            if (q0 + a < N && lane < nw)
                H[(q0 + a) * (int64_t)W + w0 + lane] = greater(cnt[a], T);
    }
}

// Model preparation: one thread per output word of the compacted rows,
// packing the caller's unpacked bytes (nonzero = the element -1) of the
// kept dims d = s0 + k*stride.
//   rows [0, F):      ID row f (id_bits: F x D bytes)
//   rows [F, F + L):  level l, bit d = l >= flip[d] ? hi[d] : lo[d]
__global__ void levelid_prepare_kernel(const uint8_t *__restrict__ id_bits, const uint8_t *__restrict__ lo_bits,
                                       const uint8_t *__restrict__ hi_bits, const int32_t *__restrict__ flip, int F,
                                       int L, int64_t D, int64_t s0, int64_t stride, int64_t Dk, int Wk,
                                       uint32_t *__restrict__ id, uint32_t *__restrict__ lv)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)(F + L) * Wk) return;
    const int r = (int)(i / Wk), kw = (int)(i % Wk);
    uint32_t word = 0;
    for (int j = 0; j < 32; j++) {
        const int64_t k = (int64_t)kw * 32 + j;
        if (k >= Dk) break;
        const int64_t d = s0 + k * stride;
        uint8_t b;
        if (r < F) {
            b = id_bits[(int64_t)r * D + d];
        } else {
            const int l = r - F;
            b = l >= flip[d] ? hi_bits[d] : lo_bits[d];
        }
        word |= (uint32_t)(b != 0) << j;
    }
    if (r < F) id[(int64_t)r * Wk + kw] = word;
    else lv[(int64_t)(r - F) * Wk + kw] = word;
}

__global__ void flip_check_kernel(const int32_t *__restrict__ flip, int D, int L, int *__restrict__ bad)
{
    for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < D; d += gridDim.x * blockDim.x)
        if (flip[d] < 1 || flip[d] > L - 1) atomicOr(bad, 1);
}

struct LevelLayout {
    size_t id, lv, total;
};

LevelLayout level_layout(int F, int L, int Wk)
{
    LevelLayout Ly;
    size_t off = 0;
    Ly.id = off; off = align_up(off + (size_t)F * Wk * 4, kAlign);
    Ly.lv = off; off = align_up(off + (size_t)L * Wk * 4, kAlign);
    Ly.total = off;
    return Ly;
}

size_t encode_smem(int F, int L) { return (size_t)(F + L) * LWC * 4; }

}  // namespace
}  // namespace hdc

using namespace hdc;

extern "C" hdc_status hdc_levelid_model_bytes(int32_t F, int32_t D, int32_t L, const hdc_approx_config *cfg,
                                              size_t *bytes)
{
    Perf p;
    if (!bytes || F <= 0 || D <= 0 || L < 2 || (cfg && cfg->struct_size < sizeof(hdc_approx_config)) ||
        !perf_of(D, cfg, &p))
        return HDC_ERR_INVALID_ARG;
    if (F >= 8 * 1024 || encode_smem(F, L) > 200 * 1024) return HDC_ERR_UNSUPPORTED;
    *bytes = level_layout(F, L, words_for(p.Dk)).total;
    return HDC_OK;
}

extern "C" hdc_status hdc_levelid_prepare(const uint8_t *id_bits, const uint8_t *lo_bits, const uint8_t *hi_bits,
                                          const int32_t *flip, int32_t F, int32_t D, int32_t L, float x_lo,
                                          float x_hi, const hdc_approx_config *cfg, void *buf, size_t buf_bytes,
                                          int32_t *flip_error, hdc_levelid_model *out, hdc_stream_t stream)
{
    size_t need = 0;
    hdc_status s = hdc_levelid_model_bytes(F, D, L, cfg, &need);
    if (s != HDC_OK) return s;
    if (!id_bits || !lo_bits || !hi_bits || !flip || !out || !buf || ((uintptr_t)buf % kAlign) != 0 ||
        !(x_hi > x_lo) || !std::isfinite(x_lo) || !std::isfinite(x_hi))
        return HDC_ERR_INVALID_ARG;
    if (buf_bytes < need) return HDC_ERR_WORKSPACE;
    Perf p;
    perf_of(D, cfg, &p);
    const int Wk = words_for(p.Dk);
    const LevelLayout Ly = level_layout(F, L, Wk);
    cudaStream_t st = (cudaStream_t)stream;
    char *b = (char *)buf;
    if (flip_error) {
        if (cudaMemsetAsync(flip_error, 0, sizeof(int32_t), st) != cudaSuccess) return HDC_ERR_CUDA;
        flip_check_kernel<<<(D + 255) / 256 < 1024 ? (D + 255) / 256 : 1024, 256, 0, st>>>(flip, D, L, flip_error);
        if (cudaGetLastError() != cudaSuccess) return HDC_ERR_CUDA;
    }
    const int64_t n = (int64_t)(F + L) * Wk;
    levelid_prepare_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        id_bits, lo_bits, hi_bits, flip, F, L, (int64_t)D, p.s0, p.stride, p.Dk, Wk, (uint32_t *)(b + Ly.id),
        (uint32_t *)(b + Ly.lv));
    if (cudaGetLastError() != cudaSuccess) return HDC_ERR_CUDA;
    hdc_levelid_model m;
    memset(&m, 0, sizeof(m));
    m.struct_size = sizeof(m);
    m.F = F;
    m.D = D;
    m.Dk = (int32_t)p.Dk;
    m.L = L;
    m.W = Wk;
    m.lo = x_lo;
    m.scale = (float)((double)L / ((double)x_hi - (double)x_lo));
    m.id = (const uint32_t *)(b + Ly.id);
    m.level = (const uint32_t *)(b + Ly.lv);
    *out = m;
    return HDC_OK;
}

extern "C" hdc_status hdc_levelid_encode(const float *X, int64_t N, const hdc_levelid_model *m, uint32_t *H,
                                         hdc_stream_t stream)
{
    if (N < 0 || !m || m->struct_size < sizeof(hdc_levelid_model) || m->F <= 0 || m->L < 2 || m->Dk <= 0 ||
        m->W != words_for(m->Dk) || !m->id || !m->level || encode_smem(m->F, m->L) > 200 * 1024 || m->F >= 8 * 1024)
        return HDC_ERR_INVALID_ARG;
    if (N == 0) return HDC_OK;
    if (!X || !H) return HDC_ERR_INVALID_ARG;
    const size_t smem = encode_smem(m->F, m->L) + LOFF_BYTES;
    // counter planes for floor(F / 16) (F < 8192: at most 9)
    auto k = hp_for(m->F) == 6 ? levelid_encode_kernel<6> : levelid_encode_kernel<9>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return HDC_ERR_CUDA;
    const dim3 grid((unsigned)((N + LQ - 1) / LQ), (unsigned)((m->W + LWC - 1) / LWC));
    if (grid.y > 65535) return HDC_ERR_UNSUPPORTED;
    k<<<grid, LWARPS * 32, smem, (cudaStream_t)stream>>>(X, N, m->F, m->L, m->W, m->lo, m->scale, m->id, m->level, H);
    return cudaGetLastError() == cudaSuccess ? HDC_OK : HDC_ERR_CUDA;
}
