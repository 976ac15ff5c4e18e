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
// query (carry-save adders over groups of 8 rows, then a ripple-carry add of
// the weight-8 plane), then compares the counter against floor(F/2)
// bit-sliced.
#include <cmath>
#include <cstring>

#include "hdc_internal.cuh"

namespace hdc {
namespace {

constexpr int LQ = 32;       // queries per block
constexpr int LWC = 32;      // words per block (one per lane)
constexpr int LWARPS = 8;
constexpr int HPLANES = 10;  // counter planes of weight 8, 16, ...: F < 8 * 2^10

__device__ __forceinline__ void csa(uint32_t &h, uint32_t &l, uint32_t a, uint32_t b, uint32_t c)
{
    // full adder per bit position: l = a ^ b ^ c (weight 1), h = majority (weight 2)
    const uint32_t u = a ^ b;
    h = (a & b) | (u & c);
    l = u ^ c;
}

__device__ __forceinline__ int quant_level(float x, float lo, float scale, int L)
{
    // separate FP32 rounding of the difference and the product (no FMA), as the oracle
    const float t = __fmul_rn(__fsub_rn(x, lo), scale);
    if (t >= (float)L) return L - 1;
    if (t > 0.f) return (int)t;  // floor of a positive value
    return 0;                    // t <= 0, or NaN
}

// Add 8 rows of weight 1 into the counter (ones, twos, fours, hp): a
// carry-save tree to one row of weight 8, then a ripple-carry add of it.
__device__ __forceinline__ void add8(uint32_t &ones, uint32_t &twos, uint32_t &fours, uint32_t (&hp)[HPLANES],
                                     const uint32_t (&r)[8])
{
    uint32_t t2a, t2b, t4a, t4b, e8;
    csa(t2a, ones, ones, r[0], r[1]);
    csa(t2b, ones, ones, r[2], r[3]);
    csa(t4a, twos, twos, t2a, t2b);
    csa(t2a, ones, ones, r[4], r[5]);
    csa(t2b, ones, ones, r[6], r[7]);
    csa(t4b, twos, twos, t2a, t2b);
    csa(e8, fours, fours, t4a, t4b);
    uint32_t c = e8;
#pragma unroll
    for (int k = 0; k < HPLANES; k++) {
        const uint32_t t = hp[k] & c;
        hp[k] ^= c;
        c = t;
    }
}

// Add one row of weight 1 (ripple carry through every plane).
__device__ __forceinline__ void add1(uint32_t &ones, uint32_t &twos, uint32_t &fours, uint32_t (&hp)[HPLANES],
                                     uint32_t c)
{
    uint32_t t = ones & c; ones ^= c; c = t;
    t = twos & c; twos ^= c; c = t;
    t = fours & c; fours ^= c; c = t;
#pragma unroll
    for (int k = 0; k < HPLANES; k++) {
        const uint32_t u = hp[k] & c;
        hp[k] ^= c;
        c = u;
    }
}

// cnt > T per bit position, from the most significant plane down.
__device__ __forceinline__ uint32_t greater(uint32_t ones, uint32_t twos, uint32_t fours,
                                            const uint32_t (&hp)[HPLANES], uint32_t T)
{
    uint32_t gt = 0, eq = 0xffffffffu;
#pragma unroll
    for (int k = HPLANES - 1; k >= 0; k--) {
        const uint32_t cp = hp[k];
        if ((T >> (k + 3)) & 1u) eq &= cp;
        else { gt |= eq & cp; eq &= ~cp; }
    }
    const uint32_t pl[3] = {fours, twos, ones};
#pragma unroll
    for (int k = 2; k >= 0; k--) {
        const uint32_t cp = pl[2 - k];
        if ((T >> k) & 1u) eq &= cp;
        else { gt |= eq & cp; eq &= ~cp; }
    }
    return gt;
}

// A warp encodes QW queries at once (independent counter chains; each ID
// word loaded once for all of them).
constexpr int QW = 4;

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
        uint32_t ones[QW], twos[QW], fours[QW], hp[QW][HPLANES];
#pragma unroll
        for (int a = 0; a < QW; a++) {
            ones[a] = twos[a] = fours[a] = 0;
#pragma unroll
            for (int k = 0; k < HPLANES; k++) hp[a][k] = 0;
        }
        for (int f0 = 0; f0 < F; f0 += 32) {
            const int f = f0 + lane;
            int my[QW];   // level of feature f of each query (rows past N: level 0, not stored)
#pragma unroll
            for (int a = 0; a < QW; a++)
                my[a] = (f < F && q0 + a < N) ? quant_level(X[(q0 + a) * (int64_t)F + f], lo, scale, L) : 0;
            const int nf = min(32, F - f0);
            int j = 0;
            for (; j + 8 <= nf; j += 8) {
                uint32_t idw[8];
#pragma unroll
                for (int u = 0; u < 8; u++) idw[u] = sid[(f0 + j + u) * LWC + lane];
#pragma unroll
                for (int a = 0; a < QW; a++) {
                    uint32_t r[8];
#pragma unroll
                    for (int u = 0; u < 8; u++) {
                        const int l = __shfl_sync(0xffffffffu, my[a], j + u);
                        r[u] = idw[u] ^ slv[l * LWC + lane];
                    }
                    add8(ones[a], twos[a], fours[a], hp[a], r);
                }
            }
            for (; j < nf; j++) {
                const uint32_t idw = sid[(f0 + j) * LWC + lane];
#pragma unroll
                for (int a = 0; a < QW; a++) {
                    const int l = __shfl_sync(0xffffffffu, my[a], j);
                    add1(ones[a], twos[a], fours[a], hp[a], idw ^ slv[l * LWC + lane]);
                }
            }
        }
#pragma unroll
        for (int a = 0; a < QW; a++)
            if (q0 + a < N && lane < nw)
                H[(q0 + a) * (int64_t)W + w0 + lane] = greater(ones[a], twos[a], fours[a], hp[a], T);
    }
}

// Model preparation: one thread per output word of the compacted rows.
//   rows [0, F):      ID row f, kept dims gathered from id_bits (W(D) words per row)
//   rows [F, F + L):  level l, bit d = l >= flip[d] ? hi[d] : lo[d]
__global__ void levelid_prepare_kernel(const uint32_t *__restrict__ id_bits, const uint32_t *__restrict__ lo_hv,
                                       const uint32_t *__restrict__ hi_hv, const int32_t *__restrict__ flip, int F,
                                       int L, int WD, int64_t s0, int64_t stride, int64_t Dk, int Wk,
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
        uint32_t bit;
        if (r < F) {
            bit = (id_bits[(int64_t)r * WD + (d >> 5)] >> (d & 31)) & 1u;
        } else {
            const int l = r - F;
            const uint32_t *src = l >= flip[d] ? hi_hv : lo_hv;
            bit = (src[d >> 5] >> (d & 31)) & 1u;
        }
        word |= bit << j;
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

extern "C" hdc_status hdc_levelid_prepare(const uint32_t *id_bits, const uint32_t *lo_hv, const uint32_t *hi_hv,
                                          const int32_t *flip, int32_t F, int32_t D, int32_t L, float x_lo,
                                          float x_hi, const hdc_approx_config *cfg, void *buf, size_t buf_bytes,
                                          int32_t *flip_error, hdc_levelid_model *out, hdc_stream_t stream)
{
    size_t need = 0;
    hdc_status s = hdc_levelid_model_bytes(F, D, L, cfg, &need);
    if (s != HDC_OK) return s;
    if (!id_bits || !lo_hv || !hi_hv || !flip || !out || !buf || ((uintptr_t)buf % kAlign) != 0 ||
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
        id_bits, lo_hv, hi_hv, flip, F, L, words_for(D), p.s0, p.stride, p.Dk, Wk, (uint32_t *)(b + Ly.id),
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
    const size_t smem = encode_smem(m->F, m->L);
    if (cudaFuncSetAttribute(levelid_encode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return HDC_ERR_CUDA;
    const dim3 grid((unsigned)((N + LQ - 1) / LQ), (unsigned)((m->W + LWC - 1) / LWC));
    if (grid.y > 65535) return HDC_ERR_UNSUPPORTED;
    levelid_encode_kernel<<<grid, LWARPS * 32, smem, (cudaStream_t)stream>>>(X, N, m->F, m->L, m->W, m->lo, m->scale,
                                                                            m->id, m->level, H);
    return cudaGetLastError() == cudaSuccess ? HDC_OK : HDC_ERR_CUDA;
}
