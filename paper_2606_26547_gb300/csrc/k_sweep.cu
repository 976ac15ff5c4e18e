// K7: batched evaluation of approximation configurations (the candidate
// evaluations of the paper's tuning loop, Sec. 3, done in one launch).
//
// For one trained model: validation hypervectors H (N x W words, encoded
// once at the full D) are scored under every (class width b, perforation
// entry (s0, e0, s)) pair.  Strides are powers of two <= 32, so the kept
// dims of an entry inside any word are the bits at positions = s0 (mod s):
// one constant mask per entry (0x55555555 << (s0 mod 2) for s = 2, ...),
// cleared below s0 in the first word and from e0 on in the last, and the
// configurations share every load.
//   b = 1       Hamming over the stride's dims          -> arg-min
//   b = 4, 8    cosine with b-bit class values (planes) -> arg-max
//   b = 0       cosine with the int32 accumulators themselves (32 planes)
// The b-bit quantisation, the sums and the norms are those of hdc_classify
// (per class over the full D; sums and norms over each stride's dims), so
// every configuration's predictions equal hdc_classify's.
#include <math.h>

#include "hdc_internal.cuh"

namespace hdc {
namespace {

constexpr int MAXS = HDC_SWEEP_MAX_STRIDES;
constexpr int MAXB = HDC_SWEEP_MAX_BITS;

struct SweepConf {
    int ns, nb;
    int stride[MAXS];
    uint32_t mask[MAXS];    // kept bit positions inside a word
    int64_t s0[MAXS];       // first kept dim of each entry
    int sw[MAXS];           // word holding s0
    uint32_t shead[MAXS];   // bits of word sw at or above s0
    int64_t e0[MAXS];       // end dim (exclusive) of each entry
    int ew[MAXS];           // words fully below e0
    uint32_t etail[MAXS];   // kept bits of word ew (below e0)
    int bits[MAXB];
    int planes[MAXB];       // planes of each width
    int plane_off[MAXB];    // first plane of each width in the plane array
    int total_planes;
};

__host__ __device__ inline int nplanes(int b) { return b == 0 ? 32 : b; }

// value of a class element under width b (b = 0: the accumulator itself)
__device__ __forceinline__ long long class_value(long long a, int b, long long M)
{
    if (b == 0) return a;
    if (b == 1) return a < 0 ? -1 : 1;
    if (M == 0) return 0;
    const long long Q = (1ll << (b - 1)) - 1;
    const long long mag = a < 0 ? -a : a;
    const long long r = (2 * mag * Q + M) / (2 * M);
    return a < 0 ? -r : r;
}

// One block per class: planes of every width over all D dims, and per
// (width, stride) the sum and the norm of the class values over the
// stride's dims.
__global__ void __launch_bounds__(256) sweep_prep_kernel(const int32_t *__restrict__ acc, int D, int C, int W,
                                                         SweepConf cf, uint32_t *__restrict__ planes,
                                                         long long *__restrict__ sums, double *__restrict__ norms)
{
    __shared__ long long s_max;
    __shared__ long long s_sum[MAXB * MAXS], s_sq[MAXB * MAXS];
    const int c = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int32_t *a = acc + (int64_t)c * D;
    if (threadIdx.x == 0) s_max = 0;
    if (threadIdx.x < MAXB * MAXS) { s_sum[threadIdx.x] = 0; s_sq[threadIdx.x] = 0; }
    __syncthreads();
    long long m = 0;
    for (int d = threadIdx.x; d < D; d += blockDim.x) {
        const long long v = a[d];
        m = max(m, v < 0 ? -v : v);
    }
    atomicMax(&s_max, m);
    __syncthreads();
    const long long M = s_max;
    long long lsum[MAXB * MAXS], lsq[MAXB * MAXS];
#pragma unroll
    for (int k = 0; k < MAXB * MAXS; k++) { lsum[k] = 0; lsq[k] = 0; }
    for (int w = warp; w < W; w += nw) {
        const int d = w * 32 + lane;
        const bool valid = d < D;
        const long long x = valid ? (long long)a[d] : 0;
#pragma unroll
        for (int j = 0; j < MAXB; j++) {
            if (j >= cf.nb) break;
            const int b = cf.bits[j];
            const long long v = valid ? class_value(x, b, M) : 0;
            for (int p = 0; p < cf.planes[j]; p++) {
                const bool bit = b == 1 ? v < 0 : ((v >> p) & 1) != 0;
                const unsigned bal = __ballot_sync(0xffffffffu, valid && bit);
                if (lane == 0) planes[((int64_t)(cf.plane_off[j] + p) * C + c) * W + w] = bal;
            }
#pragma unroll
            for (int i = 0; i < MAXS; i++)
                if (i < cf.ns && valid && d >= cf.s0[i] && (d - cf.s0[i]) % cf.stride[i] == 0 && d < cf.e0[i]) {
                    lsum[j * MAXS + i] += v;
                    lsq[j * MAXS + i] += v * v;
                }
        }
    }
#pragma unroll
    for (int k = 0; k < MAXB * MAXS; k++) {
        long long s = lsum[k], q = lsq[k];
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, o);
            q += __shfl_xor_sync(0xffffffffu, q, o);
        }
        if (lane == 0 && (s || q)) {
            atomicAdd((unsigned long long *)&s_sum[k], (unsigned long long)s);
            atomicAdd((unsigned long long *)&s_sq[k], (unsigned long long)q);
        }
    }
    __syncthreads();
    if (threadIdx.x < MAXB * MAXS) {
        const int j = threadIdx.x / MAXS, i = threadIdx.x % MAXS;
        if (j < cf.nb && i < cf.ns) {
            sums[((int64_t)j * cf.ns + i) * C + c] = s_sum[threadIdx.x];
            norms[((int64_t)j * cf.ns + i) * C + c] = sqrt((double)s_sq[threadIdx.x]);
        }
    }
}

// Per-stride sums over one chunk of words for a class with NP planes
// (NP = 1: Hamming, popc(q ^ c); NP = 4, 8: b-bit cosine, popc(q & plane)
// weighted 2^p, the top plane negative).  Counts stay int32 per (plane,
// stride) and are weighted once per chunk.
// Mask of entry i for global word w: the entry's bit pattern, cut below s0
// and from e0 on.
__device__ __forceinline__ uint32_t entry_mask(const SweepConf &cf, int i, int w)
{
    uint32_t m = (w < cf.sw[i] || w > cf.ew[i]) ? 0u : cf.mask[i];
    if (w == cf.sw[i]) m &= cf.shead[i];
    if (w == cf.ew[i]) m &= cf.etail[i];
    return m;
}

template <int NP>
__device__ __forceinline__ void chunk_counts(const uint32_t *sq, int QLD, int tid, const uint32_t *spc,
                                             int pstride, int nw, int w0, const SweepConf &cf, long long *out)
{
    int cnt[NP][MAXS];
#pragma unroll
    for (int p = 0; p < NP; p++)
#pragma unroll
        for (int i = 0; i < MAXS; i++) cnt[p][i] = 0;
    for (int j = 0; j < nw; j++) {
        const uint32_t qw = sq[(size_t)j * QLD + tid];
        uint32_t m[MAXS];
#pragma unroll
        for (int i = 0; i < MAXS; i++) m[i] = i < cf.ns ? entry_mask(cf, i, w0 + j) : 0u;
#pragma unroll
        for (int p = 0; p < NP; p++) {
            const uint32_t cw = spc[(size_t)p * pstride + j];
            const uint32_t x = NP == 1 ? qw ^ cw : qw & cw;
#pragma unroll
            for (int i = 0; i < MAXS; i++)
                if (i < cf.ns) cnt[p][i] += __popc(x & m[i]);
        }
    }
#pragma unroll
    for (int i = 0; i < MAXS; i++) {
        long long s = 0;
#pragma unroll
        for (int p = 0; p < NP; p++)
            s += NP == 1 ? (long long)cnt[p][i]
                         : (p == NP - 1 ? -((long long)cnt[p][i] << p) : ((long long)cnt[p][i] << p));
        out[i] = s;
    }
}

// One query per thread.  Shared memory: the chunk's query words [WCH][TPB+1],
// the chunk's class planes [planes][C][WCH], and the per-(config, class)
// partial sums [ns*C][TPB] (int64) of the block's class width.
__global__ void sweep_eval_kernel(const uint32_t *__restrict__ H, const int32_t *__restrict__ y, int64_t N, int C,
                                  int W, int WCH, SweepConf cf, const uint32_t *__restrict__ planes,
                                  const long long *__restrict__ sums, const double *__restrict__ norms,
                                  int32_t *__restrict__ correct, int32_t *__restrict__ labels)
{
    // blockIdx.y = class-width entry jb: blocks of different widths share
    // the query words through L2 and run side by side
    extern __shared__ __align__(16) uint8_t sm[];
    const int TPB = blockDim.x, tid = threadIdx.x;
    const int jb = blockIdx.y;
    const int np = cf.planes[jb], p0 = cf.plane_off[jb];
    const int ns = cf.ns;
    long long *accs = reinterpret_cast<long long *>(sm);                         // ns*C x TPB
    const int QLD = TPB + 1;  // padded: conflict-free stores and loads
    uint32_t *sq = reinterpret_cast<uint32_t *>(accs + (size_t)ns * C * TPB);      // WCH x QLD
    uint32_t *sp = sq + (size_t)WCH * QLD;                                       // np x C x WCH
    const int64_t row = (int64_t)blockIdx.x * TPB + tid;
    const bool valid = row < N;
    for (int k = 0; k < ns * C; k++) accs[(size_t)k * TPB + tid] = 0;

    for (int w0 = 0; w0 < W; w0 += WCH) {
        const int nw = min(WCH, W - w0);
        __syncthreads();
        // query words: coalesced over each row's chunk, stored [word][thread]
        for (int i = tid; i < TPB * WCH; i += TPB) {
            const int r = i / WCH, j = i % WCH;
            const int64_t gr = (int64_t)blockIdx.x * TPB + r;
            sq[(size_t)j * QLD + r] = (gr < N && j < nw) ? H[gr * W + w0 + j] : 0u;
        }
        for (int i = tid; i < np * C * WCH; i += TPB) {
            const int pc = i / WCH, j = i % WCH;
            sp[i] = j < nw ? planes[((int64_t)p0 * C + pc) * W + w0 + j] : 0u;
        }
        __syncthreads();
        for (int c = 0; c < C; c++) {
            long long part[MAXS];
            const uint32_t *spc = sp + (size_t)c * WCH;
            if (np == 1) {
                chunk_counts<1>(sq, QLD, tid, spc, C * WCH, nw, w0, cf, part);
            } else if (np == 4) {
                chunk_counts<4>(sq, QLD, tid, spc, C * WCH, nw, w0, cf, part);
            } else if (np == 8) {
                chunk_counts<8>(sq, QLD, tid, spc, C * WCH, nw, w0, cf, part);
            } else {  // unquantised accumulators: 32 planes, int64 weights
#pragma unroll
                for (int i = 0; i < MAXS; i++) part[i] = 0;
                for (int j = 0; j < nw; j++) {
                    const uint32_t qw = sq[(size_t)j * QLD + tid];
                    for (int p = 0; p < np; p++) {
                        const uint32_t x = qw & sp[((size_t)p * C + c) * WCH + j];
                        const long long wp = p == np - 1 ? -(1ll << p) : (1ll << p);
#pragma unroll
                        for (int i = 0; i < MAXS; i++)
                            if (i < ns) part[i] += wp * __popc(x & entry_mask(cf, i, w0 + j));
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < MAXS; i++)
                if (i < ns) accs[((size_t)i * C + c) * TPB + tid] += part[i];
        }
    }
    // arg-min / arg-max per stride, counts of correct predictions
    const int lane = tid & 31;
    const int yv = valid ? y[row] : -1;
    for (int i = 0; i < ns; i++) {
        const int k = jb * ns + i;
        int best = 0;
        if (cf.bits[jb] == 1) {
            long long bv = accs[((size_t)i * C) * TPB + tid];
            for (int c = 1; c < C; c++) {
                const long long v = accs[((size_t)i * C + c) * TPB + tid];
                if (v < bv) { bv = v; best = c; }
            }
        } else {
            double bs = 0.0;
            for (int c = 0; c < C; c++) {
                const double nrm = norms[(int64_t)k * C + c];
                const double sc = nrm == 0.0 ? 0.0
                                             : (double)(sums[(int64_t)k * C + c] -
                                                        2 * accs[((size_t)i * C + c) * TPB + tid]) / nrm;
                if (c == 0 || sc > bs) { bs = sc; best = c; }
            }
        }
        if (valid && labels) labels[(int64_t)k * N + row] = best;
        const unsigned hit = __ballot_sync(0xffffffffu, valid && best == yv);
        if (lane == 0 && hit) atomicAdd(correct + k, __popc(hit));
    }
}

bool is_pow2_le32(int s) { return s >= 1 && s <= 32 && (s & (s - 1)) == 0; }

bool make_conf(const hdc_sweep_spec *sp, int64_t D, SweepConf *cf)
{
    if (!sp || sp->struct_size < sizeof(hdc_sweep_spec)) return false;
    if (sp->n_strides < 1 || sp->n_strides > MAXS || sp->n_bits < 1 || sp->n_bits > MAXB) return false;
    cf->ns = sp->n_strides;
    cf->nb = sp->n_bits;
    for (int i = 0; i < MAXS; i++) {
        cf->stride[i] = 1;
        cf->mask[i] = 0;
        cf->s0[i] = 0;
        cf->sw[i] = 0;
        cf->shead[i] = 0;
        cf->e0[i] = D;
        cf->ew[i] = 0;
        cf->etail[i] = 0;
    }
    for (int i = 0; i < cf->ns; i++) {
        const int s = sp->strides[i];
        if (!is_pow2_le32(s)) return false;
        // start and end of entry i: floor(fraction * D) formed in double, as
        // for hdc_classify
        const float start = sp->starts[i], end = sp->ends[i];
        if (!(start >= 0.f) || !(start < 1.f) || !(end >= 0.f) || end > 1.f) return false;
        const int64_t s0 = (int64_t)floor((double)start * (double)D);
        const int64_t e0 = end == 0.f ? D : (int64_t)floor((double)end * (double)D);
        if (e0 <= s0) return false;  // keeps at least dim s0
        uint32_t m = 0;
        for (int b = (int)(s0 % s); b < 32; b += s) m |= 1u << b;
        cf->stride[i] = s;
        cf->mask[i] = m;
        cf->s0[i] = s0;
        cf->sw[i] = (int)(s0 >> 5);
        cf->shead[i] = ~0u << (s0 & 31);
        cf->e0[i] = e0;
        cf->ew[i] = (int)(e0 >> 5);
        cf->etail[i] = (1u << (e0 & 31)) - 1u;
    }
    int off = 0;
    for (int j = 0; j < MAXB; j++) { cf->bits[j] = 1; cf->planes[j] = 0; cf->plane_off[j] = 0; }
    for (int j = 0; j < cf->nb; j++) {
        const int b = sp->bits[j];
        if (b != 0 && b != 1 && b != 4 && b != 8) return false;
        cf->bits[j] = b;
        cf->planes[j] = nplanes(b);
        cf->plane_off[j] = off;
        off += nplanes(b);
    }
    cf->total_planes = off;
    return true;
}

struct SweepLayout {
    size_t planes, sums, norms, total;
};

SweepLayout sweep_layout(int D, int C, const SweepConf &cf)
{
    SweepLayout L;
    size_t off = 0;
    const int W = words_for(D);
    const size_t ncfg = (size_t)cf.nb * cf.ns;
    L.planes = off; off = align_up(off + (size_t)cf.total_planes * C * W * 4, kAlign);
    L.sums = off;   off = align_up(off + ncfg * C * 8, kAlign);
    L.norms = off;  off = align_up(off + ncfg * C * 8, kAlign);
    L.total = off;
    return L;
}

}  // namespace
}  // namespace hdc

using namespace hdc;

extern "C" hdc_status hdc_sweep_workspace_bytes(int32_t D, int32_t C, const hdc_sweep_spec *spec, size_t *bytes)
{
    SweepConf cf;
    if (!bytes || D <= 0 || C <= 0 || !make_conf(spec, D, &cf)) return HDC_ERR_INVALID_ARG;
    *bytes = sweep_layout(D, C, cf).total;
    return HDC_OK;
}

extern "C" hdc_status hdc_sweep_eval(const uint32_t *H, const int32_t *y, int64_t N, int32_t D, int32_t C,
                                     const int32_t *acc, const hdc_sweep_spec *spec, int32_t *correct,
                                     int32_t *labels, void *ws, size_t ws_bytes, hdc_stream_t stream)
{
    SweepConf cf;
    if (N < 0 || D <= 0 || C <= 0 || !make_conf(spec, D, &cf) || !correct || !acc) return HDC_ERR_INVALID_ARG;
    if (N > 0 && (!H || !y || ((uintptr_t)H % 16) != 0)) return HDC_ERR_INVALID_ARG;
    const int tpb = spec->block_threads ? spec->block_threads : 128;
    if (tpb != 64 && tpb != 128 && tpb != 256) return HDC_ERR_INVALID_ARG;
    int wch = spec->words_per_chunk ? spec->words_per_chunk : 32;
    if (wch <= 0 || wch % 4 != 0) return HDC_ERR_INVALID_ARG;
    const int W = words_for(D);
    if (wch > W) wch = W;
    const SweepLayout L = sweep_layout(D, C, cf);
    if (!ws || ws_bytes < L.total || ((uintptr_t)ws % kAlign) != 0) return HDC_ERR_WORKSPACE;
    const size_t ncfg = (size_t)cf.nb * cf.ns;
    int maxp = 0;
    for (int j = 0; j < cf.nb; j++) maxp = cf.planes[j] > maxp ? cf.planes[j] : maxp;
    const size_t smem = (size_t)cf.ns * C * tpb * 8 + (size_t)wch * (tpb + 1) * 4 + (size_t)maxp * C * wch * 4;
    if (smem > 220 * 1024) return HDC_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    char *w = (char *)ws;
    if (cudaMemsetAsync(correct, 0, ncfg * sizeof(int32_t), st) != cudaSuccess) return HDC_ERR_CUDA;
    sweep_prep_kernel<<<C, 256, 0, st>>>(acc, D, C, W, cf, (uint32_t *)(w + L.planes), (long long *)(w + L.sums),
                                         (double *)(w + L.norms));
    if (cudaGetLastError() != cudaSuccess) return HDC_ERR_CUDA;
    if (N == 0) return HDC_OK;
    if (cudaFuncSetAttribute(sweep_eval_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return HDC_ERR_CUDA;
    const int64_t blocks = (N + tpb - 1) / tpb;
    sweep_eval_kernel<<<dim3((unsigned)blocks, (unsigned)cf.nb), tpb, smem, st>>>(H, y, N, C, W, wch, cf, (const uint32_t *)(w + L.planes),
                                                          (const long long *)(w + L.sums),
                                                          (const double *)(w + L.norms), correct, labels);
    return cudaGetLastError() == cudaSuccess ? HDC_OK : HDC_ERR_CUDA;
}
