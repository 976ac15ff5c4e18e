// K4: similarity of packed query hypervectors to C class hypervectors and
// the nearest class (Listing 1: __hetero_hdc_hamming_distance, red_perf,
// __hetero_hdc_arg_min; Sec. 4.2 Automatic Binarization: xor + popcount).
//
//  NB == 1  Hamming distance, dist = sum_w popc((q ^ c) & mask), arg-min.
//           The mask selects the kept dims of a perforated reduction
//           (all ones without perforation; pad bits are zero in q and c).
//  NB  > 1  cosine on b-bit class hypervectors stored as two's-complement
//           bit planes: with q_d = 1 - 2*bit_d,
//             dot_c = sum_d q_d chat_d = S_c - 2 * sum_j w_j popc(plane_j & q)
//           (S_c = sum_d chat_d, w_j = 2^j, w_{b-1} = -2^{b-1});
//           score = dot / ||chat|| in IEEE FP64, arg-max.
// Ties go to the lowest class index.
//
// One query per thread, 128 per block; class words are staged through shared
// memory in chunks of WCH words, partial sums live in shared memory
// (acc[c][thread]) so C is a runtime value.
#include "bitslice.cuh"
#include "hdc_internal.cuh"

namespace hdc {
namespace {

constexpr int TPB = 128;

template <int NB>
__global__ void __launch_bounds__(TPB) similarity_kernel(const uint32_t *__restrict__ Q, int64_t N,
                                                         const uint32_t *__restrict__ planes, int C, int W, int WCH,
                                                         int use_mask, int64_t s0, int64_t e0, int64_t stride,
                                                         const int32_t *__restrict__ csum,
                                                         const double *__restrict__ cnorm,
                                                         int32_t *__restrict__ labels, int32_t *__restrict__ dists,
                                                         double *__restrict__ scores)
{
    extern __shared__ __align__(16) uint32_t smem[];
    int32_t *acc = reinterpret_cast<int32_t *>(smem);        // C x TPB
    uint32_t *cw = smem + (size_t)C * TPB;                    // NB x C x WCH
    uint32_t *mk = cw + (size_t)NB * C * WCH;                 // WCH
    const int tid = threadIdx.x;
    const int64_t row = (int64_t)blockIdx.x * TPB + tid;
    const bool valid = row < N;
    const uint32_t *qrow = Q + (valid ? row : 0) * (int64_t)W;

    for (int c = 0; c < C; c++) acc[c * TPB + tid] = 0;

    for (int w0 = 0; w0 < W; w0 += WCH) {
        const int nw = min(WCH, W - w0);
        __syncthreads();
        for (int i = tid; i < NB * C * WCH; i += TPB) {
            const int pc = i / WCH, j = i % WCH;   // pc = plane*C + class
            cw[i] = j < nw ? planes[(int64_t)pc * W + w0 + j] : 0u;
        }
        for (int j = tid; j < WCH; j += TPB) {
            uint32_t m = 0xffffffffu;
            if (use_mask) {  // kept dims s0, s0+stride, ... < e0 inside this word
                m = 0;
                const int64_t base = (int64_t)(w0 + j) * 32;
                const int64_t lo = max(s0, base), hi = min(e0, base + 32);
                if (lo < hi) {
                    const int64_t r = (lo - s0) % stride;
                    for (int64_t d = r ? lo + (stride - r) : lo; d < hi; d += stride) m |= 1u << (d - base);
                }
            }
            mk[j] = j < nw ? m : 0u;
        }
        __syncthreads();
        for (int j0 = 0; j0 < nw; j0 += 4) {  // W and WCH are multiples of 4
            uint4 qv = valid ? *reinterpret_cast<const uint4 *>(qrow + w0 + j0) : make_uint4(0, 0, 0, 0);
            uint32_t q[4] = {qv.x & mk[j0], qv.y & mk[j0 + 1], qv.z & mk[j0 + 2], qv.w & mk[j0 + 3]};
            if (NB == 1) {
                for (int c = 0; c < C; c++) {
                    const uint4 cv = *reinterpret_cast<const uint4 *>(cw + c * WCH + j0);
                    const int part = __popc(q[0] ^ (cv.x & mk[j0])) + __popc(q[1] ^ (cv.y & mk[j0 + 1])) +
                                     __popc(q[2] ^ (cv.z & mk[j0 + 2])) + __popc(q[3] ^ (cv.w & mk[j0 + 3]));
                    acc[c * TPB + tid] += part;
                }
            } else {
                for (int c = 0; c < C; c++) {
                    int part = 0;
#pragma unroll
                    for (int p = 0; p < NB; p++) {
                        const uint4 pv = *reinterpret_cast<const uint4 *>(cw + (p * C + c) * WCH + j0);
                        const int cnt = __popc(q[0] & pv.x) + __popc(q[1] & pv.y) + __popc(q[2] & pv.z) +
                                        __popc(q[3] & pv.w);
                        part += (p == NB - 1) ? -(cnt << p) : (cnt << p);
                    }
                    acc[c * TPB + tid] += part;
                }
            }
        }
    }
    if (!valid) return;
    if (NB == 1) {
        int best = 0, bv = acc[tid];
        for (int c = 0; c < C; c++) {
            const int v = acc[c * TPB + tid];
            if (dists) dists[row * C + c] = v;
            if (v < bv) { bv = v; best = c; }
        }
        labels[row] = best;
    } else {
        int best = 0;
        double bs = 0.0;
        for (int c = 0; c < C; c++) {
            const double nrm = cnorm[c];
            const double s = nrm == 0.0 ? 0.0 : (double)(csum[c] - 2 * acc[c * TPB + tid]) / nrm;
            if (scores) scores[row * C + c] = s;
            if (c == 0 || s > bs) { bs = s; best = c; }
        }
        labels[row] = best;
    }
}

// Hamming arg-min for C <= CMAX with the distances in registers.  A block
// stages RB = 128 / S queries x RWCH words coalesced into shared memory,
// transposed ([word][query], padded), with the chunk's class words and
// masks; every class word is then a broadcast read.  S threads share a
// query when the batch gives fewer than twelve 128-query blocks per SM
// (S = 4; 10^5 queries of 512 words ran ~15 % faster so, 3 * 10^5 of 32
// words ~5 % slower): thread (r, s) counts the words s, s + S, ... of each
// chunk for query r, and the partial distances are summed through shared
// memory before the arg-min.
constexpr int RWCH = 32;

template <int CMAX, int S>
__global__ void __launch_bounds__(TPB) hamming_reg_kernel(const uint32_t *__restrict__ Q, int64_t N,
                                                          const uint32_t *__restrict__ cls, int C, int W,
                                                          int use_mask, int64_t s0, int64_t e0, int64_t stride,
                                                          int32_t *__restrict__ labels, int32_t *__restrict__ dists)
{
    constexpr int RB = TPB / S;
    __shared__ uint32_t sq[RWCH][RB + 1];
    __shared__ uint32_t sc[CMAX][RWCH];
    __shared__ uint32_t mk[RWCH];
    __shared__ int32_t sd[S > 1 ? S - 1 : 1][CMAX][RB];
    const int tid = threadIdx.x;
    const int r = tid % RB, s = tid / RB;  // a warp holds 32 consecutive queries of one s
    const int64_t row0 = (int64_t)blockIdx.x * RB;
    const int64_t row = row0 + r;
    int best = 0, bv = 0x7fffffff;
    // classes in chunks of CMAX (one chunk when C <= CMAX); chunks ascend, so
    // a strict comparison keeps the lowest class on ties
    for (int cb = 0; cb < C; cb += CMAX) {
        const int cn = min(CMAX, C - cb);
        int dist[CMAX];
#pragma unroll
        for (int c = 0; c < CMAX; c++) dist[c] = 0;
        for (int w0 = 0; w0 < W; w0 += RWCH) {
            const int nw = min(RWCH, W - w0);
            __syncthreads();
            for (int i = tid; i < RB * RWCH; i += TPB) {  // consecutive threads: consecutive words of a row
                const int rr = i / RWCH, j = i % RWCH;
                sq[j][rr] = (row0 + rr < N && j < nw) ? __ldg(Q + (row0 + rr) * W + w0 + j) : 0u;
            }
            for (int i = tid; i < CMAX * RWCH; i += TPB) {
                const int c = i / RWCH, j = i % RWCH;
                sc[c][j] = (c < cn && j < nw) ? __ldg(cls + (int64_t)(cb + c) * W + w0 + j) : 0u;
            }
            if (tid < RWCH) {
                uint32_t m = tid < nw ? 0xffffffffu : 0u;
                if (use_mask && tid < nw) {  // kept dims s0, s0+stride, ... < e0 inside this word
                    m = 0;
                    const int64_t base = (int64_t)(w0 + tid) * 32;
                    const int64_t lo = max(s0, base), hi = min(e0, base + 32);
                    if (lo < hi) {
                        const int64_t r = (lo - s0) % stride;
                        for (int64_t d = r ? lo + (stride - r) : lo; d < hi; d += stride) m |= 1u << (d - base);
                    }
                }
                mk[tid] = m;
            }
            __syncthreads();
            for (int j = s; j < nw; j += S) {
                const uint32_t m = mk[j];
                const uint32_t q = sq[j][r] & m;
#pragma unroll
                for (int c = 0; c < CMAX; c++)
                    if (c < cn) dist[c] += __popc(q ^ (sc[c][j] & m));
            }
        }
        if (S > 1) {  // the next write of sd follows the next chunk loop's barriers
            if (s > 0)
#pragma unroll
                for (int c = 0; c < CMAX; c++) sd[s - 1][c][r] = dist[c];
            __syncthreads();
            if (s == 0)
#pragma unroll
                for (int c = 0; c < CMAX; c++)
#pragma unroll
                    for (int t = 0; t < S - 1; t++) dist[c] += sd[t][c][r];
        }
        if (s == 0 && row < N) {
#pragma unroll
            for (int c = 0; c < CMAX; c++)
                if (c < cn) {
                    if (dists) dists[row * C + cb + c] = dist[c];
                    if (dist[c] < bv) { bv = dist[c]; best = cb + c; }
                }
        }
    }
    if (s == 0 && row < N) labels[row] = best;
}

// 16-byte asynchronous global -> shared copy; with full == false nothing is
// read and the 16 bytes are zero-filled.
__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool full)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(full ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory");
}

constexpr int QRING = 8;   // query-word slots per thread of the carry-save arg-min

// Kept dims of a perforation (s0, s0 + stride, ... < e0) inside 32-dim word w.
__device__ __forceinline__ uint32_t perf_word_mask(int64_t w, int64_t s0, int64_t e0, int64_t stride)
{
    uint32_t m = 0;
    const int64_t base = w * 32;
    const int64_t lo = max(s0, base), hi = min(e0, base + 32);
    if (lo < hi) {
        const int64_t r = (lo - s0) % stride;
        for (int64_t d = r ? lo + (stride - r) : lo; d < hi; d += stride) m |= 1u << (d - base);
    }
    return m;
}

// Hamming arg-min for at most 16 binary classes (CM = C rounded up to even).
// Four threads per query: thread s takes the 16-byte groups of four words
// 4s, 4s + 16, 4s + 32, ... of its query (a warp reads eight 64-byte runs),
// streamed through a per-thread ring of QRING shared-memory slots.
// The class words of a chunk of WC words sit in shared memory (zero past C;
// both the class words and the query words are ANDed with the kept-dim mask,
// so (q ^ c) counts only kept dims).  Per class, the four mismatch words
// x = q ^ c enter a bit-sliced carry-save counter of planes of weight 1 and
// 2 (three full adders); only the carry of weight 4 is popcounted, one
// popcount per four words instead of four, the remaining work being 3-input
// logic operations.  dist = 4 * sum popc(e4) + 2 popc(c2) + popc(c1), summed
// over the four threads by shuffles.  With HIST, the kernel also counts the
// groups of a retraining epoch: a sample whose prediction differs from its
// label y goes to group y (added) and group C + prediction (subtracted).
template <int CM, bool MASKED, bool HIST>
__global__ void __launch_bounds__(TPB) hamming_csa_kernel(const uint32_t *__restrict__ Q, int64_t N,
                                                          const uint32_t *__restrict__ cls, int C, int W, int WC,
                                                          int64_t s0, int64_t e0, int64_t stride,
                                                          int32_t *__restrict__ labels, int32_t *__restrict__ dists,
                                                          const int32_t *__restrict__ y, int32_t *__restrict__ hist)
{
    extern __shared__ __align__(16) uint32_t smem[];
    uint4 *qr = reinterpret_cast<uint4 *>(smem);                    // QRING x TPB query slots
    uint32_t *sc = smem + QRING * TPB * 4;                          // CM x WC
    uint32_t *mk = sc + CM * WC;                                    // WC (MASKED)
    __shared__ int32_t sh[2 * CM];
    const int tid = threadIdx.x, s = tid & 3;
    const int64_t row = (int64_t)blockIdx.x * (TPB / 4) + (tid >> 2);
    const bool valid = row < N;
    const uint32_t *q = Q + (valid ? row : 0) * (int64_t)W;
    uint32_t c1[CM], c2[CM];
    int d4[CM];
#pragma unroll
    for (int c = 0; c < CM; c++) {
        c1[c] = 0;
        c2[c] = 0;
        d4[c] = 0;
    }
    if (HIST && tid < 2 * CM) sh[tid] = 0;
    const uint4 zero = make_uint4(0, 0, 0, 0);
    for (int w0 = 0; w0 < W; w0 += WC) {
        const int nw = min(WC, W - w0);   // a multiple of 4
        const int n16 = (nw + 15) & ~15;
        __syncthreads();
        if (MASKED)
            for (int j = tid; j < n16; j += TPB) mk[j] = j < nw ? perf_word_mask(w0 + j, s0, e0, stride) : 0u;
        if (MASKED) __syncthreads();
        for (int i = tid; i < CM * (n16 >> 2); i += TPB) {
            const int c = i / (n16 >> 2), j = (i % (n16 >> 2)) * 4;
            uint4 v = zero;
            if (c < C && j < nw) {
                v = __ldg(reinterpret_cast<const uint4 *>(cls + (int64_t)c * W + w0 + j));
                if (MASKED) {
                    v.x &= mk[j];
                    v.y &= mk[j + 1];
                    v.z &= mk[j + 2];
                    v.w &= mk[j + 3];
                }
            }
            *reinterpret_cast<uint4 *>(sc + c * WC + j) = v;
        }
        __syncthreads();
        // the thread's query words stream through its own ring of QRING
        // 16-byte slots (cp.async, QRING - 1 groups ahead of the one counted;
        // a thread reads back only what it copied, so no block barrier)
        auto issue = [&](int k) {
            const int j = k + 4 * s;
            const bool ok = valid && k < n16 && j < nw;
            cp_async16(qr + (k >> 4) % QRING * TPB + tid, ok ? (const void *)(q + w0 + j) : (const void *)Q, ok);
            cp_async_commit();
        };
#pragma unroll
        for (int p = 0; p < QRING - 1; p++) issue(16 * p);
        for (int k = 0; k < n16; k += 16) {
            const int j = k + 4 * s;
            issue(k + 16 * (QRING - 1));
            cp_async_wait<QRING - 1>();
            uint4 qv = qr[(k >> 4) % QRING * TPB + tid];
            if (MASKED) {
                const uint4 m = *reinterpret_cast<const uint4 *>(mk + j);
                qv.x &= m.x;
                qv.y &= m.y;
                qv.z &= m.z;
                qv.w &= m.w;
            }
#pragma unroll
            for (int c = 0; c < CM; c++) {
                const uint4 v = *reinterpret_cast<const uint4 *>(sc + c * WC + j);
                uint32_t a2, b2, e4;
                csa(a2, c1[c], c1[c], qv.x ^ v.x, qv.y ^ v.y);
                csa(b2, c1[c], c1[c], qv.z ^ v.z, qv.w ^ v.w);
                csa(e4, c2[c], c2[c], a2, b2);
                d4[c] += __popc(e4);
            }
        }
        cp_async_wait<0>();   // the ring's trailing zero-fills land before the next chunk reuses it
    }
    int best = 0, bv = 0x7fffffff;
#pragma unroll
    for (int c = 0; c < CM; c++) {
        int v = 4 * d4[c] + 2 * __popc(c2[c]) + __popc(c1[c]);
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        if (c < C) {
            if (dists && valid && s == 0) dists[row * C + c] = v;
            if (v < bv) {
                bv = v;
                best = c;
            }
        }
    }
    if (valid && s == 0) {
        labels[row] = best;
        if (HIST) {
            const int yc = y[row];
            if (yc >= 0 && yc < C && yc != best) {
                atomicAdd(&sh[yc], 1);
                atomicAdd(&sh[C + best], 1);
            }
        }
    }
    if (HIST) {
        __syncthreads();
        if (tid < 2 * C && sh[tid]) atomicAdd(hist + tid, sh[tid]);
    }
}

template <int CM, bool MASKED, bool HIST>
cudaError_t launch_csa_cm(const uint32_t *Q, int64_t N, const uint32_t *cls, int C, int W, int64_t s0, int64_t e0,
                          int64_t stride, int32_t *labels, int32_t *dists, const int32_t *y, int32_t *hist,
                          cudaStream_t st)
{
    const int w16 = (W + 15) & ~15;
    const int WC = w16 < 512 ? w16 : 512;
    const size_t smem = ((size_t)QRING * TPB * 4 + (size_t)CM * WC + (MASKED ? WC : 0)) * sizeof(uint32_t);
    auto k = hamming_csa_kernel<CM, MASKED, HIST>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int64_t blocks = (N + TPB / 4 - 1) / (TPB / 4);
    k<<<(unsigned)blocks, TPB, smem, st>>>(Q, N, cls, C, W, WC, s0, e0, stride, labels, dists, y, hist);
    return cudaGetLastError();
}

template <bool MASKED, bool HIST>
cudaError_t launch_csa(const uint32_t *Q, int64_t N, const uint32_t *cls, int C, int W, int64_t s0, int64_t e0,
                       int64_t stride, int32_t *labels, int32_t *dists, const int32_t *y, int32_t *hist,
                       cudaStream_t st)
{
    switch ((C + 1) / 2) {
    case 1: return launch_csa_cm<2, MASKED, HIST>(Q, N, cls, C, W, s0, e0, stride, labels, dists, y, hist, st);
    case 2: return launch_csa_cm<4, MASKED, HIST>(Q, N, cls, C, W, s0, e0, stride, labels, dists, y, hist, st);
    case 3: return launch_csa_cm<6, MASKED, HIST>(Q, N, cls, C, W, s0, e0, stride, labels, dists, y, hist, st);
    case 4: return launch_csa_cm<8, MASKED, HIST>(Q, N, cls, C, W, s0, e0, stride, labels, dists, y, hist, st);
    case 5: return launch_csa_cm<10, MASKED, HIST>(Q, N, cls, C, W, s0, e0, stride, labels, dists, y, hist, st);
    case 6: return launch_csa_cm<12, MASKED, HIST>(Q, N, cls, C, W, s0, e0, stride, labels, dists, y, hist, st);
    case 7: return launch_csa_cm<14, MASKED, HIST>(Q, N, cls, C, W, s0, e0, stride, labels, dists, y, hist, st);
    case 8: return launch_csa_cm<16, MASKED, HIST>(Q, N, cls, C, W, s0, e0, stride, labels, dists, y, hist, st);
    default: return cudaErrorNotSupported;
    }
}

int device_sms()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
                                                     cudaSuccess)
            n = 0;
    }
    return n > 0 ? n : 152;
}

template <int CMAX>
cudaError_t launch_reg(const uint32_t *Q, int64_t N, const uint32_t *cls, int C, int W, int64_t D, const Perf *p,
                       int32_t *labels, int32_t *dists, cudaStream_t st)
{
    const int use_mask = p != nullptr;
    const int64_t s0 = p ? p->s0 : 0, e0 = p ? p->e0 : D, stride = p ? p->stride : 1;
    if ((N + TPB - 1) / TPB < 12 * (int64_t)device_sms()) {  // short batch: four threads per query
        const int64_t blocks = (N + TPB / 4 - 1) / (TPB / 4);
        hamming_reg_kernel<CMAX, 4><<<(unsigned)blocks, TPB, 0, st>>>(Q, N, cls, C, W, use_mask, s0, e0, stride,
                                                                      labels, dists);
    } else {
        const int64_t blocks = (N + TPB - 1) / TPB;
        hamming_reg_kernel<CMAX, 1><<<(unsigned)blocks, TPB, 0, st>>>(Q, N, cls, C, W, use_mask, s0, e0, stride,
                                                                      labels, dists);
    }
    return cudaGetLastError();
}

template <int NB>
cudaError_t launch_nb(const uint32_t *Q, int64_t N, const uint32_t *planes, int C, int W, int64_t D, const Perf *p,
                      const int32_t *csum, const double *cnorm, int32_t *labels, int32_t *dists, double *scores,
                      cudaStream_t st)
{
    // words per staged chunk: multiple of 4 with NB*C*WCH*4 bytes <= 64 KB
    int WCH = (16384 / (NB * C)) / 4 * 4;
    if (WCH < 4) return cudaErrorNotSupported;
    if (WCH > 256) WCH = 256;
    if (WCH > W) WCH = W;
    const size_t smem = ((size_t)C * TPB + (size_t)NB * C * WCH + WCH) * sizeof(uint32_t);
    if (smem > 200 * 1024) return cudaErrorNotSupported;
    cudaError_t e = cudaFuncSetAttribute(similarity_kernel<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int use_mask = p != nullptr;
    const int64_t s0 = p ? p->s0 : 0, e0 = p ? p->e0 : D, stride = p ? p->stride : 1;
    const int64_t blocks = (N + TPB - 1) / TPB;
    similarity_kernel<NB><<<(unsigned)blocks, TPB, smem, st>>>(Q, N, planes, C, W, WCH, use_mask, s0, e0, stride,
                                                               csum, cnorm, labels, dists, scores);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_similarity(const uint32_t *Q, int64_t N, const uint32_t *planes, int C, int W, int nb, int64_t D,
                              const Perf *p, const int32_t *csum, const double *cnorm, int32_t *labels,
                              int32_t *dists, double *scores, cudaStream_t st)
{
    if (N <= 0) return cudaSuccess;
    if (nb == 1 && C <= 16) {
        if (p) return launch_csa<true, false>(Q, N, planes, C, W, p->s0, p->e0, p->stride, labels, dists, nullptr,
                                              nullptr, st);
        return launch_csa<false, false>(Q, N, planes, C, W, 0, D, 1, labels, dists, nullptr, nullptr, st);
    }
    if (nb == 1 && C <= 32) return launch_reg<32>(Q, N, planes, C, W, D, p, labels, dists, st);
    // 33..256 binary classes: the distances as a tensor-core product of the
    // rows expanded to +-1 (the popcount loop is bound by the popcount unit,
    // ~16 per clock per SM; up to 32 classes it measured faster, the
    // expansion not yet amortised: 0.24 vs 0.35 ms for 10^6 x 1,024 dims x 26)
    if (nb == 1 && C > 32 && hamming_packed_ok(C, W))
        return launch_hamming_packed(Q, N, planes, C, W, D, p ? p->s0 : 0, p ? p->e0 : D, p ? p->stride : 1, labels,
                                     dists, st);
    if (nb == 1) return launch_reg<64>(Q, N, planes, C, W, D, p, labels, dists, st);   // chunks of 64 classes
    switch (nb) {
    case 1: return launch_nb<1>(Q, N, planes, C, W, D, p, csum, cnorm, labels, dists, scores, st);
    case 4: return launch_nb<4>(Q, N, planes, C, W, D, nullptr, csum, cnorm, labels, dists, scores, st);
    case 8: return launch_nb<8>(Q, N, planes, C, W, D, nullptr, csum, cnorm, labels, dists, scores, st);
    default: return cudaErrorNotSupported;
    }
}

cudaError_t launch_argmin_groups(const uint32_t *H, int64_t N, const uint32_t *cls, int C, int W, const int32_t *y,
                                int32_t *pred, int32_t *hist, cudaStream_t st)
{
    if (N <= 0) return cudaSuccess;
    if (C > 16) return cudaErrorNotSupported;
    return launch_csa<false, true>(H, N, cls, C, W, 0, (int64_t)W * 32, 1, pred, nullptr, y, hist, st);
}

}  // namespace hdc
