// K5 / K6: training of binary class hypervectors.
//
// Bundling (Sec. 2.1 training stage): acc[c][d] = sum over samples of class
// c of the +-1 element h[n][d] = 1 - 2*bit[n][d]; normalisation of a bundle
// is its sign (class bit = acc < 0).
// Retraining (TRAIN_ITERATIONS, Sec. 4.2 custom parameters; the perceptron
// rule applied once per epoch is our reading of the unstated update):
// samples whose Hamming arg-min prediction pred_n differs from y_n add h_n to
// acc[y_n] and subtract it from acc[pred_n].
//
// Both are class-grouped signed bit counts: for a set S of samples of one
// class, sum_{n in S} (1 - 2 bit[n][d]) = |S| - 2 * count_{n in S} bit[n][d].
// The samples are grouped by class with a counting sort (histogram -- folded
// into the arg-min of a retraining epoch for up to 16 classes --, scan,
// scatter of indices).  A counting work item is a chunk of at most 252 of
// one group's samples; a block streams the item's rows, 16 at a time, for a
// range of words through a ring of shared-memory stages filled by cp.async
// (several stages in flight per block, so the gathered rows stream at HBM
// rate instead of one load latency per 16 rows), and each thread counts the
// set bits of one 32-dim word: a carry-save tree of 15 full adders per 16
// rows (bit-sliced planes of weight 1, 2, 4, 8, 32 dims per logic operation)
// whose weight-16 carry is added four dims per 32-bit add into byte lanes;
// at the end of the item count = 16 * carries + planes <= 255 per byte.
// The item's byte lanes go to a partial buffer; a reduce kernel then sums,
// per (class, word), |S| - 2*count over the class's items (signed by group),
// writes or adds acc and packs the sign bits: no global atomics, and the
// re-binarisation is part of the same pass.  Integer sums: exact and
// independent of order.
#include "bitslice.cuh"
#include "hdc_internal.cuh"

namespace hdc {
namespace {

constexpr int CH = 252;  // samples per counting work item (byte-lane counters hold <= 255)

// Groups of sample n: bundling -> group y_n (G = C groups); retraining ->
// a misclassified sample is in group y_n (added) and in group C + pred_n
// (subtracted), G = 2C.  Returns the number of groups (0, 1 or 2).
__device__ __forceinline__ int keys_of(const int32_t *y, const int32_t *pred, int64_t n, int C, int mode, int (&k)[2])
{
    const int yc = y[n];
    if (yc < 0 || yc >= C) return 0;
    k[0] = yc;
    if (mode == 0) return 1;
    const int pc = pred[n];
    if (pc == yc) return 0;
    k[1] = C + pc;
    return 2;
}

// Group sizes; counted in shared memory while G groups fit (G <= 12,288),
// else straight into hist.
__global__ void hist_kernel(const int32_t *__restrict__ y, const int32_t *__restrict__ pred, int64_t N, int C,
                            int mode, int G, bool in_shared, int32_t *__restrict__ hist)
{
    extern __shared__ int32_t sh[];
    int32_t *h = in_shared ? sh : hist;
    if (in_shared) {
        for (int g = threadIdx.x; g < G; g += blockDim.x) sh[g] = 0;
        __syncthreads();
    }
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        int k[2];
        const int nk = keys_of(y, pred, n, C, mode, k);
        for (int i = 0; i < nk; i++) atomicAdd(&h[k[i]], 1);
    }
    if (in_shared) {
        __syncthreads();
        for (int g = threadIdx.x; g < G; g += blockDim.x)
            if (sh[g]) atomicAdd(&hist[g], sh[g]);
    }
}

// offsets[g] = sum of hist[0..g), offsets[G] = total; items[g] = counting
// work items of the groups before g (ceil(hist / CH) each); cursors reset;
// the count of the first C groups (the misclassified samples when
// retraining) is added to *n_updates when given.
__global__ void scan_kernel(const int32_t *__restrict__ hist, int G, int C, int32_t *__restrict__ offsets,
                            int32_t *__restrict__ items, int32_t *__restrict__ cursor,
                            int32_t *__restrict__ n_updates)
{
    if (threadIdx.x != 0) return;
    int32_t s = 0, it = 0;
    for (int g = 0; g < G; g++) {
        offsets[g] = s;
        items[g] = it;
        cursor[g] = 0;
        s += hist[g];
        it += (hist[g] + CH - 1) / CH;
    }
    offsets[G] = s;
    items[G] = it;
    if (n_updates) *n_updates += offsets[C < G ? C : G];
}

// The scan above for G <= SEG_SMEM_G groups, done by the first warp of a
// block into shared memory (off[0..G], first[0..G] when first != NULL):
// lane l scans a run of ceil(G / 32) groups, the run totals are scanned
// across the warp with shuffles.  The caller synchronises the block after.
constexpr int SEG_SMEM_G = 1024;  // groups whose offsets are formed in shared memory
__device__ void warp_scan_groups(const int32_t *__restrict__ hist, int G, int32_t *off, int32_t *first)
{
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    const int per = (G + 31) / 32;
    const int g0 = min(G, lane * per), g1 = min(G, g0 + per);
    int32_t s = 0, it = 0;
    for (int g = g0; g < g1; g++) {
        const int32_t h = hist[g];
        s += h;
        it += (h + CH - 1) / CH;
    }
    int32_t ps = s, pi = it;   // inclusive scans of the run totals
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t a = __shfl_up_sync(0xffffffffu, ps, o), b = __shfl_up_sync(0xffffffffu, pi, o);
        if (lane >= o) {
            ps += a;
            pi += b;
        }
    }
    s = ps - s;
    it = pi - it;
    for (int g = g0; g < g1; g++) {
        const int32_t h = hist[g];
        off[g] = s;
        if (first) first[g] = it;
        s += h;
        it += (h + CH - 1) / CH;
    }
    if (lane == 31) {
        off[G] = ps;
        if (first) first[G] = pi;
    }
}

// Scatter of the sample indices into their groups.  Each block takes a
// contiguous run of `run` samples (a multiple of 256 giving about four blocks
// per SM): it counts the run's entries per group
// in shared memory, reserves each group's range with one global atomic per
// group, then places the entries inside its ranges with shared-memory
// atomics (the order inside a group does not matter: the counts are sums).
// With hist (G <= SEG_SMEM_G) the group offsets are formed here from the
// histogram; otherwise they come from the scan kernel, and the per-block
// counts stay in global memory-backed atomics per warp (large G).
__global__ void __launch_bounds__(256) scatter_kernel(const int32_t *__restrict__ y, const int32_t *__restrict__ pred,
                                                      int64_t N, int64_t run, int C, int mode,
                                                      const int32_t *__restrict__ hist,
                                                      int G, const int32_t *__restrict__ offsets_in,
                                                      int32_t *__restrict__ cursor, int32_t *__restrict__ perm)
{
    __shared__ int32_t s_off[SEG_SMEM_G + 1];
    __shared__ int32_t s_cnt[SEG_SMEM_G];
    __shared__ int32_t s_base[SEG_SMEM_G];
    const int64_t n0 = (int64_t)blockIdx.x * run;
    const int64_t n1 = min(N, n0 + run);
    if (hist) {
        warp_scan_groups(hist, G, s_off, nullptr);
        for (int g = threadIdx.x; g < G; g += blockDim.x) s_cnt[g] = 0;
        __syncthreads();
        for (int64_t n = n0 + threadIdx.x; n < n1; n += blockDim.x) {
            int k[2];
            const int nk = keys_of(y, pred, n, C, mode, k);
            for (int i = 0; i < nk; i++) atomicAdd(&s_cnt[k[i]], 1);
        }
        __syncthreads();
        for (int g = threadIdx.x; g < G; g += blockDim.x) {
            const int c = s_cnt[g];
            s_base[g] = c ? s_off[g] + atomicAdd(&cursor[g], c) : 0;
            s_cnt[g] = 0;
        }
        __syncthreads();
        for (int64_t n = n0 + threadIdx.x; n < n1; n += blockDim.x) {
            int k[2];
            const int nk = keys_of(y, pred, n, C, mode, k);
            for (int i = 0; i < nk; i++) perm[s_base[k[i]] + atomicAdd(&s_cnt[k[i]], 1)] = (int32_t)n;
        }
        return;
    }
    // many groups: lanes of a warp with the same group take their slots with
    // one global atomic (blockDim.x is a multiple of 32, the loop warp-uniform)
    const int lane = threadIdx.x & 31;
    for (int64_t base = n0; base < n1; base += blockDim.x) {
        const int64_t n = base + threadIdx.x;
        int k[2];
        const int nk = n < n1 ? keys_of(y, pred, n, C, mode, k) : 0;
        for (int i = 0; i < (mode == 0 ? 1 : 2); i++) {
            const int key = i < nk ? k[i] : -1;
            const unsigned peers = __match_any_sync(0xffffffffu, key);
            const int leader = __ffs(peers) - 1;
            int slot = 0;
            if (lane == leader && key >= 0) slot = atomicAdd(&cursor[key], __popc(peers));
            slot = __shfl_sync(0xffffffffu, slot, leader) + __popc(peers & ((1u << lane) - 1u));
            if (key >= 0) perm[offsets_in[key] + slot] = (int32_t)n;
        }
    }
}

// 16-byte asynchronous global -> shared copy; with full == false nothing is
// read and the 16 bytes are zero-filled.
__device__ __forceinline__ void cp_async16(uint32_t *dst, const void *src, bool full)
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

// Group of work item `it`: the last g with first[g] <= it (an empty group has
// first[g] == first[g + 1], so the last such g is never empty).
__device__ __forceinline__ int group_of(const int32_t *first, int G, int it)
{
    int lo_g = 0, hi_g = G - 1;
    while (lo_g < hi_g) {
        const int mid = (lo_g + hi_g + 1) >> 1;
        if (first[mid] <= it) lo_g = mid;
        else hi_g = mid - 1;
    }
    return lo_g;
}

// Work item = (group g, chunk of at most CH of its samples); block = TW
// consecutive words, thread = word.  Grid row y counts the items y,
// y + gridDim.y, ...; rows arrive through a ring of NST stages of RS rows.
// Output: partial[it][word][j] = byte lanes of the item's set-bit counts,
// byte k of lane j = count of dim 32 * word + j + 8k.
constexpr int RS = 16;            // rows per stage (one carry-save tree)
constexpr int NST = 4;            // stages in the ring (three in flight while one is counted)
// With G <= SEG_SMEM_G the block forms the offsets and first items from
// hist itself, and block (0, 0) stores them for the reduce kernel and adds
// the count of the first C groups (the updated samples of a retraining
// epoch) to *n_updates; otherwise the scan kernel has done both.
template <int TW>
__global__ void __launch_bounds__(TW) count_kernel(const uint32_t *__restrict__ H, int W,
                                                   const int32_t *__restrict__ perm,
                                                   const int32_t *__restrict__ hist,
                                                   int32_t *__restrict__ offsets,
                                                   int32_t *__restrict__ items, int G, int C,
                                                   int32_t *__restrict__ n_updates,
                                                   uint32_t *__restrict__ partial)
{
    constexpr int CPR = TW / 4;   // 16-byte chunks of a row's TW words; RS * CPR = 4 * TW per stage
    __shared__ __align__(16) uint32_t ring[NST][RS][TW];
    __shared__ int32_t s_rows[CH];
    __shared__ int32_t s_off[SEG_SMEM_G + 1];
    __shared__ int32_t s_items[SEG_SMEM_G + 1];
    const bool small = G <= SEG_SMEM_G;
    if (small) {
        warp_scan_groups(hist, G, s_off, s_items);
        __syncthreads();
        if (blockIdx.x == 0 && blockIdx.y == 0) {
            for (int g = threadIdx.x; g <= G; g += TW) {
                offsets[g] = s_off[g];
                items[g] = s_items[g];
            }
            if (threadIdx.x == 0 && n_updates) *n_updates += s_off[C < G ? C : G];
        }
    }
    const int32_t *off = small ? s_off : offsets;
    const int32_t *first = small ? s_items : items;
    const int wbase = blockIdx.x * TW;
    const int word = wbase + threadIdx.x;
    const int total = first[G];
    for (int it = blockIdx.y; it < total; it += gridDim.y) {  // uniform across the block
        const int g = group_of(first, G, it);
        const int r0 = off[g] + (it - first[g]) * CH;
        const int n = min(off[g + 1], r0 + CH) - r0;
        __syncthreads();   // the previous item's last stage has been counted
        for (int r = threadIdx.x; r < n; r += TW) s_rows[r] = __ldg(perm + r0 + r);
        __syncthreads();
        const int nst = (n + RS - 1) / RS;
        // stage st: rows st*RS .. st*RS + 15 of the item (zero past n and past W)
        auto issue = [&](int st) {
            if (st < nst) {
                uint32_t *slot = &ring[st % NST][0][0];
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const int i = threadIdx.x + k * TW;
                    const int rr = i / CPR, c4 = (i % CPR) * 4;
                    const int r = st * RS + rr;
                    const bool ok = r < n && wbase + c4 < W;
                    cp_async16(slot + rr * TW + c4, ok ? (const void *)(H + (int64_t)s_rows[r] * W + wbase + c4)
                                                       : (const void *)H, ok);
                }
            }
            cp_async_commit();   // an empty group past the last stage keeps the count uniform
        };
#pragma unroll
        for (int st = 0; st < NST - 1; st++) issue(st);
        // CH <= 252: 16 * (carries <= 15) + (planes <= 15) fits a byte lane
        uint32_t lanes[8];
#pragma unroll
        for (int j = 0; j < 8; j++) lanes[j] = 0;
        uint32_t c1 = 0, c2 = 0, c4 = 0, c8 = 0;
        for (int st = 0; st < nst; st++) {
            issue(st + NST - 1);
            cp_async_wait<NST - 1>();   // stage st has landed (this thread's copies)
            __syncthreads();            // ... and every other thread's
            uint32_t w[RS];
#pragma unroll
            for (int u = 0; u < RS; u++) w[u] = ring[st % NST][u][threadIdx.x];
            const uint32_t e16 = csa16(c1, c2, c4, c8, w);
#pragma unroll
            for (int j = 0; j < 8; j++) lanes[j] += (e16 >> j) & 0x01010101u;  // dims j, j+8, j+16, j+24
            __syncthreads();            // the slot is refilled by the next iteration's issue
        }
        if (word < W) {
#pragma unroll
            for (int j = 0; j < 8; j++)
                lanes[j] = (lanes[j] << 4) + ((c1 >> j) & 0x01010101u) + (((c2 >> j) & 0x01010101u) << 1) +
                           (((c4 >> j) & 0x01010101u) << 2) + (((c8 >> j) & 0x01010101u) << 3);
            uint4 *dst = reinterpret_cast<uint4 *>(partial + ((int64_t)it * W + word) * 8);
            dst[0] = make_uint4(lanes[0], lanes[1], lanes[2], lanes[3]);
            dst[1] = make_uint4(lanes[4], lanes[5], lanes[6], lanes[7]);
        }
    }
    cp_async_wait<0>();
}

// A block = 32 (class c, word w, byte lane j) slots, i.e. the dims
// 32w + j + 8k, k = 0..3, times 8 warps that take every eighth counting item
// of the slot's groups: each sums |S| - 2 * count over its items of group c
// (and subtracts those of group C + c when retraining); warp 0 adds the 8
// partial sums, writes acc (accumulate: adds to it) for the dims below D,
// and, with cls, the eight lanes of a word OR their sign bits into the
// packed word (pad bits 0).
constexpr int RED_SLICES = 8;
__global__ void __launch_bounds__(32 * RED_SLICES) reduce_kernel(const uint32_t *__restrict__ partial, int W, int D,
                                                                 const int32_t *__restrict__ offsets,
                                                                 const int32_t *__restrict__ items, int G, int C,
                                                                 int accumulate, int32_t *__restrict__ acc,
                                                                 uint32_t *__restrict__ cls)
{
    __shared__ int32_t s_sum[RED_SLICES][4][32];
    const int lane = threadIdx.x & 31, slice = threadIdx.x >> 5;
    const int64_t t = (int64_t)blockIdx.x * 32 + lane;
    const bool live = t < (int64_t)C * W * 8;
    const int j = (int)(t & 7);
    const int64_t cw = live ? t >> 3 : 0;
    const int c = (int)(cw / W), w = (int)(cw % W);
    int sum[4] = {0, 0, 0, 0};
    if (live) {
        for (int side = 0; side < (G > C ? 2 : 1); side++) {
            const int g = side ? C + c : c;
            const int i0 = items[g], i1 = items[g + 1], o0 = offsets[g], o1 = offsets[g + 1];
            for (int it = i0 + slice; it < i1; it += RED_SLICES) {
                const int r0 = o0 + (it - i0) * CH;
                const int n = min(o1, r0 + CH) - r0;
                const uint32_t ln = __ldg(partial + ((int64_t)it * W + w) * 8 + j);
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const int v = n - 2 * (int)((ln >> (8 * k)) & 0xffu);
                    sum[k] += side ? -v : v;
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 4; k++) s_sum[slice][k][lane] = sum[k];
    __syncthreads();
    if (slice != 0) return;
#pragma unroll
    for (int k = 0; k < 4; k++)
#pragma unroll
        for (int q = 1; q < RED_SLICES; q++) sum[k] += s_sum[q][k][lane];
    uint32_t bits = 0;
    if (live) {
        const int64_t base = (int64_t)c * D;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int d = w * 32 + j + 8 * k;
            if (d < D) {
                const int v = sum[k] + (accumulate ? acc[base + d] : 0);
                acc[base + d] = v;
                bits |= (uint32_t)(v < 0) << (j + 8 * k);
            }
        }
    }
    // the eight lanes of one word are lanes 8i .. 8i + 7 of the warp
    bits |= __shfl_xor_sync(0xffffffffu, bits, 1);
    bits |= __shfl_xor_sync(0xffffffffu, bits, 2);
    bits |= __shfl_xor_sync(0xffffffffu, bits, 4);
    if (live && cls && j == 0) cls[cw] = bits;
}

// One warp per (class, word): ballot of acc < 0 over the word's 32 dims,
// after adding delta (the summed shard updates of an epoch) when given.
__global__ void binarise_kernel(int32_t *__restrict__ acc, const int32_t *__restrict__ delta, int C, int D,
                                uint32_t *__restrict__ cls, int W)
{
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= (int64_t)C * W) return;
    const int c = (int)(gw / W), w = (int)(gw % W);
    const int d = w * 32 + lane;
    bool neg = false;
    if (d < D) {
        const int64_t i = (int64_t)c * D + d;
        int32_t v = acc[i];
        if (delta) {
            v += delta[i];
            acc[i] = v;
        }
        neg = v < 0;
    }
    const unsigned b = __ballot_sync(0xffffffffu, neg);
    if (lane == 0) cls[gw] = b;
}

int sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
                                                     cudaSuccess)
        return 152;
    return n > 0 ? n : 152;
}

// Group the counted samples (hist already counted when hist_ready), count
// their bits per item and reduce into acc (and cls): G = C groups for
// bundling, 2C for retraining (one pass for both updates).
cudaError_t group_and_count(const uint32_t *H, int W, const int32_t *y, const int32_t *pred, int64_t N, int D, int C,
                            int mode, bool hist_ready, int accumulate, int32_t *acc, uint32_t *cls,
                            int32_t *n_updates, const TrainScratch &s, cudaStream_t st)
{
    const int G = mode == 0 ? C : 2 * C;
    const int sms = sm_count();
    int64_t blocks = (N + 255) / 256;
    if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
    if (blocks < 1) blocks = 1;
    if (!hist_ready) {
        const bool in_shared = (size_t)G * sizeof(int32_t) <= 48 * 1024;
        hist_kernel<<<(unsigned)blocks, 256, in_shared ? (size_t)G * sizeof(int32_t) : 0, st>>>(y, pred, N, C, mode,
                                                                                                G, in_shared, s.hist);
    }
    // up to SEG_SMEM_G groups the scatter and counting kernels scan the
    // histogram themselves; the cursors were zeroed with it
    const bool small = G <= SEG_SMEM_G;
    if (!small) scan_kernel<<<1, 32, 0, st>>>(s.hist, G, C, s.offsets, s.items, s.cursor, n_updates);
    int64_t run = (N + (int64_t)sms * 4 - 1) / ((int64_t)sms * 4);
    run = (run + 255) / 256 * 256;
    scatter_kernel<<<(unsigned)((N + run - 1) / run), 256, 0, st>>>(y, pred, N, run, C, mode, small ? s.hist : nullptr,
                                                                   G, s.offsets, s.cursor, s.perm);
    // items: at most ceil(entries / CH) + G, entries <= (G / C) * N; one
    // block per (item, word block), extra grid rows exit at once
    const int64_t max_items = train_max_items(N, C);
    const int wtile = W >= 128 ? 128 : W >= 64 ? 64 : 32;
    const int wblocks = (W + wtile - 1) / wtile;
    int64_t rows = max_items < 65535 ? max_items : 65535;
    const dim3 grid((unsigned)wblocks, (unsigned)rows);
    int32_t *nu = small ? n_updates : nullptr;
    if (wtile == 128)
        count_kernel<128><<<grid, 128, 0, st>>>(H, W, s.perm, s.hist, s.offsets, s.items, G, C, nu, s.partial);
    else if (wtile == 64)
        count_kernel<64><<<grid, 64, 0, st>>>(H, W, s.perm, s.hist, s.offsets, s.items, G, C, nu, s.partial);
    else
        count_kernel<32><<<grid, 32, 0, st>>>(H, W, s.perm, s.hist, s.offsets, s.items, G, C, nu, s.partial);
    const int64_t threads = (int64_t)C * W * 8;
    reduce_kernel<<<(unsigned)((threads + 31) / 32), 32 * RED_SLICES, 0, st>>>(s.partial, W, D, s.offsets, s.items, G, C,
                                                                      accumulate, acc, cls);
    return cudaGetLastError();
}

}  // namespace

int64_t train_max_items(int64_t N, int C)
{
    // retraining: up to 2N entries over 2C groups
    return (2 * N + CH - 1) / CH + 2 * (int64_t)C;
}

cudaError_t launch_train_pass(const uint32_t *H, int W, const int32_t *y, int64_t N, int D, int C, int mode,
                              const uint32_t *cls_in, int32_t *pred, int32_t *acc, uint32_t *cls_out,
                              int32_t *n_updates, const TrainScratch &s, cudaStream_t st)
{
    if (N <= 0 || D <= 0 || C <= 0) return cudaSuccess;
    const int G = mode == 0 ? C : 2 * C;
    // the group histogram and the scatter cursors start from zero (adjacent
    // in the workspace: one memset)
    cudaError_t e = cudaMemsetAsync(s.hist, 0, (size_t)4 * C * sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    bool hist_ready = false;
    if (mode != 0) {
        // prediction with the start-of-epoch classes; for up to 16 classes
        // the same kernel counts the retraining groups
        e = launch_argmin_groups(H, N, cls_in, C, W, y, pred, s.hist, st);
        if (e == cudaSuccess) {
            hist_ready = true;
        } else if (e == cudaErrorNotSupported) {
            e = launch_argmin_ws(H, N, cls_in, C, W, D, nullptr, pred, s.signs, st);
            if (e != cudaSuccess) return e;
        } else {
            return e;
        }
    }
    return group_and_count(H, W, y, pred, N, D, C, mode == 0 ? 0 : 1, hist_ready, mode == 1, acc, cls_out,
                           mode == 0 ? nullptr : n_updates, s, st);
}

cudaError_t launch_apply_binarise(const int32_t *delta, int32_t *acc, int C, int D, uint32_t *cls, int W,
                                  cudaStream_t st)
{
    const int64_t warps = (int64_t)C * W;
    if (warps <= 0) return cudaSuccess;
    const int64_t blocks = (warps * 32 + 255) / 256;
    binarise_kernel<<<(unsigned)blocks, 256, 0, st>>>(acc, delta, C, D, cls, W);
    return cudaGetLastError();
}

cudaError_t launch_binarise(const int32_t *acc, int C, int D, uint32_t *cls, int W, cudaStream_t st)
{
    // without a delta the kernel only reads acc
    return launch_apply_binarise(nullptr, const_cast<int32_t *>(acc), C, D, cls, W, st);
}

size_t class_sign_bytes(int C, int W)
{
    if (C <= 32 || !hamming_packed_ok(C, W)) return 0;
    return (size_t)((C + 15) / 16 * 16) * hamming_packed_ldcs(W);
}

cudaError_t launch_argmin_ws(const uint32_t *H, int64_t N, const uint32_t *cls, int C, int W, int64_t D,
                             const Perf *p, int32_t *labels, uint8_t *signs, cudaStream_t st)
{
    if (N <= 0) return cudaSuccess;
    if (signs && class_sign_bytes(C, W) > 0) {
        // expand the classes once, then stream them to the tensor-core route
        const int Cp = (C + 15) / 16 * 16;
        cudaError_t e = launch_class_sign(cls, C, W, (int)D, Cp, hamming_packed_ldcs(W), signs, st);
        if (e != cudaSuccess) return e;
        return launch_hamming_packed(H, N, cls, C, W, D, p ? p->s0 : 0, p ? p->e0 : D, p ? p->stride : 1, labels,
                                     nullptr, st, signs);
    }
    return launch_similarity(H, N, cls, C, W, 1, D, p, nullptr, nullptr, labels, nullptr, nullptr, st);
}

}  // namespace hdc
