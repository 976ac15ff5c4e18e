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
// The samples are grouped by class with a counting sort (histogram, scan,
// scatter of indices), then each thread counts the set bits of one 32-dim
// word over a chunk of at most 252 of one class's samples: sixteen rows at a
// time through a carry-save tree of 15 full adders (bit-sliced planes of
// weight 1, 2, 4, 8, 32 dims per logic operation), whose weight-16 carry is
// added four dims per 32-bit add into byte lanes; at the end of the chunk
// count = 16 * carries + planes <= 255 per byte.  It then adds
// |S| - 2*count to acc with one atomic per (chunk, dim).  Integer sums:
// exact and independent of order.
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

// Lanes of a warp with the same group take their slots with one atomic (a
// few classes would otherwise serialise every sample on a few cursors).
// blockDim.x is a multiple of 32 and the loop is warp-uniform.
__global__ void scatter_kernel(const int32_t *__restrict__ y, const int32_t *__restrict__ pred, int64_t N, int C,
                               int mode, const int32_t *__restrict__ offsets, int32_t *__restrict__ cursor,
                               int32_t *__restrict__ perm)
{
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < N; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t n = base + threadIdx.x;
        int k[2];
        const int nk = n < N ? keys_of(y, pred, n, C, mode, k) : 0;
        for (int i = 0; i < (mode == 0 ? 1 : 2); i++) {
            const int key = i < nk ? k[i] : -1;
            const unsigned peers = __match_any_sync(0xffffffffu, key);
            const int leader = __ffs(peers) - 1;
            int slot = 0;
            if (lane == leader && key >= 0) slot = atomicAdd(&cursor[key], __popc(peers));
            slot = __shfl_sync(0xffffffffu, slot, leader) + __popc(peers & ((1u << lane) - 1u));
            if (key >= 0) perm[offsets[key] + slot] = (int32_t)n;
        }
    }
}

// Work item = (group g, chunk of at most CH of its samples); thread = word.
// Group g adds to class g mod C, with sign -1 for the groups C..2C-1 of
// retraining.  Grid row y counts the items y, y + gridDim.y, ...; the group
// of an item is found by binary search over items[] (first item per group).
constexpr int SEG_SMEM_G = 1024;  // groups whose offsets are staged in shared memory
__global__ void __launch_bounds__(128, 8) segment_count_kernel(const uint32_t *__restrict__ H, int W, int D,
                                                            const int32_t *__restrict__ perm,
                                                            const int32_t *__restrict__ offsets,
                                                            const int32_t *__restrict__ items, int G, int C,
                                                            int32_t *__restrict__ acc)
{
    __shared__ int32_t s_off[SEG_SMEM_G + 1];
    __shared__ int32_t s_items[SEG_SMEM_G + 1];
    __shared__ int32_t s_rows[CH];
    const bool small = G <= SEG_SMEM_G;
    if (small)
        for (int g = threadIdx.x; g <= G; g += blockDim.x) {
            s_off[g] = offsets[g];
            s_items[g] = items[g];
        }
    __syncthreads();
    const int32_t *off = small ? s_off : offsets;
    const int32_t *first = small ? s_items : items;
    const int word = blockIdx.x * blockDim.x + threadIdx.x;
    const int total = first[G];
    for (int it = blockIdx.y; it < total; it += gridDim.y) {  // uniform across the block
        // the last g with first[g] <= it owns item it (an empty group has
        // first[g] == first[g + 1], so the last such g is never empty)
        int lo_g = 0, hi_g = G - 1;
        while (lo_g < hi_g) {
            const int mid = (lo_g + hi_g + 1) >> 1;
            if (first[mid] <= it) lo_g = mid;
            else hi_g = mid - 1;
        }
        const int g = lo_g;
        const int c = g < C ? g : g - C;
        const int sign = g < C ? 1 : -1;
        const int r0 = off[g] + (it - first[g]) * CH;
        const int r1 = min(off[g + 1], r0 + CH);
        {
            __syncthreads();
            for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) s_rows[r - r0] = __ldg(perm + r);
            __syncthreads();
            if (word >= W) continue;
            // CH <= 252: 16 * (carries <= 15) + (planes <= 15) fits a byte lane
            uint32_t lanes[8];
#pragma unroll
            for (int j = 0; j < 8; j++) lanes[j] = 0;
            uint32_t c1 = 0, c2 = 0, c4 = 0, c8 = 0;
            const int n = r1 - r0;
            // sixteen gathered row loads in flight per thread, and the next
            // sixteen issued before the current ones are counted: the pass is
            // bound by how many bytes each SM has outstanding.  Rows past n
            // read as zero words (no bits counted; n enters the sum below).
            uint32_t nxt[16];
#pragma unroll
            for (int u = 0; u < 16; u++) nxt[u] = u < n ? __ldg(H + (int64_t)s_rows[u] * W + word) : 0u;
            for (int r = 0; r < n; r += 16) {
                uint32_t w[16];
#pragma unroll
                for (int u = 0; u < 16; u++) w[u] = nxt[u];
                if (r + 16 < n) {
#pragma unroll
                    for (int u = 0; u < 16; u++)
                        nxt[u] = r + 16 + u < n ? __ldg(H + (int64_t)s_rows[r + 16 + u] * W + word) : 0u;
                }
                const uint32_t e16 = csa16(c1, c2, c4, c8, w);
#pragma unroll
                for (int j = 0; j < 8; j++) lanes[j] += (e16 >> j) & 0x01010101u;  // dims j, j+8, j+16, j+24
            }
#pragma unroll
            for (int j = 0; j < 8; j++)
                lanes[j] = (lanes[j] << 4) + ((c1 >> j) & 0x01010101u) + (((c2 >> j) & 0x01010101u) << 1) +
                           (((c4 >> j) & 0x01010101u) << 2) + (((c8 >> j) & 0x01010101u) << 3);
            int cnt[32];
#pragma unroll
            for (int j = 0; j < 8; j++)
#pragma unroll
                for (int k = 0; k < 4; k++) cnt[j + 8 * k] = (lanes[j] >> (8 * k)) & 0xffu;
#pragma unroll
            for (int b = 0; b < 32; b++) {
                const int d = word * 32 + b;
                if (d < D) atomicAdd(acc + (int64_t)c * D + d, sign * (n - 2 * cnt[b]));
            }
        }
    }
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

// Group the counted samples and add their signed bit counts to acc: G = C
// groups for bundling, 2C for retraining (one pass for both updates).
cudaError_t group_and_count(const uint32_t *H, int W, const int32_t *y, const int32_t *pred, int64_t N, int D, int C,
                            int mode, int32_t *acc, int32_t *n_updates, const TrainScratch &s, cudaStream_t st)
{
    const int G = mode == 0 ? C : 2 * C;
    cudaError_t e = cudaMemsetAsync(s.hist, 0, (size_t)G * sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    const int sms = sm_count();
    int64_t blocks = (N + 255) / 256;
    if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
    if (blocks < 1) blocks = 1;
    const bool in_shared = (size_t)G * sizeof(int32_t) <= 48 * 1024;
    hist_kernel<<<(unsigned)blocks, 256, in_shared ? (size_t)G * sizeof(int32_t) : 0, st>>>(y, pred, N, C, mode, G,
                                                                                            in_shared, s.hist);
    scan_kernel<<<1, 32, 0, st>>>(s.hist, G, C, s.offsets, s.items, s.cursor, n_updates);
    scatter_kernel<<<(unsigned)blocks, 256, 0, st>>>(y, pred, N, C, mode, s.offsets, s.cursor, s.perm);
    // items: at most ceil(entries / CH) + G, entries <= (G / C) * N.  A block
    // spans up to 128 words (narrow rows take a narrower block); about 32
    // warps per SM, grid rows striding over the items.
    const int64_t max_items = ((G / C) * N + CH - 1) / CH + G;
    const int threads = W >= 128 ? 128 : (W + 31) / 32 * 32;
    const int wblocks = (W + threads - 1) / threads;
    int64_t rows = (int64_t)sms * (1024 / threads) / wblocks + 1;
    if (rows > max_items) rows = max_items;
    if (rows > 65535) rows = 65535;
    segment_count_kernel<<<dim3(wblocks, (unsigned)rows), threads, 0, st>>>(H, W, D, s.perm, s.offsets, s.items, G,
                                                                            C, acc);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_train_count(const uint32_t *H, int W, const int32_t *y, const int32_t *pred, int64_t N, int D,
                               int C, int mode, int32_t *acc, int32_t *n_updates, const TrainScratch &s,
                               cudaStream_t st)
{
    if (N <= 0 || D <= 0 || C <= 0) return cudaSuccess;
    return group_and_count(H, W, y, pred, N, D, C, mode, acc, mode == 0 ? nullptr : n_updates, s, st);
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

}  // namespace hdc
