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
// word over a chunk of one class's samples, four dims per 32-bit add (byte
// lanes, flushed every 255 rows), and adds |S| - 2*count to acc with one
// atomic per (chunk, dim).  Integer sums: exact and independent of order.
#include "hdc_internal.cuh"

namespace hdc {
namespace {

constexpr int CH = 252;  // samples per counting work item (byte-lane counters hold <= 255)

// key of sample n: bundling -> y_n; retraining -> y_n (which == 0) or
// pred_n (which == 1) for misclassified samples only; -1 = not counted.
__device__ __forceinline__ int key_of(const int32_t *y, const int32_t *pred, int64_t n, int C, int mode, int which)
{
    const int yc = y[n];
    if (yc < 0 || yc >= C) return -1;
    if (mode == 0) return yc;
    const int pc = pred[n];
    if (pc == yc) return -1;
    return which == 0 ? yc : pc;
}

__global__ void hist_kernel(const int32_t *__restrict__ y, const int32_t *__restrict__ pred, int64_t N, int C,
                            int mode, int which, int32_t *__restrict__ hist)
{
    extern __shared__ int32_t sh[];
    for (int c = threadIdx.x; c < C; c += blockDim.x) sh[c] = 0;
    __syncthreads();
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        const int k = key_of(y, pred, n, C, mode, which);
        if (k >= 0) atomicAdd(&sh[k], 1);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x)
        if (sh[c]) atomicAdd(&hist[c], sh[c]);
}

// offsets[c] = sum of hist[0..c), offsets[C] = total; cursors reset; the
// total is also added to *n_updates when given (retraining).
__global__ void scan_kernel(const int32_t *__restrict__ hist, int C, int32_t *__restrict__ offsets,
                            int32_t *__restrict__ cursor, int32_t *__restrict__ n_updates)
{
    if (threadIdx.x != 0) return;
    int32_t s = 0;
    for (int c = 0; c < C; c++) {
        offsets[c] = s;
        cursor[c] = 0;
        s += hist[c];
    }
    offsets[C] = s;
    if (n_updates) *n_updates += s;
}

__global__ void scatter_kernel(const int32_t *__restrict__ y, const int32_t *__restrict__ pred, int64_t N, int C,
                               int mode, int which, const int32_t *__restrict__ offsets,
                               int32_t *__restrict__ cursor, int32_t *__restrict__ perm)
{
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        const int k = key_of(y, pred, n, C, mode, which);
        if (k >= 0) perm[offsets[k] + atomicAdd(&cursor[k], 1)] = (int32_t)n;
    }
}

// Work item = (class c, chunk of at most CH of its samples); thread = word.
__global__ void __launch_bounds__(128) segment_count_kernel(const uint32_t *__restrict__ H, int W, int D,
                                                            const int32_t *__restrict__ perm,
                                                            const int32_t *__restrict__ offsets, int C, int sign,
                                                            int32_t *__restrict__ acc)
{
    __shared__ int32_t s_off[257];
    __shared__ int32_t s_rows[CH];
    const bool small = C <= 256;
    if (small)
        for (int c = threadIdx.x; c <= C; c += blockDim.x) s_off[c] = offsets[c];
    __syncthreads();
    auto off = [&](int c) { return small ? s_off[c] : offsets[c]; };
    const int word = blockIdx.x * blockDim.x + threadIdx.x;
    // walk the work items of this grid row
    int64_t item = 0;
    for (int c = 0; c < C; c++) {
        const int lo = off(c), hi = off(c + 1);
        for (int r0 = lo; r0 < hi; r0 += CH, item++) {
            if (item % gridDim.y != blockIdx.y) continue;  // uniform across the block
            const int r1 = min(hi, r0 + CH);
            __syncthreads();
            for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) s_rows[r - r0] = __ldg(perm + r);
            __syncthreads();
            if (word >= W) continue;
            // CH <= 255: the byte lanes cannot overflow within one item
            uint32_t lanes[8];
#pragma unroll
            for (int j = 0; j < 8; j++) lanes[j] = 0;
            const int n = r1 - r0;
            int r = 0;
            // sixteen independent gathered row loads in flight per thread: the
            // pass is bound by how many bytes each SM has outstanding
            for (; r + 16 <= n; r += 16) {
                uint32_t w[16];
#pragma unroll
                for (int u = 0; u < 16; u++) w[u] = __ldg(H + (int64_t)s_rows[r + u] * W + word);
#pragma unroll
                for (int u = 0; u < 16; u++)
#pragma unroll
                    for (int j = 0; j < 8; j++) lanes[j] += (w[u] >> j) & 0x01010101u;  // dims j, j+8, j+16, j+24
            }
            for (; r + 4 <= n; r += 4) {
                uint32_t w[4];
#pragma unroll
                for (int u = 0; u < 4; u++) w[u] = __ldg(H + (int64_t)s_rows[r + u] * W + word);
#pragma unroll
                for (int u = 0; u < 4; u++)
#pragma unroll
                    for (int j = 0; j < 8; j++) lanes[j] += (w[u] >> j) & 0x01010101u;
            }
            for (; r < n; r++) {
                const uint32_t w = __ldg(H + (int64_t)s_rows[r] * W + word);
#pragma unroll
                for (int j = 0; j < 8; j++) lanes[j] += (w >> j) & 0x01010101u;
            }
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

// One warp per (class, word): ballot of acc < 0 over the word's 32 dims.
__global__ void binarise_kernel(const int32_t *__restrict__ acc, int C, int D, uint32_t *__restrict__ cls, int W)
{
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= (int64_t)C * W) return;
    const int c = (int)(gw / W), w = (int)(gw % W);
    const int d = w * 32 + lane;
    const bool neg = d < D && acc[(int64_t)c * D + d] < 0;
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

// Group the counted samples by key and add their signed bit counts to acc.
cudaError_t group_and_count(const uint32_t *H, int W, const int32_t *y, const int32_t *pred, int64_t N, int D, int C,
                            int mode, int which, int sign, int32_t *acc, int32_t *n_updates, const TrainScratch &s,
                            cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(s.hist, 0, (size_t)C * sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    const int sms = sm_count();
    int64_t blocks = (N + 255) / 256;
    if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
    if (blocks < 1) blocks = 1;
    hist_kernel<<<(unsigned)blocks, 256, (size_t)C * sizeof(int32_t), st>>>(y, pred, N, C, mode, which, s.hist);
    scan_kernel<<<1, 32, 0, st>>>(s.hist, C, s.offsets, s.cursor, n_updates);
    scatter_kernel<<<(unsigned)blocks, 256, 0, st>>>(y, pred, N, C, mode, which, s.offsets, s.cursor, s.perm);
    // items: at most ceil(N / CH) + C; spread over grid rows
    const int64_t max_items = (N + CH - 1) / CH + C;
    const int wblocks = (W + 127) / 128;
    int64_t rows = (int64_t)sms * 4 / wblocks + 1;
    if (rows > max_items) rows = max_items;
    if (rows > 65535) rows = 65535;
    segment_count_kernel<<<dim3(wblocks, (unsigned)rows), 128, 0, st>>>(H, W, D, s.perm, s.offsets, C, sign, acc);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_train_count(const uint32_t *H, int W, const int32_t *y, const int32_t *pred, int64_t N, int D,
                               int C, int mode, int32_t *acc, int32_t *n_updates, const TrainScratch &s,
                               cudaStream_t st)
{
    if (N <= 0 || D <= 0 || C <= 0) return cudaSuccess;
    if (mode == 0) return group_and_count(H, W, y, pred, N, D, C, 0, 0, +1, acc, nullptr, s, st);
    cudaError_t e = group_and_count(H, W, y, pred, N, D, C, 1, 0, +1, acc, n_updates, s, st);
    if (e != cudaSuccess) return e;
    return group_and_count(H, W, y, pred, N, D, C, 1, 1, -1, acc, nullptr, s, st);
}

cudaError_t launch_binarise(const int32_t *acc, int C, int D, uint32_t *cls, int W, cudaStream_t st)
{
    const int64_t warps = (int64_t)C * W;
    if (warps <= 0) return cudaSuccess;
    const int64_t blocks = (warps * 32 + 255) / 256;
    binarise_kernel<<<(unsigned)blocks, 256, 0, st>>>(acc, C, D, cls, W);
    return cudaGetLastError();
}

}  // namespace hdc
