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
// The count kernel gives each thread one dimension of a 256-dim column
// block and keeps per-class partial counts in shared memory (cnt[c][thread]);
// a grid of (column blocks x row chunks) adds them to acc with atomics, so
// the result is exact and independent of the order of the rows.
#include "hdc_internal.cuh"

namespace hdc {
namespace {

constexpr int CB = 256;  // dims per column block = threads per block

__global__ void __launch_bounds__(CB) train_count_kernel(const uint32_t *__restrict__ H, int W,
                                                         const int32_t *__restrict__ y,
                                                         const int32_t *__restrict__ pred, int64_t N, int D, int C,
                                                         int mode, int64_t rows_per_chunk,
                                                         int32_t *__restrict__ acc, int32_t *__restrict__ n_updates)
{
    extern __shared__ int32_t cnt[];  // C x CB
    const int t = threadIdx.x;
    const int d = blockIdx.x * CB + t;
    const int word = d >> 5, bit = d & 31;
    for (int c = 0; c < C; c++) cnt[c * CB + t] = 0;
    const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
    const int64_t r1 = min(N, r0 + rows_per_chunk);
    int64_t upd = 0;
    for (int64_t n = r0; n < r1; n++) {
        const int yc = __ldg(y + n);
        if (yc < 0 || yc >= C) continue;
        int pc = -1;
        if (mode == 1) {
            pc = __ldg(pred + n);
            if (pc == yc) continue;
            upd++;
        }
        if (d < D) {
            const uint32_t w = __ldg(H + n * W + word);
            const int h = 1 - 2 * (int)((w >> bit) & 1u);
            cnt[yc * CB + t] += h;
            if (mode == 1 && pc >= 0 && pc < C) cnt[pc * CB + t] -= h;
        }
    }
    if (d < D)
        for (int c = 0; c < C; c++) {
            const int v = cnt[c * CB + t];
            if (v) atomicAdd(acc + (int64_t)c * D + d, v);
        }
    if (mode == 1 && n_updates && blockIdx.x == 0 && t == 0 && upd) atomicAdd(n_updates, (int)upd);
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

}  // namespace

cudaError_t launch_train_count(const uint32_t *H, int W, const int32_t *y, const int32_t *pred, int64_t N, int D,
                               int C, int mode, int32_t *acc, int32_t *n_updates, cudaStream_t st)
{
    if (N <= 0 || D <= 0 || C <= 0) return cudaSuccess;
    const size_t smem = (size_t)C * CB * sizeof(int32_t);
    if (smem > 200 * 1024) return cudaErrorNotSupported;
    cudaError_t e = cudaFuncSetAttribute(train_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int colb = (D + CB - 1) / CB;
    // enough row chunks for about four blocks per SM, at least 256 rows each
    int64_t chunks = (4 * 152 + colb - 1) / colb;
    int64_t rpc = (N + chunks - 1) / chunks;
    if (rpc < 256) rpc = 256;
    chunks = (N + rpc - 1) / rpc;
    if (chunks > 65535) { chunks = 65535; rpc = (N + chunks - 1) / chunks; }
    dim3 grid(colb, (unsigned)chunks);
    train_count_kernel<<<grid, CB, smem, st>>>(H, W, y, pred, N, D, C, mode, rpc, acc, n_updates);
    return cudaGetLastError();
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
