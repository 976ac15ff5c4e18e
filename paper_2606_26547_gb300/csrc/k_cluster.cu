// HD-Clustering (Sec. 5.1): K-means over binary hypervectors, built from the
// classification kernels.  Per iteration:
//   assign   every point to the nearest cluster hypervector: Hamming over the
//            kept dims of the training similarity, arg-min (lowest index on
//            ties)                         -> launch_similarity (K4)
//   changes  points whose cluster differs from the previous iteration
//   update   every cluster hypervector = the bundle of its members (sign of
//            the int32 sum over all D; a cluster without members bundles to
//            zero, i.e. all +1)             -> hdc_train_epoch mode 0 (K5/K6)
// then a final assignment under the inference similarity's kept dims.  The
// two similarity ops are perforated independently, as the paper's tuner
// treats them.
#include <algorithm>

#include "hdc_internal.cuh"

namespace hdc {
namespace {

__global__ void count_changes_kernel(const int32_t *__restrict__ cur, const int32_t *__restrict__ prev, int64_t N,
                                     int first, int32_t *__restrict__ out)
{
    int n = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        n += first || cur[i] != prev[i];
#pragma unroll
    for (int o = 16; o; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(out, n);
}

struct ClusterLayout {
    size_t lab0, lab1, signs, train, total;
};

bool cluster_layout(int64_t N, int D, int K, ClusterLayout *L)
{
    size_t tb = 0;
    if (hdc_train_workspace_bytes(N, D, K, &tb) != HDC_OK) return false;
    size_t off = 0;
    L->lab0 = off;  off = align_up(off + (size_t)N * 4, kAlign);
    L->lab1 = off;  off = align_up(off + (size_t)N * 4, kAlign);
    // the cluster hypervectors expanded to bytes for the assignment (K > 32)
    L->signs = off; off = align_up(off + class_sign_bytes(K, words_for(D)), kAlign);
    L->train = off; off = align_up(off + tb, kAlign);
    L->total = off;
    return true;
}

bool sim_ok(const hdc_approx_config *c)
{
    return !c || (c->struct_size >= sizeof(hdc_approx_config) && c->class_bits == 1);
}

// The kept dims of a similarity op (NULL when every dim of D is kept).
const Perf *perf_or_null(int64_t D, const hdc_approx_config *c, Perf *p)
{
    if (!c || !perf_of(D, c, p)) return nullptr;
    return (p->s0 == 0 && p->e0 == D && p->stride == 1) ? nullptr : p;
}

}  // namespace
}  // namespace hdc

using namespace hdc;

extern "C" hdc_status hdc_cluster_workspace_bytes(int64_t N, int32_t D, int32_t K, size_t *bytes)
{
    ClusterLayout L;
    if (!bytes || N < 0 || D <= 0 || K <= 0) return HDC_ERR_INVALID_ARG;
    if (N > kMaxTrainRows || K > kMaxTrainClasses) return HDC_ERR_UNSUPPORTED;
    if (!cluster_layout(N, D, K, &L)) return HDC_ERR_INVALID_ARG;
    *bytes = L.total;
    return HDC_OK;
}

extern "C" hdc_status hdc_cluster(const uint32_t *H, int64_t N, int32_t D, int32_t K, int32_t iters,
                                  const hdc_approx_config *train_sim, const hdc_approx_config *infer_sim,
                                  uint32_t *cls, int32_t *acc, int32_t *labels, int32_t *changes, void *ws,
                                  size_t ws_bytes, hdc_stream_t stream)
{
    if (N < 0 || D <= 0 || K <= 0 || iters < 0 || !cls || !acc || !labels || !sim_ok(train_sim) ||
        !sim_ok(infer_sim))
        return HDC_ERR_INVALID_ARG;
    // the perforations must keep at least one dim (checked by the Hamming entry on use)
    if (hdc_kept_dims(D, train_sim) <= 0 || hdc_kept_dims(D, infer_sim) <= 0) return HDC_ERR_INVALID_ARG;
    if (N > 0 && (!H || ((uintptr_t)H % 16) != 0)) return HDC_ERR_INVALID_ARG;
    if (((uintptr_t)cls % 16) != 0) return HDC_ERR_INVALID_ARG;
    if (N > kMaxTrainRows || K > kMaxTrainClasses) return HDC_ERR_UNSUPPORTED;
    ClusterLayout L;
    if (!cluster_layout(N, D, K, &L)) return HDC_ERR_INVALID_ARG;
    if (N > 0 && (!ws || ws_bytes < L.total || ((uintptr_t)ws % kAlign) != 0)) return HDC_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    char *w = (char *)ws;
    int32_t *lab[2] = {(int32_t *)(w + L.lab0), (int32_t *)(w + L.lab1)};
    uint8_t *signs = class_sign_bytes(K, words_for(D)) ? (uint8_t *)(w + L.signs) : nullptr;
    const int W = words_for(D);
    Perf pt, pi;
    const Perf *ptrain = perf_or_null(D, train_sim, &pt), *pinfer = perf_or_null(D, infer_sim, &pi);
    if (changes && iters > 0 && cudaMemsetAsync(changes, 0, (size_t)iters * sizeof(int32_t), st) != cudaSuccess)
        return HDC_ERR_CUDA;
    if (N == 0) return HDC_OK;
    for (int t = 0; t < iters; t++) {
        int32_t *cur = lab[t & 1], *prev = lab[(t + 1) & 1];
        if (launch_argmin_ws(H, N, cls, K, W, D, ptrain, cur, signs, st) != cudaSuccess) return HDC_ERR_CUDA;
        if (changes) {
            const int blocks = (int)std::min<int64_t>((N + 255) / 256, 4096);
            count_changes_kernel<<<blocks, 256, 0, st>>>(cur, prev, N, t == 0, changes + t);
            if (cudaGetLastError() != cudaSuccess) return HDC_ERR_CUDA;
        }
        hdc_status s = hdc_train_epoch(H, cur, N, D, K, 0, acc, cls, nullptr, w + L.train, ws_bytes - L.train,
                                       stream);
        if (s != HDC_OK) return s;
    }
    return launch_argmin_ws(H, N, cls, K, W, D, pinfer, labels, signs, st) == cudaSuccess ? HDC_OK : HDC_ERR_CUDA;
}
