// hdc_classify_host: classification of query rows that live in host memory
// (copy in, classify, copy labels out, all on the caller's stream).
#include "hdc_internal.cuh"

extern "C" hdc_status hdc_classify_host(const float *const *parts_host, const int64_t *part_rows, int32_t n_parts,
                                        const hdc_model *m, float *X_dev, int32_t *labels_dev,
                                        int32_t *labels_host, void *ws, size_t ws_bytes, hdc_stream_t stream)
{
    if (n_parts < 0 || !m || m->F <= 0 || (n_parts > 0 && (!parts_host || !part_rows))) return HDC_ERR_INVALID_ARG;
    int64_t N = 0;
    for (int32_t i = 0; i < n_parts; i++) {
        if (part_rows[i] < 0 || (part_rows[i] > 0 && !parts_host[i])) return HDC_ERR_INVALID_ARG;
        N += part_rows[i];
    }
    if (N == 0) return HDC_OK;
    if (!X_dev || !labels_dev || !labels_host) return HDC_ERR_INVALID_ARG;
    size_t need = 0;
    hdc_status s = hdc_workspace_bytes(N, m, &need);
    if (s != HDC_OK) return s;
    if (ws_bytes < need) return HDC_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t row_bytes = (size_t)m->F * sizeof(float);
    int64_t r = 0;
    for (int32_t i = 0; i < n_parts; i++) {  // one copy per row block, in order
        if (part_rows[i] == 0) continue;
        if (cudaMemcpyAsync((char *)X_dev + r * row_bytes, parts_host[i], (size_t)part_rows[i] * row_bytes,
                            cudaMemcpyHostToDevice, st) != cudaSuccess)
            return HDC_ERR_CUDA;
        r += part_rows[i];
    }
    s = hdc_classify(X_dev, N, m, labels_dev, nullptr, nullptr, ws, ws_bytes, stream);
    if (s != HDC_OK) return s;
    if (cudaMemcpyAsync(labels_host, labels_dev, (size_t)N * sizeof(int32_t), cudaMemcpyDeviceToHost, st) !=
        cudaSuccess)
        return HDC_ERR_CUDA;
    return HDC_OK;
}
