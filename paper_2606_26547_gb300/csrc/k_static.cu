// hdc_classify_static: classification whose scratch memory is a fixed array
// compiled into this library, for callers that cannot allocate device memory.
//
// The paper has no counterpart; this is a deployment convenience.  Some hosts
// give a component no way to allocate: a plugin or callback inside a serving
// process whose device memory is owned by someone else's allocator, a
// process that must stay inside a device-memory budget fixed at start-up, or
// a latency-critical loop that may not call cudaMalloc (it can synchronise
// the device).  Such callers pass only their inputs and outputs; the
// quantised queries and packed hypervectors that hdc_classify keeps in the
// caller's workspace live here in g_static_scratch instead.
#include <mutex>

#include "hdc_internal.cuh"

namespace {

// Scratch of hdc_classify_static.  Every GPU that loads libhdc holds these
// HDC_STATIC_SCRATCH_BYTES bytes until the process exits.  Host code may not
// hand the symbol itself to a kernel (on the host it names a host-side
// stand-in); its device address comes from cudaGetSymbolAddress.
__device__ __align__(256) unsigned char g_static_scratch[HDC_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_addr[kMaxDevices];  // device address of g_static_scratch, per device

}  // namespace

extern "C" hdc_status hdc_classify_static(const float *X, int64_t N, const hdc_model *m, int32_t *labels,
                                          int32_t *dists, double *scores, hdc_stream_t stream)
{
    size_t need = 0;
    hdc_status s = hdc_workspace_bytes(N, m, &need);
    if (s != HDC_OK) return s;
    if (need > HDC_STATIC_SCRATCH_BYTES) return HDC_ERR_WORKSPACE;  // too many queries for one call
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HDC_ERR_CUDA;
    void *scratch = nullptr;
    {
        // set-up, once per device, with that device current
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return HDC_ERR_CUDA;
            g_scratch_addr[dev] = p;
        }
        scratch = g_scratch_addr[dev];
    }
    // the workspace path fully writes every scratch byte it later reads, so
    // the array needs no clearing between calls
    return hdc_classify(X, N, m, labels, dists, scores, scratch, HDC_STATIC_SCRATCH_BYTES, stream);
}
