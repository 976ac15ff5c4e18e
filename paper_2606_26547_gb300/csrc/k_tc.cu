// Tensor-core (tcgen05) encoder: placeholder until the kernel lands.
#include "hdc_internal.cuh"

namespace hdc {

bool tc_supported(const TcArgs &) { return false; }
cudaError_t launch_tc_encode(const TcArgs &, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t tc_read_status(cudaStream_t, int *status)
{
    *status = 0;
    return cudaSuccess;
}

}  // namespace hdc
