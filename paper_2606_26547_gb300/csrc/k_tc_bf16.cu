// Tensor-core encoder instances for BF16 operands (tcgen05.mma kind::f16).
#include "tc_kernel.cuh"

namespace hdc {
namespace tc {

cudaError_t launch_bf16(const CUtensorMap &ma, const CUtensorMap &mb, const CUtensorMap &mc, const Params &p,
                        unsigned grid, bool classify,
                        cudaStream_t st)
{
    return launch_enc<HDC_ENC_BF16>(ma, mb, mc, p, grid, classify, st);
}

cudaError_t status_bf16(cudaStream_t st, int *status) { return read_status(st, status); }

}  // namespace tc
}  // namespace hdc
