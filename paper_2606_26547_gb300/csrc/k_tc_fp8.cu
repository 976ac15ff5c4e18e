// Tensor-core encoder instances for FP8 E4M3 operands (tcgen05.mma kind::f8f6f4).
#include "tc_fcos16.cuh"

namespace hdc {
namespace tc {

cudaError_t launch_fp8(const CUtensorMap &ma, const CUtensorMap &mb, const CUtensorMap &mc, const Params &p,
                        unsigned grid, bool classify,
                       cudaStream_t st)
{
    return launch_enc<HDC_ENC_FP8_E4M3>(ma, mb, mc, p, grid, classify, st);
}

cudaError_t status_fp8(cudaStream_t st, int *status) { return read_status(st, status); }

cudaError_t launch_hamming_fp8(const CUtensorMap &ma, const CUtensorMap &mb, const CUtensorMap &ms,
                               const HParams &p, unsigned grid, cudaStream_t st)
{
    return launch_hamming_enc<HDC_ENC_FP8_E4M3>(ma, mb, ms, p, grid, st);
}

cudaError_t launch_fcos_fp8(const CUtensorMap &ma, const CUtensorMap &mb, const CUtensorMap &mv,
                         const FCParams &p, unsigned grid, cudaStream_t st)
{
    return launch_fcos_enc<HDC_ENC_FP8_E4M3>(ma, mb, mv, p, grid, st);
}

cudaError_t launch_fcos16_fp8(const CUtensorMap &ma, const CUtensorMap &mb, const CUtensorMap &mv,
                               const CUtensorMap &ms, const FCParams &p, unsigned grid, cudaStream_t st)
{
    return launch_fcos16_enc<HDC_ENC_FP8_E4M3>(ma, mb, mv, ms, p, grid, st);
}

}  // namespace tc
}  // namespace hdc
