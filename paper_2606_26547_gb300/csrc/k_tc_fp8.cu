// Tensor-core encoder instances for FP8 E4M3 operands (tcgen05.mma kind::f8f6f4).
#include "tc_fcos.cuh"

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

// Failure-detection self-test: thread 0 waits, through the bounded-wait
// routine of the tensor-core kernels, on an mbarrier that nothing arrives
// on; the expiry records status 1 (timeout) in this unit's status word.
__global__ void __launch_bounds__(32, 1) wait_selftest_kernel(unsigned long long limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(su32(&bar), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (threadIdx.x == 0) (void)mbar_wait(su32(&bar), 0, &abort_flag, limit_ns);
}

}  // namespace tc

cudaError_t launch_wait_selftest(unsigned long long limit_ns, cudaStream_t st)
{
    tc::wait_selftest_kernel<<<1, 32, 0, st>>>(limit_ns);
    return cudaGetLastError();
}

}  // namespace hdc
