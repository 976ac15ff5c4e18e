// Auxiliary tensor-core kernels in a translation unit of their own (with
// its own device status word): the Hamming arg-min of packed hypervectors
// and the failure-detection self-test.
#include <string.h>

#include "tc_hamming_packed.cuh"

namespace hdc {

// Tensor map of E4M3 class bytes (Cp rows of ldcs bytes, boxes of 128 bytes x
// Cp rows, 128-byte swizzle), defined with the other map builders.
bool make_class_sign_map(CUtensorMap *m, const uint8_t *signs, int ldcs, int Cp);
namespace tc {

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

bool hamming_packed_ok(int C, int W)
{
    return C > 16 && C <= tc::HP_CMAX && W > 0 && W <= tc::HP_MAX_W && W % 4 == 0;
}

int hamming_packed_ldcs(int W) { return (W + 7) / 8 * 256; }

cudaError_t launch_hamming_packed(const uint32_t *Q, int64_t N, const uint32_t *cls, int C, int W, int64_t D,
                                  int64_t s0, int64_t e0, int64_t stride, int32_t *labels, int32_t *dists,
                                  cudaStream_t st, const uint8_t *cls_sign)
{
    if (N <= 0) return cudaSuccess;
    if (!hamming_packed_ok(C, W) || stride < 1) return cudaErrorNotSupported;
    CUtensorMap mc;
    memset(&mc, 0, sizeof(mc));
    if (cls_sign && !make_class_sign_map(&mc, cls_sign, hamming_packed_ldcs(W), (C + 15) / 16 * 16))
        return cudaErrorInvalidValue;
    tc::HPParams p;
    p.Q = Q;
    p.cls = cls;
    p.N = N;
    p.W = W;
    p.C = C;
    p.Cp = (C + 15) / 16 * 16;
    p.nt = (W + 7) / 8;
    p.D = D;
    p.s0 = s0;
    p.e0 = e0;
    p.stride = stride;
    p.labels = labels;
    p.dists = dists;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                     cudaSuccess || sms <= 0)
        sms = 152;
    const int64_t tiles = (N + tc::BM - 1) / tc::BM;
    // Up to 128 padded classes the query tile lives in tensor memory, two
    // CTAs per SM (256 TMEM columns each, two class-tile buffers).  Above,
    // two CTAs per SM with the query tile in shared memory where they fit
    // (two class-tile buffers, else one), else one CTA with the query tile in
    // tensor memory and all 512 columns: measured, the two-CTA forms win up
    // to ~176 classes (10^5 x 16,384 dims, 144 classes: 0.339 vs 0.377 ms)
    // and the one-CTA tensor-memory form above (256 classes: 0.397 vs 0.459
    // ms with the one-CTA shared-memory form).  The one-CTA form asks for at
    // least 120 KB of shared memory, so that no second CTA shares the SM and
    // waits for its 512 columns.
    auto fits2 = [](size_t bytes) { return 2 * (bytes + 1024) <= 228 * 1024; };
    const size_t smem2 = tc::hp_smem_bytes(p.Cp, W, 2), smem1 = tc::hp_smem_bytes(p.Cp, W, 1);
    const size_t smta = tc::hp_smem_bytes(p.Cp, W, 2, true);
    const int form = p.Cp <= tc::HP_TA_CMAX ? 0 : fits2(smem2) ? 1 : fits2(smem1) ? 2 : 3;
    const bool two = form < 3;
    const size_t smem = form == 0 ? smta : form == 1 ? smem2 : form == 2 ? smem1
                      : (smta >= (size_t)120 * 1024 ? smta : (size_t)120 * 1024);
    auto k = cls_sign ? (form == 0   ? tc::tc_hamming_packed_kernel<2, 2, true, true>
                         : form == 1 ? tc::tc_hamming_packed_kernel<2, 2, true>
                         : form == 2 ? tc::tc_hamming_packed_kernel<2, 1, true>
                                     : tc::tc_hamming_packed_kernel<1, 2, true, true>)
                      : (form == 0   ? tc::tc_hamming_packed_kernel<2, 2, false, true>
                         : form == 1 ? tc::tc_hamming_packed_kernel<2, 2, false>
                         : form == 2 ? tc::tc_hamming_packed_kernel<2, 1, false>
                                     : tc::tc_hamming_packed_kernel<1, 2, false, true>);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t slots = (int64_t)sms * (two ? 2 : 1);
    const unsigned grid = (unsigned)(tiles < slots ? tiles : slots);
    k<<<grid, tc::HP_THREADS, smem, st>>>(p, mc);
    return cudaGetLastError();
}

cudaError_t launch_wait_selftest(unsigned long long limit_ns, cudaStream_t st)
{
    tc::wait_selftest_kernel<<<1, 32, 0, st>>>(limit_ns);
    return cudaGetLastError();
}

cudaError_t tc_aux_read_status(cudaStream_t st, int *status) { return tc::read_status(st, status); }

}  // namespace hdc
