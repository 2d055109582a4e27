// fvv_selftest.cu -- diagnostic of the bounded waits of the tensor-core
// kernels.  One CTA waits on an mbarrier through the same tc::mbar_wait the
// convolution kernel uses; when nothing arrives, the wait must give up after
// its limit, raise the error flag and let the kernel exit normally.
#include "fvv_runtime.h"
#include "fvv_tc.cuh"

namespace fvv {
namespace {

__global__ void k_selftest_wait(int arrive, uint64_t limit_ns, int* err)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        tc::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (arrive) tc::mbar_arrive(&bar);
        tc::mbar_wait(&bar, 0, err, 7, limit_ns);
    }
    __syncthreads();
}

}  // namespace
}  // namespace fvv

using fvv::fail;

fvv_status fvv_selftest_bounded_wait(int32_t arrive, uint32_t limit_us, void* stream)
{
    if (limit_us < 1 || limit_us > 2000000u) return fail(FVV_ERR_INVALID_ARG, "limit_us must be in [1, 2000000]");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int* flag = nullptr;
    FVV_CUDA(cudaMalloc(&flag, sizeof(int)));
    int h = -1;
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        fvv::k_selftest_wait<<<1, 32, 0, s>>>(arrive ? 1 : 0, uint64_t(limit_us) * 1000ull, flag);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(flag);
    if (e != cudaSuccess) return fail(FVV_ERR_CUDA, std::string("fvv_selftest_bounded_wait: ") + cudaGetErrorString(e));
    if (h != 0)
        return fail(FVV_ERR_TIMEOUT, "fvv_selftest_bounded_wait: the wait ran out (code " + std::to_string(h) + ")");
    return FVV_OK;
}
