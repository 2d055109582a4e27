// fvv_selftest.cu -- diagnostic of the bounded waits of the tensor-core
// kernels.  One CTA waits on an mbarrier through the same tc::mbar_wait the
// convolution kernel uses; when nothing arrives, the wait must give up after
// its limit, raise the error flag and let the kernel exit normally.
#include <cstring>
#include <string>

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

// The persistent serving kernel's bounded waits, on an empty ring: the wait
// for work (barrier = 0: nothing is posted; the kernel returns after its idle
// limit) and a grid barrier (barrier = 1: one batch is posted, but the
// barrier's count starts so far off that it never completes; every CTA gives
// up after the limit and the kernel reports it).  Nothing else is read.
fvv_status fvv_selftest_persistent_wait(int32_t barrier, uint32_t limit_us, void* stream)
{
    if (limit_us < 1 || limit_us > 2000000u) return fail(FVV_ERR_INVALID_ARG, "limit_us must be in [1, 2000000]");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    fvv::PersistQueue* q = nullptr;
    fvv::PersistQueue* qd = nullptr;
    fvv::PersistSync* sync = nullptr;
    FVV_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&q), sizeof(fvv::PersistQueue), cudaHostAllocMapped));
    std::memset(q, 0, sizeof(fvv::PersistQueue));
    cudaError_t e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&qd), q, 0);
    if (e == cudaSuccess) e = cudaMalloc(&sync, sizeof(fvv::PersistSync));
    fvv::PersistSync init{};
    if (barrier) {
        q->posted = 1;                         // work is there, but the first barrier cannot complete
        init.count = 1u << 30;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(sync, &init, sizeof init, cudaMemcpyHostToDevice, s);
    int ctas = 0;
    const uint64_t ns = uint64_t(limit_us) * 1000ull;
    if (e == cudaSuccess)
        e = fvv::launch_serve_persistent(qd, sync, 0, 64, 1, barrier ? 2000000000ull : ns,
                                         barrier ? ns : ns + 2000000000ull, s, &ctas);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    const int err = q->err;
    const uint32_t done = q->done;
    if (sync) cudaFree(sync);
    cudaFreeHost(q);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(FVV_ERR_CUDA, std::string("fvv_selftest_persistent_wait: ") + cudaGetErrorString(e));
    }
    if (done != 0) return fail(FVV_ERR_STATE, "fvv_selftest_persistent_wait: a batch completed on an empty ring");
    if (barrier) {
        if (err != fvv::kPersistErrBarrier)
            return fail(FVV_ERR_STATE, "fvv_selftest_persistent_wait: the barrier did not report its limit");
        return fail(FVV_ERR_TIMEOUT, "fvv_selftest_persistent_wait: barrier wait ran out (code " +
                                         std::to_string(err) + ", " + std::to_string(ctas) + " CTAs)");
    }
    if (err != 0) return fail(FVV_ERR_STATE, "fvv_selftest_persistent_wait: unexpected error code");
    return fail(FVV_ERR_TIMEOUT, "fvv_selftest_persistent_wait: idle wait for work ran out (" +
                                     std::to_string(ctas) + " CTAs)");
}
