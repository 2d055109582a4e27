// fvv_refine.cu -- C ABI of the refinement network's layer operations.
#include <mutex>
#include <string>

#include "fvv_runtime.h"
#include "fvv_unet.h"

namespace fvv {

namespace {

std::mutex g_flag_mu;
int* g_flags[64] = {};

// A zeroed device int per device: tensor-core kernels raise it when a
// bounded wait runs out.
fvv_status device_flag(int** out)
{
    int dev = 0;
    FVV_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(FVV_ERR_CUDA, "device index out of range");
    std::lock_guard<std::mutex> lk(g_flag_mu);
    if (!g_flags[dev]) {
        FVV_CUDA(cudaMalloc(&g_flags[dev], sizeof(int)));
        FVV_CUDA(cudaMemset(g_flags[dev], 0, sizeof(int)));
    }
    *out = g_flags[dev];
    return FVV_OK;
}

fvv_status check_flag(int* flag, cudaStream_t s, const char* what)
{
    int h = 0;
    FVV_CUDA(cudaMemcpyAsync(&h, flag, sizeof h, cudaMemcpyDeviceToHost, s));
    FVV_CUDA(cudaStreamSynchronize(s));
    if (h) {
        FVV_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), s));
        FVV_CUDA(cudaStreamSynchronize(s));
        return fail(FVV_ERR_TIMEOUT, std::string(what) + ": a bounded wait ran out (code " + std::to_string(h) + ")");
    }
    return FVV_OK;
}

bool on_device(const void* p) { return p && mem_kind(p) == MemKind::Device; }

}  // namespace

}  // namespace fvv

using fvv::fail;

extern "C" {

fvv_status fvv_unet_conv3x3(const void* x, int32_t n, int32_t h, int32_t w, int32_t cin, const void* wt,
                            const float* bias, int32_t cout, int32_t relu, const void* mask, void* y,
                            void* stream)
{
    if (!fvv::on_device(x) || !fvv::on_device(wt) || !fvv::on_device(y))
        return fail(FVV_ERR_INVALID_ARG, "x, w and y must be device memory");
    if ((bias && !fvv::on_device(bias)) || (mask && !fvv::on_device(mask)))
        return fail(FVV_ERR_INVALID_ARG, "bias and mask must be device memory");
    if (n < 1 || h < 1 || w < 1 || cin < 32 || cin % 32 || cin > 4096)
        return fail(FVV_ERR_INVALID_ARG, "need n, h, w >= 1 and cin a multiple of 32");
    if (!fvv::conv_cout_supported(cout))
        return fail(FVV_ERR_INVALID_ARG, "cout must be 32, 64, 96, 128 or 192");
    if (uint64_t(n) * h * ((w + 127) / 128) >= (uint64_t(1) << 31))
        return fail(FVV_ERR_INVALID_ARG, "too many pixel tiles");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int* flag = nullptr;
    FVV_TRY(fvv::device_flag(&flag));
    fvv::ConvArgs a{};
    a.bias = bias;
    a.y = static_cast<__nv_bfloat16*>(y);
    a.relu = relu;
    a.mask = static_cast<const __nv_bfloat16*>(mask);
    a.err = flag;
    FVV_CUDA(fvv::launch_conv3x3(x, n, h, w, cin, wt, cout, a, s));
    return fvv::check_flag(flag, s, "fvv_unet_conv3x3");
}

}  // extern "C"
