// fvv_unet.h -- kernels of the refinement network (not part of the public ABI).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace fvv {

// Arguments of one tensor-core 3x3 convolution (pad 1), NHWC bf16.
struct ConvArgs {
    int NB, H, W, Cin;              // input; Cin % 32 == 0
    int tiles_x;                    // ceil(W / 128), set by the launcher
    const float* bias;              // [Cout] or null
    __nv_bfloat16* y;               // [NB][H][W][Cout]
    int relu;                       // 1: max(0, .)
    const __nv_bfloat16* mask;      // optional [NB][H][W][Cout]: zero where mask <= 0
    int* err;                       // device flag: a bounded wait ran out (never reset here)
};

bool conv_cout_supported(int cout);
cudaError_t make_act_map(CUtensorMap* m, const void* x, int NB, int H, int W, int C);
cudaError_t make_weight_map(CUtensorMap* m, const void* w, int cout, int K);
// y = relu?(conv3x3(x, w) + bias) [* (mask > 0)]; w is bf16 [Cout][3][3][Cin].
cudaError_t launch_conv3x3(const void* x, int NB, int H, int W, int Cin, const void* w, int Cout, ConvArgs a,
                           cudaStream_t s);

}  // namespace fvv
