// fvv_unet.h -- kernels of the refinement network (not part of the public ABI).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

namespace fvv {

// Arguments of one tensor-core 3x3 convolution (pad 1), NHWC.
struct ConvArgs {
    int NB, H, W, Cin;              // input; Cin a multiple of 8 (bf16) or 16 (e4m3)
    int xstride;                    // input channels per pixel in memory (0: Cin); channels
                                    // Cin..xstride-1 are read but must hold zeros
    int tiles_x;                    // tiles per image row, set by the launcher
    int x_quads;                    // set by the launcher: 16-byte pixels copied four to a row
    const float* bias;              // [Cout] or null (16-byte aligned)
    __nv_bfloat16* y;               // output pixel p, channel c at y[p * ldy + coff + c] (e4m3: bytes)
    int ldy, coff;                  // output channel stride (0: Cout) and offset
    int up2;                        // 1: store each output pixel (y, x) at the four pixels
                                    // (2y + dy, 2x + dx) of a [NB][2H][2W][ldy] tensor
    int relu;                       // 1: max(0, .)
    const __nv_bfloat16* mask;      // optional [NB][H][W][Cout] (bf16 only): zero where mask <= 0
    int fp8;                        // 1: x, w and y are e4m3
    float acc_scale;                // accumulator multiplier before the bias (0: 1)
    float out_inv_scale;            // e4m3 output = value * out_inv_scale (0: 1)
    int* err;                       // device flag: a bounded wait ran out (never reset here)
    __nv_bfloat16* pool_y;          // optional (relu, not up2/mask, conv_pool_supported): also the
                                    // 2x2 max pooling [NB][H/2][W/2][Cout] of the output (e4m3: bytes)
    uint8_t* pool_arg;              // optional with pool_y (bf16): the window position 0..3 of each max
    // optional fused 1x1 head (relu, dense output, conv_pool_supported): y is not
    // stored; per pixel p, s = rgb / 255 + head_w d1 + head_b (head_w [3][Cout],
    // d1 the rounded outputs; e4m3: decoded codes times head_scale), then
    // head_out[row * head_pitch + 3 x + k] = round(255 clamp(s_k, 0, 1)) and/or
    // head_f32[3 p + k] = clamp(s_k, 0, 1) (rows of W pixels, images stacked)
    const float* head_w;
    const float* head_b;
    float head_scale;
    const uint8_t* head_rgb;        // [NB * H * W][3]
    uint8_t* head_out;
    size_t head_pitch;
    float* head_f32;
};

// cuTensorMapEncodeTiled from the driver (NULL when it cannot be found).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

bool conv_cout_supported(int cout);
bool conv_pool_supported(int cout);
// y = relu?(acc_scale conv3x3(x, w) + bias) [* (mask > 0)]; w is [Cout][3][3][Cin]
// in the element type of x, Cout one of conv_cout_supported.
cudaError_t launch_conv3x3(const void* x, int NB, int H, int W, int Cin, const void* w, int Cout, ConvArgs a,
                           cudaStream_t s);

}  // namespace fvv

namespace fvv {

// fvv_unet_ops.cu (CUDA-core layers)
cudaError_t launch_pack_features(size_t npx, const uint8_t* rgb, const float* depth, const uint8_t* hole,
                                 const float* top3, float z_far, __nv_bfloat16* out, cudaStream_t s);
// x (pixel stride ldx channels) -> y [B][H/2][W/2][C] and the window position
cudaError_t launch_maxpool2(int B, int H, int W, int C, const __nv_bfloat16* x, int ldx, __nv_bfloat16* y,
                            uint8_t* arg, cudaStream_t s);
// dx = route(dy by arg) + add, zeroed where mask (pixel stride ldm) <= 0
cudaError_t launch_maxpool2_bwd(int B, int H, int W, int C, const __nv_bfloat16* dy, const uint8_t* arg,
                                const __nv_bfloat16* add, const __nv_bfloat16* mask, int ldm, __nv_bfloat16* dx,
                                cudaStream_t s);
// backward of cat = [up2(lo) | skip]: up_act is up2(lo) inside a full-resolution
// tensor of pixel stride ldu (lo's ReLU mask)
cudaError_t launch_up2_concat_bwd(int B, int H, int W, int C1, int C2, const __nv_bfloat16* dcat,
                                  const __nv_bfloat16* up_act, int ldu, __nv_bfloat16* dlo, __nv_bfloat16* dskip,
                                  cudaStream_t s);
bool head_width_supported(int c1);              // w1 of the 1x1 head: 32, 48 or 64
cudaError_t launch_head_fwd(size_t npx, int C1, const __nv_bfloat16* d1, const float* wout, const float* bout,
                            const uint8_t* rgb, float* sbuf, uint8_t* out, int W, size_t out_pitch,
                            float* out_f32, cudaStream_t s);
// Loss, head gradients (overwritten) and dd1, deterministic: scratch holds
// head_bwd_scratch_floats() per-warp partial sums.
constexpr int kHeadPixelsPerWarp = 256;
size_t head_bwd_scratch_floats(size_t npx, int C1);
cudaError_t launch_head_bwd(size_t npx, int C1, const __nv_bfloat16* d1, const float* wout, const float* sbuf,
                            const uint8_t* target, float* loss, float* dwout, float* dbout, __nv_bfloat16* dd1,
                            float* scratch, size_t scratch_floats, cudaStream_t s);
// e4m3 inference forms: activations are e4m3 codes with per-tensor scales
cudaError_t launch_pack_features_e4m3(size_t npx, const uint8_t* rgb, const float* depth, const uint8_t* hole,
                                      const float* top3, float z_far, float s0, uint8_t* out, cudaStream_t s);
cudaError_t launch_maxpool2_e4m3(int B, int H, int W, int C, const uint8_t* x, int ldx, uint8_t* y, cudaStream_t s);
cudaError_t launch_head_fwd_e4m3(size_t npx, int C1, const uint8_t* d1, float s_d1, const float* wout,
                                 const float* bout, const uint8_t* rgb, uint8_t* out, int W, size_t out_pitch,
                                 float* out_f32, cudaStream_t s);
// out = max(out, max |x|) over npix pixels of C channels, pixel stride ld
cudaError_t launch_amax(size_t npix, int C, const __nv_bfloat16* x, int ld, float* out, cudaStream_t s);

// fvv_unet_wgrad.cu (tensor cores): dw[co][3][3][ci] and db[co] (both
// overwritten, fp32) of a 3x3 convolution from its input x ([B][H][W] pixels
// of xstride channels, the first Cin used) and output gradient dz
// ([B][H][W][Cout]).  Cin, xstride and Cout multiples of 8; x, dz 16-byte
// aligned.  scratch holds the per-split partial sums: wgrad_scratch_floats()
// floats give the full split count, fewer give fewer splits (at least
// Cout * (9 Cin + 1) floats).  err: device flag raised when a bounded wait
// runs out.  db may be NULL.
size_t wgrad_scratch_floats(int B, int H, int W, int Cin, int Cout);
cudaError_t launch_wgrad3x3_tc(int B, int H, int W, int Cin, int xstride, int Cout, const __nv_bfloat16* x,
                               const __nv_bfloat16* dz, float* dw, float* db, float* scratch,
                               size_t scratch_floats, int* err, cudaStream_t s);
cudaError_t launch_flip_weights(int Cout, int Cin, const float* w, __nv_bfloat16* wbf, __nv_bfloat16* wt,
                                cudaStream_t s);
// out = sum over splits of part[split][n] in a fixed order (see fvv_unet_ops.cu);
// element i goes to out0[i] (i < n0), out1[i - n0] (i < n0 + n1), else out2.
cudaError_t launch_sum_splits(const float* part, int splits, size_t n, float* out0, size_t n0, float* out1,
                              size_t n1, float* out2, cudaStream_t s);

// Adam over several tensors in one launch (weights of 3x3 layers also
// refresh their bf16 copy wbf and flipped transpose wt when those are set).
constexpr int kAdamMaxTensors = 24;
struct AdamTensor {
    float* w;
    const float* g;
    float* m;
    float* v;
    __nv_bfloat16* wbf;      // or NULL
    __nv_bfloat16* wt;       // or NULL
    int cout, cin;
};
struct AdamList {
    AdamTensor t[kAdamMaxTensors];
    size_t off[kAdamMaxTensors + 1];  // prefix sums of the element counts
    int count;
};
cudaError_t launch_adam_multi(const AdamList& L, float lr, int t, cudaStream_t s);

}  // namespace fvv
