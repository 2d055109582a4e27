// fvv_unet_ops.cu -- the refinement network's non-GEMM layers (CUDA cores):
// input packing, 2x2 max pooling, nearest 2x upsampling + channel concat,
// the 1x1 output head with clamp and the mean-squared-error loss, weight and
// bias gradients of the 3x3 convolutions, the weight flip used by the
// transposed (data-gradient) convolution, and Adam.
// All activations are NHWC bf16; gradients of weights and biases are fp32.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "fvv_internal.h"
#include "fvv_unet.h"

namespace fvv {

namespace {

__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }

// ---- input features ----------------------------------------------------------
// 8 channels: RGB / 255, depth / z_far, hole, top-3 weights, stored densely
// in 16 bytes per pixel (bf16: the 8 channels; e4m3: 8 codes and 8 zero
// bytes, the smallest row a tensor map takes).  The convolution's halo copy
// reads these 16 bytes and fills the rest of its 64-byte rows with zeros
// (channels past the tensor's extent), so no padding lives in memory.
__device__ __forceinline__ void features(size_t p, const uint8_t* __restrict__ rgb, const float* __restrict__ depth,
                                         const uint8_t* __restrict__ hole, const float* __restrict__ top3,
                                         float inv_zfar, float f[8])
{
    f[0] = float(rgb[3 * p + 0]) * (1.0f / 255.0f);
    f[1] = float(rgb[3 * p + 1]) * (1.0f / 255.0f);
    f[2] = float(rgb[3 * p + 2]) * (1.0f / 255.0f);
    f[3] = depth[p] * inv_zfar;
    f[4] = float(hole[p]);
    f[5] = top3[3 * p + 0];
    f[6] = top3[3 * p + 1];
    f[7] = top3[3 * p + 2];
}

__global__ void k_pack_features(size_t npx, const uint8_t* __restrict__ rgb, const float* __restrict__ depth,
                                const uint8_t* __restrict__ hole, const float* __restrict__ top3, float inv_zfar,
                                __nv_bfloat16* __restrict__ out)
{
    const size_t p = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (p >= npx) return;
    float f[8];
    features(p, rgb, depth, hole, top3, inv_zfar, f);
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
        w[i] = *reinterpret_cast<const uint32_t*>(&h);
    }
    reinterpret_cast<uint4*>(out)[p] = make_uint4(w[0], w[1], w[2], w[3]);
}

// e4m3 codes of feature / s0 in bytes 0..7, zero in 8..15
__global__ void k_pack_features_e4m3(size_t npx, const uint8_t* __restrict__ rgb, const float* __restrict__ depth,
                                     const uint8_t* __restrict__ hole, const float* __restrict__ top3,
                                     float inv_zfar, float inv_s0, uint8_t* __restrict__ out)
{
    const size_t p = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (p >= npx) return;
    float f[8];
    features(p, rgb, depth, hole, top3, inv_zfar, f);
    uint32_t w[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const __nv_fp8x2_storage_t lo =
            __nv_cvt_float2_to_fp8x2(make_float2(f[4 * i] * inv_s0, f[4 * i + 1] * inv_s0), __NV_SATFINITE, __NV_E4M3);
        const __nv_fp8x2_storage_t hi = __nv_cvt_float2_to_fp8x2(
            make_float2(f[4 * i + 2] * inv_s0, f[4 * i + 3] * inv_s0), __NV_SATFINITE, __NV_E4M3);
        w[i] = uint32_t(lo) | (uint32_t(hi) << 16);
    }
    reinterpret_cast<uint4*>(out)[p] = make_uint4(w[0], w[1], 0u, 0u);
}

// ---- 8-channel vectors: every channel count here is a multiple of 8 ---------
__device__ __forceinline__ void unpack8(const uint4 q, float f[8])
{
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&w[j]);
        f[2 * j] = __bfloat162float(h.x);
        f[2 * j + 1] = __bfloat162float(h.y);
    }
}

__device__ __forceinline__ uint4 pack8(const float f[8])
{
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(f[2 * j], f[2 * j + 1]);
        w[j] = *reinterpret_cast<const uint32_t*>(&h);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

__device__ __forceinline__ uint4 ld8(const __nv_bfloat16* p) { return *reinterpret_cast<const uint4*>(p); }
__device__ __forceinline__ void st8(__nv_bfloat16* p, const uint4 v) { *reinterpret_cast<uint4*>(p) = v; }

// ---- pooling -----------------------------------------------------------------
// One thread per output pixel and 8 channels.  The first maximum of the 2x2
// window, in the order (0,0), (0,1), (1,0), (1,1), wins; its position is kept.
__global__ void k_maxpool2(int B, int H, int W, int C, const __nv_bfloat16* __restrict__ x, int ldx,
                           __nv_bfloat16* __restrict__ y, uint8_t* __restrict__ arg)
{
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int h2 = H / 2, w2 = W / 2, cv = C >> 3;
    const size_t n_out = size_t(B) * h2 * w2 * cv;
    if (i >= n_out) return;
    const int c = int(i % cv) * 8;
    size_t r = i / cv;
    const int ox = int(r % w2);
    r /= w2;
    const int oy = int(r % h2);
    const int b = int(r / h2);
    const size_t base = ((size_t(b) * H + 2 * oy) * W + 2 * ox) * ldx + c;
    const uint4 q[4] = {ld8(x + base), ld8(x + base + ldx), ld8(x + base + size_t(W) * ldx),
                        ld8(x + base + size_t(W) * ldx + ldx)};
    float v[4][8];
#pragma unroll
    for (int k = 0; k < 4; ++k) unpack8(q[k], v[k]);
    const uint16_t* raw[4] = {reinterpret_cast<const uint16_t*>(&q[0]), reinterpret_cast<const uint16_t*>(&q[1]),
                              reinterpret_cast<const uint16_t*>(&q[2]), reinterpret_cast<const uint16_t*>(&q[3])};
    uint16_t outv[8];
    uint8_t outa[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        int a = 0;
#pragma unroll
        for (int k = 1; k < 4; ++k)
            if (v[k][j] > v[a][j]) a = k;
        outa[j] = uint8_t(a);
        outv[j] = a == 0 ? raw[0][j] : a == 1 ? raw[1][j] : a == 2 ? raw[2][j] : raw[3][j];
    }
    const size_t o = i * 8;
    *reinterpret_cast<uint4*>(y + o) = *reinterpret_cast<const uint4*>(outv);
    *reinterpret_cast<uint2*>(arg + o) = *reinterpret_cast<const uint2*>(outa);
}

// dx = route(dy by arg) + add, then zero where mask <= 0 (add, mask nullable);
// one thread per input pixel and 8 channels
__global__ void k_maxpool2_bwd(int B, int H, int W, int C, const __nv_bfloat16* __restrict__ dy,
                               const uint8_t* __restrict__ arg, const __nv_bfloat16* __restrict__ add,
                               const __nv_bfloat16* __restrict__ mask, int ldm, __nv_bfloat16* __restrict__ dx)
{
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int cv = C >> 3;
    const size_t n = size_t(B) * H * W * cv;
    if (i >= n) return;
    const int c = int(i % cv) * 8;
    size_t r = i / cv;
    const size_t r0 = r;                                  // input pixel index
    const int x = int(r % W);
    r /= W;
    const int yy = int(r % H);
    const int b = int(r / H);
    const int h2 = H / 2, w2 = W / 2;
    const size_t j = ((size_t(b) * h2 + yy / 2) * w2 + x / 2) * C + c;
    const int k = (yy & 1) * 2 + (x & 1);
    float g[8], ad[8], m[8];
    unpack8(ld8(dy + j), g);
    const uint2 av = *reinterpret_cast<const uint2*>(arg + j);
    const uint8_t* a8 = reinterpret_cast<const uint8_t*>(&av);
    if (add) unpack8(ld8(add + i * 8), ad);
    if (mask) unpack8(ld8(mask + r0 * ldm + c), m);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        float v = a8[q] == k ? g[q] : 0.0f;
        if (add) v += ad[q];
        if (mask && !(m[q] > 0.0f)) v = 0.0f;
        g[q] = v;
    }
    st8(dx + i * 8, pack8(g));
}

// ---- upsampling + concat (backward) -----------------------------------------
// dlo = (sum over each 2x2 block of dcat[..., 0:C1]) * (lo > 0), lo read from its
// upsampled copy up_act (full resolution, pixel stride ldu); dskip = dcat[..., C1:]
__global__ void k_up2_concat_bwd(int B, int H, int W, int C1, int C2, const __nv_bfloat16* __restrict__ dcat,
                                 const __nv_bfloat16* __restrict__ up_act, int ldu, __nv_bfloat16* __restrict__ dlo,
                                 __nv_bfloat16* __restrict__ dskip)
{
    const int C = C1 + C2, cv1 = C1 >> 3, cv2 = C2 >> 3;
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int h2 = H / 2, w2 = W / 2;
    const size_t n_lo = size_t(B) * h2 * w2 * cv1;
    const size_t n_sk = size_t(B) * H * W * cv2;
    if (i < n_lo) {
        const int c = int(i % cv1) * 8;
        size_t r = i / cv1;
        const int x = int(r % w2);
        r /= w2;
        const int yy = int(r % h2);
        const int b = int(r / h2);
        const size_t p00 = (size_t(b) * H + 2 * yy) * W + 2 * x;
        float s0[8], s1[8], s2[8], s3[8], a[8];
        unpack8(ld8(dcat + p00 * C + c), s0);
        unpack8(ld8(dcat + (p00 + 1) * C + c), s1);
        unpack8(ld8(dcat + (p00 + W) * C + c), s2);
        unpack8(ld8(dcat + (p00 + W + 1) * C + c), s3);
        unpack8(ld8(up_act + p00 * ldu + c), a);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float v = s0[q] + s1[q] + s2[q] + s3[q];
            s0[q] = a[q] > 0.0f ? v : 0.0f;
        }
        st8(dlo + i * 8, pack8(s0));
    }
    if (i < n_sk) {
        const int c = int(i % cv2);
        const size_t p = i / cv2;
        st8(dskip + i * 8, ld8(dcat + p * C + C1 + 8 * c));
    }
}

// ---- e4m3 forms for inference: 16 channels (16 bytes) per thread -------------
__device__ __forceinline__ float e4m3_val(uint8_t b)
{
    return __half2float(__half(__nv_cvt_fp8_to_halfraw(__nv_fp8_storage_t(b), __NV_E4M3)));
}

// 2x2 max pooling of e4m3 codes (one scale in and out); the first maximum wins
__global__ void k_maxpool2_e4m3(int B, int H, int W, int C, const uint8_t* __restrict__ x, int ldx,
                                uint8_t* __restrict__ y)
{
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int h2 = H / 2, w2 = W / 2, cv = C >> 4;
    const size_t n_out = size_t(B) * h2 * w2 * cv;
    if (i >= n_out) return;
    const int c = int(i % cv) * 16;
    size_t r = i / cv;
    const int ox = int(r % w2);
    r /= w2;
    const int oy = int(r % h2);
    const int b = int(r / h2);
    const size_t base = ((size_t(b) * H + 2 * oy) * W + 2 * ox) * ldx + c;
    uint4 q[4];
    q[0] = *reinterpret_cast<const uint4*>(x + base);
    q[1] = *reinterpret_cast<const uint4*>(x + base + ldx);
    q[2] = *reinterpret_cast<const uint4*>(x + base + size_t(W) * ldx);
    q[3] = *reinterpret_cast<const uint4*>(x + base + size_t(W) * ldx + ldx);
    const uint8_t* v[4] = {reinterpret_cast<const uint8_t*>(&q[0]), reinterpret_cast<const uint8_t*>(&q[1]),
                           reinterpret_cast<const uint8_t*>(&q[2]), reinterpret_cast<const uint8_t*>(&q[3])};
    uint8_t o[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        uint8_t best = v[0][j];
        float bv = e4m3_val(best);
#pragma unroll
        for (int k = 1; k < 4; ++k) {
            const float f = e4m3_val(v[k][j]);
            if (f > bv) {
                bv = f;
                best = v[k][j];
            }
        }
        o[j] = best;
    }
    *reinterpret_cast<uint4*>(y + i * 16) = *reinterpret_cast<const uint4*>(o);
}

// ---- 1x1 head ---------------------------------------------------------------
// d1 activations of one pixel as floats: bf16, or e4m3 codes times s_d1
template <int C1>
__device__ __forceinline__ void load_d1(const __nv_bfloat16* d1, size_t p, float a[C1])
{
    const uint4* src = reinterpret_cast<const uint4*>(d1 + size_t(C1) * p);
#pragma unroll
    for (int v = 0; v < C1 / 8; ++v) unpack8(src[v], a + 8 * v);
}

template <int C1>
__device__ __forceinline__ void load_d1(const uint8_t* d1, size_t p, float a[C1], float s_d1)
{
    const uint4* src = reinterpret_cast<const uint4*>(d1 + size_t(C1) * p);
#pragma unroll
    for (int v = 0; v < C1 / 16; ++v) {
        const uint4 q = src[v];
        const uint8_t* b = reinterpret_cast<const uint8_t*>(&q);
#pragma unroll
        for (int j = 0; j < 16; ++j) a[16 * v + j] = e4m3_val(b[j]) * s_d1;
    }
}

// s = rgb / 255 + (W d1 + b); out = round(255 clamp(s, 0, 1)).  T = bf16 or
// e4m3 codes (then scaled by s_d1).
template <int C1, typename T>
__global__ void k_head_fwd(size_t npx, const T* __restrict__ d1, float s_d1, const float* __restrict__ wout,
                           const float* __restrict__ bout, const uint8_t* __restrict__ rgb, float* __restrict__ s,
                           uint8_t* __restrict__ out, int W, size_t out_pitch, float* __restrict__ out_f32)
{
    __shared__ float sw[3 * C1 + 3];
    for (int i = threadIdx.x; i < 3 * C1 + 3; i += blockDim.x) sw[i] = i < 3 * C1 ? wout[i] : bout[i - 3 * C1];
    __syncthreads();
    const size_t p = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (p >= npx) return;
    float a[C1];
    if constexpr (sizeof(T) == 1)
        load_d1<C1>(d1, p, a, s_d1);
    else
        load_d1<C1>(d1, p, a);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float r = sw[3 * C1 + c];
#pragma unroll
        for (int k = 0; k < C1; ++k) r += sw[C1 * c + k] * a[k];
        const float sv = float(rgb[3 * p + c]) * (1.0f / 255.0f) + r;
        if (s) s[3 * p + c] = sv;
        const float pr = fminf(fmaxf(sv, 0.0f), 1.0f);
        if (out_f32) out_f32[3 * p + c] = pr;
        if (out) {
            const size_t y = p / W, x = p % W;
            out[y * out_pitch + 3 * x + c] = uint8_t(floorf(pr * 255.0f + 0.5f));
        }
    }
}

// Loss and the head's backward pass.  diff = clamp(s) - target / 255;
// loss = sum diff^2 inv_count; ds = 2 diff inv_count on 0 < s < 1;
// dW = ds d1^T; db = ds; dd1 = (W^T ds) * (d1 > 0).  Deterministic: warp g
// reduces the fixed pixel range [g ppw, (g + 1) ppw) in pixel order (lane k
// owns output channels k and k + 32 of d1) and writes its partial sums to
// part[g][3 C1 + 4] (dW, db, loss); launch_sum_splits adds them in warp order.
template <int C1>
__global__ void __launch_bounds__(128) k_head_bwd(size_t npx, const __nv_bfloat16* __restrict__ d1,
                                                  const float* __restrict__ wout, const float* __restrict__ s,
                                                  const uint8_t* __restrict__ target, float inv_count, size_t ppw,
                                                  float* __restrict__ part, __nv_bfloat16* __restrict__ dd1)
{
    constexpr int KPL = (C1 + 31) / 32;                 // d1 channels per lane
    __shared__ float sw[3 * C1];
    for (int i = threadIdx.x; i < 3 * C1; i += blockDim.x) sw[i] = wout[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const size_t gw = (size_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const size_t p0 = gw * ppw;
    if (p0 >= npx) return;                              // whole warps leave together
    const size_t p1 = min(npx, p0 + ppw);
    float aw[3][KPL] = {}, ab[3] = {0.0f, 0.0f, 0.0f}, l = 0.0f;
    for (size_t base = p0; base < p1; base += 32) {
        const size_t p = base + lane;
        float ds[3] = {0.0f, 0.0f, 0.0f};
        if (p < p1) {
            float a[C1];
            load_d1<C1>(d1, p, a);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float sv = s[3 * p + c];
                const float d = fminf(fmaxf(sv, 0.0f), 1.0f) - float(target[3 * p + c]) * (1.0f / 255.0f);
                l += d * d;
                ds[c] = (sv > 0.0f && sv < 1.0f) ? 2.0f * d * inv_count : 0.0f;
            }
            float g[C1];
#pragma unroll
            for (int k = 0; k < C1; ++k) {
                const float v = sw[k] * ds[0] + sw[C1 + k] * ds[1] + sw[2 * C1 + k] * ds[2];
                g[k] = a[k] > 0.0f ? v : 0.0f;
            }
            uint4* dst = reinterpret_cast<uint4*>(dd1 + size_t(C1) * p);
#pragma unroll
            for (int v = 0; v < C1 / 8; ++v) dst[v] = pack8(g + 8 * v);
        }
        const int nj = int(min(size_t(32), p1 - base));
        for (int j = 0; j < nj; ++j) {
            const float e0 = __shfl_sync(0xffffffffu, ds[0], j);
            const float e1 = __shfl_sync(0xffffffffu, ds[1], j);
            const float e2 = __shfl_sync(0xffffffffu, ds[2], j);
            const __nv_bfloat16* row = d1 + size_t(C1) * (base + j);
#pragma unroll
            for (int q = 0; q < KPL; ++q) {
                const int k = lane + 32 * q;
                if (k < C1) {
                    const float a = __bfloat162float(row[k]);
                    aw[0][q] += e0 * a;
                    aw[1][q] += e1 * a;
                    aw[2][q] += e2 * a;
                }
            }
            ab[0] += e0;
            ab[1] += e1;
            ab[2] += e2;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    float* out = part + gw * (3 * C1 + 4);
#pragma unroll
    for (int q = 0; q < KPL; ++q) {
        const int k = lane + 32 * q;
        if (k < C1)
            for (int c = 0; c < 3; ++c) out[C1 * c + k] = aw[c][q];
    }
    if (lane == 0) {
        out[3 * C1 + 0] = ab[0];
        out[3 * C1 + 1] = ab[1];
        out[3 * C1 + 2] = ab[2];
        out[3 * C1 + 3] = l * inv_count;
    }
}

// Deterministic sum over splits: out[i] = sum_s part[s][i] (i < n), with a
// fixed association: warp g of a block sums the splits g, g + 8, ... in
// order for 32 consecutive elements, then the eight warp sums are added in
// warp order.  Element i goes to out0[i] (i < n0), out1[i - n0] (i < n0 + n1)
// or out2[i - n0 - n1]; a NULL output is skipped.
__global__ void __launch_bounds__(256) k_sum_splits(const float* __restrict__ part, int splits, size_t n,
                                                    float* out0, size_t n0, float* out1, size_t n1, float* out2)
{
    __shared__ float red[8][32];
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    const size_t i = size_t(blockIdx.x) * 32 + lane;
    float a = 0.0f;
    if (i < n)
        for (int sp = g; sp < splits; sp += 8) a += part[size_t(sp) * n + i];
    red[g][lane] = a;
    __syncthreads();
    if (g != 0 || i >= n) return;
    float t = red[0][lane];
#pragma unroll
    for (int w = 1; w < 8; ++w) t += red[w][lane];
    if (i < n0) {
        if (out0) out0[i] = t;
    } else if (i < n0 + n1) {
        if (out1) out1[i - n0] = t;
    } else if (out2) {
        out2[i - n0 - n1] = t;
    }
}

// wt[ci][ky][kx][co] = w[co][2-ky][2-kx][ci] (bf16), the weights of the
// transposed convolution that gives the input gradient.
__global__ void k_flip_weights(int Cout, int Cin, const float* __restrict__ w, __nv_bfloat16* __restrict__ wbf,
                               __nv_bfloat16* __restrict__ wt)
{
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const size_t n = size_t(Cout) * 9 * Cin;
    if (i >= n) return;
    const int ci = int(i % Cin);
    const int tap = int((i / Cin) % 9);
    const int co = int(i / (size_t(9) * Cin));
    const __nv_bfloat16 v = __float2bfloat16_rn(w[i]);
    wbf[i] = v;
    if (wt) wt[(size_t(ci) * 9 + (8 - tap)) * Cout + co] = v;
}

// Adam over every parameter tensor of the network in one launch; for a 3x3
// layer's weights also the bf16 copy and its flipped transpose (as
// k_flip_weights).  Element e of the concatenation lies in the tensor k with
// off[k] <= e < off[k + 1].
__global__ void k_adam_multi(AdamList L, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const size_t stride = size_t(gridDim.x) * blockDim.x;
    for (size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x; e < L.off[L.count]; e += stride) {
        int lo = 0, hi = L.count - 1;                    // the last k with off[k] <= e
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (L.off[mid] <= e) lo = mid; else hi = mid - 1;
        }
        const AdamTensor& T = L.t[lo];
        const size_t i = e - L.off[lo];
        const float gi = T.g[i];
        const float mi = b1 * T.m[i] + (1.0f - b1) * gi;
        const float vi = b2 * T.v[i] + (1.0f - b2) * gi * gi;
        T.m[i] = mi;
        T.v[i] = vi;
        const float w = T.w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        T.w[i] = w;
        if (T.wbf) {
            const int ci = int(i % T.cin);
            const int tap = int((i / T.cin) % 9);
            const int co = int(i / (size_t(9) * T.cin));
            const __nv_bfloat16 v = __float2bfloat16_rn(w);
            T.wbf[i] = v;
            if (T.wt) T.wt[(size_t(ci) * 9 + (8 - tap)) * T.cout + co] = v;
        }
    }
}

// out = max(out, max |x|) over npix pixels of C channels at pixel stride ld
// (out >= 0 on entry; non-negative floats order like their bits)
__global__ void k_amax(size_t npix, int C, const __nv_bfloat16* __restrict__ x, int ld, float* __restrict__ out)
{
    const int cv = C >> 3;
    const size_t n8 = npix * cv;
    float m = 0.0f;
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n8; i += size_t(gridDim.x) * blockDim.x) {
        float f[8];
        unpack8(ld8(x + (i / cv) * ld + 8 * (i % cv)), f);
#pragma unroll
        for (int j = 0; j < 8; ++j) m = fmaxf(m, fabsf(f[j]));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<unsigned int*>(out), __float_as_uint(m));
}

unsigned blocks(size_t n, int t) { return unsigned((n + t - 1) / t); }

}  // namespace

cudaError_t launch_pack_features(size_t npx, const uint8_t* rgb, const float* depth, const uint8_t* hole,
                                 const float* top3, float z_far, __nv_bfloat16* out, cudaStream_t s)
{
    k_pack_features<<<blocks(npx, 256), 256, 0, s>>>(npx, rgb, depth, hole, top3, 1.0f / z_far, out);
    return cudaGetLastError();
}

cudaError_t launch_maxpool2(int B, int H, int W, int C, const __nv_bfloat16* x, int ldx, __nv_bfloat16* y,
                            uint8_t* arg, cudaStream_t s)
{
    const size_t n = size_t(B) * (H / 2) * (W / 2) * (C / 8);
    k_maxpool2<<<blocks(n, 256), 256, 0, s>>>(B, H, W, C, x, ldx, y, arg);
    return cudaGetLastError();
}

cudaError_t launch_maxpool2_bwd(int B, int H, int W, int C, const __nv_bfloat16* dy, const uint8_t* arg,
                                const __nv_bfloat16* add, const __nv_bfloat16* mask, int ldm, __nv_bfloat16* dx,
                                cudaStream_t s)
{
    const size_t n = size_t(B) * H * W * (C / 8);
    k_maxpool2_bwd<<<blocks(n, 256), 256, 0, s>>>(B, H, W, C, dy, arg, add, mask, ldm, dx);
    return cudaGetLastError();
}

cudaError_t launch_up2_concat_bwd(int B, int H, int W, int C1, int C2, const __nv_bfloat16* dcat,
                                  const __nv_bfloat16* up_act, int ldu, __nv_bfloat16* dlo, __nv_bfloat16* dskip,
                                  cudaStream_t s)
{
    const size_t n_sk = size_t(B) * H * W * (C2 / 8), n_lo = size_t(B) * (H / 2) * (W / 2) * (C1 / 8);
    const size_t n = n_sk > n_lo ? n_sk : n_lo;
    k_up2_concat_bwd<<<blocks(n, 256), 256, 0, s>>>(B, H, W, C1, C2, dcat, up_act, ldu, dlo, dskip);
    return cudaGetLastError();
}

bool head_width_supported(int c1) { return c1 == 32 || c1 == 48 || c1 == 64; }

cudaError_t launch_head_fwd(size_t npx, int C1, const __nv_bfloat16* d1, const float* wout, const float* bout,
                            const uint8_t* rgb, float* sbuf, uint8_t* out, int W, size_t out_pitch,
                            float* out_f32, cudaStream_t s)
{
    switch (C1) {
    case 32: k_head_fwd<32><<<blocks(npx, 128), 128, 0, s>>>(npx, d1, 1.0f, wout, bout, rgb, sbuf, out, W, out_pitch, out_f32); break;
    case 48: k_head_fwd<48><<<blocks(npx, 128), 128, 0, s>>>(npx, d1, 1.0f, wout, bout, rgb, sbuf, out, W, out_pitch, out_f32); break;
    case 64: k_head_fwd<64><<<blocks(npx, 128), 128, 0, s>>>(npx, d1, 1.0f, wout, bout, rgb, sbuf, out, W, out_pitch, out_f32); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_head_fwd_e4m3(size_t npx, int C1, const uint8_t* d1, float s_d1, const float* wout,
                                 const float* bout, const uint8_t* rgb, uint8_t* out, int W, size_t out_pitch,
                                 float* out_f32, cudaStream_t s)
{
    switch (C1) {
    case 32: k_head_fwd<32><<<blocks(npx, 128), 128, 0, s>>>(npx, d1, s_d1, wout, bout, rgb, nullptr, out, W, out_pitch, out_f32); break;
    case 48: k_head_fwd<48><<<blocks(npx, 128), 128, 0, s>>>(npx, d1, s_d1, wout, bout, rgb, nullptr, out, W, out_pitch, out_f32); break;
    case 64: k_head_fwd<64><<<blocks(npx, 128), 128, 0, s>>>(npx, d1, s_d1, wout, bout, rgb, nullptr, out, W, out_pitch, out_f32); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

size_t head_bwd_scratch_floats(size_t npx, int C1)
{
    const size_t nwarps = (npx + kHeadPixelsPerWarp - 1) / kHeadPixelsPerWarp;
    return nwarps * size_t(3 * C1 + 4);
}

cudaError_t launch_head_bwd(size_t npx, int C1, const __nv_bfloat16* d1, const float* wout, const float* sbuf,
                            const uint8_t* target, float* loss, float* dwout, float* dbout, __nv_bfloat16* dd1,
                            float* scratch, size_t scratch_floats, cudaStream_t s)
{
    if (npx == 0 || !scratch || scratch_floats < head_bwd_scratch_floats(npx, C1)) return cudaErrorInvalidValue;
    const float inv = 1.0f / float(npx * 3);
    const size_t ppw = kHeadPixelsPerWarp;
    const size_t nwarps = (npx + ppw - 1) / ppw;
    const unsigned grid = unsigned((nwarps + 3) / 4);
    switch (C1) {
    case 32: k_head_bwd<32><<<grid, 128, 0, s>>>(npx, d1, wout, sbuf, target, inv, ppw, scratch, dd1); break;
    case 48: k_head_bwd<48><<<grid, 128, 0, s>>>(npx, d1, wout, sbuf, target, inv, ppw, scratch, dd1); break;
    case 64: k_head_bwd<64><<<grid, 128, 0, s>>>(npx, d1, wout, sbuf, target, inv, ppw, scratch, dd1); break;
    default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_sum_splits(scratch, int(nwarps), size_t(3 * C1 + 4), dwout, size_t(3 * C1), dbout, 3, loss, s);
}

cudaError_t launch_amax(size_t npix, int C, const __nv_bfloat16* x, int ld, float* out, cudaStream_t s)
{
    unsigned g = blocks(npix * (C / 8), 256);
    const unsigned cap = unsigned(device_sms()) * 8;
    if (g > cap) g = cap;
    if (g == 0) g = 1;
    k_amax<<<g, 256, 0, s>>>(npix, C, x, ld, out);
    return cudaGetLastError();
}

cudaError_t launch_pack_features_e4m3(size_t npx, const uint8_t* rgb, const float* depth, const uint8_t* hole,
                                      const float* top3, float z_far, float s0, uint8_t* out, cudaStream_t s)
{
    k_pack_features_e4m3<<<blocks(npx, 256), 256, 0, s>>>(npx, rgb, depth, hole, top3, 1.0f / z_far, 1.0f / s0, out);
    return cudaGetLastError();
}

cudaError_t launch_maxpool2_e4m3(int B, int H, int W, int C, const uint8_t* x, int ldx, uint8_t* y, cudaStream_t s)
{
    const size_t n = size_t(B) * (H / 2) * (W / 2) * (C / 16);
    k_maxpool2_e4m3<<<blocks(n, 256), 256, 0, s>>>(B, H, W, C, x, ldx, y);
    return cudaGetLastError();
}

cudaError_t launch_flip_weights(int Cout, int Cin, const float* w, __nv_bfloat16* wbf, __nv_bfloat16* wt,
                                cudaStream_t s)
{
    const size_t n = size_t(Cout) * 9 * Cin;
    k_flip_weights<<<blocks(n, 256), 256, 0, s>>>(Cout, Cin, w, wbf, wt);
    return cudaGetLastError();
}

cudaError_t launch_sum_splits(const float* part, int splits, size_t n, float* out0, size_t n0, float* out1,
                              size_t n1, float* out2, cudaStream_t s)
{
    if (n == 0 || splits < 1) return cudaSuccess;
    k_sum_splits<<<unsigned((n + 31) / 32), 256, 0, s>>>(part, splits, n, out0, n0, out1, n1, out2);
    return cudaGetLastError();
}

cudaError_t launch_adam_multi(const AdamList& L, float lr, int t, cudaStream_t s)
{
    if (L.count < 1 || L.count > kAdamMaxTensors) return cudaErrorInvalidValue;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, float(t)), c2 = 1.0f - powf(b2, float(t));
    const size_t n = L.off[L.count];
    unsigned g = blocks(n, 256);
    const unsigned cap = unsigned(device_sms()) * 8;
    if (g > cap) g = cap;
    k_adam_multi<<<g, 256, 0, s>>>(L, lr, b1, b2, 1e-8f, c1, c2);
    return cudaGetLastError();
}

}  // namespace fvv
