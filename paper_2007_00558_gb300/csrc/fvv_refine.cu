// fvv_refine.cu -- the learned refinement of synthesised views: a 3-level
// U-Net trained and run with the library's own kernels (the 3x3
// convolutions and their input gradients on the tcgen05 tensor cores, the
// rest on CUDA cores).  The paper has no learned stage; the network refines
// the plain synthesis (blended RGB, depth, hole mask, top-3 blend weights)
// into a residual added to the blended colour.
//
// Network (widths w1/w2/w3): e1 = conv(conv(x)) [w1]; e2 = conv(conv(pool e1))
// [w2]; bt = conv(conv(pool e2)) [w3]; d2 = conv(conv([up bt | e2])) [w2];
// d1 = conv(conv([up d2 | e1])) [w1]; out = clamp(rgb + W d1 + b, 0, 1).
// 3x3 convolutions with pad 1 and ReLU; 2x2 max pooling; nearest 2x
// upsampling; mean-squared error against the held-out camera; Adam.
// Master weights, gradients and Adam moments are fp32; activations and
// activation gradients are bf16 (NHWC); GEMM accumulation is fp32.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <random>
#include <string>
#include <vector>

#include <cuda_fp8.h>

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

// the 8 input features: 16 bytes per pixel (e4m3: 8 codes, 8 zero bytes)
constexpr int kX0Stride = 8;      // bf16 channels
constexpr int kX0StrideQ = 16;    // e4m3 bytes


}  // namespace

struct ConvLayer {
    int cin_true = 0, cin = 0, cout = 0;
    float *w = nullptr, *b = nullptr, *gw = nullptr, *gb = nullptr;
    float *mw = nullptr, *vw = nullptr, *mb = nullptr, *vb = nullptr;
    __nv_bfloat16 *wbf = nullptr, *wt = nullptr;
    // e4m3 inference: codes [cout][9][cin_q] (cin_q = cin rounded up to 16), scales
    uint8_t* wq = nullptr;
    int cin_q = 0;
    float acc_scale = 1.0f, out_inv_scale = 1.0f;
    size_t nw() const { return size_t(cout) * 9 * cin; }
};

struct RefineNet {
    int w1 = 32, w2 = 64, w3 = 128;
    float z_far = 8000.0f;
    ConvLayer L[10];
    float *wout = nullptr, *bout = nullptr, *gwout = nullptr, *gbout = nullptr;
    float *mwo = nullptr, *vwo = nullptr, *mbo = nullptr, *vbo = nullptr;
    int step = 0;
    std::vector<std::pair<void*, size_t>> params;     // device allocations of parameters
    // activations (and their gradients) for up to `cap` pixels: every buffer
    // is dense NHWC over the batch, so any (B, H, W) with B*H*W <= cap and H, W
    // multiples of 4 fits at the full, half and quarter resolutions
    size_t cap = 0, gcap = 0;
    std::vector<std::pair<void*, size_t>> acts, grads;
    __nv_bfloat16 *x0, *e1a, *p1, *e2a, *p2, *ba, *cat2, *d2a, *cat1, *d1a, *d1;
    uint8_t *arg1, *arg2;
    float* s;
    __nv_bfloat16 *g_d1b, *g_d1a, *g_cat1, *g_skip1, *g_d2b, *g_d2a, *g_cat2, *g_skip2, *g_bb, *g_ba, *g_p2,
        *g_e2b, *g_e2a, *g_p1, *g_e1b, *g_e1a;
    float* loss = nullptr;
    // per-split partial sums of the tensor-core weight gradients
    float* wscratch = nullptr;
    size_t wscratch_floats = 0;
    // e4m3 inference: per-tensor scales of the ten conv outputs, the input
    // scale, and e4m3 activations for (qB, qH, qW)
    int precision = FVV_PREC_BF16;
    bool q_ready = false;
    float s_act[10] = {};
    float s0 = 1.0f / 256.0f;
    float* amax = nullptr;
    size_t qcap = 0;                                  // e4m3 activations, pixels
    std::vector<std::pair<void*, size_t>> acts8;
    uint8_t *q_x0, *q_e1a, *q_p1, *q_e2a, *q_p2, *q_ba, *q_cat2, *q_d2a, *q_cat1, *q_d1a, *q_d1;
    // plain-synthesis outputs feeding fvv_synthesize_refined
    int sH = 0, sW = 0;
    std::vector<std::pair<void*, size_t>> syn;
    uint8_t *syn_rgb = nullptr, *syn_hole = nullptr, *syn_out = nullptr;
    float *syn_depth = nullptr, *syn_top3 = nullptr;
};

namespace {

fvv_status alloc_into(fvv_ctx* c, std::vector<std::pair<void*, size_t>>& list, void** p, size_t bytes)
{
    FVV_TRY(dev_alloc(c, p, bytes));
    list.push_back({*p, bytes});
    return FVV_OK;
}

void free_list(fvv_ctx* c, std::vector<std::pair<void*, size_t>>& list)
{
    for (auto& a : list) dev_free(c, a.first, a.second);
    list.clear();
}

template <class T>
fvv_status alloc_t(fvv_ctx* c, std::vector<std::pair<void*, size_t>>& list, T** p, size_t n)
{
    void* v = nullptr;
    FVV_TRY(alloc_into(c, list, &v, n * sizeof(T)));
    *p = static_cast<T*>(v);
    return FVV_OK;
}

// parameters in the flat host layout: per 3x3 layer W[cout][3][3][cin_true]
// then b[cout]; then the head W[3][w1] and b[3]
size_t flat_count(const RefineNet& N)
{
    size_t n = 0;
    for (const ConvLayer& l : N.L) n += size_t(l.cout) * 9 * l.cin_true + l.cout;
    return n + 3 * size_t(N.w1) + 3;
}

enum class Buf { Param, Grad, M, V };

void layer_bufs(ConvLayer& l, Buf b, float** w, float** bias)
{
    switch (b) {
    case Buf::Param: *w = l.w; *bias = l.b; break;
    case Buf::Grad: *w = l.gw; *bias = l.gb; break;
    case Buf::M: *w = l.mw; *bias = l.mb; break;
    case Buf::V: *w = l.vw; *bias = l.vb; break;
    }
}

void head_bufs(RefineNet& N, Buf b, float** w, float** bias)
{
    switch (b) {
    case Buf::Param: *w = N.wout; *bias = N.bout; break;
    case Buf::Grad: *w = N.gwout; *bias = N.gbout; break;
    case Buf::M: *w = N.mwo; *bias = N.mbo; break;
    case Buf::V: *w = N.vwo; *bias = N.vbo; break;
    }
}

fvv_status get_flat(RefineNet& N, Buf which, float* out)
{
    size_t o = 0;
    std::vector<float> tmp;
    for (ConvLayer& l : N.L) {
        float *w, *b;
        layer_bufs(l, which, &w, &b);
        tmp.resize(l.nw());
        FVV_CUDA(cudaMemcpy(tmp.data(), w, l.nw() * 4, cudaMemcpyDeviceToHost));
        for (int co = 0; co < l.cout; ++co)
            for (int t = 0; t < 9; ++t)
                for (int ci = 0; ci < l.cin_true; ++ci)
                    out[o++] = tmp[(size_t(co) * 9 + t) * l.cin + ci];
        FVV_CUDA(cudaMemcpy(out + o, b, size_t(l.cout) * 4, cudaMemcpyDeviceToHost));
        o += l.cout;
    }
    float *w, *b;
    head_bufs(N, which, &w, &b);
    FVV_CUDA(cudaMemcpy(out + o, w, size_t(3) * N.w1 * 4, cudaMemcpyDeviceToHost));
    o += 3 * size_t(N.w1);
    FVV_CUDA(cudaMemcpy(out + o, b, 3 * 4, cudaMemcpyDeviceToHost));
    return FVV_OK;
}

fvv_status refresh_weights(RefineNet& N, cudaStream_t s)
{
    N.q_ready = false;                        // e4m3 weights are stale
    N.precision = FVV_PREC_BF16;
    for (ConvLayer& l : N.L)
        FVV_CUDA(launch_flip_weights(l.cout, l.cin, l.w, l.wbf, l.wt, s));
    return FVV_OK;
}

fvv_status set_flat(RefineNet& N, Buf which, const float* in, cudaStream_t s)
{
    size_t o = 0;
    std::vector<float> tmp;
    for (ConvLayer& l : N.L) {
        float *w, *b;
        layer_bufs(l, which, &w, &b);
        tmp.assign(l.nw(), 0.0f);
        for (int co = 0; co < l.cout; ++co)
            for (int t = 0; t < 9; ++t)
                for (int ci = 0; ci < l.cin_true; ++ci)
                    tmp[(size_t(co) * 9 + t) * l.cin + ci] = in[o++];
        FVV_CUDA(cudaMemcpy(w, tmp.data(), l.nw() * 4, cudaMemcpyHostToDevice));
        FVV_CUDA(cudaMemcpy(b, in + o, size_t(l.cout) * 4, cudaMemcpyHostToDevice));
        o += l.cout;
    }
    float *w, *b;
    head_bufs(N, which, &w, &b);
    FVV_CUDA(cudaMemcpy(w, in + o, size_t(3) * N.w1 * 4, cudaMemcpyHostToDevice));
    o += 3 * size_t(N.w1);
    FVV_CUDA(cudaMemcpy(b, in + o, 3 * 4, cudaMemcpyHostToDevice));
    if (which == Buf::Param) FVV_TRY(refresh_weights(N, s));
    return FVV_OK;
}

fvv_status ensure_acts(fvv_ctx* c, RefineNet& N, size_t pixels)
{
    if (pixels <= N.cap) return FVV_OK;
    FVV_CUDA(cudaDeviceSynchronize());
    free_list(c, N.acts);
    N.cap = 0;
    const size_t p1 = pixels, p2 = p1 / 4, p3 = p1 / 16;
    const int w1 = N.L[1].cout, w2 = N.L[3].cout, w3 = N.L[5].cout;
    auto A = [&](__nv_bfloat16** p, size_t n) { return alloc_t(c, N.acts, p, n); };
    FVV_TRY(A(&N.x0, p1 * kX0Stride));
    FVV_TRY(A(&N.e1a, p1 * w1));
    FVV_TRY(A(&N.p1, p2 * w1));
    FVV_TRY(A(&N.e2a, p2 * w2));
    FVV_TRY(A(&N.p2, p3 * w2));
    FVV_TRY(A(&N.ba, p3 * w3));
    FVV_TRY(A(&N.cat2, p2 * (w3 + w2)));
    FVV_TRY(A(&N.d2a, p2 * w2));
    FVV_TRY(A(&N.cat1, p1 * (w2 + w1)));
    FVV_TRY(A(&N.d1a, p1 * w1));
    FVV_TRY(A(&N.d1, p1 * w1));
    FVV_TRY(alloc_t(c, N.acts, &N.arg1, p2 * w1));
    FVV_TRY(alloc_t(c, N.acts, &N.arg2, p3 * w2));
    FVV_TRY(alloc_t(c, N.acts, &N.s, p1 * 3));
    FVV_CUDA(cudaDeviceSynchronize());
    N.cap = pixels;
    return FVV_OK;
}

// Activation gradients (training) for up to `pixels` pixels.
fvv_status ensure_grads(fvv_ctx* c, RefineNet& N, size_t pixels)
{
    if (pixels <= N.gcap) return FVV_OK;
    FVV_CUDA(cudaDeviceSynchronize());
    free_list(c, N.grads);
    N.gcap = 0;
    const size_t p1 = pixels, p2 = p1 / 4, p3 = p1 / 16;
    const int w1 = N.L[1].cout, w2 = N.L[3].cout, w3 = N.L[5].cout;
    auto A = [&](__nv_bfloat16** p, size_t n) { return alloc_t(c, N.grads, p, n); };
    FVV_TRY(A(&N.g_d1b, p1 * w1));
    FVV_TRY(A(&N.g_d1a, p1 * w1));
    FVV_TRY(A(&N.g_cat1, p1 * (w2 + w1)));
    FVV_TRY(A(&N.g_skip1, p1 * w1));
    FVV_TRY(A(&N.g_d2b, p2 * w2));
    FVV_TRY(A(&N.g_d2a, p2 * w2));
    FVV_TRY(A(&N.g_cat2, p2 * (w3 + w2)));
    FVV_TRY(A(&N.g_skip2, p2 * w2));
    FVV_TRY(A(&N.g_bb, p3 * w3));
    FVV_TRY(A(&N.g_ba, p3 * w3));
    FVV_TRY(A(&N.g_p2, p3 * w2));
    FVV_TRY(A(&N.g_e2b, p2 * w2));
    FVV_TRY(A(&N.g_e2a, p2 * w2));
    FVV_TRY(A(&N.g_p1, p2 * w1));
    FVV_TRY(A(&N.g_e1b, p1 * w1));
    FVV_TRY(A(&N.g_e1a, p1 * w1));
    N.gcap = pixels;
    return FVV_OK;
}

// Partial sums of the weight-gradient kernels for a batch of B images H x W:
// the largest layer's full split count, capped at 64 MiB (the kernels then
// use fewer splits).
fvv_status ensure_wscratch(fvv_ctx* c, RefineNet& N, int B, int H, int W)
{
    size_t need = 0;
    const int hs[10] = {H, H, H / 2, H / 2, H / 4, H / 4, H / 2, H / 2, H, H};
    const int ws[10] = {W, W, W / 2, W / 2, W / 4, W / 4, W / 2, W / 2, W, W};
    for (int i = 0; i < 10; ++i)
        need = std::max(need, wgrad_scratch_floats(B, hs[i], ws[i], N.L[i].cin, N.L[i].cout));
    need = std::min(need, size_t(16) << 20);             // 64 MiB
    for (int i = 0; i < 10; ++i)                          // but one split of every layer
        need = std::max(need, size_t(N.L[i].cout) * (9 * size_t(N.L[i].cin) + 1));
    // the head's backward pass uses the same buffer first
    need = std::max(need, head_bwd_scratch_floats(size_t(B) * H * W, N.L[9].cout));
    if (need <= N.wscratch_floats) return FVV_OK;
    FVV_CUDA(cudaDeviceSynchronize());
    if (N.wscratch) dev_free(c, N.wscratch, N.wscratch_floats * 4);
    N.wscratch = nullptr;
    N.wscratch_floats = 0;
    void* p = nullptr;
    FVV_TRY(dev_alloc(c, &p, need * 4));
    N.wscratch = static_cast<float*>(p);
    N.wscratch_floats = need;
    return FVV_OK;
}

// Where a conv writes: channel stride and offset of the output, whether it
// stores the 2x nearest upsampling (into a concatenation's first part), and
// optionally the 2x2 max pooling of the output (and its window positions).
struct Out {
    int ldy = 0, coff = 0, up2 = 0;
    void* pool_y = nullptr;
    uint8_t* pool_arg = nullptr;
};

// The 1x1 head fused into the last convolution (inference only: the
// activations d1 are then never stored).
struct Head {
    const float *w = nullptr, *b = nullptr;
    float scale = 1.0f;
    const uint8_t* rgb = nullptr;
    uint8_t* out = nullptr;
    size_t pitch = 0;
    float* f32 = nullptr;
};

void set_head(ConvArgs& a, const Head& h)
{
    a.head_w = h.w;
    a.head_b = h.b;
    a.head_scale = h.scale;
    a.head_rgb = h.rgb;
    a.head_out = h.out;
    a.head_pitch = h.pitch;
    a.head_f32 = h.f32;
}

fvv_status conv(const ConvLayer& l, const __nv_bfloat16* x, int B, int H, int W, __nv_bfloat16* y, int* err,
                cudaStream_t s, int xstride = 0, Out o = Out(), Head h = Head())
{
    ConvArgs a{};
    set_head(a, h);
    a.ldy = o.ldy;
    a.coff = o.coff;
    a.up2 = o.up2;
    a.pool_y = static_cast<__nv_bfloat16*>(o.pool_y);
    a.pool_arg = o.pool_arg;
    a.bias = l.b;
    a.y = y;
    a.relu = 1;
    a.err = err;
    a.xstride = xstride;
    FVV_CUDA(launch_conv3x3(x, B, H, W, l.cin, l.wbf, l.cout, a, s));
    return FVV_OK;
}

// weight and bias gradients of layer l (tensor cores, written whole), and its
// input gradient (masked).  The input gradient is the convolution of dz with
// the flipped weights wt[ci][ky][kx][co]; for a concatenated input (split >
// 0) it runs once per part, ci in [0, split) and [split, cin), into channel
// slices of dx.
fvv_status conv_bwd(const RefineNet& N, const ConvLayer& l, const __nv_bfloat16* x, const __nv_bfloat16* dz, int B,
                    int H, int W, __nv_bfloat16* dx, const __nv_bfloat16* mask, int* err, cudaStream_t s,
                    int split = 0, int xstride = 0)
{
    FVV_CUDA(launch_wgrad3x3_tc(B, H, W, l.cin, xstride ? xstride : l.cin, l.cout, x, dz, l.gw, l.gb, N.wscratch,
                                N.wscratch_floats, err, s));
    if (dx) {
        const int parts = split > 0 ? 2 : 1;
        for (int p = 0; p < parts; ++p) {
            const int c0 = p == 0 ? 0 : split;
            const int n = parts == 1 ? l.cin : (p == 0 ? split : l.cin - split);
            ConvArgs a{};
            a.y = dx;
            a.ldy = l.cin;
            a.coff = c0;
            a.relu = 0;
            a.mask = parts == 1 ? mask : nullptr;
            a.err = err;
            FVV_CUDA(launch_conv3x3(dz, B, H, W, l.cout, l.wt + size_t(c0) * 9 * l.cout, n, a, s));
        }
    }
    return FVV_OK;
}

fvv_status forward(RefineNet& N, const fvv_refine_batch& b, int* err, cudaStream_t s, uint8_t* out,
                   size_t out_pitch, float* out_f32)
{
    const int B = b.n, H = b.height, W = b.width;
    const size_t npx = size_t(B) * H * W;
    const int H2 = H / 2, W2 = W / 2, H4 = H / 4, W4 = W / 4;
    const int w1 = N.L[1].cout, w2 = N.L[3].cout, w3 = N.L[5].cout;
    // e1b and e2b write straight into the second part of the concatenations
    // cat1 = [up2(d2b) | e1b] and cat2 = [up2(bb) | e2b]; bb and d2b write their
    // 2x upsampling into the first parts.  No separate copies of e1b, e2b,
    // bb or d2b exist.
    const int l1 = w2 + w1, l2 = w3 + w2;
    FVV_CUDA(launch_pack_features(npx, b.rgb, b.depth, b.hole, b.top3, N.z_far, N.x0, s));
    FVV_TRY(conv(N.L[0], N.x0, B, H, W, N.e1a, err, s, kX0Stride));
    // the pooling runs in the epilogue of the conv before it where the tile
    // shape allows (cout <= 64), else as a kernel of its own
    const bool fp1 = conv_pool_supported(w1), fp2 = conv_pool_supported(w2);
    FVV_TRY(conv(N.L[1], N.e1a, B, H, W, N.cat1, err, s, 0, Out{l1, w2, 0, fp1 ? N.p1 : nullptr, fp1 ? N.arg1 : nullptr}));
    if (!fp1) FVV_CUDA(launch_maxpool2(B, H, W, w1, N.cat1 + w2, l1, N.p1, N.arg1, s));
    FVV_TRY(conv(N.L[2], N.p1, B, H2, W2, N.e2a, err, s));
    FVV_TRY(conv(N.L[3], N.e2a, B, H2, W2, N.cat2, err, s, 0, Out{l2, w3, 0, fp2 ? N.p2 : nullptr, fp2 ? N.arg2 : nullptr}));
    if (!fp2) FVV_CUDA(launch_maxpool2(B, H2, W2, w2, N.cat2 + w3, l2, N.p2, N.arg2, s));
    FVV_TRY(conv(N.L[4], N.p2, B, H4, W4, N.ba, err, s));
    FVV_TRY(conv(N.L[5], N.ba, B, H4, W4, N.cat2, err, s, 0, Out{l2, 0, 1}));
    FVV_TRY(conv(N.L[6], N.cat2, B, H2, W2, N.d2a, err, s));
    FVV_TRY(conv(N.L[7], N.d2a, B, H2, W2, N.cat1, err, s, 0, Out{l1, 0, 1}));
    FVV_TRY(conv(N.L[8], N.cat1, B, H, W, N.d1a, err, s));
    if (out || out_f32) {
        // inference: the head runs in d1b's epilogue (d1 and s are training state)
        Head h;
        h.w = N.wout;
        h.b = N.bout;
        h.rgb = b.rgb;
        h.out = out;
        h.pitch = out_pitch;
        h.f32 = out_f32;
        FVV_TRY(conv(N.L[9], N.d1a, B, H, W, N.d1, err, s, 0, Out(), h));
        return FVV_OK;
    }
    FVV_TRY(conv(N.L[9], N.d1a, B, H, W, N.d1, err, s));
    FVV_CUDA(launch_head_fwd(npx, w1, N.d1, N.wout, N.bout, b.rgb, N.s, out, W, out_pitch, out_f32, s));
    return FVV_OK;
}

fvv_status backward(RefineNet& N, const fvv_refine_batch& b, int* err, cudaStream_t s)
{
    const int B = b.n, H = b.height, W = b.width;
    const size_t npx = size_t(B) * H * W;
    const int H2 = H / 2, W2 = W / 2, H4 = H / 4, W4 = W / 4;
    const int w1 = N.L[1].cout, w2 = N.L[3].cout, w3 = N.L[5].cout;
    FVV_CUDA(launch_head_bwd(npx, w1, N.d1, N.wout, N.s, b.target, N.loss, N.gwout, N.gbout, N.g_d1b, N.wscratch,
                             N.wscratch_floats, s));
    FVV_TRY(conv_bwd(N, N.L[9], N.d1a, N.g_d1b, B, H, W, N.g_d1a, N.d1a, err, s));
    FVV_TRY(conv_bwd(N, N.L[8], N.cat1, N.g_d1a, B, H, W, N.g_cat1, nullptr, err, s, w2));
    FVV_CUDA(launch_up2_concat_bwd(B, H, W, w2, w1, N.g_cat1, N.cat1, w2 + w1, N.g_d2b, N.g_skip1, s));
    FVV_TRY(conv_bwd(N, N.L[7], N.d2a, N.g_d2b, B, H2, W2, N.g_d2a, N.d2a, err, s));
    FVV_TRY(conv_bwd(N, N.L[6], N.cat2, N.g_d2a, B, H2, W2, N.g_cat2, nullptr, err, s, w3));
    FVV_CUDA(launch_up2_concat_bwd(B, H2, W2, w3, w2, N.g_cat2, N.cat2, w3 + w2, N.g_bb, N.g_skip2, s));
    FVV_TRY(conv_bwd(N, N.L[5], N.ba, N.g_bb, B, H4, W4, N.g_ba, N.ba, err, s));
    FVV_TRY(conv_bwd(N, N.L[4], N.p2, N.g_ba, B, H4, W4, N.g_p2, nullptr, err, s));
    FVV_CUDA(launch_maxpool2_bwd(B, H2, W2, w2, N.g_p2, N.arg2, N.g_skip2, N.cat2 + w3, w3 + w2, N.g_e2b, s));
    FVV_TRY(conv_bwd(N, N.L[3], N.e2a, N.g_e2b, B, H2, W2, N.g_e2a, N.e2a, err, s));
    FVV_TRY(conv_bwd(N, N.L[2], N.p1, N.g_e2a, B, H2, W2, N.g_p1, nullptr, err, s));
    FVV_CUDA(launch_maxpool2_bwd(B, H, W, w1, N.g_p1, N.arg1, N.g_skip1, N.cat1 + w2, w2 + w1, N.g_e1b, s));
    FVV_TRY(conv_bwd(N, N.L[1], N.e1a, N.g_e1b, B, H, W, N.g_e1a, N.e1a, err, s));
    FVV_TRY(conv_bwd(N, N.L[0], N.x0, N.g_e1a, B, H, W, nullptr, nullptr, err, s, 0, kX0Stride));
    return FVV_OK;
}

fvv_status ensure_acts8(fvv_ctx* c, RefineNet& N, size_t pixels)
{
    if (pixels <= N.qcap) return FVV_OK;
    FVV_CUDA(cudaDeviceSynchronize());
    free_list(c, N.acts8);
    N.qcap = 0;
    const size_t p1 = pixels, p2 = p1 / 4, p3 = p1 / 16;
    const int w1 = N.L[1].cout, w2 = N.L[3].cout, w3 = N.L[5].cout;
    auto A = [&](uint8_t** p, size_t n) { return alloc_t(c, N.acts8, p, n); };
    FVV_TRY(A(&N.q_x0, p1 * kX0StrideQ));
    FVV_TRY(A(&N.q_e1a, p1 * w1));
    FVV_TRY(A(&N.q_p1, p2 * w1));
    FVV_TRY(A(&N.q_e2a, p2 * w2));
    FVV_TRY(A(&N.q_p2, p3 * w2));
    FVV_TRY(A(&N.q_ba, p3 * w3));
    FVV_TRY(A(&N.q_cat2, p2 * (w3 + w2)));
    FVV_TRY(A(&N.q_d2a, p2 * w2));
    FVV_TRY(A(&N.q_cat1, p1 * (w2 + w1)));
    FVV_TRY(A(&N.q_d1a, p1 * w1));
    FVV_TRY(A(&N.q_d1, p1 * w1));
    N.qcap = pixels;
    return FVV_OK;
}

fvv_status conv_e4m3(const ConvLayer& l, const uint8_t* x, int B, int H, int W, uint8_t* y, int* err,
                     cudaStream_t s, int xstride = 0, Out o = Out(), Head h = Head())
{
    ConvArgs a{};
    set_head(a, h);
    a.ldy = o.ldy;
    a.coff = o.coff;
    a.up2 = o.up2;
    a.pool_y = static_cast<__nv_bfloat16*>(o.pool_y);
    a.bias = l.b;
    a.y = reinterpret_cast<__nv_bfloat16*>(y);
    a.relu = 1;
    a.fp8 = 1;
    a.acc_scale = l.acc_scale;
    a.out_inv_scale = l.out_inv_scale;
    a.err = err;
    a.xstride = xstride;
    FVV_CUDA(launch_conv3x3(x, B, H, W, l.cin_q, l.wq, l.cout, a, s));
    return FVV_OK;
}

// The forward pass on e4m3 codes (weights and scales from quantize()).
fvv_status forward_e4m3(RefineNet& N, const fvv_refine_batch& b, int* err, cudaStream_t s, uint8_t* out,
                        size_t out_pitch, float* out_f32)
{
    const int B = b.n, H = b.height, W = b.width;
    const size_t npx = size_t(B) * H * W;
    const int H2 = H / 2, W2 = W / 2, H4 = H / 4, W4 = W / 4;
    const int w1 = N.L[1].cout, w2 = N.L[3].cout, w3 = N.L[5].cout;
    FVV_CUDA(launch_pack_features_e4m3(npx, b.rgb, b.depth, b.hole, b.top3, N.z_far, N.s0, N.q_x0, s));
    const int l1 = w2 + w1, l2 = w3 + w2;                 // concatenations written in place
    FVV_TRY(conv_e4m3(N.L[0], N.q_x0, B, H, W, N.q_e1a, err, s, kX0StrideQ));
    const bool fp1 = conv_pool_supported(w1), fp2 = conv_pool_supported(w2);
    FVV_TRY(conv_e4m3(N.L[1], N.q_e1a, B, H, W, N.q_cat1, err, s, 0, Out{l1, w2, 0, fp1 ? N.q_p1 : nullptr}));
    if (!fp1) FVV_CUDA(launch_maxpool2_e4m3(B, H, W, w1, N.q_cat1 + w2, l1, N.q_p1, s));
    FVV_TRY(conv_e4m3(N.L[2], N.q_p1, B, H2, W2, N.q_e2a, err, s));
    FVV_TRY(conv_e4m3(N.L[3], N.q_e2a, B, H2, W2, N.q_cat2, err, s, 0, Out{l2, w3, 0, fp2 ? N.q_p2 : nullptr}));
    if (!fp2) FVV_CUDA(launch_maxpool2_e4m3(B, H2, W2, w2, N.q_cat2 + w3, l2, N.q_p2, s));
    FVV_TRY(conv_e4m3(N.L[4], N.q_p2, B, H4, W4, N.q_ba, err, s));
    FVV_TRY(conv_e4m3(N.L[5], N.q_ba, B, H4, W4, N.q_cat2, err, s, 0, Out{l2, 0, 1}));
    FVV_TRY(conv_e4m3(N.L[6], N.q_cat2, B, H2, W2, N.q_d2a, err, s));
    FVV_TRY(conv_e4m3(N.L[7], N.q_d2a, B, H2, W2, N.q_cat1, err, s, 0, Out{l1, 0, 1}));
    FVV_TRY(conv_e4m3(N.L[8], N.q_cat1, B, H, W, N.q_d1a, err, s));
    if (out || out_f32) {
        Head h;                                           // the head runs in d1b's epilogue
        h.w = N.wout;
        h.b = N.bout;
        h.scale = N.s_act[9];
        h.rgb = b.rgb;
        h.out = out;
        h.pitch = out_pitch;
        h.f32 = out_f32;
        FVV_TRY(conv_e4m3(N.L[9], N.q_d1a, B, H, W, N.q_d1, err, s, 0, Out(), h));
        return FVV_OK;
    }
    FVV_TRY(conv_e4m3(N.L[9], N.q_d1a, B, H, W, N.q_d1, err, s));
    FVV_CUDA(launch_head_fwd_e4m3(npx, w1, N.q_d1, N.s_act[9], N.wout, N.bout, b.rgb, out, W, out_pitch, out_f32,
                                  s));
    return FVV_OK;
}

// Scales of the input parts of layer i: {scale, channels} in channel order.
int input_parts(const RefineNet& N, int i, float sc[2], int ch[2])
{
    const int w1 = N.L[1].cout, w2 = N.L[3].cout, w3 = N.L[5].cout;
    const float* a = N.s_act;
    switch (i) {
    case 0: sc[0] = N.s0; ch[0] = 8; return 1;
    case 1: sc[0] = a[0]; ch[0] = w1; return 1;
    case 2: sc[0] = a[1]; ch[0] = w1; return 1;       // max pooling keeps e1b's scale
    case 3: sc[0] = a[2]; ch[0] = w2; return 1;
    case 4: sc[0] = a[3]; ch[0] = w2; return 1;
    case 5: sc[0] = a[4]; ch[0] = w3; return 1;
    case 6: sc[0] = a[5]; ch[0] = w3; sc[1] = a[3]; ch[1] = w2; return 2;    // [up(bb) | e2b]
    case 7: sc[0] = a[6]; ch[0] = w2; return 1;
    case 8: sc[0] = a[7]; ch[0] = w2; sc[1] = a[1]; ch[1] = w1; return 2;    // [up(d2b) | e1b]
    default: sc[0] = a[8]; ch[0] = w1; return 1;
    }
}

// e4m3 weight codes and multipliers of every layer from the fp32 masters and
// the activation scales in N.s_act (host arithmetic, one pass per quantisation).
fvv_status quantize_weights(RefineNet& N, cudaStream_t s)
{
    std::vector<float> w;
    std::vector<uint8_t> q;
    for (int i = 0; i < 10; ++i) {
        ConvLayer& l = N.L[i];
        w.resize(l.nw());
        FVV_CUDA(cudaMemcpy(w.data(), l.w, l.nw() * 4, cudaMemcpyDeviceToHost));
        float sc[2] = {1.0f, 1.0f};
        int ch[2] = {l.cin, 0};
        const int np = input_parts(N, i, sc, ch);
        std::vector<float> f(l.cin, 1.0f);            // per input channel: s_part / s_first_part
        if (np == 2)
            for (int c = ch[0]; c < l.cin; ++c) f[c] = sc[1] / sc[0];
        float amax = 0.0f;
        for (int co = 0; co < l.cout; ++co)
            for (int t = 0; t < 9; ++t)
                for (int ci = 0; ci < l.cin; ++ci)
                    amax = std::max(amax, std::fabs(w[(size_t(co) * 9 + t) * l.cin + ci] * f[ci]));
        const float sw = amax > 0.0f ? amax / 448.0f : 1.0f;
        q.assign(size_t(l.cout) * 9 * l.cin_q, 0);
        for (int co = 0; co < l.cout; ++co)
            for (int t = 0; t < 9; ++t)
                for (int ci = 0; ci < l.cin; ++ci)
                    q[(size_t(co) * 9 + t) * l.cin_q + ci] = uint8_t(__nv_cvt_float_to_fp8(
                        w[(size_t(co) * 9 + t) * l.cin + ci] * f[ci] / sw, __NV_SATFINITE, __NV_E4M3));
        FVV_CUDA(cudaMemcpyAsync(l.wq, q.data(), q.size(), cudaMemcpyHostToDevice, s));
        FVV_CUDA(cudaStreamSynchronize(s));
        l.acc_scale = sc[0] * sw;
        l.out_inv_scale = 1.0f / N.s_act[i];
    }
    return FVV_OK;
}

fvv_status adam(RefineNet& N, float lr, cudaStream_t s)
{
    const int t = ++N.step;
    // every tensor in one launch; the 3x3 weights refresh their bf16 copies
    // (and the flipped transposes of the input gradients) as they update
    AdamList L{};
    auto add = [&](float* w, const float* g, float* m, float* v, size_t n, __nv_bfloat16* wbf,
                   __nv_bfloat16* wt, int cout, int cin) {
        AdamTensor& T = L.t[L.count];
        T = AdamTensor{w, g, m, v, wbf, wt, cout, cin};
        L.off[L.count + 1] = L.off[L.count] + n;
        ++L.count;
    };
    for (ConvLayer& l : N.L) {
        add(l.w, l.gw, l.mw, l.vw, l.nw(), l.wbf, l.wt, l.cout, l.cin);
        add(l.b, l.gb, l.mb, l.vb, size_t(l.cout), nullptr, nullptr, 0, 1);
    }
    add(N.wout, N.gwout, N.mwo, N.vwo, size_t(3) * N.w1, nullptr, nullptr, 0, 1);
    add(N.bout, N.gbout, N.mbo, N.vbo, 3, nullptr, nullptr, 0, 1);
    FVV_CUDA(launch_adam_multi(L, lr, t, s));
    N.q_ready = false;                        // e4m3 weights are stale
    N.precision = FVV_PREC_BF16;
    return FVV_OK;
}

fvv_status check_batch(const RefineNet& N, const fvv_refine_batch* b, bool need_target)
{
    if (!b) return fail(FVV_ERR_INVALID_ARG, "batch is NULL");
    if (b->n < 1 || b->height < 4 || b->width < 4 || b->height % 4 || b->width % 4)
        return fail(FVV_ERR_INVALID_ARG, "batch size >= 1, height and width multiples of 4");
    if (!on_device(b->rgb) || !on_device(b->depth) || !on_device(b->hole) || !on_device(b->top3))
        return fail(FVV_ERR_INVALID_ARG, "batch inputs must be device memory");
    if (need_target && !on_device(b->target)) return fail(FVV_ERR_INVALID_ARG, "target must be device memory");
    (void)N;
    return FVV_OK;
}

RefineNet* net_of(fvv_ctx* c) { return c ? c->refine : nullptr; }

}  // namespace

void refine_destroy(fvv_ctx* c)
{
    RefineNet* N = c->refine;
    if (!N) return;
    cudaDeviceSynchronize();
    free_list(c, N->acts);
    free_list(c, N->grads);
    free_list(c, N->acts8);
    free_list(c, N->syn);
    free_list(c, N->params);
    if (N->wscratch) dev_free(c, N->wscratch, N->wscratch_floats * 4);
    delete N;
    c->refine = nullptr;
}

bool refine_ready(fvv_ctx* c) { return c && c->refine; }

fvv_status refine_reserve(fvv_ctx* c, size_t pixels)
{
    RefineNet* N = c->refine;
    if (!N) return fail(FVV_ERR_STATE, "refinement network not initialised");
    fvv::DeviceScope dev_scope(c->device);
    return N->precision == FVV_PREC_E4M3 ? ensure_acts8(c, *N, pixels) : ensure_acts(c, *N, pixels);
}

fvv_status refine_forward_async(fvv_ctx* c, const fvv_refine_batch& b, uint8_t* out_rgb, cudaStream_t s)
{
    RefineNet* N = c->refine;
    if (!N) return fail(FVV_ERR_STATE, "refinement network not initialised");
    fvv::DeviceScope dev_scope(c->device);
    int* err = nullptr;
    FVV_TRY(device_flag(&err));
    const size_t px = size_t(b.n) * b.height * b.width;
    if (N->precision == FVV_PREC_E4M3) {
        FVV_TRY(ensure_acts8(c, *N, px));
        return forward_e4m3(*N, b, err, s, out_rgb, size_t(b.width) * 3, nullptr);
    }
    FVV_TRY(ensure_acts(c, *N, px));
    return forward(*N, b, err, s, out_rgb, size_t(b.width) * 3, nullptr);
}

fvv_status refine_error_flag(int** flag) { return device_flag(flag); }

}  // namespace fvv

using fvv::fail;
using fvv::RefineNet;

extern "C" {

fvv_status fvv_unet_conv3x3(const void* x, int32_t n, int32_t h, int32_t w, int32_t cin, const void* wt,
                            const float* bias, int32_t cout, int32_t relu, const void* mask, void* y,
                            void* stream)
{
    if (!fvv::on_device(x) || !fvv::on_device(wt) || !fvv::on_device(y))
        return fail(FVV_ERR_INVALID_ARG, "x, w and y must be device memory");
    if ((bias && !fvv::on_device(bias)) || (mask && !fvv::on_device(mask)))
        return fail(FVV_ERR_INVALID_ARG, "bias and mask must be device memory");
    if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(wt) | reinterpret_cast<uintptr_t>(y) |
         reinterpret_cast<uintptr_t>(bias) | reinterpret_cast<uintptr_t>(mask)) & 15u)
        return fail(FVV_ERR_INVALID_ARG, "x, w, bias, mask and y must be 16-byte aligned");
    if (n < 1 || h < 1 || w < 1 || cin < 8 || cin % 8 || cin > 4096)
        return fail(FVV_ERR_INVALID_ARG, "need n, h, w >= 1 and cin a multiple of 8");
    if (!fvv::conv_cout_supported(cout))
        return fail(FVV_ERR_INVALID_ARG, "cout must be 32, 48, 64, 96, 128 or 192");
    if (uint64_t(n) * h * ((w + 119) / 120) >= (uint64_t(1) << 31))
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

fvv_status fvv_unet_wgrad3x3(const void* x, int32_t n, int32_t h, int32_t w, int32_t cin, int32_t xstride,
                            const void* dz, int32_t cout, float* dw, float* db, void* stream)
{
    if (!fvv::on_device(x) || !fvv::on_device(dz) || !fvv::on_device(dw) || (db && !fvv::on_device(db)))
        return fail(FVV_ERR_INVALID_ARG, "x, dz, dw and db must be device memory");
    if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(dz)) & 15u)
        return fail(FVV_ERR_INVALID_ARG, "x and dz must be 16-byte aligned");
    if (xstride == 0) xstride = cin;
    if (n < 1 || h < 1 || w < 1 || cin < 8 || cin % 8 || cin > 4096 || xstride < cin || xstride % 8 ||
        cout < 8 || cout % 8 || cout > 4096)
        return fail(FVV_ERR_INVALID_ARG, "need n, h, w >= 1, cin, xstride >= cin and cout multiples of 8");
    if (uint64_t(n) * h * w >= (uint64_t(1) << 31))
        return fail(FVV_ERR_INVALID_ARG, "too many pixels");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int* flag = nullptr;
    FVV_TRY(fvv::device_flag(&flag));
    const size_t nf = fvv::wgrad_scratch_floats(n, h, w, cin, cout);
    float* scratch = nullptr;
    FVV_CUDA(cudaMalloc(&scratch, nf * sizeof(float)));
    cudaError_t e = fvv::launch_wgrad3x3_tc(n, h, w, cin, xstride, cout, static_cast<const __nv_bfloat16*>(x),
                                            static_cast<const __nv_bfloat16*>(dz), dw, db, scratch, nf, flag, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(scratch);
    FVV_CUDA(e);
    return fvv::check_flag(flag, s, "fvv_unet_wgrad3x3");
}

fvv_status fvv_unet_conv3x3_e4m3(const void* x, int32_t n, int32_t h, int32_t w, int32_t cin, const void* wt,
                                 const float* bias, int32_t cout, int32_t relu, float acc_scale, float out_inv_scale,
                                 void* y, void* stream)
{
    if (!fvv::on_device(x) || !fvv::on_device(wt) || !fvv::on_device(y))
        return fail(FVV_ERR_INVALID_ARG, "x, w and y must be device memory");
    if (bias && !fvv::on_device(bias)) return fail(FVV_ERR_INVALID_ARG, "bias must be device memory");
    if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(wt) | reinterpret_cast<uintptr_t>(y) |
         reinterpret_cast<uintptr_t>(bias)) & 15u)
        return fail(FVV_ERR_INVALID_ARG, "x, w, bias and y must be 16-byte aligned");
    if (n < 1 || h < 1 || w < 1 || cin < 16 || cin % 16 || cin > 4096)
        return fail(FVV_ERR_INVALID_ARG, "need n, h, w >= 1 and cin a multiple of 16");
    if (!fvv::conv_cout_supported(cout))
        return fail(FVV_ERR_INVALID_ARG, "cout must be 32, 48, 64, 96, 128 or 192");
    if (!(acc_scale > 0.0f) || !(out_inv_scale > 0.0f) || !std::isfinite(acc_scale) || !std::isfinite(out_inv_scale))
        return fail(FVV_ERR_INVALID_ARG, "scales must be finite and > 0");
    if (uint64_t(n) * h * ((w + 119) / 120) >= (uint64_t(1) << 31))
        return fail(FVV_ERR_INVALID_ARG, "too many pixel tiles");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int* flag = nullptr;
    FVV_TRY(fvv::device_flag(&flag));
    fvv::ConvArgs a{};
    a.bias = bias;
    a.y = static_cast<__nv_bfloat16*>(y);
    a.relu = relu;
    a.fp8 = 1;
    a.acc_scale = acc_scale;
    a.out_inv_scale = out_inv_scale;
    a.err = flag;
    FVV_CUDA(fvv::launch_conv3x3(x, n, h, w, cin, wt, cout, a, s));
    return fvv::check_flag(flag, s, "fvv_unet_conv3x3_e4m3");
}

fvv_status fvv_unet_conv3x3_pool(const void* x, int32_t n, int32_t h, int32_t w, int32_t cin, const void* wt,
                                 const float* bias, int32_t cout, int32_t e4m3, float acc_scale,
                                 float out_inv_scale, void* y, void* pool_y, uint8_t* pool_arg, void* stream)
{
    if (!fvv::on_device(x) || !fvv::on_device(wt) || !fvv::on_device(y) || !fvv::on_device(pool_y))
        return fail(FVV_ERR_INVALID_ARG, "x, w, y and pool_y must be device memory");
    if ((bias && !fvv::on_device(bias)) || (pool_arg && !fvv::on_device(pool_arg)))
        return fail(FVV_ERR_INVALID_ARG, "bias and pool_arg must be device memory");
    if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(wt) | reinterpret_cast<uintptr_t>(y) |
         reinterpret_cast<uintptr_t>(bias) | reinterpret_cast<uintptr_t>(pool_y) |
         reinterpret_cast<uintptr_t>(pool_arg)) & 15u)
        return fail(FVV_ERR_INVALID_ARG, "every pointer must be 16-byte aligned");
    if (e4m3 != 0 && e4m3 != 1) return fail(FVV_ERR_INVALID_ARG, "e4m3 must be 0 or 1");
    if (e4m3 && pool_arg) return fail(FVV_ERR_INVALID_ARG, "pool_arg is bf16 only");
    const int q = e4m3 ? 16 : 8;
    if (n < 1 || h < 1 || w < 1 || cin < q || cin % q || cin > 4096)
        return fail(FVV_ERR_INVALID_ARG, "need n, h, w >= 1 and cin a multiple of 8 (e4m3: 16)");
    if (!fvv::conv_pool_supported(cout)) return fail(FVV_ERR_INVALID_ARG, "cout must be 32, 48 or 64");
    if (e4m3 && (!(acc_scale > 0.0f) || !(out_inv_scale > 0.0f) || !std::isfinite(acc_scale) ||
                 !std::isfinite(out_inv_scale)))
        return fail(FVV_ERR_INVALID_ARG, "scales must be finite and > 0");
    if (uint64_t(n) * h * ((w + 119) / 120) >= (uint64_t(1) << 31))
        return fail(FVV_ERR_INVALID_ARG, "too many pixel tiles");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int* flag = nullptr;
    FVV_TRY(fvv::device_flag(&flag));
    fvv::ConvArgs a{};
    a.bias = bias;
    a.y = static_cast<__nv_bfloat16*>(y);
    a.relu = 1;
    a.fp8 = e4m3;
    if (e4m3) {
        a.acc_scale = acc_scale;
        a.out_inv_scale = out_inv_scale;
    }
    a.pool_y = static_cast<__nv_bfloat16*>(pool_y);
    a.pool_arg = pool_arg;
    a.err = flag;
    FVV_CUDA(fvv::launch_conv3x3(x, n, h, w, cin, wt, cout, a, s));
    return fvv::check_flag(flag, s, "fvv_unet_conv3x3_pool");
}

fvv_status fvv_refine_default_cfg(fvv_unet_cfg* cfg)
{
    if (!cfg) return fail(FVV_ERR_INVALID_ARG, "cfg is NULL");
    cfg->widths[0] = 32;
    cfg->widths[1] = 64;
    cfg->widths[2] = 128;
    cfg->seed = 0;
    cfg->z_far = 8000.0f;
    return FVV_OK;
}

fvv_status fvv_refine_init(fvv_ctx* c, const fvv_unet_cfg* cfg_in)
{
    if (!c) return fail(FVV_ERR_INVALID_ARG, "ctx is NULL");
    fvv::DeviceScope dev_scope(c->device);
    fvv_unet_cfg cfg;
    if (cfg_in) cfg = *cfg_in; else fvv_refine_default_cfg(&cfg);
    // every forward output width and every part of every input gradient is a
    // supported conv width; the head takes w1 in {32, 48, 64}
    for (int i = 0; i < 3; ++i)
        if (!fvv::conv_cout_supported(cfg.widths[i]))
            return fail(FVV_ERR_INVALID_ARG, "widths must each be 32, 48, 64, 96, 128 or 192");
    if (!fvv::head_width_supported(cfg.widths[0]))
        return fail(FVV_ERR_INVALID_ARG, "the first width must be 32, 48 or 64");
    if (!(cfg.z_far > 0.0f)) return fail(FVV_ERR_INVALID_ARG, "z_far must be > 0");
    std::lock_guard<std::recursive_mutex> g(c->mu);
    if (fvv::serve_refining(c)) return fail(FVV_ERR_BUSY, "the serving loop is running the refinement network");
    FVV_CUDA(cudaSetDevice(c->device));
    fvv::refine_destroy(c);
    auto* N = new RefineNet();
    c->refine = N;
    N->w1 = cfg.widths[0];
    N->w2 = cfg.widths[1];
    N->w3 = cfg.widths[2];
    N->z_far = cfg.z_far;
    const int w1 = N->w1, w2 = N->w2, w3 = N->w3;
    const int cins[10] = {8, w1, w1, w2, w2, w3, w3 + w2, w2, w2 + w1, w1};
    const int couts[10] = {w1, w1, w2, w2, w3, w3, w2, w2, w1, w1};
    auto P = [&](float** p, size_t n) { return fvv::alloc_t(c, N->params, p, n); };
    auto PB = [&](__nv_bfloat16** p, size_t n) { return fvv::alloc_t(c, N->params, p, n); };
    fvv_status rc = FVV_OK;
    for (int i = 0; i < 10 && rc == FVV_OK; ++i) {
        fvv::ConvLayer& l = N->L[i];
        l.cin_true = cins[i];
        l.cin = cins[i];
        l.cin_q = (cins[i] + 15) / 16 * 16;
        l.cout = couts[i];
        const size_t nw = l.nw();
        if ((rc = P(&l.w, nw)) || (rc = P(&l.gw, nw)) || (rc = P(&l.mw, nw)) || (rc = P(&l.vw, nw)) ||
            (rc = P(&l.b, l.cout)) || (rc = P(&l.gb, l.cout)) || (rc = P(&l.mb, l.cout)) ||
            (rc = P(&l.vb, l.cout)) || (rc = PB(&l.wbf, nw)) || (rc = PB(&l.wt, nw)) ||
            (rc = fvv::alloc_t(c, N->params, &l.wq, size_t(l.cout) * 9 * l.cin_q)))
            break;
    }
    if (rc == FVV_OK) {
        float** hp[10] = {&N->wout, &N->bout, &N->gwout, &N->gbout, &N->mwo,
                          &N->vwo,  &N->mbo,  &N->vbo,   &N->loss,  &N->amax};
        const size_t hn[10] = {3 * size_t(w1), 3, 3 * size_t(w1), 3, 3 * size_t(w1), 3 * size_t(w1), 3, 3, 1, 10};
        for (int i = 0; i < 10 && rc == FVV_OK; ++i) rc = P(hp[i], hn[i]);
    }
    if (rc != FVV_OK) {
        std::string msg = fvv_last_error();
        fvv::refine_destroy(c);
        return fail(rc, msg);
    }
    for (auto& a : N->params) FVV_CUDA(cudaMemset(a.first, 0, a.second));
    // He-normal 3x3 weights, zero biases, a small head
    std::mt19937_64 rng(cfg.seed);
    std::normal_distribution<float> nd(0.0f, 1.0f);
    std::vector<float> flat(fvv::flat_count(*N));
    size_t o = 0;
    for (fvv::ConvLayer& l : N->L) {
        const float sd = std::sqrt(2.0f / (9.0f * float(l.cin_true)));
        for (size_t k = 0; k < size_t(l.cout) * 9 * l.cin_true; ++k) flat[o++] = sd * nd(rng);
        for (int k = 0; k < l.cout; ++k) flat[o++] = 0.0f;
    }
    const float sd = 0.1f * std::sqrt(1.0f / float(w1));
    for (int k = 0; k < 3 * w1; ++k) flat[o++] = sd * nd(rng);
    for (int k = 0; k < 3; ++k) flat[o++] = 0.0f;
    FVV_TRY(fvv::set_flat(*N, fvv::Buf::Param, flat.data(), c->own));
    FVV_CUDA(cudaStreamSynchronize(c->own));
    return FVV_OK;
}

fvv_status fvv_refine_param_count(fvv_ctx* c, uint64_t* n)
{
    RefineNet* N = fvv::net_of(c);
    if (!N || !n) return fail(FVV_ERR_STATE, "refinement network not initialised");
    *n = fvv::flat_count(*N);
    return FVV_OK;
}

fvv_status fvv_refine_get(fvv_ctx* c, int32_t which, float* out)
{
    RefineNet* N = fvv::net_of(c);
    if (!N) return fail(FVV_ERR_STATE, "refinement network not initialised");
    fvv::DeviceScope dev_scope(c->device);
    if (!out || which < 0 || which > 3) return fail(FVV_ERR_INVALID_ARG, "bad buffer selector or NULL");
    std::lock_guard<std::recursive_mutex> g(c->mu);
    FVV_CUDA(cudaDeviceSynchronize());
    return fvv::get_flat(*N, fvv::Buf(which), out);
}

fvv_status fvv_refine_set(fvv_ctx* c, int32_t which, const float* in)
{
    RefineNet* N = fvv::net_of(c);
    if (!N) return fail(FVV_ERR_STATE, "refinement network not initialised");
    fvv::DeviceScope dev_scope(c->device);
    if (!in || which < 0 || which > 3) return fail(FVV_ERR_INVALID_ARG, "bad buffer selector or NULL");
    std::lock_guard<std::recursive_mutex> g(c->mu);
    if (fvv::serve_refining(c)) return fail(FVV_ERR_BUSY, "the serving loop is running the refinement network");
    FVV_CUDA(cudaDeviceSynchronize());
    FVV_TRY(fvv::set_flat(*N, fvv::Buf(which), in, c->own));
    FVV_CUDA(cudaStreamSynchronize(c->own));
    return FVV_OK;
}

fvv_status fvv_refine_forward(fvv_ctx* c, const fvv_refine_batch* b, uint8_t* out_rgb, float* out_f32,
                              void* stream)
{
    RefineNet* N = fvv::net_of(c);
    if (!N) return fail(FVV_ERR_STATE, "refinement network not initialised");
    fvv::DeviceScope dev_scope(c->device);
    FVV_TRY(fvv::check_batch(*N, b, false));
    if ((out_rgb && !fvv::on_device(out_rgb)) || (out_f32 && !fvv::on_device(out_f32)))
        return fail(FVV_ERR_INVALID_ARG, "outputs must be device memory");
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : c->own;
    std::lock_guard<std::recursive_mutex> g(c->mu);
    if (fvv::serve_refining(c)) return fail(FVV_ERR_BUSY, "the serving loop is running the refinement network");
    int* err = nullptr;
    FVV_TRY(fvv::device_flag(&err));
    if (N->precision == FVV_PREC_E4M3) {
        FVV_TRY(fvv::ensure_acts8(c, *N, size_t(b->n) * b->height * b->width));
        FVV_TRY(fvv::forward_e4m3(*N, *b, err, s, out_rgb, size_t(b->width) * 3, out_f32));
    } else {
        FVV_TRY(fvv::ensure_acts(c, *N, size_t(b->n) * b->height * b->width));
        FVV_TRY(fvv::forward(*N, *b, err, s, out_rgb, size_t(b->width) * 3, out_f32));
    }
    return fvv::check_flag(err, s, "fvv_refine_forward");
}

fvv_status fvv_refine_quantize(fvv_ctx* c, const fvv_refine_batch* calib, const float* act_scales, void* stream)
{
    RefineNet* N = fvv::net_of(c);
    if (!N) return fail(FVV_ERR_STATE, "refinement network not initialised");
    fvv::DeviceScope dev_scope(c->device);
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : c->own;
    std::lock_guard<std::recursive_mutex> g(c->mu);
    if (fvv::serve_refining(c)) return fail(FVV_ERR_BUSY, "the serving loop is running the refinement network");
    float sc[10];
    if (act_scales) {
        for (int i = 0; i < 10; ++i) {
            if (!(act_scales[i] > 0.0f) || !std::isfinite(act_scales[i]))
                return fail(FVV_ERR_INVALID_ARG, "activation scales must be finite and > 0");
            sc[i] = act_scales[i];
        }
    } else {
        FVV_TRY(fvv::check_batch(*N, calib, false));
        int* err = nullptr;
        FVV_TRY(fvv::device_flag(&err));
        FVV_TRY(fvv::ensure_acts(c, *N, size_t(calib->n) * calib->height * calib->width));
        FVV_TRY(fvv::forward(*N, *calib, err, s, nullptr, 0, nullptr));
        FVV_TRY(fvv::check_flag(err, s, "fvv_refine_quantize"));
        const size_t p1 = size_t(calib->n) * calib->height * calib->width, p2 = p1 / 4, p3 = p1 / 16;
        const int w1 = N->L[1].cout, w2 = N->L[3].cout, w3 = N->L[5].cout;
        // e1b, e2b, bb, d2b live inside the concatenations (bb and d2b upsampled:
        // the same maximum)
        const __nv_bfloat16* t[10] = {N->e1a, N->cat1 + w2, N->e2a, N->cat2 + w3, N->ba,
                                      N->cat2, N->d2a, N->cat1, N->d1a, N->d1};
        const size_t np[10] = {p1, p1, p2, p2, p3, p2, p2, p1, p1, p1};
        const int ld[10] = {w1, w2 + w1, w2, w3 + w2, w3, w3 + w2, w2, w2 + w1, w1, w1};
        FVV_CUDA(cudaMemsetAsync(N->amax, 0, 10 * sizeof(float), s));
        for (int i = 0; i < 10; ++i)
            FVV_CUDA(fvv::launch_amax(np[i], N->L[i].cout, t[i], ld[i], N->amax + i, s));
        float am[10];
        FVV_CUDA(cudaMemcpyAsync(am, N->amax, sizeof am, cudaMemcpyDeviceToHost, s));
        FVV_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i < 10; ++i) sc[i] = am[i] > 0.0f && std::isfinite(am[i]) ? am[i] / 448.0f : 1.0f;
    }
    for (int i = 0; i < 10; ++i) N->s_act[i] = sc[i];
    FVV_TRY(fvv::quantize_weights(*N, s));
    N->q_ready = true;
    N->precision = FVV_PREC_E4M3;
    return FVV_OK;
}

fvv_status fvv_refine_set_precision(fvv_ctx* c, int32_t precision)
{
    RefineNet* N = fvv::net_of(c);
    if (!N) return fail(FVV_ERR_STATE, "refinement network not initialised");
    fvv::DeviceScope dev_scope(c->device);
    if (precision != FVV_PREC_BF16 && precision != FVV_PREC_E4M3)
        return fail(FVV_ERR_INVALID_ARG, "precision must be FVV_PREC_BF16 or FVV_PREC_E4M3");
    std::lock_guard<std::recursive_mutex> g(c->mu);
    if (fvv::serve_refining(c)) return fail(FVV_ERR_BUSY, "the serving loop is running the refinement network");
    if (precision == FVV_PREC_E4M3 && !N->q_ready)
        return fail(FVV_ERR_STATE, "no current e4m3 weights: call fvv_refine_quantize");
    N->precision = precision;
    return FVV_OK;
}

fvv_status fvv_refine_get_precision(fvv_ctx* c, int32_t* precision, float* act_scales)
{
    RefineNet* N = fvv::net_of(c);
    if (!N) return fail(FVV_ERR_STATE, "refinement network not initialised");
    fvv::DeviceScope dev_scope(c->device);
    if (!precision) return fail(FVV_ERR_INVALID_ARG, "precision is NULL");
    std::lock_guard<std::recursive_mutex> g(c->mu);
    *precision = N->precision;
    if (act_scales)
        for (int i = 0; i < 10; ++i) act_scales[i] = N->s_act[i];
    return FVV_OK;
}

fvv_status fvv_refine_train_step(fvv_ctx* c, const fvv_refine_batch* b, float lr, float* loss, void* stream)
{
    RefineNet* N = fvv::net_of(c);
    if (!N) return fail(FVV_ERR_STATE, "refinement network not initialised");
    fvv::DeviceScope dev_scope(c->device);
    FVV_TRY(fvv::check_batch(*N, b, true));
    if (!(lr >= 0.0f) || !std::isfinite(lr)) return fail(FVV_ERR_INVALID_ARG, "lr must be >= 0");
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : c->own;
    std::lock_guard<std::recursive_mutex> g(c->mu);
    if (fvv::serve_refining(c)) return fail(FVV_ERR_BUSY, "the serving loop is running the refinement network");
    int* err = nullptr;
    FVV_TRY(fvv::device_flag(&err));
    FVV_TRY(fvv::ensure_acts(c, *N, size_t(b->n) * b->height * b->width));
    FVV_TRY(fvv::ensure_grads(c, *N, size_t(b->n) * b->height * b->width));
    FVV_TRY(fvv::ensure_wscratch(c, *N, b->n, b->height, b->width));
    FVV_TRY(fvv::forward(*N, *b, err, s, nullptr, 0, nullptr));
    FVV_TRY(fvv::backward(*N, *b, err, s));
    if (lr > 0.0f) FVV_TRY(fvv::adam(*N, lr, s));
    float h = 0.0f;
    FVV_CUDA(cudaMemcpyAsync(&h, N->loss, 4, cudaMemcpyDeviceToHost, s));
    FVV_TRY(fvv::check_flag(err, s, "fvv_refine_train_step"));
    if (loss) *loss = h;
    return FVV_OK;
}

fvv_status fvv_refine_save(fvv_ctx* c, const char* path)
{
    RefineNet* N = fvv::net_of(c);
    if (!N) return fail(FVV_ERR_STATE, "refinement network not initialised");
    fvv::DeviceScope dev_scope(c->device);
    if (!path) return fail(FVV_ERR_INVALID_ARG, "path is NULL");
    std::lock_guard<std::recursive_mutex> g(c->mu);
    FVV_CUDA(cudaDeviceSynchronize());
    const size_t n = fvv::flat_count(*N);
    std::vector<float> buf(3 * n);
    FVV_TRY(fvv::get_flat(*N, fvv::Buf::Param, buf.data()));
    FVV_TRY(fvv::get_flat(*N, fvv::Buf::M, buf.data() + n));
    FVV_TRY(fvv::get_flat(*N, fvv::Buf::V, buf.data() + 2 * n));
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(FVV_ERR_INVALID_ARG, std::string("cannot open ") + path);
    const char magic[8] = {'F', 'V', 'V', 'U', 'N', 'E', 'T', '1'};
    const int32_t hdr[5] = {N->w1, N->w2, N->w3, N->step, 0};
    const uint64_t cnt = n;
    bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(hdr, 4, 5, f) == 5 &&
              std::fwrite(&N->z_far, 4, 1, f) == 1 && std::fwrite(&cnt, 8, 1, f) == 1 &&
              std::fwrite(buf.data(), 4, buf.size(), f) == buf.size();
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(FVV_ERR_INVALID_ARG, std::string("write failed: ") + path);
    return FVV_OK;
}

fvv_status fvv_refine_load(fvv_ctx* c, const char* path)
{
    if (!c || !path) return fail(FVV_ERR_INVALID_ARG, "NULL argument");
    fvv::DeviceScope dev_scope(c->device);
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(FVV_ERR_INVALID_ARG, std::string("cannot open ") + path);
    char magic[8];
    int32_t hdr[5];
    float z_far = 0.0f;
    uint64_t cnt = 0;
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "FVVUNET1", 8) == 0 &&
              std::fread(hdr, 4, 5, f) == 5 && std::fread(&z_far, 4, 1, f) == 1 && std::fread(&cnt, 8, 1, f) == 1;
    std::vector<float> buf;
    if (ok && cnt < (uint64_t(1) << 32)) {
        buf.resize(3 * cnt);
        ok = std::fread(buf.data(), 4, buf.size(), f) == buf.size();
    } else {
        ok = false;
    }
    std::fclose(f);
    if (!ok) return fail(FVV_ERR_INVALID_ARG, std::string("not a refinement checkpoint: ") + path);
    fvv_unet_cfg cfg;
    fvv_refine_default_cfg(&cfg);
    cfg.widths[0] = hdr[0];
    cfg.widths[1] = hdr[1];
    cfg.widths[2] = hdr[2];
    cfg.z_far = z_far;
    FVV_TRY(fvv_refine_init(c, &cfg));
    RefineNet* N = fvv::net_of(c);
    if (fvv::flat_count(*N) != cnt) return fail(FVV_ERR_INVALID_ARG, "checkpoint size mismatch");
    std::lock_guard<std::recursive_mutex> g(c->mu);
    if (fvv::serve_refining(c)) return fail(FVV_ERR_BUSY, "the serving loop is running the refinement network");
    FVV_TRY(fvv::set_flat(*N, fvv::Buf::Param, buf.data(), c->own));
    FVV_TRY(fvv::set_flat(*N, fvv::Buf::M, buf.data() + cnt, c->own));
    FVV_TRY(fvv::set_flat(*N, fvv::Buf::V, buf.data() + 2 * cnt, c->own));
    N->step = hdr[3];
    FVV_CUDA(cudaStreamSynchronize(c->own));
    return FVV_OK;
}

fvv_status fvv_synthesize_refined(fvv_ctx* c, const fvv_view* view, uint8_t* out_rgb, size_t out_pitch,
                                  void* stream)
{
    RefineNet* N = fvv::net_of(c);
    if (!N) return fail(FVV_ERR_STATE, "refinement network not initialised");
    fvv::DeviceScope dev_scope(c->device);
    if (!view || !out_rgb) return fail(FVV_ERR_INVALID_ARG, "NULL argument");
    const int H = view->height, W = view->width;
    if (H % 4 || W % 4) return fail(FVV_ERR_INVALID_ARG, "refined views need width and height multiples of 4");
    if (out_pitch < size_t(W) * 3) return fail(FVV_ERR_INVALID_ARG, "out_pitch < 3 * width");
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : c->own;
    std::lock_guard<std::recursive_mutex> g(c->mu);
    if (fvv::serve_refining(c)) return fail(FVV_ERR_BUSY, "the serving loop is running the refinement network");
    if (N->sH != H || N->sW != W) {
        FVV_CUDA(cudaDeviceSynchronize());
        fvv::free_list(c, N->syn);
        N->sH = N->sW = 0;
        const size_t np = size_t(H) * W;
        FVV_TRY(fvv::alloc_t(c, N->syn, &N->syn_rgb, np * 3));
        FVV_TRY(fvv::alloc_t(c, N->syn, &N->syn_out, np * 3));
        FVV_TRY(fvv::alloc_t(c, N->syn, &N->syn_hole, np));
        FVV_TRY(fvv::alloc_t(c, N->syn, &N->syn_depth, np));
        FVV_TRY(fvv::alloc_t(c, N->syn, &N->syn_top3, np * 3));
        N->sH = H;
        N->sW = W;
    }
    fvv_aux aux{};
    aux.depth = N->syn_depth;
    aux.hole = N->syn_hole;
    aux.top3 = N->syn_top3;
    uint8_t* outs[1] = {N->syn_rgb};
    const size_t pitches[1] = {size_t(W) * 3};
    FVV_TRY(fvv::run_batch(c, c->main, 1, view, nullptr, outs, pitches, &aux, s, true));
    fvv_refine_batch b{};
    b.n = 1;
    b.height = H;
    b.width = W;
    b.rgb = N->syn_rgb;
    b.depth = N->syn_depth;
    b.hole = N->syn_hole;
    b.top3 = N->syn_top3;
    int* err = nullptr;
    FVV_TRY(fvv::device_flag(&err));
    if (fvv::foreign(out_rgb))
        return fail(FVV_ERR_INVALID_ARG, "out_rgb must be host memory or the context's device memory");
    const bool dev_out = fvv::mem_kind(out_rgb) == fvv::MemKind::Device;
    if (N->precision == FVV_PREC_E4M3) {
        FVV_TRY(fvv::ensure_acts8(c, *N, size_t(H) * W));
        FVV_TRY(fvv::forward_e4m3(*N, b, err, s, dev_out ? out_rgb : N->syn_out,
                                  dev_out ? out_pitch : size_t(W) * 3, nullptr));
    } else {
        FVV_TRY(fvv::ensure_acts(c, *N, size_t(H) * W));
        FVV_TRY(fvv::forward(*N, b, err, s, dev_out ? out_rgb : N->syn_out, dev_out ? out_pitch : size_t(W) * 3,
                             nullptr));
    }
    if (!dev_out)
        FVV_CUDA(cudaMemcpy2DAsync(out_rgb, out_pitch, N->syn_out, size_t(W) * 3, size_t(W) * 3, size_t(H),
                                   cudaMemcpyDeviceToHost, s));
    return fvv::check_flag(err, s, "fvv_synthesize_refined");
}

}  // extern "C"
