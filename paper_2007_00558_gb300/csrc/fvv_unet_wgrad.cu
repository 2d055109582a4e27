// fvv_unet_wgrad.cu -- weight and bias gradients of the refinement network's
// 3x3 convolutions on the sm_103a tensor cores (tcgen05, TMEM accumulators,
// TMA operand tiles).
//
//   dW[co][ky][kx][ci] = sum_p dz[p][co] x[p + (ky - 1, kx - 1)][ci]
//   db[co]             = sum_p dz[p][co]
//
// The reduction runs over pixels.  Both operands are read straight from the
// NHWC tensors by TMA as 64-byte rows of 32 channels, one row per pixel, with
// the 64-byte swizzle: for the MMA that is an MN-major tile (the channel
// index contiguous, the pixel index K across rows).  A chunk is 64 pixels (a
// box of wbox x hbox pixels).  Per chunk the CTA loads
//   - nine windows of x (32 input channels), each shifted by one tap
//     (kx - 1, ky - 1); TMA fills pixels outside the image with zeros, which
//     is the convolution's zero padding;
//   - the chunk of dz (32 nb output channels, unshifted).
// Each MMA is M = 128 rows = four 32-row slots of A, so one MMA accumulates
// four taps: slots 0-8 are the taps, slot 9 a tile of ones (its rows give
// sum_p dz[p][co], the bias gradient, at no extra cost), slots 10-11 unused.
// Three MMAs (K = 16 pixels each) per 16 pixels of the chunk, into three
// 128 x N TMEM accumulators.
//
// Each CTA (one 32-channel input box, up to 128 output channels) reduces a
// fixed range of chunks and writes its fp32 partial sums; a second kernel
// adds the partials in split order.  No atomics: the result does not depend
// on scheduling, so a training run is reproducible bit for bit.
#include <algorithm>

#include "fvv_tc.cuh"
#include "fvv_internal.h"
#include "fvv_unet.h"

namespace fvv {
namespace {

constexpr int kWgThreads = 128;
constexpr int kWgBox = 4096;                    // 64 pixels x 32 channels x 2 bytes
constexpr int kWgMaxNb = 4;                     // output-channel boxes of 32 per CTA
constexpr int kWgHeader = 1024;
constexpr int kWgHaloPx = 66;                   // a one-row chunk and its two neighbours
constexpr int kWgHaloBox = 5120;                // room for 80 rows of 64 bytes, 1024-aligned

// Two layouts of the shifted x windows in a pipeline stage.
//  Nine windows (any chunk shape): tap t = 3 ky + kx at slot t (4 KiB each),
//    the ones tile at slot 9; MMA g reads slots 4g .. 4g + 3.
//  Row halos (one-row chunks, images at least 64 wide): for each ky one box
//    of the 66 pixels x0 - 1 .. x0 + 64 of row y0 + ky - 1, the ones tile as
//    a fourth box; MMA g = kx starts kx rows (64 bytes) into every box, so
//    its slots are (ky = 0, 1, 2, ones).  A third of the TMA traffic of the
//    nine windows.  (The 64-byte swizzle follows absolute shared-memory
//    address bits, so a start moved by whole rows reads the shifted window.)
template <bool kHalo>
struct WgLayout {
    static constexpr int kLbo = kHalo ? kWgHaloBox : kWgBox;          // between the slots of an MMA
    static constexpr int kABytes = kHalo ? 4 * kWgHaloBox : 12 * kWgBox;
    static constexpr int kOnes = kHalo ? 3 * kWgHaloBox : 9 * kWgBox;  // the ones tile
    static constexpr int kOnesBytes = kHalo ? kWgHaloBox : kWgBox;
    static constexpr int kStage = kABytes + kWgMaxNb * kWgBox;
    static constexpr int kStages = kHalo ? 5 : 3;
    static constexpr int kSmem = kWgHeader + kStages * kStage + 1024;  // + alignment slack
    // the tap (0..8) of slot w of MMA g, 9 for the ones slot, -1 unused
    __device__ static int tap(int g, int w)
    {
        if (kHalo) return w < 3 ? 3 * w + g : (g == 0 ? 9 : -1);
        const int s = 4 * g + w;
        return s <= 9 ? s : -1;
    }
};

struct WgradArgs {
    int B, H, W, Cin, Cout;
    int wbox, hbox;                             // chunk box, wbox * hbox = 64 pixels
    int tiles_x, tiles_y;                       // chunks along a row / a column of an image
    int n_chunks;
    int cps;                                    // chunks per split
    int nb;                                     // output-channel boxes per CTA
    float* part;                                // [splits][Cout * 9 * Cin + Cout]: dW, then db
    int* err;
};

// Descriptor of an MN-major operand tile written by TMA with the 64-byte
// swizzle: 64-byte rows of 32 MN-consecutive elements, one row per K index,
// 8-row groups (512 bytes) consecutive along K; the next 32 MN elements live
// in another tile `lbo` bytes away.
__device__ __forceinline__ uint64_t desc_mn_sw64(uint32_t saddr, uint32_t lbo)
{
    uint64_t d = 0;
    d |= uint64_t((saddr >> 4) & 0x3FFFu);          // start address
    d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;       // next 32 MN elements
    d |= uint64_t(512 >> 4) << 32;                   // next 8 K rows
    d |= uint64_t(1) << 46;                          // descriptor version
    d |= uint64_t(4) << 61;                          // 64-byte swizzle
    return d;
}

template <bool kHalo>
__global__ void __launch_bounds__(kWgThreads, 1)
k_wgrad3x3_tc(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmdz, WgradArgs P)
{
    using Lay = WgLayout<kHalo>;
    constexpr int kWgStages = Lay::kStages;
    constexpr int kWgStage = Lay::kStage;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(base);
    uint64_t* empty = full + kWgStages;
    uint64_t* acc_full = empty + kWgStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_full + 1);
    int* skip = reinterpret_cast<int*>(tmem_slot + 1);
    uint8_t* stages = base + kWgHeader;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) *skip = *reinterpret_cast<volatile int*>(P.err);
    __syncthreads();
    if (*skip) return;                                 // an earlier CTA gave up

    const int ci_boxes = (P.Cin + 31) >> 5;
    const int ci0 = (blockIdx.x % ci_boxes) * 32;
    const int co0 = (blockIdx.x / ci_boxes) * 32 * P.nb;
    const int split = blockIdx.y;
    const int c_begin = split * P.cps, c_end = min(c_begin + P.cps, P.n_chunks);
    const int nb = P.nb, N = 32 * nb;
    const uint32_t cols = N * 3 <= 32 ? 32u : N * 3 <= 64 ? 64u : N * 3 <= 128 ? 128u : N * 3 <= 256 ? 256u : 512u;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kWgStages; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(acc_full, 1);
        tc::fence_mbar_init();
        tc::prefetch_tensormap(&tmx);
        tc::prefetch_tensormap(&tmdz);
    }
    // the ones tile of every stage (bf16 1.0; the swizzle does not matter)
    for (int s = 0; s < kWgStages; ++s) {
        uint4* o = reinterpret_cast<uint4*>(stages + s * kWgStage + Lay::kOnes);
        for (int i = threadIdx.x; i < Lay::kOnesBytes / 16; i += kWgThreads)
            o[i] = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
    }
    tc::fence_proxy_async_smem();
    if (warp == 0) tc::tmem_alloc(tmem_slot, cols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    const int nk = c_end - c_begin;
    if (warp == 0 && lane == 0) {
        // ---------------------------------------------------------------- TMA
        const uint32_t bytes = (kHalo ? 3u * kWgHaloPx * 64u : 9u * kWgBox) + uint32_t(nb) * kWgBox;
        int it = 0;
        for (; it < nk; ++it) {
            const int s = it % kWgStages;
            if (it >= kWgStages &&
                !tc::mbar_wait_sleep(&empty[s], uint32_t((it / kWgStages - 1) & 1), P.err, 1, 2000))
                break;
            int c = c_begin + it;
            const int tx = c % P.tiles_x;
            c /= P.tiles_x;
            const int ty = c % P.tiles_y;
            const int b = c / P.tiles_y;
            const int x0 = tx * P.wbox, y0 = ty * P.hbox;
            uint8_t* st = stages + s * kWgStage;
            tc::mbar_arrive_expect_tx(&full[s], bytes);
            if (kHalo) {
                for (int ky = 0; ky < 3; ++ky)
                    tc::tma_load_4d(st + ky * kWgHaloBox, &tmx, &full[s], ci0, x0 - 1, y0 + ky - 1, b);
            } else {
                for (int t = 0; t < 9; ++t)
                    tc::tma_load_4d(st + t * kWgBox, &tmx, &full[s], ci0, x0 + (t % 3) - 1, y0 + (t / 3) - 1, b);
            }
            for (int j = 0; j < nb; ++j)
                tc::tma_load_4d(st + Lay::kABytes + j * kWgBox, &tmdz, &full[s], co0 + 32 * j, x0, y0, b);
        }
        // the copies of the last stages have landed before the CTA exits
        for (int k = max(0, it - kWgStages); k < it; ++k)
            tc::mbar_wait_drain(&full[k % kWgStages], uint32_t((k / kWgStages) & 1));
    } else if (warp == 1 && lane == 0) {
        // ---------------------------------------------------------------- MMA
        const uint32_t idesc = tc::idesc_bf16(128, N) | (1u << 15) | (1u << 16);   // A, B MN-major
        for (int it = 0; it < nk; ++it) {
            const int s = it % kWgStages;
            if (!tc::mbar_wait(&full[s], uint32_t((it / kWgStages) & 1), P.err, 2)) break;
            tc::fence_after_sync();
            const uint32_t a0 = tc::smem_u32(stages + s * kWgStage);
            const uint32_t b0 = a0 + Lay::kABytes;
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
#pragma unroll
                for (int g = 0; g < 3; ++g)
                    tc::mma_bf16(tmem + uint32_t(g * N),
                                 desc_mn_sw64(a0 + (kHalo ? g * 64 : g * 4 * kWgBox) + ks * 1024, Lay::kLbo),
                                 desc_mn_sw64(b0 + ks * 1024, kWgBox), idesc, (it > 0 || ks > 0) ? 1u : 0u);
            tc::mma_commit(&empty[s]);
        }
        tc::mma_commit(acc_full);                       // also after a failure: every issued MMA done
    }
    __syncwarp();

    // -------------------------------------------------------------- epilogue
    // warp w reads TMEM lanes 32w .. 32w+31: slot 4g + w of accumulator g
    bool ok = tc::mbar_wait_sleep(acc_full, 0, P.err, 3, 2000);
    tc::fence_after_sync();
    ok = __all_sync(0xffffffffu, ok && nk > 0 && *reinterpret_cast<volatile int*>(P.err) == 0);
    if (ok) {
        const int ci = ci0 + lane;
        const size_t nw = size_t(P.Cout) * 9 * P.Cin, nper = nw + size_t(P.Cout);
        for (int g = 0; g < 3; ++g) {
            const int slot = Lay::tap(g, warp);
            if (slot < 0) continue;
            for (int c32 = 0; c32 < nb; ++c32) {
                uint32_t r[32];
                tc::tmem_ld_x32(tmem + (uint32_t(32 * warp) << 16) + uint32_t(g * N + 32 * c32), r);
                tc::tmem_ld_wait();
                const int cb = co0 + 32 * c32;
                if (slot < 9) {
                    if (ci < P.Cin) {
                        float* dst = P.part + size_t(split) * nper + (size_t(cb) * 9 + slot) * P.Cin + ci;
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (cb + j < P.Cout) dst[size_t(j) * 9 * P.Cin] = __uint_as_float(r[j]);
                    }
                } else if (ci0 == 0 && lane == 0) {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (cb + j < P.Cout) P.part[size_t(split) * nper + nw + cb + j] = __uint_as_float(r[j]);
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, cols);
}

}  // namespace

namespace {

struct WgradPlan {
    int wbox, hbox, tiles_x, tiles_y, n_chunks, nb, tiles;
};

WgradPlan wgrad_plan(int B, int H, int W, int Cin, int Cout)
{
    WgradPlan p;
    // 64-pixel chunks, as wide as the image allows
    p.wbox = W >= 64 ? 64 : W >= 32 ? 32 : W >= 16 ? 16 : 8;
    p.hbox = 64 / p.wbox;
    p.tiles_x = (W + p.wbox - 1) / p.wbox;
    p.tiles_y = (H + p.hbox - 1) / p.hbox;
    p.n_chunks = B * p.tiles_x * p.tiles_y;
    const int co_boxes = (Cout + 31) / 32;
    p.nb = std::min(co_boxes, kWgMaxNb);
    p.tiles = ((Cin + 31) / 32) * ((co_boxes + p.nb - 1) / p.nb);
    return p;
}

// Splits of the chunk range: one resident wave (one CTA per SM) over all
// tiles, at least four chunks per CTA.
int wgrad_splits(const WgradPlan& p)
{
    const int want = (device_sms() + p.tiles - 1) / p.tiles;
    const int most = (p.n_chunks + 3) / 4;
    return std::max(1, std::min(want, most));
}

// x: [B][H][W][xstride] seen as (C, W, H, B) with C = the first `c` channels
cudaError_t make_map(CUtensorMap* m, const void* x, int B, int H, int W, int c, int stride, int wbox, int hbox)
{
    auto enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[4] = {cuuint64_t(c), cuuint64_t(W), cuuint64_t(H), cuuint64_t(B)};
    const cuuint64_t strides[3] = {cuuint64_t(stride) * 2, cuuint64_t(W) * stride * 2, cuuint64_t(H) * W * stride * 2};
    const cuuint32_t box[4] = {32, cuuint32_t(wbox), cuuint32_t(hbox), 1};
    const cuuint32_t el[4] = {1, 1, 1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(x), dims, strides, box, el,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

size_t wgrad_scratch_floats(int B, int H, int W, int Cin, int Cout)
{
    const WgradPlan p = wgrad_plan(B, H, W, Cin, Cout);
    return size_t(wgrad_splits(p)) * size_t(Cout) * (9 * size_t(Cin) + 1);
}

cudaError_t launch_wgrad3x3_tc(int B, int H, int W, int Cin, int xstride, int Cout, const __nv_bfloat16* x,
                               const __nv_bfloat16* dz, float* dw, float* db, float* scratch,
                               size_t scratch_floats, int* err, cudaStream_t s)
{
    if (B < 1 || H < 1 || W < 1 || Cin < 8 || Cin % 8 || Cout < 8 || Cout % 8 || xstride < Cin || xstride % 8 ||
        !x || !dz || !dw || !scratch || !err)
        return cudaErrorInvalidValue;
    if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(dz)) & 15) return cudaErrorInvalidValue;
    const WgradPlan p = wgrad_plan(B, H, W, Cin, Cout);
    const size_t per = size_t(Cout) * (9 * size_t(Cin) + 1);
    if (scratch_floats < per || p.tiles > 65535) return cudaErrorInvalidValue;
    int splits = std::min<long long>(wgrad_splits(p), (long long)(scratch_floats / per));
    const int cps = (p.n_chunks + splits - 1) / splits;
    splits = (p.n_chunks + cps - 1) / cps;                 // every split holds at least one chunk
    CUtensorMap mx, mdz;
    const bool halo = p.hbox == 1;                       // one-row chunks: row halos
    cudaError_t e = make_map(&mx, x, B, H, W, Cin, xstride, halo ? kWgHaloPx : p.wbox, p.hbox);
    if (e != cudaSuccess) return e;
    e = make_map(&mdz, dz, B, H, W, Cout, Cout, p.wbox, p.hbox);
    if (e != cudaSuccess) return e;
    WgradArgs a;
    a.B = B;
    a.H = H;
    a.W = W;
    a.Cin = Cin;
    a.Cout = Cout;
    a.wbox = p.wbox;
    a.hbox = p.hbox;
    a.tiles_x = p.tiles_x;
    a.tiles_y = p.tiles_y;
    a.n_chunks = p.n_chunks;
    a.cps = cps;
    a.nb = p.nb;
    a.part = scratch;
    a.err = err;
    const dim3 grid(unsigned(p.tiles), unsigned(splits));
    if (halo) {
        e = cudaFuncSetAttribute(k_wgrad3x3_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, WgLayout<true>::kSmem);
        if (e != cudaSuccess) return e;
        k_wgrad3x3_tc<true><<<grid, kWgThreads, WgLayout<true>::kSmem, s>>>(mx, mdz, a);
    } else {
        e = cudaFuncSetAttribute(k_wgrad3x3_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 WgLayout<false>::kSmem);
        if (e != cudaSuccess) return e;
        k_wgrad3x3_tc<false><<<grid, kWgThreads, WgLayout<false>::kSmem, s>>>(mx, mdz, a);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t nw = size_t(Cout) * 9 * Cin;
    return launch_sum_splits(scratch, splits, nw + size_t(Cout), dw, nw, db, size_t(Cout), nullptr, s);
}

}  // namespace fvv
