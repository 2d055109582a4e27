// fvv_unet_conv.cu -- 3x3 convolution (pad 1) of the refinement network as
// an implicit GEMM on the sm_103a tensor cores (tcgen05, TMEM, TMA).
//
// GEMM view: M = 128 consecutive output pixels of one image row, N = the
// output channels, K = 9 taps x input channels.  A tile is R such rows
// (R = 4 for 32 output channels, 2 for up to 64, else 1; the folded and
// wide forms below use 2).  A persistent CTA
// (one per SM) walks the tiles.  Input channels are taken in groups of one
// 64-byte row (32 bf16 or 64 e4m3 channels).  For each tile and group, ONE
// TMA copy brings the halo -- rows y0-1..y0+R, pixels x0-1..x0+128, zero
// outside the image (the convolution's padding) and beyond the last channel
// -- into shared memory as (R+2) x 130 rows of 64 bytes with the 64-byte
// swizzle.  Operand A of output row r and tap (ky, kx) is that same halo
// seen through a descriptor whose start lies 130 (r + ky) + kx rows further
// on: nine taps cost nine descriptors, not nine copies, and the halo's two
// extra rows are shared by the R output rows (narrow layers are bound by
// moving the halo).  The weights [cout][ky][kx][cin] stay
// resident in shared memory when they fit; otherwise they stream through a
// ring of one-ky slices (three taps).  The fp32 accumulators live in a TMEM
// ring: the epilogue (scale, bias, ReLU, optional ReLU-derivative mask,
// rounding to bf16 or e4m3, NHWC store -- staged through shared memory and
// TMA where the output is strided or upsampled --, optional 2x2 max pooling
// or 1x1 output head) drains tile i while the MMA thread accumulates the
// next ones.
//
// C8 (the first layer: 8 input features in 16 bytes per pixel, bf16, or 8
// e4m3 codes and 8 zero bytes): the halo is copied as rows of 16 bytes, one
// per pixel, without swizzle, and each MMA (K = 16 bytes x 2) takes two taps
// at once -- the descriptor's second K core matrix is the next pixel (tap
// kx + 1) or the next halo row (tap ky + 1) -- against a weight tile stored
// tap by tap: five MMAs per output row instead of nine, and a quarter of the
// halo bytes.  A tenth, zero weight tap pads the odd ninth.  Where the image
// width is a multiple of 4 the copy sees four pixels as one 64-byte row (a
// TMA copy costs per row): the halo then starts at pixel x0 - 4, three
// pixels before the window, and the descriptors start three pixels on.
//
// Warp roles (320 threads): 0 = TMA producer, 1 = TMEM owner and MMA issuer,
// 2..9 = epilogue in two groups of four, taking alternate tiles (warp w
// reads TMEM lanes 32 (w mod 4) .. +31); two warps per sub-partition hide
// each other's TMEM-load and store latency.
#include <algorithm>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cudaTypedefs.h>

#include "fvv_internal.h"
#include "fvv_tc.cuh"
#include "fvv_unet.h"

namespace fvv {

namespace {

constexpr int kTileM = 128;
constexpr int kRow = 64;                               // bytes of one pixel row of a channel group
constexpr int kThreads = 320;
constexpr int kMaxStages = 8;
constexpr int kSmemLimit = 227 * 1024;
constexpr int kHeader = 2048;                          // barriers (bytes 0..511) and bias (512..1279)
constexpr int kSmemFixed = 1024 + kHeader;             // alignment slack + header

// kFold (32 output channels, where a 128 x 32 MMA is bound by its issue
// cost): the three kx taps of one ky run as ONE MMA of N = 96 against the
// unshifted halo row, D[p][32 kx + c] = sum over ky of A_ky[p] W(ky, kx);
// output pixel q is then D[q][c] + D[q+1][32+c] + D[q+2][64+c], summed in
// the epilogue with warp shuffles.  Each TMEM lane quadrant (one epilogue
// warp) holds its own window of 32 halo pixels, overlapping the next by 2,
// so a warp finds all three terms of its first 30 pixels in its own lanes:
// a tile covers 4 x 30 output pixels.
// WIDE (96 and 128 output channels with streamed weights): two output rows
// per tile instead of one, so that every weight slice streamed from L2 feeds
// twice the MMAs.
template <int COUT, bool FOLD = false, bool WIDE = false>
struct ConvCfg {
    static_assert(!WIDE || (!FOLD && (COUT == 96 || COUT == 128)), "the wide form is for 96 or 128 channels");
    static_assert(!FOLD || COUT == 32, "the folded form is for 32 output channels");
    static constexpr bool kFold = FOLD;
    static constexpr int kTap = COUT * kRow;           // B tile of one tap (COUT rows of 64 bytes)
    static constexpr int kSlice = 3 * kTap;            // the three taps of one ky
    static constexpr int kGroup = 9 * kTap;            // all taps of one channel group
    static constexpr int kN = kFold ? 3 * COUT : COUT; // MMA N
    static constexpr int kAcc = (kN + 31) / 32 * 32;   // TMEM columns of one output row's accumulator
    static constexpr int kRows = kFold ? 2 : WIDE ? 2 : COUT <= 32 ? 4 : COUT <= 64 ? 2 : 1;   // rows per tile
    static constexpr int kHaloPx = kFold ? 128 : kTileM + 2;           // halo pixels per halo row
    static constexpr int kQuad = kFold ? 30 : 32;      // output pixels per lane quadrant
    static constexpr int kTileOut = 4 * kQuad;         // output pixels per tile row
    static constexpr int kTileAcc = kRows * kAcc;      // TMEM columns of one tile
    static constexpr int kNumAcc = 4 * kTileAcc <= 512 ? 4 : 2;        // accumulator ring depth
    static constexpr int kTmemCols = kNumAcc * kTileAcc <= 64 ? 64 : kNumAcc * kTileAcc <= 128 ? 128
                                   : kNumAcc * kTileAcc <= 256 ? 256 : 512;
    static constexpr int kHaloRows = kRows + 2;
    static constexpr int kHaloBytes = kHaloRows * kHaloPx * kRow;
    static constexpr int kHaloStage = (kHaloBytes + 1023) / 1024 * 1024;   // halo slot, 1024-aligned
    // Output staging for the TMA stores: each of the eight epilogue warps
    // owns a buffer of 32 pixels x one chunk of up to 64 channels,
    // 1024-byte aligned (the 128-byte swizzle's period).
    static constexpr int kChunk = COUT < 64 ? COUT : 64;
    __host__ __device__ static constexpr int out_buf(bool fp8) { return (32 * kChunk * (fp8 ? 1 : 2) + 1023) / 1024 * 1024; }
    static_assert(kTap % 1024 == 0, "tap tiles stay 1024-byte aligned");
    static_assert(kNumAcc * kTileAcc <= 512, "accumulators fit TMEM");
};

struct Plan {
    int hs, ws, resident, out, smem;
};

// Shared memory: resident weights come first (they are read by every tile),
// then the staged output, then the depth of the rings.  hs = 0: no plan fits.
template <int COUT, bool FOLD, bool WIDE = false>
Plan make_plan(int groups, bool fp8, bool want_out)
{
    using C = ConvCfg<COUT, FOLD, WIDE>;
    Plan p{};
    const int res = groups * C::kGroup;
    for (int out = want_out ? 2 : 0; out >= 0; --out) {
        const int fixed = kSmemFixed + out * 8 * C::out_buf(fp8);
        if (fixed + res + 3 * C::kHaloStage <= kSmemLimit) {
            p.resident = 1;
            p.out = out;
            p.hs = std::min(kMaxStages, (kSmemLimit - fixed - res) / C::kHaloStage);
            p.ws = 0;
            p.smem = fixed + res + p.hs * C::kHaloStage;
            return p;
        }
    }
    for (int out = want_out ? 1 : 0; out >= 0; --out) {       // streamed: weight slices before staging
        const int fixed = kSmemFixed + out * 8 * C::out_buf(fp8);
        const int ws = std::min(kMaxStages, (kSmemLimit - fixed - 3 * C::kHaloStage) / C::kSlice);
        if (ws >= 2) {
            p.resident = 0;
            p.out = out;
            p.hs = 3;
            p.ws = ws;
            p.smem = fixed + p.hs * C::kHaloStage + p.ws * C::kSlice;
            return p;
        }
    }
    return p;
}

// C8: halo rows of kC8Px pixels x 16 bytes; weights as 10 tap tiles of COUT x 16 bytes
constexpr int kC8Px = 136;
template <int COUT>
struct C8Cfg {
    static constexpr int kHaloRows = ConvCfg<COUT>::kHaloRows;
    static constexpr int kHaloBytes = kHaloRows * kC8Px * 16;
    static constexpr int kHaloStage = (kHaloBytes + 1023) / 1024 * 1024;
    static constexpr int kTap = COUT * 16;
    static constexpr int kWBytes = (10 * kTap + 1023) / 1024 * 1024;
};

template <int COUT>
Plan make_plan_c8(bool fp8, bool want_out)
{
    using C = C8Cfg<COUT>;
    Plan p{};
    for (int out = want_out ? 2 : 0; out >= 0; --out) {
        const int fixed = kSmemFixed + out * 8 * ConvCfg<COUT>::out_buf(fp8);
        if (fixed + C::kWBytes + 2 * C::kHaloStage <= kSmemLimit) {
            p.resident = 1;
            p.out = out;
            p.hs = std::min(kMaxStages, (kSmemLimit - fixed - C::kWBytes) / C::kHaloStage);
            p.ws = 0;
            p.smem = fixed + C::kWBytes + p.hs * C::kHaloStage;
            return p;
        }
    }
    return p;
}

// The 16-byte unit that logical unit j of staging row p occupies under the
// tensor map's swizzle (the 128-, 64- and 32-byte modes XOR the unit index
// with address bits 7 and up; rows of another length are not swizzled).
__device__ __forceinline__ int out_swizzle(int row_bytes, int p)
{
    return row_bytes == 128 ? (p & 7) : row_bytes == 64 ? ((p >> 1) & 3) : row_bytes == 32 ? ((p >> 2) & 1) : 0;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ uint32_t pack_e4m3x4(float a, float b, float c, float d)
{
    const __nv_fp8x2_storage_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
    const __nv_fp8x2_storage_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
    return uint32_t(lo) | (uint32_t(hi) << 16);
}

// The MMAs of one ky row of taps: kx = 0..2, NKS K-steps of 32 bytes each.
// A of tap kx starts kx halo rows further on; +2 in a descriptor's start
// field is +32 bytes (the second K-step).  Only the first MMA can start a
// fresh accumulator (acc0 = 0).
template <int COUT, bool FP8, int NKS>
__device__ __forceinline__ void mma_row(uint32_t d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc0)
{
    using Cfg = ConvCfg<COUT>;
#pragma unroll
    for (int kx = 0; kx < 3; ++kx) {
#pragma unroll
        for (int ks = 0; ks < NKS; ++ks) {
            const uint64_t a = da + uint64_t((kx * kRow) >> 4) + 2 * ks;
            const uint64_t b = db + uint64_t((kx * Cfg::kTap) >> 4) + 2 * ks;
            const uint32_t acc = (kx | ks) != 0 ? 1u : acc0;
            if (FP8)
                tc::mma_e4m3(d, a, b, idesc, acc);
            else
                tc::mma_bf16(d, a, b, idesc, acc);
        }
    }
}

// All MMAs of one channel group with resident weights: taps (ky, kx), NKS
// K-steps each, every descriptor offset a compile-time constant.
template <int COUT, bool FP8, int NKS>
__device__ __forceinline__ void mma_group(uint32_t d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc0)
{
    using Cfg = ConvCfg<COUT>;
#pragma unroll
    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
        for (int kx = 0; kx < 3; ++kx)
#pragma unroll
            for (int ks = 0; ks < NKS; ++ks) {
                const uint64_t a = da + uint64_t(((ky * Cfg::kHaloPx + kx) * kRow) >> 4) + 2 * ks;
                const uint64_t b = db + uint64_t((ky * Cfg::kSlice + kx * Cfg::kTap) >> 4) + 2 * ks;
                const uint32_t acc = (ky | kx | ks) != 0 ? 1u : acc0;
                if (FP8)
                    tc::mma_e4m3(d, a, b, idesc, acc);
                else
                    tc::mma_bf16(d, a, b, idesc, acc);
            }
}

// kFold: the MMAs of one output row and channel group, one per (ky, K-step)
// with N = 96; A of ky starts ky halo rows further on, B of ky is the
// contiguous slice of its three taps.  NKY: slices resident (3, ky from the
// group's base) or one streamed slice (1, the caller passes its ky's A).
template <bool FP8, int NKS, int NKY>
__device__ __forceinline__ void mma_fold(uint32_t d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc0)
{
    using Cfg = ConvCfg<32, true>;
#pragma unroll
    for (int ky = 0; ky < NKY; ++ky)
#pragma unroll
        for (int ks = 0; ks < NKS; ++ks) {
            const uint64_t a = da + uint64_t((ky * Cfg::kHaloPx * kRow) >> 4) + 2 * ks;
            const uint64_t b = db + uint64_t((ky * Cfg::kSlice) >> 4) + 2 * ks;
            const uint32_t acc = (ky | ks) != 0 ? 1u : acc0;
            if (FP8)
                tc::mma_e4m3(d, a, b, idesc, acc);
            else
                tc::mma_bf16(d, a, b, idesc, acc);
        }
}

// 2 x 2 max pooling of packed non-negative values (bf16 pairs or e4m3
// quads; after the ReLU a value is +0, -0 or positive, so its magnitude bits
// order it like the value and -0 ties with +0).  Candidates in window order
// (0,0), (0,1), (1,0), (1,1); a later one wins only if strictly greater, as
// in the separate pooling kernel.  *arg gets the winner's index per element.
__device__ __forceinline__ uint32_t pool4_bf16(const uint32_t (&c)[4], uint32_t* arg)
{
    uint32_t best = c[0], bk = c[0] & 0x7FFF7FFFu, a = 0;
#pragma unroll
    for (int k = 1; k < 4; ++k) {
        const uint32_t kk = c[k] & 0x7FFF7FFFu;
        const uint32_t m = __vcmpgtu2(kk, bk);
        best = (c[k] & m) | (best & ~m);
        bk = (kk & m) | (bk & ~m);
        a = ((uint32_t(k) * 0x00010001u) & m) | (a & ~m);
    }
    *arg = a;
    return best;
}

__device__ __forceinline__ uint32_t pool4_e4m3(const uint32_t (&c)[4])
{
    uint32_t best = c[0], bk = c[0] & 0x7F7F7F7Fu;
#pragma unroll
    for (int k = 1; k < 4; ++k) {
        const uint32_t kk = c[k] & 0x7F7F7F7Fu;
        const uint32_t m = __vcmpgtu4(kk, bk);
        best = (c[k] & m) | (best & ~m);
        bk = (kk & m) | (bk & ~m);
    }
    return best;
}

// FP8: e4m3 operands and output (K = 32 channels per MMA, 64 per group);
// otherwise bf16 (K = 16, 32 per group).
template <int COUT, bool FP8, bool FOLD, bool WIDE, bool C8>
__global__ void __launch_bounds__(kThreads, 1)
k_conv3x3_tc(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmw,
             const __grid_constant__ CUtensorMap tmy, const __grid_constant__ CUtensorMap tmy2, ConvArgs P,
             int n_tiles, int HS, int WS, int resident, int tma_out)
{
    using Cfg = ConvCfg<COUT, FOLD, WIDE>;
    static_assert(!C8 || (!FOLD && !WIDE && COUT <= 64), "the 16-byte-pixel form is for the first layer");
    // halo stage size and bytes per copy (C8: 16-byte pixel rows)
    constexpr int kStage = C8 ? C8Cfg<COUT>::kHaloStage : Cfg::kHaloStage;
    constexpr int kHaloTx = C8 ? C8Cfg<COUT>::kHaloBytes : Cfg::kHaloBytes;
    static_assert(512 + 4 * COUT <= kHeader, "bias fits the header");
    static_assert(COUT > 64 || 768 + 4 * (3 * COUT + 3) <= kHeader, "head weights fit the header");
    constexpr int kPerGroup = FP8 ? 64 : 32;           // channels in one 64-byte row
    constexpr int kEsize = FP8 ? 1 : 2;
    constexpr int kOutBuf = Cfg::out_buf(FP8);
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full_h = reinterpret_cast<uint64_t*>(base);
    uint64_t* empty_h = full_h + kMaxStages;
    uint64_t* full_w = empty_h + kMaxStages;
    uint64_t* empty_w = full_w + kMaxStages;
    uint64_t* acc_full = empty_w + kMaxStages;         // [kNumAcc]
    uint64_t* acc_empty = acc_full + 4;                // [kNumAcc]
    uint64_t* wready = acc_empty + 4;
    uint64_t* drain = wready + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    int* skip = reinterpret_cast<int*>(tmem_slot + 1);
    float* s_bias = reinterpret_cast<float*>(base + 512);          // [COUT] (<= 192 floats)
    float* s_head = reinterpret_cast<float*>(base + 768);          // fused head: [3][COUT] weights, [3] bias
    uint8_t* sOut = base + kHeader;                                  // [8 warps][tma_out][kOutBuf]
    uint8_t* sHalo = sOut + tma_out * 8 * kOutBuf;
    uint8_t* sW = sHalo + HS * kStage;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) *skip = *reinterpret_cast<volatile int*>(P.err);
    __syncthreads();
    if (*skip) return;                                 // an earlier CTA gave up

    const int Cin = P.Cin, H = P.H, Wd = P.W;
    const int G = C8 ? 1 : (Cin + kPerGroup - 1) / kPerGroup;
    constexpr int R = Cfg::kRows;
    const int tiles_y = (H + R - 1) / R;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kMaxStages; ++s) {
            tc::mbar_init(&full_h[s], 1);
            tc::mbar_init(&empty_h[s], 1);
            tc::mbar_init(&full_w[s], 1);
            tc::mbar_init(&empty_w[s], 1);
        }
        for (int b = 0; b < Cfg::kNumAcc; ++b) {
            tc::mbar_init(&acc_full[b], 1);
            tc::mbar_init(&acc_empty[b], 4);
        }
        tc::mbar_init(wready, 1);
        tc::mbar_init(drain, 1);
        tc::fence_mbar_init();
        tc::prefetch_tensormap(&tmx);
        tc::prefetch_tensormap(&tmw);
        if (tma_out) {
            tc::prefetch_tensormap(&tmy);
            tc::prefetch_tensormap(&tmy2);
        }
    }
    if (warp == 1) tc::tmem_alloc(tmem_slot, Cfg::kTmemCols);
    for (int i = threadIdx.x; i < COUT; i += kThreads) s_bias[i] = P.bias ? P.bias[i] : 0.0f;
    if (COUT <= 64 && P.head_w)
        for (int i = threadIdx.x; i < 3 * COUT + 3; i += kThreads) s_head[i] = i < 3 * COUT ? P.head_w[i] : P.head_b[i - 3 * COUT];
    if (C8) {
        // the zero tenth tap, visible to the tensor cores (async proxy)
        uint4* z = reinterpret_cast<uint4*>(sW + 9 * C8Cfg<COUT>::kTap);
        for (int i = threadIdx.x; i < COUT; i += kThreads) z[i] = make_uint4(0u, 0u, 0u, 0u);
        tc::fence_proxy_async_smem();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            if (C8) {
                tc::mbar_arrive_expect_tx(wready, uint32_t(9 * C8Cfg<COUT>::kTap));
                tc::tma_load_3d(sW, &tmw, wready, 0, 0, 0);
            } else if (resident) {
                tc::mbar_arrive_expect_tx(wready, uint32_t(G * Cfg::kGroup));
                for (int g = 0; g < G; ++g)
                    for (int ky = 0; ky < 3; ++ky)
                        tc::tma_load_3d(sW + g * Cfg::kGroup + ky * Cfg::kSlice, &tmw, wready, g * kPerGroup, 0,
                                        3 * ky);
            }
            uint32_t qh = 0, qw = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
                const int xt = tile % P.tiles_x, rb = tile / P.tiles_x;
                const int y0 = (rb % tiles_y) * R, n = rb / tiles_y;
                const int x0 = xt * Cfg::kTileOut;
                for (int g = 0; g < G && ok; ++g) {
                    const int sh = int(qh % uint32_t(HS));
                    if (!tc::mbar_wait_sleep(&empty_h[sh], ((qh / uint32_t(HS)) & 1u) ^ 1u, P.err, 1)) {
                        ok = false;
                        break;
                    }
                    tc::mbar_arrive_expect_tx(&full_h[sh], kHaloTx);
                    if constexpr (C8) {
                        tc::tma_load_4d(sHalo + sh * kStage, &tmx, &full_h[sh], 0, P.x_quads ? x0 / 4 - 1 : x0 - 1,
                                        y0 - 1, n);
                    } else if constexpr (Cfg::kFold) {
                        // one 32-pixel window per lane quadrant and halo row
                        for (int h = 0; h < Cfg::kHaloRows; ++h)
                            for (int k = 0; k < 4; ++k)
                                tc::tma_load_4d(sHalo + sh * kStage + (h * Cfg::kHaloPx + 32 * k) * kRow, &tmx,
                                                &full_h[sh], g * kPerGroup, x0 - 1 + Cfg::kQuad * k, y0 - 1 + h, n);
                    } else {
                        tc::tma_load_4d(sHalo + sh * kStage, &tmx, &full_h[sh], g * kPerGroup, x0 - 1, y0 - 1, n);
                    }
                    ++qh;
                    if (!resident && !C8) {
                        for (int ky = 0; ky < 3; ++ky, ++qw) {
                            const int sw = int(qw % uint32_t(WS));
                            if (!tc::mbar_wait_sleep(&empty_w[sw], ((qw / uint32_t(WS)) & 1u) ^ 1u, P.err, 2)) {
                                ok = false;
                                break;
                            }
                            tc::mbar_arrive_expect_tx(&full_w[sw], Cfg::kSlice);
                            tc::tma_load_3d(sW + sw * Cfg::kSlice, &tmw, &full_w[sw], g * kPerGroup, 0, 3 * ky);
                        }
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        // Ring slots and phase parities are running counters; every channel
        // group but the last holds two K-steps.  With resident weights a
        // group is one straight run of MMAs with compile-time descriptor
        // offsets (the issue loop is the critical path of the kernel).
        if (lane == 0) {
            constexpr uint32_t idesc = FP8 ? tc::idesc_e4m3(kTileM, Cfg::kN) : tc::idesc_bf16(kTileM, Cfg::kN);
            bool ok = (!resident && !C8) || tc::mbar_wait(wready, 0, P.err, 3);
            const int nks_last = (min(kPerGroup, Cin - (G - 1) * kPerGroup) * kEsize + 31) / 32;
            const uint64_t dh0 = tc::desc_kmajor_sw64(tc::smem_u32(sHalo));
            const uint64_t dw0 = tc::desc_kmajor_sw64(tc::smem_u32(sW));
            int sh = 0, sw = 0, b = 0;
            uint32_t ph = 0, pw = 0, pb = 0;
            for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
                if (!tc::mbar_wait(&acc_empty[b], pb ^ 1u, P.err, 4)) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t d = tmem + uint32_t(b * Cfg::kTileAcc);
                for (int g = 0; g < G; ++g) {
                    // TMA completion on the mbarrier orders the halo for the tensor
                    // cores (both async proxy): no tcgen05 fence here
                    if (!tc::mbar_wait(&full_h[sh], ph, P.err, 5)) {
                        ok = false;
                        break;
                    }
                    const uint64_t da = dh0 + uint64_t((sh * kStage) >> 4);
                    const bool two = g < G - 1 || nks_last == 2;
                    const uint32_t acc0 = g != 0 ? 1u : 0u;
                    if constexpr (C8) {
                        // per output row: (ky, 0) + (ky, 1) for ky = 0..2 (second K core
                        // matrix = the next pixel, the next weight tap), (0, 2) + (1, 2)
                        // (the next halo row, three taps on), (2, 2) + the zero tap
                        constexpr uint32_t kHR = kC8Px * 16, kT = C8Cfg<COUT>::kTap;
                        const uint32_t h0 = tc::smem_u32(sHalo + sh * kStage) + (P.x_quads ? 3u * 16u : 0u);
                        const uint32_t w0 = tc::smem_u32(sW);
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            const uint32_t dr = d + uint32_t(r * Cfg::kAcc);
                            const uint32_t hr = h0 + uint32_t(r) * kHR;
                            uint64_t a[5], bw[5];
#pragma unroll
                            for (int ky = 0; ky < 3; ++ky) {
                                a[ky] = tc::desc_kmajor_plain(hr + ky * kHR, 16, 128);
                                bw[ky] = tc::desc_kmajor_plain(w0 + 3 * ky * kT, kT, 128);
                            }
                            a[3] = tc::desc_kmajor_plain(hr + 2 * 16, kHR, 128);
                            bw[3] = tc::desc_kmajor_plain(w0 + 2 * kT, 3 * kT, 128);
                            a[4] = tc::desc_kmajor_plain(hr + 2 * kHR + 2 * 16, 16, 128);
                            bw[4] = tc::desc_kmajor_plain(w0 + 8 * kT, kT, 128);
#pragma unroll
                            for (int i = 0; i < 5; ++i) {
                                if (FP8)
                                    tc::mma_e4m3(dr, a[i], bw[i], idesc, i != 0 ? 1u : acc0);
                                else
                                    tc::mma_bf16(dr, a[i], bw[i], idesc, i != 0 ? 1u : acc0);
                            }
                        }
                    } else if (resident) {
                        const uint64_t db = dw0 + uint64_t((g * Cfg::kGroup) >> 4);
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            // output row r: its accumulator, the halo from row r on
                            const uint32_t dr = d + uint32_t(r * Cfg::kAcc);
                            const uint64_t dar = da + uint64_t((r * Cfg::kHaloPx * kRow) >> 4);
                            if constexpr (Cfg::kFold) {
                                if (two)
                                    mma_fold<FP8, 2, 3>(dr, dar, db, idesc, acc0);
                                else
                                    mma_fold<FP8, 1, 3>(dr, dar, db, idesc, acc0);
                            } else {
                                if (two)
                                    mma_group<COUT, FP8, 2>(dr, dar, db, idesc, acc0);
                                else
                                    mma_group<COUT, FP8, 1>(dr, dar, db, idesc, acc0);
                            }
                        }
                    } else {
                        for (int ky = 0; ky < 3; ++ky) {
                            if (!tc::mbar_wait(&full_w[sw], pw, P.err, 6)) {
                                ok = false;
                                break;
                            }
                            const uint64_t db = dw0 + uint64_t((sw * Cfg::kSlice) >> 4);
                            const uint32_t a0 = acc0 | (ky != 0 ? 1u : 0u);
#pragma unroll
                            for (int r = 0; r < R; ++r) {
                                const uint32_t dr = d + uint32_t(r * Cfg::kAcc);
                                const uint64_t dak = da + uint64_t(((r + ky) * Cfg::kHaloPx * kRow) >> 4);
                                if constexpr (Cfg::kFold) {
                                    if (two)
                                        mma_fold<FP8, 2, 1>(dr, dak, db, idesc, a0);
                                    else
                                        mma_fold<FP8, 1, 1>(dr, dak, db, idesc, a0);
                                } else {
                                    if (two)
                                        mma_row<COUT, FP8, 2>(dr, dak, db, idesc, a0);
                                    else
                                        mma_row<COUT, FP8, 1>(dr, dak, db, idesc, a0);
                                }
                            }
                            tc::mma_commit(&empty_w[sw]);      // the slice is free once these finish
                            if (++sw == WS) {
                                sw = 0;
                                pw ^= 1u;
                            }
                        }
                        if (!ok) break;
                    }
                    tc::mma_commit(&empty_h[sh]);              // the halo slot is free once these finish
                    if (++sh == HS) {
                        sh = 0;
                        ph ^= 1u;
                    }
                }
                if (!ok) break;
                tc::mma_commit(&acc_full[b]);                  // the tile's accumulator is complete
                if (++b == Cfg::kNumAcc) {
                    b = 0;
                    pb ^= 1u;
                }
            }
            tc::mma_commit(drain);                             // every issued MMA has finished
        }
    } else {
        // ------------------------------------------------------------ epilogue
        // Group eg = (w - 2) / 4 takes the tiles tl = eg, eg + 2, ... of this
        // CTA.  Thread (warp w, lane l) owns output pixel x0 + 32 (w mod 4) + l
        // of each row; every lane runs the arithmetic (the shuffles of the
        // pooling need the whole warp) and only lanes inside the image load
        // or store.  With tma_out the rounded values go, one chunk of up to 64
        // channels at a time, into the warp's staging buffer (rows of 32
        // pixels, swizzled like the tensor map) and lane 0 stores the chunk
        // with one TMA store (four with up2) while the warp moves on;
        // otherwise every thread stores its pixel's channels itself.
        //
        // With pool_y (cout <= 64, an even number of rows per tile) the packed
        // outputs of the top row of each row pair stay in registers; at the
        // bottom row lanes 2i and 2i+1 pool pixel pair i unit by unit, the
        // even lane taking the first half of each unit's channels.
        const int qd = warp & 3, ew = warp - 2, eg = ew >> 2;
        constexpr int kPoolW = COUT <= 64 ? (FP8 ? COUT / 4 : COUT / 2) : 1;   // packed words per pixel
        uint32_t ptop[kPoolW];
#pragma unroll
        for (int i = 0; i < kPoolW; ++i) ptop[i] = 0u;
        const bool ev = (lane & 1) == 0;
        int nst = 0;                                               // chunks this warp has staged
        for (int tile = blockIdx.x + eg * gridDim.x, tl = eg; tile < n_tiles; tile += 2 * gridDim.x, tl += 2) {
            const int b = tl % Cfg::kNumAcc;
            if (!tc::mbar_wait_sleep(&acc_full[b], (tl / Cfg::kNumAcc) & 1, P.err, 7)) break;
            tc::fence_after_sync();
            const int xt = tile % P.tiles_x, rb = tile / P.tiles_x;
            const int y0 = (rb % tiles_y) * R, n = rb / tiles_y;
            const int xw = xt * Cfg::kTileOut + qd * Cfg::kQuad, x = xw + lane;
            const bool xin = lane < Cfg::kQuad && x < Wd;
            const bool pair_in = lane < Cfg::kQuad && (x | 1) < Wd;   // both pixels of this lane's pooling pair
            const bool stage = tma_out && xw < Wd;                 // (uniform over the warp)
#pragma unroll 1
            for (int rr = 0; rr < R; ++rr) {
                const int y = y0 + rr;
                if (y >= H) break;                                 // rows past the image (last tile)
                size_t opix = (size_t(n) * H + y) * Wd + x;
                if (P.up2)                                         // top-left of the 2 x 2 block
                    opix = (size_t(n) * 2 * H + 2 * y) * (2 * size_t(Wd)) + 2 * size_t(x);
                const size_t rowstep = 2 * size_t(Wd);            // up2: the next output row
                const size_t pp = (size_t(n) * (H / 2) + (y >> 1)) * size_t(Wd / 2) + (x >> 1);   // pooled pixel
                const bool pool_row = COUT <= 64 && P.pool_y && (rr & 1);
                // the head's colour input, fetched before the accumulator is read
                float hrgb[3] = {0.0f, 0.0f, 0.0f};
                if (COUT <= 64 && P.head_w && xin) {
                    const size_t p = (size_t(n) * H + y) * Wd + x;
#pragma unroll
                    for (int k = 0; k < 3; ++k) hrgb[k] = float(P.head_rgb[3 * p + k]);
                }
                const uint32_t taddr = tmem + (uint32_t(qd * 32) << 16) + uint32_t(b * Cfg::kTileAcc + rr * Cfg::kAcc);
                // up to 64 columns per TMEM round trip, in units of 16
#pragma unroll 1
                for (int c0 = 0; c0 < COUT; c0 += 64) {
                    uint32_t r[4][16];
                    const int nu = COUT <= 64 ? COUT / 16 : min(4, (COUT - c0) / 16);
                    const int row_bytes = nu * 16 * kEsize;
                    uint8_t* const obuf = sOut + (ew * tma_out + (tma_out == 2 ? (nst & 1) : 0)) * kOutBuf;
                    uint8_t* ob = obuf + lane * row_bytes;
                    const int swz = out_swizzle(row_bytes, lane);
                    if (stage) {
                        if (lane == 0) {                           // the buffer's previous store has read it
                            if (tma_out == 2)
                                tc::bulk_wait_read<1>();
                            else
                                tc::bulk_wait_read<0>();
                        }
                        __syncwarp();
                    }
                    if constexpr (Cfg::kFold) {
                        // the three kx partial sums of output pixel x are in lanes l, l+1, l+2
                        uint32_t t0[32], t1[32], t2[32];
                        tc::tmem_ld_x32(taddr, t0);
                        tc::tmem_ld_x32(taddr + 32u, t1);
                        tc::tmem_ld_x32(taddr + 64u, t2);
                        tc::tmem_ld_wait();
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const float s1 = __uint_as_float(__shfl_down_sync(~0u, t1[j], 1));
                            const float s2 = __uint_as_float(__shfl_down_sync(~0u, t2[j], 2));
                            r[j >> 4][j & 15] = __float_as_uint(__uint_as_float(t0[j]) + s1 + s2);
                        }
                    }
                    // as few TMEM loads as the chunk allows (32 columns each, 16 for an odd unit)
#pragma unroll
                    for (int h = 0; h < 2 && !Cfg::kFold; ++h) {
                        if (2 * h + 1 < nu) {
                            uint32_t t[32];
                            tc::tmem_ld_x32(taddr + uint32_t(c0 + 32 * h), t);
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                r[2 * h][j] = t[j];
                                r[2 * h + 1][j] = t[16 + j];
                            }
                        } else if (2 * h < nu) {
                            tc::tmem_ld_x16(taddr + uint32_t(c0 + 32 * h), r[2 * h]);
                        }
                    }
                    tc::tmem_ld_wait();
                    // fused 1x1 head: one chain per output channel over the
                    // rounded activations in channel order
                    float hr[3] = {0.0f, 0.0f, 0.0f};
                    if (COUT <= 64 && P.head_w)
                        for (int k = 0; k < 3; ++k) hr[k] = s_head[3 * COUT + k];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (u >= nu) break;
                        const int c = c0 + 16 * u;
                        float v[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[u][j]) * P.acc_scale + s_bias[c + j];
                        if (P.relu) {
#pragma unroll
                            for (int j = 0; j < 16; ++j) v[j] = fmaxf(v[j], 0.0f);
                        }
                        // the unit as packed words: 4 of 4 e4m3 codes or 8 of 2 bf16
                        constexpr int kW = FP8 ? 4 : 8;
                        uint32_t w[kW];
                        if (FP8) {
                            const float sc = P.out_inv_scale;
#pragma unroll
                            for (int m = 0; m < 4; ++m)
                                w[m] = pack_e4m3x4(v[4 * m] * sc, v[4 * m + 1] * sc, v[4 * m + 2] * sc, v[4 * m + 3] * sc);
                        } else {
                            if (P.mask && xin) {
                                const __nv_bfloat16* mk = P.mask + opix * COUT + c;
#pragma unroll
                                for (int j = 0; j < 16; j += 2) {
                                    const __nv_bfloat162 mm = *reinterpret_cast<const __nv_bfloat162*>(mk + j);
                                    if (!(__bfloat162float(mm.x) > 0.0f)) v[j] = 0.0f;
                                    if (!(__bfloat162float(mm.y) > 0.0f)) v[j + 1] = 0.0f;
                                }
                            }
#pragma unroll
                            for (int m = 0; m < kW; ++m) w[m % kW] = pack_bf16x2(v[2 * m], v[2 * m + 1]);
                        }
                        if constexpr (COUT <= 64) {
                            if (P.head_w) {
#pragma unroll
                                for (int j = 0; j < 16; ++j) {
                                    float a;
                                    if (FP8) {
                                        const __nv_fp8_storage_t b8 =
                                            __nv_fp8_storage_t((w[(j >> 2) % kW] >> (8 * (j & 3))) & 0xFFu);
                                        a = __half2float(__half(__nv_cvt_fp8_to_halfraw(b8, __NV_E4M3))) * P.head_scale;
                                    } else {
                                        const uint32_t wj = w[(j >> 1) % kW];
                                        a = __uint_as_float((j & 1) ? (wj & 0xFFFF0000u) : (wj << 16));
                                    }
#pragma unroll
                                    for (int k = 0; k < 3; ++k) {
                                        const float4 w4 = reinterpret_cast<const float4*>(s_head + k * COUT + c)[j >> 2];
                                        const float wk = (j & 3) == 0 ? w4.x : (j & 3) == 1 ? w4.y : (j & 3) == 2 ? w4.z : w4.w;
                                        hr[k] += wk * a;
                                    }
                                }
                                continue;                          // the activations themselves are not stored
                            }
                            if (P.pool_y) {
                                if (!pool_row) {
#pragma unroll
                                    for (int m = 0; m < kW; ++m) ptop[(kW * u + m) % kPoolW] = w[m];
                                } else {
                                    // candidates in window order: (top, even), (top, odd), (bottom, even), (bottom, odd)
                                    constexpr int kH = kW / 2;
                                    uint32_t pw[kH], pa[kH];
#pragma unroll
                                    for (int i = 0; i < kH; ++i) {
                                        const uint32_t t_lo = ptop[(kW * u + i) % kPoolW], t_hi = ptop[(kW * u + kH + i) % kPoolW];
                                        const uint32_t ot = __shfl_xor_sync(~0u, ev ? t_hi : t_lo, 1);
                                        const uint32_t obm = __shfl_xor_sync(~0u, ev ? w[kH + i] : w[i], 1);
                                        const uint32_t mt = ev ? t_lo : t_hi, mb = ev ? w[i] : w[kH + i];
                                        const uint32_t cand[4] = {ev ? mt : ot, ev ? ot : mt, ev ? mb : obm, ev ? obm : mb};
                                        pa[i] = 0u;
                                        pw[i] = FP8 ? pool4_e4m3(cand) : pool4_bf16(cand, &pa[i]);
                                    }
                                    if (pair_in) {
                                        // this lane's 8 channels of the unit: c + 8 (odd lane)
                                        const size_t pc = pp * COUT + c + (ev ? 0 : 8);
                                        if (FP8) {
                                            *reinterpret_cast<uint2*>(reinterpret_cast<uint8_t*>(P.pool_y) + pc) =
                                                make_uint2(pw[0], pw[1 % kH]);
                                        } else {
                                            *reinterpret_cast<uint4*>(P.pool_y + pc) =
                                                make_uint4(pw[0], pw[1 % kH], pw[2 % kH], pw[3 % kH]);
                                            if (P.pool_arg) {
                                                uint32_t ab[2];
#pragma unroll
                                                for (int i = 0; i < 2; ++i) {
                                                    const uint32_t a0 = pa[(2 * i) % kH], a1 = pa[(2 * i + 1) % kH];
                                                    ab[i] = (a0 & 0xFFu) | ((a0 >> 16) << 8) | ((a1 & 0xFFu) << 16) |
                                                            ((a1 >> 16) << 24);
                                                }
                                                *reinterpret_cast<uint2*>(P.pool_arg + pc) = make_uint2(ab[0], ab[1]);
                                            }
                                        }
                                    }
                                }
                            }
                        }
                        if (stage) {
                            if (FP8) {
                                *reinterpret_cast<uint4*>(ob + ((u ^ swz) << 4)) = make_uint4(w[0], w[1], w[2], w[3]);
                            } else {
                                *reinterpret_cast<uint4*>(ob + (((2 * u) ^ swz) << 4)) =
                                    make_uint4(w[0], w[1], w[2], w[3]);
                                *reinterpret_cast<uint4*>(ob + (((2 * u + 1) ^ swz) << 4)) =
                                    make_uint4(w[4 % kW], w[5 % kW], w[6 % kW], w[7 % kW]);
                            }
                            continue;
                        }
                        if (!xin) continue;
                        if (FP8) {
                            uint8_t* dst = reinterpret_cast<uint8_t*>(P.y) + opix * P.ldy + P.coff + c;
                            const uint4 q = make_uint4(w[0], w[1], w[2], w[3]);
                            *reinterpret_cast<uint4*>(dst) = q;
                            if (P.up2) {
                                const size_t ld = size_t(P.ldy);
                                *reinterpret_cast<uint4*>(dst + ld) = q;
                                *reinterpret_cast<uint4*>(dst + rowstep * ld) = q;
                                *reinterpret_cast<uint4*>(dst + (rowstep + 1) * ld) = q;
                            }
                        } else {
                            __nv_bfloat16* dst = P.y + opix * P.ldy + P.coff + c;
                            const uint4 q0 = make_uint4(w[0], w[1], w[2], w[3]);
                            const uint4 q1 = make_uint4(w[4 % kW], w[5 % kW], w[6 % kW], w[7 % kW]);
                            const int nst = P.up2 ? 4 : 1;
                            for (int k = 0; k < nst; ++k) {
                                const size_t off = (k >> 1) * rowstep + (k & 1);     // pixels from the first
                                uint4* d4 = reinterpret_cast<uint4*>(dst + off * P.ldy);
                                d4[0] = q0;
                                d4[1] = q1;
                            }
                        }
                    }
                    if (COUT <= 64 && P.head_w && xin) {
                        // s = rgb / 255 + (W d1 + b); out = round(255 clamp(s, 0, 1))
                        const size_t p = (size_t(n) * H + y) * Wd + x;
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            const float sv = hrgb[k] * (1.0f / 255.0f) + hr[k];
                            const float pr = fminf(fmaxf(sv, 0.0f), 1.0f);
                            if (P.head_f32) P.head_f32[3 * p + k] = pr;
                            if (P.head_out) {
                                const size_t yy = p / size_t(Wd), xx = p % size_t(Wd);
                                P.head_out[yy * P.head_pitch + 3 * xx + k] = uint8_t(floorf(pr * 255.0f + 0.5f));
                            }
                        }
                    }
                    if (stage) {
                        tc::fence_proxy_async_smem();              // the staged rows, visible to the TMA unit
                        __syncwarp();
                        if (lane == 0) {                           // pixels past the image are clipped
                            const CUtensorMap* m = (COUT <= 64 || c0 + 64 <= COUT) ? &tmy : &tmy2;
                            const uint8_t* src = obuf;
                            const int row = n * H + y;
                            if (P.up2) {
                                for (int k = 0; k < 4; ++k) tc::tma_store_5d(m, src, c0, k & 1, xw, k >> 1, row);
                            } else {
                                tc::tma_store_3d(m, src, c0, xw, row);
                            }
                            tc::bulk_commit();
                        }
                        ++nst;
                    }
                }
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&acc_empty[b]);
        }
        if (tma_out && lane == 0) tc::bulk_wait<0>();          // the last stores are complete
    }
    if (warp == 1 && lane == 0) tc::mbar_wait_drain(drain, 0);  // before TMEM is released
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) tc::tmem_dealloc(tmem, Cfg::kTmemCols);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// x: [NB][H][W][C], halo box {one 64-byte channel group, px pixels, rows, 1 image}
cudaError_t make_halo_map(CUtensorMap* m, const void* x, int NB, int H, int W, int C, bool fp8, int px, int rows)
{
    auto enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t es = fp8 ? 1 : 2;
    const cuuint64_t dims[4] = {cuuint64_t(C), cuuint64_t(W), cuuint64_t(H), cuuint64_t(NB)};
    const cuuint64_t strides[3] = {cuuint64_t(C) * es, cuuint64_t(W) * C * es, cuuint64_t(H) * W * C * es};
    const cuuint32_t box[4] = {cuuint32_t(kRow / es), cuuint32_t(px), cuuint32_t(rows), 1};
    const cuuint32_t el[4] = {1, 1, 1, 1};
    CUresult r = enc(m, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4,
                     const_cast<void*>(x), dims, strides, box, el, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// w: [cout][9][cin] seen as (cin, cout, tap); box {one channel group, cout, 3 taps}
cudaError_t make_weight_map(CUtensorMap* m, const void* w, int cout, int cin, bool fp8)
{
    auto enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t es = fp8 ? 1 : 2;
    const cuuint64_t dims[3] = {cuuint64_t(cin), cuuint64_t(cout), 9};
    const cuuint64_t strides[2] = {cuuint64_t(9) * cin * es, cuuint64_t(cin) * es};
    const cuuint32_t box[3] = {cuuint32_t(kRow / es), cuuint32_t(cout), 3};
    const cuuint32_t el[3] = {1, 1, 1};
    CUresult r = enc(m, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                     const_cast<void*>(w), dims, strides, box, el, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// C8: x [NB][H][W] pixels of 16 bytes (8 bf16 channels, or 16 e4m3 bytes),
// halo box {16 bytes, kC8Px pixels, rows, 1 image}, no swizzle; quads (W a
// multiple of 4): the same bytes as rows of four pixels, box {64 bytes,
// kC8Px / 4 quads, rows, 1}
cudaError_t make_halo_map_c8(CUtensorMap* m, const void* x, int NB, int H, int W, bool fp8, int rows, bool quads)
{
    auto enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t px = quads ? 4 : 1;                          // pixels per copied row
    const cuuint64_t ch = (fp8 ? 16 : 8) * px;
    const cuuint64_t dims[4] = {ch, cuuint64_t(W) / px, cuuint64_t(H), cuuint64_t(NB)};
    const cuuint64_t strides[3] = {16 * px, cuuint64_t(W) * 16, cuuint64_t(H) * W * 16};
    const cuuint32_t box[4] = {cuuint32_t(ch), cuuint32_t(kC8Px / px), cuuint32_t(rows), 1};
    const cuuint32_t el[4] = {1, 1, 1, 1};
    CUresult r = enc(m, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4,
                     const_cast<void*>(x), dims, strides, box, el, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// C8: w [cout][9][16 bytes] seen as (16 bytes, cout, tap); one box of all nine
// taps lands tap by tap, each tap a COUT x 16-byte tile
cudaError_t make_weight_map_c8(CUtensorMap* m, const void* w, int cout, bool fp8)
{
    auto enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t ch = fp8 ? 16 : 8;
    const cuuint64_t dims[3] = {ch, cuuint64_t(cout), 9};
    const cuuint64_t strides[2] = {9 * 16, 16};
    const cuuint32_t box[3] = {cuuint32_t(ch), cuuint32_t(cout), 9};
    const cuuint32_t el[3] = {1, 1, 1};
    CUresult r = enc(m, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                     const_cast<void*>(w), dims, strides, box, el, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

int num_sms()
{
    static int n = 0;
    if (!n) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            n = v;
        else
            n = 1;
    }
    return n;
}

// y: channel c of output pixel p at y[p * ldy + coff + c]; box {chunk channels,
// 32 pixels, 1 row}.  Plain: dims (cout, W, NB*H).  up2: the [NB][2H][2W]
// tensor seen as (cout, dx, W, dy, NB*H), so that one box written at
// (c, dx, x, dy, row) lands on the pixels (2 row + dy, 2 x + dx).
cudaError_t make_out_map(CUtensorMap* m, void* y, int NB, int H, int W, int ldy, int coff, int cout, int chunk,
                         int quad, bool fp8, bool up2)
{
    auto enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t es = fp8 ? 1 : 2;
    const cuuint64_t px = cuuint64_t(ldy) * es;
    char* base = static_cast<char*>(y) + size_t(coff) * es;
    if ((reinterpret_cast<uintptr_t>(base) & 15) || (px & 15)) return cudaErrorInvalidValue;
    const int row_bytes = chunk * int(es);
    const CUtensorMapSwizzle sw = row_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                  : row_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                  : row_bytes == 32 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_NONE;
    const CUtensorMapDataType dt = fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    CUresult r;
    if (up2) {
        const cuuint64_t dims[5] = {cuuint64_t(cout), 2, cuuint64_t(W), 2, cuuint64_t(NB) * H};
        const cuuint64_t strides[4] = {px, 2 * px, 2 * cuuint64_t(W) * px, 4 * cuuint64_t(W) * px};
        const cuuint32_t box[5] = {cuuint32_t(chunk), 1, cuuint32_t(quad), 1, 1};
        const cuuint32_t el[5] = {1, 1, 1, 1, 1};
        r = enc(m, dt, 5, base, dims, strides, box, el, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
        const cuuint64_t dims[3] = {cuuint64_t(cout), cuuint64_t(W), cuuint64_t(NB) * H};
        const cuuint64_t strides[2] = {px, cuuint64_t(W) * px};
        const cuuint32_t box[3] = {cuuint32_t(chunk), cuuint32_t(quad), 1};
        const cuuint32_t el[3] = {1, 1, 1};
        r = enc(m, dt, 3, base, dims, strides, box, el, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int COUT, bool FP8, bool FOLD = false, bool WIDE = false, bool C8 = false>
cudaError_t launch_conv(const void* x, const void* w, ConvArgs a, cudaStream_t s)
{
    constexpr int kPerGroup = FP8 ? 64 : 32;
    const int G = (a.Cin + kPerGroup - 1) / kPerGroup;
    // Staged TMA stores pay where a warp's own stores would scatter: into a
    // channel slice of a wider tensor, or four times for the upsampling.  A
    // dense output is already written in whole lines by the threads.
    const bool want_out = a.up2 || a.ldy != COUT || a.coff != 0;
    Plan p = C8 ? make_plan_c8<COUT>(FP8, want_out) : make_plan<COUT, FOLD, WIDE>(G, FP8, want_out);
    if (p.hs < 2 || (!p.resident && p.ws < 2)) return cudaErrorInvalidValue;
    CUtensorMap mx, mw, my, my2;
    using C = ConvCfg<COUT, FOLD, WIDE>;
    a.tiles_x = (a.W + C::kTileOut - 1) / C::kTileOut;
    a.x_quads = C8 && a.W % 4 == 0;
    cudaError_t e = C8         ? make_halo_map_c8(&mx, x, a.NB, a.H, a.W, FP8, C::kHaloRows, a.x_quads != 0)
                    : C::kFold ? make_halo_map(&mx, x, a.NB, a.H, a.W, a.xstride, FP8, 32, 1)
                               : make_halo_map(&mx, x, a.NB, a.H, a.W, a.xstride, FP8, C::kHaloPx, C::kHaloRows);
    if (e != cudaSuccess) return e;
    e = C8 ? make_weight_map_c8(&mw, w, COUT, FP8) : make_weight_map(&mw, w, COUT, a.Cin, FP8);
    if (e != cudaSuccess) return e;
    my = mw;                                           // unused unless the output maps are made
    my2 = mw;
    if (p.out) {
        // a layout the tensor maps cannot describe keeps the per-thread stores
        const int tail = COUT > 64 ? COUT % 64 : 0;
        if (make_out_map(&my, a.y, a.NB, a.H, a.W, a.ldy, a.coff, COUT, C::kChunk, C::kQuad, FP8, a.up2 != 0) !=
                cudaSuccess ||
            (tail && make_out_map(&my2, a.y, a.NB, a.H, a.W, a.ldy, a.coff, COUT, tail, C::kQuad, FP8, a.up2 != 0) !=
                         cudaSuccess))
            p.out = 0;
    }
    e = cudaFuncSetAttribute(k_conv3x3_tc<COUT, FP8, FOLD, WIDE, C8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             p.smem);
    if (e != cudaSuccess) return e;
    const long long tiles = (long long)a.tiles_x * a.NB * ((a.H + C::kRows - 1) / C::kRows);
    const int grid = int(std::min<long long>(tiles, num_sms()));
    k_conv3x3_tc<COUT, FP8, FOLD, WIDE, C8><<<grid, kThreads, p.smem, s>>>(mx, mw, my, my2, a, int(tiles), p.hs, p.ws,
                                                                      p.resident, p.out);
    return cudaGetLastError();
}

// Whether the one-row plan of a layer streams its weights.
template <int COUT>
bool streamed(const ConvArgs& a, bool fp8)
{
    const int G = (a.Cin + (fp8 ? 64 : 32) - 1) / (fp8 ? 64 : 32);
    const bool want_out = a.up2 || (a.ldy && a.ldy != COUT) || a.coff != 0;
    return !make_plan<COUT, false>(G, fp8, want_out).resident;
}

template <bool FP8>
cudaError_t dispatch(const void* x, const void* w, int Cout, const ConvArgs& a, cudaStream_t s)
{
    // 16-byte pixels (the network's input features): two taps per MMA
    const bool c8 = a.xstride * (FP8 ? 1 : 2) == 16;
    switch (Cout) {
    case 32:
        if (c8) return launch_conv<32, FP8, false, false, true>(x, w, a, s);
        // the folded form pays where the MMAs outweigh the epilogue: two or
        // more channel groups per tile.  It is kept to dense outputs without
        // the fused head (the network's uses of it)
        if (a.Cin > (FP8 ? 64 : 32) && !a.up2 && a.ldy == 32 && a.coff == 0 && !a.head_w)
            return launch_conv<32, FP8, true>(x, w, a, s);
        return launch_conv<32, FP8>(x, w, a, s);
    case 48:
        if (c8) return launch_conv<48, FP8, false, false, true>(x, w, a, s);
        return launch_conv<48, FP8>(x, w, a, s);
    case 64: return launch_conv<64, FP8>(x, w, a, s);
    case 96:
        if (streamed<96>(a, FP8)) return launch_conv<96, FP8, false, true>(x, w, a, s);
        return launch_conv<96, FP8>(x, w, a, s);
    case 128:
        if (streamed<128>(a, FP8)) return launch_conv<128, FP8, false, true>(x, w, a, s);
        return launch_conv<128, FP8>(x, w, a, s);
    case 192: return launch_conv<192, FP8>(x, w, a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() { return encode_fn(); }

bool conv_cout_supported(int cout)
{
    return cout == 32 || cout == 48 || cout == 64 || cout == 96 || cout == 128 || cout == 192;
}

bool conv_pool_supported(int cout)
{
    return cout == 32 || cout == 48 || cout == 64;                // an even number of rows per tile
}

cudaError_t launch_conv3x3(const void* x, int NB, int H, int W, int Cin, const void* w, int Cout, ConvArgs a,
                           cudaStream_t s)
{
    const bool fp8 = a.fp8 != 0;
    if (Cin < 1 || Cin % (fp8 ? 16 : 8) || NB < 1 || H < 1 || W < 1 || !conv_cout_supported(Cout))
        return cudaErrorInvalidValue;
    a.NB = NB;
    a.H = H;
    a.W = W;
    a.Cin = Cin;
    if (a.xstride == 0) a.xstride = Cin;
    if (a.mask && (a.up2 || a.coff || (a.ldy && a.ldy != Cout))) return cudaErrorInvalidValue;
    if ((a.pool_y || a.pool_arg) && (!conv_pool_supported(Cout) || !a.pool_y || !a.relu || a.up2 || a.mask))
        return cudaErrorInvalidValue;
    if (a.pool_arg && fp8) return cudaErrorInvalidValue;
    if (a.head_w && (!conv_pool_supported(Cout) || !a.head_b || !a.relu || a.up2 || a.mask || a.pool_y || a.coff ||
                     (a.ldy && a.ldy != Cout) || !a.head_rgb || (!a.head_out && !a.head_f32)))
        return cudaErrorInvalidValue;
    if (a.head_w && fp8 && !(a.head_scale > 0.0f)) return cudaErrorInvalidValue;
    if (a.xstride < Cin || a.xstride % (fp8 ? 16 : 8)) return cudaErrorInvalidValue;
    if (a.ldy == 0) a.ldy = Cout;
    if (a.acc_scale == 0.0f) a.acc_scale = 1.0f;
    if (a.out_inv_scale == 0.0f) a.out_inv_scale = 1.0f;
    return fp8 ? dispatch<true>(x, w, Cout, a, s) : dispatch<false>(x, w, Cout, a, s);
}

}  // namespace fvv
