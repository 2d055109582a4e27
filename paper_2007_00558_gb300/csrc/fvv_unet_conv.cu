// fvv_unet_conv.cu -- 3x3 convolution (pad 1) of the refinement network as
// an implicit GEMM on the sm_103a tensor cores (tcgen05, TMEM, TMA).
//
// GEMM view: M = 128 consecutive output pixels of one image row, N = the
// output channels, K = 9 taps x input channels.  For tap (ky, kx) and a
// 32-channel block, TMA loads the 128 x 32 input patch at pixel offset
// (kx - 1, ky - 1) straight from the NHWC activation tensor (zero fill
// outside the image is the convolution's padding) and the matching
// COUT x 32 block of the weights [cout][ky][kx][cin].  A 4-stage mbarrier
// ring feeds one MMA-issuing thread; the fp32 accumulators live in TMEM and
// four epilogue warps add the bias, apply ReLU and an optional ReLU-derivative
// mask, round to bf16 and store NHWC.
//
// Warp roles (192 threads): 0 = TMA producer, 1 = TMEM owner + MMA issuer,
// 2..5 = epilogue (warp w reads TMEM lanes 32 (w mod 4) .. +31).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "fvv_internal.h"
#include "fvv_tc.cuh"
#include "fvv_unet.h"

namespace fvv {

namespace {

constexpr int kStages = 4;
constexpr int kTileM = 128;
constexpr int kBlockK = 32;                       // channels per stage (64-byte rows)
constexpr int kABytes = kTileM * kBlockK * 2;     // 8 KiB

template <int COUT>
struct ConvCfg {
    static constexpr int kBBytes = COUT * kBlockK * 2;
    static constexpr int kBStride = (kBBytes + 1023) / 1024 * 1024;
    static constexpr int kTmemCols = COUT <= 32 ? 32 : COUT <= 64 ? 64 : COUT <= 128 ? 128 : 256;
    static constexpr int kSmem = 1024 + kStages * (kABytes + kBStride) + 256;
};

template <int COUT>
__global__ void __launch_bounds__(192, 1)
k_conv3x3_tc(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmw, ConvArgs P)
{
    using Cfg = ConvCfg<COUT>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = base;
    uint8_t* sB = base + kStages * kABytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + kStages * Cfg::kBStride);
    uint64_t* empty = full + kStages;
    uint64_t* done = empty + kStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    int* skip = reinterpret_cast<int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) *skip = *reinterpret_cast<volatile int*>(P.err);
    __syncthreads();
    if (*skip) return;                             // an earlier CTA gave up: do nothing

    const int tile = blockIdx.x;
    const int xt = tile % P.tiles_x;
    const int row = tile / P.tiles_x;             // n * H + y
    const int yy = row % P.H, n = row / P.H;
    const int x0 = xt * kTileM;
    const int cblocks = P.Cin / kBlockK;
    const int n_k = 9 * cblocks;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(done, 1);
        tc::fence_mbar_init();
        tc::prefetch_tensormap(&tmx);
        tc::prefetch_tensormap(&tmw);
    }
    if (warp == 1) tc::tmem_alloc(tmem_slot, Cfg::kTmemCols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {                          // TMA producer
            int issued = 0;
            for (int it = 0; it < n_k; ++it) {
                const int s = it % kStages;
                const uint32_t ph = (it / kStages) & 1;
                if (!tc::mbar_wait(&empty[s], ph ^ 1, P.err, 1)) break;
                const int tap = it / cblocks, cb = it - tap * cblocks;
                const int ky = tap / 3, kx = tap - 3 * ky;
                tc::mbar_arrive_expect_tx(&full[s], kABytes + Cfg::kBBytes);
                tc::tma_load_4d(sA + s * kABytes, &tmx, &full[s], cb * kBlockK, x0 + kx - 1, yy + ky - 1, n);
                tc::tma_load_2d(sB + s * Cfg::kBStride, &tmw, &full[s], tap * P.Cin + cb * kBlockK, 0);
                ++issued;
            }
            if (issued < n_k) {
                // gave up: let the copies still in flight land before exiting
                for (int it = (issued > kStages ? issued - kStages : 0); it < issued; ++it)
                    tc::mbar_wait_drain(&full[it % kStages], (it / kStages) & 1);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {                          // MMA issuer
            constexpr uint32_t idesc = tc::idesc_bf16(kTileM, COUT);
            for (int it = 0; it < n_k; ++it) {
                const int s = it % kStages;
                const uint32_t ph = (it / kStages) & 1;
                if (!tc::mbar_wait(&full[s], ph, P.err, 2)) break;
                tc::fence_after_sync();
                const uint32_t a = tc::smem_u32(sA + s * kABytes);
                const uint32_t b = tc::smem_u32(sB + s * Cfg::kBStride);
#pragma unroll
                for (int ks = 0; ks < kBlockK / 16; ++ks)
                    tc::mma_bf16(tmem, tc::desc_kmajor_sw64(a + 32 * ks), tc::desc_kmajor_sw64(b + 32 * ks),
                                 idesc, (it | ks) != 0);
                tc::mma_commit(&empty[s]);        // the stage is free once these MMAs finish
            }
            tc::mma_commit(done);                 // every issued MMA has finished
        }
    } else {                                      // epilogue
        const int q = warp & 3;
        const bool ok = tc::mbar_wait(done, 0, P.err, 3);
        tc::fence_after_sync();
        const int px = q * 32 + lane;
        const int x = x0 + px;
        const size_t obase = ((size_t(n) * P.H + yy) * P.W + x) * COUT;
        if (ok) {
#pragma unroll 1
            for (int c0 = 0; c0 < COUT; c0 += 32) {
                uint32_t r[32];
                tc::tmem_ld_x32(tmem + (uint32_t(q * 32) << 16) + uint32_t(c0), r);
                tc::tmem_ld_wait();
                if (x < P.W) {
                    uint32_t packed[16];
#pragma unroll
                    for (int j = 0; j < 32; j += 2) {
                        float v0 = __uint_as_float(r[j]), v1 = __uint_as_float(r[j + 1]);
                        if (P.bias) {
                            v0 += P.bias[c0 + j];
                            v1 += P.bias[c0 + j + 1];
                        }
                        if (P.relu) {
                            v0 = fmaxf(v0, 0.0f);
                            v1 = fmaxf(v1, 0.0f);
                        }
                        if (P.mask) {
                            const __nv_bfloat162 m =
                                *reinterpret_cast<const __nv_bfloat162*>(P.mask + obase + c0 + j);
                            if (!(__bfloat162float(m.x) > 0.0f)) v0 = 0.0f;
                            if (!(__bfloat162float(m.y) > 0.0f)) v1 = 0.0f;
                        }
                        const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
                        packed[j >> 1] = *reinterpret_cast<const uint32_t*>(&h);
                    }
                    uint4* dst = reinterpret_cast<uint4*>(P.y + obase + c0);
#pragma unroll
                    for (int v = 0; v < 4; ++v)
                        dst[v] = make_uint4(packed[4 * v], packed[4 * v + 1], packed[4 * v + 2], packed[4 * v + 3]);
                }
            }
        }
    }
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

template <int COUT>
cudaError_t launch_conv(const CUtensorMap& mx, const CUtensorMap& mw, const ConvArgs& a, cudaStream_t s)
{
    using Cfg = ConvCfg<COUT>;
    cudaError_t e = cudaFuncSetAttribute(k_conv3x3_tc<COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         Cfg::kSmem);
    if (e != cudaSuccess) return e;
    const unsigned tiles = unsigned(a.tiles_x) * unsigned(a.NB) * unsigned(a.H);
    k_conv3x3_tc<COUT><<<tiles, 192, Cfg::kSmem, s>>>(mx, mw, a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t make_act_map(CUtensorMap* m, const void* x, int NB, int H, int W, int C)
{
    auto enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[4] = {cuuint64_t(C), cuuint64_t(W), cuuint64_t(H), cuuint64_t(NB)};
    const cuuint64_t strides[3] = {cuuint64_t(C) * 2, cuuint64_t(W) * C * 2, cuuint64_t(H) * W * C * 2};
    const cuuint32_t box[4] = {cuuint32_t(kBlockK), cuuint32_t(kTileM), 1, 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(x), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t make_weight_map(CUtensorMap* m, const void* w, int cout, int K)
{
    auto enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {cuuint64_t(K), cuuint64_t(cout)};
    const cuuint64_t strides[1] = {cuuint64_t(K) * 2};
    const cuuint32_t box[2] = {cuuint32_t(kBlockK), cuuint32_t(cout)};
    const cuuint32_t es[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(w), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

bool conv_cout_supported(int cout)
{
    return cout == 32 || cout == 64 || cout == 96 || cout == 128 || cout == 192;
}

cudaError_t launch_conv3x3(const void* x, int NB, int H, int W, int Cin, const void* w, int Cout, ConvArgs a,
                           cudaStream_t s)
{
    CUtensorMap mx, mw;
    cudaError_t e = make_act_map(&mx, x, NB, H, W, Cin);
    if (e != cudaSuccess) return e;
    e = make_weight_map(&mw, w, Cout, 9 * Cin);
    if (e != cudaSuccess) return e;
    a.NB = NB;
    a.H = H;
    a.W = W;
    a.Cin = Cin;
    a.tiles_x = (W + kTileM - 1) / kTileM;
    switch (Cout) {
    case 32: return launch_conv<32>(mx, mw, a, s);
    case 64: return launch_conv<64>(mx, mw, a, s);
    case 96: return launch_conv<96>(mx, mw, a, s);
    case 128: return launch_conv<128>(mx, mw, a, s);
    case 192: return launch_conv<192>(mx, mw, a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace fvv
