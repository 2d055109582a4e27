// fvv_codec.cu -- the depth codec of the transmission chain (Sec. IV-A, V-A):
// 16-bit depth -> Eq. (1) correction -> Eq. (2) 12-bit disparity -> Eq. (3)
// and the bit re-arrangement onto an 8-bit YUV420 frame, and back.
//
// Both directions go through per-camera tables built on the host in FP64
// (encode: every uint16 depth code -> 12-bit code; decode: every 12-bit code
// -> uint16 depth code), so the kernels are integer-only and bound by memory:
// one thread per 2x2 block reads 4 Y bytes, one U and one V byte and writes
// four depth codes (decode), or the reverse (encode).  The decode runs fused
// into the frame upload (fvv_upload_frame_yuv): the decoded depth lands
// directly in the frame ring.
//
// Readings where the paper is silent: Eq. (2) rounds half up; bit i of the
// first pixel's 4 MSBs goes to bit 2i of U (V), the second pixel's to bit
// 2i + 1; the decoder inverts Eq. (2) as 1 / (1/z_far + (Y - 2)(1/z_near -
// 1/z_far) / 4093) and rounds to depth codes in [1, 65534]; reserved code 1
// (out of range or no depth) decodes to depth code 0 and code 0 (background)
// to the background signal 65535; depth code 0 encodes to 1 and the signal
// to 0.
#include <cmath>
#include <cstring>
#include <vector>

#include "fvv_runtime.h"

namespace fvv {

struct CodecState {
    std::vector<int> set;                   // per camera: tables built
    std::vector<fvv_depth_codec> prm;
    std::vector<uint16_t*> dec;             // [4096] per camera
    std::vector<uint16_t*> enc;             // [65536] per camera
    std::vector<uint8_t*> stage;            // host-upload staging of Y, U, V
    std::vector<size_t> stage_bytes;
};

namespace {

constexpr double kLevels = 4093.0;          // 2^12 - 3

// 12-bit code of depth code d (FP64, the operation order of the reading)
uint16_t encode_code(int d, const fvv_depth_codec& p, double unit)
{
    if (d == 0) return 1;                       // no depth
    if (d == int(kDepthBg)) return 0;           // background signal
    const double z = double(d) * unit;
    const double zc = (p.alpha * z + p.beta) * z;               // Eq. (1)
    if (!(zc >= p.z_near && zc <= p.z_far)) return 1;
    const double inv_n = 1.0 / p.z_near, inv_f = 1.0 / p.z_far;
    const double v = kLevels * (1.0 / zc - inv_f) / (inv_n - inv_f) + 2.0;   // Eq. (2)
    return uint16_t(std::floor(v + 0.5));
}

uint16_t decode_code(int y, const fvv_depth_codec& p, double unit)
{
    if (y == 0) return kDepthBg;
    if (y == 1) return 0;
    const double inv_n = 1.0 / p.z_near, inv_f = 1.0 / p.z_far;
    const double z = 1.0 / (inv_f + (double(y) - 2.0) * (inv_n - inv_f) / kLevels);
    const double d = std::floor(z / unit + 0.5);
    return uint16_t(d < 1.0 ? 1.0 : d > 65534.0 ? 65534.0 : d);
}

__device__ __forceinline__ uint32_t interleave4(uint32_t a, uint32_t b)
{
    uint32_t u = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) u |= (((a >> i) & 1u) << (2 * i)) | (((b >> i) & 1u) << (2 * i + 1));
    return u;
}

__device__ __forceinline__ void deinterleave4(uint32_t u, uint32_t& a, uint32_t& b)
{
    a = b = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        a |= ((u >> (2 * i)) & 1u) << i;
        b |= ((u >> (2 * i + 1)) & 1u) << i;
    }
}

// Eq. (3): the Y byte of a 12-bit code, and its inverse given the MSBs
__device__ __forceinline__ uint32_t fold(uint32_t y12)
{
    const uint32_t lsb = y12 & 255u;
    return ((y12 >> 8) & 1u) ? 255u - lsb : lsb;
}

__device__ __forceinline__ uint32_t unfold(uint32_t ybyte, uint32_t msb)
{
    return (msb << 8) | ((msb & 1u) ? 255u - ybyte : ybyte);
}

// Grid-stride over 2x2 blocks; the 8 KB decode table is read through the L1
// (it stays cached: staging a copy per CTA cost more traffic than the frame).
__device__ __forceinline__ void decode_block(const YuvDepth& f, const uint16_t* lut, int bx, int by,
                                             uint16_t* out, size_t opitch)
{
    const uint8_t* y0 = f.y + size_t(2 * by) * f.y_pitch + 2 * bx;
    const uint8_t* y1 = y0 + f.y_pitch;
    uint32_t m11, m12, m21, m22;
    deinterleave4(f.u[size_t(by) * f.uv_pitch + bx], m11, m12);
    deinterleave4(f.v[size_t(by) * f.uv_pitch + bx], m21, m22);
    uint16_t* r0 = reinterpret_cast<uint16_t*>(reinterpret_cast<uint8_t*>(out) + size_t(2 * by) * opitch) + 2 * bx;
    uint16_t* r1 = reinterpret_cast<uint16_t*>(reinterpret_cast<uint8_t*>(r0) + opitch);
    const uint32_t a = __ldg(lut + unfold(y0[0], m11)), b = __ldg(lut + unfold(y0[1], m12));
    const uint32_t c = __ldg(lut + unfold(y1[0], m21)), d = __ldg(lut + unfold(y1[1], m22));
    *reinterpret_cast<uint32_t*>(r0) = a | (b << 16);
    *reinterpret_cast<uint32_t*>(r1) = c | (d << 16);
}

__global__ void __launch_bounds__(512) k_yuv_decode(YuvDepth f, int bw, int bh, uint16_t* __restrict__ out,
                                                    size_t opitch)
{
    const size_t n = size_t(bw) * bh;
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
        decode_block(f, f.lut, int(i % bw), int(i / bw), out, opitch);
}

// 16 x 2 pixels (eight 2x2 blocks) per thread with 16-byte accesses: two
// 16-byte Y row pieces, 8 bytes of U and of V, four 16-byte stores of codes.
// The 4 MSBs of a pixel are the even (left pixel) or odd (right pixel) bits
// of its block's U (top row) or V (bottom row) byte, gathered by two
// mask-and-shift steps.
__device__ __forceinline__ uint32_t msb_of(uint32_t uvbyte, uint32_t right)
{
    uint32_t m = (uvbyte >> right) & 0x55u;
    m = (m | (m >> 1)) & 0x33u;
    return (m | (m >> 2)) & 0x0Fu;
}

__device__ __forceinline__ void decode_16x2(const uint8_t* y0, const uint8_t* y1, const uint8_t* u, const uint8_t* v,
                                            const uint16_t* __restrict__ lut, uint16_t* o0, uint16_t* o1)
{
    const uint4 Y0 = *reinterpret_cast<const uint4*>(y0);
    const uint4 Y1 = *reinterpret_cast<const uint4*>(y1);
    const uint2 U = *reinterpret_cast<const uint2*>(u);
    const uint2 V = *reinterpret_cast<const uint2*>(v);
    const uint32_t yw[2][4] = {{Y0.x, Y0.y, Y0.z, Y0.w}, {Y1.x, Y1.y, Y1.z, Y1.w}};
    const uint32_t cw[2][2] = {{U.x, U.y}, {V.x, V.y}};
    uint32_t out[2][8];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {                 // pixels 4q .. 4q + 3: blocks 2q, 2q + 1
            const uint32_t cb = cw[r][q >> 1] >> (16 * (q & 1));
#pragma unroll
            for (int h = 0; h < 2; ++h) {             // block 2q + h: pixels 4q + 2h (left), 4q + 2h + 1 (right)
                const uint32_t byte = (cb >> (8 * h)) & 0xFFu;
                uint32_t codes = 0;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const uint32_t yb = (yw[r][q] >> (8 * (2 * h + e))) & 0xFFu;
                    const uint32_t m = msb_of(byte, uint32_t(e));
                    const uint32_t y12 = (m << 8) | ((m & 1u) ? 255u - yb : yb);
                    codes |= uint32_t(__ldg(lut + y12)) << (16 * e);
                }
                out[r][2 * q + h] = codes;
            }
        }
    }
    uint4* d0 = reinterpret_cast<uint4*>(o0);
    uint4* d1 = reinterpret_cast<uint4*>(o1);
    d0[0] = make_uint4(out[0][0], out[0][1], out[0][2], out[0][3]);
    d0[1] = make_uint4(out[0][4], out[0][5], out[0][6], out[0][7]);
    d1[0] = make_uint4(out[1][0], out[1][1], out[1][2], out[1][3]);
    d1[1] = make_uint4(out[1][4], out[1][5], out[1][6], out[1][7]);
}

// Frames of cameras 0 .. n-1 of one size: camera k's planes at y/u/v + k *
// cam_stride, its codes at out + k * out_cam_stride.  Work item = (camera,
// block row, 16-pixel column group), grid-stride.
struct YuvFrames {
    const uint8_t *y, *u, *v;
    size_t y_pitch, uv_pitch, cam_stride;
    uint16_t* out;
    size_t out_pitch, out_cam_stride;
    int groups, block_rows, n;
    const uint16_t* lut[kMaxCams];
};

__global__ void __launch_bounds__(256) k_yuv_decode16(const __grid_constant__ YuvFrames f)
{
    const size_t per_cam = size_t(f.groups) * f.block_rows;
    const size_t n = per_cam * f.n;
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
        const int k = int(i / per_cam);
        const size_t r = i - size_t(k) * per_cam;
        const int by = int(r / f.groups), g = int(r - size_t(by) * f.groups);
        const size_t cs = size_t(k) * f.cam_stride;
        const uint8_t* y0 = f.y + cs + size_t(2 * by) * f.y_pitch + 16 * g;
        const size_t uvo = cs + size_t(by) * f.uv_pitch + 8 * g;
        uint16_t* o0 = reinterpret_cast<uint16_t*>(reinterpret_cast<uint8_t*>(f.out) + size_t(k) * f.out_cam_stride +
                                                   size_t(2 * by) * f.out_pitch) + 16 * g;
        uint16_t* o1 = reinterpret_cast<uint16_t*>(reinterpret_cast<uint8_t*>(o0) + f.out_pitch);
        decode_16x2(y0, y0 + f.y_pitch, f.u + uvo, f.v + uvo, f.lut[k], o0, o1);
    }
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// The 16-byte form applies when every access it makes is aligned.
bool vec16_ok(const YuvFrames& f, int width)
{
    return width % 16 == 0 && aligned(f.y, 16) && f.y_pitch % 16 == 0 && aligned(f.u, 8) && aligned(f.v, 8) &&
           f.uv_pitch % 8 == 0 && f.cam_stride % 16 == 0 && aligned(f.out, 16) && f.out_pitch % 16 == 0 &&
           f.out_cam_stride % 16 == 0;
}

int device_sm_count()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
            sms = 1;
    }
    return sms;
}

cudaError_t launch_decode16(const YuvFrames& f, cudaStream_t s)
{
    const size_t n = size_t(f.groups) * f.block_rows * f.n;
    if (n == 0) return cudaSuccess;
    const size_t want = (n + 255) / 256, cap = size_t(device_sm_count()) * 8;
    k_yuv_decode16<<<unsigned(want < cap ? want : cap), 256, 0, s>>>(f);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_yuv_encode(const uint16_t* __restrict__ depth, size_t dpitch, int bw,
                                                    int bh, const uint16_t* __restrict__ lut, uint8_t* __restrict__ y,
                                                    size_t ypitch, uint8_t* __restrict__ u, uint8_t* __restrict__ v,
                                                    size_t uvpitch)
{
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= size_t(bw) * bh) return;
    const int bx = int(i % bw), by = int(i / bw);
    const uint16_t* d0 =
        reinterpret_cast<const uint16_t*>(reinterpret_cast<const uint8_t*>(depth) + size_t(2 * by) * dpitch) + 2 * bx;
    const uint16_t* d1 = reinterpret_cast<const uint16_t*>(reinterpret_cast<const uint8_t*>(d0) + dpitch);
    const uint32_t p11 = __ldg(lut + d0[0]), p12 = __ldg(lut + d0[1]);
    const uint32_t p21 = __ldg(lut + d1[0]), p22 = __ldg(lut + d1[1]);
    uint8_t* yr0 = y + size_t(2 * by) * ypitch + 2 * bx;
    uint8_t* yr1 = yr0 + ypitch;
    yr0[0] = uint8_t(fold(p11));
    yr0[1] = uint8_t(fold(p12));
    yr1[0] = uint8_t(fold(p21));
    yr1[1] = uint8_t(fold(p22));
    u[size_t(by) * uvpitch + bx] = uint8_t(interleave4(p11 >> 8, p12 >> 8));
    v[size_t(by) * uvpitch + bx] = uint8_t(interleave4(p21 >> 8, p22 >> 8));
}

bool on_dev(const void* p) { return p && mem_kind(p) == MemKind::Device; }

fvv_status check_cam(fvv_ctx* c, int32_t cam)
{
    if (!c) return fail(FVV_ERR_INVALID_ARG, "ctx is NULL");
    if (cam < 0 || cam >= c->n_cams) return fail(FVV_ERR_INVALID_ARG, "camera index out of range");
    if (c->cams[cam].width % 2 || c->cams[cam].height % 2)
        return fail(FVV_ERR_INVALID_ARG, "YUV420 depth needs even width and height");
    if (!c->codec || !c->codec->set[cam]) return fail(FVV_ERR_STATE, "no depth codec set for this camera");
    return FVV_OK;
}

}  // namespace

cudaError_t launch_yuv_decode(const YuvDepth& f, int width, int height, uint16_t* out, size_t out_pitch,
                              cudaStream_t s)
{
    const int bw = width / 2, bh = height / 2;
    const size_t n = size_t(bw) * bh;
    if (n == 0) return cudaSuccess;
    YuvFrames v{};
    v.y = f.y;
    v.u = f.u;
    v.v = f.v;
    v.y_pitch = f.y_pitch;
    v.uv_pitch = f.uv_pitch;
    v.cam_stride = 0;
    v.out = out;
    v.out_pitch = out_pitch;
    v.out_cam_stride = 0;
    v.groups = width / 16;
    v.block_rows = bh;
    v.n = 1;
    v.lut[0] = f.lut;
    if (vec16_ok(v, width)) return launch_decode16(v, s);
    const int sms = device_sm_count();
    const size_t want = (n + 511) / 512;
    const unsigned grid = unsigned(want < size_t(2 * sms) ? want : size_t(2 * sms));
    k_yuv_decode<<<grid, 512, 0, s>>>(f, bw, bh, out, out_pitch);
    return cudaGetLastError();
}

const uint16_t* codec_decode_table(fvv_ctx* c, int cam)
{
    CodecState* K = c->codec;
    if (!K || cam < 0 || cam >= int(K->set.size()) || !K->set[cam]) return nullptr;
    return K->dec[cam];
}

void codec_destroy(fvv_ctx* c)
{
    CodecState* K = c->codec;
    if (!K) return;
    for (int k = 0; k < c->n_cams; ++k) {
        dev_free(c, K->dec[k], 4096 * sizeof(uint16_t));
        dev_free(c, K->enc[k], 65536 * sizeof(uint16_t));
        dev_free(c, K->stage[k], K->stage_bytes[k]);
    }
    delete K;
    c->codec = nullptr;
}

}  // namespace fvv

using fvv::fail;

extern "C" {

fvv_status fvv_depth_codec_default(fvv_depth_codec* p)
{
    if (!p) return fail(FVV_ERR_INVALID_ARG, "codec is NULL");
    p->z_near = 0.3;
    p->z_far = 10.0;
    p->alpha = 0.0;
    p->beta = 1.0;
    return FVV_OK;
}

fvv_status fvv_set_depth_codec(fvv_ctx* c, int32_t cam, const fvv_depth_codec* p)
{
    if (!c || !p) return fail(FVV_ERR_INVALID_ARG, "NULL argument");
    if (cam < 0 || cam >= c->n_cams) return fail(FVV_ERR_INVALID_ARG, "camera index out of range");
    if (!(p->z_near > 0.0) || !(p->z_far > p->z_near) || !std::isfinite(p->z_far) || !std::isfinite(p->alpha) ||
        !std::isfinite(p->beta))
        return fail(FVV_ERR_INVALID_ARG, "need 0 < z_near < z_far and finite alpha, beta");
    std::lock_guard<std::recursive_mutex> g(c->mu);
    fvv::DeviceScope dev_scope(c->device);
    if (!c->codec) {
        auto* K = new fvv::CodecState();
        K->set.assign(c->n_cams, 0);
        K->prm.resize(c->n_cams);
        K->dec.assign(c->n_cams, nullptr);
        K->enc.assign(c->n_cams, nullptr);
        K->stage.assign(c->n_cams, nullptr);
        K->stage_bytes.assign(c->n_cams, 0);
        c->codec = K;
    }
    fvv::CodecState* K = c->codec;
    if (!K->dec[cam]) FVV_TRY(fvv::dev_alloc(c, reinterpret_cast<void**>(&K->dec[cam]), 4096 * sizeof(uint16_t)));
    if (!K->enc[cam]) FVV_TRY(fvv::dev_alloc(c, reinterpret_cast<void**>(&K->enc[cam]), 65536 * sizeof(uint16_t)));
    std::vector<uint16_t> dec(4096), enc(65536);
    for (int y = 0; y < 4096; ++y) dec[y] = fvv::decode_code(y, *p, c->depth_unit_m);
    for (int d = 0; d < 65536; ++d) enc[d] = fvv::encode_code(d, *p, c->depth_unit_m);
    // the tables may be read by work in flight on the context's stream
    FVV_CUDA(cudaStreamSynchronize(c->own));
    FVV_CUDA(cudaMemcpy(K->dec[cam], dec.data(), dec.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
    FVV_CUDA(cudaMemcpy(K->enc[cam], enc.data(), enc.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
    K->prm[cam] = *p;
    K->set[cam] = 1;
    return FVV_OK;
}

fvv_status fvv_depth_encode_yuv(fvv_ctx* c, int32_t cam, const uint16_t* depth, size_t depth_pitch, uint8_t* y,
                                size_t y_pitch, uint8_t* u, uint8_t* v, size_t uv_pitch, void* stream)
{
    FVV_TRY(fvv::check_cam(c, cam));
    fvv::DeviceScope dev_scope(c->device);
    const int W = c->cams[cam].width, H = c->cams[cam].height;
    if (!fvv::on_dev(depth) || !fvv::on_dev(y) || !fvv::on_dev(u) || !fvv::on_dev(v))
        return fail(FVV_ERR_INVALID_ARG, "depth and the Y, U, V planes must be device memory");
    if (depth_pitch < size_t(W) * 2 || depth_pitch % 4 || y_pitch < size_t(W) || uv_pitch < size_t(W / 2) ||
        reinterpret_cast<uintptr_t>(depth) % 4)
        return fail(FVV_ERR_INVALID_ARG, "pitch too small, or depth not 4-byte aligned");
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : c->own;
    const int bw = W / 2, bh = H / 2;
    const size_t n = size_t(bw) * bh;
    fvv::k_yuv_encode<<<unsigned((n + 255) / 256), 256, 0, s>>>(depth, depth_pitch, bw, bh, c->codec->enc[cam], y,
                                                               y_pitch, u, v, uv_pitch);
    FVV_CUDA(cudaGetLastError());
    return FVV_OK;
}

fvv_status fvv_depth_decode_yuv(fvv_ctx* c, int32_t cam, const uint8_t* y, size_t y_pitch, const uint8_t* u,
                                const uint8_t* v, size_t uv_pitch, uint16_t* depth, size_t depth_pitch, void* stream)
{
    FVV_TRY(fvv::check_cam(c, cam));
    fvv::DeviceScope dev_scope(c->device);
    const int W = c->cams[cam].width, H = c->cams[cam].height;
    if (!fvv::on_dev(depth) || !fvv::on_dev(y) || !fvv::on_dev(u) || !fvv::on_dev(v))
        return fail(FVV_ERR_INVALID_ARG, "depth and the Y, U, V planes must be device memory");
    if (depth_pitch < size_t(W) * 2 || depth_pitch % 4 || y_pitch < size_t(W) || uv_pitch < size_t(W / 2) ||
        reinterpret_cast<uintptr_t>(depth) % 4)
        return fail(FVV_ERR_INVALID_ARG, "pitch too small, or depth not 4-byte aligned");
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : c->own;
    const fvv::YuvDepth f{y, u, v, y_pitch, uv_pitch, c->codec->dec[cam]};
    std::lock_guard<std::recursive_mutex> g(c->mu);
    return fvv::run_kernel(c, fvv::kDecode, s, [&] { return fvv::launch_yuv_decode(f, W, H, depth, depth_pitch, s); });
}

fvv_status fvv_depth_decode_yuv_frames(fvv_ctx* c, int32_t n_cams, const uint8_t* yuv, size_t yuv_cam_stride,
                                       uint16_t* depth, size_t depth_cam_stride, size_t depth_pitch, void* stream)
{
    if (!c) return fail(FVV_ERR_INVALID_ARG, "ctx is NULL");
    if (n_cams < 1 || n_cams > c->n_cams) return fail(FVV_ERR_INVALID_ARG, "n_cams out of range");
    fvv::DeviceScope dev_scope(c->device);
    for (int k = 0; k < n_cams; ++k) {
        FVV_TRY(fvv::check_cam(c, k));
        if (c->cams[k].width != c->cams[0].width || c->cams[k].height != c->cams[0].height)
            return fail(FVV_ERR_INVALID_ARG, "cameras of one size only");
    }
    const int W = c->cams[0].width, H = c->cams[0].height;
    const size_t frame = size_t(W) * H + 2 * size_t(W / 2) * (H / 2);
    if (!fvv::on_dev(yuv) || !fvv::on_dev(depth))
        return fail(FVV_ERR_INVALID_ARG, "yuv and depth must be device memory");
    if (yuv_cam_stride < frame || depth_pitch < size_t(W) * 2 || depth_cam_stride < depth_pitch * size_t(H) ||
        depth_pitch % 4 || depth_cam_stride % 4 || reinterpret_cast<uintptr_t>(depth) % 4)
        return fail(FVV_ERR_INVALID_ARG, "stride or pitch too small, or depth not 4-byte aligned");
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : c->own;
    fvv::YuvFrames f{};
    f.y = yuv;
    f.u = yuv + size_t(W) * H;
    f.v = f.u + size_t(W / 2) * (H / 2);
    f.y_pitch = size_t(W);
    f.uv_pitch = size_t(W / 2);
    f.cam_stride = yuv_cam_stride;
    f.out = depth;
    f.out_pitch = depth_pitch;
    f.out_cam_stride = depth_cam_stride;
    f.groups = W / 16;
    f.block_rows = H / 2;
    f.n = n_cams;
    for (int k = 0; k < n_cams; ++k) f.lut[k] = c->codec->dec[k];
    std::lock_guard<std::recursive_mutex> g(c->mu);
    if (fvv::vec16_ok(f, W))
        return fvv::run_kernel(c, fvv::kDecode, s, [&] { return fvv::launch_decode16(f, s); });
    // unaligned or ragged: the per-frame form, camera after camera
    return fvv::run_kernel(c, fvv::kDecode, s, [&] {
        for (int k = 0; k < n_cams; ++k) {
            const uint8_t* y = yuv + size_t(k) * yuv_cam_stride;
            const fvv::YuvDepth d{y, y + size_t(W) * H, y + size_t(W) * H + size_t(W / 2) * (H / 2), size_t(W),
                                  size_t(W / 2), c->codec->dec[k]};
            uint16_t* o = reinterpret_cast<uint16_t*>(reinterpret_cast<uint8_t*>(depth) + size_t(k) * depth_cam_stride);
            const cudaError_t e = fvv::launch_yuv_decode(d, W, H, o, depth_pitch, s);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    });
}

fvv_status fvv_upload_frame_yuv(fvv_ctx* c, int32_t cam, const uint8_t* rgb, size_t rgb_pitch, const uint8_t* y,
                                size_t y_pitch, const uint8_t* u, const uint8_t* v, size_t uv_pitch, uint64_t tick,
                                void* stream)
{
    FVV_TRY(fvv::check_cam(c, cam));
    fvv::DeviceScope dev_scope(c->device);
    if (!y || !u || !v) return fail(FVV_ERR_INVALID_ARG, "Y, U and V must be non-NULL");
    const int W = c->cams[cam].width, H = c->cams[cam].height;
    if (y_pitch < size_t(W) || uv_pitch < size_t(W / 2)) return fail(FVV_ERR_INVALID_ARG, "pitch too small");
    if (fvv::foreign(rgb) || fvv::foreign(y) || fvv::foreign(u) || fvv::foreign(v))
        return fail(FVV_ERR_INVALID_ARG, "frame buffers must be host memory or the context's device memory");
    const bool dy = fvv::on_dev(y), du = fvv::on_dev(u), dv = fvv::on_dev(v);
    if (dy != du || dy != dv) return fail(FVV_ERR_INVALID_ARG, "Y, U, V must all be host or all device memory");
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : c->own;
    std::lock_guard<std::recursive_mutex> g(c->mu);
    fvv::CodecState* K = c->codec;
    fvv::YuvDepth f{y, u, v, y_pitch, uv_pitch, K->dec[cam]};
    if (!dy) {
        // host planes: one copy per plane into dense staging
        const size_t yb = size_t(W) * H, cb = size_t(W / 2) * (H / 2);
        if (K->stage_bytes[cam] < yb + 2 * cb) {
            FVV_CUDA(cudaStreamSynchronize(s));
            fvv::dev_free(c, K->stage[cam], K->stage_bytes[cam]);
            K->stage[cam] = nullptr;
            K->stage_bytes[cam] = 0;
            FVV_TRY(fvv::dev_alloc(c, reinterpret_cast<void**>(&K->stage[cam]), yb + 2 * cb));
            K->stage_bytes[cam] = yb + 2 * cb;
        }
        uint8_t* sy = K->stage[cam];
        if (y_pitch == size_t(W) && uv_pitch == size_t(W / 2) && u == y + yb && v == u + cb) {
            // one planar I420 buffer: a single copy
            FVV_CUDA(cudaMemcpyAsync(sy, y, yb + 2 * cb, cudaMemcpyHostToDevice, s));
        } else {
            FVV_CUDA(cudaMemcpy2DAsync(sy, W, y, y_pitch, W, H, cudaMemcpyHostToDevice, s));
            FVV_CUDA(cudaMemcpy2DAsync(sy + yb, W / 2, u, uv_pitch, W / 2, H / 2, cudaMemcpyHostToDevice, s));
            FVV_CUDA(cudaMemcpy2DAsync(sy + yb + cb, W / 2, v, uv_pitch, W / 2, H / 2, cudaMemcpyHostToDevice, s));
        }
        f = fvv::YuvDepth{sy, sy + yb, sy + yb + cb, size_t(W), size_t(W / 2), K->dec[cam]};
    }
    return fvv::upload_frame(c, cam, rgb, rgb_pitch, nullptr, 0, &f, tick, s);
}

}  // extern "C"
