// fvv_upload.cu -- batched frame upload: one tick of every camera of equal
// size lands in a frame-ring slot in one launch (RGB8 -> RGBA8 packing and
// the depth rows), after at most two bulk host-to-device copies.
#include "fvv_runtime.h"

namespace fvv {

namespace {

// every camera of one tick: RGB8 -> RGBA8 and depth rows into the slot; one
// thread per texel of row blockIdx.y of camera blockIdx.z
__global__ void __launch_bounds__(256) k_upload_all(const UploadAll u)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, k = blockIdx.z;
    if (x >= u.W)
        return;
    const uint8_t* p = u.rgb + k * u.rgb_cam_stride + size_t(y) * u.rgb_pitch + 3 * size_t(x);
    uint32_t* rgba = reinterpret_cast<uint32_t*>(u.slot + u.off_rgba[k]);
    rgba[size_t(y) * u.rpitch + x] = uint32_t(p[0]) | (uint32_t(p[1]) << 8) | (uint32_t(p[2]) << 16);
    uint16_t* dd = u.ddst[k] ? u.ddst[k] : reinterpret_cast<uint16_t*>(u.slot + u.off_depth[k]);
    uint32_t code;
    if (u.yuv) {
        // Eq. (3) inverted for one pixel: its Y byte, the 4 MSBs from the U
        // (top row of the 2x2 block) or V (bottom row) byte, bit i of the
        // left pixel at bit 2i and of the right one at bit 2i + 1
        const uint8_t* blk = u.depth + k * u.depth_cam_stride;
        const size_t yb = size_t(u.W) * u.H, cb = size_t(u.W / 2) * (u.H / 2);
        const uint32_t ybyte = blk[size_t(y) * u.W + x];
        const uint32_t uv = blk[yb + ((y & 1) ? cb : 0) + size_t(y >> 1) * (u.W / 2) + (x >> 1)];
        uint32_t msb = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) msb |= ((uv >> (2 * i + (x & 1))) & 1u) << i;
        const uint32_t y12 = (msb << 8) | ((msb & 1u) ? 255u - ybyte : ybyte);
        code = __ldg(u.lut[k] + y12);
    } else {
        code = reinterpret_cast<const uint16_t*>(u.depth + k * u.depth_cam_stride + size_t(y) * u.depth_pitch)[x];
    }
    dd[size_t(y) * u.dpitch + x] = uint16_t(code);
}

}  // namespace

cudaError_t launch_upload_all(const UploadAll& u, cudaStream_t stream)
{
    if (u.W <= 0 || u.H <= 0 || u.n_cams <= 0) return cudaSuccess;
    dim3 grid(static_cast<unsigned>((u.W + 255) / 256), static_cast<unsigned>(u.H), static_cast<unsigned>(u.n_cams));
    k_upload_all<<<grid, 256, 0, stream>>>(u);
    return cudaGetLastError();
}

}  // namespace fvv
