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
    const uint16_t* d =
        reinterpret_cast<const uint16_t*>(u.depth + k * u.depth_cam_stride + size_t(y) * u.depth_pitch);
    uint16_t* dd = reinterpret_cast<uint16_t*>(u.slot + u.off_depth[k]);
    dd[size_t(y) * u.dpitch + x] = d[x];
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
