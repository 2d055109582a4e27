// fvv_noalloc.cu -- view synthesis for callers that cannot allocate device
// memory.
//
// Some callers must never call cudaMalloc: a process whose device memory is
// owned by another allocator (a framework's caching allocator that has
// reserved the GPU), or a latency-critical render thread on which cudaMalloc /
// cudaFree would synchronise the device and stall other streams.  For them,
// fvv_synthesize_noalloc runs the same three kernels as fvv_synthesize_batch
// (clear, splat, resolve) on one view, with its scratch -- the z-buffer keys
// and the launch parameters -- in file-scope device arrays of fixed size.
// The caller passes the camera frames (already on the device, in the
// library's RGBA8 + uint16 layout) and the output buffer.
//
// The arrays are module globals: every GPU that loads the library holds them
// (about 16 MiB + 16 KiB) until the process exits, and every call shares
// them.  Calls whose GPU work overlaps (e.g. on two streams without ordering)
// race on that scratch.  The clear kernel resets the keys at the start of
// every call; the parameters are rewritten by every call.
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "fvv.h"
#include "fvv_internal.h"

namespace {

constexpr size_t kMaxPixels = FVV_NOALLOC_MAX_PIXELS;   // keys: 16 MiB
constexpr int kMaxDevices = 64;

struct NoAllocParams {
    fvv::ViewDesc view;
    fvv::CamGeom geom[fvv::kMaxCams];
    fvv::FrameRef frames[fvv::kMaxCams];
};

static __device__ __align__(256) unsigned long long g_keys[kMaxPixels];
static __device__ __align__(256) NoAllocParams g_params;

// Device addresses of the two arrays, looked up once per device.  In host
// code g_keys / g_params name host-side stand-ins, never device memory.
struct DeviceScratch {
    bool ready = false;
    unsigned long long* keys = nullptr;
    NoAllocParams* params = nullptr;
};
DeviceScratch g_scratch[kMaxDevices];
std::mutex g_scratch_mu;

fvv_status fail(fvv_status code, const char* msg)
{
    fvv::set_last_error(msg);               // failure path only
    return code;
}

// The launch parameters travel by value as a kernel argument (no host
// staging buffer, no host synchronisation) and are stored into g_params.
__global__ void k_store_params(const NoAllocParams p, NoAllocParams* dst)
{
    const unsigned* src = reinterpret_cast<const unsigned*>(&p);
    unsigned* d = reinterpret_cast<unsigned*>(dst);
    for (unsigned i = threadIdx.x; i < sizeof(NoAllocParams) / 4; i += blockDim.x)
        d[i] = src[i];
}

// Device (or managed) memory of device `dev`: the kernels run on the current
// device and would otherwise dereference another GPU's memory.
bool device_memory(const void* p, int dev)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

// The resolve kernel indexes a frame in 32 bits: (H - 1) * pitch + W must
// stay below 2^32 elements.
bool pitch_fits(size_t pitch_elems, int W, int H)
{
    return pitch_elems <= size_t(INT32_MAX) &&
           uint64_t(H - 1) * uint64_t(pitch_elems) + uint64_t(W) < (uint64_t(1) << 32);
}

bool camera_sane(const fvv_camera& c)
{
    if (c.width < 1 || c.height < 1 || c.width > 65535 || c.height > 65535) return false;
    if (uint64_t(c.width) * uint64_t(c.height) > FVV_MAX_SRC_PIXELS) return false;
    const double v[4] = {c.fx, c.fy, c.cx, c.cy};
    for (double x : v)
        if (!std::isfinite(x)) return false;
    if (c.fx == 0.0 || c.fy == 0.0) return false;
    for (double x : c.R)
        if (!std::isfinite(x)) return false;
    for (double x : c.t)
        if (!std::isfinite(x)) return false;
    return true;
}

}  // namespace

extern "C" fvv_status fvv_synthesize_noalloc(const fvv_rig* rig, const fvv_options* opt,
                                             const uint16_t* const* depth, const size_t* depth_pitch,
                                             const uint32_t* const* rgba, const size_t* rgba_pitch,
                                             const fvv_view* view, uint8_t* out_rgb, size_t out_pitch,
                                             void* stream)
{
    if (!rig || !view || !depth || !depth_pitch || !rgba || !rgba_pitch || !out_rgb)
        return fail(FVV_ERR_INVALID_ARG, "fvv_synthesize_noalloc: NULL argument");
    if (rig->n_cams < 1 || rig->n_cams > FVV_MAX_CAMS || !rig->cams)
        return fail(FVV_ERR_INVALID_ARG, "fvv_synthesize_noalloc: n_cams must be in [1, 64]");
    if (!(rig->depth_unit_m > 0.0) || !std::isfinite(rig->depth_unit_m))
        return fail(FVV_ERR_INVALID_ARG, "fvv_synthesize_noalloc: depth_unit_m must be > 0");
    fvv_options o;
    if (opt) o = *opt; else fvv_default_options(&o);
    if (o.layered)
        return fail(FVV_ERR_INVALID_ARG,
                    "fvv_synthesize_noalloc: layered synthesis needs a context (fvv_set_bg_depth)");
    if (o.n_ref < 0 || o.n_ref > rig->n_cams || o.d_lo < 1 || o.d_hi > 65534 || o.d_lo > o.d_hi ||
        !(o.tau_crack >= 0.0f) || !(o.tau_vis >= 0.0f) || !(o.z_min >= 0.0f) || !std::isfinite(o.z_min))
        return fail(FVV_ERR_INVALID_ARG, "fvv_synthesize_noalloc: invalid options");
    if (!camera_sane(*view))
        return fail(FVV_ERR_INVALID_ARG, "fvv_synthesize_noalloc: invalid view camera");
    const size_t np = size_t(view->width) * size_t(view->height);
    if (np > kMaxPixels) {
        char msg[256];
        std::snprintf(msg, sizeof msg,
                      "fvv_synthesize_noalloc: the view has %zu pixels; this allocation-free entry "
                      "point holds scratch for at most %zu (use fvv_synthesize for larger views)",
                      np, kMaxPixels);
        return fail(FVV_ERR_INVALID_ARG, msg);
    }
    if (out_pitch < size_t(view->width) * 3)
        return fail(FVV_ERR_INVALID_ARG, "fvv_synthesize_noalloc: out_pitch < 3 * width");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return fail(FVV_ERR_CUDA, "fvv_synthesize_noalloc: no usable current device");
    }
    if (!device_memory(out_rgb, dev))
        return fail(FVV_ERR_INVALID_ARG, "fvv_synthesize_noalloc: out_rgb must be memory of the current device");
    for (int k = 0; k < rig->n_cams; ++k) {
        if (!camera_sane(rig->cams[k]))
            return fail(FVV_ERR_INVALID_ARG, "fvv_synthesize_noalloc: invalid rig camera");
        if (!depth[k] || !rgba[k] || !device_memory(depth[k], dev) || !device_memory(rgba[k], dev))
            return fail(FVV_ERR_INVALID_ARG, "fvv_synthesize_noalloc: frames must be memory of the current device");
        const int W = rig->cams[k].width, H = rig->cams[k].height;
        if (depth_pitch[k] % 2 || depth_pitch[k] < size_t(W) * 2 ||
            rgba_pitch[k] % 4 || rgba_pitch[k] < size_t(W) * 4 ||
            (reinterpret_cast<uintptr_t>(depth[k]) & 1) || (reinterpret_cast<uintptr_t>(rgba[k]) & 3))
            return fail(FVV_ERR_INVALID_ARG, "fvv_synthesize_noalloc: bad frame pitch or alignment");
        if (!pitch_fits(depth_pitch[k] / 2, W, H) || !pitch_fits(rgba_pitch[k] / 4, W, H))
            return fail(FVV_ERR_INVALID_ARG,
                        "fvv_synthesize_noalloc: frame pitch too large ((H - 1) * pitch + W must be below 2^32 elements)");
    }
    if (fvv::resolve_smem_bytes(view->width, rig->n_cams) > size_t(227) * 1024)
        return fail(FVV_ERR_INVALID_ARG, "fvv_synthesize_noalloc: view too wide");

    // once per device, with that device current: device addresses of the
    // scratch arrays (a device reset after this point is not supported: the
    // module may come back at other addresses)
    DeviceScratch S;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        DeviceScratch& D = g_scratch[dev];
        if (!D.ready) {
            void* k = nullptr;
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&k, g_keys);
            if (e == cudaSuccess) e = cudaGetSymbolAddress(&p, g_params);
            if (e != cudaSuccess) {
                cudaGetLastError();
                char msg[256];
                std::snprintf(msg, sizeof msg, "fvv_synthesize_noalloc: cudaGetSymbolAddress: %s",
                              cudaGetErrorString(e));
                return fail(FVV_ERR_CUDA, msg);
            }
            D.keys = static_cast<unsigned long long*>(k);
            D.params = static_cast<NoAllocParams*>(p);
            D.ready = true;
        }
        S = D;
    }

    NoAllocParams P;
    std::memset(&P, 0, sizeof P);
    const int nc = rig->n_cams;
    fvv::compose_view_into(nc, rig->cams, rig->look_at, rig->depth_unit_m, o.n_ref, *view, P.geom);
    fvv::ViewDesc& D = P.view;
    D.Wv = view->width;
    D.Hv = view->height;
    D.n_cams = nc;
    D.slot = 0;
    D.flags = (o.crack_filter ? fvv::kFlagCrack : 0) | (o.hole_fill ? fvv::kFlagFill : 0) |
              (o.pixel_weights ? fvv::kFlagPixelWeights : 0);
    D.tau_crack = o.tau_crack;
    D.tau_vis = o.tau_vis;
    D.z_min = o.z_min;
    D.d_lo = o.d_lo;
    D.d_hi = o.d_hi;
    D.vk[0] = float(view->cx);
    D.vk[1] = float(view->cy);
    D.vk[2] = float(1.0 / view->fx);
    D.vk[3] = float(1.0 / view->fy);
    D.keys = S.keys;
    D.out_rgb = out_rgb;
    D.out_pitch = int64_t(out_pitch);
    D.geom = S.params->geom;                 // device addresses inside g_params
    int na = 0, segs = 0;
    D.chunk_begin[0] = 0;
    for (int k = 0; k < nc; ++k) {
        fvv::FrameRef& F = P.frames[k];
        F.depth = depth[k];
        F.rgba = rgba[k];
        F.W = rig->cams[k].width;
        F.H = rig->cams[k].height;
        F.dpitch = int32_t(depth_pitch[k] / 2);
        F.rpitch = int32_t(rgba_pitch[k] / 4);
        if (P.geom[k].w > 0.0f) {
            D.active[na] = k;
            segs += F.H * ((F.W + fvv::kSplatSeg - 1) / fvv::kSplatSeg);
            D.chunk_begin[++na] = segs;
        }
    }
    D.n_active = na;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const fvv::ViewDesc* vdev = &S.params->view;
    const fvv::FrameRef* fdev = S.params->frames;
    k_store_params<<<1, 256, 0, s>>>(P, S.params);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = fvv::launch_clear_keys(S.keys, (np + 15) & ~size_t(15), s);
    if (e == cudaSuccess) e = fvv::launch_warp_splat(vdev, 1, segs, fdev, s);
    if (e == cudaSuccess)
        e = fvv::launch_resolve(vdev, 1, view->height, view->width, nc, false, fdev, s, false, o.pixel_weights != 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        char msg[256];
        std::snprintf(msg, sizeof msg, "fvv_synthesize_noalloc: launch failed: %s", cudaGetErrorString(e));
        return fail(FVV_ERR_CUDA, msg);
    }
    return FVV_OK;
}
