// fvv_internal.h -- device-side descriptors shared by the kernels and the
// host runtime of libfvv.  Not part of the public ABI (see include/fvv.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace fvv {

constexpr int kMaxCams = 64;
constexpr int kSrcBits = 26;
constexpr unsigned long long kKeyEmpty = ~0ull;
constexpr uint16_t kDepthBg = 65535;   // depth code of a background pixel
constexpr int kSplatSeg = 256;       // source pixels per splat warp (8 per lane, stride 32)
constexpr int kSplatThreads = 256;
constexpr int kResolveThreads = 256;
constexpr int kResolveBand = 2;      // output rows per resolve CTA

constexpr int kFlagCrack = 1;
constexpr int kFlagFill = 2;
constexpr int kFlagLayered = 4;
constexpr int kFlagPixelWeights = 8;

// Per (view, camera) quantities, composed on the host in FP64 and rounded
// to FP32 once (Sec. VI geometry).  M maps (u z, v z, z, 1) of the camera to
// (X, Y, Z) of the view; N maps (x Z, y Z, Z, 1) of the view to the camera.
struct alignas(16) CamGeom {
    float M[12];
    float N[12];
    float w;          // blend weight, 0 = inactive
    float pad[3];     // the camera's centre in the view's frame, depth units (per-pixel weights)
};

// One camera's frame in one slot of the device-resident frame ring.
struct alignas(16) FrameRef {
    const uint16_t* depth;   // [H][dpitch] depth codes, 0 = none, kDepthBg = background
    const uint32_t* rgba;    // [H][rpitch] R | G << 8 | B << 16
    const uint16_t* bg;      // [H][dpitch] static background depth model, or NULL
    int32_t W, H;
    int32_t dpitch;          // elements; rows 128-B aligned
    int32_t rpitch;          // elements
};

// One view of a batched launch.
struct alignas(16) ViewDesc {
    int32_t Wv, Hv;
    int32_t n_cams;
    int32_t n_active;
    int32_t slot;
    int32_t flags;
    float tau_crack, tau_vis, z_min;
    uint32_t d_lo, d_hi;
    int32_t pad0;
    float vk[4];                     // the view's cx, cy, 1/fx, 1/fy (per-pixel weights)
    unsigned long long* keys;        // scratch z-buffer [Hv * Wv] (the FG layer when layered)
    unsigned long long* keys_bg;     // layered: the BG layer's z-buffer [Hv * Wv], else NULL
    unsigned long long* keys_bgf;    // layered: the BG layer after the crack filter (keys_bg without it)
    unsigned long long* keys_next;   // nullable [Hv * Wv]: set to the empty key by the resolve (the
                                     // next batch's z-buffer, so that it needs no clear; single layer)
    uint8_t* out_rgb;                // [Hv] rows of 3 * Wv bytes
    int64_t out_pitch;               // bytes
    float* out_depth;                // nullable [Hv * Wv]
    uint8_t* out_hole;               // nullable [Hv * Wv]
    float* out_top3;                 // nullable [Hv * Wv * 3]
    unsigned long long* out_keys;    // nullable [Hv * Wv], after the crack filter
    const CamGeom* geom;             // [n_cams]
    int32_t active[kMaxCams];        // cameras with w > 0, ascending
    int32_t chunk_begin[kMaxCams + 1];  // prefix of splat warp segments over `active`
};

// Persistent serving kernel (fvv_kernels.cu): one cooperative launch that
// takes batches of views from a ring the host writes, and runs steps a-e of
// each (clear, splat, resolve, separated by grid barriers).  The ring lives
// in pinned, mapped host memory; the kernel reads it through its device
// alias.  Every wait of the kernel is bounded by %globaltimer.
struct PersistBatch {
    const ViewDesc* views;             // device: the batch's parameter block
    const FrameRef* frames;            // device: the frame ring's table
    unsigned long long* keys;          // the batch's z-buffers, cleared first
    unsigned long long n_keys;
    int32_t n_views, max_h, band, splat_bx;
    int32_t pixel_weights, pad[3];
};
constexpr int kPersistRing = 16;
struct PersistQueue {
    PersistBatch batch[kPersistRing];   // batch b at b % kPersistRing
    volatile uint32_t posted;           // batches written so far (set after the batch)
    volatile uint32_t stop;             // 1: return at the next wait for work
    volatile uint32_t done;             // batches completed (set after their outputs)
    volatile int32_t err;               // 0, or the code of the wait that ran out
};
// Device memory of the kernel's grid barrier; zeroed before every launch.
struct PersistSync {
    unsigned int count, gen;
    int cmd;                            // 0: run the batch, 1: return
    int err;
};
constexpr int kPersistErrBarrier = 11;  // a grid barrier ran out
// Launch the kernel on `stream` (cooperative, every CTA resident) to take
// batches first, first + 1, ...; it returns after idle_ns without work, on
// q->stop, or when a grid barrier waits longer than wait_ns.  max_w, n_cams
// size its shared memory.  *ctas: the grid size.
cudaError_t launch_serve_persistent(PersistQueue* q_dev, PersistSync* sync, uint32_t first, int max_w, int n_cams,
                                    uint64_t idle_ns, uint64_t wait_ns, cudaStream_t stream, int* ctas);
// The grid of that kernel for views up to max_w wide (0: none fits).
int persist_grid(int max_w, int n_cams);
// The band and the splat's CTAs per view the kernel uses for a batch.
void persist_batch_shape(int n_views, int max_h, int max_chunks, int ctas, int* band, int* splat_bx);

// Launchers (fvv_kernels.cu).  All asynchronous on `stream`.
cudaError_t launch_clear_keys(unsigned long long* keys, size_t n, cudaStream_t stream);
// layered: FG/BG layers (each view's keys_bg set, frames' bg models used).
cudaError_t launch_warp_splat(const ViewDesc* views, int n_views, int max_chunks,
                              const FrameRef* frames, cudaStream_t stream, bool layered = false);
// Layered: the crack filter of the BG layer (keys_bg -> keys_bgf), one pass.
cudaError_t launch_crack_bg(const ViewDesc* views, int n_views, int max_h, int max_w, cudaStream_t stream);
cudaError_t launch_resolve(const ViewDesc* views, int n_views, int max_h, int max_w, int n_cams,
                           bool top3, const FrameRef* frames, cudaStream_t stream, bool layered = false,
                           bool pixel_weights = false);
cudaError_t launch_pack_rgba(const uint8_t* rgb, size_t rgb_pitch, uint32_t* rgba,
                             int rpitch, int W, int H, cudaStream_t stream);
size_t resolve_smem_bytes(int max_w, int n_cams, bool layered = false);
// The current device's streaming-multiprocessor count (1 if it cannot be read).
int device_sms();

}  // namespace fvv

struct fvv_camera;
namespace fvv {
// fvv_api.cu: message returned by fvv_last_error() on this thread.
void set_last_error(const char* msg);
// fvv_api.cu: FP64 composition of one view (maps M, N and weights w per camera).
void compose_view_into(int n_cams, const fvv_camera* cams, const double look_at[3],
                       double depth_unit_m, int n_ref, const fvv_camera& view, CamGeom* g);
}  // namespace fvv
