// fvv_runtime.h -- host runtime internals shared by fvv_api.cu (context,
// uploads, batched synthesis) and fvv_serve.cu (the serving loop).  Not part
// of the public ABI.
#pragma once

#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "fvv.h"
#include "fvv_internal.h"

namespace fvv {

// Records `msg` for fvv_last_error() on this thread and returns `code`.
fvv_status fail(fvv_status code, const std::string& msg);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

#define FVV_CUDA(call)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            cudaGetLastError();                                                          \
            return ::fvv::fail(e_ == cudaErrorMemoryAllocation ? FVV_ERR_OUT_OF_MEMORY    \
                                                               : FVV_ERR_CUDA,            \
                               std::string(#call) + ": " + cudaGetErrorString(e_));      \
        }                                                                                \
    } while (0)

#define FVV_TRY(expr)                      \
    do {                                   \
        fvv_status s_ = (expr);            \
        if (s_ != FVV_OK) return s_;       \
    } while (0)

// Where a caller's buffer lives: device memory that the current device's
// kernels may use (its own, or managed), host memory (pageable or pinned),
// or device memory of another GPU.  Entry points refuse the last kind for
// buffers their kernels read or write: the kernels would dereference the
// pointer on the wrong device.
enum class MemKind { Device, Host, Foreign };
MemKind mem_kind(const void* p);
inline bool foreign(const void* p) { return p && mem_kind(p) == MemKind::Foreign; }

// Makes a context's device current for the rest of an entry point (its
// launches, allocations and pointer checks) and gives the caller's current
// device back on return.
class DeviceScope {
public:
    explicit DeviceScope(int dev)
    {
        if (cudaGetDevice(&prev_) != cudaSuccess) {
            cudaGetLastError();
            prev_ = -1;
        }
        if (prev_ != dev) cudaSetDevice(dev);
    }
    ~DeviceScope()
    {
        int cur = -1;
        if (prev_ >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev_) cudaSetDevice(prev_);
    }
    DeviceScope(const DeviceScope&) = delete;
    DeviceScope& operator=(const DeviceScope&) = delete;

private:
    int prev_ = -1;
};

// Valid pinhole camera (also used for views); `why` gets the reason.
bool camera_ok(const fvv_camera& c, std::string* why);

struct ParamBlock {
    uint8_t* host = nullptr;    // pinned
    uint8_t* dev = nullptr;
    size_t cap = 0;
    cudaEvent_t done = nullptr;
    bool pending = false;
};

enum Kid { kClear = 0, kSplat, kResolve, kPack, kDecode, kJbf, kCrackBg, kNumKernels };
extern const char* const kKernelName[kNumKernels];

struct KernelStat {
    uint64_t launches = 0;
    uint64_t timed = 0;
    double ms = 0.0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
};

// Readers of the frame ring: the context's own scratch (0) and up to 16
// serving lanes; each records its own "last read" event per slot.
constexpr int kMaxReaders = 17;

struct SlotState {
    uint64_t tick = 0;
    uint64_t mask = 0;
    bool any = false;
    cudaEvent_t uploaded = nullptr;            // after the last upload into this slot
    cudaEvent_t read[kMaxReaders] = {};        // after each reader's last synthesis of it
    bool read_pending[kMaxReaders] = {};
    uint32_t persist_reads = 0;                // persistent serving: batch index + 1 of its last reader
};

// Device scratch of batched launches: the z-buffer keys, the staging area
// for host outputs and a ring of parameter blocks.  The context's own
// scratch grows on demand; a serving lane's is sized once from its budget.
struct BatchScratch {
    unsigned long long* keys = nullptr;
    size_t keys_cap = 0;                  // elements
    // A growable scratch holds two z-buffers: a single-layer batch splats
    // into keys_buf(cur) while its resolve empties the same view regions of
    // the other one, so a next batch of the same layout starts without a
    // clear.  clean[b]: the per-view key counts whose regions buffer b is
    // known to hold empty (none: clear before use).
    unsigned long long* keys2 = nullptr;
    int cur = 0;
    std::vector<size_t> clean[2];
    uint8_t* out_stage = nullptr;
    size_t out_stage_cap = 0;             // bytes
    std::vector<ParamBlock> pring;
    int pnext = 0;
    cudaEvent_t done = nullptr;           // after the last batch using this scratch
    bool pending = false;
    bool growable = true;
    int reader = 0;                       // index into SlotState::read
    int max_batch = 0;                    // views per launch the parameter blocks hold
};

struct ServeState;                        // fvv_serve.cu
struct RefineNet;                         // fvv_refine.cu

}  // namespace fvv

namespace fvv {
struct CodecState;

// One tick of every camera (all W x H) into a frame-ring slot: camera k's RGB8
// rows at rgb + k * rgb_cam_stride (pitch rgb_pitch) become RGBA8 rows at
// slot + off_rgba[k] (pitch rpitch texels), its uint16 depth rows at
// depth + k * depth_cam_stride (pitch depth_pitch bytes) are copied to
// slot + off_depth[k] (pitch dpitch elements).
// With yuv set, camera i's depth is a dense planar YUV420 depth frame (Eq.
// (3)) at depth + i * depth_cam_stride (Y rows of W bytes, then U and V rows
// of W/2), decoded through lut[i]; ddst[i], when set, replaces the slot as
// the destination of camera i's depth rows (pitch dpitch).
struct UploadAll {
    const uint8_t* rgb;
    size_t rgb_cam_stride, rgb_pitch;
    const uint8_t* depth;
    size_t depth_cam_stride, depth_pitch;
    uint8_t* slot;
    int W, H, n_cams, dpitch, rpitch;
    int yuv;
    uint64_t off_depth[kMaxCams], off_rgba[kMaxCams];
    const uint16_t* lut[kMaxCams];
    uint16_t* ddst[kMaxCams];
};
cudaError_t launch_upload_all(const UploadAll& u, cudaStream_t stream);

// A YUV420 depth frame in device memory and the decode table of its camera.
struct YuvDepth {
    const uint8_t *y, *u, *v;
    size_t y_pitch, uv_pitch;
    const uint16_t* lut;
};
}  // namespace fvv

struct fvv_ctx {
    int device = 0;
    int n_cams = 0;
    std::vector<fvv_camera> cams;
    double look_at[3] = {0, 0, 0};
    double depth_unit_m = 0.001;
    fvv_options opt{};
    cudaStream_t own = nullptr;
    size_t smem_optin = 0;

    int slots = 0;
    std::vector<int> dpitch, rpitch;            // elements
    std::vector<size_t> off_depth, off_rgba;    // within a slot
    size_t slot_bytes = 0;
    uint8_t* arena = nullptr;
    size_t arena_bytes = 0;
    fvv::FrameRef* frames_dev = nullptr;
    std::vector<fvv::SlotState> slot;
    uint64_t full_mask = 0;
    uint64_t latest = 0;                        // newest tick holding every camera
    bool have_latest = false;
    bool have_any = false;                      // some camera of some tick uploaded

    std::vector<uint16_t*> bg;                  // per camera: static BG depth model [H][dpitch] or NULL
    std::vector<uint16_t*> jbf_tmp;             // per camera: unfiltered codes [H][dpitch] (depth pre-filter)
    std::vector<uint8_t*> stage_rgb;            // per camera, for host uploads
    // batched host uploads: two staging buffers used in turn, so that a
    // tick's host-to-device copy (on one stream) can run while the previous
    // tick's packing kernel (on another) still reads the other buffer
    uint8_t* stage_all[2] = {};
    size_t stage_all_bytes[2] = {};
    cudaEvent_t stage_all_free[2] = {};         // last reader of each
    int stage_all_next = 0;
    cudaEvent_t stage_free = nullptr;           // last reader of the per-camera staging buffers
    fvv::BatchScratch main;                     // scratch of fvv_synthesize(_batch)

    bool profiling = false;
    fvv::KernelStat kstat[fvv::kNumKernels];
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> event_pool;
    size_t held = 0;                            // device bytes held

    // Guards the frame-ring state, the kernel statistics and the scratch
    // against the serving thread.
    std::recursive_mutex mu;
    fvv::ServeState* serve = nullptr;
    fvv::RefineNet* refine = nullptr;
    fvv::CodecState* codec = nullptr;           // depth codec tables (fvv_codec.cu)
};

namespace fvv {

fvv_status dev_alloc(fvv_ctx* c, void** p, size_t bytes);
// Upload one camera's frame for `tick` into the frame ring: depth from uint16
// rows (yuv NULL) or decoded from a YUV420 depth frame.  Caller holds c->mu.
fvv_status upload_frame(fvv_ctx* c, int cam, const uint8_t* rgb, size_t rgb_pitch, const uint16_t* depth,
                        size_t depth_pitch, const YuvDepth* yuv, uint64_t tick, cudaStream_t s);
cudaError_t launch_yuv_decode(const YuvDepth& f, int width, int height, uint16_t* out, size_t out_pitch,
                              cudaStream_t s);
void codec_destroy(fvv_ctx* c);
// Camera cam's decode table (4096 depth codes) or NULL when it has no codec.
const uint16_t* codec_decode_table(fvv_ctx* c, int cam);
// The refinement network for the serving loop: whether it is initialised, and
// its forward pass on `s` without waiting (device batch; out_rgb is
// [n][h][w][3] uint8).  A bounded-wait timeout leaves the device flag raised
// for the next synchronous refinement call to report.
bool refine_ready(fvv_ctx* c);
fvv_status refine_forward_async(fvv_ctx* c, const fvv_refine_batch& b, uint8_t* out_rgb, cudaStream_t s);
// Grow the network's activations (current precision) to `pixels` per batch.
fvv_status refine_reserve(fvv_ctx* c, size_t pixels);
// The device int the network's kernels raise when a bounded wait runs out.
fvv_status refine_error_flag(int** flag);
// True while a serving loop with refinement runs (the network is in use).
bool serve_refining(fvv_ctx* c);
void dev_free(fvv_ctx* c, void* p, size_t bytes);

// Launch through `fn` (returns cudaError_t), counting it and, when profiling
// is on, bracketing it with events on the launching stream.
template <class Fn>
fvv_status run_kernel(fvv_ctx* c, Kid id, cudaStream_t s, Fn fn)
{
    KernelStat& K = c->kstat[id];
    std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
    if (c->profiling) {
        if (c->event_pool.empty()) {
            FVV_CUDA(cudaEventCreate(&ev.first));
            FVV_CUDA(cudaEventCreate(&ev.second));
        } else {
            ev = c->event_pool.back();
            c->event_pool.pop_back();
        }
        FVV_CUDA(cudaEventRecord(ev.first, s));
    }
    cudaError_t e = fn();
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (ev.first) c->event_pool.push_back(ev);
        return fail(FVV_ERR_CUDA, std::string("launch of ") + kKernelName[id] + ": " + cudaGetErrorString(e));
    }
    ++K.launches;
    if (ev.first) {
        FVV_CUDA(cudaEventRecord(ev.second, s));
        K.pending.push_back(ev);
    }
    return FVV_OK;
}

// Allocate `S` with room for `keys` z-buffer entries, `stage` staging bytes
// and `n_blocks` parameter blocks of `max_batch` views; growable = false.
fvv_status scratch_alloc(fvv_ctx* c, BatchScratch& S, size_t keys, size_t stage, int max_batch,
                         int n_blocks);
void scratch_free(fvv_ctx* c, BatchScratch& S);

// Keys (elements) and host-output staging bytes one view needs (layered:
// two z-buffers).
size_t view_keys(const fvv_view& v, bool layered = false);
size_t view_stage_bytes(const fvv_view& v, uint8_t* out_rgb, const fvv_aux* aux);

// A batch for the persistent serving kernel: what run_batch fills instead
// of launching (ctas: the kernel's grid, set by the caller).
struct PersistPost {
    int ctas = 0;
    PersistBatch batch{};
    std::vector<int> slots;                    // frame-ring slots the batch reads
};

// One batched launch of steps a-e for n views on stream s, with scratch S.
// ticks[i] selects view i's tick (NULL = newest complete).  With sync_host
// the call waits for host outputs; without, the caller orders on the stream.
// With post (device outputs, no aux, single-layer context) nothing is
// launched: the parameter copy and the waits for the frames' uploads are
// queued on s and *post describes the batch for the persistent kernel.
// The caller holds c->mu.
fvv_status run_batch(fvv_ctx* c, BatchScratch& S, int n, const fvv_view* views,
                     const uint64_t* ticks, uint8_t* const* out_rgb, const size_t* out_pitch,
                     const fvv_aux* aux, cudaStream_t s, bool sync_host, PersistPost* post = nullptr);

// Persistent serving: before an upload overwrites `slot`, wait (up to 2 s,
// relaunching the kernel if it returned with the batch pending) until the
// batches that read it are done.  The caller holds c->mu.
fvv_status serve_wait_slot(fvv_ctx* c, const SlotState& slot);

// fvv_serve.cu: stop a running serving loop (fvv_destroy calls it).
void serve_shutdown(fvv_ctx* c);
// fvv_refine.cu: free the refinement network (fvv_destroy calls it).
void refine_destroy(fvv_ctx* c);

}  // namespace fvv
