// fvv_api.cu -- host runtime behind the C ABI of include/fvv.h.
//
// Owns the device-resident frame ring (every camera's RGBA8 + depth for
// `frame_slots` capture ticks), the per-view z-buffer scratch, a ring of
// pinned/device parameter blocks for batched launches, and the FP64 pose
// composition (Sec. VI geometry) whose FP32-rounded results the kernels use.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "fvv.h"
#include "fvv_internal.h"
#include "fvv_jbf.h"
#include "fvv_runtime.h"

using fvv::BatchScratch;
using fvv::CamGeom;
using fvv::FrameRef;
using fvv::MemKind;
using fvv::ParamBlock;
using fvv::SlotState;
using fvv::ViewDesc;
using fvv::align_up;
using fvv::camera_ok;
using fvv::dev_alloc;
using fvv::dev_free;
using fvv::fail;
using fvv::mem_kind;
using fvv::run_kernel;
using fvv::kClear;
using fvv::kPack;
using fvv::kResolve;
using fvv::kSplat;
using fvv::kNumKernels;
using fvv::kKernelName;

namespace {
thread_local std::string g_err;
}  // namespace

fvv_status fvv::fail(fvv_status code, const std::string& msg)
{
    g_err = msg;
    return code;
}

const char* const fvv::kKernelName[fvv::kNumKernels] = {"clear_keys", "warp_splat", "resolve",
                                                        "pack_rgba", "yuv_decode", "jbf", "crack_bg"};

fvv::MemKind fvv::mem_kind(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return MemKind::Host;
    }
    if (a.type == cudaMemoryTypeManaged) return MemKind::Device;
    if (a.type != cudaMemoryTypeDevice) return MemKind::Host;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) {
        cudaGetLastError();
        return MemKind::Foreign;
    }
    return a.device == cur ? MemKind::Device : MemKind::Foreign;
}

namespace {

bool finite_all(const double* v, int n)
{
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

}  // namespace

bool fvv::camera_ok(const fvv_camera& c, std::string* why)
{
    if (c.width < 1 || c.height < 1 || c.width > 65535 || c.height > 65535) {
        *why = "width/height must be in [1, 65535]";
        return false;
    }
    if (uint64_t(c.width) * uint64_t(c.height) > FVV_MAX_SRC_PIXELS) {
        *why = "width*height exceeds the 26-bit source-pixel field of a key";
        return false;
    }
    const double k[4] = {c.fx, c.fy, c.cx, c.cy};
    if (!finite_all(k, 4) || c.fx == 0.0 || c.fy == 0.0) {
        *why = "intrinsics must be finite with fx, fy != 0";
        return false;
    }
    if (!finite_all(c.R, 9) || !finite_all(c.t, 3)) {
        *why = "R and t must be finite";
        return false;
    }
    return true;
}

namespace {

bool options_ok(const fvv_options& o, int n_cams, std::string* why)
{
    if (o.n_ref < 0 || o.n_ref > n_cams) { *why = "n_ref must be in [0, n_cams]"; return false; }
    if (!(o.tau_crack >= 0.0f) || !std::isfinite(o.tau_crack)) { *why = "tau_crack must be >= 0"; return false; }
    if (!(o.tau_vis >= 0.0f) || !std::isfinite(o.tau_vis)) { *why = "tau_vis must be >= 0"; return false; }
    // Z > z_min >= 0 keeps every projected depth positive, so X / Z is never NaN
    if (!(o.z_min >= 0.0f) || !std::isfinite(o.z_min)) { *why = "z_min must be finite and >= 0"; return false; }
    if (o.d_lo < 1 || o.d_hi > 65534 || o.d_lo > o.d_hi) {
        *why = "need 1 <= d_lo <= d_hi <= 65534 (65535 is the background signal)";
        return false;
    }
    if (o.layered != 0 && o.layered != 1) { *why = "layered must be 0 or 1"; return false; }
    if (o.pixel_weights != 0 && o.pixel_weights != 1) { *why = "pixel_weights must be 0 or 1"; return false; }
    if (!fvv::jbf_options_ok(o, why)) return false;
    if (o.frame_slots < 1 || o.frame_slots > 1024) { *why = "frame_slots must be in [1, 1024]"; return false; }
    if (o.max_batch < 1 || o.max_batch > 4096) { *why = "max_batch must be in [1, 4096]"; return false; }
    return true;
}

// ---------------------------------------------------------------------------
// Sec. VI geometry, FP64.  Maps (u z, v z, z, 1) of camera s to (X, Y, Z) of
// camera d: [A | b] with A = K_d R_rel K_s^-1 and b = K_d t_rel, where
// R_rel = R_d R_s^T and t_rel = (t_d - R_rel t_s) / depth_unit_m.  A's columns
// are KR[:,0] / fx_s, KR[:,1] / fy_s and KR[:,2] - KR[:,0] cx_s / fx_s -
// KR[:,1] cy_s / fy_s (exact when the cameras share intrinsics and
// orientation).  Rounded to FP32 once.
// ---------------------------------------------------------------------------
void compose_map(const fvv_camera& s, const fvv_camera& d, double scale, float out[12])
{
    double Rrel[3][3], trel[3], KR[3][3], Kt[3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int m = 0; m < 3; ++m) acc += d.R[3 * i + m] * s.R[3 * j + m];
            Rrel[i][j] = acc;
        }
    for (int i = 0; i < 3; ++i) {
        double acc = 0.0;
        for (int j = 0; j < 3; ++j) acc += Rrel[i][j] * s.t[j];
        trel[i] = (d.t[i] - acc) * scale;
    }
    for (int j = 0; j < 3; ++j) {
        KR[0][j] = d.fx * Rrel[0][j] + d.cx * Rrel[2][j];
        KR[1][j] = d.fy * Rrel[1][j] + d.cy * Rrel[2][j];
        KR[2][j] = Rrel[2][j];
    }
    Kt[0] = d.fx * trel[0] + d.cx * trel[2];
    Kt[1] = d.fy * trel[1] + d.cy * trel[2];
    Kt[2] = trel[2];
    for (int i = 0; i < 3; ++i) {
        const double c0 = KR[i][0] / s.fx;
        const double c1 = KR[i][1] / s.fy;
        const double c2 = (KR[i][2] - (KR[i][0] * s.cx) / s.fx) - (KR[i][1] * s.cy) / s.fy;
        out[4 * i + 0] = float(c0);
        out[4 * i + 1] = float(c1);
        out[4 * i + 2] = float(c2);
        out[4 * i + 3] = float(Kt[i]);
    }
}

void centre_of(const fvv_camera& c, double C[3])
{
    for (int j = 0; j < 3; ++j)
        C[j] = -(c.R[0 + j] * c.t[0] + c.R[3 + j] * c.t[1] + c.R[6 + j] * c.t[2]);
}

// Sec. VI weights a reference camera by its distance from the virtual
// camera, read as the angle between the two viewing directions from the
// rig's look-at point: theta = atan2(|a x b|, a . b).
double angle_about(const double Cv[3], const double Ck[3], const double O[3])
{
    double a[3], b[3], c[3];
    for (int j = 0; j < 3; ++j) {
        a[j] = Cv[j] - O[j];
        b[j] = Ck[j] - O[j];
    }
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
    const double cn = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    const double dt = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
    return std::atan2(cn, dt);
}

// The n cameras of smallest angle to the view (ties to the lower index), as
// a bit mask: the active references of a view (n = n_ref) and the cameras a
// tick must carry for it (n = N_Tx, Sec. V-C adaptive view transmission).
uint64_t nearest_cameras(int n_cams, const fvv_camera* cams, const double look_at[3], const fvv_camera& view,
                         int n)
{
    double Cv[3], theta[fvv::kMaxCams];
    centre_of(view, Cv);
    for (int k = 0; k < n_cams; ++k) {
        double Ck[3];
        centre_of(cams[k], Ck);
        theta[k] = angle_about(Cv, Ck, look_at);
    }
    if (n <= 0 || n > n_cams) n = n_cams;
    uint64_t m = 0;
    for (int r = 0; r < n; ++r) {
        int best = -1;
        for (int k = 0; k < n_cams; ++k)
            if (!((m >> k) & 1u) && (best < 0 || theta[k] < theta[best])) best = k;
        m |= uint64_t(1) << best;
    }
    return m;
}

// Per-camera maps and weights of one view: the n_ref cameras of smallest
// angle get w = 1 / (theta + 1e-3), the rest 0; a view sitting on a camera
// (same centre within 1e-9 m, same optical axis) is one-hot on it.
void compose_view(int n_cams, const fvv_camera* cams, const double look_at[3],
                  double depth_unit_m, int n_ref, const fvv_camera& view, CamGeom* g)
{
    const double scale = 1.0 / depth_unit_m;
    double Cv[3], theta[fvv::kMaxCams];
    bool chosen[fvv::kMaxCams];
    centre_of(view, Cv);
    int onehot = -1;
    for (int k = 0; k < n_cams; ++k) {
        compose_map(cams[k], view, scale, g[k].M);
        compose_map(view, cams[k], scale, g[k].N);
        double Ck[3];
        centre_of(cams[k], Ck);
        // the camera's centre in the view's frame, R_v C_k + t_v, depth units
        for (int i = 0; i < 3; ++i) {
            double acc = 0.0;
            for (int j = 0; j < 3; ++j) acc += view.R[3 * i + j] * Ck[j];
            g[k].pad[i] = float((acc + view.t[i]) * scale);
        }
        theta[k] = angle_about(Cv, Ck, look_at);
        chosen[k] = false;
        const double dx = Cv[0] - Ck[0], dy = Cv[1] - Ck[1], dz = Cv[2] - Ck[2];
        const double dist = std::sqrt(dx * dx + dy * dy + dz * dz);
        const double axis = view.R[6] * cams[k].R[6] + view.R[7] * cams[k].R[7] +
                            view.R[8] * cams[k].R[8];
        if (onehot < 0 && dist < 1e-9 && axis > 1.0 - 1e-12) onehot = k;
    }
    if (n_ref <= 0 || n_ref > n_cams) n_ref = n_cams;
    if (onehot >= 0) {
        for (int k = 0; k < n_cams; ++k) g[k].w = k == onehot ? 1.0f : 0.0f;
        return;
    }
    for (int r = 0; r < n_ref; ++r) {
        int best = -1;
        for (int k = 0; k < n_cams; ++k)
            if (!chosen[k] && (best < 0 || theta[k] < theta[best])) best = k;
        chosen[best] = true;
    }
    for (int k = 0; k < n_cams; ++k)
        g[k].w = chosen[k] ? float(1.0 / (theta[k] + 1e-3)) : 0.0f;
}

}  // namespace

namespace fvv {
// Message for fvv_last_error() from code outside this file (failure paths).
void set_last_error(const char* msg) { g_err = msg; }

// Host-side composition of one view's per-camera maps and weights (the same
// routine the batched path uses); writes into caller storage only.
void compose_view_into(int n_cams, const fvv_camera* cams, const double look_at[3],
                       double depth_unit_m, int n_ref, const fvv_camera& view, CamGeom* g)
{
    compose_view(n_cams, cams, look_at, depth_unit_m, n_ref, view, g);
}
}  // namespace fvv

fvv_status fvv::dev_alloc(fvv_ctx* c, void** p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) return FVV_OK;
    if (c->opt.memory_budget && c->held + bytes > c->opt.memory_budget)
        return fail(FVV_ERR_BUDGET, "device memory budget exceeded (" + std::to_string(c->held + bytes) +
                                        " > " + std::to_string(c->opt.memory_budget) + " bytes)");
    FVV_CUDA(cudaMalloc(p, bytes));
    c->held += bytes;
    return FVV_OK;
}

void fvv::dev_free(fvv_ctx* c, void* p, size_t bytes)
{
    if (p) {
        cudaFree(p);
        c->held -= bytes;
    }
}

namespace {

size_t param_bytes(int n, int n_cams)
{
    return align_up(size_t(n) * sizeof(ViewDesc), 256) + size_t(n) * n_cams * sizeof(CamGeom);
}

fvv_status ensure_keys(fvv_ctx* c, BatchScratch& S, size_t n)
{
    if (n <= S.keys_cap) return FVV_OK;
    if (!S.growable)
        return fail(FVV_ERR_BUDGET, "batch needs " + std::to_string(n) + " z-buffer keys; the scratch holds " +
                                        std::to_string(S.keys_cap));
    if (S.keys) {
        FVV_CUDA(cudaDeviceSynchronize());
        dev_free(c, S.keys, S.keys_cap * 8);
        dev_free(c, S.keys2, S.keys_cap * 8);
        S.keys = nullptr;
        S.keys2 = nullptr;
        S.keys_cap = 0;
    }
    S.clean[0].clear();
    S.clean[1].clear();
    S.cur = 0;
    const size_t cap = align_up(n, 1 << 16);
    FVV_TRY(dev_alloc(c, reinterpret_cast<void**>(&S.keys), cap * 8));
    S.keys_cap = cap;
    // the second z-buffer only where the memory budget leaves room for it
    // (without it every batch clears its z-buffer first)
    if (!c->opt.memory_budget || c->held + cap * 8 <= c->opt.memory_budget)
        FVV_TRY(dev_alloc(c, reinterpret_cast<void**>(&S.keys2), cap * 8));
    return FVV_OK;
}

fvv_status ensure_out_stage(fvv_ctx* c, BatchScratch& S, size_t bytes)
{
    if (bytes <= S.out_stage_cap) return FVV_OK;
    if (!S.growable)
        return fail(FVV_ERR_BUDGET, "batch needs " + std::to_string(bytes) +
                                        " bytes of output staging; the scratch holds " +
                                        std::to_string(S.out_stage_cap));
    if (S.out_stage) {
        FVV_CUDA(cudaDeviceSynchronize());
        dev_free(c, S.out_stage, S.out_stage_cap);
        S.out_stage = nullptr;
        S.out_stage_cap = 0;
    }
    const size_t cap = align_up(bytes, 1 << 20);
    FVV_TRY(dev_alloc(c, reinterpret_cast<void**>(&S.out_stage), cap));
    S.out_stage_cap = cap;
    return FVV_OK;
}

fvv_status upload_one(fvv_ctx* c, int cam, const uint8_t* rgb, size_t rgb_pitch,
                      const uint16_t* depth, size_t depth_pitch, uint64_t tick, cudaStream_t s)
{
    return fvv::upload_frame(c, cam, rgb, rgb_pitch, depth, depth_pitch, nullptr, tick, s);
}

}  // namespace

fvv_status fvv::upload_frame(fvv_ctx* c, int cam, const uint8_t* rgb, size_t rgb_pitch, const uint16_t* depth,
                             size_t depth_pitch, const YuvDepth* yuv, uint64_t tick, cudaStream_t s)
{
    const fvv_camera& C = c->cams[cam];
    if (!rgb || (!depth && !yuv)) return fail(FVV_ERR_INVALID_ARG, "rgb and depth must be non-NULL");
    if (foreign(rgb) || foreign(depth) || (yuv && (foreign(yuv->y) || foreign(yuv->u) || foreign(yuv->v))))
        return fail(FVV_ERR_INVALID_ARG, "frame buffers must be host memory or the context's device memory");
    if (rgb_pitch < size_t(C.width) * 3) return fail(FVV_ERR_INVALID_ARG, "rgb_pitch < 3 * width");
    if (!yuv && depth_pitch < size_t(C.width) * 2) return fail(FVV_ERR_INVALID_ARG, "depth_pitch < 2 * width");
    const int si = int(tick % uint64_t(c->slots));
    SlotState& S = c->slot[si];
    if (S.any && tick < S.tick)
        return fail(FVV_ERR_STATE, "tick " + std::to_string(tick) + " is older than tick " +
                                       std::to_string(S.tick) + " held by its slot");
    if (!S.any || tick > S.tick) {
        S.any = true;
        S.tick = tick;
        S.mask = 0;
    }
    FVV_TRY(fvv::serve_wait_slot(c, S));
    for (int r = 0; r < fvv::kMaxReaders; ++r)
        if (S.read_pending[r]) FVV_CUDA(cudaStreamWaitEvent(s, S.read[r], 0));
    uint8_t* base = c->arena + size_t(si) * c->slot_bytes;
    uint16_t* ddst = reinterpret_cast<uint16_t*>(base + c->off_depth[cam]);
    uint32_t* rdst = reinterpret_cast<uint32_t*>(base + c->off_rgba[cam]);
    const bool staged = mem_kind(rgb) == MemKind::Host;
    // with the depth pre-filter the unfiltered codes go to a per-camera
    // buffer (or are read in place from device memory) and the filter
    // writes the slot
    const bool jbf = c->opt.jbf_radius > 0;
    const uint16_t* jsrc = nullptr;
    int64_t jpitch = 0;
    uint16_t* dfirst = ddst;
    if (jbf) {
        if (!c->jbf_tmp[cam])
            FVV_TRY(dev_alloc(c, reinterpret_cast<void**>(&c->jbf_tmp[cam]), size_t(C.height) * c->dpitch[cam] * 2));
        if (!yuv && mem_kind(depth) == MemKind::Device && depth_pitch % 2 == 0 &&
            (reinterpret_cast<uintptr_t>(depth) & 1) == 0) {
            jsrc = depth;
            jpitch = int64_t(depth_pitch / 2);
            dfirst = nullptr;
        } else {
            dfirst = c->jbf_tmp[cam];
            jsrc = dfirst;
            jpitch = c->dpitch[cam];
        }
    }
    if (staged || jbf) FVV_CUDA(cudaStreamWaitEvent(s, c->stage_free, 0));   // a previous upload may still read them
    if (yuv)
        FVV_TRY(run_kernel(c, kDecode, s, [&] {
            return fvv::launch_yuv_decode(*yuv, C.width, C.height, dfirst, size_t(c->dpitch[cam]) * 2, s);
        }));
    else if (dfirst)
        FVV_CUDA(cudaMemcpy2DAsync(dfirst, size_t(c->dpitch[cam]) * 2, depth, depth_pitch, size_t(C.width) * 2,
                                   size_t(C.height), cudaMemcpyDefault, s));
    const uint8_t* src = rgb;
    size_t spitch = rgb_pitch;
    if (staged) {
        if (!c->stage_rgb[cam]) {
            void* p = nullptr;
            FVV_TRY(dev_alloc(c, &p, size_t(C.width) * 3 * size_t(C.height)));
            c->stage_rgb[cam] = static_cast<uint8_t*>(p);
        }
        FVV_CUDA(cudaMemcpy2DAsync(c->stage_rgb[cam], size_t(C.width) * 3, rgb, rgb_pitch,
                                   size_t(C.width) * 3, size_t(C.height), cudaMemcpyHostToDevice, s));
        src = c->stage_rgb[cam];
        spitch = size_t(C.width) * 3;
    }
    FVV_TRY(run_kernel(c, kPack, s, [&] {
        return fvv::launch_pack_rgba(src, spitch, rdst, c->rpitch[cam], C.width, C.height, s);
    }));
    if (jbf) {
        JbfParams P;
        jbf_params(c->opt, C.width, C.height, &P);
        P.cam[0] = JbfCam{src, int64_t(spitch), jsrc, jpitch, ddst, int64_t(c->dpitch[cam])};
        FVV_TRY(run_kernel(c, kJbf, s, [&] { return launch_jbf(P, 1, s); }));
    }
    if (staged || jbf) FVV_CUDA(cudaEventRecord(c->stage_free, s));
    FVV_CUDA(cudaEventRecord(S.uploaded, s));
    S.mask |= uint64_t(1) << cam;
    c->have_any = true;
    if (S.mask == c->full_mask && (!c->have_latest || tick > c->latest)) {
        c->latest = tick;
        c->have_latest = true;
    }
    return FVV_OK;
}

// The cameras of `mask` (all of one size) for one tick in one launch, after
// at most two bulk host-to-device copies into the context's staging buffer;
// camera blocks are packed in ascending camera order.
// With yuv, each camera's depth block is a dense planar YUV420 depth frame
// (Eq. (3)) decoded on the way in; dp is unused then.
static fvv_status upload_all(fvv_ctx* c, uint64_t mask, const uint8_t* rgb, size_t rcs, size_t rp,
                             const uint8_t* depth, size_t dcs, size_t dp, uint64_t tick, cudaStream_t s, bool host,
                             bool yuv = false)
{
    using namespace fvv;
    int cams[kMaxCams], K = 0;
    for (int k = 0; k < c->n_cams; ++k)
        if ((mask >> k) & 1u) cams[K++] = k;
    if (K == 0) return fail(FVV_ERR_INVALID_ARG, "camera mask selects no camera");
    const int W = c->cams[cams[0]].width, H = c->cams[cams[0]].height;
    if (rp < size_t(W) * 3) return fail(FVV_ERR_INVALID_ARG, "rgb_pitch < 3 * width");
    const size_t yuv_bytes = size_t(W) * H + 2 * (size_t(W / 2) * (H / 2));
    if (yuv) {
        if (W % 2 || H % 2) return fail(FVV_ERR_INVALID_ARG, "YUV420 depth needs even width and height");
        if (dcs < yuv_bytes) return fail(FVV_ERR_INVALID_ARG, "depth camera stride < one YUV420 frame");
        for (int i = 0; i < K; ++i)
            if (!codec_decode_table(c, cams[i]))
                return fail(FVV_ERR_STATE, "camera " + std::to_string(cams[i]) + " has no depth codec");
    } else {
        if (dp < size_t(W) * 2 || dp % 2) return fail(FVV_ERR_INVALID_ARG, "depth_pitch < 2 * width or odd");
        if (dcs % 2) return fail(FVV_ERR_INVALID_ARG, "depth camera stride must be even");
    }
    const int si = int(tick % uint64_t(c->slots));
    SlotState& S = c->slot[si];
    if (S.any && tick < S.tick)
        return fail(FVV_ERR_STATE, "tick " + std::to_string(tick) + " is older than tick " +
                                       std::to_string(S.tick) + " held by its slot");
    if (!S.any || tick > S.tick) {
        S.any = true;
        S.tick = tick;
        S.mask = 0;
    }
    const uint8_t* r = rgb;
    const uint8_t* d = depth;
    const int sb = c->stage_all_next;
    if (host) {
        c->stage_all_next ^= 1;
        const size_t rspan = size_t(K - 1) * rcs + size_t(H - 1) * rp + size_t(W) * 3;
        const size_t dspan = size_t(K - 1) * dcs + (yuv ? yuv_bytes : size_t(H - 1) * dp + size_t(W) * 2);
        const size_t doff = align_up(rspan, 256);
        if (c->stage_all_bytes[sb] < doff + dspan) {
            FVV_CUDA(cudaEventSynchronize(c->stage_all_free[sb]));
            dev_free(c, c->stage_all[sb], c->stage_all_bytes[sb]);
            c->stage_all[sb] = nullptr;
            c->stage_all_bytes[sb] = 0;
            void* p = nullptr;
            FVV_TRY(dev_alloc(c, &p, doff + dspan));
            c->stage_all[sb] = static_cast<uint8_t*>(p);
            c->stage_all_bytes[sb] = doff + dspan;
        }
        FVV_CUDA(cudaStreamWaitEvent(s, c->stage_all_free[sb], 0));   // an earlier upload may still read it
        FVV_CUDA(cudaMemcpyAsync(c->stage_all[sb], rgb, rspan, cudaMemcpyHostToDevice, s));
        FVV_CUDA(cudaMemcpyAsync(c->stage_all[sb] + doff, depth, dspan, cudaMemcpyHostToDevice, s));
        r = c->stage_all[sb];
        d = c->stage_all[sb] + doff;
    }
    // only the writes into the slot wait for syntheses still reading it: the
    // copies into the staging buffer above may already run
    FVV_TRY(fvv::serve_wait_slot(c, S));
    for (int rd = 0; rd < kMaxReaders; ++rd)
        if (S.read_pending[rd]) FVV_CUDA(cudaStreamWaitEvent(s, S.read[rd], 0));
    UploadAll u{};
    u.rgb = r;
    u.rgb_cam_stride = rcs;
    u.rgb_pitch = rp;
    u.depth = d;
    u.depth_cam_stride = dcs;
    u.depth_pitch = dp;
    u.slot = c->arena + size_t(si) * c->slot_bytes;
    u.W = W;
    u.H = H;
    u.n_cams = K;
    u.dpitch = c->dpitch[cams[0]];
    u.rpitch = c->rpitch[cams[0]];
    u.yuv = yuv ? 1 : 0;
    const bool jbf = c->opt.jbf_radius > 0;
    for (int i = 0; i < K; ++i) {
        u.off_depth[i] = c->off_depth[cams[i]];
        u.off_rgba[i] = c->off_rgba[cams[i]];
        u.lut[i] = yuv ? codec_decode_table(c, cams[i]) : nullptr;
        u.ddst[i] = nullptr;
        if (yuv && jbf) {
            // the decoded codes go to the camera's unfiltered-code buffer;
            // the pre-filter then writes the slot
            const int k = cams[i];
            if (!c->jbf_tmp[k])
                FVV_TRY(dev_alloc(c, reinterpret_cast<void**>(&c->jbf_tmp[k]),
                                  size_t(c->cams[k].height) * c->dpitch[k] * 2));
            u.ddst[i] = c->jbf_tmp[k];
        }
    }
    FVV_TRY(run_kernel(c, kPack, s, [&] { return launch_upload_all(u, s); }));
    if (c->opt.jbf_radius > 0) {
        // the pre-filter reads the unfiltered codes where they came from and
        // overwrites the slot's depth rows
        JbfParams P;
        jbf_params(c->opt, W, H, &P);
        for (int i = 0; i < K; ++i)
            P.cam[i] = JbfCam{r + size_t(i) * rcs, int64_t(rp),
                              yuv ? u.ddst[i] : reinterpret_cast<const uint16_t*>(d + size_t(i) * dcs),
                              yuv ? int64_t(c->dpitch[cams[i]]) : int64_t(dp / 2),
                              reinterpret_cast<uint16_t*>(u.slot + c->off_depth[cams[i]]),
                              int64_t(c->dpitch[cams[i]])};
        FVV_TRY(run_kernel(c, kJbf, s, [&] { return launch_jbf(P, K, s); }));
    }
    if (host) FVV_CUDA(cudaEventRecord(c->stage_all_free[sb], s));
    FVV_CUDA(cudaEventRecord(S.uploaded, s));
    S.mask |= mask;
    c->have_any = true;
    if (S.mask == c->full_mask && (!c->have_latest || tick > c->latest)) {
        c->latest = tick;
        c->have_latest = true;
    }
    return FVV_OK;
}

fvv_status fvv::scratch_alloc(fvv_ctx* c, BatchScratch& S, size_t keys, size_t stage, int max_batch,
                              int n_blocks)
{
    S.growable = false;
    if (keys) {
        FVV_TRY(dev_alloc(c, reinterpret_cast<void**>(&S.keys), keys * 8));
        S.keys_cap = keys;
    }
    if (stage) {
        FVV_TRY(dev_alloc(c, reinterpret_cast<void**>(&S.out_stage), stage));
        S.out_stage_cap = stage;
    }
    const size_t pb = param_bytes(max_batch, c->n_cams);
    S.max_batch = max_batch;
    S.pring.resize(n_blocks);
    for (auto& p : S.pring) {
        FVV_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&p.host), pb, cudaHostAllocDefault));
        FVV_TRY(dev_alloc(c, reinterpret_cast<void**>(&p.dev), pb));
        p.cap = pb;
        FVV_CUDA(cudaEventCreateWithFlags(&p.done, cudaEventDisableTiming));
    }
    FVV_CUDA(cudaEventCreateWithFlags(&S.done, cudaEventDisableTiming));
    return FVV_OK;
}

void fvv::scratch_free(fvv_ctx* c, BatchScratch& S)
{
    for (auto& p : S.pring) {
        if (p.host) cudaFreeHost(p.host);
        dev_free(c, p.dev, p.cap);
        if (p.done) cudaEventDestroy(p.done);
    }
    S.pring.clear();
    dev_free(c, S.keys, S.keys_cap * 8);
    dev_free(c, S.keys2, S.keys_cap * 8);
    dev_free(c, S.out_stage, S.out_stage_cap);
    S.keys2 = nullptr;
    S.clean[0].clear();
    S.clean[1].clear();
    S.keys = nullptr;
    S.out_stage = nullptr;
    S.keys_cap = S.out_stage_cap = 0;
    if (S.done) cudaEventDestroy(S.done);
    S.done = nullptr;
}

size_t fvv::view_keys(const fvv_view& v, bool layered)
{
    // layered: the FG z-buffer, the BG z-buffer and the BG layer after its
    // crack filter
    return align_up(size_t(v.width) * v.height, 16) * (layered ? 3 : 1);
}

size_t fvv::view_stage_bytes(const fvv_view& v, uint8_t* out_rgb, const fvv_aux* aux)
{
    const size_t np = size_t(v.width) * v.height;
    size_t b = 0;
    if (mem_kind(out_rgb) == MemKind::Host) b += align_up(np * 3, 256);
    if (aux) {
        if (aux->depth && mem_kind(aux->depth) == MemKind::Host) b += align_up(np * 4, 256);
        if (aux->hole && mem_kind(aux->hole) == MemKind::Host) b += align_up(np, 256);
        if (aux->top3 && mem_kind(aux->top3) == MemKind::Host) b += align_up(np * 12, 256);
        if (aux->keys && mem_kind(aux->keys) == MemKind::Host) b += align_up(np * 8, 256);
    }
    return b;
}

fvv_status fvv::run_batch(fvv_ctx* c, BatchScratch& S, int n, const fvv_view* views,
                          const uint64_t* ticks, uint8_t* const* out_rgb, const size_t* out_pitch,
                          const fvv_aux* aux, cudaStream_t s, bool sync_host, PersistPost* post)
{
    if (n < 1 || n > S.max_batch)
        return fail(FVV_ERR_INVALID_ARG, "batch size must be in [1, max_batch]");
    if (!views || !out_rgb || !out_pitch) return fail(FVV_ERR_INVALID_ARG, "NULL views/out_rgb/out_pitch");
    FVV_CUDA(cudaSetDevice(c->device));

    // validate views, compose their per-camera maps and weights, and
    // resolve their frame slots: a view needs the frames of its active
    // cameras only (a tick may carry a subset of the cameras, Sec. V-C)
    std::string why;
    std::vector<int> slot_of(n);
    std::vector<CamGeom> geom(size_t(n) * c->n_cams);
    size_t key_total = 0, stage_total = 0;
    int max_w = 0, max_h = 0;
    for (int i = 0; i < n; ++i) {
        const fvv_view& V = views[i];
        if (!camera_ok(V, &why)) return fail(FVV_ERR_INVALID_ARG, "view " + std::to_string(i) + ": " + why);
        if (fvv::resolve_smem_bytes(V.width, c->n_cams, c->opt.layered != 0) > c->smem_optin)
            return fail(FVV_ERR_INVALID_ARG, "view " + std::to_string(i) + ": width too large");
        if (!out_rgb[i]) return fail(FVV_ERR_INVALID_ARG, "out_rgb[" + std::to_string(i) + "] is NULL");
        if (foreign(out_rgb[i]) ||
            (aux && (foreign(aux[i].depth) || foreign(aux[i].hole) || foreign(aux[i].top3) || foreign(aux[i].keys))))
            return fail(FVV_ERR_INVALID_ARG, "view " + std::to_string(i) +
                                                 ": outputs must be host memory or the context's device memory");
        if (out_pitch[i] < size_t(V.width) * 3) return fail(FVV_ERR_INVALID_ARG, "out_pitch < 3 * width");
        CamGeom* g = geom.data() + size_t(i) * c->n_cams;
        compose_view(c->n_cams, c->cams.data(), c->look_at, c->depth_unit_m, c->opt.n_ref, V, g);
        uint64_t need = 0;
        for (int k = 0; k < c->n_cams; ++k)
            if (g[k].w > 0.0f) need |= uint64_t(1) << k;
        uint64_t t = 0;
        if (ticks) {
            t = ticks[i];
            const SlotState& T = c->slot[t % uint64_t(c->slots)];
            if (!T.any || T.tick != t || (T.mask & need) != need)
                return fail(FVV_ERR_NOT_READY, "tick " + std::to_string(t) +
                                                   " does not hold the view's cameras or is no longer resident");
        } else {
            // the newest resident tick holding every camera the view uses
            bool found = false;
            for (int si = 0; si < c->slots; ++si) {
                const SlotState& T = c->slot[si];
                if (T.any && (T.mask & need) == need && (!found || T.tick > t)) {
                    t = T.tick;
                    found = true;
                }
            }
            if (!found) return fail(FVV_ERR_NOT_READY, "no resident tick holds the cameras of view " + std::to_string(i));
        }
        slot_of[i] = int(t % uint64_t(c->slots));
        const size_t np = size_t(V.width) * V.height;
        key_total += view_keys(V, c->opt.layered != 0);
        max_w = std::max(max_w, V.width);
        max_h = std::max(max_h, V.height);
        if (mem_kind(out_rgb[i]) == MemKind::Host) stage_total += align_up(np * 3, 256);
        if (aux) {
            const fvv_aux& A = aux[i];
            if (A.depth && mem_kind(A.depth) == MemKind::Host) stage_total += align_up(np * 4, 256);
            if (A.hole && mem_kind(A.hole) == MemKind::Host) stage_total += align_up(np, 256);
            if (A.top3 && mem_kind(A.top3) == MemKind::Host) stage_total += align_up(np * 12, 256);
            if (A.keys && mem_kind(A.keys) == MemKind::Host) stage_total += align_up(np * 8, 256);
        }
    }
    FVV_TRY(ensure_keys(c, S, key_total));
    FVV_TRY(ensure_out_stage(c, S, stage_total));

    // parameter block
    ParamBlock& P = S.pring[S.pnext];
    S.pnext = (S.pnext + 1) % int(S.pring.size());
    if (P.pending) FVV_CUDA(cudaEventSynchronize(P.done));
    ViewDesc* vd = reinterpret_cast<ViewDesc*>(P.host);
    const size_t geom_off = align_up(size_t(n) * sizeof(ViewDesc), 256);
    CamGeom* gh = reinterpret_cast<CamGeom*>(P.host + geom_off);
    const CamGeom* gd = reinterpret_cast<const CamGeom*>(P.dev + geom_off);

    // the z-buffer this batch splats into, and the one its resolve empties
    const bool ahead = S.keys2 != nullptr && !c->opt.layered && !post;
    unsigned long long* const kx = ahead && S.cur ? S.keys2 : S.keys;
    unsigned long long* const ky = ahead ? (S.cur ? S.keys : S.keys2) : nullptr;
    std::vector<size_t> layout;

    struct HostCopy { void* dst; size_t dpitch; const void* src; size_t spitch, width, height; };
    std::vector<HostCopy> d2h;
    std::vector<std::pair<void*, const void*>> raw_copies;   // keys_raw
    std::vector<size_t> raw_bytes;
    size_t koff = 0, soff = 0;
    int max_chunks = 0;
    bool any_host = false;
    for (int i = 0; i < n; ++i) {
        const fvv_view& V = views[i];
        ViewDesc& D = vd[i];
        std::memset(&D, 0, sizeof D);
        const size_t np = size_t(V.width) * V.height;
        D.Wv = V.width;
        D.Hv = V.height;
        D.n_cams = c->n_cams;
        D.slot = slot_of[i];
        D.flags = (c->opt.crack_filter ? fvv::kFlagCrack : 0) | (c->opt.hole_fill ? fvv::kFlagFill : 0) |
                  (c->opt.layered ? fvv::kFlagLayered : 0) | (c->opt.pixel_weights ? fvv::kFlagPixelWeights : 0);
        D.vk[0] = float(V.cx);
        D.vk[1] = float(V.cy);
        D.vk[2] = float(1.0 / V.fx);
        D.vk[3] = float(1.0 / V.fy);
        D.tau_crack = c->opt.tau_crack;
        D.tau_vis = c->opt.tau_vis;
        D.z_min = c->opt.z_min;
        D.d_lo = c->opt.d_lo;
        D.d_hi = c->opt.d_hi;
        D.keys = kx + koff;
        D.keys_next = ky ? ky + koff : nullptr;
        layout.push_back(align_up(np, 16));
        koff += align_up(np, 16);
        D.keys_bg = nullptr;
        D.keys_bgf = nullptr;
        if (c->opt.layered) {
            D.keys_bg = S.keys + koff;
            koff += align_up(np, 16);
            D.keys_bgf = c->opt.crack_filter ? S.keys + koff : D.keys_bg;
            koff += align_up(np, 16);
        }
        CamGeom* g = gh + size_t(i) * c->n_cams;
        std::memcpy(g, geom.data() + size_t(i) * c->n_cams, sizeof(CamGeom) * c->n_cams);
        D.geom = gd + size_t(i) * c->n_cams;
        int na = 0, chunks = 0;
        D.chunk_begin[0] = 0;
        for (int k = 0; k < c->n_cams; ++k)
            if (g[k].w > 0.0f) {
                D.active[na] = k;
                chunks += c->cams[k].height * ((c->cams[k].width + fvv::kSplatSeg - 1) / fvv::kSplatSeg);
                D.chunk_begin[++na] = chunks;
            }
        D.n_active = na;
        max_chunks = std::max(max_chunks, chunks);
        auto stage = [&](size_t bytes) {
            uint8_t* p = S.out_stage + soff;
            soff += align_up(bytes, 256);
            return p;
        };
        if (mem_kind(out_rgb[i]) == MemKind::Host) {
            D.out_rgb = stage(np * 3);
            D.out_pitch = int64_t(V.width) * 3;
            d2h.push_back({out_rgb[i], out_pitch[i], D.out_rgb, size_t(V.width) * 3, size_t(V.width) * 3,
                           size_t(V.height)});
        } else {
            D.out_rgb = out_rgb[i];
            D.out_pitch = int64_t(out_pitch[i]);
        }
        if (aux) {
            const fvv_aux& A = aux[i];
            auto plan = [&](void* user, size_t elem, void** dev_field) {
                if (!user) return;
                if (mem_kind(user) == MemKind::Host) {
                    uint8_t* p = stage(np * elem);
                    *dev_field = p;
                    d2h.push_back({user, np * elem, p, np * elem, np * elem, 1});
                } else {
                    *dev_field = user;
                }
            };
            plan(A.depth, 4, reinterpret_cast<void**>(&D.out_depth));
            plan(A.hole, 1, reinterpret_cast<void**>(&D.out_hole));
            plan(A.top3, 12, reinterpret_cast<void**>(&D.out_top3));
            plan(A.keys, 8, reinterpret_cast<void**>(&D.out_keys));
            if (A.keys_raw) {
                raw_copies.push_back({A.keys_raw, D.keys});
                raw_bytes.push_back(np * 8);
                if (mem_kind(A.keys_raw) == MemKind::Host) any_host = true;
            }
        }
    }
    if (!d2h.empty()) any_host = true;
    bool want_top3 = false;
    for (int i = 0; aux && i < n; ++i) want_top3 = want_top3 || aux[i].top3 != nullptr;
    const size_t pbytes = geom_off + size_t(n) * c->n_cams * sizeof(CamGeom);
    FVV_CUDA(cudaMemcpyAsync(P.dev, P.host, pbytes, cudaMemcpyHostToDevice, s));
    const ViewDesc* vdev = reinterpret_cast<const ViewDesc*>(P.dev);

    std::vector<int> used(c->slots, 0);
    for (int i = 0; i < n; ++i) used[slot_of[i]] = 1;
    for (int si = 0; si < c->slots; ++si)
        if (used[si]) FVV_CUDA(cudaStreamWaitEvent(s, c->slot[si].uploaded, 0));

    // the z-buffer scratch and output staging are shared by all batches using
    // S: a batch on another stream waits for the previous one
    if (S.pending) FVV_CUDA(cudaStreamWaitEvent(s, S.done, 0));
    if (post) {
        if (c->opt.layered || any_host || want_top3 || aux)
            return fail(FVV_ERR_INVALID_ARG, "persistent batches take device outputs and no aux outputs");
        int band = 1, sbx = 1;
        fvv::persist_batch_shape(n, max_h, max_chunks, post->ctas, &band, &sbx);
        post->batch = PersistBatch{vdev, c->frames_dev, S.keys, koff, n, max_h, band, sbx,
                                   c->opt.pixel_weights != 0 ? 1 : 0, {0, 0, 0}};
        post->slots.clear();
        for (int si = 0; si < c->slots; ++si)
            if (used[si]) post->slots.push_back(si);
        FVV_CUDA(cudaEventRecord(P.done, s));
        P.pending = true;
        return FVV_OK;
    }
    // a buffer whose view regions an earlier resolve emptied for this layout needs no clear
    const bool clean = ahead && S.clean[S.cur] == layout;
    S.clean[0].clear();
    S.clean[1].clear();
    if (!clean) FVV_TRY(run_kernel(c, kClear, s, [&] { return fvv::launch_clear_keys(kx, koff, s); }));
    FVV_TRY(run_kernel(c, kSplat, s, [&] {
        return fvv::launch_warp_splat(vdev, n, max_chunks, c->frames_dev, s, c->opt.layered != 0);
    }));
    if (c->opt.layered && c->opt.crack_filter)
        FVV_TRY(run_kernel(c, fvv::kCrackBg, s, [&] { return fvv::launch_crack_bg(vdev, n, max_h, max_w, s); }));
    for (size_t r = 0; r < raw_copies.size(); ++r)
        FVV_CUDA(cudaMemcpyAsync(raw_copies[r].first, raw_copies[r].second, raw_bytes[r],
                                 cudaMemcpyDefault, s));
    FVV_TRY(run_kernel(c, kResolve, s, [&] {
        return fvv::launch_resolve(vdev, n, max_h, max_w, c->n_cams, want_top3, c->frames_dev, s,
                                   c->opt.layered != 0, c->opt.pixel_weights != 0);
    }));
    if (ahead) {
        S.clean[1 - S.cur] = layout;
        S.cur ^= 1;
    }
    for (const HostCopy& h : d2h)
        FVV_CUDA(cudaMemcpy2DAsync(h.dst, h.dpitch, h.src, h.spitch, h.width, h.height,
                                   cudaMemcpyDeviceToHost, s));
    FVV_CUDA(cudaEventRecord(P.done, s));
    P.pending = true;
    FVV_CUDA(cudaEventRecord(S.done, s));
    S.pending = true;
    for (int si = 0; si < c->slots; ++si)
        if (used[si]) {
            SlotState& T = c->slot[si];
            if (!T.read[S.reader])
                FVV_CUDA(cudaEventCreateWithFlags(&T.read[S.reader], cudaEventDisableTiming));
            FVV_CUDA(cudaEventRecord(T.read[S.reader], s));
            T.read_pending[S.reader] = true;
        }
    if (any_host && sync_host) FVV_CUDA(cudaStreamSynchronize(s));
    return FVV_OK;
}

fvv_status fvv_synthesize_batch(fvv_ctx* c, int32_t n, const fvv_view* views, const uint64_t* ticks,
                                uint8_t* const* out_rgb, const size_t* out_pitch, const fvv_aux* aux,
                                void* stream)
{
    if (!c) return fail(FVV_ERR_INVALID_ARG, "ctx is NULL");
    if (n < 1 || n > c->opt.max_batch)
        return fail(FVV_ERR_INVALID_ARG, "batch size must be in [1, max_batch]");
    fvv::DeviceScope dev_scope(c->device);
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : c->own;
    std::lock_guard<std::recursive_mutex> lock(c->mu);
    return fvv::run_batch(c, c->main, n, views, ticks, out_rgb, out_pitch, aux, s, true);
}

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

fvv_status fvv_default_options(fvv_options* o)
{
    if (!o) return fail(FVV_ERR_INVALID_ARG, "options pointer is NULL");
    std::memset(o, 0, sizeof *o);
    o->n_ref = 0;
    o->crack_filter = 1;
    o->hole_fill = 1;
    o->tau_crack = 0.05f;
    o->tau_vis = 0.03f;
    o->z_min = 1.0f;
    o->d_lo = 1;
    o->d_hi = 65534;
    o->frame_slots = 2;
    o->max_batch = 64;
    o->memory_budget = 0;
    o->layered = 0;
    o->jbf_radius = 0;
    o->jbf_sigma_s = 2.0f;
    o->jbf_sigma_c = 10.0f;
    o->jbf_min_valid = 3;
    o->pixel_weights = 0;
    return FVV_OK;
}

const char* fvv_last_error(void) { return g_err.c_str(); }

static fvv_status check_rig(const fvv_rig* rig)
{
    if (!rig) return fail(FVV_ERR_INVALID_ARG, "rig is NULL");
    if (rig->n_cams < 1 || rig->n_cams > FVV_MAX_CAMS)
        return fail(FVV_ERR_INVALID_ARG, "n_cams must be in [1, 64]");
    if (!rig->cams) return fail(FVV_ERR_INVALID_ARG, "rig->cams is NULL");
    if (!(rig->depth_unit_m > 0.0) || !std::isfinite(rig->depth_unit_m))
        return fail(FVV_ERR_INVALID_ARG, "depth_unit_m must be > 0");
    if (!finite_all(rig->look_at, 3)) return fail(FVV_ERR_INVALID_ARG, "look_at must be finite");
    std::string why;
    for (int k = 0; k < rig->n_cams; ++k)
        if (!camera_ok(rig->cams[k], &why))
            return fail(FVV_ERR_INVALID_ARG, "camera " + std::to_string(k) + ": " + why);
    return FVV_OK;
}

fvv_status fvv_view_params(const fvv_rig* rig, const fvv_options* opt, const fvv_view* view,
                           float* M, float* N, float* w)
{
    FVV_TRY(check_rig(rig));
    fvv_options o;
    if (opt) o = *opt; else fvv_default_options(&o);
    std::string why;
    if (!options_ok(o, rig->n_cams, &why)) return fail(FVV_ERR_INVALID_ARG, why);
    if (!view || !camera_ok(*view, &why)) return fail(FVV_ERR_INVALID_ARG, "view: " + why);
    std::vector<CamGeom> g(rig->n_cams);
    compose_view(rig->n_cams, rig->cams, rig->look_at, rig->depth_unit_m, o.n_ref, *view, g.data());
    for (int k = 0; k < rig->n_cams; ++k) {
        if (M) std::memcpy(M + 12 * k, g[k].M, 12 * sizeof(float));
        if (N) std::memcpy(N + 12 * k, g[k].N, 12 * sizeof(float));
        if (w) w[k] = g[k].w;
    }
    return FVV_OK;
}

fvv_status fvv_destroy(fvv_ctx* c)
{
    if (!c) return FVV_OK;
    {   // the context's device for the teardown, the caller's again after it
        fvv::DeviceScope dev_scope(c->device);
        fvv::serve_shutdown(c);
        fvv::refine_destroy(c);
        fvv::codec_destroy(c);
        if (c->own) cudaStreamSynchronize(c->own);
        cudaDeviceSynchronize();
        fvv::scratch_free(c, c->main);
        for (auto& S : c->slot) {
            if (S.uploaded) cudaEventDestroy(S.uploaded);
            for (cudaEvent_t e : S.read)
                if (e) cudaEventDestroy(e);
        }
        for (auto& K : c->kstat)
            for (auto& ev : K.pending) c->event_pool.push_back(ev);
        for (auto& ev : c->event_pool) {
            cudaEventDestroy(ev.first);
            cudaEventDestroy(ev.second);
        }
        for (int k = 0; k < c->n_cams; ++k)
            if (c->stage_rgb[k])
                dev_free(c, c->stage_rgb[k], size_t(c->cams[k].width) * 3 * size_t(c->cams[k].height));
        for (size_t k = 0; k < c->bg.size(); ++k)
            dev_free(c, c->bg[k], size_t(c->cams[k].height) * c->dpitch[k] * 2);
        for (size_t k = 0; k < c->jbf_tmp.size(); ++k)
            dev_free(c, c->jbf_tmp[k], size_t(c->cams[k].height) * c->dpitch[k] * 2);
        dev_free(c, c->frames_dev, sizeof(FrameRef) * size_t(c->slots) * c->n_cams);
        dev_free(c, c->arena, c->arena_bytes);
        for (int i = 0; i < 2; ++i) {
            if (c->stage_all[i]) dev_free(c, c->stage_all[i], c->stage_all_bytes[i]);
            if (c->stage_all_free[i]) cudaEventDestroy(c->stage_all_free[i]);
        }
        if (c->stage_free) cudaEventDestroy(c->stage_free);
        if (c->own) cudaStreamDestroy(c->own);
        cudaGetLastError();
    }
    delete c;
    return FVV_OK;
}

fvv_status fvv_create(const fvv_rig* rig, const fvv_options* opt, fvv_ctx** out)
{
    if (!out) return fail(FVV_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    FVV_TRY(check_rig(rig));
    fvv_options o;
    if (opt) o = *opt; else fvv_default_options(&o);
    std::string why;
    if (!options_ok(o, rig->n_cams, &why)) return fail(FVV_ERR_INVALID_ARG, why);

    fvv_ctx* c = new fvv_ctx();
    c->n_cams = rig->n_cams;
    c->cams.assign(rig->cams, rig->cams + rig->n_cams);
    std::memcpy(c->look_at, rig->look_at, sizeof c->look_at);
    c->depth_unit_m = rig->depth_unit_m;
    c->opt = o;
    c->slots = o.frame_slots;
    c->full_mask = c->n_cams == 64 ? ~uint64_t(0) : ((uint64_t(1) << c->n_cams) - 1);
    c->stage_rgb.assign(c->n_cams, nullptr);
    c->bg.assign(c->n_cams, nullptr);
    c->jbf_tmp.assign(c->n_cams, nullptr);

    auto bail = [&](fvv_status s) {
        std::string msg = g_err;
        fvv_destroy(c);
        g_err = msg;
        return s;
    };
#define FVV_CREATE_TRY(expr)                 \
    do {                                     \
        fvv_status s_ = (expr);              \
        if (s_ != FVV_OK) return bail(s_);   \
    } while (0)
#define FVV_CREATE_CUDA(call)                                                                      \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            cudaGetLastError();                                                                    \
            return bail(fail(FVV_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)));  \
        }                                                                                          \
    } while (0)

    FVV_CREATE_CUDA(cudaGetDevice(&c->device));
    int optin = 0;
    FVV_CREATE_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    c->smem_optin = size_t(optin);
    FVV_CREATE_CUDA(cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking));

    // frame ring layout: per camera depth then RGBA8, rows padded to 128 B
    c->dpitch.resize(c->n_cams);
    c->rpitch.resize(c->n_cams);
    c->off_depth.resize(c->n_cams);
    c->off_rgba.resize(c->n_cams);
    size_t off = 0;
    for (int k = 0; k < c->n_cams; ++k) {
        const fvv_camera& C = c->cams[k];
        c->dpitch[k] = int(align_up(size_t(C.width) * 2, 128) / 2);
        c->rpitch[k] = int(align_up(size_t(C.width) * 4, 128) / 4);
        c->off_depth[k] = off;
        off = align_up(off + size_t(C.height) * c->dpitch[k] * 2, 256);
        c->off_rgba[k] = off;
        off = align_up(off + size_t(C.height) * c->rpitch[k] * 4, 256);
    }
    c->slot_bytes = off;
    c->arena_bytes = off * size_t(c->slots);
    FVV_CREATE_TRY(dev_alloc(c, reinterpret_cast<void**>(&c->arena), c->arena_bytes));
    FVV_CREATE_CUDA(cudaMemsetAsync(c->arena, 0, c->arena_bytes, c->own));

    std::vector<FrameRef> fr(size_t(c->slots) * c->n_cams);
    for (int s = 0; s < c->slots; ++s)
        for (int k = 0; k < c->n_cams; ++k) {
            FrameRef& F = fr[size_t(s) * c->n_cams + k];
            uint8_t* base = c->arena + size_t(s) * c->slot_bytes;
            F.depth = reinterpret_cast<const uint16_t*>(base + c->off_depth[k]);
            F.rgba = reinterpret_cast<const uint32_t*>(base + c->off_rgba[k]);
            F.W = c->cams[k].width;
            F.H = c->cams[k].height;
            F.dpitch = c->dpitch[k];
            F.rpitch = c->rpitch[k];
        }
    FVV_CREATE_TRY(dev_alloc(c, reinterpret_cast<void**>(&c->frames_dev), sizeof(FrameRef) * fr.size()));
    FVV_CREATE_CUDA(cudaMemcpyAsync(c->frames_dev, fr.data(), sizeof(FrameRef) * fr.size(),
                                    cudaMemcpyHostToDevice, c->own));

    c->slot.resize(c->slots);
    for (auto& S : c->slot) {
        FVV_CREATE_CUDA(cudaEventCreateWithFlags(&S.uploaded, cudaEventDisableTiming));
        FVV_CREATE_CUDA(cudaEventRecord(S.uploaded, c->own));
    }
    FVV_CREATE_CUDA(cudaEventCreateWithFlags(&c->stage_free, cudaEventDisableTiming));
    FVV_CREATE_CUDA(cudaEventRecord(c->stage_free, c->own));
    for (int i = 0; i < 2; ++i) {
        FVV_CREATE_CUDA(cudaEventCreateWithFlags(&c->stage_all_free[i], cudaEventDisableTiming));
        FVV_CREATE_CUDA(cudaEventRecord(c->stage_all_free[i], c->own));
    }
    FVV_CREATE_TRY(fvv::scratch_alloc(c, c->main, 0, 0, o.max_batch, 4));
    c->main.growable = true;
    FVV_CREATE_CUDA(cudaStreamSynchronize(c->own));
#undef FVV_CREATE_TRY
#undef FVV_CREATE_CUDA
    *out = c;
    return FVV_OK;
}

fvv_status fvv_upload_frame(fvv_ctx* c, int32_t cam, const uint8_t* rgb, size_t rgb_pitch,
                            const uint16_t* depth, size_t depth_pitch, uint64_t tick, void* stream)
{
    if (!c) return fail(FVV_ERR_INVALID_ARG, "ctx is NULL");
    if (cam < 0 || cam >= c->n_cams) return fail(FVV_ERR_INVALID_ARG, "camera index out of range");
    fvv::DeviceScope dev_scope(c->device);
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : c->own;
    std::lock_guard<std::recursive_mutex> lock(c->mu);
    return upload_one(c, cam, rgb, rgb_pitch, depth, depth_pitch, tick, s);
}

fvv_status fvv_set_bg_depth(fvv_ctx* c, int32_t cam, const uint16_t* depth, size_t pitch)
{
    if (!c) return fail(FVV_ERR_INVALID_ARG, "ctx is NULL");
    if (cam < 0 || cam >= c->n_cams) return fail(FVV_ERR_INVALID_ARG, "camera index out of range");
    const fvv_camera& C = c->cams[cam];
    if (depth && (pitch < size_t(C.width) * 2 || pitch % 2))
        return fail(FVV_ERR_INVALID_ARG, "pitch must be even and >= 2 * width");
    std::lock_guard<std::recursive_mutex> lock(c->mu);
    fvv::DeviceScope dev_scope(c->device);
    // kernels in flight may read the model: replace it only when they are done
    FVV_CUDA(cudaDeviceSynchronize());
    const size_t bytes = size_t(C.height) * c->dpitch[cam] * 2;
    uint16_t* m = c->bg[cam];
    if (!depth) {
        dev_free(c, m, bytes);
        m = nullptr;
    } else {
        if (!m) FVV_TRY(dev_alloc(c, reinterpret_cast<void**>(&m), bytes));
        c->bg[cam] = m;
        FVV_CUDA(cudaMemset(m, 0, bytes));
        FVV_CUDA(cudaMemcpy2D(m, size_t(c->dpitch[cam]) * 2, depth, pitch, size_t(C.width) * 2, size_t(C.height),
                              cudaMemcpyDefault));
    }
    c->bg[cam] = m;
    // every slot's frame record of this camera points at the model
    const uint16_t* p = m;
    for (int s = 0; s < c->slots; ++s)
        FVV_CUDA(cudaMemcpy(&c->frames_dev[size_t(s) * c->n_cams + cam].bg, &p, sizeof p, cudaMemcpyHostToDevice));
    return FVV_OK;
}

fvv_status fvv_upload_frames_subset(fvv_ctx* c, uint64_t cam_mask, const uint8_t* rgb, size_t rgb_cam_stride,
                                    size_t rgb_pitch, const uint16_t* depth, size_t depth_cam_stride,
                                    size_t depth_pitch, uint64_t tick, void* stream)
{
    if (!c) return fail(FVV_ERR_INVALID_ARG, "ctx is NULL");
    if (!rgb || !depth) return fail(FVV_ERR_INVALID_ARG, "rgb and depth must be non-NULL");
    if (cam_mask == 0 || (cam_mask & ~c->full_mask) != 0)
        return fail(FVV_ERR_INVALID_ARG, "camera mask empty or naming cameras the rig does not have");
    fvv::DeviceScope dev_scope(c->device);
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : c->own;
    std::lock_guard<std::recursive_mutex> lock(c->mu);
    int first = -1;
    bool uniform = true;
    for (int k = 0; k < c->n_cams; ++k) {
        if (!((cam_mask >> k) & 1u)) continue;
        if (first < 0) first = k;
        uniform = uniform && c->cams[k].width == c->cams[first].width &&
                  c->cams[k].height == c->cams[first].height;
    }
    const fvv::MemKind kr = fvv::mem_kind(rgb), kd = fvv::mem_kind(depth);
    if (kr == fvv::MemKind::Foreign || kd == fvv::MemKind::Foreign)
        return fail(FVV_ERR_INVALID_ARG, "frame buffers must be host memory or the context's device memory");
    // the batched kernel reads depth as uint16: device rows must be 2-byte aligned
    const bool aligned = depth_pitch % 2 == 0 && depth_cam_stride % 2 == 0 &&
                         (kd == fvv::MemKind::Host || (reinterpret_cast<uintptr_t>(depth) & 1) == 0);
    if (uniform && kr == kd && aligned)
        return upload_all(c, cam_mask, rgb, rgb_cam_stride, rgb_pitch, reinterpret_cast<const uint8_t*>(depth),
                          depth_cam_stride, depth_pitch, tick, s, kr == fvv::MemKind::Host);
    int i = 0;
    for (int k = 0; k < c->n_cams; ++k) {
        if (!((cam_mask >> k) & 1u)) continue;
        const uint8_t* r = rgb + size_t(i) * rgb_cam_stride;
        const uint16_t* d = reinterpret_cast<const uint16_t*>(
            reinterpret_cast<const uint8_t*>(depth) + size_t(i) * depth_cam_stride);
        FVV_TRY(upload_one(c, k, r, rgb_pitch, d, depth_pitch, tick, s));
        ++i;
    }
    return FVV_OK;
}

fvv_status fvv_upload_frames_yuv(fvv_ctx* c, const uint8_t* rgb, size_t rgb_cam_stride, size_t rgb_pitch,
                                 const uint8_t* yuv, size_t yuv_cam_stride, uint64_t tick, void* stream)
{
    if (!c) return fail(FVV_ERR_INVALID_ARG, "ctx is NULL");
    if (!rgb || !yuv) return fail(FVV_ERR_INVALID_ARG, "rgb and yuv must be non-NULL");
    fvv::DeviceScope dev_scope(c->device);
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : c->own;
    std::lock_guard<std::recursive_mutex> lock(c->mu);
    for (int k = 1; k < c->n_cams; ++k)
        if (c->cams[k].width != c->cams[0].width || c->cams[k].height != c->cams[0].height)
            return fail(FVV_ERR_INVALID_ARG, "fvv_upload_frames_yuv needs cameras of one size");
    const fvv::MemKind kr = fvv::mem_kind(rgb), ky = fvv::mem_kind(yuv);
    if (kr == fvv::MemKind::Foreign || ky == fvv::MemKind::Foreign)
        return fail(FVV_ERR_INVALID_ARG, "frame buffers must be host memory or the context's device memory");
    if (kr != ky) return fail(FVV_ERR_INVALID_ARG, "rgb and yuv must both be host or both device memory");
    return upload_all(c, c->full_mask, rgb, rgb_cam_stride, rgb_pitch, yuv, yuv_cam_stride, 0, tick, s,
                      kr == fvv::MemKind::Host, true);
}

fvv_status fvv_upload_frames(fvv_ctx* c, const uint8_t* rgb, size_t rgb_cam_stride, size_t rgb_pitch,
                             const uint16_t* depth, size_t depth_cam_stride, size_t depth_pitch,
                             uint64_t tick, void* stream)
{
    if (!c) return fail(FVV_ERR_INVALID_ARG, "ctx is NULL");
    return fvv_upload_frames_subset(c, c->full_mask, rgb, rgb_cam_stride, rgb_pitch, depth, depth_cam_stride,
                                    depth_pitch, tick, stream);
}

fvv_status fvv_select_cameras(const fvv_rig* rig, int32_t n_views, const fvv_view* views, int32_t n_tx,
                              uint64_t* mask)
{
    FVV_TRY(check_rig(rig));
    if (n_views < 1 || !views || !mask) return fail(FVV_ERR_INVALID_ARG, "need n_views >= 1, views and mask");
    if (n_tx < 1 || n_tx > rig->n_cams) return fail(FVV_ERR_INVALID_ARG, "n_tx must be in [1, n_cams]");
    std::string why;
    uint64_t m = 0;
    for (int i = 0; i < n_views; ++i) {
        if (!camera_ok(views[i], &why)) return fail(FVV_ERR_INVALID_ARG, "view " + std::to_string(i) + ": " + why);
        m |= nearest_cameras(rig->n_cams, rig->cams, rig->look_at, views[i], n_tx);
    }
    *mask = m;
    return FVV_OK;
}

fvv_status fvv_latest_tick(fvv_ctx* c, uint64_t* tick)
{
    if (!c || !tick) return fail(FVV_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::recursive_mutex> lock(c->mu);
    if (!c->have_latest) return fail(FVV_ERR_NOT_READY, "no complete frame tick uploaded yet");
    *tick = c->latest;
    return FVV_OK;
}

fvv_status fvv_profile_enable(fvv_ctx* c, int32_t on)
{
    if (!c) return fail(FVV_ERR_INVALID_ARG, "ctx is NULL");
    std::lock_guard<std::recursive_mutex> lock(c->mu);
    c->profiling = on != 0;
    return FVV_OK;
}

fvv_status fvv_profile_read(fvv_ctx* c, fvv_kernel_stats* out, int32_t* n, int32_t reset)
{
    if (!c || !n) return fail(FVV_ERR_INVALID_ARG, "NULL argument");
    fvv::DeviceScope dev_scope(c->device);
    std::lock_guard<std::recursive_mutex> lock(c->mu);
    for (auto& K : c->kstat) {
        for (auto& ev : K.pending) {
            FVV_CUDA(cudaEventSynchronize(ev.second));
            float ms = 0.0f;
            FVV_CUDA(cudaEventElapsedTime(&ms, ev.first, ev.second));
            K.ms += double(ms);
            ++K.timed;
            c->event_pool.push_back(ev);
        }
        K.pending.clear();
    }
    if (out) {
        const int m = std::min<int>(*n, kNumKernels);
        for (int i = 0; i < m; ++i) {
            std::memset(&out[i], 0, sizeof out[i]);
            std::snprintf(out[i].name, sizeof out[i].name, "%s", kKernelName[i]);
            out[i].launches = c->kstat[i].launches;
            out[i].timed = c->kstat[i].timed;
            out[i].total_ms = c->kstat[i].ms;
        }
    }
    *n = kNumKernels;
    if (reset)
        for (auto& K : c->kstat) {
            K.launches = 0;
            K.timed = 0;
            K.ms = 0.0;
        }
    return FVV_OK;
}

fvv_status fvv_synthesize(fvv_ctx* c, const fvv_view* view, uint8_t* out_rgb, size_t out_pitch,
                          const fvv_aux* aux, void* stream)
{
    return fvv_synthesize_batch(c, 1, view, nullptr, &out_rgb, &out_pitch, aux, stream);
}

}  // extern "C"
