/*
 * fvv.h -- C ABI of the GB300 view-synthesis library (libfvv.so).
 *
 * The library implements the real-time view-synthesis stage of FVV Live
 * (Sec. VI "View synthesis"): depth-image-based rendering (DIBR) of a
 * virtual camera, chosen by the viewer, from calibrated multiview colour
 * plus depth frames.  Every step runs in the library's CUDA kernels for
 * sm_103a:
 *   (a) per-camera unproject/reproject warp of every pixel with depth
 *       (Sec. VI: a pixel of a calibrated camera is a ray, and its depth
 *       fixes the 3D point on that ray);
 *   (b) z-buffer splat with 64-bit atomicMin on packed keys
 *       bits(Z) << 32 | camera << 26 | source pixel;
 *   (c) crack / outlier filter on the key image (Sec. VI: cracks from
 *       magnification, handled by backward warping plus filtering);
 *   (d) backward fetch and blend, each camera weighted by its angular
 *       distance from the virtual camera (Sec. VI weighs the cameras'
 *       contributions by that distance);
 *   (e) row-wise hole filling from the background side (Sec. VI names
 *       disocclusions; the paper leaves them black, Sec. IX, fig. of test
 *       screenshots -- the fill can be switched off).
 *
 * Conventions
 *   - Cameras: pinhole, pixel (u, v) has its centre at integer (u, v);
 *     x right, y down, z forward; R, t map world -> camera; t in metres.
 *   - Depth frames: uint16 codes, 0 = no depth, FVV_DEPTH_BG = a background
 *     pixel (Sec. V-A reserves the 12-bit code 0 for it; Sec. IV-B: its
 *     depth is not sent);
 *     other codes * depth_unit_m metres of camera-space z.  Colour frames:
 *     RGB8 interleaved.
 *   - Every call returns an fvv_status; on failure fvv_last_error() holds a
 *     message for the calling thread.
 *   - Buffers passed in may be host memory (pageable or pinned) or device
 *     memory of the context's device (the device current at fvv_create);
 *     the kind is detected per pointer.  Device memory of another GPU is
 *     refused with FVV_ERR_INVALID_ARG wherever a kernel would read or
 *     write it.  A call on a context makes the context's device current for
 *     its duration and gives the caller's current device back on return;
 *     calls without a context use the current device.  The library keeps
 *     no pointer to a caller buffer after a call returns.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the library's own
 *     stream).  Calls enqueue their GPU work on that stream; a call that
 *     writes host memory returns after that data is written.  Calls on one
 *     context must not be made from several threads at once.
 */
#ifndef FVV_H
#define FVV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t fvv_status;
#define FVV_OK                0
#define FVV_ERR_INVALID_ARG   1   /* bad pointer, size, index or option */
#define FVV_ERR_OUT_OF_MEMORY 2   /* a device or pinned allocation failed */
#define FVV_ERR_BUDGET        3   /* the request exceeds the memory budget */
#define FVV_ERR_CUDA          4   /* a CUDA call failed (message has the name) */
#define FVV_ERR_TIMEOUT       5   /* a bounded wait ran out */
#define FVV_ERR_BUSY          6   /* no free slot right now */
#define FVV_ERR_NOT_READY     7   /* no complete frame tick / result not ready */
#define FVV_ERR_STATE         8   /* call not valid in the context's state */

#define FVV_MAX_CAMS       64          /* 6-bit camera field of a key */
#define FVV_MAX_SRC_PIXELS (1u << 26)  /* 26-bit source-pixel field of a key */
#define FVV_KEY_EMPTY      (~(uint64_t)0)
#define FVV_DEPTH_BG       65535u      /* depth code signalling a background pixel */

typedef struct fvv_ctx fvv_ctx;

/* One calibrated pinhole camera, or the virtual camera of a view. */
typedef struct fvv_camera {
    int32_t width, height;      /* pixels, >= 1; width * height <= FVV_MAX_SRC_PIXELS */
    double fx, fy, cx, cy;      /* intrinsics, pixels */
    double R[9];                /* world -> camera rotation, row-major */
    double t[3];                /* world -> camera translation, metres */
} fvv_camera;

typedef fvv_camera fvv_view;

/* The reference-camera rig (Sec. III/IX: cameras on an arc around the scene). */
typedef struct fvv_rig {
    int32_t n_cams;             /* 1 .. FVV_MAX_CAMS */
    const fvv_camera* cams;     /* n_cams entries, copied by fvv_create */
    double look_at[3];          /* point the rig faces; centre of the angular weights */
    double depth_unit_m;        /* metres per depth code (0.001 = millimetres) */
} fvv_rig;

/* Options.  Initialise with fvv_default_options, then override fields. */
typedef struct fvv_options {
    int32_t n_ref;              /* active reference cameras: the n_ref of smallest angle
                                   to the view (Sec. VI: typically three); 0 = all */
    int32_t crack_filter;       /* 1 = apply step (c) */
    int32_t hole_fill;          /* 1 = apply step (e) */
    float tau_crack;            /* (c) relative depth tolerance, default 0.05 */
    float tau_vis;              /* (d) visibility tolerance |d - Z| <= tau_vis Z, default 0.03 */
    float z_min;                /* smallest accepted projected depth (depth units), >= 0, default 1 */
    uint32_t d_lo, d_hi;        /* accepted depth codes, default [1, 65534] (d_hi <= 65534:
                                   FVV_DEPTH_BG is never a depth) */
    int32_t frame_slots;        /* device-resident frame ticks kept (ring), default 2 */
    int32_t max_batch;          /* most views per batched call, default 64 */
    uint64_t memory_budget;     /* device bytes the context may hold, 0 = unlimited.  Within it
                                   the batch z-buffer is held twice (a batch's resolve empties
                                   the other copy, so the next batch of the same view sizes
                                   needs no clear); without room for that, once. */
    int32_t layered;            /* 1 = layered FG/BG synthesis (see fvv_set_bg_depth), default 0 */
    /* joint bilateral depth pre-filter on upload (see fvv_depth_jbf) */
    int32_t jbf_radius;         /* window radius 0..7, 0 = off (default) */
    float jbf_sigma_s;          /* spatial sigma, pixels, default 2 */
    float jbf_sigma_c;          /* colour sigma per RGB channel, default 10 */
    int32_t jbf_min_valid;      /* fill only with at least this many valid neighbours, default 3 */
    int32_t pixel_weights;      /* 1 = per-pixel angular weights in (d), see below; default 0 */
} fvv_options;

/* Optional per-view outputs (device or host pointers; NULL = not wanted).
 * Each is dense row-major over the view's height x width. */
typedef struct fvv_aux {
    float* depth;               /* [H][W] virtual-camera depth Z (depth units); 0 where no fill */
    uint8_t* hole;              /* [H][W] 1 = no reference camera contributed (before fill) */
    float* top3;                /* [H][W][3] three largest normalised blend weights, descending */
    uint64_t* keys;             /* [H][W] z-buffer keys after the crack filter */
    uint64_t* keys_raw;         /* [H][W] z-buffer keys before the crack filter */
} fvv_aux;

/* Per-pixel angular weights (pixel_weights = 1).  The n_ref cameras are
 * chosen per view as always; each contribution at output pixel (x, y) of
 * depth Z is then weighted by the angle at its surface point P = ((x - cx) /
 * fx Z, (y - cy) / fy Z, Z) (view frame) between the rays to camera k's
 * centre c_k and to the view's centre: w = 1 / (sqrt(2 (1 - cos)) + 0.001),
 * in FP32 as  lb = |P|, a = c_k - P, la = |a|, q = (a . P) / (la lb),
 * t = max(1 + q, 0), w = 1 / (sqrt(t + t) + 0.001f), dot products
 * ((x x + y y) + z z), c_k and 1/fx, 1/fy composed in FP64 and rounded once. */

/* Fill `opt` with the defaults listed above. */
fvv_status fvv_default_options(fvv_options* opt);

/* Message of the last failing call on this thread ("" if none).  The
 * pointer stays valid until the next failing call on this thread. */
const char* fvv_last_error(void);

/* Create a context on the current CUDA device: copies the rig, allocates the
 * frame ring (frame_slots ticks of every camera: RGBA8 + uint16 depth) and
 * scratch.  Errors: INVALID_ARG (rig/options), BUDGET, OUT_OF_MEMORY, CUDA. */
fvv_status fvv_create(const fvv_rig* rig, const fvv_options* opt, fvv_ctx** out);

/* Release every resource of `ctx` (waits for its work).  NULL is a no-op. */
fvv_status fvv_destroy(fvv_ctx* ctx);

/* Upload one camera's frame for capture tick `tick` (the per-tick input of
 * Sec. VI: decoded colour + depth of a reference camera).
 *   rgb:   height rows of width*3 bytes, row pitch `rgb_pitch` bytes
 *   depth: height rows of width uint16, row pitch `depth_pitch` bytes
 * Tick t lives in slot t % frame_slots.  A tick is complete once all cameras
 * have been uploaded for it; later syntheses see it.  Uploading into a slot
 * waits on the GPU for syntheses still reading that slot.  Errors:
 * INVALID_ARG, STATE (tick older than the one held by the slot), CUDA. */
fvv_status fvv_upload_frame(fvv_ctx* ctx, int32_t cam, const uint8_t* rgb,
                            size_t rgb_pitch, const uint16_t* depth,
                            size_t depth_pitch, uint64_t tick, void* stream);

/* Upload all cameras of one tick.  Camera k's rows start at
 * rgb + k * rgb_cam_stride and depth + k * depth_cam_stride (bytes). */
fvv_status fvv_upload_frames(fvv_ctx* ctx, const uint8_t* rgb, size_t rgb_cam_stride,
                             size_t rgb_pitch, const uint16_t* depth,
                             size_t depth_cam_stride, size_t depth_pitch,
                             uint64_t tick, void* stream);

/* ---- adaptive view transmission (Sec. V-C) -------------------------------
 * Only the N_Tx cameras nearest the viewers' viewpoints need to be sent for
 * a tick.  A tick may therefore carry a subset of the cameras: a view is
 * synthesised from the newest resident tick that holds all of its active
 * reference cameras (the n_ref of smallest angle), or from the tick named
 * in fvv_synthesize_batch's ticks if that one holds them (else NOT_READY).
 * fvv_latest_tick still reports the newest tick holding every camera. */

/* The cameras of cam_mask (bit k = camera k) for one tick; their blocks are
 * packed in ascending camera order: the i-th selected camera's rows start at
 * rgb + i * rgb_cam_stride and depth + i * depth_cam_stride.  Errors as
 * fvv_upload_frame; INVALID_ARG for an empty mask or one naming missing
 * cameras. */
fvv_status fvv_upload_frames_subset(fvv_ctx* ctx, uint64_t cam_mask, const uint8_t* rgb,
                                    size_t rgb_cam_stride, size_t rgb_pitch, const uint16_t* depth,
                                    size_t depth_cam_stride, size_t depth_pitch, uint64_t tick,
                                    void* stream);

/* The n_tx cameras of smallest angle to each of the n_views views (the
 * angle the blend weights use; ties to the lower index), OR-ed over the
 * views into *mask: the cameras the capture side must send for them.  With
 * n_tx >= the context's n_ref every view's references are included.  Needs
 * no GPU.  Errors: INVALID_ARG. */
fvv_status fvv_select_cameras(const fvv_rig* rig, int32_t n_views, const fvv_view* views, int32_t n_tx,
                              uint64_t* mask);

/* ---- layered FG/BG synthesis (Sec. VI: per-camera FG and BG layers) -----
 * With fvv_options.layered = 1 each camera's pixels split by the depth
 * signalling.  A depth code in [d_lo, d_hi] is a foreground (FG) point at
 * that depth.  FVV_DEPTH_BG is a background (BG) point at the depth of the
 * camera's static BG model, with the live colour (a BG pixel where the model
 * holds 0, or of a camera without a model, is not warped).  0 is neither.
 * Steps (a)-(d) run on each layer on its own: its own z-buffer and crack
 * filter, and in (d) the visibility test against that layer's depth in the
 * other cameras (FG: their live codes; BG: their model where they signal
 * BG), with the same angular weights.  The FG layer is then stacked over the
 * BG layer (a pixel shows FG wherever the filtered FG layer is present) and
 * (e) fills what neither covers.  aux.keys gives each pixel's key in the
 * layer shown, aux.keys_raw the FG layer's keys before the filter.  The
 * z-buffer scratch doubles.  Without layered, BG pixels have no depth. */

/* Set camera `cam`'s static BG depth model: height rows of width uint16
 * depth codes (0 = no model depth) at row pitch `pitch` bytes, host or device
 * memory, copied.  Waits for the device's work first.  depth = NULL removes
 * the model.  Errors: INVALID_ARG, BUDGET, OUT_OF_MEMORY, CUDA. */
fvv_status fvv_set_bg_depth(fvv_ctx* ctx, int32_t cam, const uint16_t* depth, size_t pitch);

/* ---- joint bilateral depth pre-filter (Sec. VI) ------------------------
 * A joint bilateral filter guided by the colour frame fills small gaps in
 * the live depth, in particular along object boundaries.  A pixel
 * without depth (0) takes the weighted mean of the valid codes (in [d_lo,
 * d_hi], not FVV_DEPTH_BG) of its (2 jbf_radius + 1)^2 window, visited in
 * row-major order; the weight is s(dx, dy) c(|dR|) c(|dG|) c(|dB|) with
 * s = exp(-(dx^2 + dy^2) / (2 jbf_sigma_s^2)) and c(t) = exp(-t^2 / (2
 * jbf_sigma_c^2)), each evaluated in FP64 and rounded to FP32 once, products
 * and sums in FP32 round-to-nearest in that order.  The code is
 * floor(sum w d / sum w + 0.5) clamped to [d_lo, d_hi], written when at
 * least jbf_min_valid neighbours are valid; other pixels keep their code.
 * With fvv_options.jbf_radius > 0 every uploaded frame (all upload calls)
 * is filtered before it enters the frame ring.  This call runs the filter
 * on one frame: rgb (height rows of width*3 bytes), depth and out (height
 * rows of width uint16, even pitches) in device memory; out must not overlap
 * depth.  Asynchronous on `stream`.  Errors: INVALID_ARG (options with
 * jbf_radius = 0 included), CUDA. */
fvv_status fvv_depth_jbf(const uint8_t* rgb, size_t rgb_pitch, const uint16_t* depth, size_t depth_pitch,
                         uint16_t* out, size_t out_pitch, int32_t width, int32_t height,
                         const fvv_options* opt, void* stream);

/* Newest complete tick, or NOT_READY if none. */
fvv_status fvv_latest_tick(fvv_ctx* ctx, uint64_t* tick);

/* Synthesise one virtual view from the newest complete tick: steps (a)-(e).
 *   out_rgb: height rows of width*3 bytes, row pitch `out_pitch` >= 3*width
 *   aux:     optional extra outputs (NULL = none)
 * Errors: INVALID_ARG, NOT_READY (no complete tick), BUDGET, CUDA. */
fvv_status fvv_synthesize(fvv_ctx* ctx, const fvv_view* view, uint8_t* out_rgb,
                          size_t out_pitch, const fvv_aux* aux, void* stream);

/* Synthesise n views in one batched pass (three kernel launches for the
 * whole batch).  ticks[i] selects view i's frame tick (must be complete and
 * still resident); ticks = NULL uses the newest complete tick for all.
 * aux may be NULL or an array of n entries.  Views may differ in size. */
fvv_status fvv_synthesize_batch(fvv_ctx* ctx, int32_t n, const fvv_view* views,
                                const uint64_t* ticks, uint8_t* const* out_rgb,
                                const size_t* out_pitch, const fvv_aux* aux,
                                void* stream);

/* Host-only: the per-camera quantities the kernels use for `view`, composed
 * in FP64 and rounded to FP32 once.  M: n_cams x 12 forward maps (camera ->
 * view, acting on (u z, v z, z, 1)); N: n_cams x 12 backward maps (view ->
 * camera); w: n_cams blend weights (0 = inactive).  Any output may be NULL.
 * Needs no GPU. */
fvv_status fvv_view_params(const fvv_rig* rig, const fvv_options* opt,
                           const fvv_view* view, float* M, float* N, float* w);

/* ---- depth codec of the transmission chain (Sec. IV-A Eq. (1), Sec. V-A Eq. (2), (3))
 * The capture side corrects depth (Eq. (1): z_post = (alpha z + beta) z, z in
 * metres), quantises it to 12-bit disparity (Eq. (2): Y = (2^12 - 3)(1/z -
 * 1/z_far) / (1/z_near - 1/z_far) + 2, rounded half up, for z in [z_near,
 * z_far]; code 1 marks values out of that range and pixels without depth,
 * code 0 background) and packs each 2x2 block onto 8-bit YUV420: pixel p's
 * Y value is its 8 LSBs, complemented when its 4 MSBs are odd (Eq. (3)); the
 * 4 MSBs of the top pair are bit-interleaved into U (bit i of the left pixel
 * at bit 2i, of the right pixel at bit 2i + 1), those of the bottom pair into
 * V.  The view-synthesis side inverts the packing and Eq. (2) on upload,
 * depth code = round(z / depth_unit_m) clamped to [1, 65534]; code 1
 * decodes to 0 (no depth) and code 0 to FVV_DEPTH_BG, which also encodes
 * back to code 0.
 * Both directions use per-camera tables built in FP64 on the host, so the
 * kernels are integer lookups.  Frames need even width and height. */
typedef struct fvv_depth_codec {
    double z_near, z_far;       /* clipping planes of Eq. (2), metres, 0 < z_near < z_far */
    double alpha, beta;         /* Eq. (1) correction; identity: alpha = 0, beta = 1 */
} fvv_depth_codec;

/* z_near 0.3 m, z_far 10 m, alpha 0, beta 1. */
fvv_status fvv_depth_codec_default(fvv_depth_codec* codec);
/* Set camera `cam`'s codec (builds its tables; waits for the context's
 * stream).  Errors: INVALID_ARG, OUT_OF_MEMORY, BUDGET, CUDA. */
fvv_status fvv_set_depth_codec(fvv_ctx* ctx, int32_t cam, const fvv_depth_codec* codec);
/* Capture side: camera `cam`'s uint16 depth codes (height rows, pitch
 * depth_pitch bytes, 4-byte aligned) -> Y (height rows of width bytes, pitch
 * y_pitch), U and V (height/2 rows of width/2 bytes, pitch uv_pitch); all
 * device memory; asynchronous on `stream`.  Errors: INVALID_ARG, STATE (no
 * codec set), CUDA. */
fvv_status fvv_depth_encode_yuv(fvv_ctx* ctx, int32_t cam, const uint16_t* depth, size_t depth_pitch, uint8_t* y,
                                size_t y_pitch, uint8_t* u, uint8_t* v, size_t uv_pitch, void* stream);
/* The inverse: Y, U, V planes -> uint16 depth codes; device memory;
 * asynchronous on `stream`.  Errors as for the encoder. */
fvv_status fvv_depth_decode_yuv(fvv_ctx* ctx, int32_t cam, const uint8_t* y, size_t y_pitch, const uint8_t* u,
                                const uint8_t* v, size_t uv_pitch, uint16_t* depth, size_t depth_pitch,
                                void* stream);
/* The decoder over every camera 0 .. n_cams-1 of one tick in one launch:
 * camera k's depth as one dense planar YUV420 frame at yuv + k *
 * yuv_cam_stride (Y: height rows of width bytes, then U and V: height/2 rows
 * of width/2 bytes each, the layout fvv_upload_frames_yuv takes), its codes
 * at depth + k * depth_cam_stride (height rows, pitch depth_pitch bytes).
 * Cameras of one size, even width and height, each with a codec set; device
 * memory; asynchronous on `stream`.  With width a multiple of 16 and 16-byte
 * aligned frames, strides and pitches the kernel moves 16 bytes per access;
 * otherwise it decodes frame after frame like fvv_depth_decode_yuv.  Errors:
 * INVALID_ARG (sizes, strides, pitches, host memory), STATE (a camera without
 * codec), CUDA. */
fvv_status fvv_depth_decode_yuv_frames(fvv_ctx* ctx, int32_t n_cams, const uint8_t* yuv, size_t yuv_cam_stride,
                                       uint16_t* depth, size_t depth_cam_stride, size_t depth_pitch, void* stream);
/* fvv_upload_frame with the depth given as a YUV420 depth frame: the decode
 * runs fused into the upload and writes the frame ring directly.  rgb and
 * the planes may be host or device memory (the three planes alike). */
fvv_status fvv_upload_frame_yuv(fvv_ctx* ctx, int32_t cam, const uint8_t* rgb, size_t rgb_pitch, const uint8_t* y,
                                size_t y_pitch, const uint8_t* u, const uint8_t* v, size_t uv_pitch, uint64_t tick,
                                void* stream);

/* Every camera of one tick with YUV420 depth, in one batched upload: camera
 * k's RGB8 rows at rgb + k * rgb_cam_stride (pitch rgb_pitch) and its depth
 * as one dense planar YUV420 frame at yuv + k * yuv_cam_stride (Y: height
 * rows of width bytes, then U and V: height/2 rows of width/2 bytes each).
 * Cameras of one size, even width and height, each with a codec set; rgb and
 * yuv both host or both device memory.  Decoded like fvv_upload_frame_yuv
 * (and pre-filtered when jbf_radius > 0).  Errors: INVALID_ARG, STATE (a
 * camera without codec, or a tick older than its slot's), CUDA. */
fvv_status fvv_upload_frames_yuv(fvv_ctx* ctx, const uint8_t* rgb, size_t rgb_cam_stride, size_t rgb_pitch,
                                 const uint8_t* yuv, size_t yuv_cam_stride, uint64_t tick, void* stream);

/* ---- serving loop (continuous batching of many viewers' requests) ------
 * The paper serves one viewer whose viewpoint commands reach the edge server
 * and wait for the next synthesised frame (Sec. VIII, motion-to-photon
 * delay).  Here many viewers submit viewpoint requests of any resolution; a
 * scheduler thread inside the library packs queued requests, in arrival
 * order, into batched launches of steps (a)-(e) on `lanes` CUDA streams.
 * Each lane owns device scratch sized from `memory_budget`; a batch is formed
 * when a lane is free, from the oldest requests that fit its scratch, so
 * requests arriving while others run join the next batch (continuous
 * batching) and batches on different lanes overlap on the GPU.  Every batch
 * renders from the newest complete frame tick when it is formed; frames keep
 * being uploaded with fvv_upload_frame(s) meanwhile.  Latency is measured
 * from fvv_serve_submit to the completion of the request's output write. */
/* With refine = 1 (fvv_refine_init first) each batch renders the plain views
 * into lane scratch, then the refinement network (in its current precision,
 * bf16 or E4M3) runs on one refinement stream shared by the lanes and writes
 * the requests' outputs.  A batch then holds requests of one size: the
 * oldest queued request and later ones of its width and height.  Views need
 * width and height multiples of 4.  The network's own activations are not
 * part of memory_budget.  While such a session runs, the fvv_refine_* calls
 * that use or change the network return FVV_ERR_BUSY. */
/* With persistent = 1 (plain views only: refine 0, no layered context) the
 * batches do not become kernel launches: one cooperative kernel, resident on
 * every SM, takes them from a ring of batch descriptors in pinned host
 * memory that the scheduler writes, runs steps (a)-(e) of each (grid
 * barriers between the steps), and publishes each batch's completion in
 * that memory, where a poller thread of the library sees it.  The kernel
 * returns after idle_us without work and is launched again for the next
 * batch.  It leaves room on every SM (registers for a small kernel) so
 * that frame uploads run beside it.  Views may be at most max_width wide (it sizes the kernel's shared
 * memory) and outputs must be device memory.  Every wait of the kernel is
 * bounded; a grid barrier that runs out ends the kernel and fails its
 * batches with FVV_ERR_TIMEOUT.  An upload into a frame slot that a posted
 * batch still reads waits (up to 2 s) for that batch. */
typedef struct fvv_serve_cfg {
    int32_t lanes;              /* batches in flight on the GPU, 1..16, default 3 */
    int32_t max_batch;          /* views per batched launch, default 16 */
    int32_t max_pending;        /* submitted and not yet polled, default 4096 */
    uint64_t memory_budget;     /* device bytes of serving scratch (all lanes), default 768 MiB */
    int32_t refine;             /* 1: every view also runs the refinement network (see below) */
    int32_t persistent;         /* 1: batches run in one persistent kernel (see above), default 0 */
    int32_t max_width;          /* persistent: widest view, default 1920 */
    uint32_t idle_us;           /* persistent: the kernel returns after this long without work, default 20000 */
    uint32_t batch_window_us;   /* coalescing window, default 0 (see below) */
} fvv_serve_cfg;

typedef struct fvv_serve_report {
    uint64_t submitted, completed, failed;
    uint64_t batches;           /* batched launches */
    double mean_batch;          /* views per launch */
    double p50_ms, p99_ms, max_ms;   /* per-view latency, submission -> output written */
    double views_per_s;         /* completed / (last completion - first submission) */
    int32_t in_flight;          /* submitted, not yet finished */
} fvv_serve_report;

/* batch_window_us > 0 trades latency for batch size: while fewer than
 * max_batch requests are queued, a batch waits until its oldest request has
 * been queued for batch_window_us (at most 1 s) before it leaves.  At light
 * load (each request finds the GPU idle) the default 0 gives batches of one. */
fvv_status fvv_serve_default_cfg(fvv_serve_cfg* cfg);

/* Start the scheduler thread and allocate the lanes' scratch.  Errors:
 * INVALID_ARG, STATE (already running), BUDGET (budget too small), CUDA. */
fvv_status fvv_serve_start(fvv_ctx* ctx, const fvv_serve_cfg* cfg);

/* Queue one view for `viewer`; `out` (device or host) receives height rows of
 * 3 * width bytes with row pitch `pitch` and must stay valid until the
 * ticket is polled.  Errors: INVALID_ARG, NOT_READY (no complete tick), BUSY
 * (max_pending outstanding), BUDGET (view larger than a lane's scratch),
 * STATE (not running / stopping). */
fvv_status fvv_serve_submit(fvv_ctx* ctx, uint32_t viewer, const fvv_view* view, uint8_t* out,
                            size_t pitch, uint64_t* ticket);

/* Wait up to timeout_us (0 = do not wait, < 0 = until done) for a ticket.
 * OK once the result is written (the ticket is then released), NOT_READY /
 * TIMEOUT if not finished, INVALID_ARG for an unknown ticket, CUDA if the
 * batch failed. */
fvv_status fvv_serve_poll(fvv_ctx* ctx, uint64_t ticket, int64_t timeout_us);

/* Throughput and latency percentiles since start or the last reset. */
fvv_status fvv_serve_stats(fvv_ctx* ctx, fvv_serve_report* out, int32_t reset);

/* Finish every queued and running request, then stop the thread and free
 * the lanes.  fvv_destroy stops a running loop too. */
fvv_status fvv_serve_stop(fvv_ctx* ctx);

/* ---- profiling (per-stage timing, after the paper's per-stage times of
 * Sec. VIII: decode, synthesis, end-to-end) ------------------------------ */

/* Per-kernel statistics of one context. */
typedef struct fvv_kernel_stats {
    char name[32];              /* "clear_keys", "warp_splat", "resolve", "pack_rgba", "yuv_decode" */
    uint64_t launches;          /* launches since the last reset */
    uint64_t timed;             /* of which bracketed by CUDA events */
    double total_ms;            /* summed event durations of the timed launches */
} fvv_kernel_stats;

/* on = 1: bracket every kernel launch of `ctx` with CUDA events recorded on
 * the launching stream (adds two event records per launch); 0: counts only. */
fvv_status fvv_profile_enable(fvv_ctx* ctx, int32_t on);

/* Copy up to *n entries into `out` (NULL = only return the count in *n);
 * waits for the recorded events.  reset = 1 clears the statistics. */
fvv_status fvv_profile_read(fvv_ctx* ctx, fvv_kernel_stats* out, int32_t* n, int32_t reset);

/* ---- diagnostics ----------------------------------------------------------
 * Self-test of the bounded waits that every tensor-core kernel of this
 * library uses (the paper has no counterpart).  One CTA initialises an
 * mbarrier expecting one arrival; if `arrive` != 0 a thread arrives on it;
 * then a thread waits for the phase to complete, giving up after limit_us
 * microseconds (1 .. 2,000,000).  A wait that gives up records an error code
 * in a device flag and the kernel exits normally, so the context stays
 * usable.  Allocates and frees one device int; waits for completion on
 * `stream` (NULL = the legacy default stream).
 * Returns OK when the phase completed, TIMEOUT when the wait ran out,
 * INVALID_ARG for a limit outside the range, CUDA on a launch failure. */
fvv_status fvv_selftest_bounded_wait(int32_t arrive, uint32_t limit_us, void* stream);

/* Diagnostic of the persistent serving kernel's bounded waits, on an empty
 * ring of batches (a context with an n_cams-camera rig is not needed).
 * barrier = 0: the kernel waits for work that never comes and returns after
 * idle_us.  barrier = 1: work is posted but the grid barrier's count is set
 * so that it never completes; every CTA gives up after limit_us.  Waits on
 * `stream`.  Returns TIMEOUT with the kernel's code in the message when the
 * limit ran out as intended (the wait for work: "idle", the barrier:
 * "barrier"), INVALID_ARG for limits outside [1, 2000000] us, CUDA. */
fvv_status fvv_selftest_persistent_wait(int32_t barrier, uint32_t limit_us, void* stream);

/* ---- refinement network: layer operations -------------------------------
 * The learned refinement (a U-Net; the paper has none) runs on the sm_103a
 * tensor cores.  Its layers are exposed for tests and custom pipelines.
 * Tensors are device memory, NHWC, bf16 unless stated. */

/* y = relu?(conv3x3(x, w) + bias), pad 1, stride 1, then optionally zeroed
 * where mask <= 0 (the ReLU derivative of a previous layer, for backward
 * passes).  Implicit GEMM on tcgen05 with fp32 accumulation in TMEM.
 *   x: [n][h][w][cin], cin a multiple of 8 (at most 4096)
 *   wt: [cout][3][3][cin]; bias: float [cout] or NULL
 *   cout: 32, 48, 64, 96, 128 or 192; mask: [n][h][w][cout] or NULL
 *   every pointer 16-byte aligned
 *   y: [n][h][w][cout]
 * Waits for completion on `stream`.  Errors: INVALID_ARG, TIMEOUT (a bounded
 * wait inside the kernel ran out), CUDA. */
fvv_status fvv_unet_conv3x3(const void* x, int32_t n, int32_t h, int32_t w, int32_t cin,
                            const void* wt, const float* bias, int32_t cout, int32_t relu,
                            const void* mask, void* y, void* stream);

/* Weight and bias gradients of that convolution on the tensor cores (the
 * paper has no network; these are the training step's kernels):
 *   dw[co][ky][kx][ci] = sum_p dz[p][co] x[p + (ky - 1, kx - 1)][ci],
 *   db[co] = sum_p dz[p][co]   (zero padding outside the image)
 *   x: [n][h][w] pixels of xstride bf16 channels, the first cin used
 *      (xstride 0 = cin); dz: [n][h][w][cout] bf16; cin, xstride and cout
 *      multiples of 8; x and dz 16-byte aligned
 *   dw: float [cout][3][3][cin], db: float [cout] or NULL (overwritten)
 * The pixels are split into fixed ranges whose fp32 partial sums are added
 * in a fixed order, so the result is reproducible bit for bit.  Allocates
 * its partial-sum scratch (cudaMalloc) for the call and waits for
 * completion on `stream`.  Errors: INVALID_ARG, OUT_OF_MEMORY, TIMEOUT (a
 * bounded wait inside the kernel ran out), CUDA. */
fvv_status fvv_unet_wgrad3x3(const void* x, int32_t n, int32_t h, int32_t w, int32_t cin, int32_t xstride,
                             const void* dz, int32_t cout, float* dw, float* db, void* stream);

/* FP8 form of the same convolution.  x, wt and y hold OCP E4M3 bytes (1
 * sign, 4 exponent bits with bias 7, 3 mantissa bits; largest finite 448).
 * With per-tensor scales s_x, s_w, s_y (x = s_x X, w = s_w W, y = s_y Y for
 * the stored codes X, W, Y):
 *   Y = e4m3(relu?(acc_scale * sum X W + bias) * out_inv_scale),
 * acc_scale = s_x s_w, out_inv_scale = 1 / s_y; e4m3() rounds to nearest
 * even and saturates to +-448.  Products accumulate in fp32 (tcgen05
 * kind::f8f6f4).  x: [n][h][w][cin], cin a multiple of 16; wt:
 * [cout][3][3][cin]; bias: float [cout] or NULL; y: [n][h][w][cout]; every
 * pointer 16-byte aligned.  Waits for completion on `stream`.
 * Errors: INVALID_ARG, TIMEOUT, CUDA. */
fvv_status fvv_unet_conv3x3_e4m3(const void* x, int32_t n, int32_t h, int32_t w, int32_t cin, const void* wt,
                                 const float* bias, int32_t cout, int32_t relu, float acc_scale,
                                 float out_inv_scale, void* y, void* stream);

/* The convolution (ReLU on) with the network's 2x2 max pooling of its output
 * fused into the same kernel, as the encoder uses it: y as
 * fvv_unet_conv3x3 (bf16) or fvv_unet_conv3x3_e4m3 (e4m3 = 1; acc_scale,
 * out_inv_scale as there), and pool_y[n][h/2][w/2][cout] (floors) the
 * maximum of each 2x2 window of y (the stored values; -0 ties with +0).
 * pool_arg (bf16 only, may be NULL): the window position 0..3 of each
 * maximum in the order (0,0), (0,1), (1,0), (1,1), the first one winning a
 * tie.  cout 32, 48 or 64.  Every pointer 16-byte aligned device memory.
 * Waits for completion on `stream`.  Errors: INVALID_ARG, TIMEOUT, CUDA. */
fvv_status fvv_unet_conv3x3_pool(const void* x, int32_t n, int32_t h, int32_t w, int32_t cin, const void* wt,
                                 const float* bias, int32_t cout, int32_t e4m3, float acc_scale,
                                 float out_inv_scale, void* y, void* pool_y, uint8_t* pool_arg, void* stream);

/* ---- refinement network ---------------------------------------------------
 * A 3-level U-Net refines a plain synthesis (the paper has none; it leaves
 * disocclusions black, Sec. IX).  Input: the blended RGB / 255, depth / z_far,
 * the hole mask and the three largest blend weights; output: clamp(RGB +
 * residual, 0, 1).  3x3 convolutions (pad 1) + ReLU at widths w1/w2/w3, 2x2
 * max pooling, nearest 2x upsampling with channel-concatenated skips, a 1x1
 * head; trained with mean-squared error against a held-out camera and Adam.
 * The 3x3 convolutions and their input gradients run on the tcgen05 tensor
 * cores (bf16 operands, fp32 accumulation); master weights are fp32. */
typedef struct fvv_unet_cfg {
    int32_t widths[3];          /* default 32, 64, 128; each one of 32, 48, 64, 96, 128, 192,
                                   widths[0] one of 32, 48, 64 */
    uint64_t seed;              /* weight initialisation */
    float z_far;                /* depth normalisation (depth units), default 8000 */
} fvv_unet_cfg;

/* One batch of plain-synthesis outputs (device memory, dense). */
typedef struct fvv_refine_batch {
    int32_t n, height, width;   /* height and width multiples of 4 */
    const uint8_t* rgb;         /* [n][h][w][3] blended colour */
    const float* depth;         /* [n][h][w] virtual depth (fvv_aux.depth) */
    const uint8_t* hole;        /* [n][h][w] hole mask (fvv_aux.hole) */
    const float* top3;          /* [n][h][w][3] top-3 blend weights (fvv_aux.top3) */
    const uint8_t* target;      /* [n][h][w][3] held-out camera colour (training only) */
} fvv_refine_batch;

/* Buffers addressable by fvv_refine_get / fvv_refine_set, each a flat fp32
 * vector of fvv_refine_param_count entries: per 3x3 layer (e1a, e1b, e2a,
 * e2b, ba, bb, d2a, d2b, d1a, d1b) W[cout][3][3][cin] then b[cout], then the
 * head W[3][w1] and b[3]. */
#define FVV_REFINE_PARAMS 0
#define FVV_REFINE_GRADS  1
#define FVV_REFINE_ADAM_M 2
#define FVV_REFINE_ADAM_V 3

fvv_status fvv_refine_default_cfg(fvv_unet_cfg* cfg);
/* (Re)create the network of `ctx` with fresh weights. */
fvv_status fvv_refine_init(fvv_ctx* ctx, const fvv_unet_cfg* cfg);
fvv_status fvv_refine_param_count(fvv_ctx* ctx, uint64_t* n);
/* Copy a buffer to / from host memory (waits for the device). */
fvv_status fvv_refine_get(fvv_ctx* ctx, int32_t which, float* out);
fvv_status fvv_refine_set(fvv_ctx* ctx, int32_t which, const float* in);
/* Forward pass: out_rgb [n][h][w][3] uint8 and/or out_f32 (clamped
 * prediction in [0, 1]); device memory, either may be NULL.  Waits. */
fvv_status fvv_refine_forward(fvv_ctx* ctx, const fvv_refine_batch* batch, uint8_t* out_rgb,
                              float* out_f32, void* stream);
/* Forward, backward and (lr > 0) one Adam step; *loss = mean squared error
 * of the batch before the update.  lr = 0 leaves the gradients readable with
 * FVV_REFINE_GRADS and changes nothing else.  Waits. */
fvv_status fvv_refine_train_step(fvv_ctx* ctx, const fvv_refine_batch* batch, float lr, float* loss,
                                 void* stream);
/* Checkpoint: widths, step, z_far, weights and Adam moments. */
fvv_status fvv_refine_save(fvv_ctx* ctx, const char* path);
fvv_status fvv_refine_load(fvv_ctx* ctx, const char* path);
/* ---- FP8 (E4M3) inference ------------------------------------------------
 * Post-training quantisation of the trained network.  Every activation
 * tensor is stored as E4M3 codes with one scale per tensor: the input
 * features with 2^-8, each 3x3 conv output t with s_t = amax_t / 448, where
 * amax_t is the largest |value| of t in a bf16 forward pass over `calib`
 * (act_scales NULL), or s_t = act_scales[t] for the ten conv outputs in layer
 * order (e1a ... d1b).  Weights get one scale per layer, s_w = amax(W') / 448,
 * where W' folds the scale ratio of a concatenated input's two parts into the
 * weights (W' = W s_part / s_first_part per input channel), so one fp32
 * accumulator multiplier per layer restores real units.  The 3x3 convs run
 * as fvv_unet_conv3x3_e4m3; pooling and upsampling move codes; the head
 * dequantises.  After this call fvv_refine_forward and fvv_synthesize_refined
 * run in E4M3 until fvv_refine_set_precision(FVV_PREC_BF16) or any change of
 * the weights (init, set, load, a training step), which returns to bf16.
 * calib: device memory as for fvv_refine_forward (ignored when act_scales is
 * given).  Waits.  Errors: STATE (no network), INVALID_ARG, TIMEOUT, CUDA. */
#define FVV_PREC_BF16 0
#define FVV_PREC_E4M3 1
fvv_status fvv_refine_quantize(fvv_ctx* ctx, const fvv_refine_batch* calib, const float* act_scales,
                               void* stream);
/* FVV_PREC_E4M3 needs quantised weights that are current (else STATE). */
fvv_status fvv_refine_set_precision(fvv_ctx* ctx, int32_t precision);
/* *precision, and (if not NULL) the ten activation scales in use. */
fvv_status fvv_refine_get_precision(fvv_ctx* ctx, int32_t* precision, float* act_scales);

/* Plain synthesis of `view` from the newest complete tick, then the
 * network; out_rgb device or host.  Width and height multiples of 4. */
fvv_status fvv_synthesize_refined(fvv_ctx* ctx, const fvv_view* view, uint8_t* out_rgb,
                                  size_t out_pitch, void* stream);

/* ---- allocation-free variant ------------------------------------------- */

/* Largest view (width * height) fvv_synthesize_noalloc accepts. */
#define FVV_NOALLOC_MAX_PIXELS (1u << 21)

/* Synthesise one view (steps a-e, the same kernels and results as
 * fvv_synthesize) without allocating any memory.  The paper has no
 * counterpart: this call exists for callers that must not call cudaMalloc --
 * a process whose device memory is owned by another allocator (a framework's
 * caching allocator that has reserved the GPU), or a latency-critical render
 * thread on which cudaMalloc / cudaFree would synchronise the device and
 * stall other streams.  It needs no context: the caller passes the frames
 * and the output, all in device memory.
 *   rig, opt:       as for fvv_create (opt NULL = defaults; frame_slots,
 *                   max_batch and memory_budget are ignored)
 *   depth[k]:       camera k's depth codes, uint16 rows of pitch depth_pitch[k]
 *                   bytes (even), 0 = no depth
 *   rgba[k]:        camera k's colour, one uint32 per pixel R | G << 8 | B << 16,
 *                   rows of pitch rgba_pitch[k] bytes (multiple of 4)
 *                   (each pitch in elements, p, must keep (H - 1) * p + W
 *                   below 2^32; depth, rgba and out_rgb must be memory of
 *                   the current device)
 *   view:           the virtual camera, width * height <= FVV_NOALLOC_MAX_PIXELS
 *   out_rgb:        height rows of 3 * width bytes, row pitch out_pitch
 *   stream:         cudaStream_t as void* (NULL = the legacy default stream);
 *                   the call is asynchronous on it
 * Scratch: file-scope device arrays (FVV_NOALLOC_MAX_PIXELS 64-bit z-buffer
 * keys = 16 MiB, plus about 10 KiB of launch parameters), which every GPU that
 * loads the library holds until the process exits.  Larger views are rejected
 * with FVV_ERR_INVALID_ARG.  The first call on a device looks up the device
 * address of that scratch (cudaGetSymbolAddress) with the device current;
 * make that first call before any stream capture.  The address is kept for
 * the life of the process, so a device reset (cudaDeviceReset) after the
 * first call is not supported.  Every call shares the
 * scratch and it keeps the last call's contents (the keys are reset at the
 * start of each call): calls whose GPU work overlaps, e.g. on two unordered
 * streams, race -- order them on one stream.  On success nothing is
 * allocated, on the host or the device.
 * Errors: INVALID_ARG (NULL, non-device pointer, size, pitch, options), CUDA. */
fvv_status fvv_synthesize_noalloc(const fvv_rig* rig, const fvv_options* opt,
                                  const uint16_t* const* depth, const size_t* depth_pitch,
                                  const uint32_t* const* rgba, const size_t* rgba_pitch,
                                  const fvv_view* view, uint8_t* out_rgb, size_t out_pitch,
                                  void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FVV_H */
