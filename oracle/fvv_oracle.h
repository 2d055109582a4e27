/*
 * fvv_oracle.h -- plain, slow CPU oracle of the view-synthesis hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this code; the library never does.
 * It shares no code with the CUDA path.
 *
 * What it computes (FVV Live, Sec. VI "View synthesis"): depth-image-based
 * rendering of a virtual camera from calibrated multiview RGB8 + depth.
 * Each reference pixel with depth is a 3D point that is projected into the
 * virtual camera; cracks from magnification are handled by backward warping
 * plus filtering; several reference cameras are mixed according to their
 * distance to the virtual camera; disocclusions stay holes (Sec. IX shows
 * them black) unless the optional row-wise hole fill is on.
 *
 * The paper prints no formula for any of these steps.  The readings taken
 * here (FP32 warp in explicitly rounded operations, 64-bit z-buffer keys,
 * the 3x3 crack rule, the
 * angular weights, the visibility test, the hole-fill rule) are stated
 * beside each function in fvv_oracle.c.
 *
 * Units: camera poses in metres (FP64); depth codes in depth units
 * (millimetres for depth_unit_m = 0.001); all per-pixel arithmetic in FP32
 * on depth-unit lengths.
 */
#ifndef FVV_ORACLE_H
#define FVV_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_KEY_EMPTY (~(uint64_t)0)

typedef struct {
    int width, height;
    double fx, fy, cx, cy;
    double R[9];   /* world -> camera rotation, row-major */
    double t[3];   /* world -> camera translation, metres */
} or_camera;

typedef struct {
    int n_ref;          /* active reference cameras (0 = all) */
    int crack_filter;   /* 1 = apply the 3x3 crack/outlier rule */
    int hole_fill;      /* 1 = row-wise background-side fill */
    float tau_crack;    /* relative depth tolerance of the crack rule */
    float tau_vis;      /* relative depth tolerance of the visibility test */
    float z_min;        /* smallest accepted projected depth, depth units */
    uint32_t d_lo;      /* accepted depth codes [d_lo, d_hi] (d_lo >= 1) */
    uint32_t d_hi;
    int pixel_weights;  /* 1 = per-pixel angular weights (R9) instead of per-view ones */
} or_options;

/* Per-camera quantities of one virtual view, composed in FP64 and rounded
 * to FP32 once. */
typedef struct {
    float M[12];  /* forward  3x4: (u z, v z, z, 1) of camera k -> virtual (X, Y, Z) */
    float N[12];  /* backward 3x4: (x Z, y Z, Z, 1) of the view  -> camera k (X, Y, Z) */
    float w;      /* blend weight, 0 = camera not among the active references */
    float cv[3];  /* camera k's centre in the view's camera frame, depth units */
    float vk[4];  /* the view's cx, cy, 1/fx, 1/fy (the same for every k) */
} or_xform;

void oracle_default_options(or_options* o);

/* Host-side composition for one view (Sec. VI, DIBR geometry). */
void oracle_compose(int n_cams, const or_camera* cams, const or_camera* view,
                    const double look_at[3], double depth_unit_m, int n_ref,
                    or_xform* out);

/* Step a+b: warp every valid source pixel and keep the minimum key. */
void oracle_warp_splat(int n_cams, const or_camera* cams,
                       const uint16_t* const* depth, const size_t* depth_pitch,
                       const or_xform* xf, int Wv, int Hv, const or_options* opt,
                       uint64_t* keys);

/* Step c: one out-of-place pass of the 3x3 crack/outlier rule. */
void oracle_crack_filter(const uint64_t* keys_in, int Wv, int Hv, float tau,
                         uint64_t* keys_out);

/* Step d: backward fetch and weighted blend.  out_rgb is [Hv][Wv][3].
 * Optional (nullable): out_depth [Hv][Wv], out_hole [Hv][Wv],
 * out_top3 [Hv][Wv][3], out_nvis [Hv][Wv] (number of contributing cameras). */
void oracle_fetch_blend(int n_cams, const or_camera* cams,
                        const uint8_t* const* rgb, const size_t* rgb_pitch,
                        const uint16_t* const* depth, const size_t* depth_pitch,
                        const or_xform* xf, const uint64_t* keys, int Wv, int Hv,
                        const or_options* opt, uint8_t* out_rgb, float* out_depth,
                        uint8_t* out_hole, float* out_top3, uint8_t* out_nvis);

/* Step e: fill hole pixels of each row from the background side. */
void oracle_hole_fill(int Wv, int Hv, const uint8_t* hole, uint8_t* rgb,
                      float* depth);

/* All steps.  keys_raw / keys_filt / out_depth / out_hole / out_top3 are
 * nullable.  Returns 0, or -1 on invalid arguments. */
int oracle_synthesize(int n_cams, const or_camera* cams,
                      const uint8_t* const* rgb, const size_t* rgb_pitch,
                      const uint16_t* const* depth, const size_t* depth_pitch,
                      const double look_at[3], double depth_unit_m,
                      const or_camera* view, const or_options* opt,
                      uint8_t* out_rgb, float* out_depth, uint8_t* out_hole,
                      float* out_top3, uint64_t* keys_raw, uint64_t* keys_filt);

#ifdef __cplusplus
}
#endif
#endif
