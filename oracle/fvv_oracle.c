/*
 * fvv_oracle.c -- plain, slow CPU oracle of FVV Live's view synthesis
 * (Sec. VI).  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the
 * benchmark's CPU-baseline leg load it; the library never does.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -shared -fPIC.
 * FP32 expressions are written one rounded operation at a time, with the
 * evaluation order spelled out by parentheses, and contraction into FMA is
 * disabled, so every FP32 result is the IEEE round-to-nearest value of that
 * exact sequence of operations.
 *
 * Readings of the paper (it gives the method in prose only):
 *   R1  units: lengths in depth units (mm); poses in metres, FP64 on the host.
 *   R2  the DIBR geometry of Sec. VI: a reference pixel (u, v) with depth z is
 *       the point z * K_k^-1 (u, v, 1); it is mapped to the virtual camera by
 *       K_v [R_v R_k^T | t_v - R_v R_k^T t_k] and the 3x4 product is rounded
 *       to FP32 once (M_k).  The backward map N_k swaps the roles.
 *   R3  forward projection (FMA-free):  a = ((m0 u + m1 v) + m2);
 *       X = a z + m3, likewise Y, Z; reject !(Z > z_min); u' = X / Z,
 *       v' = Y / Z; target pixel floor(u' + 0.5) (ties round up).
 *   R4  z-buffer: the smallest 64-bit key  bits(Z) << 32 | k << 26 | src
 *       wins; positive floats order like their bit patterns, so the key
 *       orders by depth, then camera, then source pixel.
 *   R5  crack/outlier filter (Sec. VI names cracks and "backward warping
 *       combined with filtering" but gives no rule): see oracle_crack_filter.
 *   R6  Sec. VI weights each reference camera by its distance from the
 *       virtual camera; read as the angular distance about the rig's
 *       look-at point: w_k = 1 / (theta_k + 1e-3) for the n_ref nearest
 *       cameras, 0 for the rest; one-hot when the view sits on a camera.
 *   R7  backward fetch: a non-winning camera contributes when the
 *       back-projected point lands in its image on a pixel with depth d and
 *       |d - Z_k| <= tau_vis * Z_k.
 *   R8  holes (disocclusions, Sec. VI) stay holes (black, as Sec. IX shows)
 *       unless the hole fill is on: a hole takes the nearer-left or
 *       nearer-right non-hole of its row, whichever is deeper (ties: left).
 *   R9  per-pixel angular weights (option): the n_ref cameras are chosen as
 *       in R6, but each contribution is weighted by the angle at the
 *       surface point between the rays to camera k and to the view, as the
 *       chord between their unit directions: see pixel_weight.
 */
#include "fvv_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAX_CAMS 64
#define OR_SRC_BITS 26

void oracle_default_options(or_options* o)
{
    o->n_ref = 0;
    o->crack_filter = 1;
    o->hole_fill = 1;
    o->tau_crack = 0.05f;
    o->tau_vis = 0.03f;
    o->z_min = 1.0f;
    o->d_lo = 1;
    o->d_hi = 65534;   /* 65535 signals a background pixel (Sec. V-A, code 0) */
    o->pixel_weights = 0;
}

static float key_depth(uint64_t key)
{
    uint32_t b = (uint32_t)(key >> 32);
    float f;
    memcpy(&f, &b, sizeof f);
    return f;
}

static uint32_t float_bits(float f)
{
    uint32_t b;
    memcpy(&b, &f, sizeof b);
    return b;
}

/* ------------------------------------------------------------------------
 * R2: FP64 composition.  Maps the homogeneous point (u z, v z, z, 1) of
 * camera `s` to (X, Y, Z) of camera `d`, with X / Z, Y / Z its pixel and Z
 * its depth in `d`.  Translation is converted from metres to depth units.
 * A = K_d R_rel K_s^-1 is formed column by column as
 *   A[:,0] = KR[:,0] / fx_s,  A[:,1] = KR[:,1] / fy_s,
 *   A[:,2] = (KR[:,2] - KR[:,0] cx_s / fx_s) - KR[:,1] cy_s / fy_s,
 * which is exact when the two cameras share intrinsics and orientation.
 * ---------------------------------------------------------------------- */
static void compose_pair(const or_camera* s, const or_camera* d, double scale,
                         float out[12])
{
    double Rrel[3][3], trel[3], KR[3][3], Kt[3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int m = 0; m < 3; ++m)
                acc += d->R[3 * i + m] * s->R[3 * j + m];
            Rrel[i][j] = acc;
        }
    for (int i = 0; i < 3; ++i) {
        double acc = 0.0;
        for (int j = 0; j < 3; ++j)
            acc += Rrel[i][j] * s->t[j];
        trel[i] = (d->t[i] - acc) * scale;
    }
    for (int j = 0; j < 3; ++j) {
        KR[0][j] = d->fx * Rrel[0][j] + d->cx * Rrel[2][j];
        KR[1][j] = d->fy * Rrel[1][j] + d->cy * Rrel[2][j];
        KR[2][j] = Rrel[2][j];
    }
    Kt[0] = d->fx * trel[0] + d->cx * trel[2];
    Kt[1] = d->fy * trel[1] + d->cy * trel[2];
    Kt[2] = trel[2];
    for (int i = 0; i < 3; ++i) {
        double a0 = KR[i][0] / s->fx;
        double a1 = KR[i][1] / s->fy;
        double a2 = (KR[i][2] - (KR[i][0] * s->cx) / s->fx) - (KR[i][1] * s->cy) / s->fy;
        out[4 * i + 0] = (float)a0;
        out[4 * i + 1] = (float)a1;
        out[4 * i + 2] = (float)a2;
        out[4 * i + 3] = (float)Kt[i];
    }
}

static void camera_center(const or_camera* c, double C[3])
{
    for (int j = 0; j < 3; ++j)
        C[j] = -(c->R[0 + j] * c->t[0] + c->R[3 + j] * c->t[1] + c->R[6 + j] * c->t[2]);
}

/* R6: angle between (C_v - O) and (C_k - O), atan2(|a x b|, a . b). */
static double view_angle(const double Cv[3], const double Ck[3], const double O[3])
{
    double a[3], b[3], c[3];
    for (int j = 0; j < 3; ++j) {
        a[j] = Cv[j] - O[j];
        b[j] = Ck[j] - O[j];
    }
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
    double cn = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    double dt = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
    return atan2(cn, dt);
}

void oracle_compose(int n_cams, const or_camera* cams, const or_camera* view,
                    const double look_at[3], double depth_unit_m, int n_ref,
                    or_xform* out)
{
    double scale = 1.0 / depth_unit_m;
    double Cv[3], theta[OR_MAX_CAMS];
    int chosen[OR_MAX_CAMS];
    camera_center(view, Cv);
    int onehot = -1;
    for (int k = 0; k < n_cams; ++k) {
        compose_pair(&cams[k], view, scale, out[k].M);
        compose_pair(view, &cams[k], scale, out[k].N);
        /* R9: camera k's centre in the view's frame, R_v C_k + t_v, depth units */
        double Ck0[3];
        camera_center(&cams[k], Ck0);
        for (int i = 0; i < 3; ++i) {
            double acc = 0.0;
            for (int j = 0; j < 3; ++j)
                acc += view->R[3 * i + j] * Ck0[j];
            out[k].cv[i] = (float)((acc + view->t[i]) * scale);
        }
        out[k].vk[0] = (float)view->cx;
        out[k].vk[1] = (float)view->cy;
        out[k].vk[2] = (float)(1.0 / view->fx);
        out[k].vk[3] = (float)(1.0 / view->fy);
        double Ck[3];
        camera_center(&cams[k], Ck);
        theta[k] = view_angle(Cv, Ck, look_at);
        chosen[k] = 0;
        double dx = Cv[0] - Ck[0], dy = Cv[1] - Ck[1], dz = Cv[2] - Ck[2];
        double dist = sqrt(dx * dx + dy * dy + dz * dz);
        double axis = view->R[6] * cams[k].R[6] + view->R[7] * cams[k].R[7] +
                      view->R[8] * cams[k].R[8];
        if (onehot < 0 && dist < 1e-9 && axis > 1.0 - 1e-12)
            onehot = k;
    }
    if (n_ref <= 0 || n_ref > n_cams)
        n_ref = n_cams;
    if (onehot >= 0) {
        for (int k = 0; k < n_cams; ++k)
            out[k].w = (k == onehot) ? 1.0f : 0.0f;
        return;
    }
    /* the n_ref smallest angles; ties go to the lower camera index */
    for (int r = 0; r < n_ref; ++r) {
        int best = -1;
        for (int k = 0; k < n_cams; ++k)
            if (!chosen[k] && (best < 0 || theta[k] < theta[best]))
                best = k;
        chosen[best] = 1;
    }
    for (int k = 0; k < n_cams; ++k)
        out[k].w = chosen[k] ? (float)(1.0 / (theta[k] + 1e-3)) : 0.0f;
}

/* ------------------------------------------------------------------------
 * Steps a + b: warp and z-buffer (R3, R4).  `keys` must hold Wv * Hv
 * entries; it is reset to empty first.
 * ---------------------------------------------------------------------- */
void oracle_warp_splat(int n_cams, const or_camera* cams,
                       const uint16_t* const* depth, const size_t* depth_pitch,
                       const or_xform* xf, int Wv, int Hv, const or_options* opt,
                       uint64_t* keys)
{
    for (size_t i = 0; i < (size_t)Wv * (size_t)Hv; ++i)
        keys[i] = OR_KEY_EMPTY;
    const float maxu = (float)(Wv - 1), maxv = (float)(Hv - 1);
    for (int k = 0; k < n_cams; ++k) {
        if (!(xf[k].w > 0.0f))
            continue;
        const float* m = xf[k].M;
        const int W = cams[k].width, H = cams[k].height;
        for (int v = 0; v < H; ++v) {
            const uint16_t* row = (const uint16_t*)((const char*)depth[k] + (size_t)v * depth_pitch[k]);
            const float fv = (float)v;
            for (int u = 0; u < W; ++u) {
                uint32_t d = row[u];
                if (d == 0 || d < opt->d_lo || d > opt->d_hi)
                    continue;
                const float fu = (float)u;
                const float z = (float)d;
                float a0 = ((m[0] * fu) + (m[1] * fv)) + m[2];
                float a1 = ((m[4] * fu) + (m[5] * fv)) + m[6];
                float a2 = ((m[8] * fu) + (m[9] * fv)) + m[10];
                float X = (a0 * z) + m[3];
                float Y = (a1 * z) + m[7];
                float Z = (a2 * z) + m[11];
                if (!(Z > opt->z_min))
                    continue;
                float up = X / Z;
                float vp = Y / Z;
                if (!isfinite(up) || !isfinite(vp))
                    continue;
                float tu = floorf(up + 0.5f);
                float tv = floorf(vp + 0.5f);
                if (!(tu >= 0.0f && tu <= maxu && tv >= 0.0f && tv <= maxv))
                    continue;
                size_t p = (size_t)(int)tv * (size_t)Wv + (size_t)(int)tu;
                uint64_t key = ((uint64_t)float_bits(Z) << 32) |
                               ((uint64_t)k << OR_SRC_BITS) |
                               (uint64_t)((size_t)v * (size_t)W + (size_t)u);
                if (key < keys[p])
                    keys[p] = key;
            }
        }
    }
}

/* ------------------------------------------------------------------------
 * Step c (R5).  For pixel p the neighbour pairs (left, right), (up, down),
 * (up-left, down-right), (up-right, down-left) are visited in that order.
 * A pair is consistent when both keys are non-empty and
 * zmax <= (1 + tau) * zmin.  An empty p takes min(key_a, key_b) of the
 * first consistent pair (closes magnification cracks); a non-empty p takes
 * it from the first consistent pair with z_p > (1 + tau) * zmax (removes
 * background seen through a foreground crack).  Off-image neighbours are
 * empty.  The filled key keeps the neighbour's camera and source fields.
 * ---------------------------------------------------------------------- */
static uint64_t key_at(const uint64_t* keys, int Wv, int Hv, int x, int y)
{
    if (x < 0 || y < 0 || x >= Wv || y >= Hv)
        return OR_KEY_EMPTY;
    return keys[(size_t)y * (size_t)Wv + (size_t)x];
}

void oracle_crack_filter(const uint64_t* keys_in, int Wv, int Hv, float tau,
                         uint64_t* keys_out)
{
    static const int pa[4][2] = {{-1, 0}, {0, -1}, {-1, -1}, {1, -1}};
    static const int pb[4][2] = {{1, 0}, {0, 1}, {1, 1}, {-1, 1}};
    const float f = 1.0f + tau;
    for (int y = 0; y < Hv; ++y)
        for (int x = 0; x < Wv; ++x) {
            uint64_t kp = keys_in[(size_t)y * Wv + x];
            uint64_t res = kp;
            for (int q = 0; q < 4; ++q) {
                uint64_t a = key_at(keys_in, Wv, Hv, x + pa[q][0], y + pa[q][1]);
                uint64_t b = key_at(keys_in, Wv, Hv, x + pb[q][0], y + pb[q][1]);
                if (a == OR_KEY_EMPTY || b == OR_KEY_EMPTY)
                    continue;
                float za = key_depth(a), zb = key_depth(b);
                float zlo = za < zb ? za : zb;
                float zhi = za < zb ? zb : za;
                if (!(zhi <= f * zlo))
                    continue;
                if (kp == OR_KEY_EMPTY || key_depth(kp) > f * zhi) {
                    res = a < b ? a : b;
                    break;
                }
            }
            keys_out[(size_t)y * Wv + x] = res;
        }
}

/* ------------------------------------------------------------------------
 * R9: per-pixel angular weight of camera k at output pixel (x, y) of depth
 * Z.  The surface point in the view's frame is P = ((x - cx) / fx Z,
 * (y - cy) / fy Z, Z); the weight falls with the angle at P between the
 * rays to camera k's centre c and to the view's centre (the origin),
 * measured by the chord between the two unit directions,
 * sqrt(2 (1 - cos)), so w = 1 / (chord + 1e-3).  FP32, in this order:
 *   px = ((x - cx) * (1/fx)) * Z,  py likewise,  pz = Z
 *   lb = sqrt((px px + py py) + pz pz)
 *   a = c - P,  la = sqrt((ax ax + ay ay) + az az)
 *   q = ((ax px + ay py) + az pz) / (la lb)       (= -cos)
 *   t = max(1 + q, 0),  chord = sqrt(t + t),  w = 1 / (chord + 0.001f)
 * ---------------------------------------------------------------------- */
static float pixel_weight(const or_xform* xk, float x, float y, float Z)
{
    const float px = ((x - xk->vk[0]) * xk->vk[2]) * Z;
    const float py = ((y - xk->vk[1]) * xk->vk[3]) * Z;
    const float pz = Z;
    const float lb = sqrtf((px * px + py * py) + pz * pz);
    const float ax = xk->cv[0] - px, ay = xk->cv[1] - py, az = xk->cv[2] - pz;
    const float la = sqrtf((ax * ax + ay * ay) + az * az);
    const float q = ((ax * px + ay * py) + az * pz) / (la * lb);
    float t = 1.0f + q;
    if (!(t > 0.0f))
        t = 0.0f;
    const float chord = sqrtf(t + t);
    return 1.0f / (chord + 0.001f);
}

/* ------------------------------------------------------------------------
 * Step d (R6, R7).  The winning key gives depth Z, camera w and source pixel
 * s.  acc = w_w * rgb_w[s]; then each other active camera k, in ascending
 * order, back-projects (x, y, Z) with N_k (same FMA-free order as R3), takes
 * the nearest pixel, and contributes w_k * rgb_k there when visible.
 * Output channel = min(255, floor(acc / wsum + 0.5)).  Aux: Z, hole flag,
 * the three largest normalised contributing weights (descending, ties by
 * lower camera index), number of contributing cameras.
 * ---------------------------------------------------------------------- */
void oracle_fetch_blend(int n_cams, const or_camera* cams,
                        const uint8_t* const* rgb, const size_t* rgb_pitch,
                        const uint16_t* const* depth, const size_t* depth_pitch,
                        const or_xform* xf, const uint64_t* keys, int Wv, int Hv,
                        const or_options* opt, uint8_t* out_rgb, float* out_depth,
                        uint8_t* out_hole, float* out_top3, uint8_t* out_nvis)
{
    for (int y = 0; y < Hv; ++y)
        for (int x = 0; x < Wv; ++x) {
            size_t p = (size_t)y * Wv + x;
            uint64_t key = keys[p];
            uint8_t* o = out_rgb + 3 * p;
            if (key == OR_KEY_EMPTY) {
                o[0] = o[1] = o[2] = 0;
                if (out_depth) out_depth[p] = 0.0f;
                if (out_hole) out_hole[p] = 1;
                if (out_top3) out_top3[3 * p] = out_top3[3 * p + 1] = out_top3[3 * p + 2] = 0.0f;
                if (out_nvis) out_nvis[p] = 0;
                continue;
            }
            const float Z = key_depth(key);
            const int w = (int)((key >> OR_SRC_BITS) & 63u);
            const uint32_t s = (uint32_t)(key & ((1u << OR_SRC_BITS) - 1u));
            const int su = (int)(s % (uint32_t)cams[w].width);
            const int sv = (int)(s / (uint32_t)cams[w].width);
            const uint8_t* c = rgb[w] + (size_t)sv * rgb_pitch[w] + 3 * (size_t)su;
            const float fx = (float)x, fy = (float)y;
            const float ww = opt->pixel_weights ? pixel_weight(&xf[w], fx, fy, Z) : xf[w].w;
            float acc[3], wsum = ww;
            float cw[OR_MAX_CAMS];
            int ck[OR_MAX_CAMS], nc = 0;
            for (int ch = 0; ch < 3; ++ch)
                acc[ch] = ww * (float)c[ch];
            cw[nc] = ww;
            ck[nc++] = w;
            for (int k = 0; k < n_cams; ++k) {
                if (k == w || !(xf[k].w > 0.0f))
                    continue;
                const float* n = xf[k].N;
                float a0 = ((n[0] * fx) + (n[1] * fy)) + n[2];
                float a1 = ((n[4] * fx) + (n[5] * fy)) + n[6];
                float a2 = ((n[8] * fx) + (n[9] * fy)) + n[10];
                float Xk = (a0 * Z) + n[3];
                float Yk = (a1 * Z) + n[7];
                float Zk = (a2 * Z) + n[11];
                if (!(Zk > opt->z_min))
                    continue;
                float up = Xk / Zk;
                float vp = Yk / Zk;
                if (!isfinite(up) || !isfinite(vp))
                    continue;
                float tu = floorf(up + 0.5f);
                float tv = floorf(vp + 0.5f);
                if (!(tu >= 0.0f && tu <= (float)(cams[k].width - 1) &&
                      tv >= 0.0f && tv <= (float)(cams[k].height - 1)))
                    continue;
                int uk = (int)tu, vk = (int)tv;
                const uint16_t* drow = (const uint16_t*)((const char*)depth[k] + (size_t)vk * depth_pitch[k]);
                uint32_t dk = drow[uk];
                if (dk == 0 || dk < opt->d_lo || dk > opt->d_hi)
                    continue;
                float diff = fabsf((float)dk - Zk);
                if (!(diff <= opt->tau_vis * Zk))
                    continue;
                const uint8_t* ckp = rgb[k] + (size_t)vk * rgb_pitch[k] + 3 * (size_t)uk;
                const float wk = opt->pixel_weights ? pixel_weight(&xf[k], fx, fy, Z) : xf[k].w;
                for (int ch = 0; ch < 3; ++ch)
                    acc[ch] = acc[ch] + wk * (float)ckp[ch];
                wsum = wsum + wk;
                cw[nc] = wk;
                ck[nc++] = k;
            }
            for (int ch = 0; ch < 3; ++ch) {
                float val = floorf(acc[ch] / wsum + 0.5f);
                o[ch] = (uint8_t)(val > 255.0f ? 255.0f : val);
            }
            if (out_depth) out_depth[p] = Z;
            if (out_hole) out_hole[p] = 0;
            if (out_nvis) out_nvis[p] = (uint8_t)nc;
            if (out_top3) {
                int used[OR_MAX_CAMS] = {0};
                for (int r = 0; r < 3; ++r) {
                    int best = -1;
                    for (int i = 0; i < nc; ++i)
                        if (!used[i] && (best < 0 || cw[i] > cw[best] ||
                                         (cw[i] == cw[best] && ck[i] < ck[best])))
                            best = i;
                    if (best < 0) {
                        out_top3[3 * p + r] = 0.0f;
                    } else {
                        used[best] = 1;
                        out_top3[3 * p + r] = cw[best] / wsum;
                    }
                }
            }
        }
}

/* ------------------------------------------------------------------------
 * Step e (R8).  left[x] / right[x] = nearest non-hole at or left / right of
 * x.  A hole copies colour and depth from the deeper of the two (ties: the
 * left one), from the only one that exists, or stays black.  The hole flags
 * are left as they are.
 * ---------------------------------------------------------------------- */
void oracle_hole_fill(int Wv, int Hv, const uint8_t* hole, uint8_t* rgb,
                      float* depth)
{
    int* left = (int*)malloc(sizeof(int) * (size_t)Wv);
    int* right = (int*)malloc(sizeof(int) * (size_t)Wv);
    for (int y = 0; y < Hv; ++y) {
        const size_t r = (size_t)y * Wv;
        int last = -1;
        for (int x = 0; x < Wv; ++x) {
            if (!hole[r + x]) last = x;
            left[x] = last;
        }
        last = -1;
        for (int x = Wv - 1; x >= 0; --x) {
            if (!hole[r + x]) last = x;
            right[x] = last;
        }
        for (int x = 0; x < Wv; ++x) {
            if (!hole[r + x])
                continue;
            int l = left[x], rr = right[x], src;
            if (l < 0 && rr < 0)
                continue;
            if (l < 0) src = rr;
            else if (rr < 0) src = l;
            else src = depth[r + rr] > depth[r + l] ? rr : l;
            for (int ch = 0; ch < 3; ++ch)
                rgb[3 * (r + x) + ch] = rgb[3 * (r + src) + ch];
            depth[r + x] = depth[r + src];
        }
    }
    free(left);
    free(right);
}

int oracle_synthesize(int n_cams, const or_camera* cams,
                      const uint8_t* const* rgb, const size_t* rgb_pitch,
                      const uint16_t* const* depth, const size_t* depth_pitch,
                      const double look_at[3], double depth_unit_m,
                      const or_camera* view, const or_options* opt,
                      uint8_t* out_rgb, float* out_depth, uint8_t* out_hole,
                      float* out_top3, uint64_t* keys_raw, uint64_t* keys_filt)
{
    if (n_cams < 1 || n_cams > OR_MAX_CAMS || !view || view->width < 1 ||
        view->height < 1 || !(depth_unit_m > 0.0))
        return -1;
    for (int k = 0; k < n_cams; ++k)
        if (cams[k].width < 1 || cams[k].height < 1 ||
            (size_t)cams[k].width * (size_t)cams[k].height > ((size_t)1 << OR_SRC_BITS))
            return -1;
    const int Wv = view->width, Hv = view->height;
    const size_t np = (size_t)Wv * Hv;
    or_xform xf[OR_MAX_CAMS];
    oracle_compose(n_cams, cams, view, look_at, depth_unit_m, opt->n_ref, xf);
    uint64_t* k0 = (uint64_t*)malloc(np * sizeof(uint64_t));
    uint64_t* k1 = (uint64_t*)malloc(np * sizeof(uint64_t));
    float* dep = (float*)malloc(np * sizeof(float));
    uint8_t* hole = (uint8_t*)malloc(np);
    oracle_warp_splat(n_cams, cams, depth, depth_pitch, xf, Wv, Hv, opt, k0);
    if (opt->crack_filter)
        oracle_crack_filter(k0, Wv, Hv, opt->tau_crack, k1);
    else
        memcpy(k1, k0, np * sizeof(uint64_t));
    oracle_fetch_blend(n_cams, cams, rgb, rgb_pitch, depth, depth_pitch, xf, k1,
                       Wv, Hv, opt, out_rgb, dep, hole, out_top3, NULL);
    if (opt->hole_fill)
        oracle_hole_fill(Wv, Hv, hole, out_rgb, dep);
    if (out_depth) memcpy(out_depth, dep, np * sizeof(float));
    if (out_hole) memcpy(out_hole, hole, np);
    if (keys_raw) memcpy(keys_raw, k0, np * sizeof(uint64_t));
    if (keys_filt) memcpy(keys_filt, k1, np * sizeof(uint64_t));
    free(k0);
    free(k1);
    free(dep);
    free(hole);
    return 0;
}
