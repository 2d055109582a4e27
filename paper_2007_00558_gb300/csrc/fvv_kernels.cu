// fvv_kernels.cu -- CUDA kernels (sm_103a) of the view-synthesis hot path.
//
// FVV Live, Sec. VI: each reference pixel with depth is a 3D point that is
// projected into the virtual camera; cracks from magnification are handled
// by backward warping plus filtering; the contributions of several reference
// cameras are mixed according to their distance to the virtual camera;
// disoccluded pixels are holes.
//
//   k_clear_keys   reset the per-view z-buffers to the empty key
//   k_warp_splat   (a) forward warp + (b) 64-bit atomicMin z-buffer splat
//   k_resolve      (c) crack filter + (d) backward fetch and blend +
//                  (e) row hole fill, fused: one CTA per output row
//   k_pack_rgba    upload: RGB8 rows -> RGBA8 (one aligned 32-bit gather per texel)
//
// Layered form (Sec. VI, per-camera FG and BG layers): a pixel signalled BG
// (kDepthBg) is a point of the BG layer at its camera's static model depth,
// every other valid pixel a point of the FG layer; each layer has its own
// z-buffer, crack filter and visibility test, and the FG layer is stacked
// over the BG layer before the hole fill.  The kernels take it as a
// template parameter, so the single-layer form carries none of it.
//
// Every FP32 operation of the warp, the filter and the blend is an explicit
// round-to-nearest intrinsic (__fmul_rn / __fadd_rn / __fsub_rn / __fdiv_rn)
// in a fixed, FMA-free order -- each product and each sum rounded once, each
// quotient a correctly rounded division -- so the results are exactly the
// IEEE values of that sequence.
#include <climits>

#include "fvv_internal.h"

namespace fvv {

namespace {

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

constexpr int kGeomFloats = 20;   // per-camera record of the resolve kernel
constexpr int kRing = 4;          // key rows kept in shared memory (3 in use + 1 in flight)

struct SmemLayout {
    size_t ring, rgb, dep, hole, geom, rowt, frames, active, pos, scan, total;
};

__host__ __device__ inline SmemLayout resolve_layout(int W, int n_cams, bool layered)
{
    SmemLayout L;
    size_t o = 0;
    (void)layered;                // the layered form reads its BG keys from the filtered z-buffer
    L.ring = o;   o = align16(o + size_t(kRing) * W * sizeof(unsigned long long));
    L.rgb = o;    o = align16(o + size_t(W) * 4);
    L.dep = o;    o = align16(o + size_t(W) * 4);
    L.hole = o;   o = align16(o + size_t(W));
    // (the hole fill's nearest-left / nearest-right indices live in the key
    // ring's slot of the row above, which no pixel reads any more by then)
    L.geom = o;   o = align16(o + size_t(n_cams) * kGeomFloats * sizeof(float));
    L.rowt = o;   o = align16(o + size_t(n_cams) * 4 * sizeof(float));
    L.frames = o; o = align16(o + size_t(n_cams) * sizeof(FrameRef));
    L.active = o; o = align16(o + size_t(kMaxCams) * sizeof(int));
    L.pos = o;    o = align16(o + size_t(kMaxCams) * sizeof(int));
    L.scan = o;   o = align16(o + 64 * sizeof(int));
    L.total = o;
    return L;
}

__device__ __forceinline__ float key_z(unsigned long long k)
{
    return __uint_as_float(static_cast<uint32_t>(k >> 32));
}

}  // namespace

// ---------------------------------------------------------------------------
// z-buffer reset
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_clear_keys(unsigned long long* __restrict__ keys, size_t n)
{
    const size_t stride = size_t(gridDim.x) * blockDim.x;
    const size_t i0 = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    const size_t npair = n >> 1;
    for (size_t j = i0; j < npair; j += stride)
        asm volatile("st.global.L2::cache_hint.v2.u64 [%0], {%1, %2}, %3;" ::"l"(keys + 2 * j),
                     "l"(kKeyEmpty), "l"(kKeyEmpty), "l"(pol)
                     : "memory");
    if ((n & 1) && i0 == 0)
        keys[n - 1] = kKeyEmpty;
}

// ---------------------------------------------------------------------------
// cache-policy helpers (PTX createpolicy / cache_hint forms, sm_80+)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t policy_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint64_t policy_evict_last()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// fire-and-forget 64-bit atomic minimum, kept in L2
__device__ __forceinline__ void red_min_key(unsigned long long* ptr, unsigned long long v, uint64_t pol)
{
    asm volatile("red.global.min.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(ptr), "l"(v), "l"(pol)
                 : "memory");
}

// streaming 2-byte load (read once)
__device__ __forceinline__ uint32_t ld_stream_u16(const uint16_t* ptr, uint64_t pol)
{
    unsigned short v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u16 %0, [%1], %2;"
                 : "=h"(v) : "l"(ptr), "l"(pol));
    return v;
}

// Exact integer <-> float conversions on the FP32/ALU pipes: for 0 <= d < 2^23,
// 2^23 + d is exactly representable and its low mantissa bits are d.
__device__ __forceinline__ float u23_to_float(uint32_t d)
{
    return __fsub_rn(__uint_as_float(0x4B000000u | d), 8388608.0f);
}

__device__ __forceinline__ uint32_t float_to_u23(float f)   // f integral, 0 <= f < 2^23
{
    return __float_as_uint(__fadd_rn(f, 8388608.0f)) & 0x7FFFFFu;
}

// ---------------------------------------------------------------------------
// (a) + (b): forward warp and z-buffer splat.
// One warp = one segment of kSplatSeg consecutive source pixels of one row
// of one active camera; lane l takes pixels l, l + 32, l + 64, ... so every
// warp-wide load and atomic touches 32 consecutive source pixels, whose
// targets are neighbours in the view (few L2 sectors per atomic).  Segments
// of a view are numbered camera-major over the active cameras:
// chunk_begin[a] .. chunk_begin[a+1).  Each CTA belongs to one view and
// stages its maps and frame table in shared memory.
// ---------------------------------------------------------------------------
template <bool kLayered>
__global__ void __launch_bounds__(kSplatThreads, 5)
k_warp_splat(const ViewDesc* __restrict__ views, const FrameRef* __restrict__ frames)
{
    __shared__ __align__(16) float s_M[kMaxCams][12];
    __shared__ __align__(16) FrameRef s_F[kMaxCams];
    __shared__ int s_cb[kMaxCams + 1];
    __shared__ int s_act[kMaxCams];
    constexpr int kWarps = kSplatThreads / 32;
    const ViewDesc* V = views + blockIdx.y;
    const int na = V->n_active;
    const int first = blockIdx.x * kWarps;
    if (first >= V->chunk_begin[na])
        return;                                   // uniform over the CTA
    for (int i = threadIdx.x; i < na * 12; i += kSplatThreads) {
        const int a = i / 12;
        s_M[a][i - a * 12] = V->geom[V->active[a]].M[i - a * 12];
    }
    for (int i = threadIdx.x; i < na; i += kSplatThreads) {
        s_act[i] = V->active[i];
        s_F[i] = frames[V->slot * V->n_cams + V->active[i]];
    }
    for (int i = threadIdx.x; i <= na; i += kSplatThreads)
        s_cb[i] = V->chunk_begin[i];
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int total = s_cb[na];
    const float zmin = V->z_min;
    const uint32_t dlo = V->d_lo, dspan = V->d_hi - V->d_lo;
    const uint32_t Wv = uint32_t(V->Wv);
    const float maxu = u23_to_float(Wv - 1), maxv = u23_to_float(uint32_t(V->Hv - 1));
    unsigned long long* __restrict__ keys = V->keys;
    unsigned long long* __restrict__ keys_bg = V->keys_bg;
    const uint64_t pol_stream = policy_evict_first();
    const uint64_t pol_keys = policy_evict_last();

    // persistent warps: segment seg, seg + stride, ... of this view
    for (int seg = first + int(threadIdx.x >> 5); seg < total; seg += gridDim.x * kWarps) {
        int a = 0;
        while (seg >= s_cb[a + 1])
            ++a;
        const int k = s_act[a];
        const FrameRef& F = s_F[a];
        const int spr = (F.W + kSplatSeg - 1) / kSplatSeg;
        const int local = seg - s_cb[a];
        const int v = local / spr;
        const int u0 = (local - v * spr) * kSplatSeg;
        const uint16_t* row = F.depth + size_t(v) * F.dpitch;

        uint32_t d[kSplatSeg / 32];
#pragma unroll
        for (int j = 0; j < kSplatSeg / 32; ++j) {
            const int u = u0 + lane + 32 * j;
            d[j] = u < F.W ? ld_stream_u16(row + u, pol_stream) : 0u;
        }
        // layered: a BG-signalled pixel takes its depth from the model and
        // splats into the BG layer (bit j of bgm)
        uint32_t bgm = 0;
        if (kLayered) {
            const uint16_t* brow = F.bg ? F.bg + size_t(v) * F.dpitch : nullptr;
#pragma unroll
            for (int j = 0; j < kSplatSeg / 32; ++j)
                if (d[j] == kDepthBg) {
                    d[j] = brow ? ld_stream_u16(brow + u0 + lane + 32 * j, pol_stream) : 0u;
                    bgm |= 1u << j;
                }
        }

        const float* m = s_M[a];
        const float m0 = m[0], m2 = m[2], m3 = m[3];
        const float m4 = m[4], m6 = m[6], m7 = m[7];
        const float m8 = m[8], m10 = m[10], m11 = m[11];
        const float fv = u23_to_float(uint32_t(v));
        // per-row products m1 v, m5 v, m9 v (the order stays ((m0 u + m1 v) + m2))
        const float r0 = __fmul_rn(m[1], fv), r1 = __fmul_rn(m[5], fv), r2 = __fmul_rn(m[9], fv);
        const unsigned long long khi = static_cast<unsigned long long>(k) << kSrcBits;
        const uint32_t src0 = uint32_t(v) * uint32_t(F.W) + uint32_t(u0 + lane);
        const float fu0 = u23_to_float(uint32_t(u0 + lane));

        // branch-free per point (only the atomic is predicated), so the eight
        // independent projections and divisions of a lane can interleave
#pragma unroll
        for (int j = 0; j < kSplatSeg / 32; ++j) {
            const uint32_t dd = d[j];
            const float fu = __fadd_rn(fu0, float(32 * j));  // exact: small integers
            const float z = u23_to_float(dd);
            const float a0 = __fadd_rn(__fadd_rn(__fmul_rn(m0, fu), r0), m2);
            const float a1 = __fadd_rn(__fadd_rn(__fmul_rn(m4, fu), r1), m6);
            const float a2 = __fadd_rn(__fadd_rn(__fmul_rn(m8, fu), r2), m10);
            const float X = __fadd_rn(__fmul_rn(a0, z), m3);
            const float Y = __fadd_rn(__fmul_rn(a1, z), m7);
            const float Z = __fadd_rn(__fmul_rn(a2, z), m11);
            const float tu = floorf(__fadd_rn(__fdiv_rn(X, Z), 0.5f));
            const float tv = floorf(__fadd_rn(__fdiv_rn(Y, Z), 0.5f));
            // the bounds test also rejects NaN and +-inf, as a finiteness test would
            // dd in [dlo, dhi] (dlo >= 1, so a code of 0 wraps above the span)
            const bool ok = dd - dlo <= dspan && Z > zmin && tu >= 0.0f && tu <= maxu && tv >= 0.0f &&
                            tv <= maxv;
            if (ok) {
                const uint32_t pix = float_to_u23(tv) * Wv + float_to_u23(tu);
                const unsigned long long key =
                    (static_cast<unsigned long long>(__float_as_uint(Z)) << 32) | khi |
                    static_cast<unsigned long long>(src0 + uint32_t(32 * j));
                unsigned long long* dst = (kLayered && ((bgm >> j) & 1u)) ? keys_bg : keys;
                red_min_key(dst + pix, key, pol_keys);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// (c) crack / outlier rule on the three staged key rows.  Pairs, in order:
// (left, right), (up, down), (up-left, down-right), (up-right, down-left).
// A pair is consistent when both keys are present and zmax <= (1+tau) zmin.
// An empty pixel takes min(a, b) of the first consistent pair; a present
// pixel takes it from the first consistent pair with z_p > (1+tau) zmax.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long nb_key(const unsigned long long* row, int Wv, int x)
{
    return (x < 0 || x >= Wv) ? kKeyEmpty : row[x];
}

// The rule for a pixel whose neighbour at (dy, dx) is get(dy, dx).
template <class Get>
__device__ __forceinline__ unsigned long long crack_rule_at(Get get, unsigned long long kp, float f1)
{
    const int ady[4] = {0, -1, -1, -1}, adx[4] = {-1, 0, -1, 1};
    const int bdy[4] = {0, 1, 1, 1}, bdx[4] = {1, 0, 1, -1};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const unsigned long long a = get(ady[q], adx[q]);
        const unsigned long long b = get(bdy[q], bdx[q]);
        if (a == kKeyEmpty || b == kKeyEmpty)
            continue;
        const float za = key_z(a), zb = key_z(b);
        const float zlo = za < zb ? za : zb;
        const float zhi = za < zb ? zb : za;
        if (!(zhi <= __fmul_rn(f1, zlo)))
            continue;
        if (kp == kKeyEmpty || key_z(kp) > __fmul_rn(f1, zhi))
            return a < b ? a : b;
    }
    return kp;
}

__device__ __forceinline__ unsigned long long crack_rule(const unsigned long long* up,
                                                         const unsigned long long* mid,
                                                         const unsigned long long* dn, int Wv, int x,
                                                         unsigned long long kp, float f1)
{
    const unsigned long long* rows[3] = {up, mid, dn};
    return crack_rule_at([&](int dy, int dx) { return nb_key(rows[dy + 1], Wv, x + dx); }, kp, f1);
}

// Layered form: the BG layer's crack filter as its own pass, read straight
// from the z-buffer (L1/L2), so the resolve stages one key ring only.
__global__ void __launch_bounds__(256) k_crack_bg(const ViewDesc* __restrict__ views)
{
    const ViewDesc* V = views + blockIdx.z;
    const int Wv = V->Wv, Hv = V->Hv;
    const int x = blockIdx.x * 256 + threadIdx.x, y = blockIdx.y;
    if (x >= Wv || y >= Hv)
        return;
    const unsigned long long* kb = V->keys_bg;
    const float f1 = __fadd_rn(1.0f, V->tau_crack);
    auto get = [&](int dy, int dx) {
        const int yy = y + dy, xx = x + dx;
        return (yy < 0 || yy >= Hv || xx < 0 || xx >= Wv) ? kKeyEmpty : __ldg(kb + size_t(yy) * Wv + xx);
    };
    V->keys_bgf[size_t(y) * Wv + x] = crack_rule_at(get, __ldg(kb + size_t(y) * Wv + x), f1);
}

__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc)
{
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gsrc) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ bool w_before(float wa, int ka, float wb, int kb)
{
    return wa > wb || (wa == wb && ka < kb);
}

__device__ __forceinline__ uint32_t blend_channel(float acc, float wsum)
{
    float v = floorf(__fadd_rn(__fdiv_rn(acc, wsum), 0.5f));
    v = v > 255.0f ? 255.0f : v;
    return uint32_t(v);
}

// Block-wide exclusive prefix max (over lower thread ids), -1 for thread 0.
__device__ __forceinline__ int block_excl_prefix_max(int v, int* s_scan)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc = max(inc, t);
    }
    if (lane == 31) s_scan[wid] = inc;
    __syncthreads();
    int acc = -1;
    for (int i = 0; i < wid; ++i) acc = max(acc, s_scan[i]);
    int excl = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) excl = -1;
    __syncthreads();
    return max(acc, excl);
}

// Block-wide exclusive suffix min (over higher thread ids), INT_MAX for the last.
__device__ __forceinline__ int block_excl_suffix_min(int v, int* s_scan)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_down_sync(0xffffffffu, inc, o);
        if (lane + o < 32) inc = min(inc, t);
    }
    if (lane == 0) s_scan[wid] = inc;
    __syncthreads();
    int acc = INT_MAX;
    for (int i = wid + 1; i < nw; ++i) acc = min(acc, s_scan[i]);
    int excl = __shfl_down_sync(0xffffffffu, inc, 1);
    if (lane == 31) excl = INT_MAX;
    __syncthreads();
    return min(acc, excl);
}

// ---------------------------------------------------------------------------
// (c) + (d) + (e).  One CTA walks a band of consecutive output rows of one
// view.  The key rows y-1, y, y+1 sit in a 4-row ring in shared memory; row
// y+2 is copied in asynchronously (cp.async) while row y is resolved.
// kTop3: also track the three largest contributing weights (only when that
// output is requested).
// ---------------------------------------------------------------------------
// Per-pixel angular weight of a camera whose centre in the view's frame is
// (cx, cy, cz), at the surface point (px, py, pz) at distance lb from the
// view's centre: 1 / (chord + 0.001) with chord = sqrt(2 (1 - cos)) of the
// angle at the point between the rays to the camera and to the view.
__device__ __forceinline__ float pixel_weight(float cx, float cy, float cz, float px, float py, float pz, float lb)
{
    const float ax = __fsub_rn(cx, px), ay = __fsub_rn(cy, py), az = __fsub_rn(cz, pz);
    const float la = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(ax, ax), __fmul_rn(ay, ay)), __fmul_rn(az, az)));
    const float dot = __fadd_rn(__fadd_rn(__fmul_rn(ax, px), __fmul_rn(ay, py)), __fmul_rn(az, pz));
    const float q = __fdiv_rn(dot, __fmul_rn(la, lb));
    float t = __fadd_rn(1.0f, q);
    t = t > 0.0f ? t : 0.0f;
    const float chord = __fsqrt_rn(__fadd_rn(t, t));
    return __fdiv_rn(1.0f, __fadd_rn(chord, 0.001f));
}

// kPixW: per-pixel angular weights (each contribution weighted by the angle
// at its surface point) instead of the view's per-camera weights.
// Three CTAs per SM (a 64-register cap for four cost more in the gathers'
// overlap than the extra warps gained).
template <bool kTop3, bool kLayered, bool kPixW>
__global__ void __launch_bounds__(kResolveThreads, 3)
k_resolve(const ViewDesc* __restrict__ views, const FrameRef* __restrict__ frames, int band)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const ViewDesc* V = views + blockIdx.y;
    const int Wv = V->Wv, Hv = V->Hv;
    const int y0 = blockIdx.x * band;
    if (y0 >= Hv)
        return;                                    // uniform over the CTA
    const int y1 = min(Hv, y0 + band);
    const int nc = V->n_cams, na = V->n_active;
    const SmemLayout L = resolve_layout(Wv, nc, kLayered);
    unsigned long long* s_ring = reinterpret_cast<unsigned long long*>(smem + L.ring);
    uint32_t* s_rgb = reinterpret_cast<uint32_t*>(smem + L.rgb);
    float* s_dep = reinterpret_cast<float*>(smem + L.dep);
    uint8_t* s_hole = smem + L.hole;
    float* s_geom = reinterpret_cast<float*>(smem + L.geom);
    float* s_rowt = reinterpret_cast<float*>(smem + L.rowt);
    FrameRef* s_fr = reinterpret_cast<FrameRef*>(smem + L.frames);
    int* s_act = reinterpret_cast<int*>(smem + L.active);
    int* s_pos = reinterpret_cast<int*>(smem + L.pos);        // camera -> position in s_act
    int* s_scan = reinterpret_cast<int*>(smem + L.scan);
    const int tid = threadIdx.x;
    constexpr int NT = kResolveThreads;
    const unsigned long long* keys = V->keys;

    const unsigned long long* keys_bgf = V->keys_bgf;
    auto ring_row = [&](int yy) { return s_ring + size_t((yy + kRing) & (kRing - 1)) * Wv; };
    auto fetch_row = [&](int yy) {           // async copy of key row yy (empty outside)
        unsigned long long* dst = ring_row(yy);
        if (yy >= 0 && yy < Hv) {
            const unsigned long long* src = keys + size_t(yy) * Wv;
            for (int x = tid; x < Wv; x += NT) cp_async8(dst + x, src + x);
        } else {
            for (int x = tid; x < Wv; x += NT) dst[x] = kKeyEmpty;
        }
    };
    fetch_row(y0 - 1);
    fetch_row(y0);
    fetch_row(y0 + 1);
    cp_async_commit();

    // per camera, 20 floats: N[0..11], w, 3 unused, W - 1, H - 1, 2 unused
    for (int i = tid; i < nc * kGeomFloats; i += NT) {
        const int k = i / kGeomFloats, j = i - k * kGeomFloats;
        float val = 0.0f;
        if (j < 12) val = V->geom[k].N[j];
        else if (j == 12) val = V->geom[k].w;
        else if (j < 16) val = V->geom[k].pad[j - 13];     // centre in the view's frame (per-pixel weights)
        else if (j == 16) val = float(frames[V->slot * nc + k].W - 1);
        else if (j == 17) val = float(frames[V->slot * nc + k].H - 1);
        s_geom[i] = val;
    }
    for (int i = tid; i < nc; i += NT)
        s_fr[i] = frames[V->slot * nc + i];
    for (int i = tid; i < na; i += NT)
        s_act[i] = V->active[i];
    for (int k = tid; k < kMaxCams; k += NT) {     // 0 for inactive cameras keeps every index in range
        int p = 0;
        for (int i = 0; i < na; ++i)
            if (V->active[i] == k) p = i;
        s_pos[k] = p;
    }

    const bool crack = (V->flags & kFlagCrack) != 0;
    const bool fill = (V->flags & kFlagFill) != 0;
    const float f1 = __fadd_rn(1.0f, V->tau_crack);
    const float tau_vis = V->tau_vis, zmin = V->z_min;
    const uint32_t dlo = V->d_lo, dspan = V->d_hi - V->d_lo;
    float* __restrict__ top3 = V->out_top3;
    unsigned long long* __restrict__ okeys = V->out_keys;
    const float4* g4 = reinterpret_cast<const float4*>(s_geom);
    __syncthreads();                          // s_geom, s_fr, s_act staged

    for (int y = y0; y < y1; ++y) {
        // the ring slot of row y+2 held row y-2, last read before the end of
        // the previous iteration
        if (y + 1 < y1)
            fetch_row(y + 2);
        cp_async_commit();
        // per-row products N1 y, N5 y, N9 y (the order stays ((N0 x + N1 y) + N2))
        const float fy = u23_to_float(uint32_t(y));
        for (int i = tid; i < nc * 3; i += NT) {
            const int k = i / 3, j = i - k * 3;
            s_rowt[4 * k + j] = __fmul_rn(s_geom[kGeomFloats * k + 1 + 4 * j], fy);
        }
        cp_async_wait<1>();                   // rows y-1 .. y+1 have landed
        __syncthreads();

        const unsigned long long* rU = ring_row(y - 1);
        const unsigned long long* rC = ring_row(y);
        const unsigned long long* rD = ring_row(y + 1);
        const size_t rowbase = size_t(y) * Wv;
        bool any_hole = false;
        for (int x = tid; x < Wv; x += NT) {
            const unsigned long long kp = rC[x];
            unsigned long long key = crack ? crack_rule(rU, rC, rD, Wv, x, kp, f1) : kp;
            // layered: the FG layer is stacked over the BG layer, so the BG
            // layer is resolved only where the filtered FG layer is empty
            bool bg_layer = false;
            if (kLayered && key == kKeyEmpty) {
                key = keys_bgf[rowbase + x];          // filtered by k_crack_bg (raw without the filter)
                bg_layer = true;
            }
            if (okeys) okeys[rowbase + x] = key;
            if (key == kKeyEmpty) {
                s_rgb[x] = 0u;
                s_dep[x] = 0.0f;
                s_hole[x] = 1;
                any_hole = true;
                if (kTop3 && top3) {
                    top3[3 * (rowbase + x) + 0] = 0.0f;
                    top3[3 * (rowbase + x) + 1] = 0.0f;
                    top3[3 * (rowbase + x) + 2] = 0.0f;
                }
                continue;
            }
            const float Z = key_z(key);
            const int w = int((key >> kSrcBits) & 63u);
            const uint32_t s = uint32_t(key & ((1u << kSrcBits) - 1u));
            const FrameRef& Fw = s_fr[w];
            const uint32_t sv = s / uint32_t(Fw.W);
            const uint32_t su = s - sv * uint32_t(Fw.W);
            const uint32_t cw = __ldg(Fw.rgba + sv * uint32_t(Fw.rpitch) + su);
            const float fx = u23_to_float(uint32_t(x));
            // per-pixel weights: the surface point in the view's frame
            float px = 0.0f, py = 0.0f, lb = 0.0f;
            if (kPixW) {
                px = __fmul_rn(__fmul_rn(__fsub_rn(fx, V->vk[0]), V->vk[2]), Z);
                py = __fmul_rn(__fmul_rn(__fsub_rn(fy, V->vk[1]), V->vk[3]), Z);
                lb = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(px, px), __fmul_rn(py, py)), __fmul_rn(Z, Z)));
            }
            auto weight_of = [&](int k) {
                if (!kPixW) return s_geom[kGeomFloats * k + 12];
                const float* gk = s_geom + kGeomFloats * k;
                return pixel_weight(gk[13], gk[14], gk[15], px, py, Z, lb);
            };
            const float ww = weight_of(w);
            float acc0 = __fmul_rn(ww, u23_to_float(cw & 255u));
            float acc1 = __fmul_rn(ww, u23_to_float((cw >> 8) & 255u));
            float acc2 = __fmul_rn(ww, u23_to_float((cw >> 16) & 255u));
            float wsum = ww;
            float t0 = ww, t1 = -1.0f, t2 = -1.0f;
            int k0 = w, k1 = INT_MAX, k2 = INT_MAX;
            // the other active cameras (the winner is always active: only
            // active cameras splat), in ascending order, in groups of four:
            // project all four and issue their depth and colour gathers
            // before any is consumed, then accumulate in order
            const int pw = s_pos[w], nother = na - 1;
            for (int g0 = 0; g0 < nother; g0 += 4) {
                uint32_t dk[4], ck[4], di[4];
                float zk[4];
                int kk[4];
                bool ok[4];
                // branch-free projection of the group (only the gathers are
                // predicated), so the four chains can interleave
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int ii = min(g0 + j, nother - 1);
                    const int k = s_act[ii + (ii >= pw ? 1 : 0)];
                    kk[j] = k;
                    const float4 A = g4[5 * k + 0], Bq = g4[5 * k + 1], Cq = g4[5 * k + 2],
                                 Eq = g4[5 * k + 4];
                    const float4 Rt = reinterpret_cast<const float4*>(s_rowt)[k];
                    const float a0 = __fadd_rn(__fadd_rn(__fmul_rn(A.x, fx), Rt.x), A.z);
                    const float a1 = __fadd_rn(__fadd_rn(__fmul_rn(Bq.x, fx), Rt.y), Bq.z);
                    const float a2 = __fadd_rn(__fadd_rn(__fmul_rn(Cq.x, fx), Rt.z), Cq.z);
                    const float Xk = __fadd_rn(__fmul_rn(a0, Z), A.w);
                    const float Yk = __fadd_rn(__fmul_rn(a1, Z), Bq.w);
                    const float Zk = __fadd_rn(__fmul_rn(a2, Z), Cq.w);
                    const float tu = floorf(__fadd_rn(__fdiv_rn(Xk, Zk), 0.5f));
                    const float tv = floorf(__fadd_rn(__fdiv_rn(Yk, Zk), 0.5f));
                    // the bounds test also rejects NaN and +-inf, as a finiteness test would
                    ok[j] = g0 + j < nother && Zk > zmin && tu >= 0.0f && tu <= Eq.x &&
                            tv >= 0.0f && tv <= Eq.y;
                    zk[j] = Zk;
                    dk[j] = 0u;
                    ck[j] = 0u;
                    di[j] = 0u;
                    if (ok[j]) {
                        const FrameRef& Fk = s_fr[k];
                        const uint32_t uk = float_to_u23(tu), vk = float_to_u23(tv);
                        di[j] = vk * uint32_t(Fk.dpitch) + uk;
                        dk[j] = __ldg(Fk.depth + di[j]);
                        ck[j] = __ldg(Fk.rgba + vk * uint32_t(Fk.rpitch) + uk);
                    }
                }
                // the BG layer's depth in camera k: its model where camera k
                // signals BG, none elsewhere (there camera k sees FG)
                if (kLayered && bg_layer) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if (!ok[j])
                            continue;
                        const FrameRef& Fk = s_fr[kk[j]];
                        dk[j] = (dk[j] == kDepthBg && Fk.bg) ? uint32_t(__ldg(Fk.bg + di[j])) : 0u;
                    }
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (!ok[j])
                        continue;
                    if (dk[j] - dlo > dspan)         // outside [dlo, dhi]; 0 wraps above
                        continue;
                    const float diff = fabsf(__fsub_rn(u23_to_float(dk[j]), zk[j]));
                    if (!(diff <= __fmul_rn(tau_vis, zk[j])))
                        continue;
                    const int k = kk[j];
                    const float wk = weight_of(k);
                    const uint32_t c = ck[j];
                    acc0 = __fadd_rn(acc0, __fmul_rn(wk, u23_to_float(c & 255u)));
                    acc1 = __fadd_rn(acc1, __fmul_rn(wk, u23_to_float((c >> 8) & 255u)));
                    acc2 = __fadd_rn(acc2, __fmul_rn(wk, u23_to_float((c >> 16) & 255u)));
                    wsum = __fadd_rn(wsum, wk);
                    if (kTop3) {
                        if (w_before(wk, k, t0, k0)) {
                            t2 = t1; k2 = k1; t1 = t0; k1 = k0; t0 = wk; k0 = k;
                        } else if (w_before(wk, k, t1, k1)) {
                            t2 = t1; k2 = k1; t1 = wk; k1 = k;
                        } else if (w_before(wk, k, t2, k2)) {
                            t2 = wk; k2 = k;
                        }
                    }
                }
            }
            s_rgb[x] = blend_channel(acc0, wsum) | (blend_channel(acc1, wsum) << 8) | (blend_channel(acc2, wsum) << 16);
            s_dep[x] = Z;
            s_hole[x] = 0;
            if (kTop3 && top3) {
                top3[3 * (rowbase + x) + 0] = __fdiv_rn(t0, wsum);
                top3[3 * (rowbase + x) + 1] = t1 >= 0.0f ? __fdiv_rn(t1, wsum) : 0.0f;
                top3[3 * (rowbase + x) + 2] = t2 >= 0.0f ? __fdiv_rn(t2, wsum) : 0.0f;
            }
        }
        // (e) hole fill: nearest non-hole left / right, the deeper one wins
        const bool row_has_hole = __syncthreads_or(any_hole) != 0;
        if (fill && row_has_hole) {
            // the ring slot of row y - 1: every thread has finished reading
            // it (the barrier above), and row y + 3 lands in it only after
            // the barrier that ends this row
            int16_t* s_left = reinterpret_cast<int16_t*>(const_cast<unsigned long long*>(rU));
            int16_t* s_right = s_left + Wv;
            const int seg = (Wv + NT - 1) / NT;
            const int x0 = min(tid * seg, Wv), x1 = min(x0 + seg, Wv);
            int last = -1;
            for (int x = x0; x < x1; ++x)
                if (!s_hole[x]) last = x;
            int run = block_excl_prefix_max(last, s_scan);
            for (int x = x0; x < x1; ++x) {
                if (!s_hole[x]) run = x;
                s_left[x] = int16_t(run);
            }
            int first = INT_MAX;
            for (int x = x1 - 1; x >= x0; --x)
                if (!s_hole[x]) first = x;
            run = block_excl_suffix_min(first, s_scan);
            for (int x = x1 - 1; x >= x0; --x) {
                if (!s_hole[x]) run = x;
                s_right[x] = int16_t(run == INT_MAX ? -1 : run);
            }
            __syncthreads();
            for (int x = tid; x < Wv; x += NT) {
                if (!s_hole[x])
                    continue;
                const int l = s_left[x], r = s_right[x];
                if (l < 0 && r < 0)
                    continue;
                const int src = l < 0 ? r : (r < 0 ? l : (s_dep[r] > s_dep[l] ? r : l));
                s_rgb[x] = s_rgb[src];
                s_dep[x] = s_dep[src];
            }
            __syncthreads();
        }

        uint8_t* orow = V->out_rgb + size_t(y) * size_t(V->out_pitch);
        const int nbytes = 3 * Wv;
        int done = 0;
        if ((reinterpret_cast<uintptr_t>(orow) & 3u) == 0) {
            const int nw = nbytes >> 2;
            uint32_t* o32 = reinterpret_cast<uint32_t*>(orow);
            for (int i = tid; i < nw; i += NT) {
                uint32_t word = 0;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int byte = 4 * i + b;
                    const int x = byte / 3;
                    word |= ((s_rgb[x] >> (8 * (byte - 3 * x))) & 255u) << (8 * b);
                }
                o32[i] = word;
            }
            done = nw << 2;
        }
        for (int i = done + tid; i < nbytes; i += NT) {
            const int x = i / 3;
            orow[i] = uint8_t(s_rgb[x] >> (8 * (i - 3 * x)));
        }
        if (V->out_depth)
            for (int x = tid; x < Wv; x += NT) V->out_depth[rowbase + x] = s_dep[x];
        if (V->out_hole)
            for (int x = tid; x < Wv; x += NT) V->out_hole[rowbase + x] = s_hole[x];
        __syncthreads();        // s_rgb / s_dep / s_hole / s_rowt are rewritten next row
    }
}

// ---------------------------------------------------------------------------
// upload: RGB8 rows -> RGBA8 rows (R | G << 8 | B << 16)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_pack_rgba(const uint8_t* __restrict__ rgb, size_t pitch,
                                                   uint32_t* __restrict__ rgba, int rpitch, int W)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W)
        return;
    const uint8_t* p = rgb + size_t(y) * pitch + 3 * size_t(x);
    rgba[size_t(y) * rpitch + x] = uint32_t(p[0]) | (uint32_t(p[1]) << 8) | (uint32_t(p[2]) << 16);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
size_t resolve_smem_bytes(int max_w, int n_cams, bool layered)
{
    return resolve_layout(max_w, n_cams, layered).total;
}

cudaError_t launch_clear_keys(unsigned long long* keys, size_t n, cudaStream_t stream)
{
    if (n == 0) return cudaSuccess;
    size_t blocks = ((n >> 1) + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_clear_keys<<<unsigned(blocks), 256, 0, stream>>>(keys, n);
    return cudaGetLastError();
}

cudaError_t launch_warp_splat(const ViewDesc* views, int n_views, int max_chunks,
                              const FrameRef* frames, cudaStream_t stream, bool layered)
{
    if (n_views <= 0 || max_chunks <= 0) return cudaSuccess;
    constexpr int kWarps = kSplatThreads / 32;      // one warp per segment at a time
    // persistent warps: about two resident waves over all views of the batch
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int want = (2 * 5 * sms + n_views - 1) / n_views;
    const int need = (max_chunks + kWarps - 1) / kWarps;
    const int bx = need < want ? need : (want < 1 ? 1 : want);
    dim3 grid(static_cast<unsigned>(bx), static_cast<unsigned>(n_views));
    if (layered)
        k_warp_splat<true><<<grid, kSplatThreads, 0, stream>>>(views, frames);
    else
        k_warp_splat<false><<<grid, kSplatThreads, 0, stream>>>(views, frames);
    return cudaGetLastError();
}

cudaError_t launch_crack_bg(const ViewDesc* views, int n_views, int max_h, int max_w, cudaStream_t stream)
{
    if (n_views <= 0 || max_h <= 0 || max_w <= 0) return cudaSuccess;
    dim3 grid(static_cast<unsigned>((max_w + 255) / 256), static_cast<unsigned>(max_h),
              static_cast<unsigned>(n_views));
    k_crack_bg<<<grid, 256, 0, stream>>>(views);
    return cudaGetLastError();
}

cudaError_t launch_resolve(const ViewDesc* views, int n_views, int max_h, int max_w, int n_cams,
                           bool top3, const FrameRef* frames, cudaStream_t stream, bool layered,
                           bool pixel_weights)
{
    if (n_views <= 0 || max_h <= 0) return cudaSuccess;
    // the layout grows with the width and the camera count, so the widest
    // view of the batch bounds every CTA's shared memory
    const size_t smem = resolve_smem_bytes(max_w, n_cams, layered);
    const int band = kResolveBand;
    dim3 grid(static_cast<unsigned>((max_h + band - 1) / band), static_cast<unsigned>(n_views));
    auto go = [&](auto kernel) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        kernel<<<grid, kResolveThreads, smem, stream>>>(views, frames, band);
        return cudaGetLastError();
    };
    if (pixel_weights) {
        if (layered) return top3 ? go(k_resolve<true, true, true>) : go(k_resolve<false, true, true>);
        return top3 ? go(k_resolve<true, false, true>) : go(k_resolve<false, false, true>);
    }
    if (layered) return top3 ? go(k_resolve<true, true, false>) : go(k_resolve<false, true, false>);
    return top3 ? go(k_resolve<true, false, false>) : go(k_resolve<false, false, false>);
}

cudaError_t launch_pack_rgba(const uint8_t* rgb, size_t rgb_pitch, uint32_t* rgba, int rpitch,
                             int W, int H, cudaStream_t stream)
{
    if (W <= 0 || H <= 0) return cudaSuccess;
    dim3 grid(static_cast<unsigned>((W + 255) / 256), static_cast<unsigned>(H));
    k_pack_rgba<<<grid, 256, 0, stream>>>(rgb, rgb_pitch, rgba, rpitch, W);
    return cudaGetLastError();
}

}  // namespace fvv
