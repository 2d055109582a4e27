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
//                  (e) row hole fill, fused: one CTA per band of output rows
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
#include <algorithm>
#include <climits>
#include <cstdlib>

#include "fvv_internal.h"

namespace fvv {

namespace {

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

constexpr int kRing = 4;          // key rows kept in shared memory (3 in use + 1 in flight)
constexpr int kGroup = 8;         // back-projections issued together per pixel

// Per active camera of a view, staged in the resolve kernel's shared memory
// and indexed by the camera's position in the view's active list.  The first
// 80 bytes are what every back-projection reads.
struct alignas(16) RCam {
    float4 gx;                 // N0, N2, N3, N1 y   (the row product, rewritten per row)
    float4 gy;                 // N4, N6, N7, N5 y
    float4 gz;                 // N8, N10, N11, N9 y
    const uint16_t* depth;     // the camera's frame in the view's slot
    const uint32_t* rgba;
    int32_t dpitch, rpitch;    // elements
    uint32_t maxu, maxv;       // W - 1, H - 1
    float w;                   // per-view blend weight
    int32_t k;                 // camera index
    uint32_t magic, shift;     // s / W == (s * magic) >> shift for every s < 2^26
    const uint16_t* bg;        // layered: the static BG depth model, or NULL
    float unused[2];
    float4 rowc;               // N1, N5, N9 (coefficients of the row products)
    float4 cen;                // the camera's centre in the view's frame (per-pixel weights)
};
static_assert(sizeof(RCam) == 144, "RCam layout");

struct SmemLayout {
    size_t ring, rgb, dep, hole, cams, pos, scan, total;
};

// Key rows carry one EMPTY sentinel on each side (Wv + 2 entries), so the
// crack filter reads x - 1 and x + 1 without bounds tests.
__host__ __device__ inline size_t ring_pitch(int W) { return size_t(W) + 2; }

__host__ __device__ inline SmemLayout resolve_layout(int W, int n_cams, bool layered)
{
    SmemLayout L;
    size_t o = 0;
    (void)layered;                // the layered form reads its BG keys from the filtered z-buffer
    L.ring = o;   o = align16(o + size_t(kRing) * ring_pitch(W) * sizeof(unsigned long long));
    L.rgb = o;    o = align16(o + size_t(W) * 4);
    L.dep = o;    o = align16(o + size_t(W) * 4);
    L.hole = o;   o = align16(o + size_t(W));
    // (the hole fill's nearest-left / nearest-right indices live in the key
    // ring's slot of the row above, which no pixel reads any more by then)
    L.cams = o;   o = align16(o + size_t(n_cams) * sizeof(RCam));
    L.pos = o;    o = align16(o + size_t(kMaxCams) * sizeof(int));
    L.scan = o;   o = align16(o + 64 * sizeof(int));
    L.total = o;
    return L;
}

__device__ __forceinline__ float key_z(unsigned long long k)
{
    return __uint_as_float(static_cast<uint32_t>(k >> 32));
}

__device__ __forceinline__ uint32_t key_zbits(unsigned long long k)
{
    return static_cast<uint32_t>(k >> 32);
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

// streaming loads (read once)
__device__ __forceinline__ uint32_t ld_stream_u16(const uint16_t* ptr, uint64_t pol)
{
    unsigned short v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u16 %0, [%1], %2;"
                 : "=h"(v) : "l"(ptr), "l"(pol));
    return v;
}

__device__ __forceinline__ uint4 ld_stream_v4(const void* ptr, uint64_t pol)
{
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(ptr), "l"(pol));
    return v;
}

// Loads of frame data.  kCoh = false: the read-only (non-coherent) paths,
// for kernels during whose life the frames do not change.  kCoh = true
// (the persistent serving kernel, which outlives frame uploads): weak loads,
// which a gpu-scope acquire fence makes observe the latest writes.
template <bool kCoh, class T>
__device__ __forceinline__ T ld_frame(const T* p)
{
    if constexpr (kCoh) return *p;
    else return __ldg(p);
}

template <bool kCoh>
__device__ __forceinline__ uint32_t ld_depth_stream(const uint16_t* ptr, uint64_t pol)
{
    if constexpr (kCoh) return *ptr;
    else return ld_stream_u16(ptr, pol);
}

// Exact integer -> float conversion on the FP32/ALU pipes: for 0 <= d < 2^23,
// 2^23 + d is exactly representable and its low mantissa bits are d.
__device__ __forceinline__ float u23_to_float(uint32_t d)
{
    return __fsub_rn(__uint_as_float(0x4B000000u | d), 8388608.0f);
}

// R3's target pixel of a projected point: u' = X / Z and v' = Y / Z by
// correctly rounded division, then floor(u' + 0.5) (ties up), and the bounds
// test 0 <= t <= max as one unsigned compare per axis.  The float -> int
// floor saturates, so +-inf and out-of-range values fail the test as in the
// FP32 form; Z > z_min >= 0 (validated on the host) and a finite X, Y rule
// out NaN.
__device__ __forceinline__ bool target_pixel(float X, float Y, float Z, uint32_t maxu, uint32_t maxv,
                                             uint32_t& ui, uint32_t& vi)
{
    ui = static_cast<uint32_t>(__float2int_rd(__fadd_rn(__fdiv_rn(X, Z), 0.5f)));
    vi = static_cast<uint32_t>(__float2int_rd(__fadd_rn(__fdiv_rn(Y, Z), 0.5f)));
    return ui <= maxu && vi <= maxv;
}

// ---------------------------------------------------------------------------
// (a) + (b): forward warp and z-buffer splat.
// One warp = one segment of kSplatSeg consecutive source pixels of one row
// of one active camera.  kVec = false: lane l takes pixels l, l + 32, ...
// (2-byte loads), so every warp-wide atomic touches 32 consecutive source
// pixels, whose targets are neighbours in the view (few L2 sectors per
// atomic).  kVec = true: lane l takes the 8 consecutive pixels 8l .. 8l+7
// with one 16-byte load.  Segments of a view are numbered camera-major over
// the active cameras: chunk_begin[a] .. chunk_begin[a+1).  Each CTA belongs
// to one view and stages its maps and frame table in shared memory.
// ---------------------------------------------------------------------------
// The work of one CTA (bx, by) of a grid of gdx x (views) CTAs; the kernel
// below is its one-launch form, the persistent serving kernel calls it for
// virtual CTAs in turn (kCoh: coherent frame loads, see ld_frame).
template <bool kLayered, bool kVec, bool kCoh>
__device__ __forceinline__ void splat_cta(const ViewDesc* __restrict__ views, const FrameRef* __restrict__ frames,
                                          int bx, int by, int gdx)
{
    // per active camera: (m0, m2, m3, m1), (m4, m6, m7, m5), (m8, m10, m11, m9)
    __shared__ __align__(16) float4 s_M[kMaxCams][3];
    __shared__ __align__(16) FrameRef s_F[kMaxCams];
    __shared__ int s_cb[kMaxCams + 1];
    __shared__ int s_act[kMaxCams];
    __shared__ uint2 s_div[kMaxCams];              // segment -> row: (magic, shift) of segments per row
    constexpr int kWarps = kSplatThreads / 32;
    constexpr int kPer = kSplatSeg / 32;           // pixels per lane per segment
    static_assert(kPer == 8, "a 16-byte load holds 8 depth codes");
    if (kCoh) __syncthreads();                     // the previous virtual CTA's reads of the staging are done
    const ViewDesc* V = views + by;
    const int na = V->n_active;
    const int first = bx * kWarps;
    if (first >= V->chunk_begin[na])
        return;                                   // uniform over the CTA
    for (int i = threadIdx.x; i < na * 3; i += kSplatThreads) {
        const int a = i / 3, r = i - a * 3;
        const float* m = V->geom[V->active[a]].M + 4 * r;
        s_M[a][r] = make_float4(m[0], m[2], m[3], m[1]);
    }
    for (int i = threadIdx.x; i < na; i += kSplatThreads) {
        s_act[i] = V->active[i];
        const FrameRef F = frames[V->slot * V->n_cams + V->active[i]];
        s_F[i] = F;
        // local / spr for local < 2^26 as (local * magic) >> shift, with
        // shift = 26 + ceil(log2 spr) and magic = ceil(2^shift / spr): the
        // excess local * e / 2^shift stays below 1 / spr
        const uint32_t spr = uint32_t((F.W + kSplatSeg - 1) / kSplatSeg);
        const uint32_t lg = spr > 1 ? 32u - uint32_t(__clz(spr - 1)) : 0u;
        s_div[i] = make_uint2(uint32_t(((1ull << (26u + lg)) + spr - 1) / spr), 26u + lg);
    }
    for (int i = threadIdx.x; i <= na; i += kSplatThreads)
        s_cb[i] = V->chunk_begin[i];
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int total = s_cb[na];
    const float zmin = V->z_min;
    const uint32_t dlo = V->d_lo, dspan = V->d_hi - V->d_lo;
    const uint32_t Wv = uint32_t(V->Wv);
    const uint32_t maxu = Wv - 1, maxv = uint32_t(V->Hv - 1);
    unsigned long long* __restrict__ keys = V->keys;
    unsigned long long* __restrict__ keys_bg = V->keys_bg;
    const uint64_t pol_stream = policy_evict_first();
    const uint64_t pol_keys = policy_evict_last();

    // persistent warps: segment seg, seg + stride, ... of this view; the
    // segments grow, so the camera search resumes where it stopped
    int a = 0;
    for (int seg = first + int(threadIdx.x >> 5); seg < total; seg += gdx * kWarps) {
        while (seg >= s_cb[a + 1])
            ++a;
        const int k = s_act[a];
        const FrameRef& F = s_F[a];
        const int spr = (F.W + kSplatSeg - 1) / kSplatSeg;
        const uint32_t local = uint32_t(seg - s_cb[a]);
        const uint2 dv = s_div[a];
        const int v = int((static_cast<unsigned long long>(local) * dv.x) >> dv.y);
        const int u0 = (int(local) - v * spr) * kSplatSeg;
        const uint16_t* row = F.depth + size_t(v) * F.dpitch;
        // the lane's first pixel and the step between its pixels
        const int ub = u0 + (kVec ? kPer * lane : lane);
        constexpr int kStep = kVec ? 1 : 32;

        uint32_t d[kPer];
        // 16-byte loads need 16-byte aligned rows; a vector lies wholly
        // inside or wholly past the row's pitch (pitch and ub multiples of 8)
        if (kVec && !kCoh && (F.dpitch & 7) == 0 && (reinterpret_cast<uintptr_t>(F.depth) & 15u) == 0) {
            uint4 q = make_uint4(0u, 0u, 0u, 0u);
            if (ub < F.dpitch)
                q = ld_stream_v4(row + ub, pol_stream);
            d[0] = q.x & 0xFFFFu; d[1] = q.x >> 16; d[2] = q.y & 0xFFFFu; d[3] = q.y >> 16;
            d[4] = q.z & 0xFFFFu; d[5] = q.z >> 16; d[6] = q.w & 0xFFFFu; d[7] = q.w >> 16;
#pragma unroll
            for (int j = 0; j < kPer; ++j)
                if (ub + j >= F.W) d[j] = 0u;
        } else {
#pragma unroll
            for (int j = 0; j < kPer; ++j) {
                const int u = ub + kStep * j;
                d[j] = u < F.W ? ld_depth_stream<kCoh>(row + u, pol_stream) : 0u;
            }
        }
        // layered: a BG-signalled pixel takes its depth from the model and
        // splats into the BG layer (bit j of bgm)
        uint32_t bgm = 0;
        if (kLayered) {
            const uint16_t* brow = F.bg ? F.bg + size_t(v) * F.dpitch : nullptr;
#pragma unroll
            for (int j = 0; j < kPer; ++j)
                if (d[j] == kDepthBg) {
                    d[j] = brow ? ld_depth_stream<kCoh>(brow + ub + kStep * j, pol_stream) : 0u;
                    bgm |= 1u << j;
                }
        }

        const float4 Mx = s_M[a][0], My = s_M[a][1], Mz = s_M[a][2];
        const float fv = u23_to_float(uint32_t(v));
        // per-row products m1 v, m5 v, m9 v (the order stays ((m0 u + m1 v) + m2))
        const float rx = __fmul_rn(Mx.w, fv), ry = __fmul_rn(My.w, fv), rz = __fmul_rn(Mz.w, fv);
        const unsigned long long khi = static_cast<unsigned long long>(k) << kSrcBits;
        const uint32_t src0 = uint32_t(v) * uint32_t(F.W) + uint32_t(ub);
        const float fu0 = u23_to_float(uint32_t(ub));

        // branch-free per point (only the atomic is predicated), so the eight
        // independent projections and divisions of a lane can interleave
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const uint32_t dd = d[j];
            const float fu = __fadd_rn(fu0, float(kStep * j));   // exact: small integers
            const float z = u23_to_float(dd);
            const float a0 = __fadd_rn(__fadd_rn(__fmul_rn(Mx.x, fu), rx), Mx.y);
            const float a1 = __fadd_rn(__fadd_rn(__fmul_rn(My.x, fu), ry), My.y);
            const float a2 = __fadd_rn(__fadd_rn(__fmul_rn(Mz.x, fu), rz), Mz.y);
            const float X = __fadd_rn(__fmul_rn(a0, z), Mx.z);
            const float Y = __fadd_rn(__fmul_rn(a1, z), My.z);
            const float Z = __fadd_rn(__fmul_rn(a2, z), Mz.z);
            uint32_t tu, tv;
            const bool hit = target_pixel(X, Y, Z, maxu, maxv, tu, tv);
            // dd in [dlo, dhi] (dlo >= 1, so a code of 0 wraps above the span)
            if (dd - dlo <= dspan && Z > zmin && hit) {
                const unsigned long long key =
                    (static_cast<unsigned long long>(__float_as_uint(Z)) << 32) | khi |
                    static_cast<unsigned long long>(src0 + uint32_t(kStep * j));
                unsigned long long* dst = (kLayered && ((bgm >> j) & 1u)) ? keys_bg : keys;
                red_min_key(dst + (tv * Wv + tu), key, pol_keys);
            }
        }
    }
}

template <bool kLayered, bool kVec>
__global__ void __launch_bounds__(kSplatThreads, 5)
k_warp_splat(const ViewDesc* __restrict__ views, const FrameRef* __restrict__ frames)
{
    splat_cta<kLayered, kVec, false>(views, frames, int(blockIdx.x), int(blockIdx.y), int(gridDim.x));
}

// ---------------------------------------------------------------------------
// (c) crack / outlier rule on the three staged key rows.  Pairs, in order:
// (left, right), (up, down), (up-left, down-right), (up-right, down-left).
// A pair is consistent when both keys are present and zmax <= (1+tau) zmin.
// An empty pixel takes min(a, b) of the first consistent pair; a present
// pixel takes it from the first consistent pair with z_p > (1+tau) zmax.
// ---------------------------------------------------------------------------
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

// The rule on padded shared-memory rows (index -1 and Wv hold EMPTY).  A
// present pixel no deeper than (1+tau) times its nearest present neighbour
// keeps its key without the pair walk: every consistent pair's far depth is
// at least that neighbour's, and the rounded product is monotone, so no pair
// can satisfy z_p > (1+tau) zmax.  With no present neighbour no pair is
// consistent either.
__device__ __forceinline__ unsigned long long crack_rule_rows(const unsigned long long* up,
                                                              const unsigned long long* mid,
                                                              const unsigned long long* dn, int x,
                                                              unsigned long long kp, float f1)
{
    const unsigned long long n[3][3] = {{up[x - 1], up[x], up[x + 1]},
                                        {mid[x - 1], kp, mid[x + 1]},
                                        {dn[x - 1], dn[x], dn[x + 1]}};
    if (kp != kKeyEmpty) {
        // positive depths order like their bit patterns; EMPTY's are the largest
        const uint32_t zb =
            min(min(min(key_zbits(n[0][0]), key_zbits(n[0][1])), min(key_zbits(n[0][2]), key_zbits(n[1][0]))),
                min(min(key_zbits(n[1][2]), key_zbits(n[2][0])), min(key_zbits(n[2][1]), key_zbits(n[2][2]))));
        if (zb == 0xFFFFFFFFu || !(key_z(kp) > __fmul_rn(f1, __uint_as_float(zb))))
            return kp;
    }
    return crack_rule_at([&](int dy, int dx) { return n[dy + 1][dx + 1]; }, kp, f1);
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

// ---------------------------------------------------------------------------
// (c) + (d) + (e).  One CTA walks a band of consecutive output rows of one
// view (two rows, or one for small batches), launched view after view so
// that the resident CTAs share one view's frames in L2.  The key rows y-1, y, y+1 sit in a 4-row ring in shared
// memory; row y+2 is copied in asynchronously (cp.async) while row y is
// resolved.  Each thread resolves the pixels x = tid, tid + 256, ... of a
// row: the winner's colour, then the other active cameras in ascending
// order, in groups of eight (kGroup) whose projections and gathers are
// issued before any is consumed.
// kTop3: also track the three largest contributing weights (only when that
// output is requested).  kPixW: per-pixel angular weights (each contribution
// weighted by the angle at its surface point) instead of the view's
// per-camera weights.
// ---------------------------------------------------------------------------
template <bool kTop3, bool kLayered, bool kPixW, bool kCoh>
__device__ __forceinline__ void resolve_cta(const ViewDesc* __restrict__ views, const FrameRef* __restrict__ frames,
                                            int band, int bx, int by, unsigned char* smem)
{
    if (kCoh) __syncthreads();                     // the previous virtual CTA is done with the shared memory
    const ViewDesc* V = views + by;
    const int Wv = V->Wv, Hv = V->Hv;
    const int y0 = bx * band;
    if (y0 >= Hv)
        return;                                    // uniform over the CTA
    const int y1 = min(Hv, y0 + band);
    if (!kLayered && V->keys_next) {
        // the next batch's z-buffer rows of this band, emptied while the key
        // rows below are in flight (kept in L2 for that batch's splat)
        const uint64_t pol = policy_evict_last();
        unsigned long long* kn = V->keys_next + size_t(y0) * Wv;
        const int m = (y1 - y0) * Wv;
        for (int i = threadIdx.x; i < m; i += kResolveThreads)
            asm volatile("st.global.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(kn + i), "l"(kKeyEmpty), "l"(pol)
                         : "memory");
    }
    const int nc = V->n_cams, na = V->n_active;
    const SmemLayout L = resolve_layout(Wv, nc, kLayered);
    const size_t RP = ring_pitch(Wv);
    unsigned long long* s_ring = reinterpret_cast<unsigned long long*>(smem + L.ring);
    uint32_t* s_rgb = reinterpret_cast<uint32_t*>(smem + L.rgb);
    float* s_dep = reinterpret_cast<float*>(smem + L.dep);
    uint8_t* s_hole = smem + L.hole;
    RCam* s_cam = reinterpret_cast<RCam*>(smem + L.cams);
    int* s_pos = reinterpret_cast<int*>(smem + L.pos);        // camera -> position in the active list
    int* s_scan = reinterpret_cast<int*>(smem + L.scan);
    const int tid = threadIdx.x;
    constexpr int NT = kResolveThreads;
    const unsigned long long* keys = V->keys;

    const unsigned long long* keys_bgf = V->keys_bgf;
    auto ring_row = [&](int yy) { return s_ring + size_t((yy + kRing) & (kRing - 1)) * RP; };
    auto fetch_row = [&](int yy) {           // async copy of key row yy (empty outside), with sentinels
        unsigned long long* dst = ring_row(yy);
        if (tid == 0) dst[0] = kKeyEmpty;
        if (tid == NT - 1) dst[Wv + 1] = kKeyEmpty;
        if (yy >= 0 && yy < Hv) {
            const unsigned long long* src = keys + size_t(yy) * Wv;
            if (kCoh) {
                // written by other CTAs of the same kernel: L2 loads
                for (int x = tid; x < Wv; x += NT) dst[1 + x] = __ldcg(src + x);
            } else {
                for (int x = tid; x < Wv; x += NT) cp_async8(dst + 1 + x, src + x);
            }
        } else {
            for (int x = tid; x < Wv; x += NT) dst[1 + x] = kKeyEmpty;
        }
    };
    fetch_row(y0 - 1);
    fetch_row(y0);
    fetch_row(y0 + 1);
    cp_async_commit();

    // the active cameras' records, in active order
    for (int a = tid; a < na; a += NT) {
        const int k = V->active[a];
        const CamGeom& G = V->geom[k];
        const FrameRef& F = frames[V->slot * nc + k];
        RCam C;
        C.gx = make_float4(G.N[0], G.N[2], G.N[3], 0.0f);
        C.gy = make_float4(G.N[4], G.N[6], G.N[7], 0.0f);
        C.gz = make_float4(G.N[8], G.N[10], G.N[11], 0.0f);
        C.depth = F.depth;
        C.rgba = F.rgba;
        C.dpitch = F.dpitch;
        C.rpitch = F.rpitch;
        C.maxu = uint32_t(F.W - 1);
        C.maxv = uint32_t(F.H - 1);
        C.w = G.w;
        C.k = k;
        // s / W for s < 2^26: shift = 26 + ceil(log2 W), magic = ceil(2^shift / W);
        // then s * magic / 2^shift = s / W + e with 0 <= e < s / 2^shift < 1 / W,
        // which never carries past the next integer
        const uint32_t lg = F.W > 1 ? 32u - uint32_t(__clz(uint32_t(F.W - 1))) : 0u;
        C.shift = 26u + lg;
        C.magic = uint32_t(((1ull << C.shift) + uint64_t(F.W) - 1) / uint64_t(F.W));
        C.bg = F.bg;
        C.unused[0] = C.unused[1] = 0.0f;
        C.rowc = make_float4(G.N[1], G.N[5], G.N[9], 0.0f);
        C.cen = make_float4(G.pad[0], G.pad[1], G.pad[2], 0.0f);
        s_cam[a] = C;
    }
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
    const int nother = na - 1;
    __syncthreads();                          // s_cam, s_pos staged

    for (int y = y0; y < y1; ++y) {
        // the ring slot of row y+2 held row y-2, last read before the end of
        // the previous iteration
        if (y + 1 < y1)
            fetch_row(y + 2);
        cp_async_commit();
        // per-row products N1 y, N5 y, N9 y (the order stays ((N0 x + N1 y) + N2))
        const float fy = u23_to_float(uint32_t(y));
        for (int a = tid; a < na; a += NT) {
            const float4 rc = s_cam[a].rowc;
            s_cam[a].gx.w = __fmul_rn(rc.x, fy);
            s_cam[a].gy.w = __fmul_rn(rc.y, fy);
            s_cam[a].gz.w = __fmul_rn(rc.z, fy);
        }
        cp_async_wait<1>();                   // rows y-1 .. y+1 have landed
        __syncthreads();

        const unsigned long long* rU = ring_row(y - 1) + 1;
        const unsigned long long* rC = ring_row(y) + 1;
        const unsigned long long* rD = ring_row(y + 1) + 1;
        const size_t rowbase = size_t(y) * Wv;
        bool any_hole = false;
        for (int x = tid; x < Wv; x += NT) {
            const unsigned long long kp = rC[x];
            unsigned long long key = crack ? crack_rule_rows(rU, rC, rD, x, kp, f1) : kp;
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
            // the winner is always active (only active cameras splat)
            const int pw = s_pos[w];
            const RCam& Cw = s_cam[pw];
            const uint32_t sv = uint32_t((static_cast<unsigned long long>(s) * Cw.magic) >> Cw.shift);
            const uint32_t su = s - sv * (Cw.maxu + 1u);
            const uint32_t cw = ld_frame<kCoh>(Cw.rgba + sv * uint32_t(Cw.rpitch) + su);
            const float fx = u23_to_float(uint32_t(x));
            // per-pixel weights: the surface point in the view's frame
            float px = 0.0f, py = 0.0f, lb = 0.0f;
            if (kPixW) {
                px = __fmul_rn(__fmul_rn(__fsub_rn(fx, V->vk[0]), V->vk[2]), Z);
                py = __fmul_rn(__fmul_rn(__fsub_rn(fy, V->vk[1]), V->vk[3]), Z);
                lb = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(px, px), __fmul_rn(py, py)), __fmul_rn(Z, Z)));
            }
            auto weight_of = [&](const RCam& C) {
                if (!kPixW) return C.w;
                const float4 c = C.cen;
                return pixel_weight(c.x, c.y, c.z, px, py, Z, lb);
            };
            const float ww = weight_of(Cw);
            // the winner's colour is consumed after the first group's gathers
            // are in flight (its load latency overlaps their projections)
            float acc0 = 0.0f, acc1 = 0.0f, acc2 = 0.0f;
            auto init_acc = [&]() {
                acc0 = __fmul_rn(ww, u23_to_float(cw & 255u));
                acc1 = __fmul_rn(ww, u23_to_float((cw >> 8) & 255u));
                acc2 = __fmul_rn(ww, u23_to_float((cw >> 16) & 255u));
            };
            if (nother <= 0)
                init_acc();
            float wsum = ww;
            float t0 = ww, t1 = -1.0f, t2 = -1.0f;
            int k0 = w, k1 = INT_MAX, k2 = INT_MAX;
            for (int g0 = 0; g0 < nother; g0 += kGroup) {
                uint32_t dk[kGroup], ck[kGroup], di[kGroup];
                float zk[kGroup];
                int ak[kGroup];
                bool ok[kGroup];
                // branch-free projection of the group (only the gathers are
                // predicated), so the chains can interleave
#pragma unroll
                for (int j = 0; j < kGroup; ++j) {
                    const int ii = min(g0 + j, nother - 1);
                    const int a = ii + (ii >= pw ? 1 : 0);
                    ak[j] = a;
                    const RCam& C = s_cam[a];
                    const float4 gx = C.gx, gy = C.gy, gz = C.gz;
                    const float a0 = __fadd_rn(__fadd_rn(__fmul_rn(gx.x, fx), gx.w), gx.y);
                    const float a1 = __fadd_rn(__fadd_rn(__fmul_rn(gy.x, fx), gy.w), gy.y);
                    const float a2 = __fadd_rn(__fadd_rn(__fmul_rn(gz.x, fx), gz.w), gz.y);
                    const float Xk = __fadd_rn(__fmul_rn(a0, Z), gx.z);
                    const float Yk = __fadd_rn(__fmul_rn(a1, Z), gy.z);
                    const float Zk = __fadd_rn(__fmul_rn(a2, Z), gz.z);
                    uint32_t uk, vk;
                    const bool hit = target_pixel(Xk, Yk, Zk, C.maxu, C.maxv, uk, vk);
                    ok[j] = g0 + j < nother && Zk > zmin && hit;
                    zk[j] = Zk;
                    dk[j] = 0u;
                    ck[j] = 0u;
                    di[j] = 0u;
                    if (ok[j]) {
                        di[j] = vk * uint32_t(C.dpitch) + uk;
                        dk[j] = ld_frame<kCoh>(C.depth + di[j]);
                        ck[j] = ld_frame<kCoh>(C.rgba + vk * uint32_t(C.rpitch) + uk);
                    }
                }
                // the BG layer's depth in camera k: its model where camera k
                // signals BG, none elsewhere (there camera k sees FG)
                if (kLayered && bg_layer) {
#pragma unroll
                    for (int j = 0; j < kGroup; ++j) {
                        if (!ok[j])
                            continue;
                        const uint16_t* bgk = s_cam[ak[j]].bg;
                        dk[j] = (dk[j] == kDepthBg && bgk) ? uint32_t(ld_frame<kCoh>(bgk + di[j])) : 0u;
                    }
                }
                if (g0 == 0)
                    init_acc();
#pragma unroll
                for (int j = 0; j < kGroup; ++j) {
                    if (!ok[j])
                        continue;
                    if (dk[j] - dlo > dspan)         // outside [dlo, dhi]; 0 wraps above
                        continue;
                    const float diff = fabsf(__fsub_rn(u23_to_float(dk[j]), zk[j]));
                    if (!(diff <= __fmul_rn(tau_vis, zk[j])))
                        continue;
                    const RCam& C = s_cam[ak[j]];
                    const float wk = weight_of(C);
                    const uint32_t c = ck[j];
                    acc0 = __fadd_rn(acc0, __fmul_rn(wk, u23_to_float(c & 255u)));
                    acc1 = __fadd_rn(acc1, __fmul_rn(wk, u23_to_float((c >> 8) & 255u)));
                    acc2 = __fadd_rn(acc2, __fmul_rn(wk, u23_to_float((c >> 16) & 255u)));
                    wsum = __fadd_rn(wsum, wk);
                    if (kTop3) {
                        const int k = C.k;
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
        // (e) hole fill: nearest non-hole left / right, the deeper one wins.
        // The row is cut into 32-pixel chunks, a warp owning a run of them;
        // a chunk's non-hole mask is one ballot, the nearest non-hole inside
        // a chunk one bit search, and across chunks and warps a carry.
        const bool row_has_hole = __syncthreads_or(any_hole) != 0;
        if (fill && row_has_hole) {
            constexpr int NW = NT / 32;
            const int lane = tid & 31, wid = tid >> 5;
            // the ring slot of row y - 1: every thread has finished reading
            // it (the barrier above), and row y + 3 lands in it only after
            // the barrier that ends this row (which also restores its sentinels)
            int16_t* s_left = reinterpret_cast<int16_t*>(ring_row(y - 1));
            uint32_t* s_mask = reinterpret_cast<uint32_t*>(s_left + ((Wv + 1) & ~1));
            const int nch = (Wv + 31) >> 5;
            const int cpw = (nch + NW - 1) / NW;
            const int c0 = min(wid * cpw, nch), c1 = min(c0 + cpw, nch);
            int last = -1, first = INT_MAX;
            for (int c = c0; c < c1; ++c) {
                const int x = (c << 5) + lane;
                const uint32_t m = __ballot_sync(0xffffffffu, x < Wv && !s_hole[x]);
                if (m) {
                    last = (c << 5) + 31 - __clz(m);
                    if (first == INT_MAX) first = (c << 5) + __ffs(m) - 1;
                }
                if (lane == 0) s_mask[c] = m;
            }
            if (lane == 0) {
                s_scan[wid] = last;
                s_scan[NW + wid] = first;
            }
            __syncthreads();
            int carry = -1;                          // nearest non-hole left of the chunk
            for (int i = 0; i < wid; ++i) carry = max(carry, s_scan[i]);
            const uint32_t upto = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);   // bits <= lane
            for (int c = c0; c < c1; ++c) {
                const uint32_t m = s_mask[c];
                const uint32_t ml = m & upto;
                const int x = (c << 5) + lane;
                if (x < Wv) s_left[x] = int16_t(ml ? (c << 5) + 31 - __clz(ml) : carry);
                if (m) carry = (c << 5) + 31 - __clz(m);
            }
            __syncwarp();
            carry = INT_MAX;                         // nearest non-hole right of the chunk
            for (int i = wid + 1; i < NW; ++i) carry = min(carry, s_scan[NW + i]);
            const uint32_t from = ~((1u << lane) - 1u);                             // bits >= lane
            for (int c = c1 - 1; c >= c0; --c) {
                const uint32_t m = s_mask[c];
                const uint32_t mr = m & from;
                const int x = (c << 5) + lane;
                const int r0 = mr ? (c << 5) + __ffs(mr) - 1 : carry;
                if (m) carry = (c << 5) + __ffs(m) - 1;
                if (x >= Wv || !s_hole[x])
                    continue;
                const int l = s_left[x], r = r0 == INT_MAX ? -1 : r0;
                if (l < 0 && r < 0)
                    continue;
                // only holes are written and only non-holes are read
                const int src = l < 0 ? r : (r < 0 ? l : (s_dep[r] > s_dep[l] ? r : l));
                s_rgb[x] = s_rgb[src];
                s_dep[x] = s_dep[src];
            }
            __syncthreads();
        }

        // RGB8 row: four pixels -> three aligned 32-bit words where the row
        // allows it, single bytes for the rest
        uint8_t* orow = V->out_rgb + size_t(y) * size_t(V->out_pitch);
        int xdone = 0;
        if ((reinterpret_cast<uintptr_t>(orow) & 3u) == 0) {
            const int nq = Wv >> 2;
            uint32_t* o32 = reinterpret_cast<uint32_t*>(orow);
            const uint4* p4 = reinterpret_cast<const uint4*>(s_rgb);
            for (int q = tid; q < nq; q += NT) {
                const uint4 p = p4[q];
                o32[3 * q + 0] = __byte_perm(p.x, p.y, 0x4210);
                o32[3 * q + 1] = __byte_perm(p.y, p.z, 0x5421);
                o32[3 * q + 2] = __byte_perm(p.z, p.w, 0x6542);
            }
            xdone = nq << 2;
        }
        for (int i = 3 * xdone + tid; i < 3 * Wv; i += NT) {
            const int x = i / 3;
            orow[i] = uint8_t(s_rgb[x] >> (8 * (i - 3 * x)));
        }
        if (V->out_depth)
            for (int x = tid; x < Wv; x += NT) V->out_depth[rowbase + x] = s_dep[x];
        if (V->out_hole)
            for (int x = tid; x < Wv; x += NT) V->out_hole[rowbase + x] = s_hole[x];
        __syncthreads();        // s_rgb / s_dep / s_hole / row products are rewritten next row
    }
}

template <bool kTop3, bool kLayered, bool kPixW>
__global__ void __launch_bounds__(kResolveThreads, 3)
k_resolve(const ViewDesc* __restrict__ views, const FrameRef* __restrict__ frames, int band)
{
    extern __shared__ __align__(16) unsigned char smem[];
    resolve_cta<kTop3, kLayered, kPixW, false>(views, frames, band, int(blockIdx.x), int(blockIdx.y), smem);
}

// ---------------------------------------------------------------------------
// Persistent serving kernel.  One cooperative launch (every CTA resident)
// loops: CTA 0 waits for the next posted batch, then all CTAs run its clear,
// splat and resolve as virtual CTAs, with a grid barrier between the steps
// and a gpu-scope fence after each barrier (so weak loads see the other
// CTAs' writes and the frames uploaded before the batch was posted), and
// CTA 0 publishes the batch's completion.  It returns when no batch comes
// for idle_ns, on q->stop, or when a barrier runs out (sync->err, then
// q->err).
// ---------------------------------------------------------------------------
namespace {

__device__ __forceinline__ uint64_t gtimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Sense-counting grid barrier with a bounded wait (limit_ns); false once any
// CTA gave up.
__device__ bool persist_barrier(PersistSync* sync, unsigned int& gen, uint64_t limit_ns)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int g = gen;
        __threadfence();
        if (atomicAdd(&sync->count, 1u) == gridDim.x - 1) {
            atomicExch(&sync->count, 0u);
            __threadfence();
            atomicExch(&sync->gen, g + 1);
        } else {
            const uint64_t t0 = gtimer();
            while (*reinterpret_cast<volatile unsigned int*>(&sync->gen) == g) {
                if (*reinterpret_cast<volatile int*>(&sync->err) != 0) break;
                if (gtimer() - t0 > limit_ns) {
                    atomicCAS(&sync->err, 0, kPersistErrBarrier);
                    break;
                }
                __nanosleep(256);
            }
        }
        __threadfence();                      // acquire: later loads see the writes before the barrier
        gen = g + 1;
        s_ok = *reinterpret_cast<volatile int*>(&sync->err) == 0;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace

__global__ void __launch_bounds__(kResolveThreads, 3)
k_serve_persistent(PersistQueue* q, PersistSync* sync, uint32_t first, uint64_t idle_ns, uint64_t wait_ns)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ PersistBatch s_b;
    __shared__ int s_cmd;
    unsigned int gen = 0;                     // the host zeroes *sync before the launch
    for (uint32_t b = first;; ++b) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            int cmd = 1;
            const uint64_t t0 = gtimer();
            for (;;) {
                if (q->stop) break;
                if (q->posted > b) {
                    cmd = 0;
                    break;
                }
                if (gtimer() - t0 > idle_ns) break;
                __nanosleep(1000);
            }
            sync->cmd = cmd;
        }
        if (!persist_barrier(sync, gen, wait_ns)) break;
        if (threadIdx.x == 0) {
            s_cmd = *reinterpret_cast<volatile int*>(&sync->cmd);
            if (!s_cmd) {
                // field by field through volatile reads: the host wrote it
                const volatile PersistBatch& src = q->batch[b % kPersistRing];
                s_b.views = src.views;
                s_b.frames = src.frames;
                s_b.keys = src.keys;
                s_b.n_keys = src.n_keys;
                s_b.n_views = src.n_views;
                s_b.max_h = src.max_h;
                s_b.band = src.band;
                s_b.splat_bx = src.splat_bx;
                s_b.pixel_weights = src.pixel_weights;
            }
        }
        __syncthreads();
        if (s_cmd) break;
        const PersistBatch B = s_b;
        // (a0) the batch's z-buffers
        const size_t stride = size_t(gridDim.x) * blockDim.x;
        for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < B.n_keys; i += stride)
            B.keys[i] = kKeyEmpty;
        if (!persist_barrier(sync, gen, wait_ns)) break;
        // (a) + (b)
        for (int v = int(blockIdx.x); v < B.splat_bx * B.n_views; v += int(gridDim.x))
            splat_cta<false, false, true>(B.views, B.frames, v % B.splat_bx, v / B.splat_bx, B.splat_bx);
        if (!persist_barrier(sync, gen, wait_ns)) break;
        // (c) + (d) + (e)
        const int nb = (B.max_h + B.band - 1) / B.band;
        for (int v = int(blockIdx.x); v < nb * B.n_views; v += int(gridDim.x)) {
            if (B.pixel_weights)
                resolve_cta<false, false, true, true>(B.views, B.frames, B.band, v % nb, v / nb, smem);
            else
                resolve_cta<false, false, false, true>(B.views, B.frames, B.band, v % nb, v / nb, smem);
        }
        if (!persist_barrier(sync, gen, wait_ns)) break;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            __threadfence_system();           // the batch's outputs before its completion
            q->done = b + 1;
            __threadfence_system();
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        q->err = *reinterpret_cast<volatile int*>(&sync->err);
        __threadfence_system();
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
int device_sms()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        sms = 1;
    }
    return sms;
}

namespace {

// Splat depth loads: 16-byte vectors (8 pixels per lane) or 2-byte loads at
// a stride of 32 pixels.  FVV_SPLAT_VEC=0/1 picks one for measurements.
bool splat_vec()
{
    static const int v = [] {
        const char* e = std::getenv("FVV_SPLAT_VEC");
        return e ? (e[0] == '1' ? 1 : 0) : 0;
    }();
    return v != 0;
}

}  // namespace

size_t resolve_smem_bytes(int max_w, int n_cams, bool layered)
{
    return resolve_layout(max_w, n_cams, layered).total;
}

cudaError_t launch_clear_keys(unsigned long long* keys, size_t n, cudaStream_t stream)
{
    if (n == 0) return cudaSuccess;
    size_t blocks = ((n >> 1) + 255) / 256;
    const size_t cap = size_t(device_sms()) * 16;
    if (blocks < 1) blocks = 1;
    if (blocks > cap) blocks = cap;
    k_clear_keys<<<unsigned(blocks), 256, 0, stream>>>(keys, n);
    return cudaGetLastError();
}

cudaError_t launch_warp_splat(const ViewDesc* views, int n_views, int max_chunks,
                              const FrameRef* frames, cudaStream_t stream, bool layered)
{
    if (n_views <= 0 || max_chunks <= 0) return cudaSuccess;
    constexpr int kWarps = kSplatThreads / 32;      // one warp per segment at a time
    // persistent warps: about two resident waves over all views of the batch
    const int sms = device_sms();
    const int want = (2 * 5 * sms + n_views - 1) / n_views;
    const int need = (max_chunks + kWarps - 1) / kWarps;
    const int bx = need < want ? need : (want < 1 ? 1 : want);
    dim3 grid(static_cast<unsigned>(bx), static_cast<unsigned>(n_views));
    const bool vec = splat_vec();
    if (layered) {
        if (vec) k_warp_splat<true, true><<<grid, kSplatThreads, 0, stream>>>(views, frames);
        else k_warp_splat<true, false><<<grid, kSplatThreads, 0, stream>>>(views, frames);
    } else {
        if (vec) k_warp_splat<false, true><<<grid, kSplatThreads, 0, stream>>>(views, frames);
        else k_warp_splat<false, false><<<grid, kSplatThreads, 0, stream>>>(views, frames);
    }
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
    const int sms = device_sms();
    auto go = [&](auto kernel) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        // Bands of two rows, launched view after view: the CTAs resident at
        // one time then cover about one view, whose frames stay in L2 for
        // its gathers (a single wave of all views' bands streams every
        // view's frames at once and doubled the DRAM reads).  Single rows
        // when two-row bands would not fill the resident slots.
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kResolveThreads, smem);
        if (e != cudaSuccess) return e;
        const long long slots = (long long)(per_sm > 0 ? per_sm : 1) * sms;
        const int band = (long long)max_h * n_views >= 2 * kResolveBand * slots ? kResolveBand : 1;
        dim3 grid(static_cast<unsigned>((max_h + band - 1) / band), static_cast<unsigned>(n_views));
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

void persist_batch_shape(int n_views, int max_h, int max_chunks, int ctas, int* band, int* splat_bx)
{
    // two-row bands when they fill the CTAs, else single rows; the splat's
    // segments spread over about one virtual CTA per real one
    *band = (long long)max_h * n_views >= 2LL * kResolveBand * ctas ? kResolveBand : 1;
    constexpr int kWarps = kSplatThreads / 32;
    const int need = (max_chunks + kWarps - 1) / kWarps;
    const int want = (ctas + n_views - 1) / n_views;
    *splat_bx = std::max(1, std::min(need, want));
}

int persist_grid(int max_w, int n_cams)
{
    const size_t smem = resolve_smem_bytes(max_w, n_cams, false);
    int per_sm = 0;
    if (cudaFuncSetAttribute(k_serve_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_serve_persistent, kResolveThreads, smem) !=
            cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    // other kernels (the frame uploads: 256 threads of at most 32 registers)
    // must fit beside the persistent one instead of waiting for it to idle:
    // when its CTAs leave fewer registers than that, one CTA per SM less
    cudaFuncAttributes fa{};
    int regs_sm = 65536;
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaFuncGetAttributes(&fa, k_serve_persistent) != cudaSuccess ||
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess) {
        cudaGetLastError();
        return (per_sm > 1 ? per_sm - 1 : 1) * device_sms();
    }
    const int free_regs = regs_sm - per_sm * kResolveThreads * fa.numRegs;
    if (free_regs < 256 * 32 && per_sm > 1) --per_sm;
    return per_sm * device_sms();
}

cudaError_t launch_serve_persistent(PersistQueue* q_dev, PersistSync* sync, uint32_t first, int max_w, int n_cams,
                                    uint64_t idle_ns, uint64_t wait_ns, cudaStream_t stream, int* ctas)
{
    const size_t smem = resolve_smem_bytes(max_w, n_cams, false);
    const int grid = persist_grid(max_w, n_cams);
    if (grid < 1) return cudaErrorInvalidValue;
    *ctas = grid;
    void* args[] = {&q_dev, &sync, &first, &idle_ns, &wait_ns};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_serve_persistent), dim3(unsigned(grid)),
                                       dim3(kResolveThreads), args, smem, stream);
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
