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
// Every FP32 operation of the warp, the filter and the blend is an explicit
// round-to-nearest intrinsic (__fmul_rn / __fadd_rn / __fsub_rn / __fdiv_rn)
// in a fixed order with no FMA contraction, so the results are exactly the
// IEEE values of that operation sequence.
#include <climits>

#include "fvv_internal.h"

namespace fvv {

namespace {

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

struct SmemLayout {
    size_t keys, rgb, dep, hole, geom, frames, active, scan, total;
};

__host__ __device__ inline SmemLayout resolve_layout(int W, int n_cams)
{
    SmemLayout L;
    size_t o = 0;
    L.keys = o;   o = align16(o + size_t(3) * W * sizeof(unsigned long long));
    L.rgb = o;    o = align16(o + size_t(W) * 4);
    L.dep = o;    o = align16(o + size_t(W) * 4);
    L.hole = o;   o = align16(o + size_t(W));
    L.geom = o;   o = align16(o + size_t(n_cams) * 16 * sizeof(float));
    L.frames = o; o = align16(o + size_t(n_cams) * sizeof(FrameRef));
    L.active = o; o = align16(o + size_t(kMaxCams) * sizeof(int));
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

// streaming 16-byte load: read once, do not keep in L1, evict first from L2
__device__ __forceinline__ uint4 ld_stream_u4(const void* ptr, uint64_t pol)
{
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(ptr), "l"(pol));
    return v;
}

// z-buffer read at L2 (the value may be stale, but keys only ever decrease,
// so a stale value is never below the current one)
__device__ __forceinline__ unsigned long long ld_key(const unsigned long long* ptr, uint64_t pol)
{
    unsigned long long v;
    asm volatile("ld.global.cg.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(ptr), "l"(pol));
    return v;
}

// fire-and-forget 64-bit atomic minimum, kept in L2
__device__ __forceinline__ void red_min_key(unsigned long long* ptr, unsigned long long v, uint64_t pol)
{
    asm volatile("red.global.min.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(ptr), "l"(v), "l"(pol)
                 : "memory");
}

// ---------------------------------------------------------------------------
// (a) + (b): forward warp and z-buffer splat.
// One thread = 16 consecutive source pixels of one row of one active camera
// (two 16-byte depth loads).  Threads of a view are numbered camera-major
// over the active cameras: chunk_begin[a] .. chunk_begin[a+1).  Every CTA
// belongs to one view, whose maps and frame table it stages in shared memory.
// A point is splatted only when its key is below the key read at its target
// pixel first: keys only decrease, so the skipped atomics could not win.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSplatThreads)
k_warp_splat(const ViewDesc* __restrict__ views, const FrameRef* __restrict__ frames)
{
    __shared__ __align__(16) float s_M[kMaxCams][12];
    __shared__ __align__(16) FrameRef s_F[kMaxCams];
    __shared__ int s_cb[kMaxCams + 1];
    __shared__ int s_act[kMaxCams];
    const ViewDesc* V = views + blockIdx.y;
    const int na = V->n_active;
    const int first = blockIdx.x * kSplatThreads;
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

    const int chunk = first + threadIdx.x;
    if (chunk >= s_cb[na])
        return;
    int a = 0;
    while (chunk >= s_cb[a + 1])
        ++a;
    const int k = s_act[a];
    const FrameRef F = s_F[a];
    const int cpr = (F.W + kSplatPix - 1) / kSplatPix;
    const int local = chunk - s_cb[a];
    const int v = local / cpr;
    const int u0 = (local - v * cpr) * kSplatPix;
    const uint16_t* row = F.depth + size_t(v) * F.dpitch;
    const uint64_t pol_stream = policy_evict_first();
    const uint64_t pol_keys = policy_evict_last();

    uint32_t dw[kSplatPix / 2];                   // two depth codes per word
    if (u0 + kSplatPix <= F.W) {
        const uint4 q0 = ld_stream_u4(row + u0, pol_stream);
        const uint4 q1 = ld_stream_u4(row + u0 + 8, pol_stream);
        dw[0] = q0.x; dw[1] = q0.y; dw[2] = q0.z; dw[3] = q0.w;
        dw[4] = q1.x; dw[5] = q1.y; dw[6] = q1.z; dw[7] = q1.w;
    } else {
#pragma unroll
        for (int i = 0; i < kSplatPix / 2; ++i) {
            const uint32_t lo = (u0 + 2 * i < F.W) ? uint32_t(row[u0 + 2 * i]) : 0u;
            const uint32_t hi = (u0 + 2 * i + 1 < F.W) ? uint32_t(row[u0 + 2 * i + 1]) : 0u;
            dw[i] = lo | (hi << 16);
        }
    }

    const float* m = s_M[a];
    const float m0 = m[0], m2 = m[2], m3 = m[3];
    const float m4 = m[4], m6 = m[6], m7 = m[7];
    const float m8 = m[8], m10 = m[10], m11 = m[11];
    const float fv = float(v);
    const float r0 = __fmul_rn(m[1], fv), r1 = __fmul_rn(m[5], fv), r2 = __fmul_rn(m[9], fv);
    const float zmin = V->z_min;
    const uint32_t dlo = V->d_lo, dhi = V->d_hi;
    const int Wv = V->Wv;
    const float maxu = float(Wv - 1), maxv = float(V->Hv - 1);
    unsigned long long* __restrict__ keys = V->keys;
    const unsigned long long khi = static_cast<unsigned long long>(k) << kSrcBits;
    const uint32_t src0 = uint32_t(v) * uint32_t(F.W) + uint32_t(u0);

#pragma unroll
    for (int h = 0; h < kSplatPix; h += 8) {
        unsigned long long key[8];
        uint32_t pix[8];
        bool ok[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int ii = h + i;
            const uint32_t dd = (dw[ii >> 1] >> (16 * (ii & 1))) & 0xFFFFu;
            ok[i] = false;
            key[i] = kKeyEmpty;
            pix[i] = 0;
            if (dd == 0u || dd < dlo || dd > dhi)
                continue;
            const float fu = float(u0 + ii);
            const float z = float(dd);
            const float a0 = __fadd_rn(__fadd_rn(__fmul_rn(m0, fu), r0), m2);
            const float a1 = __fadd_rn(__fadd_rn(__fmul_rn(m4, fu), r1), m6);
            const float a2 = __fadd_rn(__fadd_rn(__fmul_rn(m8, fu), r2), m10);
            const float X = __fadd_rn(__fmul_rn(a0, z), m3);
            const float Y = __fadd_rn(__fmul_rn(a1, z), m7);
            const float Z = __fadd_rn(__fmul_rn(a2, z), m11);
            if (!(Z > zmin))
                continue;
            const float tu = floorf(__fadd_rn(__fdiv_rn(X, Z), 0.5f));
            const float tv = floorf(__fadd_rn(__fdiv_rn(Y, Z), 0.5f));
            // also rejects NaN and +-inf, as a finiteness test would
            if (!(tu >= 0.0f && tu <= maxu && tv >= 0.0f && tv <= maxv))
                continue;
            ok[i] = true;
            pix[i] = uint32_t(int(tv)) * uint32_t(Wv) + uint32_t(int(tu));
            key[i] = (static_cast<unsigned long long>(__float_as_uint(Z)) << 32) | khi |
                     static_cast<unsigned long long>(src0 + uint32_t(ii));
        }
        unsigned long long cur[8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
            cur[i] = ok[i] ? ld_key(keys + pix[i], pol_keys) : 0ull;
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (ok[i] && key[i] < cur[i])
                red_min_key(keys + pix[i], key[i], pol_keys);
    }
}

// ---------------------------------------------------------------------------
// (c) crack / outlier rule on the three staged key rows.  Pairs, in order:
// (left, right), (up, down), (up-left, down-right), (up-right, down-left).
// A pair is consistent when both keys are present and zmax <= (1+tau) zmin.
// An empty pixel takes min(a, b) of the first consistent pair; a present
// pixel takes it from the first consistent pair with z_p > (1+tau) zmax.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long nb_key(const unsigned long long* s, int Wv, int x, int r)
{
    return (x < 0 || x >= Wv) ? kKeyEmpty : s[r * Wv + x];
}

__device__ __forceinline__ unsigned long long crack_rule(const unsigned long long* s, int Wv, int x,
                                                         unsigned long long kp, float f1)
{
    const int ax[4] = {-1, 0, -1, 1}, ar[4] = {1, 0, 0, 0};
    const int bx[4] = {1, 0, 1, -1}, br[4] = {1, 2, 2, 2};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const unsigned long long a = nb_key(s, Wv, x + ax[q], ar[q]);
        const unsigned long long b = nb_key(s, Wv, x + bx[q], br[q]);
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
// (c) + (d) + (e), one CTA per output row of one view.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kResolveThreads, 3)
k_resolve(const ViewDesc* __restrict__ views, const FrameRef* __restrict__ frames)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const ViewDesc* V = views + blockIdx.y;
    const int Wv = V->Wv, Hv = V->Hv;
    const int y = blockIdx.x;
    if (y >= Hv)
        return;
    const int nc = V->n_cams, na = V->n_active;
    const SmemLayout L = resolve_layout(Wv, nc);
    unsigned long long* s_keys = reinterpret_cast<unsigned long long*>(smem + L.keys);
    uint32_t* s_rgb = reinterpret_cast<uint32_t*>(smem + L.rgb);
    float* s_dep = reinterpret_cast<float*>(smem + L.dep);
    uint8_t* s_hole = smem + L.hole;
    float* s_geom = reinterpret_cast<float*>(smem + L.geom);
    FrameRef* s_fr = reinterpret_cast<FrameRef*>(smem + L.frames);
    int* s_act = reinterpret_cast<int*>(smem + L.active);
    int* s_scan = reinterpret_cast<int*>(smem + L.scan);
    const int tid = threadIdx.x;
    constexpr int NT = kResolveThreads;

    // stage the backward maps, weights, frame table and active list.  Per
    // camera, 16 floats: N[0..11], then w and the row terms N1 y, N5 y, N9 y
    // (the products the per-pixel projection would form; same rounding).
    const float fy = float(y);
    for (int i = tid; i < nc * 16; i += NT) {
        const int k = i >> 4, j = i & 15;
        const float* Nk = V->geom[k].N;
        float val;
        if (j < 12) val = Nk[j];
        else if (j == 12) val = V->geom[k].w;
        else val = __fmul_rn(Nk[1 + 4 * (j - 13)], fy);
        s_geom[i] = val;
    }
    for (int i = tid; i < nc; i += NT)
        s_fr[i] = frames[V->slot * nc + i];
    for (int i = tid; i < na; i += NT)
        s_act[i] = V->active[i];
    // stage key rows y-1, y, y+1 (empty outside the image)
    const unsigned long long* keys = V->keys;
    for (int r = 0; r < 3; ++r) {
        const int yy = y - 1 + r;
        unsigned long long* dst = s_keys + size_t(r) * Wv;
        if (yy >= 0 && yy < Hv) {
            const unsigned long long* src = keys + size_t(yy) * Wv;
            for (int x = tid; x < Wv; x += NT) dst[x] = src[x];
        } else {
            for (int x = tid; x < Wv; x += NT) dst[x] = kKeyEmpty;
        }
    }
    __syncthreads();

    const bool crack = (V->flags & kFlagCrack) != 0;
    const float f1 = __fadd_rn(1.0f, V->tau_crack);
    const float tau_vis = V->tau_vis, zmin = V->z_min;
    const uint32_t dlo = V->d_lo, dhi = V->d_hi;
    float* __restrict__ top3 = V->out_top3;
    unsigned long long* __restrict__ okeys = V->out_keys;
    const size_t rowbase = size_t(y) * Wv;
    const float4* g4 = reinterpret_cast<const float4*>(s_geom);

    for (int x = tid; x < Wv; x += NT) {
        const unsigned long long kp = s_keys[Wv + x];
        const unsigned long long key = crack ? crack_rule(s_keys, Wv, x, kp, f1) : kp;
        if (okeys) okeys[rowbase + x] = key;
        if (key == kKeyEmpty) {
            s_rgb[x] = 0u;
            s_dep[x] = 0.0f;
            s_hole[x] = 1;
            if (top3) {
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
        const uint32_t cw = __ldg(Fw.rgba + size_t(sv) * Fw.rpitch + su);
        const float ww = s_geom[w * 16 + 12];
        float acc0 = __fmul_rn(ww, float(cw & 255u));
        float acc1 = __fmul_rn(ww, float((cw >> 8) & 255u));
        float acc2 = __fmul_rn(ww, float((cw >> 16) & 255u));
        float wsum = ww;
        float t0 = ww, t1 = -1.0f, t2 = -1.0f;
        int k0 = w, k1 = INT_MAX, k2 = INT_MAX;
        const float fx = float(x);
        // cameras in groups of four: project all four and issue their depth
        // and colour gathers before any is consumed, then accumulate in
        // ascending camera order
        for (int g0 = 0; g0 < na; g0 += 4) {
            uint32_t dk[4], ck[4];
            float zk[4];
            int kk[4];
            bool ok[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                ok[j] = false;
                dk[j] = 0u;
                ck[j] = 0u;
                zk[j] = 0.0f;
                kk[j] = 0;
                const int ai = g0 + j;
                if (ai >= na)
                    continue;
                const int k = s_act[ai];
                kk[j] = k;
                if (k == w)
                    continue;
                const float4 A = g4[4 * k + 0], Bq = g4[4 * k + 1], Cq = g4[4 * k + 2],
                             Dq = g4[4 * k + 3];
                const float a0 = __fadd_rn(__fadd_rn(__fmul_rn(A.x, fx), Dq.y), A.z);
                const float a1 = __fadd_rn(__fadd_rn(__fmul_rn(Bq.x, fx), Dq.z), Bq.z);
                const float a2 = __fadd_rn(__fadd_rn(__fmul_rn(Cq.x, fx), Dq.w), Cq.z);
                const float Xk = __fadd_rn(__fmul_rn(a0, Z), A.w);
                const float Yk = __fadd_rn(__fmul_rn(a1, Z), Bq.w);
                const float Zk = __fadd_rn(__fmul_rn(a2, Z), Cq.w);
                if (!(Zk > zmin))
                    continue;
                const float tu = floorf(__fadd_rn(__fdiv_rn(Xk, Zk), 0.5f));
                const float tv = floorf(__fadd_rn(__fdiv_rn(Yk, Zk), 0.5f));
                const FrameRef& Fk = s_fr[k];
                // also rejects NaN and +-inf, as a finiteness test would
                if (!(tu >= 0.0f && tu <= float(Fk.W - 1) && tv >= 0.0f && tv <= float(Fk.H - 1)))
                    continue;
                const int uk = int(tu), vk = int(tv);
                ok[j] = true;
                zk[j] = Zk;
                dk[j] = __ldg(Fk.depth + size_t(vk) * Fk.dpitch + uk);
                ck[j] = __ldg(Fk.rgba + size_t(vk) * Fk.rpitch + uk);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (!ok[j])
                    continue;
                if (dk[j] == 0u || dk[j] < dlo || dk[j] > dhi)
                    continue;
                const float diff = fabsf(__fsub_rn(float(dk[j]), zk[j]));
                if (!(diff <= __fmul_rn(tau_vis, zk[j])))
                    continue;
                const int k = kk[j];
                const float wk = s_geom[16 * k + 12];
                const uint32_t c = ck[j];
                acc0 = __fadd_rn(acc0, __fmul_rn(wk, float(c & 255u)));
                acc1 = __fadd_rn(acc1, __fmul_rn(wk, float((c >> 8) & 255u)));
                acc2 = __fadd_rn(acc2, __fmul_rn(wk, float((c >> 16) & 255u)));
                wsum = __fadd_rn(wsum, wk);
                if (w_before(wk, k, t0, k0)) {
                    t2 = t1; k2 = k1; t1 = t0; k1 = k0; t0 = wk; k0 = k;
                } else if (w_before(wk, k, t1, k1)) {
                    t2 = t1; k2 = k1; t1 = wk; k1 = k;
                } else if (w_before(wk, k, t2, k2)) {
                    t2 = wk; k2 = k;
                }
            }
        }
        s_rgb[x] = blend_channel(acc0, wsum) | (blend_channel(acc1, wsum) << 8) |
                   (blend_channel(acc2, wsum) << 16);
        s_dep[x] = Z;
        s_hole[x] = 0;
        if (top3) {
            top3[3 * (rowbase + x) + 0] = __fdiv_rn(t0, wsum);
            top3[3 * (rowbase + x) + 1] = t1 >= 0.0f ? __fdiv_rn(t1, wsum) : 0.0f;
            top3[3 * (rowbase + x) + 2] = t2 >= 0.0f ? __fdiv_rn(t2, wsum) : 0.0f;
        }
    }
    __syncthreads();

    // (e) hole fill: nearest non-hole left / right of each hole, the deeper wins
    if (V->flags & kFlagFill) {
        int* s_left = reinterpret_cast<int*>(s_keys);     // key rows are no longer needed
        int* s_right = s_left + Wv;
        const int seg = (Wv + NT - 1) / NT;
        const int x0 = min(tid * seg, Wv), x1 = min(x0 + seg, Wv);
        int last = -1;
        for (int x = x0; x < x1; ++x)
            if (!s_hole[x]) last = x;
        int run = block_excl_prefix_max(last, s_scan);
        for (int x = x0; x < x1; ++x) {
            if (!s_hole[x]) run = x;
            s_left[x] = run;
        }
        int first = INT_MAX;
        for (int x = x1 - 1; x >= x0; --x)
            if (!s_hole[x]) first = x;
        run = block_excl_suffix_min(first, s_scan);
        for (int x = x1 - 1; x >= x0; --x) {
            if (!s_hole[x]) run = x;
            s_right[x] = run;
        }
        __syncthreads();
        for (int x = tid; x < Wv; x += NT) {
            if (!s_hole[x])
                continue;
            const int l = s_left[x];
            const int r = s_right[x] == INT_MAX ? -1 : s_right[x];
            if (l < 0 && r < 0)
                continue;
            const int src = l < 0 ? r : (r < 0 ? l : (s_dep[r] > s_dep[l] ? r : l));
            s_rgb[x] = s_rgb[src];
            s_dep[x] = s_dep[src];
        }
        __syncthreads();
    }

    uint8_t* orow = V->out_rgb + size_t(y) * size_t(V->out_pitch);
    for (int i = tid; i < 3 * Wv; i += NT) {
        const int x = i / 3;
        const int c = i - 3 * x;
        orow[i] = uint8_t(s_rgb[x] >> (8 * c));
    }
    if (V->out_depth)
        for (int x = tid; x < Wv; x += NT) V->out_depth[rowbase + x] = s_dep[x];
    if (V->out_hole)
        for (int x = tid; x < Wv; x += NT) V->out_hole[rowbase + x] = s_hole[x];
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
size_t resolve_smem_bytes(int max_w, int n_cams) { return resolve_layout(max_w, n_cams).total; }

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
                              const FrameRef* frames, cudaStream_t stream)
{
    if (n_views <= 0 || max_chunks <= 0) return cudaSuccess;
    dim3 grid(static_cast<unsigned>((max_chunks + kSplatThreads - 1) / kSplatThreads), static_cast<unsigned>(n_views));
    k_warp_splat<<<grid, kSplatThreads, 0, stream>>>(views, frames);
    return cudaGetLastError();
}

cudaError_t launch_resolve(const ViewDesc* views, int n_views, int max_h, int max_w, int n_cams,
                           const FrameRef* frames, cudaStream_t stream)
{
    if (n_views <= 0 || max_h <= 0) return cudaSuccess;
    // the layout grows with the width and the camera count, so the widest
    // view of the batch bounds every CTA's shared memory
    const size_t smem = resolve_smem_bytes(max_w, n_cams);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_resolve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(smem));
        if (e != cudaSuccess) return e;
    }
    dim3 grid(static_cast<unsigned>(max_h), static_cast<unsigned>(n_views));
    k_resolve<<<grid, kResolveThreads, smem, stream>>>(views, frames);
    return cudaGetLastError();
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
