// fvv_jbf.cu -- joint bilateral depth pre-filter (Sec. VI: a colour-guided
// joint bilateral filter fills small gaps in the live depth, in particular
// along object boundaries).
//
// A pixel without depth (code 0) takes the weighted mean of the valid codes
// in its (2r+1) x (2r+1) window; every other pixel keeps its code.  The
// weight of neighbour q is s[dy][dx] * c[|dR|] * c[|dG|] * c[|dB|] with
// s = exp(-(dx^2 + dy^2) / (2 sigma_s^2)) and c[t] = exp(-t^2 / (2
// sigma_c^2)), both evaluated on the host in FP64 and rounded to FP32 once.
// Neighbours are visited in row-major window order and every FP32 operation
// is an explicit round-to-nearest intrinsic, so the result is exactly that
// of the stated operation sequence.  The code is floor(acc / wsum + 0.5)
// clamped to [d_lo, d_hi], written only when at least min_valid neighbours
// are valid codes; the background signal is neither a source nor filled.
// One pass, out of place.
//
// The filter reads 2 + 3 bytes and writes 2 bytes per pixel: it is bound by
// HBM bandwidth once the few pixels without depth, the only ones that visit
// their window, no longer hold up whole warps (see k_jbf).
#include <cmath>
#include <cstring>

#include "fvv_jbf.h"
#include "fvv_runtime.h"

namespace fvv {

namespace {

__device__ __forceinline__ float code_to_float(uint32_t d)   // exact for d < 2^23
{
    return __fsub_rn(__uint_as_float(0x4B000000u | d), 8388608.0f);
}

// A CTA filters a kTileW x kTileH tile of camera blockIdx.z.  Phase 1
// stages the tile and its halo (codes and colour bytes) in shared memory:
// the tile's own columns as 16-byte loads and stores when the rows are
// 16-byte aligned, the halo columns and ragged edges element by element.
// Phase 2 writes the tile's codes back out 8 at a time and lists the pixels
// without one.  Phase 3 deals the listed pixels out to the threads, so a
// tile's few holes are filtered by many threads at once instead of idling
// the rest of their warps; each filtered pixel walks its window in shared
// memory in the stated order (the radius is a template parameter, so the
// window unrolls and its loads are in flight together) and overwrites its
// output.
constexpr int kTileW = 64, kTileH = 16, kThreads = 256;
constexpr int kDM = 8, kCM = 32;          // left margins of the staged rows: pixels, colour bytes
constexpr int kDW = kDM + kTileW + kDM;   // staged code row, pixels
constexpr int kCW = kCM + 3 * kTileW + kCM;   // staged colour row, bytes
static_assert(kJbfMaxRadius <= kDM && 3 * kJbfMaxRadius <= kCM, "halo wider than the margins");

template <int R>
__global__ void __launch_bounds__(kThreads) k_jbf(const JbfParams P)
{
    constexpr int side = 2 * R + 1;
    constexpr int hh = kTileH + 2 * R;
    __shared__ __align__(16) uint16_t s_d[hh][kDW];
    __shared__ __align__(16) uint8_t s_c[hh][kCW];
    // per staged pixel: the code as FP32 (-1 when it is no source) and the
    // colour packed R | G << 8 | B << 16, for the window walks of phase 3
    // (rows padded by a word so that neighbouring rows fall in other banks)
    __shared__ float s_df[hh][kDW + 1];
    __shared__ uint32_t s_cc[hh][kDW + 1];
    __shared__ uint16_t s_list[kTileW * kTileH];
    __shared__ float s_ws[side * side];
    __shared__ float s_wc[256];
    __shared__ int s_n;
    const JbfCam& C = P.cam[blockIdx.z];
    const int x0 = blockIdx.x * kTileW, y0 = blockIdx.y * kTileH;
    const int W = P.width;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool vec = C.vec != 0;
    if (tid == 0) s_n = 0;
    // the weight tables in shared memory: the filtered pixels of a warp
    // index them at different places, which parameter (constant) memory
    // would serialise
    for (int i = tid; i < side * side; i += kThreads) s_ws[i] = P.s[i];
    for (int i = tid; i < 256; i += kThreads) s_wc[i] = P.c[i];
    // phase 1: a warp per staged row.  Tasks 0-7: the tile's codes, 8 pixels
    // each; 8-19: its colour, 16 bytes each; then the halo elements (R codes
    // and 3R colour bytes on each side).  Outside the image a code of 0
    // (never a source) and colour 0.
    constexpr int kTasks = 8 + 12 + 8 * R;
    for (int hy = warp; hy < hh; hy += kThreads / 32) {
        const int gy = y0 - R + hy;
        const bool row_in = gy >= 0 && gy < P.height;
        const uint16_t* drow = C.src + size_t(row_in ? gy : 0) * C.src_pitch;
        const uint8_t* crow = C.rgb + size_t(row_in ? gy : 0) * C.rgb_pitch;
        for (int t = lane; t < kTasks; t += 32) {
            if (t < 8) {
                const int x = x0 + 8 * t;
                uint16_t* dst = &s_d[hy][kDM + 8 * t];
                if (row_in && vec && x + 8 <= W) {
                    *reinterpret_cast<uint4*>(dst) = __ldg(reinterpret_cast<const uint4*>(drow + x));
                } else {
#pragma unroll
                    for (int e = 0; e < 8; ++e) dst[e] = (row_in && x + e < W) ? __ldg(drow + x + e) : uint16_t(0);
                }
            } else if (t < 20) {
                const int b = 3 * x0 + 16 * (t - 8);
                uint8_t* dst = &s_c[hy][kCM + 16 * (t - 8)];
                if (row_in && vec && b + 16 <= 3 * W) {
                    *reinterpret_cast<uint4*>(dst) = __ldg(reinterpret_cast<const uint4*>(crow + b));
                } else {
#pragma unroll
                    for (int e = 0; e < 16; ++e) dst[e] = (row_in && b + e < 3 * W) ? __ldg(crow + b + e) : uint8_t(0);
                }
            } else if (t < 20 + 2 * R) {
                const int h = t - 20;                              // left R codes, then right R
                const int tx = h < R ? h - R : kTileW + (h - R);
                const int x = x0 + tx;
                s_d[hy][kDM + tx] = (row_in && x >= 0 && x < W) ? __ldg(drow + x) : uint16_t(0);
            } else {
                const int h = t - 20 - 2 * R;                      // left 3R bytes, then right 3R
                const int tb = h < 3 * R ? h - 3 * R : 3 * kTileW + (h - 3 * R);
                const int b = 3 * x0 + tb;
                s_c[hy][kCM + tb] = (row_in && b >= 0 && b < 3 * W) ? __ldg(crow + b) : uint8_t(0);
            }
        }
    }
    __syncthreads();
    // phase 1b: sources and packed colour of every staged pixel
    constexpr int sw = kTileW + 2 * R;
    for (int i = tid; i < hh * sw; i += kThreads) {
        const int hy = i / sw, col = kDM - R + (i - hy * sw);
        const uint32_t q = s_d[hy][col];
        const bool src = q >= P.d_lo && q <= P.d_hi && q != kDepthBg;
        s_df[hy][col] = src ? code_to_float(q) : -1.0f;
        const uint8_t* c = &s_c[hy][kCM + 3 * (col - kDM)];
        s_cc[hy][col] = uint32_t(c[0]) | (uint32_t(c[1]) << 8) | (uint32_t(c[2]) << 16);
    }
    // phase 2: the tile's codes go out 8 at a time (pixels without one as
    // 0 for now) and those pixels are listed
    if (tid < kTileH * (kTileW / 8)) {
        const int ty = tid >> 3, c8 = tid & 7;
        const int y = y0 + ty, x = x0 + 8 * c8;
        if (y < P.height && x < W) {
            const uint4 v = *reinterpret_cast<const uint4*>(&s_d[ty + R][kDM + 8 * c8]);
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
            uint16_t* orow = C.dst + size_t(y) * C.dst_pitch;
            const int ne = min(8, W - x);
            if (vec && ne == 8)
                *reinterpret_cast<uint4*>(orow + x) = v;
            for (int e = 0; e < ne; ++e) {
                const uint16_t d = uint16_t(w[e >> 1] >> (16 * (e & 1)));
                if (!(vec && ne == 8)) orow[x + e] = d;
                if (d == 0) s_list[atomicAdd(&s_n, 1)] = uint16_t(ty * kTileW + 8 * c8 + e);
            }
        }
    }
    __syncthreads();
    // phase 3: one listed pixel per thread at a time
    const int n_holes = s_n;
    for (int j = tid; j < n_holes; j += kThreads) {
        const int i = s_list[j];
        const int ty = i / kTileW, tx = i - ty * kTileW;
        const int cy = ty + R, cx = kDM + tx;                      // centre in the staged tile
        const uint32_t c0 = s_cc[cy][cx];
        float acc = 0.0f, wsum = 0.0f;
        int n = 0;
#pragma unroll
        for (int dy = -R; dy <= R; ++dy) {
#pragma unroll
            for (int dx = -R; dx <= R; ++dx) {
                const float qf = s_df[cy + dy][cx + dx];
                if (qf < 0.0f)
                    continue;
                const uint32_t ad = __vabsdiffu4(c0, s_cc[cy + dy][cx + dx]);   // |dR|, |dG|, |dB| bytes
                const float w = __fmul_rn(__fmul_rn(__fmul_rn(s_ws[(dy + R) * side + (dx + R)], s_wc[ad & 255u]),
                                                    s_wc[(ad >> 8) & 255u]),
                                          s_wc[(ad >> 16) & 255u]);
                acc = __fadd_rn(acc, __fmul_rn(w, qf));
                wsum = __fadd_rn(wsum, w);
                ++n;
            }
        }
        uint32_t out = 0u;
        if (n >= P.min_valid && wsum > 0.0f) {
            float v = floorf(__fadd_rn(__fdiv_rn(acc, wsum), 0.5f));
            v = fminf(fmaxf(v, float(P.d_lo)), float(P.d_hi));
            out = uint32_t(v);
        }
        if (out != 0u)
            C.dst[size_t(y0 + ty) * C.dst_pitch + (x0 + tx)] = uint16_t(out);
    }
}

}  // namespace

bool jbf_options_ok(const fvv_options& o, std::string* why)
{
    if (o.jbf_radius < 0 || o.jbf_radius > kJbfMaxRadius) {
        *why = "jbf_radius must be in [0, 7]";
        return false;
    }
    if (o.jbf_radius == 0) return true;
    if (!(o.jbf_sigma_s > 0.0f) || !std::isfinite(o.jbf_sigma_s) || !(o.jbf_sigma_c > 0.0f) ||
        !std::isfinite(o.jbf_sigma_c)) {
        *why = "jbf_sigma_s and jbf_sigma_c must be finite and > 0";
        return false;
    }
    const int side = 2 * o.jbf_radius + 1;
    if (o.jbf_min_valid < 1 || o.jbf_min_valid >= side * side) {
        *why = "jbf_min_valid must be in [1, (2 jbf_radius + 1)^2 - 1]";
        return false;
    }
    return true;
}

void jbf_params(const fvv_options& o, int width, int height, JbfParams* P)
{
    std::memset(P, 0, sizeof *P);
    P->width = width;
    P->height = height;
    P->radius = o.jbf_radius;
    P->min_valid = o.jbf_min_valid;
    P->d_lo = o.d_lo;
    P->d_hi = o.d_hi;
    const int R = o.jbf_radius, side = 2 * R + 1;
    const double ss = double(o.jbf_sigma_s), sc = double(o.jbf_sigma_c);
    for (int dy = -R; dy <= R; ++dy)
        for (int dx = -R; dx <= R; ++dx)
            P->s[(dy + R) * side + (dx + R)] = float(std::exp(-double(dx * dx + dy * dy) / (2.0 * ss * ss)));
    for (int t = 0; t < 256; ++t) P->c[t] = float(std::exp(-double(t * t) / (2.0 * sc * sc)));
}

cudaError_t launch_jbf(const JbfParams& P_in, int n_cams, cudaStream_t stream)
{
    if (n_cams <= 0 || P_in.width <= 0 || P_in.height <= 0) return cudaSuccess;
    if (n_cams > kJbfMaxCams) return cudaErrorInvalidValue;
    // 16-byte accesses where every row of a camera starts 16-byte aligned
    // (a tile's first column sits 128 code bytes and 192 colour bytes on)
    JbfParams P = P_in;
    auto a16 = [](const void* p, int64_t pitch_bytes) {
        return (reinterpret_cast<uintptr_t>(p) & 15u) == 0 && pitch_bytes % 16 == 0;
    };
    for (int k = 0; k < n_cams; ++k) {
        JbfCam& c = P.cam[k];
        c.vec = a16(c.rgb, c.rgb_pitch) && a16(c.src, c.src_pitch * 2) && a16(c.dst, c.dst_pitch * 2) ? 1 : 0;
    }
    dim3 grid(unsigned((P.width + kTileW - 1) / kTileW), unsigned((P.height + kTileH - 1) / kTileH),
              unsigned(n_cams));
    switch (P.radius) {
    case 1: k_jbf<1><<<grid, kThreads, 0, stream>>>(P); break;
    case 2: k_jbf<2><<<grid, kThreads, 0, stream>>>(P); break;
    case 3: k_jbf<3><<<grid, kThreads, 0, stream>>>(P); break;
    case 4: k_jbf<4><<<grid, kThreads, 0, stream>>>(P); break;
    case 5: k_jbf<5><<<grid, kThreads, 0, stream>>>(P); break;
    case 6: k_jbf<6><<<grid, kThreads, 0, stream>>>(P); break;
    case 7: k_jbf<7><<<grid, kThreads, 0, stream>>>(P); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace fvv

using fvv::fail;

extern "C" fvv_status fvv_depth_jbf(const uint8_t* rgb, size_t rgb_pitch, const uint16_t* depth, size_t depth_pitch,
                                    uint16_t* out, size_t out_pitch, int32_t width, int32_t height,
                                    const fvv_options* opt, void* stream)
{
    if (!rgb || !depth || !out || !opt) return fail(FVV_ERR_INVALID_ARG, "fvv_depth_jbf: NULL argument");
    if (width < 1 || height < 1) return fail(FVV_ERR_INVALID_ARG, "fvv_depth_jbf: width and height must be >= 1");
    std::string why;
    if (!fvv::jbf_options_ok(*opt, &why)) return fail(FVV_ERR_INVALID_ARG, "fvv_depth_jbf: " + why);
    if (opt->jbf_radius == 0) return fail(FVV_ERR_INVALID_ARG, "fvv_depth_jbf: jbf_radius is 0 (filter off)");
    if (opt->d_lo < 1 || opt->d_hi > 65534 || opt->d_lo > opt->d_hi)
        return fail(FVV_ERR_INVALID_ARG, "fvv_depth_jbf: need 1 <= d_lo <= d_hi <= 65534");
    if (rgb_pitch < size_t(width) * 3 || depth_pitch < size_t(width) * 2 || depth_pitch % 2 ||
        out_pitch < size_t(width) * 2 || out_pitch % 2 || (reinterpret_cast<uintptr_t>(depth) & 1) ||
        (reinterpret_cast<uintptr_t>(out) & 1))
        return fail(FVV_ERR_INVALID_ARG, "fvv_depth_jbf: bad pitch or alignment");
    const size_t ib = depth_pitch * size_t(height - 1) + size_t(width) * 2;
    const size_t ob = out_pitch * size_t(height - 1) + size_t(width) * 2;
    const uintptr_t i0 = reinterpret_cast<uintptr_t>(depth), o0 = reinterpret_cast<uintptr_t>(out);
    if (i0 < o0 + ob && o0 < i0 + ib)
        return fail(FVV_ERR_INVALID_ARG, "fvv_depth_jbf: out must not overlap depth (the filter is out of place)");
    for (const void* p : {static_cast<const void*>(rgb), static_cast<const void*>(depth),
                          static_cast<const void*>(out)})
        if (fvv::mem_kind(p) != fvv::MemKind::Device)
            return fail(FVV_ERR_INVALID_ARG, "fvv_depth_jbf: buffers must be device memory");
    fvv::JbfParams P;
    fvv::jbf_params(*opt, width, height, &P);
    P.cam[0].rgb = rgb;
    P.cam[0].rgb_pitch = int64_t(rgb_pitch);
    P.cam[0].src = depth;
    P.cam[0].src_pitch = int64_t(depth_pitch / 2);
    P.cam[0].dst = out;
    P.cam[0].dst_pitch = int64_t(out_pitch / 2);
    cudaError_t e = fvv::launch_jbf(P, 1, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(FVV_ERR_CUDA, std::string("fvv_depth_jbf: ") + cudaGetErrorString(e));
    }
    return FVV_OK;
}
