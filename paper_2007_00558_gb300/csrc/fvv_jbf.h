// fvv_jbf.h -- the joint bilateral depth pre-filter (fvv_jbf.cu).
#pragma once

#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "fvv.h"

namespace fvv {

constexpr int kJbfMaxRadius = 7;
constexpr int kJbfMaxCams = 64;

// One camera's frame: guidance colour (RGB8 rows), unfiltered codes and
// the output (pitches of the code rows in elements).
struct JbfCam {
    const uint8_t* rgb;
    int64_t rgb_pitch;          // bytes
    const uint16_t* src;
    int64_t src_pitch;
    uint16_t* dst;
    int64_t dst_pitch;
    int32_t vec;                // 1: rgb, src and dst rows all start 16-byte aligned (set by launch_jbf)
    int32_t pad;
};

// Everything a launch needs, passed by value: the weight tables (FP32,
// evaluated in FP64 on the host) and the cameras of the launch.
struct JbfParams {
    float s[(2 * kJbfMaxRadius + 1) * (2 * kJbfMaxRadius + 1)];   // [dy + r][dx + r], row stride 2r + 1
    float c[256];                                                 // colour weight of a channel difference
    int32_t width, height, radius, min_valid;
    uint32_t d_lo, d_hi;
    JbfCam cam[kJbfMaxCams];
};

bool jbf_options_ok(const fvv_options& o, std::string* why);
// Tables and scalars from the options (cameras left zero).
void jbf_params(const fvv_options& o, int width, int height, JbfParams* P);
// One launch over cameras cam[0 .. n_cams) of equal size, asynchronous.
cudaError_t launch_jbf(const JbfParams& P, int n_cams, cudaStream_t stream);

}  // namespace fvv
