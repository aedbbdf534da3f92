// backward_internal.h -- the adjoint passes as the entry points call them (not public).
#pragma once

#include "internal.h"

namespace imcl {

struct BwdArgs {
    ConvCall fwd;                 // the forward call: input image, taps, boundary rule
    const float* g = nullptr;     // upstream gradient (f32), pitch in bytes
    int64_t g_pitch_b = 0;
    float* dx = nullptr;          // input gradient (f32) or nullptr
    int64_t dx_pitch_b = 0;
    float* dw0 = nullptr;         // conv2d: taps; sepconv: row taps; harris: Sobel x
    float* dw1 = nullptr;         // sepconv: column taps; harris: Sobel y
    float* dw2 = nullptr;         // harris: window
    void* workspace = nullptr;
    size_t ws_bytes = 0;
};

size_t conv2d_backward_ws(int W, int H, int kw, int kh);
size_t sepconv_backward_ws(int W, int H, int nr, int nc);
size_t harris_backward_ws(int W, int H, int wk);
imcl_status conv2d_backward_run(const BwdArgs& b, cudaStream_t s);
imcl_status sepconv_backward_run(const BwdArgs& b, cudaStream_t s);
imcl_status harris_backward_run(const BwdArgs& b, cudaStream_t s);

}  // namespace imcl
