// abi_backward.cu -- entry points of the adjoint (backward) passes: argument checks and
// workspace sizes.  The passes themselves are in backward.cu.
#include <string>

#include "abi_internal.h"
#include "backward_internal.h"

namespace imcl {

// Checks shared by the three backward calls; fills the forward description's image part.
static imcl_status bwd_common(const imcl_image* grad_out, const imcl_image* in, const imcl_image* grad_in,
                              void* ws, size_t ws_bytes, size_t ws_need, BwdArgs* b) {
    imcl_status st;
    if ((st = check_image(grad_out, "grad_out")) != IMCL_OK) return st;
    if ((st = check_image(in, "in")) != IMCL_OK) return st;
    if (grad_out->dtype != IMCL_F32) return fail(IMCL_ERR_UNSUPPORTED, "grad_out must be f32");
    if (in->dtype != IMCL_F32 && in->dtype != IMCL_F16 && in->dtype != IMCL_BF16)
        return fail(IMCL_ERR_UNSUPPORTED, "gradients are provided for f32, f16 and bf16 images");
    if (grad_out->width != in->width || grad_out->height != in->height)
        return fail(IMCL_ERR_INVALID, "grad_out and in must have the same width and height");
    if (grad_in) {
        if ((st = check_image(grad_in, "grad_in")) != IMCL_OK) return st;
        if (grad_in->dtype != IMCL_F32) return fail(IMCL_ERR_UNSUPPORTED, "grad_in must be f32");
        if (grad_in->width != in->width || grad_in->height != in->height)
            return fail(IMCL_ERR_INVALID, "grad_in must have the size of in");
        if (images_overlap(grad_in, grad_out) || images_overlap(grad_in, in))
            return fail(IMCL_ERR_INVALID, "grad_in overlaps grad_out or in");
    }
    if (!ws || ws_bytes < ws_need)
        return fail(IMCL_ERR_INVALID, "workspace missing or smaller than the *_backward_workspace_size query");
    DeviceInfo* dev = nullptr;
    if ((st = device_info(&dev)) != IMCL_OK) return st;
    ConvCall& c = b->fwd;
    c.in = in->data;
    c.in_dtype = in->dtype;
    c.out = nullptr;
    c.out_dtype = IMCL_F32;
    c.W = in->width;
    c.H = in->height;
    c.in_pitch_b = in->pitch_bytes;
    c.status = dev->status;
    c.dev = dev;
    b->g = static_cast<const float*>(grad_out->data);
    b->g_pitch_b = grad_out->pitch_bytes;
    if (grad_in) {
        b->dx = static_cast<float*>(grad_in->data);
        b->dx_pitch_b = grad_in->pitch_bytes;
    }
    b->workspace = ws;
    b->ws_bytes = ws_bytes;
    return IMCL_OK;
}

}  // namespace imcl

using namespace imcl;

extern "C" {

size_t imagecl_conv2d_backward_workspace_size(int32_t width, int32_t height, int32_t kw, int32_t kh) {
    if (width <= 0 || height <= 0 || kw <= 0 || kh <= 0) return 0;
    return conv2d_backward_ws(width, height, kw, kh);
}

size_t imagecl_sepconv_backward_workspace_size(int32_t width, int32_t height, int32_t nrow, int32_t ncol) {
    if (width <= 0 || height <= 0 || nrow <= 0 || ncol <= 0) return 0;
    return sepconv_backward_ws(width, height, nrow, ncol);
}

size_t imagecl_harris_backward_workspace_size(int32_t width, int32_t height, int32_t wk) {
    if (width <= 0 || height <= 0 || wk <= 0) return 0;
    return harris_backward_ws(width, height, harris_kernel_side(wk));
}

imcl_status imagecl_conv2d_backward(const imcl_image* grad_out, const imcl_image* in, const float* taps, int32_t kw,
                                    int32_t kh, int32_t taps_mem, int32_t border, double border_value,
                                    const imcl_image* grad_in, float* grad_taps, void* workspace,
                                    size_t workspace_bytes, void* stream) {
    imcl_status st;
    if ((st = check_side(kw, "kw")) != IMCL_OK) return st;
    if ((st = check_side(kh, "kh")) != IMCL_OK) return st;
    if (!taps) return fail(IMCL_ERR_INVALID, "taps is NULL");
    if (taps_mem != IMCL_MEM_HOST && taps_mem != IMCL_MEM_DEVICE)
        return fail(IMCL_ERR_INVALID, "taps_mem must be IMCL_MEM_HOST or IMCL_MEM_DEVICE");
    if (in && (st = check_border(border, border_value, in->dtype)) != IMCL_OK) return st;
    BwdArgs b;
    const size_t need = (in && in->width > 0 && in->height > 0) ? conv2d_backward_ws(in->width, in->height, kw, kh) : 0;
    if ((st = bwd_common(grad_out, in, grad_in, workspace, workspace_bytes, need, &b)) != IMCL_OK) return st;
    b.fwd.kw = kw;
    b.fwd.kh = kh;
    b.fwd.taps = taps;
    b.fwd.taps_mem = taps_mem;
    b.fwd.border = border;
    b.fwd.border_value = border_value;
    b.dw0 = grad_taps;
    return conv2d_backward_run(b, static_cast<cudaStream_t>(stream));
}

imcl_status imagecl_sepconv_backward(const imcl_image* grad_out, const imcl_image* in, const float* row_taps,
                                     int32_t nrow, const float* col_taps, int32_t ncol, int32_t taps_mem,
                                     int32_t border, double border_value, const imcl_image* grad_in,
                                     float* grad_row, float* grad_col, void* workspace, size_t workspace_bytes,
                                     void* stream) {
    if (nrow <= 0 || ncol <= 0) return fail(IMCL_ERR_INVALID, "tap counts must be positive");
    if (nrow % 2 == 0 || ncol % 2 == 0) return fail(IMCL_ERR_UNSUPPORTED, "tap counts must be odd (centred taps)");
    if (nrow > kMaxSepTaps || ncol > kMaxSepTaps) return fail(IMCL_ERR_UNSUPPORTED, "more than 33 taps is not provided");
    if (!row_taps || !col_taps) return fail(IMCL_ERR_INVALID, "row_taps and col_taps must not be NULL");
    if (taps_mem != IMCL_MEM_HOST && taps_mem != IMCL_MEM_DEVICE)
        return fail(IMCL_ERR_INVALID, "taps_mem must be IMCL_MEM_HOST or IMCL_MEM_DEVICE");
    imcl_status st;
    if (in && (st = check_border(border, border_value, in->dtype)) != IMCL_OK) return st;
    BwdArgs b;
    const size_t need = (in && in->width > 0 && in->height > 0) ? sepconv_backward_ws(in->width, in->height, nrow, ncol) : 0;
    if ((st = bwd_common(grad_out, in, grad_in, workspace, workspace_bytes, need, &b)) != IMCL_OK) return st;
    b.fwd.kw = nrow;
    b.fwd.kh = ncol;
    b.fwd.taps = row_taps;
    b.fwd.taps2 = col_taps;
    b.fwd.taps_mem = taps_mem;
    b.fwd.border = border;
    b.fwd.border_value = border_value;
    b.dw0 = grad_row;
    b.dw1 = grad_col;
    return sepconv_backward_run(b, static_cast<cudaStream_t>(stream));
}

imcl_status imagecl_harris_backward(const imcl_image* grad_out, const imcl_image* in, const float* sobel_x,
                                    const float* sobel_y, const float* window, int32_t wk, float k, int32_t taps_mem,
                                    const imcl_image* grad_in, float* grad_sobel_x, float* grad_sobel_y,
                                    float* grad_window, void* workspace, size_t workspace_bytes, void* stream) {
    if (wk <= 0) return fail(IMCL_ERR_INVALID, "window side must be positive");
    if (wk > 7) return fail(IMCL_ERR_UNSUPPORTED, "window side above 7 is not provided");
    if (!sobel_x || !sobel_y || !window) return fail(IMCL_ERR_INVALID, "sobel_x, sobel_y and window must not be NULL");
    if (taps_mem != IMCL_MEM_HOST && taps_mem != IMCL_MEM_DEVICE)
        return fail(IMCL_ERR_INVALID, "taps_mem must be IMCL_MEM_HOST or IMCL_MEM_DEVICE");
    if (in && in->dtype != IMCL_F32) return fail(IMCL_ERR_UNSUPPORTED, "harris takes an f32 image");
    imcl_status st;
    BwdArgs b;
    const size_t need =
        (in && in->width > 0 && in->height > 0) ? harris_backward_ws(in->width, in->height, harris_kernel_side(wk)) : 0;
    if ((st = bwd_common(grad_out, in, grad_in, workspace, workspace_bytes, need, &b)) != IMCL_OK) return st;
    b.fwd.kw = harris_kernel_side(wk);
    b.fwd.kh = wk;
    b.fwd.taps = sobel_x;
    b.fwd.taps2 = sobel_y;
    b.fwd.taps3 = window;
    b.fwd.hk = k;
    b.fwd.taps_mem = taps_mem;
    b.fwd.border = IMCL_BORDER_CLAMP;
    b.dw0 = grad_sobel_x;
    b.dw1 = grad_sobel_y;
    b.dw2 = grad_window;
    return harris_backward_run(b, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
