// abi_harris.cu -- imagecl_harris: argument checks and variant selection.
#include <string>

#include "abi_internal.h"

namespace imcl {

// Harris calls keep the caller's window side in kh and the side of the kernels that run
// it in kw: equal for odd windows; an even window runs as the next odd one with a zero
// last row and column (tap (j, i) keeps its offset (i - wk/2, j - wk/2)).
int harris_kernel_side(int wk) { return wk % 2 ? wk : wk + 1; }

// The forward has its own kernels for the paper's 2x2 block (and the untuned kernel takes
// any side): only even windows above 2 run as the next odd one.
int harris_forward_side(int wk) { return wk == 2 ? 2 : harris_kernel_side(wk); }

ConvCall harris_problem_call(const imcl_problem& p) {
    ConvCall c = problem_call(p);
    c.in_dtype = c.out_dtype = IMCL_F32;
    c.kh = p.kw;
    c.kw = harris_forward_side(p.kw);
    return c;
}

imcl_problem harris_problem(const ConvCall& c) {
    imcl_problem p = conv_problem(c);
    p.op = IMCL_OP_HARRIS;
    p.kw = p.kh = c.kh;
    return p;
}

std::vector<const ConvEntry*> harris_entries_for(int wk, int taps_mem) {
    std::vector<const ConvEntry*> r;
    for (const ConvEntry& e : harris_table()) {
        if (e.v.kind == IMCL_KIND_PLAIN) { r.push_back(&e); continue; }
        if (e.k != wk) continue;
        if (taps_mem == IMCL_MEM_DEVICE && e.v.filt != IMCL_FILT_SMEM) continue;
        r.push_back(&e);
    }
    return r;
}

static const ConvEntry* harris_find(const ConvCall& c, const imcl_variant& v) {
    for (const ConvEntry* e : harris_entries_for(c.kw, c.taps_mem)) {
        if (v.kind == IMCL_KIND_PLAIN && e->v.kind == IMCL_KIND_PLAIN) return e;
        if (e->v.kind == v.kind && e->v.py == v.py && e->v.load == v.load && e->v.filt == v.filt) return e;
    }
    return nullptr;
}

imcl_variant harris_default_variant(const ConvCall& c) {
    imcl_variant v{};
    if (cache_lookup(harris_problem(c), &v)) return v;
    return pick_default(harris_entries_for(c.kw, c.taps_mem), c.taps_mem, tma_aligned(c), 4, 2);
}

imcl_status harris_prepare(const imcl_image* in, const imcl_image* out, const float* sx, const float* sy,
                           const float* win, int wk, float k, int taps_mem, void* ws, size_t ws_bytes,
                           ConvCall* c) {
    imcl_status st;
    if ((st = check_image(in, "in")) != IMCL_OK) return st;
    if ((st = check_image(out, "out")) != IMCL_OK) return st;
    if (in->width != out->width || in->height != out->height)
        return fail(IMCL_ERR_INVALID, "in and out must have the same width and height");
    if (images_overlap(in, out)) return fail(IMCL_ERR_INVALID, "in and out overlap (operations are out of place)");
    if (in->dtype != IMCL_F32 || out->dtype != IMCL_F32)
        return fail(IMCL_ERR_UNSUPPORTED, "harris takes an f32 image and writes f32");
    if (wk <= 0) return fail(IMCL_ERR_INVALID, "window side must be positive");
    if (wk > 7) return fail(IMCL_ERR_UNSUPPORTED, "window side above 7 is not provided");
    if (!sx || !sy || !win) return fail(IMCL_ERR_INVALID, "sobel_x, sobel_y and window must not be NULL");
    if (taps_mem != IMCL_MEM_HOST && taps_mem != IMCL_MEM_DEVICE)
        return fail(IMCL_ERR_INVALID, "taps_mem must be IMCL_MEM_HOST or IMCL_MEM_DEVICE");
    if (!(k == k)) return fail(IMCL_ERR_INVALID, "k must be a number");
    DeviceInfo* dev = nullptr;
    if ((st = device_info(&dev)) != IMCL_OK) return st;
    c->in = in->data;
    c->out = out->data;
    c->in_dtype = IMCL_F32;
    c->out_dtype = IMCL_F32;
    c->W = in->width;
    c->H = in->height;
    c->in_pitch_b = in->pitch_bytes;
    c->out_pitch_b = out->pitch_bytes;
    c->kw = harris_forward_side(wk);
    c->kh = wk;
    c->taps = sx;
    c->taps2 = sy;
    c->taps3 = win;
    c->hk = k;
    c->taps_mem = taps_mem;
    c->border = IMCL_BORDER_CLAMP;
    c->workspace = ws;
    c->ws_bytes = ws_bytes;
    c->status = dev->status;
    c->dev = dev;
    return IMCL_OK;
}

imcl_status harris_run(const ConvCall& c, const imcl_variant* variant, cudaStream_t s) {
    imcl_variant v = variant ? *variant : harris_default_variant(c);
    const ConvEntry* e = harris_find(c, v);
    if (!e) return fail(IMCL_ERR_UNSUPPORTED, "no compiled harris variant matches the request");
    if (v.kind == IMCL_KIND_TILED && (v.bx <= 0 || v.by <= 0)) { v.bx = e->v.bx; v.by = e->v.by; }
    return e->fn(c, v, s);
}

}  // namespace imcl

using namespace imcl;

extern "C" {

imcl_status imagecl_harris(const imcl_image* in, const imcl_image* out, const float* sobel_x, const float* sobel_y,
                           const float* window, int32_t wk, float k, int32_t taps_mem, const imcl_variant* variant,
                           void* workspace, size_t workspace_bytes, void* stream) {
    ConvCall c;
    imcl_status st = harris_prepare(in, out, sobel_x, sobel_y, window, wk, k, taps_mem, workspace,
                                    workspace_bytes, &c);
    if (st != IMCL_OK) return st;
    return harris_run(c, variant, static_cast<cudaStream_t>(stream));
}

size_t imagecl_harris_workspace_size(const imcl_problem* problem, const imcl_variant* variant) {
    if (!problem || problem->width <= 0 || problem->height <= 0) return 0;
    imcl_problem q = *problem;
    q.in_dtype = q.out_dtype = IMCL_F32;
    const imcl_variant v = variant ? *variant : harris_default_variant(harris_problem_call(q));
    if (v.kind == IMCL_KIND_PLAIN) return (size_t)2 * problem->width * (size_t)problem->height * sizeof(float);
    return 0;
}

}  // extern "C"
