// abi_sepconv.cu -- imagecl_sepconv: argument checks and variant selection for the
// separable correlation.
#include <algorithm>
#include <string>

#include "abi_internal.h"

namespace imcl {

imcl_problem sep_problem(const ConvCall& c) {
    imcl_problem p = conv_problem(c);
    p.op = IMCL_OP_SEPCONV;
    return p;
}

std::vector<const ConvEntry*> sep_entries_for(int in_dt, int out_dt, int nr, int nc, int taps_mem) {
    std::vector<const ConvEntry*> r;
    // a single-tap pass on both axes (radius 0) runs on the radius-1 kernels, zero-padded
    const int R = std::max(1, (std::max(nr, nc) - 1) / 2);
    for (const ConvEntry& e : sep_table()) {
        if (e.in_dtype != in_dt || e.out_dtype != out_dt) continue;
        if (e.v.kind == IMCL_KIND_PLAIN) { r.push_back(&e); continue; }
        if (e.k != R) continue;
        if (taps_mem == IMCL_MEM_DEVICE && e.v.filt != IMCL_FILT_SMEM) continue;
        r.push_back(&e);
    }
    return r;
}

static const ConvEntry* sep_find(const ConvCall& c, const imcl_variant& v) {
    for (const ConvEntry* e : sep_entries_for(c.in_dtype, c.out_dtype, c.kw, c.kh, c.taps_mem)) {
        if (v.kind == IMCL_KIND_PLAIN && e->v.kind == IMCL_KIND_PLAIN) return e;
        if (e->v.kind == v.kind && e->v.px == v.px && e->v.py == v.py && e->v.load == v.load &&
            e->v.filt == v.filt && e->v.map == v.map && e->v.unroll == v.unroll)
            return e;
    }
    return nullptr;
}

imcl_variant sep_default_variant(const ConvCall& c) {
    imcl_variant v{};
    if (cache_lookup(sep_problem(c), &v)) return v;
    return pick_default(sep_entries_for(c.in_dtype, c.out_dtype, c.kw, c.kh, c.taps_mem), c.taps_mem,
                        tma_aligned(c), 4, 8);
}

imcl_status sep_prepare(const imcl_image* in, const imcl_image* out, const float* row, int nr, const float* col,
                        int nc, int taps_mem, int border, double bv, void* ws, size_t ws_bytes, ConvCall* c) {
    imcl_status st;
    if ((st = check_image(in, "in")) != IMCL_OK) return st;
    if ((st = check_image(out, "out")) != IMCL_OK) return st;
    if (in->width != out->width || in->height != out->height)
        return fail(IMCL_ERR_INVALID, "in and out must have the same width and height");
    if (images_overlap(in, out)) return fail(IMCL_ERR_INVALID, "in and out overlap (operations are out of place)");
    if (nr <= 0 || nc <= 0) return fail(IMCL_ERR_INVALID, "tap counts must be positive");
    if (nr % 2 == 0 || nc % 2 == 0) return fail(IMCL_ERR_UNSUPPORTED, "tap counts must be odd (centred taps)");
    if (nr > kMaxSepTaps || nc > kMaxSepTaps) return fail(IMCL_ERR_UNSUPPORTED, "more than 33 taps is not provided");
    if (!row || !col) return fail(IMCL_ERR_INVALID, "row_taps and col_taps must not be NULL");
    if (taps_mem != IMCL_MEM_HOST && taps_mem != IMCL_MEM_DEVICE)
        return fail(IMCL_ERR_INVALID, "taps_mem must be IMCL_MEM_HOST or IMCL_MEM_DEVICE");
    if (is_int_dtype(in->dtype)) return fail(IMCL_ERR_UNSUPPORTED, "sepconv takes f32, f16 or bf16 images");
    if (out->dtype != IMCL_F32 && out->dtype != in->dtype)
        return fail(IMCL_ERR_UNSUPPORTED, "floating images write f32 or their own 16-bit type");
    if ((st = check_border(border, bv, in->dtype)) != IMCL_OK) return st;
    DeviceInfo* dev = nullptr;
    if ((st = device_info(&dev)) != IMCL_OK) return st;
    c->in = in->data;
    c->out = out->data;
    c->in_dtype = in->dtype;
    c->out_dtype = out->dtype;
    c->W = in->width;
    c->H = in->height;
    c->in_pitch_b = in->pitch_bytes;
    c->out_pitch_b = out->pitch_bytes;
    c->kw = nr;
    c->kh = nc;
    c->taps = row;
    c->taps2 = col;
    c->taps_mem = taps_mem;
    c->border = border;
    c->border_value = bv;
    c->workspace = ws;
    c->ws_bytes = ws_bytes;
    c->status = dev->status;
    c->dev = dev;
    return IMCL_OK;
}

imcl_status sep_run(const ConvCall& c, const imcl_variant* variant, cudaStream_t s) {
    imcl_variant v = variant ? *variant : sep_default_variant(c);
    const ConvEntry* e = sep_find(c, v);
    if (!e) return fail(IMCL_ERR_UNSUPPORTED, "no compiled sepconv variant matches the request");
    if (v.kind == IMCL_KIND_TILED && (v.bx <= 0 || v.by <= 0)) { v.bx = e->v.bx; v.by = e->v.by; }
    return e->fn(c, v, s);
}

}  // namespace imcl

using namespace imcl;

extern "C" {

imcl_status imagecl_sepconv(const imcl_image* in, const imcl_image* out, const float* row_taps, int32_t nrow,
                            const float* col_taps, int32_t ncol, int32_t taps_mem, int32_t border,
                            double border_value, const imcl_variant* variant, void* workspace,
                            size_t workspace_bytes, void* stream) {
    ConvCall c;
    imcl_status st = sep_prepare(in, out, row_taps, nrow, col_taps, ncol, taps_mem, border, border_value,
                                 workspace, workspace_bytes, &c);
    if (st != IMCL_OK) return st;
    return sep_run(c, variant, static_cast<cudaStream_t>(stream));
}

size_t imagecl_sepconv_workspace_size(const imcl_problem* problem, const imcl_variant* variant) {
    if (!problem || problem->width <= 0 || problem->height <= 0) return 0;
    const imcl_variant v = variant ? *variant : sep_default_variant(problem_call(*problem));
    if (v.kind == IMCL_KIND_PLAIN) return (size_t)problem->width * (size_t)problem->height * sizeof(float);
    return 0;
}

}  // extern "C"
