// abi.cu -- the extern "C" entry points: argument checks, variant selection and the
// tuning cache.  No exception crosses this boundary.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>

#include "abi_internal.h"

namespace imcl {

const char* last_error_text();
void clear_last_error();

imcl_status check_image(const imcl_image* im, const char* name) {
    if (!im) return fail(IMCL_ERR_INVALID, std::string(name) + " is NULL");
    if (!im->data) return fail(IMCL_ERR_INVALID, std::string(name) + ".data is NULL");
    if (im->width <= 0 || im->height <= 0)
        return fail(IMCL_ERR_INVALID, std::string(name) + " has a non-positive width or height");
    const int sz = dtype_size(im->dtype);
    if (sz == 0) return fail(IMCL_ERR_INVALID, std::string(name) + " has an unknown dtype");
    if (im->reserved != 0) return fail(IMCL_ERR_INVALID, std::string(name) + ".reserved must be 0");
    if (im->pitch_bytes < (int64_t)im->width * sz || im->pitch_bytes % sz != 0)
        return fail(IMCL_ERR_INVALID, std::string(name) + ".pitch_bytes must be >= width*elemsize and a multiple of it");
    if ((reinterpret_cast<uintptr_t>(im->data) % sz) != 0)
        return fail(IMCL_ERR_ALIGN, std::string(name) + ".data is not aligned to its element size");
    return IMCL_OK;
}

static void byte_range(const imcl_image* im, uintptr_t* lo, uintptr_t* hi) {
    *lo = reinterpret_cast<uintptr_t>(im->data);
    *hi = *lo + (uintptr_t)(im->pitch_bytes * (im->height - 1) + (int64_t)im->width * dtype_size(im->dtype));
}

bool images_overlap(const imcl_image* a, const imcl_image* b) {
    uintptr_t a0, a1, b0, b1;
    byte_range(a, &a0, &a1);
    byte_range(b, &b0, &b1);
    return a0 < b1 && b0 < a1;
}

imcl_status check_border(int border, double bv, int in_dtype) {
    if (border != IMCL_BORDER_CLAMP && border != IMCL_BORDER_CONSTANT)
        return fail(IMCL_ERR_INVALID, "border must be IMCL_BORDER_CLAMP or IMCL_BORDER_CONSTANT");
    if (border == IMCL_BORDER_CONSTANT) {
        if (!std::isfinite(bv)) return fail(IMCL_ERR_INVALID, "border_value must be finite");
        if (in_dtype == IMCL_U8 && (bv != std::floor(bv) || bv < 0 || bv > 255))
            return fail(IMCL_ERR_INVALID, "border_value for a u8 image must be an integer in 0..255");
        if (in_dtype == IMCL_I32 && (bv != std::floor(bv) || bv < -2147483648.0 || bv > 2147483647.0))
            return fail(IMCL_ERR_INVALID, "border_value for an i32 image must be an int32");
    }
    return IMCL_OK;
}

imcl_status check_side(int k, const char* what) {
    if (k <= 0) return fail(IMCL_ERR_INVALID, std::string(what) + " must be positive");
    if (k % 2 == 0) return fail(IMCL_ERR_UNSUPPORTED, std::string(what) + " must be odd (centred taps)");
    if (k > kMaxK) return fail(IMCL_ERR_UNSUPPORTED, std::string(what) + " above 15 is not provided");
    return IMCL_OK;
}

// ------------------------------------------------------------------ tuning cache
static std::mutex g_cache_mu;
static std::map<std::string, imcl_variant> g_cache;

static int size_bucket(int w, int h) {
    double px = (double)w * (double)h;
    int b = 0;
    while (px >= 2.0) { px /= 2.0; ++b; }
    return b;
}

std::string problem_key(const imcl_problem& p) {
    char buf[200];
    snprintf(buf, sizeof buf, "op=%d in=%d out=%d kw=%d kh=%d border=%d mem=%d size=%d", p.op, p.in_dtype,
             p.out_dtype, p.kw, p.kh, p.border, p.taps_mem, size_bucket(p.width, p.height));
    return buf;
}

bool cache_lookup(const imcl_problem& p, imcl_variant* v) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto it = g_cache.find(problem_key(p));
    if (it == g_cache.end()) return false;
    *v = it->second;
    return true;
}

void cache_store(const imcl_problem& p, const imcl_variant& v) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    g_cache[problem_key(p)] = v;
}

// ------------------------------------------------------------------ conv2d variants
imcl_problem conv_problem(const ConvCall& c) {
    imcl_problem p{};
    p.op = IMCL_OP_CONV2D;
    p.in_dtype = c.in_dtype;
    p.out_dtype = c.out_dtype;
    p.kw = c.kw;
    p.kh = c.kh;
    p.width = c.W;
    p.height = c.H;
    p.border = c.border;
    p.taps_mem = c.taps_mem;
    return p;
}

static bool same_axes(const imcl_variant& a, const imcl_variant& b) {
    return a.kind == b.kind && a.px == b.px && a.py == b.py && a.load == b.load && a.filt == b.filt &&
           a.map == b.map && a.unroll == b.unroll;
}

std::vector<const ConvEntry*> conv_entries_for(int in_dt, int out_dt, int kw, int kh, int taps_mem) {
    std::vector<const ConvEntry*> r;
    for (const ConvEntry& e : conv_table()) {
        if (e.in_dtype != in_dt || e.out_dtype != out_dt) continue;
        if (e.v.kind == IMCL_KIND_PLAIN) { r.push_back(&e); continue; }
        if (kw != kh || e.k != kw) continue;
        if (taps_mem == IMCL_MEM_DEVICE && e.v.filt != IMCL_FILT_SMEM) continue;
        r.push_back(&e);
    }
    return r;
}

const ConvEntry* conv_find(const ConvCall& c, const imcl_variant& v) {
    for (const ConvEntry* e : conv_entries_for(c.in_dtype, c.out_dtype, c.kw, c.kh, c.taps_mem))
        if (same_axes(e->v, v) || (v.kind == IMCL_KIND_PLAIN && e->v.kind == IMCL_KIND_PLAIN)) return e;
    return nullptr;
}

imcl_variant pick_default(const std::vector<const ConvEntry*>& entries, int taps_mem, bool tma_ok, int want_px,
                          int want_py) {
    const int filt = taps_mem == IMCL_MEM_DEVICE ? IMCL_FILT_SMEM : IMCL_FILT_PARAM;
    auto ok = [&](const ConvEntry* e) {
        return e->v.kind == IMCL_KIND_TILED && e->v.filt == filt && e->v.map == IMCL_MAP_BLOCKED &&
               (tma_ok || e->v.load != IMCL_LOAD_TMA);
    };
    const int first = tma_ok ? IMCL_LOAD_TMA : IMCL_LOAD_GLOBAL;
    // the preferred coarsening with TMA staging when the buffers allow it, else the L1 path
    for (const ConvEntry* e : entries)
        if (ok(e) && e->v.py == want_py && (want_px <= 0 || e->v.px == want_px) && e->v.load == first) return e->v;
    for (const ConvEntry* e : entries)
        if (ok(e) && e->v.py == want_py && (want_px <= 0 || e->v.px == want_px)) return e->v;
    // any feasible tiled variant, the L1 path before cooperative staging
    for (int load : {first, (int)IMCL_LOAD_GLOBAL, (int)IMCL_LOAD_SMEM})
        for (const ConvEntry* e : entries)
            if (ok(e) && e->v.load == load) return e->v;
    for (const ConvEntry* e : entries)
        if (e->v.kind == IMCL_KIND_PLAIN) return e->v;
    imcl_variant none{};
    none.kind = -1;
    return none;
}

ConvCall problem_call(const imcl_problem& p) {
    ConvCall c;
    c.in = reinterpret_cast<const void*>(uintptr_t(256));
    c.out = reinterpret_cast<void*>(uintptr_t(512));
    c.in_dtype = p.in_dtype;
    c.out_dtype = p.out_dtype;
    c.W = p.width;
    c.H = p.height;
    c.in_pitch_b = ((int64_t)p.width * dtype_size(p.in_dtype) + 127) / 128 * 128;
    c.out_pitch_b = ((int64_t)p.width * dtype_size(p.out_dtype) + 127) / 128 * 128;
    c.kw = p.kw;
    c.kh = p.kh;
    c.taps_mem = p.taps_mem;
    c.border = p.border;
    return c;
}

bool tma_aligned(const ConvCall& c) {
    return (reinterpret_cast<uintptr_t>(c.in) % 16) == 0 && (c.in_pitch_b % 16) == 0;
}

imcl_variant conv_default_variant(const ConvCall& c) {
    imcl_variant v{};
    if (cache_lookup(conv_problem(c), &v)) return v;
    return pick_default(conv_entries_for(c.in_dtype, c.out_dtype, c.kw, c.kh, c.taps_mem), c.taps_mem,
                        tma_aligned(c), 4, 4);
}

imcl_status conv_prepare(const imcl_image* in, const imcl_image* out, const void* taps, int taps_dtype,
                         int kw, int kh, int taps_mem, int border, double bv, ConvCall* c) {
    imcl_status st;
    if ((st = check_image(in, "in")) != IMCL_OK) return st;
    if ((st = check_image(out, "out")) != IMCL_OK) return st;
    if (in->width != out->width || in->height != out->height)
        return fail(IMCL_ERR_INVALID, "in and out must have the same width and height");
    if (images_overlap(in, out)) return fail(IMCL_ERR_INVALID, "in and out overlap (operations are out of place)");
    if ((st = check_side(kw, "kw")) != IMCL_OK) return st;
    if ((st = check_side(kh, "kh")) != IMCL_OK) return st;
    if (!taps) return fail(IMCL_ERR_INVALID, "taps is NULL");
    if (taps_mem != IMCL_MEM_HOST && taps_mem != IMCL_MEM_DEVICE)
        return fail(IMCL_ERR_INVALID, "taps_mem must be IMCL_MEM_HOST or IMCL_MEM_DEVICE");
    const bool int_in = is_int_dtype(in->dtype);
    if (int_in) {
        if (out->dtype != IMCL_I32) return fail(IMCL_ERR_INVALID, "integer images write an i32 output");
        if (taps_dtype != IMCL_I32) return fail(IMCL_ERR_INVALID, "integer images take i32 taps");
    } else {
        if (is_int_dtype(out->dtype)) return fail(IMCL_ERR_INVALID, "floating images write f32, f16 or bf16");
        if (taps_dtype != IMCL_F32) return fail(IMCL_ERR_INVALID, "floating images take f32 taps");
        if (out->dtype != IMCL_F32 && out->dtype != in->dtype)
            return fail(IMCL_ERR_UNSUPPORTED, "floating images write f32 or their own 16-bit type");
    }
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
    c->kw = kw;
    c->kh = kh;
    c->taps = taps;
    c->taps_mem = taps_mem;
    c->border = border;
    c->border_value = bv;
    c->status = dev->status;
    c->dev = dev;
    return IMCL_OK;
}

imcl_status conv_run(const ConvCall& c, const imcl_variant* variant, cudaStream_t s) {
    imcl_variant v = variant ? *variant : conv_default_variant(c);
    const ConvEntry* e = conv_find(c, v);
    if (!e) return fail(IMCL_ERR_UNSUPPORTED, "no compiled conv2d variant matches the request");
    if (v.kind == IMCL_KIND_TILED && (v.bx <= 0 || v.by <= 0)) { v.bx = e->v.bx; v.by = e->v.by; }
    return e->fn(c, v, s);
}

}  // namespace imcl

using namespace imcl;

extern "C" {

imcl_status imagecl_conv2d(const imcl_image* in, const imcl_image* out, const void* taps, int32_t taps_dtype,
                           int32_t kw, int32_t kh, int32_t taps_mem, int32_t border, double border_value,
                           const imcl_variant* variant, void* stream) {
    ConvCall c;
    imcl_status st = conv_prepare(in, out, taps, taps_dtype, kw, kh, taps_mem, border, border_value, &c);
    if (st != IMCL_OK) return st;
    return conv_run(c, variant, static_cast<cudaStream_t>(stream));
}

const char* imagecl_last_error(void) { return last_error_text(); }

imcl_status imagecl_device_status(int32_t* code, void* stream) {
    if (!code) return fail(IMCL_ERR_INVALID, "code is NULL");
    DeviceInfo* dev = nullptr;
    imcl_status st = device_info(&dev);
    if (st != IMCL_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    int h = 0;
    e = cudaMemcpy(&h, dev->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "status word read");
    e = cudaMemset(dev->status, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "status word reset");
    *code = h;
    return h == 0 ? IMCL_OK : fail(IMCL_ERR_TIMEOUT, "a kernel gave up on a bounded wait or check");
}

const char* imagecl_version(void) { return "imagecl-gb300 0.1 sm_103a"; }

void imagecl_tune_clear(void) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    g_cache.clear();
}

imcl_status imagecl_tune_set(const imcl_problem* p, const imcl_variant* v) {
    if (!p || !v) return fail(IMCL_ERR_INVALID, "problem and variant must not be NULL");
    cache_store(*p, *v);
    return IMCL_OK;
}

imcl_status imagecl_tune_save(const char* path) {
    if (!path) return fail(IMCL_ERR_INVALID, "path is NULL");
    DeviceInfo* dev = nullptr;
    imcl_status st = device_info(&dev);
    if (st != IMCL_OK) return st;
    std::ofstream f(path);
    if (!f) return fail(IMCL_ERR_INVALID, std::string("cannot write ") + path);
    f << "# imagecl tuning cache\tdevice=" << dev->name << "\tsms=" << dev->sm_count << "\n";
    std::lock_guard<std::mutex> lk(g_cache_mu);
    for (auto& kv : g_cache) {
        const imcl_variant& v = kv.second;
        f << kv.first << "\t" << v.kind << " " << v.bx << " " << v.by << " " << v.px << " " << v.py << " "
          << v.load << " " << v.filt << " " << v.map << " " << v.unroll << " " << v.persistent << "\n";
    }
    return f.good() ? IMCL_OK : fail(IMCL_ERR_INVALID, "write failed");
}

imcl_status imagecl_tune_load(const char* path) {
    if (!path) return fail(IMCL_ERR_INVALID, "path is NULL");
    DeviceInfo* dev = nullptr;
    imcl_status st = device_info(&dev);
    if (st != IMCL_OK) return st;
    std::ifstream f(path);
    if (!f) return fail(IMCL_ERR_INVALID, std::string("cannot read ") + path);
    std::string line;
    if (!std::getline(f, line)) return fail(IMCL_ERR_INVALID, "empty tuning cache file");
    std::ostringstream want;
    want << "device=" << dev->name << "\tsms=" << dev->sm_count;
    if (line.find(want.str()) == std::string::npos) return IMCL_OK;   // another device: nothing applies
    std::lock_guard<std::mutex> lk(g_cache_mu);
    while (std::getline(f, line)) {
        const size_t tab = line.find('\t');
        if (tab == std::string::npos) continue;
        imcl_variant v{};
        std::istringstream is(line.substr(tab + 1));
        if (is >> v.kind >> v.bx >> v.by >> v.px >> v.py >> v.load >> v.filt >> v.map >> v.unroll >> v.persistent)
            g_cache[line.substr(0, tab)] = v;
    }
    return IMCL_OK;
}

}  // extern "C"
