// tune_ops.cu -- what each operator gives the tuner: its variant list, its default
// variant, and a tuning job on scratch images of the problem's size.
#include <cmath>
#include <vector>

#include "tune_internal.h"

namespace imcl {

static ConvCall conv_call_for(const imcl_problem& p, const DeviceInfo* dev) {
    ConvCall c = problem_call(p);
    c.dev = dev;
    c.status = dev ? dev->status : nullptr;
    return c;
}

imcl_status list_variants(const imcl_problem& p, std::vector<imcl_variant>* out) {
    out->clear();
    if (p.op == IMCL_OP_CONV2D) {
        for (const ConvEntry* e : conv_entries_for(p.in_dtype, p.out_dtype, p.kw, p.kh, p.taps_mem))
            out->push_back(e->v);
        return IMCL_OK;
    }
    if (p.op == IMCL_OP_SEPCONV) {
        for (const ConvEntry* e : sep_entries_for(p.in_dtype, p.out_dtype, p.kw, p.kh, p.taps_mem))
            out->push_back(e->v);
        return IMCL_OK;
    }
    if (p.op == IMCL_OP_HARRIS) {
        for (const ConvEntry* e : harris_entries_for(harris_forward_side(p.kw), p.taps_mem)) out->push_back(e->v);
        return IMCL_OK;
    }
    return fail(IMCL_ERR_UNSUPPORTED, "unknown op");
}

imcl_status default_variant(const imcl_problem& p, imcl_variant* out) {
    if (p.op == IMCL_OP_CONV2D) {
        DeviceInfo* dev = nullptr;
        imcl_status st = device_info(&dev);
        if (st != IMCL_OK) return st;
        *out = conv_default_variant(conv_call_for(p, dev));
        if (out->kind < 0) return fail(IMCL_ERR_UNSUPPORTED, "no conv2d variant for this problem");
        return IMCL_OK;
    }
    if (p.op == IMCL_OP_SEPCONV) {
        DeviceInfo* dev = nullptr;
        imcl_status st = device_info(&dev);
        if (st != IMCL_OK) return st;
        *out = sep_default_variant(conv_call_for(p, dev));
        if (out->kind < 0) return fail(IMCL_ERR_UNSUPPORTED, "no sepconv variant for this problem");
        return IMCL_OK;
    }
    if (p.op == IMCL_OP_HARRIS) {
        DeviceInfo* dev = nullptr;
        imcl_status st = device_info(&dev);
        if (st != IMCL_OK) return st;
        ConvCall c = harris_problem_call(p);
        c.dev = dev;
        c.status = dev->status;
        *out = harris_default_variant(c);
        if (out->kind < 0) return fail(IMCL_ERR_UNSUPPORTED, "no harris variant for this problem");
        return IMCL_OK;
    }
    return fail(IMCL_ERR_UNSUPPORTED, "unknown op");
}

static imcl_status make_conv_job(const imcl_problem& p, cudaStream_t s, TuneJob* job) {
    imcl_status st;
    if ((st = check_side(p.kw, "kw")) != IMCL_OK) return st;
    if ((st = check_side(p.kh, "kh")) != IMCL_OK) return st;
    DeviceInfo* dev = nullptr;
    if ((st = device_info(&dev)) != IMCL_OK) return st;
    ConvCall c = conv_call_for(p, dev);
    void* in = nullptr;
    void* out = nullptr;
    if ((st = job->scratch.image(p.in_dtype, p.width, p.height, 1605u, &in, &c.in_pitch_b, s)) != IMCL_OK) return st;
    if ((st = job->scratch.image(p.out_dtype, p.width, p.height, 7u, &out, &c.out_pitch_b, s)) != IMCL_OK) return st;
    c.in = in;
    c.out = out;
    const int n = p.kw * p.kh;
    double l1 = 0;
    if (is_int_dtype(p.in_dtype)) {
        for (int i = 0; i < n; ++i) job->taps_i.push_back((int32_t)((i * 37 + 11) % 9) - 4);
        for (int v : job->taps_i) l1 += std::abs(v);
        l1 *= 255.0;
    } else {
        for (int i = 0; i < n; ++i) job->taps_f.push_back(std::sin(1.0 + 3.7 * i));
        for (float v : job->taps_f) l1 += std::fabs(v);
    }
    const void* host = is_int_dtype(p.in_dtype) ? (const void*)job->taps_i.data() : (const void*)job->taps_f.data();
    if (p.taps_mem == IMCL_MEM_DEVICE) {
        void* d = nullptr;
        if ((st = job->scratch.alloc(&d, n * 4)) != IMCL_OK) return st;
        cudaError_t e = cudaMemcpy(d, host, n * 4, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "tuner: taps upload");
        c.taps = d;
    } else {
        c.taps = host;
    }
    job->conv = c;
    std::vector<imcl_variant> base;
    for (const ConvEntry* e : conv_entries_for(p.in_dtype, p.out_dtype, p.kw, p.kh, p.taps_mem))
        base.push_back(e->v);
    job->candidates = expand_shapes(base);
    job->run = [job](const imcl_variant& v, cudaStream_t st2) { return conv_run(job->conv, &v, st2); };
    job->out = out;
    job->out_dtype = p.out_dtype;
    job->W = p.width;
    job->H = p.height;
    job->out_pitch_b = c.out_pitch_b;
    job->working_set_bytes = (double)c.in_pitch_b * p.height + (double)c.out_pitch_b * p.height;
    if (p.out_dtype == IMCL_F16) job->tol_abs = (float)(l1 * std::ldexp(1.0, -9));
    else if (p.out_dtype == IMCL_BF16) job->tol_abs = (float)(l1 * std::ldexp(1.0, -6));
    else job->tol_abs = (float)(l1 * 1e-5);
    return IMCL_OK;
}

static imcl_status make_sep_job(const imcl_problem& p, cudaStream_t s, TuneJob* job) {
    if (p.kw <= 0 || p.kh <= 0 || p.kw % 2 == 0 || p.kh % 2 == 0 || p.kw > kMaxSepTaps || p.kh > kMaxSepTaps)
        return fail(IMCL_ERR_UNSUPPORTED, "sepconv tap counts must be odd, 1..33");
    imcl_status st;
    DeviceInfo* dev = nullptr;
    if ((st = device_info(&dev)) != IMCL_OK) return st;
    ConvCall c = conv_call_for(p, dev);
    void *in = nullptr, *out = nullptr, *ws = nullptr;
    if ((st = job->scratch.image(p.in_dtype, p.width, p.height, 1605u, &in, &c.in_pitch_b, s)) != IMCL_OK) return st;
    if ((st = job->scratch.image(p.out_dtype, p.width, p.height, 7u, &out, &c.out_pitch_b, s)) != IMCL_OK) return st;
    const size_t ws_bytes = (size_t)p.width * p.height * sizeof(float);
    if ((st = job->scratch.alloc(&ws, ws_bytes)) != IMCL_OK) return st;
    c.in = in;
    c.out = out;
    c.workspace = ws;
    c.ws_bytes = ws_bytes;
    double l1r = 0, l1c = 0;
    for (int i = 0; i < p.kw; ++i) { job->taps_f.push_back(std::cos(0.3 * (i - p.kw / 2))); l1r += std::fabs(job->taps_f.back()); }
    for (int j = 0; j < p.kh; ++j) { job->taps_f.push_back(std::cos(0.2 * (j - p.kh / 2))); l1c += std::fabs(job->taps_f.back()); }
    const double l1 = l1r * l1c;
    if (p.taps_mem == IMCL_MEM_DEVICE) {
        void* d = nullptr;
        if ((st = job->scratch.alloc(&d, job->taps_f.size() * 4)) != IMCL_OK) return st;
        cudaError_t e = cudaMemcpy(d, job->taps_f.data(), job->taps_f.size() * 4, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "tuner: taps upload");
        c.taps = d;
        c.taps2 = static_cast<const float*>(d) + p.kw;
    } else {
        c.taps = job->taps_f.data();
        c.taps2 = job->taps_f.data() + p.kw;
    }
    job->conv = c;
    std::vector<imcl_variant> base;
    for (const ConvEntry* e : sep_entries_for(p.in_dtype, p.out_dtype, p.kw, p.kh, p.taps_mem))
        base.push_back(e->v);
    job->candidates = expand_shapes(base);
    job->run = [job](const imcl_variant& v, cudaStream_t st2) { return sep_run(job->conv, &v, st2); };
    job->out = out;
    job->out_dtype = p.out_dtype;
    job->W = p.width;
    job->H = p.height;
    job->out_pitch_b = c.out_pitch_b;
    job->working_set_bytes = (double)c.in_pitch_b * p.height + (double)c.out_pitch_b * p.height;
    if (p.out_dtype == IMCL_F16) job->tol_abs = (float)(l1 * std::ldexp(1.0, -9));
    else if (p.out_dtype == IMCL_BF16) job->tol_abs = (float)(l1 * std::ldexp(1.0, -6));
    else job->tol_abs = (float)(l1 * 1e-5);
    return IMCL_OK;
}

static imcl_status make_harris_job(const imcl_problem& p, cudaStream_t s, TuneJob* job) {
    if (p.kw <= 0 || p.kw > 7) return fail(IMCL_ERR_UNSUPPORTED, "harris window side must be 1..7");
    imcl_status st;
    DeviceInfo* dev = nullptr;
    if ((st = device_info(&dev)) != IMCL_OK) return st;
    ConvCall c = harris_problem_call(p);
    c.dev = dev;
    c.status = dev->status;
    void *in = nullptr, *out = nullptr, *ws = nullptr;
    if ((st = job->scratch.image(IMCL_F32, p.width, p.height, 1605u, &in, &c.in_pitch_b, s)) != IMCL_OK) return st;
    if ((st = job->scratch.image(IMCL_F32, p.width, p.height, 7u, &out, &c.out_pitch_b, s)) != IMCL_OK) return st;
    const size_t ws_bytes = (size_t)2 * p.width * p.height * sizeof(float);
    if ((st = job->scratch.alloc(&ws, ws_bytes)) != IMCL_OK) return st;
    c.in = in;
    c.out = out;
    c.workspace = ws;
    c.ws_bytes = ws_bytes;
    const float sob[9] = {-1, 0, 1, -2, 0, 2, -1, 0, 1};
    for (int i = 0; i < 9; ++i) job->taps_f.push_back(sob[i]);
    for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) job->taps_f.push_back(sob[i * 3 + j]);
    double gsum = 0;
    const int r = p.kw / 2;
    for (int j = 0; j < p.kw; ++j)   // a Gaussian over the window's offsets (caller's side)
        for (int i = 0; i < p.kw; ++i) {
            job->taps_f.push_back((float)std::exp(-0.5 * ((i - r) * (i - r) + (j - r) * (j - r))));
            gsum += job->taps_f.back();
        }
    c.hk = 0.04f;
    const size_t n = job->taps_f.size();
    if (p.taps_mem == IMCL_MEM_DEVICE) {
        void* d = nullptr;
        if ((st = job->scratch.alloc(&d, n * 4)) != IMCL_OK) return st;
        cudaError_t e = cudaMemcpy(d, job->taps_f.data(), n * 4, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "tuner: taps upload");
        c.taps = d;
        c.taps2 = static_cast<const float*>(d) + 9;
        c.taps3 = static_cast<const float*>(d) + 18;
    } else {
        c.taps = job->taps_f.data();
        c.taps2 = job->taps_f.data() + 9;
        c.taps3 = job->taps_f.data() + 18;
    }
    job->conv = c;
    std::vector<imcl_variant> base;
    for (const ConvEntry* e : harris_entries_for(c.kw, p.taps_mem)) base.push_back(e->v);
    job->candidates = expand_shapes(base);
    job->run = [job](const imcl_variant& v, cudaStream_t st2) { return harris_run(job->conv, &v, st2); };
    job->out = out;
    job->out_dtype = IMCL_F32;
    job->W = p.width;
    job->H = p.height;
    job->out_pitch_b = c.out_pitch_b;
    job->working_set_bytes = (double)c.in_pitch_b * p.height * 2;
    // |R| <= (1 + 2k) T^2 with T <= sum|G| * 2 * (8 max|I|)^2 and max|I| < 1
    const double T = gsum * 2.0 * 64.0;
    job->tol_abs = (float)(1e-5 * T * T);
    return IMCL_OK;
}

imcl_status make_tune_job(const imcl_problem& p, cudaStream_t s, TuneJob* job) {
    if (p.op == IMCL_OP_HARRIS) return make_harris_job(p, s, job);
    if (p.op == IMCL_OP_CONV2D) return make_conv_job(p, s, job);
    if (p.op == IMCL_OP_SEPCONV) return make_sep_job(p, s, job);
    return fail(IMCL_ERR_UNSUPPORTED, "unknown op");
}

}  // namespace imcl
