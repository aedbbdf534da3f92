// tune.cu -- the auto-tuner (§4, Fig. 2) and the variant-table queries.
//
// The paper's tuner picks tuning-parameter values, generates and compiles the kernel,
// runs and times it on the device and repeats, keeping the best.  Here every variant is
// compiled ahead of time, so one tuning step is: launch a compiled variant with a block
// shape on scratch images of the problem's size, check its output against the PLAIN
// kernel's, time it with CUDA events (median of `reps`, L2 flushed between runs when the
// working set would stay in L2), and keep the fastest.  The space is small enough (tens
// to a few hundred points) to search exhaustively within seconds, so the paper's
// model-guided sampling is not needed for it.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <functional>
#include <vector>

#include "abi_internal.h"
#include "common.cuh"
#include "tune_internal.h"

namespace imcl {

// ------------------------------------------------------------------ scratch helpers
__device__ __forceinline__ uint32_t hash32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

__global__ void k_fill_pattern(void* p, int dtype, int W, int H, long long pitch_b, uint32_t seed) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W || y >= H) return;
    const uint32_t h = hash32((uint32_t)(y * 7919 + x) ^ seed);
    char* row = static_cast<char*>(p) + (long long)y * pitch_b;
    const float u = (h >> 8) * (1.0f / 16777216.0f);
    switch (dtype) {
        case IMCL_U8: reinterpret_cast<uint8_t*>(row)[x] = (uint8_t)(h & 255u); break;
        case IMCL_I32: reinterpret_cast<int32_t*>(row)[x] = (int32_t)(h & 1023u) - 512; break;
        case IMCL_F32: reinterpret_cast<float*>(row)[x] = u; break;
        case IMCL_F16: reinterpret_cast<__half*>(row)[x] = __float2half_rn(u); break;
        case IMCL_BF16: reinterpret_cast<__nv_bfloat16*>(row)[x] = __float2bfloat16_rn(u); break;
    }
}

__device__ __forceinline__ float load_any(const char* row, int dtype, int x) {
    switch (dtype) {
        case IMCL_I32: return (float)reinterpret_cast<const int32_t*>(row)[x];
        case IMCL_F32: return reinterpret_cast<const float*>(row)[x];
        case IMCL_F16: return __half2float(reinterpret_cast<const __half*>(row)[x]);
        case IMCL_BF16: return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(row)[x]);
        default: return (float)reinterpret_cast<const uint8_t*>(row)[x];
    }
}

// res[0] = max |a - b| (as float bits), res[1] = max |b|, res[2] = count of a != b
__global__ void k_compare(const void* a, const void* b, int dtype, int W, int H, long long pitch_b,
                          unsigned int* res) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W || y >= H) return;
    const char* ra = static_cast<const char*>(a) + (long long)y * pitch_b;
    const char* rb = static_cast<const char*>(b) + (long long)y * pitch_b;
    float va = load_any(ra, dtype, x), vb = load_any(rb, dtype, x);
    bool differ;
    if (dtype == IMCL_I32) differ = reinterpret_cast<const int32_t*>(ra)[x] != reinterpret_cast<const int32_t*>(rb)[x];
    else differ = !(va == vb);
    float d = fabsf(va - vb);
    if (!(d == d)) d = 3.0e38f;   // NaN compares as a huge difference
    atomicMax(&res[0], __float_as_uint(d));
    atomicMax(&res[1], __float_as_uint(fabsf(vb)));
    if (differ) atomicAdd(&res[2], 1u);
}

TuneScratch::~TuneScratch() {
    for (void* p : allocs) cudaFree(p);
}

imcl_status TuneScratch::alloc(void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(IMCL_ERR_OOM, "tuner: scratch allocation failed");
    }
    allocs.push_back(*p);
    return IMCL_OK;
}

imcl_status TuneScratch::image(int dtype, int W, int H, uint32_t seed, void** p, int64_t* pitch_b, cudaStream_t s) {
    const int sz = dtype_size(dtype);
    *pitch_b = ((int64_t)W * sz + 127) / 128 * 128;
    imcl_status st = alloc(p, (size_t)(*pitch_b) * H);
    if (st != IMCL_OK) return st;
    dim3 grid((W + 255) / 256, H);
    k_fill_pattern<<<grid, 256, 0, s>>>(*p, dtype, W, H, *pitch_b, seed);
    return cuda_fail(cudaGetLastError(), "tuner: fill");
}

// ------------------------------------------------------------------ the search
static const int kShapes[][2] = {{32, 8}, {32, 4}, {16, 16}, {16, 8}, {64, 4}, {64, 2}, {8, 16}, {32, 2}};

std::vector<imcl_variant> expand_shapes(const std::vector<imcl_variant>& base) {
    std::vector<imcl_variant> out;
    for (const imcl_variant& b : base) {
        if (b.kind == IMCL_KIND_PLAIN) { out.push_back(b); continue; }
        out.push_back(b);   // the registered default shape first
        for (auto& sh : kShapes) {
            if (sh[0] == b.bx && sh[1] == b.by) continue;
            imcl_variant v = b;
            v.bx = sh[0];
            v.by = sh[1];
            out.push_back(v);
        }
    }
    return out;
}

imcl_status tune_search(TuneJob& job, double budget_s, int reps, cudaStream_t s, imcl_variant* best,
                        double* best_ms, double* plain_ms) {
    if (reps < 1) reps = 1;
    const auto t_start = std::chrono::steady_clock::now();
    auto elapsed = [&] {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    };
    int l2 = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, 0);
    void* flush = nullptr;
    size_t flush_bytes = 0;
    if ((double)job.working_set_bytes < 2.0 * l2) {
        flush_bytes = (size_t)l2 * 2;
        if (job.scratch.alloc(&flush, flush_bytes) != IMCL_OK) { flush = nullptr; flush_bytes = 0; }
    }
    unsigned int* res = nullptr;
    imcl_status st = job.scratch.alloc(reinterpret_cast<void**>(&res), 4 * sizeof(unsigned int));
    if (st != IMCL_OK) return st;
    void* ref = nullptr;
    st = job.scratch.alloc(&ref, (size_t)job.out_pitch_b * job.H);
    if (st != IMCL_OK) return st;

    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto time_one = [&](const imcl_variant& v, double* ms_out) -> imcl_status {
        std::vector<float> t;
        for (int r = 0; r < reps + 1; ++r) {
            if (flush) cudaMemsetAsync(flush, r & 0xff, flush_bytes, s);
            cudaEventRecord(e0, s);
            imcl_status rs = job.run(v, s);
            cudaEventRecord(e1, s);
            if (rs != IMCL_OK) return rs;
            cudaError_t ce = cudaEventSynchronize(e1);
            if (ce != cudaSuccess) return cuda_fail(ce, "tuner: timing");
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r > 0) t.push_back(ms);   // first run is the warm-up
        }
        std::sort(t.begin(), t.end());
        *ms_out = t[t.size() / 2];
        return IMCL_OK;
    };

    // the untuned reference result and time
    imcl_variant plain{};
    plain.kind = IMCL_KIND_PLAIN;
    plain.bx = 16;
    plain.by = 16;
    double t_plain = 0;
    st = time_one(plain, &t_plain);
    if (st != IMCL_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return st; }
    cudaMemcpy2DAsync(ref, job.out_pitch_b, job.out, job.out_pitch_b, (size_t)job.W * dtype_size(job.out_dtype), job.H,
                      cudaMemcpyDeviceToDevice, s);
    if (plain_ms) *plain_ms = t_plain;

    imcl_variant win = plain;
    double t_win = t_plain;
    DeviceInfo* dev = nullptr;
    device_info(&dev);
    int n_tried = 0;
    for (const imcl_variant& v : job.candidates) {
        if (n_tried > 0 && elapsed() > budget_s) break;
        if (v.kind == IMCL_KIND_PLAIN) continue;
        // correctness against the plain kernel first
        cudaMemsetAsync(job.out, 0xff, (size_t)job.out_pitch_b * job.H, s);
        imcl_status rs = job.run(v, s);
        if (rs != IMCL_OK) continue;   // shape not valid for this variant: skip
        ++n_tried;
        cudaMemsetAsync(res, 0, 4 * sizeof(unsigned int), s);
        dim3 grid((job.W + 255) / 256, job.H);
        k_compare<<<grid, 256, 0, s>>>(job.out, ref, job.out_dtype, job.W, job.H, job.out_pitch_b, res);
        unsigned int h[4] = {0, 0, 0, 0};
        cudaError_t ce = cudaMemcpyAsync(h, res, sizeof h, cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) { cudaEventDestroy(e0); cudaEventDestroy(e1); return cuda_fail(ce, "tuner: check"); }
        int code = 0;
        cudaMemcpy(&code, dev->status, sizeof(int), cudaMemcpyDeviceToHost);
        if (code != 0) { cudaMemset(dev->status, 0, sizeof(int)); continue; }
        const float dmax = __builtin_bit_cast(float, h[0]);
        bool ok;
        if (job.out_dtype == IMCL_I32) ok = h[2] == 0;
        else ok = dmax <= job.tol_abs;
        if (!ok) continue;
        double t = 0;
        if (time_one(v, &t) != IMCL_OK) continue;
        if (t < t_win) { t_win = t; win = v; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *best = win;
    if (best_ms) *best_ms = t_win;
    return IMCL_OK;
}

}  // namespace imcl

using namespace imcl;

extern "C" {

int32_t imagecl_variant_count(const imcl_problem* p) {
    std::vector<imcl_variant> v;
    if (!p || list_variants(*p, &v) != IMCL_OK) return 0;
    return (int32_t)v.size();
}

imcl_status imagecl_variant_get(const imcl_problem* p, int32_t idx, imcl_variant* out) {
    if (!p || !out) return fail(IMCL_ERR_INVALID, "problem and out must not be NULL");
    std::vector<imcl_variant> v;
    imcl_status st = list_variants(*p, &v);
    if (st != IMCL_OK) return st;
    if (idx < 0 || idx >= (int32_t)v.size()) return fail(IMCL_ERR_INVALID, "variant index out of range");
    *out = v[idx];
    return IMCL_OK;
}

imcl_status imagecl_variant_default(const imcl_problem* p, imcl_variant* out) {
    if (!p || !out) return fail(IMCL_ERR_INVALID, "problem and out must not be NULL");
    return default_variant(*p, out);
}

imcl_status imagecl_tune(const imcl_problem* p, double budget_s, int32_t reps, imcl_variant* best,
                         double* best_ms, double* plain_ms, void* stream) {
    if (!p || !best) return fail(IMCL_ERR_INVALID, "problem and best must not be NULL");
    if (p->width <= 0 || p->height <= 0) return fail(IMCL_ERR_INVALID, "problem size must be positive");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    TuneJob job;
    imcl_status st = make_tune_job(*p, s, &job);
    if (st != IMCL_OK) return st;
    st = tune_search(job, budget_s, reps, s, best, best_ms, plain_ms);
    if (st != IMCL_OK) return st;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "tuner: final sync");
    cache_store(*p, *best);
    return IMCL_OK;
}

}  // extern "C"
