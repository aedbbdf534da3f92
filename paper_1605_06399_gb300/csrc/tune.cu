// tune.cu -- the auto-tuner (§4, Fig. 2) and the variant-table queries.
//
// The paper's tuner picks tuning-parameter values, generates and compiles the kernel,
// runs and times it on the device and repeats, keeping the best.  Here every variant is
// compiled ahead of time, so one tuning step is: launch a compiled variant with a block
// shape on scratch images of the problem's size, check its output against the PLAIN
// kernel's, time it with CUDA events (median of `reps`, L2 flushed between runs when the
// working set would stay in L2), and keep the fastest.  The space is small enough (tens
// to a few hundred points) to search exhaustively within seconds; the paper's
// model-guided search (a random sample, a neural-network performance model, the best
// predicted configurations confirmed by timing) is imagecl_tune_model.
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
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= W) return;
    for (int y = blockIdx.y; y < H; y += gridDim.y) {
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
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= W) return;
    for (int y = blockIdx.y; y < H; y += gridDim.y) {
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
    dim3 grid = grid_2d(W, H, 256, 1);
    k_fill_pattern<<<grid, 256, 0, s>>>(*p, dtype, W, H, *pitch_b, seed);
    return cuda_fail(cudaGetLastError(), "tuner: fill");
}

// ------------------------------------------------------------------ the search
// Work-group shapes swept for every tiled variant: every (bx, by) with bx in 4..128,
// by in 1..64 (powers of two) and 32..256 threads (the launcher rejects the shapes a
// variant's row alignment cannot take; they count as invalid candidates).
static const int kShapes[][2] = {{32, 8}, {32, 4}, {16, 16}, {16, 8}, {64, 4}, {64, 2}, {8, 16}, {32, 2},
                                 {4, 8}, {4, 16}, {4, 32}, {4, 64}, {8, 4}, {8, 8}, {8, 32}, {16, 2},
                                 {16, 4}, {32, 1}, {64, 1}, {128, 1}, {128, 2}};

std::vector<imcl_variant> expand_shapes(const std::vector<imcl_variant>& base) {
    std::vector<imcl_variant> out;
    for (const imcl_variant& b : base) {
        if (b.kind == IMCL_KIND_PLAIN) { out.push_back(b); continue; }
        if (b.kind == IMCL_KIND_TENSOR) {   // work-unit widths (16-column blocks)
            for (int nb : {8, 4, 16, 32}) {
                imcl_variant v = b;
                v.bx = nb;
                out.push_back(v);
            }
            continue;
        }
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

// Reads n 16-byte words (the second half of the L2 flush): the loads evict what the
// first half's memset left dirty in L2.  The sink is written only for one sum value, so
// the loads are kept but nothing depends on the data.
__global__ void k_l2_read(const uint4* __restrict__ p, size_t n, unsigned int* sink) {
    unsigned int acc = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const uint4 v = __ldg(p + i);
        acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
    if (acc == 0x9e3779b9u) atomicOr(sink, 1u);
}

// Runs candidates of one tuning job: the PLAIN kernel's output is the reference; a
// candidate counts if it launches, sets no device error and matches the reference
// within the job's tolerance; its time is the median of `reps` CUDA-event timings after
// a warm-up, with L2 flushed between runs when the working set would stay in L2: a
// buffer of twice L2 is overwritten and another of the same size is read, so each timed
// run starts with L2 holding neither its own data nor dirty lines it would write back.
class TuneRunner {
public:
    TuneRunner(TuneJob& job, int reps, cudaStream_t s) : job_(job), reps_(reps < 1 ? 1 : reps), s_(s) {}
    ~TuneRunner() {
        if (e0_) cudaEventDestroy(e0_);
        if (e1_) cudaEventDestroy(e1_);
    }

    imcl_status init(double* plain_ms) {
        int l2 = 0;
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, 0);
        if ((double)job_.working_set_bytes < 2.0 * l2) {
            flush_bytes_ = (size_t)l2 * 2;
            if (job_.scratch.alloc(&flush_, 2 * flush_bytes_) != IMCL_OK) { flush_ = nullptr; flush_bytes_ = 0; }
        }
        imcl_status st = job_.scratch.alloc(reinterpret_cast<void**>(&res_), 4 * sizeof(unsigned int));
        if (st != IMCL_OK) return st;
        st = job_.scratch.alloc(&ref_, (size_t)job_.out_pitch_b * job_.H);
        if (st != IMCL_OK) return st;
        if ((st = device_info(&dev_)) != IMCL_OK) return st;
        cudaEventCreate(&e0_);
        cudaEventCreate(&e1_);
        imcl_variant plain{};
        plain.kind = IMCL_KIND_PLAIN;
        plain.bx = 16;
        plain.by = 16;
        st = time_one(plain, &plain_ms_);
        if (st != IMCL_OK) return st;
        cudaMemcpy2DAsync(ref_, job_.out_pitch_b, job_.out, job_.out_pitch_b,
                          (size_t)job_.W * dtype_size(job_.out_dtype), job_.H, cudaMemcpyDeviceToDevice, s_);
        if (plain_ms) *plain_ms = plain_ms_;
        return IMCL_OK;
    }

    double plain_ms() const { return plain_ms_; }

    // true and the time if `v` launches and is correct; false otherwise.  A CUDA error
    // of the stream itself is returned through *st.
    bool check_and_time(const imcl_variant& v, double* ms, imcl_status* st) {
        *st = IMCL_OK;
        cudaMemsetAsync(job_.out, 0xff, (size_t)job_.out_pitch_b * job_.H, s_);
        if (job_.run(v, s_) != IMCL_OK) return false;   // shape not valid for this variant
        cudaMemsetAsync(res_, 0, 4 * sizeof(unsigned int), s_);
        dim3 grid = grid_2d(job_.W, job_.H, 256, 1);
        k_compare<<<grid, 256, 0, s_>>>(job_.out, ref_, job_.out_dtype, job_.W, job_.H, job_.out_pitch_b, res_);
        unsigned int h[4] = {0, 0, 0, 0};
        cudaError_t ce = cudaMemcpyAsync(h, res_, sizeof h, cudaMemcpyDeviceToHost, s_);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s_);
        if (ce != cudaSuccess) { *st = cuda_fail(ce, "tuner: check"); return false; }
        int code = 0;
        cudaMemcpy(&code, dev_->status, sizeof(int), cudaMemcpyDeviceToHost);
        if (code != 0) { cudaMemset(dev_->status, 0, sizeof(int)); return false; }
        const float dmax = __builtin_bit_cast(float, h[0]);
        const bool ok = job_.out_dtype == IMCL_I32 ? h[2] == 0 : dmax <= job_.tol_abs;
        if (!ok) return false;
        return time_one(v, ms) == IMCL_OK;
    }

private:
    imcl_status time_one(const imcl_variant& v, double* ms_out) {
        std::vector<float> t;
        for (int r = 0; r < reps_ + 1; ++r) {
            if (flush_) {
                cudaMemsetAsync(flush_, r & 0xff, flush_bytes_, s_);
                k_l2_read<<<4 * dev_->sm_count, 256, 0, s_>>>(
                    reinterpret_cast<const uint4*>(static_cast<uint8_t*>(flush_) + flush_bytes_), flush_bytes_ / 16,
                    res_ + 3);
            }
            cudaEventRecord(e0_, s_);
            imcl_status rs = job_.run(v, s_);
            cudaEventRecord(e1_, s_);
            if (rs != IMCL_OK) return rs;
            cudaError_t ce = cudaEventSynchronize(e1_);
            if (ce != cudaSuccess) return cuda_fail(ce, "tuner: timing");
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0_, e1_);
            if (r > 0) t.push_back(ms);   // first run is the warm-up
        }
        std::sort(t.begin(), t.end());
        *ms_out = t[t.size() / 2];
        return IMCL_OK;
    }

    TuneJob& job_;
    int reps_;
    cudaStream_t s_;
    void* flush_ = nullptr;
    size_t flush_bytes_ = 0;
    unsigned int* res_ = nullptr;
    void* ref_ = nullptr;
    DeviceInfo* dev_ = nullptr;
    cudaEvent_t e0_ = nullptr, e1_ = nullptr;
    double plain_ms_ = 0;
};

imcl_status tune_search(TuneJob& job, double budget_s, int reps, cudaStream_t s, imcl_variant* best,
                        double* best_ms, double* plain_ms) {
    const auto t_start = std::chrono::steady_clock::now();
    auto elapsed = [&] {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    };
    TuneRunner run(job, reps, s);
    imcl_status st = run.init(plain_ms);
    if (st != IMCL_OK) return st;
    imcl_variant win{};
    win.kind = IMCL_KIND_PLAIN;
    win.bx = 16;
    win.by = 16;
    double t_win = run.plain_ms();
    int n_tried = 0;
    for (const imcl_variant& v : job.candidates) {
        if (n_tried > 0 && elapsed() > budget_s) break;
        if (v.kind == IMCL_KIND_PLAIN) continue;
        double t = 0;
        const bool ok = run.check_and_time(v, &t, &st);
        if (st != IMCL_OK) return st;
        ++n_tried;
        if (ok && t < t_win) { t_win = t; win = v; }
    }
    *best = win;
    if (best_ms) *best_ms = t_win;
    return IMCL_OK;
}

// ------------------------------------------------------------------ model-guided search
// splitmix64: the seeded generator of the sample and of the network's initial weights
static uint64_t splitmix64(uint64_t& x) {
    uint64_t z = (x += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
static double uniform01(uint64_t& x) { return (double)(splitmix64(x) >> 11) * (1.0 / 9007199254740992.0); }

// One-hot encoding of a configuration's axes over the values the space contains.
class Encoder {
public:
    explicit Encoder(const std::vector<imcl_variant>& space) {
        for (int a = 0; a < kAxes; ++a) {
            for (const imcl_variant& v : space) {
                const int x = axis(v, a);
                if (std::find(values_[a].begin(), values_[a].end(), x) == values_[a].end()) values_[a].push_back(x);
            }
            width_ += (int)values_[a].size();
        }
    }
    int width() const { return width_; }
    std::vector<double> encode(const imcl_variant& v) const {
        std::vector<double> f((size_t)width_, 0.0);
        int o = 0;
        for (int a = 0; a < kAxes; ++a) {
            const auto it = std::find(values_[a].begin(), values_[a].end(), axis(v, a));
            if (it != values_[a].end()) f[(size_t)(o + (it - values_[a].begin()))] = 1.0;
            o += (int)values_[a].size();
        }
        return f;
    }

private:
    static constexpr int kAxes = 8;
    static int axis(const imcl_variant& v, int a) {
        const int x[kAxes] = {v.bx, v.by, v.px, v.py, v.load, v.filt, v.map, v.unroll};
        return x[a];
    }
    std::vector<int> values_[kAxes];
    int width_ = 0;
};

// y = w2 . tanh(W1 x + b1) + b2, fitted to standardised targets by full-batch Adam with
// a small L2 penalty (the performance model of §4: an artificial neural network).
class Mlp {
public:
    Mlp(int nin, int nh, uint64_t seed) : nin_(nin), nh_(nh), w1_((size_t)nh * nin), b1_(nh, 0.0), w2_(nh) {
        uint64_t st = seed ^ 0x5eedull;
        const double a1 = 1.0 / std::sqrt((double)nin), a2 = 1.0 / std::sqrt((double)nh);
        for (double& w : w1_) w = (2.0 * uniform01(st) - 1.0) * a1;
        for (double& w : w2_) w = (2.0 * uniform01(st) - 1.0) * a2;
    }
    double predict(const std::vector<double>& x) const {
        double y = b2_;
        for (int h = 0; h < nh_; ++h) {
            double z = b1_[h];
            for (int i = 0; i < nin_; ++i) z += w1_[(size_t)h * nin_ + i] * x[i];
            y += w2_[h] * std::tanh(z);
        }
        return y;
    }
    void fit(const std::vector<std::vector<double>>& X, const std::vector<double>& y, int iters, double lr,
             double l2) {
        const size_t n1 = w1_.size(), np = n1 + nh_ + nh_ + 1;
        std::vector<double> g(np), m(np, 0.0), v(np, 0.0), hid(nh_);
        const double b1m = 0.9, b2m = 0.999, eps = 1e-8;
        for (int it = 1; it <= iters; ++it) {
            std::fill(g.begin(), g.end(), 0.0);
            for (size_t s = 0; s < X.size(); ++s) {
                double out = b2_;
                for (int h = 0; h < nh_; ++h) {
                    double z = b1_[h];
                    for (int i = 0; i < nin_; ++i) z += w1_[(size_t)h * nin_ + i] * X[s][i];
                    hid[h] = std::tanh(z);
                    out += w2_[h] * hid[h];
                }
                const double d = 2.0 * (out - y[s]) / (double)X.size();
                g[np - 1] += d;
                for (int h = 0; h < nh_; ++h) {
                    g[n1 + nh_ + h] += d * hid[h];
                    const double dz = d * w2_[h] * (1.0 - hid[h] * hid[h]);
                    g[n1 + h] += dz;
                    for (int i = 0; i < nin_; ++i) g[(size_t)h * nin_ + i] += dz * X[s][i];
                }
            }
            for (size_t k = 0; k < n1; ++k) g[k] += 2.0 * l2 * w1_[k];
            for (int h = 0; h < nh_; ++h) g[n1 + nh_ + h] += 2.0 * l2 * w2_[h];
            const double c1 = 1.0 - std::pow(b1m, it), c2 = 1.0 - std::pow(b2m, it);
            for (size_t k = 0; k < np; ++k) {
                m[k] = b1m * m[k] + (1.0 - b1m) * g[k];
                v[k] = b2m * v[k] + (1.0 - b2m) * g[k] * g[k];
                const double step = lr * (m[k] / c1) / (std::sqrt(v[k] / c2) + eps);
                if (k < n1) w1_[k] -= step;
                else if (k < n1 + nh_) b1_[k - n1] -= step;
                else if (k < n1 + 2 * nh_) w2_[k - n1 - nh_] -= step;
                else b2_ -= step;
            }
        }
    }

private:
    int nin_, nh_;
    std::vector<double> w1_, b1_, w2_;
    double b2_ = 0.0;
};

constexpr int kHoldout = 8;   // random configurations timed after training, to measure the model

imcl_status tune_model_search(TuneJob& job, int n_sample, int n_confirm, int reps, uint64_t seed, cudaStream_t s,
                              imcl_variant* best, double* best_ms, double* plain_ms, imcl_tune_report* report) {
    const auto t_start = std::chrono::steady_clock::now();
    std::vector<imcl_variant> space;
    for (const imcl_variant& v : job.candidates)
        if (v.kind != IMCL_KIND_PLAIN) space.push_back(v);
    imcl_tune_report rep{};
    rep.candidates = (int32_t)space.size();
    TuneRunner run(job, reps, s);
    imcl_status st = run.init(plain_ms);
    if (st != IMCL_OK) return st;
    imcl_variant win{};
    win.kind = IMCL_KIND_PLAIN;
    win.bx = 16;
    win.by = 16;
    double t_win = run.plain_ms();
    // random sample (Fisher-Yates with the seeded generator)
    std::vector<int> order(space.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    uint64_t rs = seed;
    for (size_t i = order.size(); i > 1; --i) std::swap(order[i - 1], order[(size_t)(splitmix64(rs) % i)]);
    const int ns = std::min<int>(std::max(n_sample, 0), (int)space.size());
    std::vector<char> timed(space.size(), 0);
    std::vector<std::vector<double>> X;
    std::vector<double> y;
    Encoder enc(space);
    auto try_one = [&](int idx) -> imcl_status {
        timed[(size_t)idx] = 1;
        double t = 0;
        imcl_status e = IMCL_OK;
        if (run.check_and_time(space[(size_t)idx], &t, &e)) {
            ++rep.valid;
            X.push_back(enc.encode(space[(size_t)idx]));
            y.push_back(std::log(std::max(t, 1e-6)));
            if (t < t_win) { t_win = t; win = space[(size_t)idx]; }
        }
        return e;
    };
    for (int k = 0; k < ns; ++k) {
        if ((st = try_one(order[(size_t)k])) != IMCL_OK) return st;
        ++rep.sampled;
    }
    // the model, on standardised log times, then the untimed configurations it ranks best
    std::vector<std::pair<double, int>> ranked;
    std::vector<double> pred(space.size(), 0.0);   // the model's log time of every configuration
    bool have_model = false;
    if (X.size() >= 3) {
        double mean = 0, var = 0;
        for (double v : y) mean += v;
        mean /= (double)y.size();
        for (double v : y) var += (v - mean) * (v - mean);
        const double sd = std::sqrt(var / (double)y.size()) + 1e-9;
        std::vector<double> yn(y.size());
        for (size_t i = 0; i < y.size(); ++i) yn[i] = (y[i] - mean) / sd;
        Mlp net(enc.width(), 16, seed);
        net.fit(X, yn, 3000, 0.01, 1e-4);
        double se = 0;
        for (size_t i = 0; i < X.size(); ++i) {
            const double d = net.predict(X[i]) * sd + mean - y[i];
            se += d * d;
        }
        rep.model_rmse = std::sqrt(se / (double)X.size());
        for (size_t i = 0; i < space.size(); ++i) pred[i] = net.predict(enc.encode(space[i])) * sd + mean;
        have_model = true;
        for (size_t i = 0; i < space.size(); ++i)
            if (!timed[i]) ranked.push_back({pred[i], (int)i});
        std::sort(ranked.begin(), ranked.end());
    } else {   // too few valid samples for a model: confirm further random draws
        for (size_t k = (size_t)ns; k < order.size(); ++k) ranked.push_back({0.0, order[k]});
    }
    for (int k = 0; k < n_confirm && k < (int)ranked.size(); ++k) {
        if ((st = try_one(ranked[(size_t)k].second)) != IMCL_OK) return st;
        ++rep.confirmed;
    }
    // held-out check of the model: configurations it neither trained on nor picked, drawn
    // at random, timed, and compared with the model's prediction (they may also win)
    if (have_model) {
        double se = 0;
        for (size_t k = (size_t)ns; k < order.size() && rep.holdout < kHoldout; ++k) {
            const int idx = order[k];
            if (timed[(size_t)idx]) continue;
            const size_t before = y.size();
            if ((st = try_one(idx)) != IMCL_OK) return st;
            ++rep.holdout;
            if (y.size() > before) {
                const double d = pred[(size_t)idx] - y.back();
                se += d * d;
                ++rep.holdout_valid;
            }
        }
        rep.holdout_rmse = rep.holdout_valid ? std::sqrt(se / rep.holdout_valid) : 0.0;
    }
    *best = win;
    if (best_ms) *best_ms = t_win;
    rep.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (report) *report = rep;
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

imcl_status imagecl_tune_model(const imcl_problem* p, int32_t n_sample, int32_t n_confirm, int32_t reps, uint64_t seed,
                               imcl_variant* best, double* best_ms, double* plain_ms, imcl_tune_report* report,
                               void* stream) {
    if (!p || !best) return fail(IMCL_ERR_INVALID, "problem and best must not be NULL");
    if (p->width <= 0 || p->height <= 0) return fail(IMCL_ERR_INVALID, "problem size must be positive");
    if (n_sample < 0 || n_confirm < 0) return fail(IMCL_ERR_INVALID, "n_sample and n_confirm must not be negative");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    TuneJob job;
    imcl_status st = make_tune_job(*p, s, &job);
    if (st != IMCL_OK) return st;
    st = tune_model_search(job, n_sample, n_confirm, reps, seed, s, best, best_ms, plain_ms, report);
    if (st != IMCL_OK) return st;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "tuner: final sync");
    cache_store(*p, *best);
    return IMCL_OK;
}

}  // extern "C"
