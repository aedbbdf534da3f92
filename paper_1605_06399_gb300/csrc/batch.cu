// batch.cu -- the ragged-batch plan: validation, the cost-sorted work list, the tile
// shape chosen by timing whole-batch launches, and the CUDA graphs that replay it.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <numeric>
#include <vector>

#include "abi_internal.h"
#include "batch_internal.h"
#include "batch_kernels.cuh"

namespace imcl {

// Tile shapes the plan chooses from: (PY, bx, by) with PX = 4 -> tile (4 bx) x (PY by).
static const int kShapes[][3] = {{4, 32, 8}, {4, 16, 16}, {2, 32, 8}, {2, 16, 16}};
constexpr int kNumShapes = 4;

int batch_side(int op, int kw, int kh) {
    const int m = std::max(kw, kh);
    const int side = std::max(3, m);
    return op == IMCL_OP_CONV2D ? side : 2 * std::max(1, (m - 1) / 2) + 1;
}

size_t batch_smem_bytes(int py, int bx, int by) {
    const int TW = 4 * bx, TH = py * by;
    const int pad = 16 / 4 * ((kBatchMaxK / 2 + 3) / 4);   // f32 PAD for the largest side
    const int sw = TW + 2 * pad;
    const size_t conv = (size_t)sw * (TH + kBatchMaxK - 1) + kBatchMaxK * kBatchMaxK;
    const size_t sep = (size_t)sw * (TH + 2 * kBatchMaxR) + (size_t)(TH + 2 * kBatchMaxR) * TW + 2 * (2 * kBatchMaxR + 1);
    return std::max(conv, sep) * sizeof(float);
}

static double tile_cost(const BImg& im, int w, int h) {
    const double px = (double)w * h;
    const double flops = im.op == IMCL_OP_CONV2D ? (double)im.K * im.K : 4.0 * im.K;
    return px * (flops + 16.0);
}

// Forward work list for a tile shape, costliest tiles first (stable order for equal cost).
static std::vector<BTile> fwd_tiles(const std::vector<BImg>& imgs, int TW, int TH) {
    std::vector<std::pair<double, BTile>> v;
    for (int i = 0; i < (int)imgs.size(); ++i) {
        const BImg& im = imgs[i];
        for (int y = 0; y < im.H; y += TH)
            for (int x = 0; x < im.W; x += TW)
                v.push_back({tile_cost(im, std::min(TW, im.W - x), std::min(TH, im.H - y)), BTile{i, BT_FWD, x, y}});
    }
    std::stable_sort(v.begin(), v.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    std::vector<BTile> t;
    t.reserve(v.size());
    for (auto& p : v) t.push_back(p.second);
    return t;
}

template <typename T>
static imcl_status upload(T** dst, const std::vector<T>& src, std::vector<void*>* owned) {
    const size_t bytes = std::max<size_t>(1, src.size()) * sizeof(T);
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dst), bytes);
    if (e != cudaSuccess) return cuda_fail(e, "batch allocation");
    owned->push_back(*dst);
    if (!src.empty()) {
        e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "batch upload");
    }
    return IMCL_OK;
}

static const void* fwd_kernel(int py) {
    return py == 4 ? (const void*)k_batch_fwd<4> : (const void*)k_batch_fwd<2>;
}

static imcl_status launch_fwd(const Batch& b, const BTile* tiles, int ntiles, int py, int bx, int by, cudaStream_t s) {
    const size_t smem = batch_smem_bytes(py, bx, by);
    const int occ = cached_occupancy(fwd_kernel(py), 256, (int)smem);
    if (occ <= 0) return fail(IMCL_ERR_UNSUPPORTED, "batch: kernel cannot be resident");
    const int grid = std::max(1, std::min(ntiles, occ * b.dev->sm_count));
    cudaError_t e = cudaMemsetAsync(b.queue, 0, sizeof(int), s);
    if (e != cudaSuccess) return cuda_fail(e, "batch queue reset");
    if (py == 4) k_batch_fwd<4><<<grid, 256, smem, s>>>(b.dimgs, tiles, ntiles, b.queue, bx, by);
    else k_batch_fwd<2><<<grid, 256, smem, s>>>(b.dimgs, tiles, ntiles, b.queue, bx, by);
    return cuda_fail(cudaGetLastError(), "batch forward launch");
}

Batch::~Batch() {
    if (fwd_exec) cudaGraphExecDestroy(fwd_exec);
    if (fwd_graph) cudaGraphDestroy(fwd_graph);
    if (bwd_exec) cudaGraphExecDestroy(bwd_exec);
    if (bwd_graph) cudaGraphDestroy(bwd_graph);
    for (void* p : owned) cudaFree(p);
    if (cap_stream) cudaStreamDestroy(cap_stream);
}

imcl_status batch_validate_item(const imcl_batch_item& it, int idx) {
    const std::string at = "item " + std::to_string(idx) + ": ";
    imcl_status st;
    if (it.op != IMCL_OP_CONV2D && it.op != IMCL_OP_SEPCONV)
        return fail(IMCL_ERR_UNSUPPORTED, at + "op must be IMCL_OP_CONV2D or IMCL_OP_SEPCONV");
    if ((st = check_image(&it.in, "in")) != IMCL_OK) return fail(st, at + imagecl_last_error());
    if ((st = check_image(&it.out, "out")) != IMCL_OK) return fail(st, at + imagecl_last_error());
    if (it.in.dtype != IMCL_F32 && it.in.dtype != IMCL_F16 && it.in.dtype != IMCL_BF16)
        return fail(IMCL_ERR_UNSUPPORTED, at + "batch images are f32, f16 or bf16");
    if (it.out.dtype != IMCL_F32 && it.out.dtype != it.in.dtype)
        return fail(IMCL_ERR_UNSUPPORTED, at + "outputs are f32 or the input's type");
    if (it.in.width != it.out.width || it.in.height != it.out.height)
        return fail(IMCL_ERR_INVALID, at + "in and out sizes differ");
    if (images_overlap(&it.in, &it.out)) return fail(IMCL_ERR_INVALID, at + "in and out overlap");
    if (it.kw <= 0 || it.kh <= 0 || it.kw % 2 == 0 || it.kh % 2 == 0)
        return fail(IMCL_ERR_UNSUPPORTED, at + "tap counts must be odd and positive");
    if (it.kw > kBatchMaxK || it.kh > kBatchMaxK) return fail(IMCL_ERR_UNSUPPORTED, at + "tap counts above 15");
    if (!it.taps || (it.op == IMCL_OP_SEPCONV && !it.taps2))
        return fail(IMCL_ERR_INVALID, at + "taps (device pointers) missing");
    if ((st = check_border(it.border, it.border_value, it.in.dtype)) != IMCL_OK) return fail(st, at + imagecl_last_error());
    return IMCL_OK;
}

static BImg make_bimg(const imcl_batch_item& it) {
    BImg b;
    memset(&b, 0, sizeof b);
    b.in = it.in.data;
    b.out = it.out.data;
    b.in_pitch = it.in.pitch_bytes / dtype_size(it.in.dtype);
    b.out_pitch = it.out.pitch_bytes / dtype_size(it.out.dtype);
    b.W = it.in.width;
    b.H = it.in.height;
    b.in_dt = it.in.dtype;
    b.out_dt = it.out.dtype;
    b.op = it.op;
    b.kw = it.kw;
    b.kh = it.kh;
    b.K = batch_side(it.op, it.kw, it.kh);
    b.taps = it.taps;
    b.taps2 = it.taps2;
    b.border = it.border;
    b.bv = (float)it.border_value;
    return b;
}

imcl_status batch_create(const imcl_batch_item* items, int n, double budget_s, Batch** out) {
    if (!items || n <= 0 || !out) return fail(IMCL_ERR_INVALID, "batch: items, a positive count and out are required");
    imcl_status st;
    for (int i = 0; i < n; ++i)
        if ((st = batch_validate_item(items[i], i)) != IMCL_OK) return st;
    DeviceInfo* dev = nullptr;
    if ((st = device_info(&dev)) != IMCL_OK) return st;
    Batch* b = new Batch();
    b->dev = dev;
    b->items.assign(items, items + n);
    for (int i = 0; i < n; ++i) b->himgs.push_back(make_bimg(items[i]));
    for (const BImg& im : b->himgs) b->pixels += (double)im.W * im.H;
    auto bail = [&](imcl_status s) { delete b; return s; };
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(cuda_fail(e, "batch stream"));
    if ((st = upload(&b->dimgs, b->himgs, &b->owned)) != IMCL_OK) return bail(st);
    e = cudaMalloc(reinterpret_cast<void**>(&b->queue), 4 * sizeof(int));
    if (e != cudaSuccess) return bail(cuda_fail(e, "batch queue"));
    b->owned.push_back(b->queue);

    // tile shape: time whole-batch launches of each candidate, keep the fastest
    std::vector<BTile*> cand_tiles(kNumShapes, nullptr);
    std::vector<int> cand_n(kNumShapes, 0);
    for (int c = 0; c < kNumShapes; ++c) {
        auto t = fwd_tiles(b->himgs, 4 * kShapes[c][1], kShapes[c][0] * kShapes[c][2]);
        cand_n[c] = (int)t.size();
        if ((st = upload(&cand_tiles[c], t, &b->owned)) != IMCL_OK) return bail(st);
        if ((st = set_smem_limit(fwd_kernel(kShapes[c][0]), (int)batch_smem_bytes(kShapes[c][0], kShapes[c][1], kShapes[c][2]))) != IMCL_OK)
            return bail(st);
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = 0;
    double best_ms = 1e30;
    const auto t_start = std::chrono::steady_clock::now();
    for (int c = 0; c < kNumShapes; ++c) {
        std::vector<float> ts;
        for (int r = 0; r < 4; ++r) {
            cudaEventRecord(e0, b->cap_stream);
            st = launch_fwd(*b, cand_tiles[c], cand_n[c], kShapes[c][0], kShapes[c][1], kShapes[c][2], b->cap_stream);
            cudaEventRecord(e1, b->cap_stream);
            if (st != IMCL_OK) break;
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) { st = cuda_fail(e, "batch tuning"); break; }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r > 0) ts.push_back(ms);
        }
        if (st != IMCL_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return bail(st); }
        std::sort(ts.begin(), ts.end());
        b->shape_ms[c] = ts[ts.size() / 2];
        if (b->shape_ms[c] < best_ms) { best_ms = b->shape_ms[c]; best = c; }
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
        if (el > budget_s && c > 0) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->py = kShapes[best][0];
    b->bx = kShapes[best][1];
    b->by = kShapes[best][2];
    b->tiles = cand_tiles[best];
    b->ntiles = cand_n[best];
    b->fwd_ms_at_create = best_ms;

    // the forward graph: queue reset + one persistent launch
    e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bail(cuda_fail(e, "batch capture"));
    st = launch_fwd(*b, b->tiles, b->ntiles, b->py, b->bx, b->by, b->cap_stream);
    e = cudaStreamEndCapture(b->cap_stream, &b->fwd_graph);
    if (st != IMCL_OK) return bail(st);
    if (e != cudaSuccess) return bail(cuda_fail(e, "batch capture end"));
    e = cudaGraphInstantiate(&b->fwd_exec, b->fwd_graph, 0);
    if (e != cudaSuccess) return bail(cuda_fail(e, "batch graph instantiate"));
    e = cudaStreamSynchronize(b->cap_stream);
    if (e != cudaSuccess) return bail(cuda_fail(e, "batch sync"));
    *out = b;
    return IMCL_OK;
}

}  // namespace imcl

using namespace imcl;

extern "C" {

imcl_status imagecl_batch_create(const imcl_batch_item* items, int32_t n, double tune_budget_s, imcl_batch** out) {
    Batch* b = nullptr;
    imcl_status st = batch_create(items, n, tune_budget_s, &b);
    if (st != IMCL_OK) return st;
    *out = reinterpret_cast<imcl_batch*>(b);
    return IMCL_OK;
}

imcl_status imagecl_batch_run(imcl_batch* h, void* stream) {
    Batch* b = reinterpret_cast<Batch*>(h);
    if (!b) return fail(IMCL_ERR_INVALID, "batch is NULL");
    return cuda_fail(cudaGraphLaunch(b->fwd_exec, static_cast<cudaStream_t>(stream)), "batch forward graph launch");
}

imcl_status imagecl_batch_info(const imcl_batch* h, imcl_batch_info_t* info) {
    const Batch* b = reinterpret_cast<const Batch*>(h);
    if (!b || !info) return fail(IMCL_ERR_INVALID, "batch and info must not be NULL");
    memset(info, 0, sizeof *info);
    info->images = (int32_t)b->himgs.size();
    info->tiles = b->ntiles;
    info->tile_w = 4 * b->bx;
    info->tile_h = b->py * b->by;
    info->pixels = b->pixels;
    info->fwd_ms_at_create = b->fwd_ms_at_create;
    for (int c = 0; c < 4; ++c) info->shape_ms[c] = b->shape_ms[c];
    info->has_backward = b->bwd_exec != nullptr;
    return IMCL_OK;
}

void imagecl_batch_destroy(imcl_batch* h) { delete reinterpret_cast<Batch*>(h); }

}  // extern "C"
