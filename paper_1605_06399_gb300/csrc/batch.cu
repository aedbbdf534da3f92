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
constexpr int kShapes[][3] = {{4, 32, 8}, {4, 16, 16}, {2, 32, 8}, {2, 16, 16}};
constexpr int kNumShapes = 4;
// The forward kernel's conversion is compiled for tile widths 64 and 128, and its compute
// maps exactly bx * by = 256 consumer threads onto a tile.
constexpr bool shapes_supported() {
    for (int c = 0; c < kNumShapes; ++c) {
        const int tw = 4 * kShapes[c][1];
        if ((tw != 64 && tw != 128) || kShapes[c][1] * kShapes[c][2] != kFwdConsumers) return false;
    }
    return true;
}
static_assert(shapes_supported(), "batch tile shapes outside what the forward kernel is compiled for");

// Byte alignment every row start of an image shares (16, 4, or 0 for less).
static int row_alignment(const void* base, int64_t pitch_bytes) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(base) | (uintptr_t)pitch_bytes;
    return (a & 15) == 0 ? 16 : ((a & 3) == 0 ? 4 : 0);
}

int batch_side(int op, int kw, int kh) {
    const int m = std::max(kw, kh);
    const int side = std::max(3, m);
    return op == IMCL_OP_CONV2D ? side : 2 * std::max(1, (m - 1) / 2) + 1;
}

size_t batch_smem_bytes(int py, int bx, int by) {
    return (size_t)fwd_layout(4 * bx, py * by).total;
}

static double tile_cost(const BImg& im, int w, int h) {
    const double px = (double)w * h;
    const double flops = im.op == IMCL_OP_CONV2D ? (double)im.K * im.K : 4.0 * im.K;
    return px * (flops + 16.0);
}

// Forward work list for a tile shape, costliest tiles first (stable order for equal cost).
static std::vector<BFwdTile> fwd_tiles(const std::vector<BImg>& imgs, int TW, int TH) {
    std::vector<std::pair<double, BFwdTile>> v;
    for (int i = 0; i < (int)imgs.size(); ++i) {
        const BImg& im = imgs[i];
        const int es = im.in_dt == IMCL_F32 ? 4 : 2;
        for (int y = 0; y < im.H; y += TH)
            for (int x = 0; x < im.W; x += TW) {
                BFwdTile t{};
                t.in = im.in;
                t.taps = im.taps;
                t.taps2 = im.taps2;
                t.pitch_b = im.in_pitch * es;
                t.W = im.W;
                t.H = im.H;
                t.K = im.K;
                t.es = es;
                t.op = im.op;
                t.kw = im.kw;
                t.kh = im.kh;
                t.img = i;
                t.x0 = x;
                t.y0 = y;
                v.push_back({tile_cost(im, std::min(TW, im.W - x), std::min(TH, im.H - y)), t});
            }
    }
    std::stable_sort(v.begin(), v.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    std::vector<BFwdTile> t;
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

template <bool ADJ = false>
static const void* fwd_kernel(int py) {
    return py == 4 ? (const void*)k_batch_fwd<4, ADJ> : (const void*)k_batch_fwd<2, ADJ>;
}

// One persistent launch of the pipelined tile kernel over `tiles`, taking indices from the
// counter `queue` (reset first), with the image descriptors `imgs`.  ADJ: the backward's
// input-gradient instantiation.
template <bool ADJ>
static imcl_status launch_fwd_list(const Batch& b, const BImg* imgs, int* queue, const BFwdTile* tiles, int ntiles,
                                   int py, int bx, int by, cudaStream_t s) {
    const size_t smem = batch_smem_bytes(py, bx, by);
    const void* fn = fwd_kernel<ADJ>(py);
    imcl_status st = set_smem_limit(fn, (int)smem);
    if (st != IMCL_OK) return st;
    const int occ = cached_occupancy(fn, kFwdThreads, (int)smem);
    if (occ <= 0) return fail(IMCL_ERR_UNSUPPORTED, "batch: kernel cannot be resident");
    const int grid = std::max(1, std::min(ntiles, occ * b.dev->sm_count));
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int), s);
    if (e != cudaSuccess) return cuda_fail(e, "batch queue reset");
    if (py == 4) k_batch_fwd<4, ADJ><<<grid, kFwdThreads, smem, s>>>(imgs, tiles, ntiles, queue, bx, by, b.dev->status);
    else k_batch_fwd<2, ADJ><<<grid, kFwdThreads, smem, s>>>(imgs, tiles, ntiles, queue, bx, by, b.dev->status);
    return cuda_fail(cudaGetLastError(), "batch tile launch");
}

static imcl_status launch_fwd(const Batch& b, const BFwdTile* tiles, int ntiles, int py, int bx, int by,
                              cudaStream_t s) {
    return launch_fwd_list<false>(b, b.dimgs, b.queue, tiles, ntiles, py, bx, by, s);
}

template <int CLS>
static const void* bwd_kernel(int py) {
    return py == 4 ? (const void*)k_batch_bwd<4, CLS> : (const void*)k_batch_bwd<2, CLS>;
}

// Shared memory of a backward phase kernel of class cls.
static size_t batch_bwd_smem_bytes(int cls, int py, int bx, int by) {
    const size_t TW = 4 * bx, TH = (size_t)py * by, K = kBatchMaxK, R = kBatchMaxR;
    if (cls == BCLS_CONV_TAPS) {
        // g (TW x TH), x staged from column x0 - 8 (the widest filter's pitch), then the
        // combine scratch and the K x K sums
        const size_t conv_xw = (size_t)round_up(wg_xpitch<kBatchMaxK>((int)TW) + 4, 8);
        return std::max(TW * TH + conv_xw * (TH + K - 1), (size_t)256 * BatchWg<kBatchMaxK>::JR * K + K * K) *
               sizeof(float);
    }
    if (cls == BCLS_SEP_TAPS) {
        // g, x, the row pass / column adjoint, taps, combine
        const size_t HH = TH + 2 * R, XW = TW + 16;
        return (TW * HH + XW * HH + std::max(TW * HH, XW * TH) + 32 + 1024) * sizeof(float);
    }
    return 256 * sizeof(float);   // the reductions' group sums
}

// One persistent launch of the backward phase kernel of class CLS over a work list.
template <int CLS>
static imcl_status launch_bwd_list(const Batch& b, const BTile* items, int n, int* queue, cudaStream_t s) {
    if (n == 0) return IMCL_OK;
    const size_t smem = batch_bwd_smem_bytes(CLS, b.py, b.bx, b.by);
    imcl_status st = set_smem_limit(bwd_kernel<CLS>(b.py), (int)smem);
    if (st != IMCL_OK) return st;
    const int occ = cached_occupancy(bwd_kernel<CLS>(b.py), 256, (int)smem);
    if (occ <= 0) return fail(IMCL_ERR_UNSUPPORTED, "batch backward: kernel cannot be resident");
    const int grid = std::max(1, std::min(n, occ * b.dev->sm_count));
    if (b.py == 4) k_batch_bwd<4, CLS><<<grid, 256, smem, s>>>(b.dimgs, items, n, queue, b.bx, b.by);
    else k_batch_bwd<2, CLS><<<grid, 256, smem, s>>>(b.dimgs, items, n, queue, b.bx, b.by);
    return cuda_fail(cudaGetLastError(), "batch backward launch");
}

// Backward plan: gradient pointers into the image descriptors, partial-sum buffers, the
// input-gradient tiles for the pipelined tile kernel (on a second set of descriptors: g as
// the image, gin as the output, a zero border, flipped taps, clamp folds at the edges),
// the tap-gradient tiles, the per-image reductions, and the graph that runs them.
static imcl_status plan_backward(Batch* b) {
    const int TW = 4 * b->bx, TH = b->py * b->by;
    std::vector<BTile> lc, ls, l3;   // conv2d tap tiles, separable tap tiles, reductions
    std::vector<BImg> dxi = b->himgs;
    std::vector<std::pair<double, BFwdTile>> dxt;
    bool any = false;
    for (int i = 0; i < (int)b->items.size(); ++i) {
        const imcl_batch_item& it = b->items[i];
        BImg& im = b->himgs[i];
        const bool has_g = it.grad_out.data != nullptr;
        if (!has_g) continue;
        imcl_status st;
        if ((st = check_image(&it.grad_out, "grad_out")) != IMCL_OK) return st;
        if (it.grad_out.dtype != IMCL_F32 || it.grad_out.width != im.W || it.grad_out.height != im.H)
            return fail(IMCL_ERR_INVALID, "item " + std::to_string(i) + ": grad_out must be f32 of the image's size");
        im.g = static_cast<const float*>(it.grad_out.data);
        im.g_pitch = it.grad_out.pitch_bytes / 4;
        im.g_vec = row_alignment(it.grad_out.data, it.grad_out.pitch_bytes);
        if (it.grad_in.data) {
            if ((st = check_image(&it.grad_in, "grad_in")) != IMCL_OK) return st;
            if (it.grad_in.dtype != IMCL_F32 || it.grad_in.width != im.W || it.grad_in.height != im.H)
                return fail(IMCL_ERR_INVALID, "item " + std::to_string(i) + ": grad_in must be f32 of the image's size");
            im.gin = static_cast<float*>(it.grad_in.data);
            im.gin_pitch = it.grad_in.pitch_bytes / 4;
        }
        im.gtaps = it.grad_taps;
        im.gtaps2 = it.op == IMCL_OP_SEPCONV ? it.grad_taps2 : nullptr;
        if (!im.gin && !im.gtaps && !im.gtaps2) continue;
        any = true;
        im.tiles_x = (im.W + TW - 1) / TW;
        im.tiles_y = (im.H + TH - 1) / TH;
        const int nt = im.tiles_x * im.tiles_y;
        const size_t nparts = it.op == IMCL_OP_CONV2D ? (size_t)nt * im.kw * im.kh : (size_t)nt * (im.kw + im.kh);
        if (im.gtaps || im.gtaps2) {
            cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&im.part), nparts * sizeof(float));
            if (e != cudaSuccess) return cuda_fail(e, "batch partial sums");
            b->owned.push_back(im.part);
        }
        if (im.gin) {
            // dx = the correlation of g with the taps rotated by 180 degrees under a zero
            // border (the separable pair each flipped: the adjoint of row then column pass),
            // plus the clamp folds at the edge pixels: the forward's own tiles, with g as the
            // f32 image and gin as the output
            BImg& d = dxi[i];
            d.in = im.g;
            d.in_dt = IMCL_F32;
            d.in_pitch = im.g_pitch;
            d.in_vec = im.g_vec;
            d.out = im.gin;
            d.out_dt = IMCL_F32;
            d.out_pitch = im.gin_pitch;
            d.border = IMCL_BORDER_CONSTANT;
            d.bv = 0.f;
            d.fold = im.border == IMCL_BORDER_CLAMP;
            for (int y = 0; y < im.H; y += TH)
                for (int x = 0; x < im.W; x += TW) {
                    BFwdTile t{};
                    t.in = im.g;
                    t.taps = im.taps;
                    t.taps2 = im.taps2;
                    t.pitch_b = im.g_pitch * 4;
                    t.W = im.W;
                    t.H = im.H;
                    t.K = im.K;
                    t.es = 4;
                    t.op = im.op;
                    t.kw = im.kw;
                    t.kh = im.kh;
                    t.img = i;
                    t.x0 = x;
                    t.y0 = y;
                    t.flip = 1;
                    dxt.push_back({tile_cost(im, std::min(TW, im.W - x), std::min(TH, im.H - y)), t});
                }
        }
        if (im.gtaps || im.gtaps2)
            for (int y = 0; y < im.H; y += TH)
                for (int x = 0; x < im.W; x += TW) {
                    if (it.op == IMCL_OP_CONV2D) lc.push_back(BTile{i, BT_CONV_DW, x, y});
                    else ls.push_back(BTile{i, BT_SEP_TAPS, x, y});
                }
        if (im.gtaps || im.gtaps2) {
            const int nchunk = it.op == IMCL_OP_CONV2D ? (im.kw * im.kh + kFinalChunk - 1) / kFinalChunk : 1;
            for (int c = 0; c < nchunk; ++c) l3.push_back(BTile{i, BT_FINAL, c, 0});
        }
    }
    if (!any) return IMCL_OK;
    // costliest first within each phase (large filters, then the rest in plan order)
    auto by_cost = [&](std::vector<BTile>& l) {
        std::stable_sort(l.begin(), l.end(), [&](const BTile& a, const BTile& c) {
            return b->himgs[a.img].K > b->himgs[c.img].K;
        });
    };
    by_cost(lc);
    by_cost(ls);
    // the reductions: images with the most tiles first
    std::stable_sort(l3.begin(), l3.end(), [&](const BTile& a, const BTile& c) {
        return b->himgs[a.img].tiles_x * b->himgs[a.img].tiles_y > b->himgs[c.img].tiles_x * b->himgs[c.img].tiles_y;
    });
    imcl_status st;
    // the descriptors now carry gradient pointers: refresh the device copy
    cudaError_t e = cudaMemcpy(b->dimgs, b->himgs.data(), b->himgs.size() * sizeof(BImg), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "batch descriptors");
    std::stable_sort(dxt.begin(), dxt.end(), [](const auto& a, const auto& c) { return a.first > c.first; });
    std::vector<BFwdTile> dx_tiles;
    dx_tiles.reserve(dxt.size());
    for (auto& p : dxt) dx_tiles.push_back(p.second);
    BImg* ddx = nullptr;
    BFwdTile* ddxt = nullptr;
    if ((st = upload(&ddx, dxi, &b->owned)) != IMCL_OK) return st;
    if ((st = upload(&ddxt, dx_tiles, &b->owned)) != IMCL_OK) return st;
    BTile *dc = nullptr, *dsp = nullptr, *d3 = nullptr;
    if ((st = upload(&dc, lc, &b->owned)) != IMCL_OK) return st;
    if ((st = upload(&dsp, ls, &b->owned)) != IMCL_OK) return st;
    if ((st = upload(&d3, l3, &b->owned)) != IMCL_OK) return st;
    const int ndx = (int)dx_tiles.size();
    for (int k = 0; k < 2; ++k) {
        e = cudaStreamCreateWithFlags(&b->br_stream[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "batch backward stream");
    }
    e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "batch backward event");
    // The graph: three branches from one fork -- the input-gradient tiles (they write only
    // grad_in), the conv2d tap tiles and the separable tap tiles (each writes its own
    // items' partial sums); the per-image reductions wait for both tap branches, and
    // everything joins at the end.
    e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "batch backward capture");
    cudaMemsetAsync(b->queue + 1, 0, (kQueueSlots - 1) * sizeof(int), b->cap_stream);
    cudaEventRecord(b->ev_fork, b->cap_stream);
    cudaStreamWaitEvent(b->br_stream[0], b->ev_fork, 0);
    cudaStreamWaitEvent(b->br_stream[1], b->ev_fork, 0);
    imcl_status lst = IMCL_OK, s1, s2, s3, s4;
    if (ndx > 0) lst = launch_fwd_list<true>(*b, ddx, b->queue + 4, ddxt, ndx, b->py, b->bx, b->by, b->br_stream[0]);
    s1 = launch_bwd_list<BCLS_CONV_TAPS>(*b, dc, (int)lc.size(), b->queue + 1, b->cap_stream);
    s2 = launch_bwd_list<BCLS_SEP_TAPS>(*b, dsp, (int)ls.size(), b->queue + 2, b->br_stream[1]);
    cudaEventRecord(b->ev_join[1], b->br_stream[1]);
    cudaStreamWaitEvent(b->cap_stream, b->ev_join[1], 0);
    s3 = launch_bwd_list<BCLS_FINAL>(*b, d3, (int)l3.size(), b->queue + 3, b->cap_stream);
    cudaEventRecord(b->ev_join[0], b->br_stream[0]);
    cudaStreamWaitEvent(b->cap_stream, b->ev_join[0], 0);
    s4 = IMCL_OK;
    cudaError_t le = cudaGetLastError();
    e = cudaStreamEndCapture(b->cap_stream, &b->bwd_graph);
    for (imcl_status q : {lst, s1, s2, s3, s4})
        if (q != IMCL_OK) return q;
    if (le != cudaSuccess) return cuda_fail(le, "batch backward launch");
    if (e != cudaSuccess) return cuda_fail(e, "batch backward capture end");
    e = cudaGraphInstantiate(&b->bwd_exec, b->bwd_graph, 0);
    if (e != cudaSuccess) return cuda_fail(e, "batch backward graph instantiate");
    b->bwd_items[0] = (int)(lc.size() + ls.size());
    b->bwd_items[1] = (int)l3.size();
    b->bwd_dx_tiles = ndx;
    return IMCL_OK;
}

Batch::~Batch() {
    if (fwd_exec) cudaGraphExecDestroy(fwd_exec);
    if (fwd_graph) cudaGraphDestroy(fwd_graph);
    if (bwd_exec) cudaGraphExecDestroy(bwd_exec);
    if (bwd_graph) cudaGraphDestroy(bwd_graph);
    if (ev_fork) cudaEventDestroy(ev_fork);
    for (int k = 0; k < 2; ++k) {
        if (ev_join[k]) cudaEventDestroy(ev_join[k]);
        if (br_stream[k]) cudaStreamDestroy(br_stream[k]);
    }
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
    b.in_vec = row_alignment(it.in.data, it.in.pitch_bytes);
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
    e = cudaMalloc(reinterpret_cast<void**>(&b->queue), kQueueSlots * sizeof(int));
    if (e != cudaSuccess) return bail(cuda_fail(e, "batch queue"));
    b->owned.push_back(b->queue);

    // tile shape: time whole-batch launches of each candidate, keep the fastest
    std::vector<BFwdTile*> cand_tiles(kNumShapes, nullptr);
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
    // The backward phases run on the same tiles and were measured 15% faster on the
    // taller (PY = 4) shapes at comparable forward times, so a plan with gradients
    // chooses among those.
    bool with_grads = false;
    for (const imcl_batch_item& it : b->items) with_grads = with_grads || it.grad_out.data != nullptr;
    for (int c = 0; c < kNumShapes; ++c) {
        if (with_grads && kShapes[c][0] != 4) continue;
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
    if ((st = plan_backward(b)) != IMCL_OK) return bail(st);
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

imcl_status imagecl_batch_backward(imcl_batch* h, void* stream) {
    Batch* b = reinterpret_cast<Batch*>(h);
    if (!b) return fail(IMCL_ERR_INVALID, "batch is NULL");
    if (!b->bwd_exec) return fail(IMCL_ERR_INVALID, "no item of this batch carries gradient buffers");
    return cuda_fail(cudaGraphLaunch(b->bwd_exec, static_cast<cudaStream_t>(stream)), "batch backward graph launch");
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
