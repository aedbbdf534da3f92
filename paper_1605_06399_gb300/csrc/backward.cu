// backward.cu -- the adjoint passes of conv2d, sepconv and Harris, composed from the
// forward kernels (zero-border correlations with flipped taps) and the building blocks
// of backward_kernels.cuh.  Every launch goes on the caller's stream; intermediate planes
// and partial sums live in the caller's workspace.
#include <algorithm>
#include <vector>

#include "abi_internal.h"
#include "backward_internal.h"
#include "backward_kernels.cuh"
#include "harris_bwd_kernels.cuh"
#include "sepbwd_kernels.cuh"

namespace imcl {

static size_t plane_pitch(int W) { return (size_t)round_up(W, 32); }              // floats (128 B)
static size_t plane_floats(int W, int H) { return plane_pitch(W) * (size_t)H; }
static int wgrad_grid(int W, int H) {
    const int tiles = ((W + kWgTileW - 1) / kWgTileW) * ((H + kWgTileH - 1) / kWgTileH);
    return std::min(tiles, kWgMaxParts);
}
constexpr size_t kTapScratch = 4 * kMaxAdjTaps + 64;                                // floats

size_t conv2d_backward_ws(int W, int H, int kw, int kh) {
    return (kTapScratch + (size_t)wgrad_grid(W, H) * kw * kh) * sizeof(float);
}
size_t sepconv_backward_ws(int W, int H, int nr, int nc) {
    return (2 * plane_floats(W, H) + kTapScratch + (size_t)wgrad_grid(W, H) * std::max(nr, nc)) * sizeof(float);
}
// CTAs (tap-gradient partial sets) of the fused Harris adjoint at most
static int harris_fused_parts(int W, int H) {
    const int tiles = ((W + kHbTileW - 1) / kHbTileW) * ((H + kHbTileH - 1) / kHbTileH);
    return std::min(tiles, kWgMaxParts);
}
size_t harris_backward_ws(int W, int H, int wk) {
    const size_t parts = std::max((size_t)3 * wgrad_grid(W, H) * wk * wk, (size_t)harris_fused_parts(W, H) * (wk * wk + 18));
    return (9 * plane_floats(W, H) + kTapScratch + parts) * sizeof(float);
}

// ------------------------------------------------------------------ helpers
// A ConvCall for an f32 -> f32 correlation of workspace / user planes.
static ConvCall f32_call(const ConvCall& base, const float* in, int64_t in_pitch_b, float* out, int64_t out_pitch_b) {
    ConvCall c = base;
    c.in = in;
    c.out = out;
    c.in_dtype = IMCL_F32;
    c.out_dtype = IMCL_F32;
    c.in_pitch_b = in_pitch_b;
    c.out_pitch_b = out_pitch_b;
    c.workspace = nullptr;
    c.ws_bytes = 0;
    return c;
}

// Taps of one operand: host vectors, or device pointers into the workspace.
struct TapSet {
    const float* orig = nullptr;       // as given (host or device)
    const float* flipped = nullptr;    // flip(w) (host or device)
    std::vector<float> host_flip;
};

static imcl_status make_taps(const float* taps, int n, int taps_mem, float* dev_slot, cudaStream_t s, TapSet* t) {
    t->orig = taps;
    if (taps_mem == IMCL_MEM_HOST) {
        t->host_flip.assign(taps, taps + n);
        std::reverse(t->host_flip.begin(), t->host_flip.end());
        t->flipped = t->host_flip.data();
        return IMCL_OK;
    }
    k_flip_taps<<<(n + 255) / 256, 256, 0, s>>>(taps, n, 1, dev_slot, nullptr);
    t->flipped = dev_slot;
    return cuda_fail(cudaGetLastError(), "flip taps");
}

// the single unit tap (row or column pass that leaves its axis alone)
static const float kOne = 1.0f;
static imcl_status unit_tap(int taps_mem, float* dev_slot, cudaStream_t s, const float** out) {
    if (taps_mem == IMCL_MEM_HOST) { *out = &kOne; return IMCL_OK; }
    k_flip_taps<<<1, 32, 0, s>>>(nullptr, 0, 0, nullptr, dev_slot);
    *out = dev_slot;
    return cuda_fail(cudaGetLastError(), "unit tap");
}

static imcl_status edges_2d(float* dx, int64_t dx_pitch, const float* g1, int64_t g1_pitch, const float* w1,
                            const float* g2, int64_t g2_pitch, const float* w2, int W, int H, int kw, int kh,
                            int taps_mem, cudaStream_t s) {
    AdjTaps tp;
    memset(&tp, 0, sizeof tp);
    const float *w1d = nullptr, *w2d = nullptr;
    if (taps_mem == IMCL_MEM_HOST) {
        memcpy(tp.w1, w1, sizeof(float) * kw * kh);
        if (w2) memcpy(tp.w2, w2, sizeof(float) * kw * kh);
    } else {
        w1d = w1;
        w2d = w2;
    }
    const int nedge = (H > 1 ? 2 * W : W) + (W > 1 ? 2 : 1) * std::max(H - 2, 0);
    k_adjoint_edges_2d<<<(nedge + 7) / 8, 256, 0, s>>>(dx, dx_pitch, g1, g1_pitch, g2, g2_pitch, W, H, kw, kh,
                                                            w1d, w2d, tp);
    return cuda_fail(cudaGetLastError(), "adjoint edges");
}

static imcl_status fold_1d(float* dst, int64_t dst_pitch, const float* g, int64_t g_pitch, int W, int H, int n,
                           int axis, const float* w, int taps_mem, cudaStream_t s) {
    TapsParam<float, 33> tp;
    for (int i = 0; i < 33; ++i) tp.w[i] = 0.f;
    const float* wd = nullptr;
    if (taps_mem == IMCL_MEM_HOST) for (int i = 0; i < n; ++i) tp.w[i] = w[i];
    else wd = w;
    const int lines = axis == 0 ? H : W;
    k_fold_1d<<<(lines + 255) / 256, 256, 0, s>>>(dst, dst_pitch, g, g_pitch, W, H, n, axis, wd, tp);
    return cuda_fail(cudaGetLastError(), "fold 1d");
}

// CTAs of a tap-gradient launch: the kernel's residency per SM (three for tap rows of up
// to 5, else two), at most the partial sets the workspace holds (one per full-height
// tile, at most kWgMaxParts); fixed for a device, an image size and a tap-row length.
static int wgrad_launch_grid(int W, int H, const DeviceInfo* dev, int kw) {
    const int resident = (kw <= 5 ? 3 : 2) * (dev ? dev->sm_count : 1);   // WgLaunch<KW>::MIN_CTAS
    return std::max(1, std::min(wgrad_grid(W, H), resident));
}

template <int KW>
static imcl_status wgrad_launch(const float* g, int64_t g_pitch, const void* x, int x_dt, int64_t x_pitch, int W,
                                int H, int kh, int border, float bvf, float* partials, int grid, cudaStream_t s) {
    const int smem = wgrad_smem_bytes<KW>(kh, 256);
    auto kfn = k_wgrad_partial<KW>;
    imcl_status st = set_smem_limit((const void*)kfn, smem);
    if (st != IMCL_OK) return st;
    const int esz = x_dt == IMCL_F32 ? 4 : 2;
    const int vec = ((reinterpret_cast<uintptr_t>(g) | (uintptr_t)(g_pitch * 4) | reinterpret_cast<uintptr_t>(x) |
                      (uintptr_t)(x_pitch * esz)) & 15) == 0;
    kfn<<<grid, 256, smem, s>>>(g, g_pitch, x, x_dt, x_pitch, W, H, kh, border, bvf, vec, partials);
    return cuda_fail(cudaGetLastError(), "tap gradient partials");
}

// The TMA-staged form (f32 operands with 16-byte aligned rows, tap rows of up to 5).
template <int KW>
static imcl_status wgrad_launch_tma(const float* g, int64_t g_pitch, const float* x, int64_t x_pitch, int W, int H,
                                    int kh, int border, float bv, float* partials, int grid, cudaStream_t s) {
    DeviceInfo* dev = nullptr;
    imcl_status st = device_info(&dev);
    if (st != IMCL_OK) return st;
    const int TH = WgTma<KW>::TH;
    CUtensorMap gmap, xmap;
    memset(&gmap, 0, sizeof gmap);
    memset(&xmap, 0, sizeof xmap);
    if ((st = encode_tmap_2d(&gmap, IMCL_F32, g, W, H, g_pitch * 4, kWgTileW, TH)) != IMCL_OK) return st;
    if ((st = encode_tmap_2d(&xmap, IMCL_F32, x, W, H, x_pitch * 4, WgTma<KW>::XW, TH + kh - 1)) != IMCL_OK)
        return st;
    const int smem = 128 + 2 * wgrad_tma_stage_bytes<KW>(kh);
    auto kfn = k_wgrad_tma<KW>;
    if ((st = set_smem_limit((const void*)kfn, smem)) != IMCL_OK) return st;
    kfn<<<grid, 256, smem, s>>>(gmap, xmap, W, H, kh, border, bv, partials, dev->status);
    return cuda_fail(cudaGetLastError(), "tap gradient partials (TMA)");
}

// Per-CTA partial sums of a kw x kh tap gradient; x of type x_dt with pitch in elements.
// `grid` CTAs write partials[0 .. grid * kw * kh).
static imcl_status wgrad_partials(const float* g, int64_t g_pitch, const void* x, int x_dt, int64_t x_pitch, int W,
                                  int H, int kw, int kh, int border, float bv, float* partials, int grid,
                                  cudaStream_t s) {
    if (kw % 2 == 0 || kw > 33 || kh < 1 || kh > 33)
        return fail(IMCL_ERR_UNSUPPORTED, "tap gradient: odd kw and kh up to 33");
    const bool aligned16 = ((reinterpret_cast<uintptr_t>(g) | reinterpret_cast<uintptr_t>(x) |
                             (uintptr_t)(g_pitch * 4) | (uintptr_t)(x_pitch * 4)) & 15) == 0;
    if (x_dt == IMCL_F32 && aligned16) {
        const float* xf = static_cast<const float*>(x);
#define IMCL_WGT(K) \
    case K: return wgrad_launch_tma<K>(g, g_pitch, xf, x_pitch, W, H, kh, border, bv, partials, grid, s);
        switch (kw) {
            IMCL_WGT(1) IMCL_WGT(3) IMCL_WGT(5) IMCL_WGT(7) IMCL_WGT(9) IMCL_WGT(11) IMCL_WGT(13) IMCL_WGT(15)
            default: break;
        }
#undef IMCL_WGT
    }
    // the constant as the pixel type reads it back
    float bvf = bv;
    if (x_dt == IMCL_F16) bvf = __half2float(__float2half_rn(bv));
    else if (x_dt == IMCL_BF16) bvf = __bfloat162float(__float2bfloat16_rn(bv));
#define IMCL_WG(K) \
    case K: return wgrad_launch<K>(g, g_pitch, x, x_dt, x_pitch, W, H, kh, border, bvf, partials, grid, s);
    switch (kw) {
        IMCL_WG(1) IMCL_WG(3) IMCL_WG(5) IMCL_WG(7) IMCL_WG(9) IMCL_WG(11) IMCL_WG(13) IMCL_WG(15)
        IMCL_WG(17) IMCL_WG(19) IMCL_WG(21) IMCL_WG(23) IMCL_WG(25) IMCL_WG(27) IMCL_WG(29) IMCL_WG(31) IMCL_WG(33)
        default: return fail(IMCL_ERR_UNSUPPORTED, "tap gradient: tap row length");
    }
#undef IMCL_WG
}

static imcl_status wgrad_any(const float* g, int64_t g_pitch, const void* x, int x_dtype, int64_t x_pitch_b, int W,
                             int H, int kw, int kh, int border, float bv, float* partials, int grid, cudaStream_t s) {
    if (x_dtype != IMCL_F32 && x_dtype != IMCL_F16 && x_dtype != IMCL_BF16)
        return fail(IMCL_ERR_UNSUPPORTED, "tap gradient: pixel type");
    const int64_t esz = x_dtype == IMCL_F32 ? 4 : 2;
    return wgrad_partials(g, g_pitch, x, x_dtype, x_pitch_b / esz, W, H, kw, kh, border, bv, partials, grid, s);
}

static imcl_status finalize(const float* partials, int nparts, int ntaps, float* out, cudaStream_t s) {
    k_wgrad_finalize<<<ntaps, 256, 0, s>>>(partials, nparts, ntaps, out, 0);
    return cuda_fail(cudaGetLastError(), "tap gradient finalize");
}

// A separable pass inside the backward runs a fused variant: the tuned one unless the
// tuning cache chose the two-kernel form (which needs a workspace these passes do not
// have), then the built-in fused default.
static imcl_status sep_run_fused(const ConvCall& c, cudaStream_t s) {
    imcl_variant v = sep_default_variant(c);
    if (v.kind != IMCL_KIND_TILED)
        v = pick_default(sep_entries_for(c.in_dtype, c.out_dtype, c.kw, c.kh, c.taps_mem), c.taps_mem,
                         tma_aligned(c), 4, 8);
    if (v.kind != IMCL_KIND_TILED) return fail(IMCL_ERR_UNSUPPORTED, "no fused separable variant for a backward pass");
    return sep_run(c, &v, s);
}

#define IMCL_TRY(x)                          \
    do {                                     \
        imcl_status _st = (x);               \
        if (_st != IMCL_OK) return _st;      \
    } while (0)

// ------------------------------------------------------------------ conv2d
imcl_status conv2d_backward_run(const BwdArgs& b, cudaStream_t s) {
    const ConvCall& f = b.fwd;
    const int W = f.W, H = f.H, n = f.kw * f.kh;
    float* ws = static_cast<float*>(b.workspace);
    float* tap_slot = ws;
    float* partials = ws + kTapScratch;
    const int wgrid = wgrad_launch_grid(W, H, f.dev, f.kw);
    if (b.dx) {
        TapSet t;
        IMCL_TRY(make_taps(static_cast<const float*>(f.taps), n, f.taps_mem, tap_slot, s, &t));
        ConvCall c = f32_call(f, b.g, b.g_pitch_b, b.dx, b.dx_pitch_b);
        c.taps = t.flipped;
        c.border = IMCL_BORDER_CONSTANT;
        c.border_value = 0.0;
        IMCL_TRY(conv_run(c, nullptr, s));
        if (f.border == IMCL_BORDER_CLAMP)
            IMCL_TRY(edges_2d(b.dx, b.dx_pitch_b / 4, b.g, b.g_pitch_b / 4, static_cast<const float*>(f.taps), nullptr, 0,
                              nullptr, W, H, f.kw, f.kh, f.taps_mem, s));
    }
    if (b.dw0) {
        IMCL_TRY(wgrad_any(b.g, b.g_pitch_b / 4, f.in, f.in_dtype, f.in_pitch_b, W, H, f.kw, f.kh, f.border,
                           (float)f.border_value, partials, wgrid, s));
        IMCL_TRY(finalize(partials, wgrid, n, b.dw0, s));
    }
    return IMCL_OK;
}

// ------------------------------------------------------------------ sepconv
// The fused separable adjoint (equal row and column radii up to kSbMaxR): one persistent
// launch for dx and both tap-gradient partial sets, then the fixed-order reductions.
template <int R>
static imcl_status sep_bwd_fused(const BwdArgs& b, float* ws, size_t ws_floats, cudaStream_t s) {
    constexpr int NT = 2 * R + 1;
    const ConvCall& f = b.fwd;
    const int W = f.W, H = f.H;
    SbTaps<R> tp;
    memset(&tp, 0, sizeof tp);
    SbArgs a{};
    if (f.taps_mem == IMCL_MEM_HOST) {
        memcpy(tp.r, f.taps, sizeof tp.r);
        memcpy(tp.c, f.taps2, sizeof tp.c);
    } else {
        a.rdev = static_cast<const float*>(f.taps);
        a.cdev = static_cast<const float*>(f.taps2);
    }
    a.g = b.g;
    a.gp = b.g_pitch_b / 4;
    a.x = f.in;
    a.x_dt = f.in_dtype;
    a.xp = f.in_pitch_b / dtype_size(f.in_dtype);
    a.dx = b.dx;
    a.dxp = b.dx ? b.dx_pitch_b / 4 : 0;
    a.W = W;
    a.H = H;
    a.border = f.border;
    const float bv = (float)f.border_value;
    a.bvt = bv;
    a.bvx = f.in_dtype == IMCL_F16 ? __half2float(__float2half_rn(bv))
          : f.in_dtype == IMCL_BF16 ? __bfloat162float(__float2bfloat16_rn(bv)) : bv;
    a.tiles_x = (W + kSbTileW - 1) / kSbTileW;
    a.ntiles = a.tiles_x * ((H + kSbTileH - 1) / kSbTileH);
    a.vec = f.in_dtype == IMCL_F32 && ((reinterpret_cast<uintptr_t>(b.g) | reinterpret_cast<uintptr_t>(f.in) |
                                         (uintptr_t)b.g_pitch_b | (uintptr_t)f.in_pitch_b) & 15) == 0;
    // f32 operands on 16-byte aligned rows: TMA staging in a two-stage ring
    CUtensorMap gmap, xmap;
    memset(&gmap, 0, sizeof gmap);
    memset(&xmap, 0, sizeof xmap);
    if (a.vec) {
        using G = SbGeo<R>;
        IMCL_TRY(encode_tmap_2d(&gmap, IMCL_F32, b.g, W, H, b.g_pitch_b, G::RW, G::RH));
        IMCL_TRY(encode_tmap_2d(&xmap, IMCL_F32, f.in, W, H, f.in_pitch_b, G::RW, G::RH));
    }
    const int smem = a.vec ? sb_smem_bytes<R, true>() : sb_smem_bytes<R, false>();
    auto kfn = a.vec ? k_sep_bwd_fused<R, true> : k_sep_bwd_fused<R, false>;
    IMCL_TRY(set_smem_limit((const void*)kfn, smem));
    const int occ = cached_occupancy((const void*)kfn, 256, smem);
    if (occ <= 0) return fail(IMCL_ERR_UNSUPPORTED, "fused separable backward cannot be resident");
    int grid = std::min(a.ntiles, occ * f.dev->sm_count);
    grid = std::max(1, std::min<int>(grid, (int)(ws_floats / (2 * NT))));   // partial sets that fit
    a.prow = ws;
    a.pcol = ws + (size_t)grid * NT;
    kfn<<<grid, 256, smem, s>>>(a, tp, gmap, xmap, f.dev->status);
    IMCL_TRY(cuda_fail(cudaGetLastError(), "fused separable backward"));
    if (b.dw0) IMCL_TRY(finalize(a.prow, grid, NT, b.dw0, s));
    if (b.dw1) IMCL_TRY(finalize(a.pcol, grid, NT, b.dw1, s));
    return IMCL_OK;
}

imcl_status sepconv_backward_run(const BwdArgs& b, cudaStream_t s) {
    const ConvCall& f = b.fwd;
    const int W = f.W, H = f.H, nr = f.kw, nc = f.kh;
    const size_t pf = plane_floats(W, H);
    if (nr == nc && (nr - 1) / 2 <= kSbMaxR) {
        float* ws0 = static_cast<float*>(b.workspace);
        const size_t wsf = 2 * pf;   // the two planes the multi-pass form uses hold the partial sums
        switch ((nr - 1) / 2) {
            case 0: return sep_bwd_fused<0>(b, ws0, wsf, s);
            case 1: return sep_bwd_fused<1>(b, ws0, wsf, s);
            case 2: return sep_bwd_fused<2>(b, ws0, wsf, s);
            case 3: return sep_bwd_fused<3>(b, ws0, wsf, s);
            case 4: return sep_bwd_fused<4>(b, ws0, wsf, s);
            case 5: return sep_bwd_fused<5>(b, ws0, wsf, s);
            case 6: return sep_bwd_fused<6>(b, ws0, wsf, s);
            case 7: return sep_bwd_fused<7>(b, ws0, wsf, s);
            default: return sep_bwd_fused<8>(b, ws0, wsf, s);
        }
    }
    const int64_t pp_b = (int64_t)plane_pitch(W) * 4;
    float* ws = static_cast<float*>(b.workspace);
    float* T = ws;
    float* DT = ws + pf;
    float* tap_slot = ws + 2 * pf;
    float* partials = tap_slot + kTapScratch;
    const int wgrid_r = wgrad_launch_grid(W, H, f.dev, nr), wgrid_c = wgrad_launch_grid(W, H, f.dev, 1);
    const float* one = nullptr;
    IMCL_TRY(unit_tap(f.taps_mem, tap_slot + 4 * kMaxAdjTaps, s, &one));
    TapSet tr, tc;
    IMCL_TRY(make_taps(static_cast<const float*>(f.taps), nr, f.taps_mem, tap_slot, s, &tr));
    IMCL_TRY(make_taps(static_cast<const float*>(f.taps2), nc, f.taps_mem, tap_slot + 64, s, &tc));

    // dt = C^T g: zero-border column correlation with the flipped column taps, then fold
    ConvCall c = f32_call(f, b.g, b.g_pitch_b, DT, pp_b);
    c.kw = 1;
    c.kh = nc;
    c.taps = one;
    c.taps2 = tc.flipped;
    c.border = IMCL_BORDER_CONSTANT;
    c.border_value = 0.0;
    IMCL_TRY(sep_run_fused(c, s));
    if (f.border == IMCL_BORDER_CLAMP)
        IMCL_TRY(fold_1d(DT, pp_b / 4, b.g, b.g_pitch_b / 4, W, H, nc, 1, static_cast<const float*>(f.taps2),
                         f.taps_mem, s));
    if (b.dx) {   // dx = R^T dt
        ConvCall r = f32_call(f, DT, pp_b, b.dx, b.dx_pitch_b);
        r.kw = nr;
        r.kh = 1;
        r.taps = tr.flipped;
        r.taps2 = one;
        r.border = IMCL_BORDER_CONSTANT;
        r.border_value = 0.0;
        IMCL_TRY(sep_run_fused(r, s));
        if (f.border == IMCL_BORDER_CLAMP)
            IMCL_TRY(fold_1d(b.dx, b.dx_pitch_b / 4, DT, pp_b / 4, W, H, nr, 0, static_cast<const float*>(f.taps),
                             f.taps_mem, s));
    }
    if (b.dw0) {  // drow[i] = sum dt(p) x_b(p + i - rr)
        IMCL_TRY(wgrad_any(DT, pp_b / 4, f.in, f.in_dtype, f.in_pitch_b, W, H, nr, 1, f.border,
                           (float)f.border_value, partials, wgrid_r, s));
        IMCL_TRY(finalize(partials, wgrid_r, nr, b.dw0, s));
    }
    if (b.dw1) {  // dcol[j] = sum g(p) t_b(p + j - rc), t the forward row pass
        ConvCall t = f;
        t.out = T;
        t.out_dtype = IMCL_F32;
        t.out_pitch_b = pp_b;
        t.kh = 1;
        t.taps2 = one;
        t.workspace = nullptr;
        t.ws_bytes = 0;
        IMCL_TRY(sep_run_fused(t, s));
        IMCL_TRY(wgrad_any(b.g, b.g_pitch_b / 4, T, IMCL_F32, pp_b, W, H, 1, nc, f.border, (float)f.border_value,
                           partials, wgrid_c, s));
        IMCL_TRY(finalize(partials, wgrid_c, nc, b.dw1, s));
    }
    return IMCL_OK;
}

// ------------------------------------------------------------------ Harris
template <int WK>
static imcl_status harris_bwd_fused(const BwdArgs& b, const float* sx, const float* sy, const float* gw, int grid,
                                    float* pw, float* psx, float* psy, cudaStream_t s) {
    const ConvCall& f = b.fwd;
    HbTaps<WK> tp;
    memset(&tp, 0, sizeof tp);
    const float *sxd = nullptr, *syd = nullptr, *gwd = nullptr;
    if (f.taps_mem == IMCL_MEM_HOST) {
        memcpy(tp.sx, sx, sizeof tp.sx);
        memcpy(tp.sy, sy, sizeof tp.sy);
        memcpy(tp.g, gw, sizeof tp.g);
    } else {
        sxd = sx;
        syd = sy;
        gwd = gw;
    }
    constexpr int smem = HbGeo<WK>::TOTAL * (int)sizeof(float);
    static_assert(HbGeo<WK>::TOTAL >= kHbThreads * HbGeo<WK>::NTAP, "the tap combine reuses the tile buffers");
    auto kfn = k_harris_bwd_fused<WK>;
    imcl_status st = set_smem_limit((const void*)kfn, smem);
    if (st != IMCL_OK) return st;
    kfn<<<grid, kHbThreads, smem, s>>>(static_cast<const float*>(f.in), f.in_pitch_b / 4, b.g, b.g_pitch_b / 4, b.dx,
                                b.dx_pitch_b / 4, f.W, f.H, f.hk, sxd, syd, gwd, tp, pw, psx, psy);
    return cuda_fail(cudaGetLastError(), "harris backward (fused)");
}

imcl_status harris_backward_run(const BwdArgs& b, cudaStream_t s) {
    const ConvCall& f = b.fwd;
    const int W = f.W, H = f.H, wk = f.kw, src = f.kh;   // kernel side, caller's window side
    const size_t pf = plane_floats(W, H);
    const int64_t pp = (int64_t)plane_pitch(W), pp_b = pp * 4;
    float* ws = static_cast<float*>(b.workspace);
    float* IX = ws;
    float* IY = ws + pf;
    float* P[3] = {ws + 2 * pf, ws + 3 * pf, ws + 4 * pf};
    float* S[3] = {ws + 5 * pf, ws + 6 * pf, ws + 7 * pf};
    float* TMP = ws + 8 * pf;
    float* tap_slot = ws + 9 * pf;
    float* partials = tap_slot + kTapScratch;
    const float* sx = static_cast<const float*>(f.taps);
    const float* sy = static_cast<const float*>(f.taps2);
    const float* gw = static_cast<const float*>(f.taps3);
    const int grid = wgrad_launch_grid(W, H, f.dev, wk), grid_s = wgrad_launch_grid(W, H, f.dev, 3);
    const dim3 eg = grid_2d(W, H, 256, 1);
    // an even window runs as the next odd one with a zero last row and column; its
    // gradient is the top-left src x src block of that window's gradient
    std::vector<float> gw_host;
    float* dwin_pad = nullptr;
    if (src != wk) {
        if (f.taps_mem == IMCL_MEM_HOST) {
            gw_host.assign((size_t)wk * wk, 0.f);
            for (int j = 0; j < src; ++j)
                for (int i = 0; i < src; ++i) gw_host[j * wk + i] = gw[j * src + i];
            gw = gw_host.data();
        } else {
            float* d = tap_slot + 192;
            IMCL_TRY(cuda_fail(cudaMemsetAsync(d, 0, sizeof(float) * wk * wk, s), "window padding"));
            IMCL_TRY(cuda_fail(cudaMemcpy2DAsync(d, sizeof(float) * wk, gw, sizeof(float) * src, sizeof(float) * src,
                                                 src, cudaMemcpyDeviceToDevice, s), "window padding"));
            gw = d;
        }
        if (b.dw2) dwin_pad = tap_slot + 256;
    }

    if (wk == 3 || wk == 5) {   // one fused tile kernel, then the tap reductions
        const int hgrid = std::max(1, std::min(harris_fused_parts(W, H), 2 * (f.dev ? f.dev->sm_count : 1)));
        float* pw = partials;
        float* psx = pw + (size_t)hgrid * wk * wk;
        float* psy = psx + (size_t)hgrid * 9;
        if (wk == 3) IMCL_TRY(harris_bwd_fused<3>(b, sx, sy, gw, hgrid, pw, psx, psy, s));
        else IMCL_TRY(harris_bwd_fused<5>(b, sx, sy, gw, hgrid, pw, psx, psy, s));
        if (b.dw2) {
            IMCL_TRY(finalize(pw, hgrid, wk * wk, dwin_pad ? dwin_pad : b.dw2, s));
            if (dwin_pad)
                IMCL_TRY(cuda_fail(cudaMemcpy2DAsync(b.dw2, sizeof(float) * src, dwin_pad, sizeof(float) * wk,
                                                     sizeof(float) * src, src, cudaMemcpyDeviceToDevice, s),
                                   "window gradient"));
        }
        if (b.dw0) IMCL_TRY(finalize(psx, hgrid, 9, b.dw0, s));
        if (b.dw1) IMCL_TRY(finalize(psy, hgrid, 9, b.dw1, s));
        return IMCL_OK;
    }

    // other window sides: forward intermediates on workspace planes, then each adjoint
    // step as its own launch.  Forward intermediates: Ix, Iy, P, S
    ConvCall base = f;
    base.kw = base.kh = 3;
    ConvCall c = f32_call(base, static_cast<const float*>(f.in), f.in_pitch_b, IX, pp_b);
    c.taps = sx;
    c.border = IMCL_BORDER_CLAMP;
    IMCL_TRY(conv_run(c, nullptr, s));
    c.out = IY;
    c.taps = sy;
    IMCL_TRY(conv_run(c, nullptr, s));
    k_harris_products<<<eg, 256, 0, s>>>(IX, IY, P[0], P[1], P[2], pp, W, H);
    IMCL_TRY(cuda_fail(cudaGetLastError(), "harris products"));
    ConvCall cw = f;
    cw.kw = cw.kh = wk;
    for (int ch = 0; ch < 3; ++ch) {
        ConvCall w = f32_call(cw, P[ch], pp_b, S[ch], pp_b);
        w.taps = gw;
        w.border = IMCL_BORDER_CLAMP;
        IMCL_TRY(conv_run(w, nullptr, s));
    }
    // dR/dS in place
    k_harris_gs<<<eg, 256, 0, s>>>(b.g, b.g_pitch_b / 4, S[0], S[1], S[2], pp, W, H, f.hk);
    IMCL_TRY(cuda_fail(cudaGetLastError(), "harris dR/dS"));
    // window gradient: sum over the three channels
    if (b.dw2) {
        for (int ch = 0; ch < 3; ++ch)
            IMCL_TRY(wgrad_partials(S[ch], pp, P[ch], IMCL_F32, pp, W, H, wk, wk, IMCL_BORDER_CLAMP, 0.f,
                                    partials + (size_t)ch * grid * wk * wk, grid, s));
        IMCL_TRY(finalize(partials, 3 * grid, wk * wk, dwin_pad ? dwin_pad : b.dw2, s));
        if (dwin_pad)
            IMCL_TRY(cuda_fail(cudaMemcpy2DAsync(b.dw2, sizeof(float) * src, dwin_pad, sizeof(float) * wk,
                                                 sizeof(float) * src, src, cudaMemcpyDeviceToDevice, s),
                               "window gradient"));
    }
    // gP = window adjoint of gS (into the P planes)
    TapSet tg;
    IMCL_TRY(make_taps(gw, wk * wk, f.taps_mem, tap_slot, s, &tg));
    for (int ch = 0; ch < 3; ++ch) {
        ConvCall w = f32_call(cw, S[ch], pp_b, P[ch], pp_b);
        w.taps = tg.flipped;
        w.border = IMCL_BORDER_CONSTANT;
        w.border_value = 0.0;
        IMCL_TRY(conv_run(w, nullptr, s));
        IMCL_TRY(edges_2d(P[ch], pp, S[ch], pp, gw, nullptr, 0, nullptr, W, H, wk, wk, f.taps_mem, s));
    }
    // through the products: gIx -> S0, gIy -> S1
    k_harris_gi<<<eg, 256, 0, s>>>(IX, IY, P[0], P[1], P[2], S[0], S[1], pp, W, H);
    IMCL_TRY(cuda_fail(cudaGetLastError(), "harris dIx dIy"));
    if (b.dx) {   // Sobel adjoints, summed, then the folded edges of both
        TapSet tx, ty;
        IMCL_TRY(make_taps(sx, 9, f.taps_mem, tap_slot + 64, s, &tx));
        IMCL_TRY(make_taps(sy, 9, f.taps_mem, tap_slot + 128, s, &ty));
        ConvCall a = f32_call(base, S[0], pp_b, b.dx, b.dx_pitch_b);
        a.taps = tx.flipped;
        a.border = IMCL_BORDER_CONSTANT;
        a.border_value = 0.0;
        IMCL_TRY(conv_run(a, nullptr, s));
        ConvCall a2 = f32_call(base, S[1], pp_b, TMP, pp_b);
        a2.taps = ty.flipped;
        a2.border = IMCL_BORDER_CONSTANT;
        a2.border_value = 0.0;
        IMCL_TRY(conv_run(a2, nullptr, s));
        k_add_plane<<<eg, 256, 0, s>>>(b.dx, b.dx_pitch_b / 4, TMP, pp, W, H);
        IMCL_TRY(cuda_fail(cudaGetLastError(), "harris dI sum"));
        IMCL_TRY(edges_2d(b.dx, b.dx_pitch_b / 4, S[0], pp, sx, S[1], pp, sy, W, H, 3, 3, f.taps_mem, s));
    }
    if (b.dw0) {
        IMCL_TRY(wgrad_partials(S[0], pp, f.in, IMCL_F32, f.in_pitch_b / 4, W, H, 3, 3, IMCL_BORDER_CLAMP, 0.f,
                                partials, grid_s, s));
        IMCL_TRY(finalize(partials, grid_s, 9, b.dw0, s));
    }
    if (b.dw1) {
        IMCL_TRY(wgrad_partials(S[1], pp, f.in, IMCL_F32, f.in_pitch_b / 4, W, H, 3, 3, IMCL_BORDER_CLAMP, 0.f,
                                partials, grid_s, s));
        IMCL_TRY(finalize(partials, grid_s, 9, b.dw1, s));
    }
    return IMCL_OK;
}

}  // namespace imcl
