// batch_kernels.cuh -- the ragged batch: many images of different sizes, each with its
// own stencil (a conv2d filter of odd side <= 15 or a separable pair of radius <= 7), in
// one persistent launch.
//
// The host sorts every tile of every image into one work list (costliest first) and the
// CTAs of a persistent grid take tiles from it with an atomic counter (no waits, so no
// CTA can block another).  Each tile is staged into shared memory as f32 (converting the
// image's storage type, applying its boundary rule), then the specialised device code
// for its operator and filter side runs: the same register-blocked conv2d and fused
// row+column separable computation as the single-image kernels.  The backward runs as
// a few such persistent phases (input-gradient tiles, separable second pass, tap-gradient
// reductions), all recorded in one CUDA graph.
#pragma once

#include "tile_common.cuh"

namespace imcl {

constexpr int kBatchMaxK = 15;    // conv2d side
constexpr int kBatchMaxR = 7;     // separable radius

// One image operation of the batch (device copy).  Pitches in elements.
struct BImg {
    const void* in;
    void* out;
    long long in_pitch, out_pitch;
    int W, H, in_dt, out_dt;
    int op, kw, kh, K;                 // K: compiled side (conv) or 2R+1 (sep) it runs with
    const float* taps;                 // conv: kw*kh; sep: row taps (kw)
    const float* taps2;                // sep: column taps (kh)
    int border;
    float bv;
    // backward
    const float* g;                    // upstream gradient (f32)
    long long g_pitch;
    float* gin;                        // input gradient (f32) or nullptr
    long long gin_pitch;
    float* gtaps;                      // tap gradients or nullptr
    float* gtaps2;
    float* dt;                         // sep: batch-owned intermediate (pitch dt_pitch)
    long long dt_pitch;
    float* part;                       // batch-owned partial sums: [tiles][ntap_parts]
    int tiles_x, tiles_y;
};

// work item kinds
enum : int {
    BT_FWD = 0,        // forward tile
    BT_CONV_DX = 1,    // conv2d: input-gradient tile (zero-border flipped correlation) + tap partials
    BT_CONV_EDGE = 2,  // conv2d: folded input gradient on the image's edge pixels (clamp rule)
    BT_SEP_DT = 3,     // sep: dt tile (column adjoint with folds) + column-tap partials
    BT_SEP_DX = 4,     // sep: dx tile (row adjoint with folds) + row-tap partials
    BT_FINAL = 5,      // reduce one image's partial sums to its tap gradients
};

struct BTile {
    int img, kind, x0, y0;   // x0, y0: tile origin (tile kinds); BT_FINAL: x0 = tap set
};

__device__ __forceinline__ float load_px(const void* base, int dt, long long pitch, int x, int y) {
    const long long o = (long long)y * pitch + x;
    switch (dt) {
        case IMCL_F16: return __half2float(ldg(static_cast<const __half*>(base) + o));
        case IMCL_BF16: return __bfloat162float(ldg(static_cast<const __nv_bfloat16*>(base) + o));
        default: return ldg(static_cast<const float*>(base) + o);
    }
}

__device__ __forceinline__ void store_px(void* base, int dt, long long pitch, int x, int y, float v) {
    const long long o = (long long)y * pitch + x;
    switch (dt) {
        case IMCL_F16: static_cast<__half*>(base)[o] = __float2half_rn(v); break;
        case IMCL_BF16: static_cast<__nv_bfloat16*>(base)[o] = __float2bfloat16_rn(v); break;
        default: static_cast<float*>(base)[o] = v; break;
    }
}

// Stage region [gx0, gx0+sw) x [gy0, gy0+sh) of an image as f32 with its boundary rule
// (mode 0), or with zeros outside (mode 1, for upstream gradients).
__device__ void stage_region(float* st, int sw, int sh, const void* img, int dt, long long pitch, int gx0, int gy0,
                             int W, int H, int border, float bv, int zero_outside, int tid, int nth) {
    for (int idx = tid; idx < sw * sh; idx += nth) {
        const int r = idx / sw, c = idx - r * sw;
        const int gx = gx0 + c, gy = gy0 + r;
        float v;
        if (gx >= 0 && gx < W && gy >= 0 && gy < H) v = load_px(img, dt, pitch, gx, gy);
        else if (zero_outside) v = 0.f;
        else if (border == IMCL_BORDER_CONSTANT) v = bv;
        else v = load_px(img, dt, pitch, clampi(gx, 0, W - 1), clampi(gy, 0, H - 1));
        st[idx] = v;
    }
}

// Store a PX-wide register row of f32 results to an image of any output type.
template <int PX>
__device__ __forceinline__ void store_row_any(void* out, int dt, long long pitch, int gx, int gy, int W, int H,
                                              const float* v) {
    if (gy >= H) return;
#pragma unroll
    for (int c = 0; c < PX; ++c)
        if (gx + c < W) store_px(out, dt, pitch, gx + c, gy, v[c]);
}

// ------------------------------------------------------------------ forward tiles
// conv2d tile: sm holds the staged region (TW + 2 PAD) x (TH + K - 1), then K*K taps.
template <int K, int PY>
__device__ void batch_conv_tile(const BImg& im, int x0, int y0, int bx, int by, float* sm, bool flipped_zero,
                                const float* g_src, long long g_pitch, void* dst, long long dst_pitch, int dst_dt,
                                const int tid, const int nth) {
    constexpr int PX = 4;
    using G = TileGeo<float, K, PX>;
    const int TW = bx * PX, TH = by * PY, SW = TW + 2 * G::PAD, SH = TH + K - 1;
    float* st = sm;
    float* w = sm + SW * SH;
    const int R = (K - 1) / 2, rx = (im.kw - 1) / 2, ry = (im.kh - 1) / 2;
    // taps, centred into K x K (zero elsewhere); flipped for the adjoint
    for (int i = tid; i < K * K; i += nth) {
        const int j = i / K, c = i % K;
        const int sj = j - (R - ry), sc = c - (R - rx);
        float v = 0.f;
        if (sj >= 0 && sj < im.kh && sc >= 0 && sc < im.kw) {
            const int o = flipped_zero ? (im.kh - 1 - sj) * im.kw + (im.kw - 1 - sc) : sj * im.kw + sc;
            v = im.taps[o];
        }
        w[i] = v;
    }
    if (flipped_zero)
        stage_region(st, SW, SH, g_src, IMCL_F32, g_pitch, x0 - G::PAD, y0 - R, im.W, im.H, IMCL_BORDER_CONSTANT, 0.f, 1,
                     tid, nth);
    else
        stage_region(st, SW, SH, im.in, im.in_dt, im.in_pitch, x0 - G::PAD, y0 - R, im.W, im.H, im.border, im.bv, 0,
                     tid, nth);
    __syncthreads();
    if (tid < bx * by) {
        const int tx = tid % bx, ty = tid / bx;
        float acc[PY][PX];
#pragma unroll
        for (int oy = 0; oy < PY; ++oy)
#pragma unroll
            for (int ox = 0; ox < PX; ++ox) acc[oy][ox] = 0.f;
#pragma unroll
        for (int yy = 0; yy < PY + K - 1; ++yy) {
            float seg[G::SEG];
            load_seg_smem<float, G>(st + (ty * PY + yy) * SW + tx * PX, seg);
            fma_row_blocked<G, K, PX, PY, 1>(yy, seg, acc, w);
        }
        const bool skip_edges = flipped_zero && im.border == IMCL_BORDER_CLAMP;   // edge items own those
#pragma unroll
        for (int oy = 0; oy < PY; ++oy) {
            const int gy = y0 + ty * PY + oy;
            if (gy >= im.H) continue;
#pragma unroll
            for (int ox = 0; ox < PX; ++ox) {
                const int gx = x0 + tx * PX + ox;
                if (gx >= im.W) continue;
                if (skip_edges && (gx == 0 || gy == 0 || gx == im.W - 1 || gy == im.H - 1)) continue;
                store_px(dst, dst_dt, dst_pitch, gx, gy, acc[oy][ox]);
            }
        }
    }
}

// separable tile (forward): sm = staged region (TW + 2 PAD) x (TH + 2R), t buffer
// (TH + 2R) x TW, 2(2R+1) taps.
template <int R, int PY>
__device__ void batch_sep_tile(const BImg& im, int x0, int y0, int bx, int by, float* sm, const int tid, const int nth) {
    constexpr int PX = 4, NT = 2 * R + 1;
    using G = TileGeo<float, NT, PX>;
    const int TW = bx * PX, TH = by * PY, SW = TW + 2 * G::PAD, SH = TH + 2 * R;
    float* st = sm;
    float* tb = st + SW * SH;
    float* w = tb + SH * TW;
    const int orr = R - (im.kw - 1) / 2, orc = R - (im.kh - 1) / 2;
    for (int i = tid; i < NT; i += nth) {
        w[i] = (i >= orr && i < orr + im.kw) ? im.taps[i - orr] : 0.f;
        w[NT + i] = (i >= orc && i < orc + im.kh) ? im.taps2[i - orc] : 0.f;
    }
    stage_region(st, SW, SH, im.in, im.in_dt, im.in_pitch, x0 - G::PAD, y0 - R, im.W, im.H, im.border, im.bv, 0, tid,
                 nth);
    __syncthreads();
    const int nseg = TW / PX;
    for (int it = tid; it < SH * nseg; it += nth) {
        const int row = it / nseg, c0 = (it - row * nseg) * PX;
        const int gy = y0 - R + row;
        float r4[PX];
        if (im.border == IMCL_BORDER_CONSTANT && (gy < 0 || gy >= im.H)) {
#pragma unroll
            for (int ox = 0; ox < PX; ++ox) r4[ox] = im.bv;
        } else {
            float seg[G::SEG];
            load_seg_smem<float, G>(st + row * SW + c0, seg);
#pragma unroll
            for (int ox = 0; ox < PX; ++ox) r4[ox] = 0.f;
#pragma unroll
            for (int i = 0; i < NT; ++i)
#pragma unroll
                for (int ox = 0; ox < PX; ++ox) r4[ox] = __fmaf_rn(w[i], seg[G::LO + ox + i], r4[ox]);
        }
        *reinterpret_cast<float4*>(tb + row * TW + c0) = make_float4(r4[0], r4[1], r4[2], r4[3]);
    }
    __syncthreads();
    if (tid < bx * by) {
        const int tx = tid % bx, ty = tid / bx;
        float acc[PY][PX];
#pragma unroll
        for (int oy = 0; oy < PY; ++oy)
#pragma unroll
            for (int ox = 0; ox < PX; ++ox) acc[oy][ox] = 0.f;
#pragma unroll
        for (int yy = 0; yy < PY + 2 * R; ++yy) {
            const float4 v = *reinterpret_cast<const float4*>(tb + (ty * PY + yy) * TW + tx * PX);
            const float tv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int oy = 0; oy < PY; ++oy) {
                const int j = yy - oy;
                if (j >= 0 && j < NT) {
                    const float cj = w[NT + j];
#pragma unroll
                    for (int ox = 0; ox < PX; ++ox) acc[oy][ox] = __fmaf_rn(cj, tv[ox], acc[oy][ox]);
                }
            }
        }
#pragma unroll
        for (int oy = 0; oy < PY; ++oy)
            store_row_any<PX>(im.out, im.out_dt, im.out_pitch, x0 + tx * PX, y0 + ty * PY + oy, im.W, im.H, acc[oy]);
    }
}

template <int PY>
__device__ __forceinline__ void batch_fwd_dispatch(const BImg& im, int x0, int y0, int bx, int by, float* sm, int tid,
                                                   int nth) {
    if (im.op == IMCL_OP_CONV2D) {
        switch (im.K) {
            case 3: batch_conv_tile<3, PY>(im, x0, y0, bx, by, sm, false, nullptr, 0, im.out, im.out_pitch, im.out_dt, tid, nth); break;
            case 5: batch_conv_tile<5, PY>(im, x0, y0, bx, by, sm, false, nullptr, 0, im.out, im.out_pitch, im.out_dt, tid, nth); break;
            case 7: batch_conv_tile<7, PY>(im, x0, y0, bx, by, sm, false, nullptr, 0, im.out, im.out_pitch, im.out_dt, tid, nth); break;
            case 9: batch_conv_tile<9, PY>(im, x0, y0, bx, by, sm, false, nullptr, 0, im.out, im.out_pitch, im.out_dt, tid, nth); break;
            case 11: batch_conv_tile<11, PY>(im, x0, y0, bx, by, sm, false, nullptr, 0, im.out, im.out_pitch, im.out_dt, tid, nth); break;
            case 13: batch_conv_tile<13, PY>(im, x0, y0, bx, by, sm, false, nullptr, 0, im.out, im.out_pitch, im.out_dt, tid, nth); break;
            default: batch_conv_tile<15, PY>(im, x0, y0, bx, by, sm, false, nullptr, 0, im.out, im.out_pitch, im.out_dt, tid, nth); break;
        }
    } else {
        switch (im.K) {
            case 3: batch_sep_tile<1, PY>(im, x0, y0, bx, by, sm, tid, nth); break;
            case 5: batch_sep_tile<2, PY>(im, x0, y0, bx, by, sm, tid, nth); break;
            case 7: batch_sep_tile<3, PY>(im, x0, y0, bx, by, sm, tid, nth); break;
            case 9: batch_sep_tile<4, PY>(im, x0, y0, bx, by, sm, tid, nth); break;
            case 11: batch_sep_tile<5, PY>(im, x0, y0, bx, by, sm, tid, nth); break;
            case 13: batch_sep_tile<6, PY>(im, x0, y0, bx, by, sm, tid, nth); break;
            default: batch_sep_tile<7, PY>(im, x0, y0, bx, by, sm, tid, nth); break;
        }
    }
}

// Persistent forward: CTAs take tiles from the work list until it is exhausted.
template <int PY>
__global__ void __launch_bounds__(256, 2)
    k_batch_fwd(const BImg* __restrict__ imgs, const BTile* __restrict__ tiles, int ntiles, int* queue, int bx, int by) {
    extern __shared__ __align__(16) float bsm[];
    __shared__ int s_next;
    const int tid = threadIdx.x, nth = blockDim.x;
    for (;;) {
        if (tid == 0) s_next = atomicAdd(queue, 1);
        __syncthreads();
        const int t = s_next;
        if (t >= ntiles) break;
        const BTile tl = tiles[t];
        const BImg im = imgs[tl.img];
        batch_fwd_dispatch<PY>(im, tl.x0, tl.y0, bx, by, bsm, tid, nth);
        __syncthreads();   // shared memory and s_next are reused by the next tile
    }
}

}  // namespace imcl
