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
#include "wgrad_tile.cuh"

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
    int in_vec, g_vec;                 // byte alignment of the rows (16, 4 or less) for staging
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
// (zero_outside = 0), or with zeros outside (1, for upstream gradients).  When the region
// starts on an 8-pixel boundary and the image rows are 16-byte aligned (vec), chunks of 8
// pixels inside the image are read with 16-byte loads, several in flight per thread.
__device__ __forceinline__ float outside_px(const void* img, int dt, long long pitch, int gx, int gy, int W, int H,
                                            int border, float bv, int zero_outside) {
    if (gx >= 0 && gx < W && gy >= 0 && gy < H) return load_px(img, dt, pitch, gx, gy);
    if (zero_outside) return 0.f;
    if (border == IMCL_BORDER_CONSTANT) return bv;
    return load_px(img, dt, pitch, clampi(gx, 0, W - 1), clampi(gy, 0, H - 1));
}

// 8 consecutive pixels of one row starting at gx (all inside the image), with the widest
// loads the row's alignment allows: 16-byte vectors (vec = 16), pairs of 16-bit pixels
// (vec = 4), or single pixels; the loads are independent, so they are in flight together.
__device__ __forceinline__ void load8_inside(const void* img, int dt, long long pitch, int gx, int gy, int vec,
                                             float* v) {
    const long long o = (long long)gy * pitch + gx;
    if (dt == IMCL_F32) {
        const float* p = static_cast<const float*>(img) + o;
        if (vec >= 16) {
            const float4 a = __ldg(reinterpret_cast<const float4*>(p));
            const float4 b = __ldg(reinterpret_cast<const float4*>(p + 4));
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
            v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = __ldg(p + e);
        }
        return;
    }
    const uint16_t* p = static_cast<const uint16_t*>(img) + o;
    uint32_t u[4];
    if (vec >= 16) {
        const uint4 q = __ldg(reinterpret_cast<const uint4*>(p));
        u[0] = q.x; u[1] = q.y; u[2] = q.z; u[3] = q.w;
    } else if (vec >= 4) {
#pragma unroll
        for (int k = 0; k < 4; ++k) u[k] = __ldg(reinterpret_cast<const unsigned int*>(p) + k);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) u[k] = (uint32_t)__ldg(p + 2 * k) | ((uint32_t)__ldg(p + 2 * k + 1) << 16);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (dt == IMCL_F16) {
            const __half2 h = *reinterpret_cast<const __half2*>(&u[k]);
            const float2 f = __half22float2(h);
            v[2 * k] = f.x;
            v[2 * k + 1] = f.y;
        } else {
            v[2 * k] = __uint_as_float(u[k] << 16);
            v[2 * k + 1] = __uint_as_float(u[k] & 0xffff0000u);
        }
    }
}

// Stage region [gx0, gx0+sw) x [gy0, gy0+sh) of an image as f32 with its boundary rule
// (zero_outside = 0), or with zeros outside (1, for upstream gradients), in chunks of 8
// pixels.  vec: the alignment in bytes of the image's rows (16, 4 or less).
__device__ void stage_region(float* st, int sw, int sh, const void* img, int dt, long long pitch, int gx0, int gy0,
                             int W, int H, int border, float bv, int zero_outside, int tid, int nth, int vec = 0) {
    if ((gx0 & 7) == 0 && (sw & 7) == 0) {
        const int nch = sw >> 3;
#pragma unroll 4
        for (int idx = tid; idx < nch * sh; idx += nth) {
            const int r = idx / nch, c = (idx - r * nch) << 3;
            const int gx = gx0 + c, gy = gy0 + r;
            float v[8];
            if (gy >= 0 && gy < H && gx >= 0 && gx + 8 <= W) {
                load8_inside(img, dt, pitch, gx, gy, vec, v);
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) v[e] = outside_px(img, dt, pitch, gx + e, gy, W, H, border, bv, zero_outside);
            }
            float* d = st + r * sw + c;
            *reinterpret_cast<float4*>(d) = make_float4(v[0], v[1], v[2], v[3]);
            *reinterpret_cast<float4*>(d + 4) = make_float4(v[4], v[5], v[6], v[7]);
        }
        return;
    }
    for (int idx = tid; idx < sw * sh; idx += nth) {
        const int r = idx / sw, c = idx - r * sw;
        st[idx] = outside_px(img, dt, pitch, gx0 + c, gy0 + r, W, H, border, bv, zero_outside);
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
    using G = TileGeo<__half, K, PX>;    // halo padded to 8 columns: 16-byte aligned staging
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
                     tid, nth, im.g_vec);
    else
        stage_region(st, SW, SH, im.in, im.in_dt, im.in_pitch, x0 - G::PAD, y0 - R, im.W, im.H, im.border, im.bv, 0,
                     tid, nth, im.in_vec);
    __syncthreads();
    if (tid < bx * by) {
        const int tx = tid % bx, ty = tid / bx;
        float acc[PY][PX];
#pragma unroll
        for (int oy = 0; oy < PY; ++oy)
#pragma unroll
            for (int ox = 0; ox < PX; ++ox) acc[oy][ox] = 0.f;
        // filter row j outermost: its K taps stay in registers while the PY output rows
        // that read input row (oy + j) accumulate (one shared-memory read per tap per tile).
        // The j loop stays rolled: one batch kernel carries every filter side, and fully
        // unrolled bodies for all of them would not fit the instruction cache together.
#pragma unroll 1
        for (int j = 0; j < K; ++j) {
            float wr[K];
#pragma unroll
            for (int i = 0; i < K; ++i) wr[i] = w[j * K + i];
#pragma unroll
            for (int oy = 0; oy < PY; ++oy) {
                float seg[G::SEG];
                load_seg_smem<float, G>(st + (ty * PY + oy + j) * SW + tx * PX, seg);
#pragma unroll
                for (int i = 0; i < K; ++i)
#pragma unroll
                    for (int ox = 0; ox < PX; ++ox) acc[oy][ox] = __fmaf_rn(wr[i], seg[G::LO + ox + i], acc[oy][ox]);
            }
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
    using G = TileGeo<__half, NT, PX>;   // halo padded to 8 columns: 16-byte aligned staging
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
                 nth, im.in_vec);
    __syncthreads();
    float rw[NT], cw[NT];                 // row and column taps, in registers for the tile
#pragma unroll
    for (int i = 0; i < NT; ++i) { rw[i] = w[i]; cw[i] = w[NT + i]; }
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
                for (int ox = 0; ox < PX; ++ox) r4[ox] = __fmaf_rn(rw[i], seg[G::LO + ox + i], r4[ox]);
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
#pragma unroll
                    for (int ox = 0; ox < PX; ++ox) acc[oy][ox] = __fmaf_rn(cw[j], tv[ox], acc[oy][ox]);
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

// ------------------------------------------------------------------ backward tiles
// Tap-gradient partial sums over one tile from staged arrays: gs (gh x gsw, the upstream
// gradient, tile rows at gs_row0) and xs (the operand region, xsw wide, tile-relative
// origin (-rx, -ry + xs_row0)); out[j*kw + i] = sum_p g(p) x(p + (i - rx, j - ry)).
__device__ void tile_wgrad(const float* gs, int gsw, int gs_row0, const float* xs, int xsw, int xs_row0, int TW,
                           int TH, int kw, int kh, float* red, float* out, int tid, int nth) {
    const int cw = (kw + 3) / 4, ngroups = kh * cw;
    const int reps = nth / ngroups > 0 ? nth / ngroups : 1;
    const int gi = tid % ngroups, rep = tid / ngroups;
    const bool active = rep < reps;
    const int j = gi / cw, i0 = (gi % cw) * 4;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    if (active) {
        for (int py = rep; py < TH; py += reps) {
            const float* gr = gs + (gs_row0 + py) * gsw;
            const float* xr = xs + (xs_row0 + py + j) * xsw + i0;
            for (int px = 0; px < TW; ++px) {
                const float gv = gr[px];
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (i0 + k < kw) acc[k] = __fmaf_rn(gv, xr[px + k], acc[k]);
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) red[tid * 4 + k] = active ? acc[k] : 0.f;
    __syncthreads();
    for (int q = tid; q < kw * kh; q += nth) {
        const int jj = q / kw, ii = q % kw;
        const int grp = jj * cw + ii / 4, lane = ii % 4;
        float sum = 0.f;
        for (int r = 0; r < reps; ++r) sum += red[(r * ngroups + grp) * 4 + lane];
        out[q] = sum;
    }
}

// conv2d: input-gradient tile (all but the image's edge pixels under the clamp rule) and
// the tile's tap partial sums.
template <int K, int PY>
__device__ void batch_conv_dx_tile(const BImg& im, int x0, int y0, int bx, int by, float* sm, int tid, int nth) {
    const int TW = 4 * bx, TH = PY * by;
    if (im.gin) {
        batch_conv_tile<K, PY>(im, x0, y0, bx, by, sm, true, im.g, im.g_pitch, im.gin, im.gin_pitch, IMCL_F32, tid, nth);
        __syncthreads();
    }
    if (im.gtaps) {
        // the K x K centred tap gradient by the register-blocked reduction; a kw x kh
        // filter (kw, kh <= K) takes its block of it
        constexpr int R = (K - 1) / 2, JR = WgCfg<K>::JR;
        const int XW = wg_xpitch<K>(TW), XH = TH + K - 1;
        float* gs = sm;
        float* xs = gs + TW * TH;
        stage_region(gs, TW, TH, im.g, IMCL_F32, im.g_pitch, x0, y0, im.W, im.H, IMCL_BORDER_CONSTANT, 0.f, 1, tid, nth,
                     im.g_vec);
        stage_region(xs, XW, XH, im.in, im.in_dt, im.in_pitch, x0 - R, y0 - R, im.W, im.H, im.border, im.bv, 0, tid,
                     nth);
        __syncthreads();
        const int G = (K + JR - 1) / JR, T = nth / G, grp = tid / T, lt = tid - grp * T;
        const bool active = grp < G;
        float acc[JR][K];
#pragma unroll
        for (int jr = 0; jr < JR; ++jr)
#pragma unroll
            for (int i = 0; i < K; ++i) acc[jr][i] = 0.f;
        if (active) wgrad_accumulate<K>(gs, TW, xs, XW, TW, TH, K, grp * JR, lt, T, acc);
        float* kk = sm + nth * JR * K;                  // the K x K sums, after the combine scratch
        wgrad_combine<K>(acc, active, sm, K, T, kk, tid, nth);
        const int tile = (y0 / TH) * im.tiles_x + x0 / TW;
        const int rx = (im.kw - 1) / 2, ry = (im.kh - 1) / 2;
        float* out = im.part + (size_t)tile * im.kw * im.kh;
        for (int q = tid; q < im.kw * im.kh; q += nth) {
            const int j = q / im.kw, i = q - j * im.kw;
            out[q] = kk[(j - ry + R) * K + (i - rx + R)];
        }
    }
}

// conv2d, clamp rule: the input gradient at a chunk of the image's edge pixels, with the
// contributions of clamped taps folded in (the transpose of the clamp).
__device__ void batch_conv_edges(const BImg& im, int chunk, int tid, int nth) {
    const int W = im.W, H = im.H;
    const int ntop = W, nside = H > 2 ? H - 2 : 0;
    const int rows = H > 1 ? 2 * ntop : ntop;
    const int nedge = rows + (W > 1 ? 2 * nside : nside);
    const int rx = (im.kw - 1) / 2, ry = (im.kh - 1) / 2;
    for (int e = chunk * 1024 + tid; e < min(nedge, (chunk + 1) * 1024); e += nth) {
        int qx, qy;
        if (e < rows) {
            qx = e % W;
            qy = e < ntop ? 0 : H - 1;
        } else {
            const int k = e - rows;
            qy = 1 + (k % nside);
            qx = k < nside ? 0 : W - 1;
        }
        const int xlo = qx == 0 ? -rx : qx, xhi = qx == W - 1 ? W - 1 + rx : qx;
        const int ylo = qy == 0 ? -ry : qy, yhi = qy == H - 1 ? H - 1 + ry : qy;
        float acc = 0.f;
        for (int ey = ylo; ey <= yhi; ++ey)
            for (int ex = xlo; ex <= xhi; ++ex)
                for (int j = 0; j < im.kh; ++j) {
                    const int sy = ey - j + ry;
                    if (sy < 0 || sy >= H) continue;
                    for (int i = 0; i < im.kw; ++i) {
                        const int sx = ex - i + rx;
                        if (sx < 0 || sx >= W) continue;
                        acc = __fmaf_rn(im.taps[j * im.kw + i], im.g[(long long)sy * im.g_pitch + sx], acc);
                    }
                }
        im.gin[(long long)qy * im.gin_pitch + qx] = acc;
    }
}

// separable, first backward pass: dt = C^T g on the tile (with the clamp folds on the
// first and last rows) into the plan's dt plane, and the column-tap partial sums
// dcol[j] = sum_p g(p) t(p + (0, j - rc)), t the forward row pass.
template <int R>
__device__ void batch_sep_dt_tile(const BImg& im, int x0, int y0, int TW, int TH, float* sm, int tid, int nth) {
    constexpr int PADR = 8;                             // >= R, 16 bytes of f32
    const int nr = im.kw, nc = im.kh, rr = (nr - 1) / 2, rc = (nc - 1) / 2;
    const int XW = TW + 2 * PADR, HH = TH + 2 * R;      // R >= rc rows of halo
    float* gs = sm;                                     // TW x HH, rows y0 - R ..
    float* w = gs + TW * HH;                            // row taps [0, 16), column taps [16, 32)
    float* red = w + 32;
    for (int i = tid; i < 32; i += nth) w[i] = i < 16 ? (i < nr ? im.taps[i] : 0.f) : (i - 16 < nc ? im.taps2[i - 16] : 0.f);
    stage_region(gs, TW, HH, im.g, IMCL_F32, im.g_pitch, x0, y0 - R, im.W, im.H, IMCL_BORDER_CONSTANT, 0.f, 1, tid, nth,
                 im.g_vec);
    __syncthreads();
    const float* cw = w + 16;
    // dt for the tile's pixels
    if (im.dt) {
        for (int k = tid; k < TW * TH; k += nth) {
            const int py = k / TW, px = k % TW;
            const int gx = x0 + px, gy = y0 + py;
            if (gx >= im.W || gy >= im.H) continue;
            float acc = 0.f;
            for (int j = 0; j < nc; ++j) acc = __fmaf_rn(cw[j], gs[(py + R + rc - j) * TW + px], acc);
            if (im.border == IMCL_BORDER_CLAMP) {
                if (gy == 0)
                    for (int e = -rc; e <= -1; ++e)
                        for (int j = 0; j < nc; ++j) {
                            const int sy = e - j + rc;   // image row, < rc
                            if (sy >= 0 && sy < im.H) acc = __fmaf_rn(cw[j], gs[(sy - y0 + R) * TW + px], acc);
                        }
                if (gy == im.H - 1)
                    for (int e = im.H; e <= im.H - 1 + rc; ++e)
                        for (int j = 0; j < nc; ++j) {
                            const int sy = e - j + rc;
                            if (sy >= 0 && sy < im.H) acc = __fmaf_rn(cw[j], gs[(sy - y0 + R) * TW + px], acc);
                        }
            }
            im.dt[(long long)gy * im.dt_pitch + gx] = acc;
        }
    }
    if (im.gtaps2) {
        // t on rows y0 - rc .. y0 + TH + rc of the tile's columns (boundary rule on x and t)
        float* xs = red + 4 * 256;                      // XW x HH
        float* ts = xs + XW * HH;                       // TW x HH
        stage_region(xs, XW, HH, im.in, im.in_dt, im.in_pitch, x0 - PADR, y0 - R, im.W, im.H, im.border, im.bv, 0,
                     tid, nth, im.in_vec);
        __syncthreads();
        for (int k = tid; k < TW * HH; k += nth) {
            const int r = k / TW, px = k % TW;
            const int gy = y0 - R + r;
            float acc = 0.f;
            if (im.border == IMCL_BORDER_CONSTANT && (gy < 0 || gy >= im.H)) {
                acc = im.bv;
            } else {
                for (int i = 0; i < nr; ++i) acc = __fmaf_rn(w[i], xs[r * XW + px + PADR - rr + i], acc);
            }
            ts[k] = acc;
        }
        __syncthreads();
        const int tile = (y0 / TH) * im.tiles_x + x0 / TW;
        // column taps: the register-blocked reduction with one tap per row (KW = 1, nc tap
        // rows); g rows of the tile start at row R of gs, t rows at offset R - rc
        constexpr int JR = WgCfg<1>::JR;
        const int G = (nc + JR - 1) / JR, T = nth / G, grp = tid / T, lt = tid - grp * T;
        const bool active = grp < G;
        float acc[JR][1];
#pragma unroll
        for (int jr = 0; jr < JR; ++jr) acc[jr][0] = 0.f;
        if (active) wgrad_accumulate<1>(gs + R * TW, TW, ts + (R - rc) * TW, TW, TW, TH, nc, grp * JR, lt, T, acc);
        wgrad_combine<1>(acc, active, red, nc, T, im.part + (size_t)tile * nc, tid, nth);
    }
}

// Row-tap partial sums of a separable tile: out[i] = sum_p dt(p) x(p + (i - rr, 0)), with
// dt staged at columns PADR.. of ds and x at columns PADR - rr + i of xs (rows XW wide).
// x reads start PADR - rr columns in: the aligned column below and D = (PADR - rr) % 4.
template <int NR>
__device__ void batch_row_wgrad(const float* ds, const float* xs, int XW, int TW, int TH, float* red, float* out,
                                int tid, int nth) {
    constexpr int PADR = 8, RR = (NR - 1) / 2, D = (PADR - RR) % 4;
    float acc[1][NR];
#pragma unroll
    for (int i = 0; i < NR; ++i) acc[0][i] = 0.f;
    wgrad_accumulate<NR, D, 1>(ds + PADR, XW, xs + (PADR - RR - D), XW, TW, TH, 1, 0, tid, nth, acc);
    wgrad_combine<NR, 1>(acc, true, red, 1, nth, out, tid, nth);
}

// separable, second backward pass: dx = R^T dt on the tile (with the clamp folds on the
// first and last columns) and the row-tap partials drow[i] = sum_p dt(p) x(p + (i - rr, 0)).
__device__ void batch_sep_dx_tile(const BImg& im, int x0, int y0, int TW, int TH, float* sm, int tid, int nth) {
    constexpr int PADR = 8;
    const int nr = im.kw, rr = (nr - 1) / 2;
    const int XW = TW + 2 * PADR;
    float* ds = sm;                                     // XW x TH, columns x0 - PADR ..
    float* xs = ds + XW * TH;                           // XW x TH
    float* w = xs + XW * TH;
    float* red = w + 16;
    for (int i = tid; i < 16; i += nth) w[i] = i < nr ? im.taps[i] : 0.f;
    stage_region(ds, XW, TH, im.dt, IMCL_F32, im.dt_pitch, x0 - PADR, y0, im.W, im.H, IMCL_BORDER_CONSTANT, 0.f, 1, tid,
                 nth, 16);
    stage_region(xs, XW, TH, im.in, im.in_dt, im.in_pitch, x0 - PADR, y0, im.W, im.H, im.border, im.bv, 0, tid, nth,
                 im.in_vec);
    __syncthreads();
    if (im.gin) {
        for (int k = tid; k < TW * TH; k += nth) {
            const int py = k / TW, px = k % TW;
            const int gx = x0 + px, gy = y0 + py;
            if (gx >= im.W || gy >= im.H) continue;
            float acc = 0.f;
            for (int i = 0; i < nr; ++i) acc = __fmaf_rn(w[i], ds[py * XW + px + PADR + rr - i], acc);
            if (im.border == IMCL_BORDER_CLAMP) {
                if (gx == 0)
                    for (int e = -rr; e <= -1; ++e)
                        for (int i = 0; i < nr; ++i) {
                            const int sx = e - i + rr;
                            if (sx >= 0 && sx < im.W) acc = __fmaf_rn(w[i], ds[py * XW + sx - x0 + PADR], acc);
                        }
                if (gx == im.W - 1)
                    for (int e = im.W; e <= im.W - 1 + rr; ++e)
                        for (int i = 0; i < nr; ++i) {
                            const int sx = e - i + rr;
                            if (sx >= 0 && sx < im.W) acc = __fmaf_rn(w[i], ds[py * XW + sx - x0 + PADR], acc);
                        }
            }
            im.gin[(long long)gy * im.gin_pitch + gx] = acc;
        }
    }
    if (im.gtaps) {
        const int tile = (y0 / TH) * im.tiles_x + x0 / TW;
        const int ntiles = im.tiles_x * im.tiles_y;
        // dt rows of the tile are ds rows 0..TH at columns PADR..; x at columns PADR - rr + i
        float* out = im.part + (size_t)ntiles * im.kh + (size_t)tile * nr;
        switch (nr) {   // row taps: the register-blocked reduction, one tap row
            case 1: batch_row_wgrad<1>(ds, xs, XW, TW, TH, red, out, tid, nth); break;
            case 3: batch_row_wgrad<3>(ds, xs, XW, TW, TH, red, out, tid, nth); break;
            case 5: batch_row_wgrad<5>(ds, xs, XW, TW, TH, red, out, tid, nth); break;
            case 7: batch_row_wgrad<7>(ds, xs, XW, TW, TH, red, out, tid, nth); break;
            case 9: batch_row_wgrad<9>(ds, xs, XW, TW, TH, red, out, tid, nth); break;
            case 11: batch_row_wgrad<11>(ds, xs, XW, TW, TH, red, out, tid, nth); break;
            case 13: batch_row_wgrad<13>(ds, xs, XW, TW, TH, red, out, tid, nth); break;
            default: batch_row_wgrad<15>(ds, xs, XW, TW, TH, red, out, tid, nth); break;
        }
    }
}

// Reduce an image's tap partial sums over its tiles (fixed order) into the gradients.
__device__ void batch_final(const BImg& im, int tid, int nth) {
    const int ntiles = im.tiles_x * im.tiles_y;
    // sum_t part[t * n + q] over the tiles, in tile order, for taps q < n
    auto reduce = [&](const float* part, int n, float* out) {
        for (int q = tid; q < n; q += nth) {
            float s = 0.f;
            for (int t = 0; t < ntiles; ++t) s += part[(size_t)t * n + q];
            out[q] = s;
        }
    };
    if (im.op == IMCL_OP_CONV2D) {
        if (im.gtaps) reduce(im.part, im.kw * im.kh, im.gtaps);
    } else {
        if (im.gtaps2) reduce(im.part, im.kh, im.gtaps2);                                // column taps
        if (im.gtaps) reduce(im.part + (size_t)ntiles * im.kh, im.kw, im.gtaps);        // row taps
    }
}

template <int PY>
__device__ void batch_bwd_dispatch(const BImg& im, const BTile& tl, int bx, int by, float* sm, int tid, int nth) {
    const int TW = 4 * bx, TH = PY * by;
    switch (tl.kind) {
        case BT_CONV_DX:
            switch (im.K) {
                case 3: batch_conv_dx_tile<3, PY>(im, tl.x0, tl.y0, bx, by, sm, tid, nth); break;
                case 5: batch_conv_dx_tile<5, PY>(im, tl.x0, tl.y0, bx, by, sm, tid, nth); break;
                case 7: batch_conv_dx_tile<7, PY>(im, tl.x0, tl.y0, bx, by, sm, tid, nth); break;
                case 9: batch_conv_dx_tile<9, PY>(im, tl.x0, tl.y0, bx, by, sm, tid, nth); break;
                case 11: batch_conv_dx_tile<11, PY>(im, tl.x0, tl.y0, bx, by, sm, tid, nth); break;
                case 13: batch_conv_dx_tile<13, PY>(im, tl.x0, tl.y0, bx, by, sm, tid, nth); break;
                default: batch_conv_dx_tile<15, PY>(im, tl.x0, tl.y0, bx, by, sm, tid, nth); break;
            }
            break;
        case BT_CONV_EDGE: batch_conv_edges(im, tl.x0, tid, nth); break;
        case BT_SEP_DT: batch_sep_dt_tile<kBatchMaxR>(im, tl.x0, tl.y0, TW, TH, sm, tid, nth); break;
        case BT_SEP_DX: batch_sep_dx_tile(im, tl.x0, tl.y0, TW, TH, sm, tid, nth); break;
        default: batch_final(im, tid, nth); break;
    }
}

// Persistent backward phase: CTAs take work items from one list until it is exhausted.
template <int PY>
__global__ void __launch_bounds__(256, 3)
    k_batch_bwd(const BImg* __restrict__ imgs, const BTile* __restrict__ items, int nitems, int* queue, int bx, int by) {
    extern __shared__ __align__(16) float bsm[];
    __shared__ int s_next;
    const int tid = threadIdx.x, nth = blockDim.x;
    for (;;) {
        if (tid == 0) s_next = atomicAdd(queue, 1);
        __syncthreads();
        const int t = s_next;
        if (t >= nitems) break;
        const BTile tl = items[t];
        const BImg im = imgs[tl.img];
        batch_bwd_dispatch<PY>(im, tl, bx, by, bsm, tid, nth);
        __syncthreads();
    }
}

}  // namespace imcl
