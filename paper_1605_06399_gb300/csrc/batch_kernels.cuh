// batch_kernels.cuh -- the ragged batch: many images of different sizes, each with its
// own stencil (a conv2d filter of odd side <= 15 or a separable pair of radius <= 7), in
// one persistent launch.
//
// The host sorts every tile of every image into one work list (costliest first) and the
// CTAs of a persistent grid take tiles from it with an atomic counter (no CTA waits on
// another).  In the forward a producer warp per CTA takes the tiles two ahead and brings
// each tile's image rows into shared memory with bulk asynchronous copies, while the
// consumer warps convert the previous tile to f32 (the image's storage type, its boundary
// rule) and run the specialised device code for its operator and filter side: register-
// blocked conv2d rows and the fused row+column separable computation.  In the backward
// the conv2d items' input gradient is that same pipelined kernel run on the upstream
// gradient with flipped taps and a zero border (the adjoint of a correlation); clamp folds
// at the image's edge pixels are added after it.  The rest of the backward runs as a few
// persistent phases of 256-thread CTAs that stage their own tiles (tap-gradient tiles,
// the separable adjoint's two passes, per-image reductions), all recorded in one CUDA
// graph.
#pragma once

#include "bulk_copy.cuh"
#include "tile_common.cuh"
#include "wgrad_tile.cuh"

namespace imcl {

constexpr int kBatchMaxK = 15;    // conv2d side
constexpr int kBatchMaxR = 7;     // separable radius
constexpr int kFinalChunk = 32;  // conv2d taps per reduction work item

// One image operation of the batch (device copy).  Pitches in elements.  16-byte
// aligned: the forward copies descriptors into shared memory with bulk copies.
struct alignas(16) BImg {
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
    float* part;                       // batch-owned partial sums: [tiles][ntap_parts]
    int tiles_x, tiles_y;
    int fold;                          // input-gradient descriptors: add the clamp folds
};

// work item kinds
enum : int {
    BT_FWD = 0,        // forward tile
    BT_CONV_DW = 1,    // conv2d: tap-gradient partial sums of one tile
    BT_SEP_TAPS = 3,   // sep: column- and row-tap partial sums of one tile
    BT_FINAL = 5,      // reduce one image's partial sums to its tap gradients (x0: tap chunk)
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

// Store 4 f32 results at (gx..gx+3, gy) to an image of any output type: one dtype
// branch per group, and 16-, 8- or 4-byte stores where the address allows.
__device__ __forceinline__ uint32_t pack2_out(int dt, float a, float b) {
    if (dt == IMCL_F16) {
        const __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<const uint32_t*>(&h);
    }
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

template <int PX>
__device__ __forceinline__ void store_row_any(void* out, int dt, long long pitch, int gx, int gy, int W, int H,
                                              const float* v) {
    static_assert(PX == 4, "groups of 4 pixels");
    if (gy >= H) return;
    const long long o = (long long)gy * pitch + gx;
    const bool full = gx + 4 <= W;
    if (dt == IMCL_F32) {
        float* p = static_cast<float*>(out) + o;
        if (full && (reinterpret_cast<uintptr_t>(p) & 15) == 0) {
            *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (full || gx + c < W) p[c] = v[c];
        }
        return;
    }
    uint16_t* p = static_cast<uint16_t*>(out) + o;
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    if (full && (a & 7) == 0) {
        *reinterpret_cast<uint2*>(p) = make_uint2(pack2_out(dt, v[0], v[1]), pack2_out(dt, v[2], v[3]));
    } else if (full && (a & 3) == 0) {
        reinterpret_cast<uint32_t*>(p)[0] = pack2_out(dt, v[0], v[1]);
        reinterpret_cast<uint32_t*>(p)[1] = pack2_out(dt, v[2], v[3]);
    } else {
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (full || gx + c < W)
                p[c] = dt == IMCL_F16 ? __half_as_ushort(__float2half_rn(v[c]))
                                      : __bfloat16_as_ushort(__float2bfloat16_rn(v[c]));
    }
}

// ------------------------------------------------------------------ forward tiles
// Tap tables in shared memory hold conv2d filter row j at w + j * kTapStride (16-byte
// aligned rows, read as broadcast vectors).
constexpr int kTapStride = 16;

// conv2d: accumulate one tile from a staged region (rows SW wide, origin (x0 - 8, y0 - R))
// and the K x K taps (rows kTapStride apart) in shared memory, and store it.
template <int K, int PY>
__device__ __forceinline__ void conv_tile_compute(const BImg& im, int x0, int y0, int bx, int by, const float* st,
                                                  int SW, const float* w, const int tid) {
    constexpr int PX = 4;
    using G = TileGeo<__half, K, PX>;    // halo padded to 8 columns: 16-byte aligned staging
    if (tid >= bx * by) return;
    const int tx = tid % bx, ty = tid / bx;
    float acc[PY][PX];
#pragma unroll
    for (int oy = 0; oy < PY; ++oy)
#pragma unroll
        for (int ox = 0; ox < PX; ++ox) acc[oy][ox] = 0.f;
    // filter row j outermost: its K taps (broadcast 16-byte loads) stay in registers while
    // the PY output rows that read input row (oy + j) accumulate.  The j loop stays rolled:
    // one batch kernel carries every filter side, and fully unrolled bodies for all of
    // them would not fit the instruction cache together.
    static_assert(K <= kTapStride, "filter rows wider than the tap table stride");
    constexpr int KV = (K + 3) / 4;
    const float* srow = st + ty * PY * SW + tx * PX;
#pragma unroll 1
    for (int j = 0; j < K; ++j) {
        float wr[4 * KV];
#pragma unroll
        for (int q = 0; q < KV; ++q) {
            const float4 t4 = *reinterpret_cast<const float4*>(w + j * kTapStride + 4 * q);
            wr[4 * q] = t4.x; wr[4 * q + 1] = t4.y; wr[4 * q + 2] = t4.z; wr[4 * q + 3] = t4.w;
        }
#pragma unroll
        for (int oy = 0; oy < PY; ++oy) {
            float seg[G::SEG];
            load_seg_smem<float, G>(srow + (oy + j) * SW, seg);
#pragma unroll
            for (int i = 0; i < K; ++i)
#pragma unroll
                for (int ox = 0; ox < PX; ++ox) acc[oy][ox] = __fmaf_rn(wr[i], seg[G::LO + ox + i], acc[oy][ox]);
        }
    }
#pragma unroll
    for (int oy = 0; oy < PY; ++oy)
        store_row_any<PX>(im.out, im.out_dt, im.out_pitch, x0 + tx * PX, y0 + ty * PY + oy, im.W, im.H, acc[oy]);
}

// The forward runs warp-specialised: 8 consumer warps (256 threads, named barrier 1)
// convert and compute tiles while one producer warp fetches the next ones.  The producer
// takes tile indices from the queue two ahead, and for each tile fills one of two slots
// with bulk asynchronous copies: the image descriptor, and every image row of the tile's
// region widened to whole 16-byte words (the region is (TW + 16) x (TH + 2R) pixels at
// (x0 - 8, y0 - R), clipped to the image).  It writes the taps (centred into the compiled
// side), the per-row byte offsets and the tile origin with plain stores, and arrives on the
// slot's `full` barrier.  A row whose widened span would leave the image's own bytes (the
// first or last row of an image whose start or end is not 16-byte aligned) is not copied:
// its offset is -1 and the consumers read it from global memory.  The consumers convert
// the raw rows to the f32 region under the image's boundary rule, release the slot on its
// `empty` barrier, and compute, so the copies of the next tiles overlap the current one.
constexpr int kFwdConsumers = 256;
constexpr int kFwdThreads = kFwdConsumers + 32;
constexpr int kFwdMaxTaps = kBatchMaxK * kTapStride;   // the largest tap table

// Per-tile record the producer reads (one per forward tile, costliest first).
struct alignas(16) BFwdTile {
    const void* in;          // image base
    const float* taps;       // conv: kh x kw; sep: row taps (kw)
    const float* taps2;      // sep: column taps (kh)
    long long pitch_b;       // row pitch in bytes
    int W, H, K, es;         // size, compiled side, bytes per pixel
    int op, kw, kh, img;     // operator, caller's tap counts, image index
    int x0, y0;              // tile origin
    int flip, pad;           // flip: conv taps read rotated by 180 degrees (the adjoint)
};

// The forward's staged rows are TW + 16 pixels, stored kFwdPitchPad floats further
// apart: a row pitch of 20 words modulo 32 spreads a warp's 16-byte loads from several
// rows over all bank groups.
constexpr int kFwdPitchPad = 4;

struct FwdLayout {
    int rows;        // region rows at the largest radius
    int rp_max;      // raw row pitch in bytes at 4 bytes per pixel
    int slot;        // bytes per slot
    int s_img, s_info, s_row, s_taps, s_raw;   // offsets within a slot
    int slot0, st, tb, w, img, total;          // offsets from the start of shared memory
};

__host__ __device__ inline FwdLayout fwd_layout(int TW, int TH) {
    FwdLayout L;
    const int sw = TW + 16;
    L.rows = TH + 2 * kBatchMaxR;
    L.rp_max = round_up(sw * 4 + 32, 16);
    int o = 0;
    L.s_img = o;  o += (int)sizeof(BImg);
    L.s_info = o; o += 16;
    L.s_row = o;  o += round_up(L.rows * 4, 16);
    L.s_taps = o; o += round_up(kFwdMaxTaps * 4, 16);
    L.s_raw = o;  o += L.rows * L.rp_max;
    L.slot = round_up(o, 128);
    L.slot0 = 128;                                   // barriers and flags below
    L.st = L.slot0 + 2 * L.slot;
    L.tb = L.st + (sw + kFwdPitchPad) * L.rows * 4;
    L.w = L.tb + L.rows * TW * 4;
    L.img = L.w + round_up(kFwdMaxTaps * 4, 16);
    L.total = L.img + (int)sizeof(BImg);
    return L;
}

__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// True on every consumer thread if `p` holds on any of them (named barrier 1).
__device__ __forceinline__ bool consumer_any(bool p) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred a, b;\n\t"
        "setp.ne.u32 a, %1, 0;\n\t"
        "bar.red.or.pred b, 1, 256, a;\n\t"
        "selp.u32 %0, 1, 0, b;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)p)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ float raw_px(const uint8_t* p, int dt) {
    switch (dt) {
        case IMCL_F16: return __half2float(*reinterpret_cast<const __half*>(p));
        case IMCL_BF16: return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(p));
        default: return *reinterpret_cast<const float*>(p);
    }
}

// Producer: fill slot `sl` with tile `ft` (all 32 lanes); tv: this lane's taps (entries
// lane + 32 k of the centred table).  Returns after the arrival on `full`.
__device__ __forceinline__ void fwd_fill(const BFwdTile& ft, const BImg* imgs, uint8_t* sl, const FwdLayout& L,
                                         int TW, int TH, const float* tv, uint64_t* full, int lane) {
    const int R = (ft.K - 1) / 2;
    const int gx0 = ft.x0 - 8, sw = TW + 16, gy0 = ft.y0 - R, sh = TH + 2 * R;
    const int cx0 = max(gx0, 0), cx1 = min(gx0 + sw, ft.W);
    const int cy0 = max(gy0, 0), cy1 = min(gy0 + sh, ft.H);
    const int rp = round_up(sw * ft.es + 32, 16);
    const uintptr_t base = reinterpret_cast<uintptr_t>(ft.in);
    const uintptr_t hi = base + ((uintptr_t)(ft.H - 1) * (uintptr_t)ft.pitch_b + (uintptr_t)ft.W * ft.es);
    int* rowinfo = reinterpret_cast<int*>(sl + L.s_row);
    uint32_t total = lane == 0 ? (uint32_t)sizeof(BImg) : 0u;
    for (int y = cy0 + lane; y < cy1; y += 32) {
        const uintptr_t row = base + (uintptr_t)y * (uintptr_t)ft.pitch_b;
        const uintptr_t s = row + (uintptr_t)cx0 * ft.es, e = row + (uintptr_t)cx1 * ft.es;
        const uintptr_t a0 = s & ~(uintptr_t)15, a1 = (e + 15) & ~(uintptr_t)15;
        if (a0 >= base && a1 <= hi) total += (uint32_t)(a1 - a0);
    }
    total = __reduce_add_sync(0xffffffffu, total);
    if (lane == 0) {
        fence_proxy_async_smem();
        mbar_expect_tx(full, total);
    }
    __syncwarp();
    if (lane == 0) bulk_g2s(sl + L.s_img, imgs + ft.img, (uint32_t)sizeof(BImg), full);
    for (int y = cy0 + lane; y < cy1; y += 32) {
        const uintptr_t row = base + (uintptr_t)y * (uintptr_t)ft.pitch_b;
        const uintptr_t s = row + (uintptr_t)cx0 * ft.es, e = row + (uintptr_t)cx1 * ft.es;
        const uintptr_t a0 = s & ~(uintptr_t)15, a1 = (e + 15) & ~(uintptr_t)15;
        const bool ok = a0 >= base && a1 <= hi;
        if (ok) bulk_g2s(sl + L.s_raw + (y - cy0) * rp, reinterpret_cast<const void*>(a0), (uint32_t)(a1 - a0), full);
        rowinfo[y - cy0] = ok ? (int)(s - a0) : -1;
    }
    float* taps = reinterpret_cast<float*>(sl + L.s_taps);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int i = lane + 32 * k;
        if (i < kFwdMaxTaps) taps[i] = tv[k];
    }
    if (lane == 0) {
        int* info = reinterpret_cast<int*>(sl + L.s_info);
        info[0] = ft.x0;
        info[1] = ft.y0;
        info[2] = rp;
        info[3] = 1;
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(full);
}

// Producer: this lane's entries of the tile's tap table (conv: K rows kTapStride apart
// with the caller's kh x kw centred, zeros elsewhere; sep: NT row taps then NT column
// taps, centred).  ADJ: the input-gradient kernel, whose tiles may ask for the taps
// rotated by 180 degrees.
template <bool ADJ>
__device__ __forceinline__ void fwd_load_taps(const BFwdTile& ft, int lane, float* tv) {
    const bool flip = ADJ && ft.flip;
    const int K = ft.K;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int i = lane + 32 * k;
        float v = 0.f;
        if (ft.op == IMCL_OP_CONV2D) {
            const int j = i / kTapStride, c = i % kTapStride;
            if (j < K && c < K) {
                const int R = (K - 1) / 2;
                const int sj = j - (R - (ft.kh - 1) / 2), sc = c - (R - (ft.kw - 1) / 2);
                if (sj >= 0 && sj < ft.kh && sc >= 0 && sc < ft.kw)
                    v = __ldg(ft.taps + (flip ? (ft.kh - 1 - sj) * ft.kw + (ft.kw - 1 - sc) : sj * ft.kw + sc));
            }
        } else if (i < 2 * K) {
            const int R = (K - 1) / 2;
            if (i < K) {
                const int o = i - (R - (ft.kw - 1) / 2);
                if (o >= 0 && o < ft.kw) v = __ldg(ft.taps + (flip ? ft.kw - 1 - o : o));
            } else {
                const int o = i - K - (R - (ft.kh - 1) / 2);
                if (o >= 0 && o < ft.kh) v = __ldg(ft.taps2 + (flip ? ft.kh - 1 - o : o));
            }
        }
        tv[k] = v;
    }
}

// 4 pixels of a raw row at p (converted to f32), with the widest loads p's alignment
// allows (uniform along a row: the groups of one row are 4 pixels apart).
template <int DT>
__device__ __forceinline__ void raw_load4(const uint8_t* p, float* v) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    if constexpr (DT == IMCL_F32) {
        if ((a & 15) == 0) {
            const float4 q = *reinterpret_cast<const float4*>(p);
            v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
        } else if ((a & 7) == 0) {
            const float2 q0 = reinterpret_cast<const float2*>(p)[0], q1 = reinterpret_cast<const float2*>(p)[1];
            v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) v[e] = reinterpret_cast<const float*>(p)[e];
        }
    } else {
        uint32_t u0, u1;
        if ((a & 7) == 0) {
            const uint2 q = *reinterpret_cast<const uint2*>(p);
            u0 = q.x; u1 = q.y;
        } else if ((a & 3) == 0) {
            u0 = reinterpret_cast<const uint32_t*>(p)[0];
            u1 = reinterpret_cast<const uint32_t*>(p)[1];
        } else {
            const uint16_t* h = reinterpret_cast<const uint16_t*>(p);
            u0 = (uint32_t)h[0] | ((uint32_t)h[1] << 16);
            u1 = (uint32_t)h[2] | ((uint32_t)h[3] << 16);
        }
        if constexpr (DT == IMCL_F16) {
            const float2 f0 = __half22float2(*reinterpret_cast<const __half2*>(&u0));
            const float2 f1 = __half22float2(*reinterpret_cast<const __half2*>(&u1));
            v[0] = f0.x; v[1] = f0.y; v[2] = f1.x; v[3] = f1.y;
        } else {
            v[0] = __uint_as_float(u0 << 16); v[1] = __uint_as_float(u0 & 0xffff0000u);
            v[2] = __uint_as_float(u1 << 16); v[3] = __uint_as_float(u1 & 0xffff0000u);
        }
    }
}

template <int DT>
__device__ __forceinline__ float raw_load1(const uint8_t* p) {
    if constexpr (DT == IMCL_F32) return *reinterpret_cast<const float*>(p);
    else if constexpr (DT == IMCL_F16) return __half2float(*reinterpret_cast<const __half*>(p));
    else return __uint_as_float((uint32_t)*reinterpret_cast<const uint16_t*>(p) << 16);
}

// conv2d forward tile from the staged region st (rows SWP apart, origin (x0 - 8, y0 - R))
// and the tap table w: a thread computes PXC consecutive pixels of one row.  Per filter
// row j it loads its row segment (PXC + K - 1 pixels) once and the K taps as broadcast
// vectors, then runs K * PXC independent-accumulator FMAs.
template <int K, int PXC>
__device__ __forceinline__ void conv_fwd_compute(const BImg& im, int x0, int y0, int TW, const float* st, int SWP,
                                                 const float* w, int tid) {
    constexpr int R = (K - 1) / 2, LO = 8 - R, USED = PXC + K - 1;
    constexpr int C0 = LO / 4 * 4, NCH = (LO + USED - 1) / 4 - LO / 4 + 1, D = LO - C0;
    constexpr int KV = (K + 3) / 4;
    static_assert(K <= kTapStride && PXC % 4 == 0, "tap rows and pixel groups");
    const int nx = TW / PXC;
    const int tx = tid % nx, ty = tid / nx;
    float acc[PXC];
#pragma unroll
    for (int ox = 0; ox < PXC; ++ox) acc[ox] = 0.f;
    const float* srow = st + ty * SWP + tx * PXC + C0;
#pragma unroll 1
    for (int j = 0; j < K; ++j) {
        float wr[4 * KV];
#pragma unroll
        for (int q = 0; q < KV; ++q) {
            const float4 t4 = *reinterpret_cast<const float4*>(w + j * kTapStride + 4 * q);
            wr[4 * q] = t4.x; wr[4 * q + 1] = t4.y; wr[4 * q + 2] = t4.z; wr[4 * q + 3] = t4.w;
        }
        float seg[4 * NCH];
#pragma unroll
        for (int q = 0; q < NCH; ++q) {
            const float4 s4 = *reinterpret_cast<const float4*>(srow + j * SWP + 4 * q);
            seg[4 * q] = s4.x; seg[4 * q + 1] = s4.y; seg[4 * q + 2] = s4.z; seg[4 * q + 3] = s4.w;
        }
#pragma unroll
        for (int i = 0; i < K; ++i)
#pragma unroll
            for (int ox = 0; ox < PXC; ++ox) acc[ox] = __fmaf_rn(wr[i], seg[D + ox + i], acc[ox]);
    }
#pragma unroll
    for (int g = 0; g < PXC / 4; ++g)
        store_row_any<4>(im.out, im.out_dt, im.out_pitch, x0 + tx * PXC + 4 * g, y0 + ty, im.W, im.H, acc + 4 * g);
}

// Consumers: raw rows of slot `sl` -> the f32 region st ((TW + 16) x (TH + 2R)) with the
// image's boundary rule, 4 pixels per item, NG items per row; unrolled so that each
// thread has several rows' loads in flight.
template <int DT, int NG>
__device__ __forceinline__ void fwd_convert_rows(const BImg& im, const int* __restrict__ info,
                                                 const int* __restrict__ rowinfo, const uint8_t* __restrict__ raw,
                                                 int TH, float* __restrict__ st, int tid) {
    constexpr int ES = DT == IMCL_F32 ? 4 : 2;
    constexpr int SW = 4 * NG + kFwdPitchPad;
    const int x0 = info[0], y0 = info[1], rp = info[2];
    const int R = (im.K - 1) / 2, W = im.W, H = im.H;
    const int gx0 = x0 - 8, gy0 = y0 - R, sh = TH + 2 * R;
    const int cx0 = max(gx0, 0), cy0 = max(gy0, 0);
    const bool cst = im.border == IMCL_BORDER_CONSTANT;
    const float bv = im.bv;
#pragma unroll 4
    for (int idx = tid; idx < NG * sh; idx += kFwdConsumers) {
        const int r = idx / NG, c0 = (idx - r * NG) * 4;
        const int gy = gy0 + r, gx = gx0 + c0;
        float v[4];
        if (cst && (gy < 0 || gy >= H)) {
#pragma unroll
            for (int e = 0; e < 4; ++e) v[e] = bv;
        } else {
            const int yy = clampi(gy, 0, H - 1);
            const int off = rowinfo[yy - cy0];
            const uint8_t* rr = raw + (yy - cy0) * rp + off;   // pixel x at rr + (x - cx0) * ES
            if (off >= 0 && gx >= 0 && gx + 4 <= W) {
                raw_load4<DT>(rr + (gx - cx0) * ES, v);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int xx = clampi(gx + e, 0, W - 1);
                    const float u = off >= 0 ? raw_load1<DT>(rr + (xx - cx0) * ES)
                                             : load_px(im.in, DT, im.in_pitch, xx, yy);
                    v[e] = (cst && xx != gx + e) ? bv : u;
                }
            }
        }
        *reinterpret_cast<float4*>(st + r * SW + c0) = make_float4(v[0], v[1], v[2], v[3]);
    }
}

template <int DT>
__device__ __forceinline__ void fwd_convert_dt(const BImg& im, const int* info, const int* rowinfo,
                                               const uint8_t* raw, int TW, int TH, float* st, int tid) {
    if (TW == 64) fwd_convert_rows<DT, 20>(im, info, rowinfo, raw, TH, st, tid);
    else fwd_convert_rows<DT, 36>(im, info, rowinfo, raw, TH, st, tid);
}

// Consumers: the slot's raw rows -> st; taps -> w; the descriptor -> cur.
__device__ __forceinline__ void fwd_convert(const uint8_t* sl, const FwdLayout& L, int TW, int TH, float* st,
                                            float* w, BImg* cur, int tid) {
    const BImg& im = *reinterpret_cast<const BImg*>(sl + L.s_img);
    const int* info = reinterpret_cast<const int*>(sl + L.s_info);
    const int* rowinfo = reinterpret_cast<const int*>(sl + L.s_row);
    const uint8_t* raw = sl + L.s_raw;
    switch (im.in_dt) {
        case IMCL_F16: fwd_convert_dt<IMCL_F16>(im, info, rowinfo, raw, TW, TH, st, tid); break;
        case IMCL_BF16: fwd_convert_dt<IMCL_BF16>(im, info, rowinfo, raw, TW, TH, st, tid); break;
        default: fwd_convert_dt<IMCL_F32>(im, info, rowinfo, raw, TW, TH, st, tid); break;
    }
    const float* taps = reinterpret_cast<const float*>(sl + L.s_taps);
    if (tid < kFwdMaxTaps) w[tid] = taps[tid];
    static_assert(sizeof(BImg) % 16 == 0, "descriptor copies move whole 16-byte words");
    if (tid < (int)(sizeof(BImg) / 16))
        reinterpret_cast<uint4*>(cur)[tid] = reinterpret_cast<const uint4*>(&im)[tid];
}

// separable tile (forward) from the staged region st ((TW + 16) x (TH + 2R)) and taps w
// (NT row taps, NT column taps); the row pass goes to tb ((TH + 2R) x TW).
template <int R, int PY>
__device__ void sep_tile_compute(const BImg& im, int x0, int y0, int bx, int by, const float* st, float* tb,
                                 const float* w, const int tid) {
    constexpr int PX = 4, NT = 2 * R + 1;
    using G = TileGeo<__half, NT, PX>;   // halo padded to 8 columns: 16-byte aligned staging
    const int TW = bx * PX, SW = TW + 2 * G::PAD + kFwdPitchPad, SH = by * PY + 2 * R;
    float rw[NT], cw[NT];                 // row and column taps, in registers for the tile
#pragma unroll
    for (int i = 0; i < NT; ++i) { rw[i] = w[i]; cw[i] = w[NT + i]; }
    const int nseg = TW / PX;
    for (int it = tid; it < SH * nseg; it += kFwdConsumers) {
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
    consumer_sync();
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
__device__ __forceinline__ void batch_fwd_dispatch(const BImg& im, int x0, int y0, int bx, int by, const float* st,
                                                   float* tb, const float* w, int tid) {
    constexpr int PXC = 4 * PY;          // (4 bx / PXC) x (PY by) = bx x by threads
    const int TW = 4 * bx, SWP = TW + 16 + kFwdPitchPad;
    if (im.op == IMCL_OP_CONV2D) {
        switch (im.K) {
            // small filters: 4 x PY blocks (contiguous stores; the segment loads are cheap)
            case 3: conv_tile_compute<3, PY>(im, x0, y0, bx, by, st, SWP, w, tid); break;
            case 5: conv_tile_compute<5, PY>(im, x0, y0, bx, by, st, SWP, w, tid); break;
            case 7: conv_tile_compute<7, PY>(im, x0, y0, bx, by, st, SWP, w, tid); break;
            // larger ones: a row of PXC pixels per thread (fewer shared-memory wavefronts per FMA)
            case 9: conv_fwd_compute<9, PXC>(im, x0, y0, TW, st, SWP, w, tid); break;
            case 11: conv_fwd_compute<11, PXC>(im, x0, y0, TW, st, SWP, w, tid); break;
            case 13: conv_fwd_compute<13, PXC>(im, x0, y0, TW, st, SWP, w, tid); break;
            default: conv_fwd_compute<15, PXC>(im, x0, y0, TW, st, SWP, w, tid); break;
        }
    } else {
        switch (im.K) {
            case 3: sep_tile_compute<1, PY>(im, x0, y0, bx, by, st, tb, w, tid); break;
            case 5: sep_tile_compute<2, PY>(im, x0, y0, bx, by, st, tb, w, tid); break;
            case 7: sep_tile_compute<3, PY>(im, x0, y0, bx, by, st, tb, w, tid); break;
            case 9: sep_tile_compute<4, PY>(im, x0, y0, bx, by, st, tb, w, tid); break;
            case 11: sep_tile_compute<5, PY>(im, x0, y0, bx, by, st, tb, w, tid); break;
            case 13: sep_tile_compute<6, PY>(im, x0, y0, bx, by, st, tb, w, tid); break;
            default: sep_tile_compute<7, PY>(im, x0, y0, bx, by, st, tb, w, tid); break;
        }
    }
}

// Input-gradient tiles of clamped images: the transpose of the clamp folds every read the
// forward made outside the image back onto the edge pixel it was clamped to.  The tile's
// main pass stored z(q) at each pixel q, the correlation of g (zero outside the image)
// with the flipped taps; z at an outside position e is the gradient the forward's read of
// e received, so an edge pixel q adds z(e) for every outside e that clamps to q.
//
// The outside positions that clamp into this tile form up to four bands: left (columns
// -rx .. -1) and right (W .. W - 1 + rx) over the tile's rows, extended by ry rows at the
// image's top and bottom (the corners), and top (rows -ry .. -1) and bottom (H .. H - 1 +
// ry) over the tile's columns.  Step 1 computes z for every band position (one position
// per thread at a time) into zb; step 2 gives each edge pixel of the tile its positions'
// sum in a fixed order (left, right, top, bottom band; rows, then columns).  g is read
// from the staged region (origin (x0 - 8, y0 - R), rows SWP apart), which holds every
// in-image g position these sums reach; terms outside the image are skipped.  conv2d: w
// is the K x K flipped table; separable: NT flipped row taps then NT column taps, the 2D
// filter being their outer product (the clamped separable forward equals the clamped 2D
// correlation with it).  Ends synchronised (named barrier of the consumers).
__device__ void fwd_fold_edges(const BImg& im, int x0, int y0, int TW, int TH, const float* st, int SWP,
                               const float* w, float* zb, int tid) {
    const int W = im.W, H = im.H, K = im.K, R = (K - 1) / 2;
    const int rx = (im.kw - 1) / 2, ry = (im.kh - 1) / 2;
    const bool top = y0 == 0, bot = y0 + TH >= H, lft = x0 == 0, rgt = x0 + TW >= W;
    const int tw = min(TW, W - x0), th = min(TH, H - y0);
    // step 1: z at the band positions
    const int Y0 = top ? -ry : y0, Y1 = bot ? H - 1 + ry : y0 + th - 1;
    const int nL = lft ? rx * (Y1 - Y0 + 1) : 0, nR = rgt ? rx * (Y1 - Y0 + 1) : 0;
    const int nT = top ? ry * tw : 0, nB = bot ? ry * tw : 0;
    const int nz = nL + nR + nT + nB;
    for (int k = tid; k < nz; k += kFwdConsumers) {
        int ex, ey, t = k;
        if (t < nL) { ey = Y0 + t / rx; ex = -rx + t % rx; }
        else if ((t -= nL) < nR) { ey = Y0 + t / rx; ex = W + t % rx; }
        else if ((t -= nR) < nT) { ey = -ry + t / tw; ex = x0 + t % tw; }
        else { t -= nT; ey = H + t / tw; ex = x0 + t % tw; }
        const int a0 = max(0, R - ey), a1 = min(K - 1, H - 1 - ey + R);
        const int b0 = max(0, R - ex), b1 = min(K - 1, W - 1 - ex + R);
        float z = 0.f;
        for (int a = a0; a <= a1; ++a) {
            // g(ex - R + b, ey + a - R) is staged at row ey + a - y0, column ex - R + b - x0 + 8
            const int gb = (ey + a - y0) * SWP + (ex - R - x0 + 8);
            if (im.op == IMCL_OP_CONV2D) {
                const float* wr = w + a * kTapStride;
                for (int b = b0; b <= b1; ++b) z = __fmaf_rn(wr[b], st[gb + b], z);
            } else {
                float rs = 0.f;
                for (int b = b0; b <= b1; ++b) rs = __fmaf_rn(w[b], st[gb + b], rs);
                z = __fmaf_rn(w[K + a], rs, z);
            }
        }
        zb[k] = z;
    }
    consumer_sync();
    // step 2: each edge pixel of the tile (top row, bottom row, then the side columns
    // without the corners) adds the z of the band positions that clamp to it
    const int ntop = top ? tw : 0, nbot = (bot && H > 1) ? tw : 0;
    const int r0 = top ? 1 : y0, r1 = bot ? H - 2 : y0 + th - 1;
    const int nside = max(0, r1 - r0 + 1);
    const int nl = lft ? nside : 0, nr = (rgt && W > 1) ? nside : 0;
    const int n = ntop + nbot + nl + nr;
    for (int k = tid; k < n; k += kFwdConsumers) {
        int qx, qy, t = k;
        if (t < ntop) { qx = x0 + t; qy = 0; }
        else if ((t -= ntop) < nbot) { qx = x0 + t; qy = H - 1; }
        else if ((t -= nbot) < nl) { qx = 0; qy = r0 + t; }
        else { t -= nl; qx = W - 1; qy = r0 + t; }
        const int ya = qy == 0 ? -ry : qy, yb = qy == H - 1 ? H - 1 + ry : qy;
        float acc = 0.f;
        if (qx == 0 && lft)
            for (int ey = ya; ey <= yb; ++ey)
                for (int c = 0; c < rx; ++c) acc += zb[(ey - Y0) * rx + c];
        if (qx == W - 1 && rgt)
            for (int ey = ya; ey <= yb; ++ey)
                for (int c = 0; c < rx; ++c) acc += zb[nL + (ey - Y0) * rx + c];
        if (qy == 0 && top)
            for (int r = 0; r < ry; ++r) acc += zb[nL + nR + r * tw + (qx - x0)];
        if (qy == H - 1 && bot)
            for (int r = 0; r < ry; ++r) acc += zb[nL + nR + nT + r * tw + (qx - x0)];
        float* o = static_cast<float*>(im.out) + (long long)qy * im.out_pitch + qx;
        *o += acc;
    }
    consumer_sync();
}

// Persistent forward (kFwdThreads threads: warps 0-7 consume, warp 8 produces).  ADJ:
// the instantiation that runs the input-gradient tiles of the backward (flipped taps,
// clamp folds); the forward's own instantiation carries neither.
template <int PY, bool ADJ>
__global__ void __launch_bounds__(kFwdThreads, 2)
    k_batch_fwd(const BImg* __restrict__ imgs, const BFwdTile* __restrict__ tiles, int ntiles, int* queue, int bx,
                int by, int* status) {
    extern __shared__ __align__(128) uint8_t fsm[];
    const int TW = 4 * bx, TH = PY * by;
    const FwdLayout L = fwd_layout(TW, TH);
    uint64_t* full = reinterpret_cast<uint64_t*>(fsm);
    uint64_t* empty = full + 2;
    volatile int* abort_flag = reinterpret_cast<volatile int*>(fsm + 64);
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init(&empty[0], kFwdConsumers / 32);
        mbar_init(&empty[1], kFwdConsumers / 32);
        *abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();

    if (tid >= kFwdConsumers) {
        // ---------------- producer warp
        const int lane = tid - kFwdConsumers;
        int raw_next = lane == 0 ? atomicAdd(queue, 1) : 0;
        int cur = __shfl_sync(0xffffffffu, raw_next, 0);
        raw_next = lane == 0 ? atomicAdd(queue, 1) : 0;
        BFwdTile ft{};
        if (cur < ntiles) ft = tiles[cur];
        int issued[2] = {-1, -1};
        for (int i = 0;; ++i) {
            const int b = i & 1;
            const int nxt = __shfl_sync(0xffffffffu, raw_next, 0);
            BFwdTile ftn{};
            if (nxt < ntiles) {
                ftn = tiles[nxt];                               // used next iteration
                raw_next = lane == 0 ? atomicAdd(queue, 1) : 0; // its index, the one after
            } else {
                raw_next = ntiles;
            }
            float tv[8];
            if (cur < ntiles) fwd_load_taps<ADJ>(ft, lane, tv);
            bool ok = true;
            if (i >= 2) ok = mbar_wait(&empty[b], ((i >> 1) - 1) & 1u, status) && !*abort_flag;
            if (!__all_sync(0xffffffffu, ok)) {
                // consumers gone: wait for this warp's copies still in flight, then leave
                for (int q = 0; q < 2; ++q)
                    if (lane == 0 && issued[q] >= 0) mbar_wait(&full[q], issued[q] & 1u, nullptr);
                break;
            }
            uint8_t* sl = fsm + L.slot0 + b * L.slot;
            if (cur >= ntiles) {
                if (lane == 0) {
                    reinterpret_cast<int*>(sl + L.s_info)[3] = 0;
                    mbar_arrive(&full[b]);
                }
                break;
            }
            fwd_fill(ft, imgs, sl, L, TW, TH, tv, &full[b], lane);
            issued[b] = i >> 1;
            cur = nxt;
            ft = ftn;
        }
        return;
    }

    // ---------------- consumers
    float* st = reinterpret_cast<float*>(fsm + L.st);
    float* tb = reinterpret_cast<float*>(fsm + L.tb);
    float* w = reinterpret_cast<float*>(fsm + L.w);
    BImg* cur = reinterpret_cast<BImg*>(fsm + L.img);
    for (int i = 0;; ++i) {
        const int b = i & 1;
        const bool ok = mbar_wait(&full[b], (i >> 1) & 1u, status);
        if (consumer_any(!ok)) {
            if (tid == 0) *abort_flag = 1;
            break;
        }
        const uint8_t* sl = fsm + L.slot0 + b * L.slot;
        const int* info = reinterpret_cast<const int*>(sl + L.s_info);
        if (info[3] == 0) break;
        const int x0 = info[0], y0 = info[1];
        fwd_convert(sl, L, TW, TH, st, w, cur, tid);
        __syncwarp();
        if ((tid & 31) == 0) mbar_arrive(&empty[b]);   // this warp is done with the slot
        consumer_sync();
        batch_fwd_dispatch<PY>(*cur, x0, y0, bx, by, st, tb, w, tid);
        consumer_sync();   // st, tb, w and cur are reused by the next tile
        if constexpr (ADJ) {
            if (cur->fold)     // the tile's own stores are visible to the consumers after the barrier
                fwd_fold_edges(*cur, x0, y0, 4 * bx, PY * by, st, 4 * bx + 16 + kFwdPitchPad, w, tb, tid);
        }
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

// Tap rows per thread in the batch's tap-gradient tiles: JR x K accumulators, the 32
// values of a 4 x 8 block of g and one x row segment must fit the registers of a kernel
// that runs three CTAs of 256 threads per SM.
template <int K>
struct BatchWg {
    static constexpr int JR = K <= 7 ? 4 : (K <= 9 ? 3 : 2);
};

// conv2d: the tap-gradient partial sums of one tile, dw[j][i] = sum_p g(p) x(p + (i - rx,
// j - ry)) over the tile's pixels, by the register-blocked reduction on the K x K centred
// form (a kw x kh filter, kw, kh <= K, takes its block of it).
template <int K>
__device__ void batch_conv_dw_tile(const BImg& im, int x0, int y0, int TW, int TH, float* sm, int tid, int nth) {
    constexpr int R = (K - 1) / 2, JR = BatchWg<K>::JR;
    // x staged from column x0 - 8 (16-byte chunks); the reduction's region starts at x0 - R,
    // (8 - R) columns in: the aligned column C below it and D = (8 - R) % 4 more
    constexpr int C = (8 - R) / 4 * 4, D = (8 - R) % 4;
    const int XW = round_up(C + wg_xpitch<K>(TW) + 4, 8), XH = TH + K - 1;
    float* gs = sm;
    float* xs = gs + TW * TH;
    stage_region(gs, TW, TH, im.g, IMCL_F32, im.g_pitch, x0, y0, im.W, im.H, IMCL_BORDER_CONSTANT, 0.f, 1, tid, nth,
                 im.g_vec);
    stage_region(xs, XW, XH, im.in, im.in_dt, im.in_pitch, x0 - 8, y0 - R, im.W, im.H, im.border, im.bv, 0, tid, nth,
                 im.in_vec);
    __syncthreads();
    const int G = (K + JR - 1) / JR, T = nth / G, grp = tid / T, lt = tid - grp * T;
    const bool active = grp < G;
    float acc[JR][K];
#pragma unroll
    for (int jr = 0; jr < JR; ++jr)
#pragma unroll
        for (int i = 0; i < K; ++i) acc[jr][i] = 0.f;
    if (active) wgrad_accumulate<K, D, JR>(gs, TW, xs + C, XW, TW, TH, K, grp * JR, lt, T, acc);
    float* kk = sm + nth * JR * K;                  // the K x K sums, after the combine scratch
    wgrad_combine_wide<K, JR>(acc, active, sm, K, T, kk, tid, nth);
    const int tile = (y0 / TH) * im.tiles_x + x0 / TW;
    const int rx = (im.kw - 1) / 2, ry = (im.kh - 1) / 2;
    float* out = im.part + (size_t)tile * im.kw * im.kh;
    for (int q = tid; q < im.kw * im.kh; q += nth) {
        const int j = q / im.kw, i = q - j * im.kw;
        out[q] = kk[(j - ry + R) * K + (i - rx + R)];
    }
}

// The forward row pass t = R x on HH staged rows (x at columns PADR = 8 .. of xs, rows
// XW wide; image row gy0 + r) into ts (TW wide), 4 pixels per item from one 20-float
// segment; the constant rule gives t the constant on rows outside the image.
template <int NR>
__device__ __forceinline__ void batch_sep_rows_t(const BImg& im, const float* xs, int XW, float* ts, int TW, int HH,
                                                 int gy0, const float* w, int tid, int nth) {
    constexpr int RR = (NR - 1) / 2, PADR = 8;
    float wr[NR];
#pragma unroll
    for (int i = 0; i < NR; ++i) wr[i] = w[i];
    const int ng = TW / 4;
    for (int k = tid; k < ng * HH; k += nth) {
        const int r = k / ng, px = (k - r * ng) * 4;
        const int gy = gy0 + r;
        float acc[4];
        if (im.border == IMCL_BORDER_CONSTANT && (gy < 0 || gy >= im.H)) {
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = im.bv;
        } else {
            float seg[20];
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                const float4 s4 = *reinterpret_cast<const float4*>(xs + r * XW + px + 4 * q);
                seg[4 * q] = s4.x; seg[4 * q + 1] = s4.y; seg[4 * q + 2] = s4.z; seg[4 * q + 3] = s4.w;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = 0.f;
#pragma unroll
            for (int i = 0; i < NR; ++i)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[q] = __fmaf_rn(wr[i], seg[PADR - RR + i + q], acc[q]);
        }
        *reinterpret_cast<float4*>(ts + r * TW + px) = make_float4(acc[0], acc[1], acc[2], acc[3]);
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
    wgrad_combine_wide<NR, 1>(acc, true, red, 1, nth, out, tid, nth);
}

// separable: the tile's tap-gradient partial sums, from one staging of g (zero outside
// the image) and of x (the image's rule), rows y0 - R .. y0 + TH + R:
//   column taps  dcol[j] = sum_p g(p) t(p + (0, j - rc)),  t = R x the forward row pass;
//   row taps     drow[i] = sum_p dt(p) x(p + (i - rr, 0)), dt = C^T g the column adjoint
//                (with the clamp folds on the image's first and last rows).
// R: the item's compiled radius (>= its column radius rc).
// The input gradient itself (R^T dt) runs in the pipelined tile kernel, so dt never
// leaves shared memory.
template <int R>
__device__ void batch_sep_taps_tile(const BImg& im, int x0, int y0, int TW, int TH, float* sm, int tid, int nth) {
    constexpr int PADR = 8;                             // >= R, 16 bytes of f32
    const int nr = im.kw, nc = im.kh, rc = (nc - 1) / 2;
    const int XW = TW + 2 * PADR, HH = TH + 2 * R;      // R >= rc rows of halo
    float* gs = sm;                                     // TW x HH, rows y0 - R ..
    float* xs = gs + TW * HH;                           // XW x HH, origin (x0 - PADR, y0 - R)
    float* u = xs + XW * HH;                            // t (TW x HH), later dt (XW x TH, columns PADR ..)
    float* w = u + max(TW * HH, XW * TH);               // row taps [0, 16), column taps [16, 32)
    float* red = w + 32;                                // the column-tap combine (nth * 4 floats)
    for (int i = tid; i < 32; i += nth) w[i] = i < 16 ? (i < nr ? im.taps[i] : 0.f) : (i - 16 < nc ? im.taps2[i - 16] : 0.f);
    stage_region(gs, TW, HH, im.g, IMCL_F32, im.g_pitch, x0, y0 - R, im.W, im.H, IMCL_BORDER_CONSTANT, 0.f, 1, tid, nth,
                 im.g_vec);
    stage_region(xs, XW, HH, im.in, im.in_dt, im.in_pitch, x0 - PADR, y0 - R, im.W, im.H, im.border, im.bv, 0, tid,
                 nth, im.in_vec);
    __syncthreads();
    const int tile = (y0 / TH) * im.tiles_x + x0 / TW;
    const int ntiles = im.tiles_x * im.tiles_y;
    if (im.gtaps2) {
        float* ts = u;
        switch (nr) {
            case 1: batch_sep_rows_t<1>(im, xs, XW, ts, TW, HH, y0 - R, w, tid, nth); break;
            case 3: batch_sep_rows_t<3>(im, xs, XW, ts, TW, HH, y0 - R, w, tid, nth); break;
            case 5: batch_sep_rows_t<5>(im, xs, XW, ts, TW, HH, y0 - R, w, tid, nth); break;
            case 7: batch_sep_rows_t<7>(im, xs, XW, ts, TW, HH, y0 - R, w, tid, nth); break;
            case 9: batch_sep_rows_t<9>(im, xs, XW, ts, TW, HH, y0 - R, w, tid, nth); break;
            case 11: batch_sep_rows_t<11>(im, xs, XW, ts, TW, HH, y0 - R, w, tid, nth); break;
            case 13: batch_sep_rows_t<13>(im, xs, XW, ts, TW, HH, y0 - R, w, tid, nth); break;
            default: batch_sep_rows_t<15>(im, xs, XW, ts, TW, HH, y0 - R, w, tid, nth); break;
        }
        __syncthreads();
        // column taps: the register-blocked reduction with one tap per row (KW = 1, nc tap
        // rows); g rows of the tile start at row R of gs, t rows at offset R - rc
        constexpr int JR = WgCfg<1>::JR;
        const int G = (nc + JR - 1) / JR, T = nth / G, grp = tid / T, lt = tid - grp * T;
        const bool active = grp < G;
        float acc[JR][1];
#pragma unroll
        for (int jr = 0; jr < JR; ++jr) acc[jr][0] = 0.f;
        if (active) wgrad_accumulate<1>(gs + R * TW, TW, ts + (R - rc) * TW, TW, TW, TH, nc, grp * JR, lt, T, acc);
        wgrad_combine_wide<1>(acc, active, red, nc, T, im.part + (size_t)tile * nc, tid, nth);   // ends synchronised
    }
    if (im.gtaps) {
        // dt = C^T g on the tile's pixels (zero outside the image), 4 pixels of a row per
        // item, into u with rows XW apart and the tile at columns PADR ..
        float* ds = u;
        const float* cw = w + 16;
        const int ng = TW / 4;
        for (int k = tid; k < ng * TH; k += nth) {
            const int py = k / ng, px = (k - py * ng) * 4;
            const int gx = x0 + px, gy = y0 + py;
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            if (gy < im.H && gx < im.W) {
                for (int j = 0; j < nc; ++j) {
                    const float4 s4 = *reinterpret_cast<const float4*>(gs + (py + R + rc - j) * TW + px);
                    acc[0] = __fmaf_rn(cw[j], s4.x, acc[0]);
                    acc[1] = __fmaf_rn(cw[j], s4.y, acc[1]);
                    acc[2] = __fmaf_rn(cw[j], s4.z, acc[2]);
                    acc[3] = __fmaf_rn(cw[j], s4.w, acc[3]);
                }
                if (im.border == IMCL_BORDER_CLAMP && (gy == 0 || gy == im.H - 1)) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (gy == 0)
                            for (int e = -rc; e <= -1; ++e)
                                for (int j = 0; j < nc; ++j) {
                                    const int sy = e - j + rc;   // image row, < rc
                                    if (sy >= 0 && sy < im.H) acc[q] = __fmaf_rn(cw[j], gs[(sy - y0 + R) * TW + px + q], acc[q]);
                                }
                        if (gy == im.H - 1)
                            for (int e = im.H; e <= im.H - 1 + rc; ++e)
                                for (int j = 0; j < nc; ++j) {
                                    const int sy = e - j + rc;
                                    if (sy >= 0 && sy < im.H) acc[q] = __fmaf_rn(cw[j], gs[(sy - y0 + R) * TW + px + q], acc[q]);
                                }
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (gx + q >= im.W) acc[q] = 0.f;
            *reinterpret_cast<float4*>(ds + py * XW + PADR + px) = make_float4(acc[0], acc[1], acc[2], acc[3]);
        }
        __syncthreads();
        // row taps: the register-blocked reduction, one tap row; x rows of the tile start at
        // row R of xs; the combine scratch takes gs, which nothing reads any more
        float* out = im.part + (size_t)ntiles * nc + (size_t)tile * nr;
        const float* xt = xs + R * XW;
        switch (nr) {
            case 1: batch_row_wgrad<1>(ds, xt, XW, TW, TH, gs, out, tid, nth); break;
            case 3: batch_row_wgrad<3>(ds, xt, XW, TW, TH, gs, out, tid, nth); break;
            case 5: batch_row_wgrad<5>(ds, xt, XW, TW, TH, gs, out, tid, nth); break;
            case 7: batch_row_wgrad<7>(ds, xt, XW, TW, TH, gs, out, tid, nth); break;
            case 9: batch_row_wgrad<9>(ds, xt, XW, TW, TH, gs, out, tid, nth); break;
            case 11: batch_row_wgrad<11>(ds, xt, XW, TW, TH, gs, out, tid, nth); break;
            case 13: batch_row_wgrad<13>(ds, xt, XW, TW, TH, gs, out, tid, nth); break;
            default: batch_row_wgrad<15>(ds, xt, XW, TW, TH, gs, out, tid, nth); break;
        }
    }
}

// Reduce an image's tap partial sums over its tiles into the gradients.  A conv2d image's
// taps are split into work items of kFinalChunk taps (chunk = the item's x0), so a large
// filter over many tiles spreads over several CTAs.  The order of the additions depends
// only on the tile count, the item's tap count m and the block size: G = min(nth / m,
// tiles) thread groups take the tiles t = g, g + G, ..., each thread keeps eight running
// sums over consecutive rounds of its tiles (eight loads in flight) and adds them in a
// fixed tree, and the group sums are added in group order.
__device__ void batch_final(const BImg& im, int chunk, float* red, int tid, int nth) {
    const int ntiles = im.tiles_x * im.tiles_y;
    // taps q0 .. q1 - 1 of a set of n: part[t * n + q] summed over the tiles t
    auto reduce = [&](const float* part, int n, int q0, int q1, float* out) {
        const int m = q1 - q0;
        const int G = max(1, min(nth / m, ntiles));
        const int g = tid / m, q = q0 + (tid - g * m);
        if (g < G) {
            float a[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            int t = g;
            for (; t + 7 * G < ntiles; t += 8 * G) {
#pragma unroll
                for (int u = 0; u < 8; ++u) a[u] += part[(size_t)(t + u * G) * n + q];
            }
            for (; t < ntiles; t += G) a[0] += part[(size_t)t * n + q];
            red[tid] = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
        }
        __syncthreads();
        if (tid < m) {
            float s = 0.f;
            for (int k = 0; k < G; ++k) s += red[k * m + tid];
            out[q0 + tid] = s;
        }
        __syncthreads();
    };
    if (im.op == IMCL_OP_CONV2D) {
        const int n = im.kw * im.kh, q0 = chunk * kFinalChunk;
        if (im.gtaps) reduce(im.part, n, q0, min(n, q0 + kFinalChunk), im.gtaps);
    } else {
        if (im.gtaps2) reduce(im.part, im.kh, 0, im.kh, im.gtaps2);                                  // column taps
        if (im.gtaps) reduce(im.part + (size_t)ntiles * im.kh, im.kw, 0, im.kw, im.gtaps);          // row taps
    }
}

// Work-item classes of the backward phases, one kernel each (a kernel then carries only
// the device code of its class, which keeps its instruction footprint and register
// budget to that class).
enum : int { BCLS_CONV_TAPS = 0, BCLS_SEP_TAPS = 1, BCLS_FINAL = 2 };

template <int PY, int CLS>
__device__ __forceinline__ void batch_bwd_dispatch(const BImg& im, const BTile& tl, int bx, int by, float* sm, int tid,
                                                   int nth) {
    const int TW = 4 * bx, TH = PY * by;
    if constexpr (CLS == BCLS_CONV_TAPS) {
        switch (im.K) {
            case 3: batch_conv_dw_tile<3>(im, tl.x0, tl.y0, TW, TH, sm, tid, nth); break;
            case 5: batch_conv_dw_tile<5>(im, tl.x0, tl.y0, TW, TH, sm, tid, nth); break;
            case 7: batch_conv_dw_tile<7>(im, tl.x0, tl.y0, TW, TH, sm, tid, nth); break;
            case 9: batch_conv_dw_tile<9>(im, tl.x0, tl.y0, TW, TH, sm, tid, nth); break;
            case 11: batch_conv_dw_tile<11>(im, tl.x0, tl.y0, TW, TH, sm, tid, nth); break;
            case 13: batch_conv_dw_tile<13>(im, tl.x0, tl.y0, TW, TH, sm, tid, nth); break;
            default: batch_conv_dw_tile<15>(im, tl.x0, tl.y0, TW, TH, sm, tid, nth); break;
        }
    } else if constexpr (CLS == BCLS_SEP_TAPS) {
        switch (im.K) {   // the staged halo rows follow the item's radius
            case 3: batch_sep_taps_tile<1>(im, tl.x0, tl.y0, TW, TH, sm, tid, nth); break;
            case 5: batch_sep_taps_tile<2>(im, tl.x0, tl.y0, TW, TH, sm, tid, nth); break;
            case 7: batch_sep_taps_tile<3>(im, tl.x0, tl.y0, TW, TH, sm, tid, nth); break;
            case 9: batch_sep_taps_tile<4>(im, tl.x0, tl.y0, TW, TH, sm, tid, nth); break;
            case 11: batch_sep_taps_tile<5>(im, tl.x0, tl.y0, TW, TH, sm, tid, nth); break;
            case 13: batch_sep_taps_tile<6>(im, tl.x0, tl.y0, TW, TH, sm, tid, nth); break;
            default: batch_sep_taps_tile<7>(im, tl.x0, tl.y0, TW, TH, sm, tid, nth); break;
        }
    } else {
        batch_final(im, tl.x0, sm, tid, nth);
    }
}

// Persistent backward phase: CTAs take work items of one class from one list until it is
// exhausted.
template <int PY, int CLS>
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
        batch_bwd_dispatch<PY, CLS>(im, tl, bx, by, bsm, tid, nth);
        __syncthreads();
    }
}

}  // namespace imcl
