// tile_common.cuh -- halo-tile staging and register-block helpers shared by the
// stencil kernels (conv2d, fused sepconv, fused Harris).
//
// A CTA stages the input region [x0 - PAD, x0 + TW + PAD) x [y0 - R, y0 + TH + R) of its
// output tile in shared memory (§5.2 "local memory", Fig. 5: the tile plus the bounding
// box of the stencil).  PAD >= R is rounded up to 16 bytes so the region's first column
// satisfies the TMA alignment rule.  Out-of-image parts follow the boundary rule of §5
// (Fig. 3) once the tile is patched.
#pragma once

#include <cstring>
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace imcl {

// The constant of the constant boundary rule as a pixel of the input type (integer
// images take it as an integer, 16-bit images round it to nearest even).
template <typename Tin>
__device__ __forceinline__ Tin border_pixel(const ConvArgs& a) {
    if constexpr (std::is_integral<Tin>::value) return (Tin)a.bv_i;
    else return Store<Tin, float>::cvt(a.bv_f);
}

template <typename Acc, int N>
struct TapsParam {
    Acc w[N];
};

// Taps as kernel parameters: one value per tap, or (w, w) pairs for the packed forms.
template <typename Acc, int N, int UNR>
using TapsParamFor = typename std::conditional<UNR == IMCL_UNROLL_PACKED, TapsParam<float2, N>, TapsParam<Acc, N>>::type;

inline void set_tap(float& d, float w) { d = w; }
inline void set_tap(int32_t& d, int32_t w) { d = w; }
inline void set_tap(float2& d, float w) { d = make_float2(w, w); }

// ------------------------------------------------------------------ tile geometry
template <typename Tin, int K, int PX>
struct TileGeo {
    static constexpr int R = (K - 1) / 2;
    static constexpr int SZ = (int)sizeof(Tin);
    static constexpr int CV = 16 / SZ;                         // elements per 16-byte chunk
    static constexpr int PAD = round_up(R > 0 ? R : 1, CV);    // staged halo columns per side
    static constexpr int VB = (PX * SZ < 16) ? PX : CV;        // elements per compute load
    static constexpr int SEG = PX + 2 * PAD;                   // row segment a thread loads
    static constexpr int LO = PAD - R;                          // first element a thread uses
    static constexpr int USED = PX + K - 1;                     // elements it uses
};

__device__ __forceinline__ bool tile_inside(int gx0, int gy0, int sw, int sh, int W, int H) {
    return gx0 >= 0 && gy0 >= 0 && gx0 + sw <= W && gy0 + sh <= H;
}

// Make the staged tile follow the boundary rule where it lies outside the image.
// Tile element (r, c) holds image pixel (gx0 + c, gy0 + r).  Requires that the tile
// starts inside the image once the halo is removed (true for every tile of the grid).
template <typename Tin>
__device__ void patch_tile(Tin* st, int sw, int sh, int gx0, int gy0, int W, int H, int border,
                           Tin bv, int tid, int nth) {
    if (border == IMCL_BORDER_CONSTANT) {
        for (int idx = tid; idx < sw * sh; idx += nth) {
            const int r = idx / sw, c = idx - r * sw;
            const int gx = gx0 + c, gy = gy0 + r;
            if (gx < 0 || gx >= W || gy < 0 || gy >= H) st[idx] = bv;
        }
        __syncthreads();
        return;
    }
    const int cl = -gx0;                  // column holding gx = 0
    const int cr = W - 1 - gx0;           // column holding gx = W-1
    const int nl = cl > 0 ? cl : 0;
    const int nr = (sw - 1 - cr) > 0 ? (sw - 1 - cr) : 0;
    const int r0 = gy0 < 0 ? -gy0 : 0;
    const int r1 = (H - gy0) < sh ? (H - gy0) : sh;   // rows [r0, r1) are inside the image
    const int ncol = nl + nr;
    if (ncol > 0) {
        for (int idx = tid; idx < (r1 - r0) * ncol; idx += nth) {
            const int r = r0 + idx / ncol, k = idx % ncol;
            const int c = k < nl ? k : (cr + 1 + (k - nl));
            st[r * sw + c] = st[r * sw + (k < nl ? cl : cr)];
        }
        __syncthreads();
    }
    const int ntop = r0, nbot = sh - r1;
    if (ntop + nbot > 0) {
        for (int idx = tid; idx < (ntop + nbot) * sw; idx += nth) {
            const int k = idx / sw, c = idx - k * sw;
            const int r = k < ntop ? k : (r1 + (k - ntop));
            const int src = k < ntop ? r0 : (r1 - 1);
            st[r * sw + c] = st[src * sw + c];
        }
        __syncthreads();
    }
}

// Cooperative clamped / constant staging of a tile with 16-byte chunks (LOAD_SMEM).
template <typename Tin>
__device__ void coop_load_tile(Tin* st, const Tin* in, long long pitch, int sw, int sh, int gx0,
                               int gy0, int W, int H, int border, Tin bv, bool vec_ok, int tid,
                               int nth) {
    constexpr int CV = 16 / (int)sizeof(Tin);
    const int nch = sw / CV;
    for (int idx = tid; idx < nch * sh; idx += nth) {
        const int r = idx / nch, c = (idx - r * nch) * CV;
        const int gy = gy0 + r, gx = gx0 + c;
        Tin* d = st + r * sw + c;
        if (vec_ok && gy >= 0 && gy < H && gx >= 0 && gx + CV <= W) {
            *reinterpret_cast<uint4*>(d) = __ldg(reinterpret_cast<const uint4*>(in + (long long)gy * pitch + gx));
        } else {
#pragma unroll
            for (int e = 0; e < CV; ++e) {
                const int x = gx + e;
                const bool inside = x >= 0 && x < W && gy >= 0 && gy < H;
                if (inside) d[e] = ldg(in + (long long)gy * pitch + x);
                else if (border == IMCL_BORDER_CONSTANT) d[e] = bv;
                else d[e] = ldg(in + (long long)clampi(gy, 0, H - 1) * pitch + clampi(x, 0, W - 1));
            }
        }
    }
}

// Load the VB-element chunks of a row segment that overlap [LO, LO+USED) from shared
// memory into registers (converted to Acc).
template <typename Tin, typename G, typename Acc>
__device__ __forceinline__ void load_seg_smem(const Tin* rowp, Acc* seg) {
#pragma unroll
    for (int c = 0; c < G::SEG; c += G::VB)
        if (c + G::VB > G::LO && c < G::LO + G::USED) load_vec<Tin, G::VB>(rowp + c, seg + c);
}

// The same from global memory, applying the boundary rule element-wise where needed.
template <typename Tin, typename G, typename Acc>
__device__ __forceinline__ void load_seg_global(const Tin* in, long long pitch, int gy, int gxs, int W,
                                                int H, int border, Acc bv, bool vec_ok, Acc* seg) {
    const bool row_in = gy >= 0 && gy < H;
    const int cy = clampi(gy, 0, H - 1);
    const Tin* rowp = in + (long long)cy * pitch;
#pragma unroll
    for (int c = 0; c < G::SEG; c += G::VB) {
        if (c + G::VB > G::LO && c < G::LO + G::USED) {
            const int gx = gxs + c;
            if (vec_ok && row_in && gx >= 0 && gx + G::VB <= W) {
                ldg_vec<Tin, G::VB>(rowp + gx, seg + c);
            } else {
#pragma unroll
                for (int e = 0; e < G::VB; ++e) {
                    const int x = gx + e;
                    if (row_in && x >= 0 && x < W) seg[c + e] = to_acc(ldg(rowp + x));
                    else if (border == IMCL_BORDER_CONSTANT) seg[c + e] = bv;
                    else seg[c + e] = to_acc(ldg(rowp + clampi(x, 0, W - 1)));
                }
            }
        }
    }
}

// Multiply-accumulate one loaded row segment into the output rows that use it.
// MAP_BLOCKED: the segment is input row (oy0 + yy) of the thread's block, used by every
// output row oy with 0 <= yy - oy < K.
template <typename G, int K, int PX, int PY, int FILT, typename Acc>
__device__ __forceinline__ void fma_row_blocked(const int yy, const Acc* seg, Acc (&acc)[PY][PX],
                                                const Acc* wp) {
#pragma unroll
    for (int oy = 0; oy < PY; ++oy) {
        const int j = yy - oy;
        if (j >= 0 && j < K) {
#pragma unroll
            for (int i = 0; i < K; ++i) {
                const Acc w = wp[j * K + i];
#pragma unroll
                for (int ox = 0; ox < PX; ++ox) acc[oy][ox] = mad(w, seg[G::LO + ox + i], acc[oy][ox]);
            }
        }
    }
}

template <typename Tout, int PX, typename Acc>
__device__ __forceinline__ void store_block_row(Tout* out, long long pitch, int gx, int gy, int W, int H,
                                                bool vec_ok, const Acc* v) {
    if (gy >= H) return;
    Tout* p = out + (long long)gy * pitch + gx;
    constexpr int SB = (PX * (int)sizeof(Tout) > 16) ? 16 / (int)sizeof(Tout) : PX;
    if (vec_ok && gx + PX <= W) {
#pragma unroll
        for (int c = 0; c < PX; c += SB) store_vec<Tout, SB>(p + c, v + c);
    } else {
#pragma unroll
        for (int c = 0; c < PX; ++c)
            if (gx + c < W) p[c] = Store<Tout, Acc>::cvt(v[c]);
    }
}

template <typename T> struct DtypeOf;
template <> struct DtypeOf<uint8_t> { static constexpr int v = IMCL_U8; };
template <> struct DtypeOf<int32_t> { static constexpr int v = IMCL_I32; };
template <> struct DtypeOf<float> { static constexpr int v = IMCL_F32; };
template <> struct DtypeOf<__half> { static constexpr int v = IMCL_F16; };
template <> struct DtypeOf<__nv_bfloat16> { static constexpr int v = IMCL_BF16; };

ConvArgs make_conv_args(const ConvCall& c, const imcl_variant& v, int in_align, int out_align);

// Occupancy of a kernel at a given block size and dynamic shared memory, cached.
int cached_occupancy(const void* fn, int threads, int smem);
imcl_status set_smem_limit(const void* fn, int smem);

}  // namespace imcl
