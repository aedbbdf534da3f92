// backward_kernels.cuh -- building blocks of the adjoint (backward) passes.
//
// A forward correlation with the clamped rule reads in(clamp(p + o)).  Write it as a
// correlation on the image extended by clamping, E in.  Its adjoint applied to an
// upstream gradient g is then
//     dx = E^T ( corr(g0, flip(w)) on the extended domain ),
// g0 being g with zeros outside the image and flip(w)[m] = w[K-1-m].  Inside the image
// (away from the first and last row and column) E^T is the identity, so the bulk of dx
// is a correlation of g with the flipped taps under a zero border: the forward kernels
// compute it.  E^T sums every extended position onto the pixel it clamps to, which only
// touches the first and last rows and columns; the edge kernels below recompute those
// pixels with the folded sums.  Under the constant rule outside reads carry no input,
// so the zero-border correlation is the whole input gradient.
//
// The tap gradient dw[o] = sum_p g(p) in_b(p + o) is reduced in two fixed-order stages
// (per-CTA partials over a static tile assignment, then a tree per tap), so results are
// deterministic run to run.
#pragma once

#include "wgrad_tile.cuh"

namespace imcl {

constexpr int kWgTileW = 128, kWgTileH = 64;  // tile of the tap-gradient reduction (largest)

// Short tap rows are memory-bound: half-height tiles and three resident CTAs per SM keep
// more loads in flight.
template <int KW>
struct WgLaunch {
    static constexpr int TH = KW <= 5 ? kWgTileH / 2 : kWgTileH;
    static constexpr int MIN_CTAS = KW <= 5 ? 3 : 2;
};
constexpr int kWgMaxParts = 1024;             // CTAs (partial sums per tap) at most
constexpr int kMaxAdjTaps = 33 * 33;

struct AdjTaps {                  // taps of up to two channels for the edge kernels
    float w1[kMaxK * kMaxK];
    float w2[kMaxK * kMaxK];
};

__device__ __forceinline__ float g0_at(const float* g, long long pitch, int x, int y, int W, int H) {
    return (x >= 0 && x < W && y >= 0 && y < H) ? g[(long long)y * pitch + x] : 0.f;
}

// Recompute dx at every pixel of the first/last row and column: the folded adjoint of
// one or two clamped correlations (kw x kh taps each, kw, kh <= 15).  Overwrites.  One
// warp per edge pixel: the lanes split the taps, then add their sums in a fixed tree.
__global__ void __launch_bounds__(256)
    k_adjoint_edges_2d(float* dx, long long dx_pitch, const float* g1, long long g1_pitch, const float* g2,
                       long long g2_pitch, int W, int H, int kw, int kh, const float* w1_dev, const float* w2_dev,
                       const __grid_constant__ AdjTaps tp) {
    const int ntop = W, nside = H > 2 ? H - 2 : 0;
    const int nedge = (H > 1 ? 2 * ntop : ntop) + (W > 1 ? 2 * nside : nside);
    const int lane = threadIdx.x & 31;
    const int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (e >= nedge) return;                       // whole warps leave together
    int qx, qy;
    const int rows = H > 1 ? 2 * ntop : ntop;
    if (e < rows) {
        qx = e % W;
        qy = e < ntop ? 0 : H - 1;
    } else {
        const int k = e - rows;
        qy = 1 + (k % nside);
        qx = k < nside ? 0 : W - 1;
    }
    const int rx = (kw - 1) / 2, ry = (kh - 1) / 2;
    const int xlo = qx == 0 ? -rx : qx, xhi = qx == W - 1 ? W - 1 + rx : qx;
    const int ylo = qy == 0 ? -ry : qy, yhi = qy == H - 1 ? H - 1 + ry : qy;
    const float* w1 = w1_dev ? w1_dev : tp.w1;
    const float* w2 = w2_dev ? w2_dev : tp.w2;
    float acc = 0.f;
    for (int ey = ylo; ey <= yhi; ++ey)
        for (int ex = xlo; ex <= xhi; ++ex)
            for (int t = lane; t < kw * kh; t += 32) {
                const int j = t / kw, i = t - j * kw;
                const int sx = ex - i + rx, sy = ey - j + ry;
                acc = __fmaf_rn(w1[t], g0_at(g1, g1_pitch, sx, sy, W, H), acc);
                if (g2) acc = __fmaf_rn(w2[t], g0_at(g2, g2_pitch, sx, sy, W, H), acc);
            }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) dx[(long long)qy * dx_pitch + qx] = acc;
}

// Add the folded contributions of a clamped 1D correlation along one axis (axis 0: x,
// axis 1: y) to the first and last column / row of dst (dst already holds the
// zero-border adjoint).  n taps, n <= 33.
__global__ void __launch_bounds__(256)
    k_fold_1d(float* dst, long long dst_pitch, const float* g, long long g_pitch, int W, int H, int n, int axis,
              const float* w_dev, const __grid_constant__ TapsParam<float, 33> tp) {
    const int L = axis == 0 ? W : H;        // length along the folded axis
    const int M = axis == 0 ? H : W;        // lines to treat
    const int line = blockIdx.x * blockDim.x + threadIdx.x;
    if (line >= M) return;
    const float* w = w_dev ? w_dev : tp.w;
    const int r = (n - 1) / 2;
    auto gat = [&](int along) -> float {
        if (along < 0 || along >= L) return 0.f;
        return axis == 0 ? g[(long long)line * g_pitch + along] : g[(long long)along * g_pitch + line];
    };
    float lo = 0.f, hi = 0.f;
    for (int e = -r; e <= -1; ++e)
        for (int j = 0; j < n; ++j) lo = __fmaf_rn(w[j], gat(e - j + r), lo);
    for (int e = L; e <= L - 1 + r; ++e)
        for (int j = 0; j < n; ++j) hi = __fmaf_rn(w[j], gat(e - j + r), hi);
    float* d0 = axis == 0 ? dst + (long long)line * dst_pitch : dst + line;
    const long long step = axis == 0 ? 1 : dst_pitch;
    if (L == 1) {
        d0[0] += lo + hi;
    } else {
        d0[0] += lo;
        d0[(long long)(L - 1) * step] += hi;
    }
}

// Per-CTA partial sums of dw[j][i] = sum_p g(p) x_b(p + (i - rx, j - ry)), KW taps per
// tap row (compile time, odd, <= 33), kh tap rows (runtime, <= 33); x is f32, f16 or
// bf16 (x_dt), bvf the constant border value as that type reads back in f32.  A CTA
// stages a kWgTileW x kWgTileH tile of g and the matching region of x (boundary rule
// applied) in shared memory -- with 16-byte loads for tiles inside the image when the
// rows are 16-byte aligned (vec) -- and reduces it with wgrad_accumulate (4 x 8 pixel
// blocks, JR tap rows x KW columns per thread; about 27 FMAs per shared-memory load for
// 11 x 11 taps).  Tiles go to CTAs statically (t = blockIdx.x + k gridDim.x) and the
// threads are combined in a fixed order: partials[blockIdx.x * KW*kh + tap],
// deterministic.
template <int KW>
constexpr int wgrad_smem_bytes(int kh, int nth) {
    return 4 * ((kWgTileW * WgLaunch<KW>::TH + wg_xpitch<KW>(kWgTileW) * (WgLaunch<KW>::TH + kh - 1)) >
                        nth * WgCfg<KW>::JR * KW
                    ? (kWgTileW * WgLaunch<KW>::TH + wg_xpitch<KW>(kWgTileW) * (WgLaunch<KW>::TH + kh - 1))
                    : nth * WgCfg<KW>::JR * KW);
}

// one x pixel of type x_dt (f32, f16 or bf16) widened to f32
__device__ __forceinline__ float load_px_f32(const void* x, int x_dt, long long o) {
    if (x_dt == IMCL_F32) return static_cast<const float*>(x)[o];
    if (x_dt == IMCL_F16) return __half2float(static_cast<const __half*>(x)[o]);
    return __bfloat162float(static_cast<const __nv_bfloat16*>(x)[o]);
}

template <int KW>
__global__ void __launch_bounds__(256, WgLaunch<KW>::MIN_CTAS)
    k_wgrad_partial(const float* g, long long g_pitch, const void* x, int x_dt, long long x_pitch, int W, int H,
                    int kh, int border, float bvf, int vec, float* partials) {
    extern __shared__ __align__(16) float wsm[];
    constexpr int JR = WgCfg<KW>::JR, XW = wg_xpitch<KW>(kWgTileW), TH_ = WgLaunch<KW>::TH;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int rx = (KW - 1) / 2, ry = (kh - 1) / 2;
    const int XH = TH_ + kh - 1;
    float* gs = wsm;                                  // TH_ x kWgTileW
    float* xs = gs + kWgTileW * TH_;             // XH x XW
    const int G = (kh + JR - 1) / JR;                 // tap-row groups
    const int T = nth / G;                            // threads per group
    const int grp = tid / T, lt = tid - grp * T;
    const bool active = grp < G;
    const int j0 = grp * JR;
    float acc[JR][KW];
#pragma unroll
    for (int jr = 0; jr < JR; ++jr)
#pragma unroll
        for (int i = 0; i < KW; ++i) acc[jr][i] = 0.f;
    const int tiles_x = (W + kWgTileW - 1) / kWgTileW, tiles_y = (H + TH_ - 1) / TH_;
    for (int t = blockIdx.x; t < tiles_x * tiles_y; t += gridDim.x) {
        const int x0 = (t % tiles_x) * kWgTileW, y0 = (t / tiles_x) * TH_;
        __syncthreads();
        if (vec && x0 + kWgTileW <= W && y0 + TH_ <= H) {
            // whole g tile inside: 16-byte loads, several in flight per thread
            // all of a thread's loads first, then its stores: 4 in flight per thread
            constexpr int NC = kWgTileW / 4, NB4 = 4;
            for (int k0 = 0; k0 < NC * TH_; k0 += NB4 * nth) {
                float4 q[NB4];
#pragma unroll
                for (int u = 0; u < NB4; ++u) {
                    const int k = k0 + u * nth + tid;
                    if (k < NC * TH_) {
                        const int r = k / NC, c = (k - r * NC) * 4;
                        q[u] = __ldg(reinterpret_cast<const float4*>(g + (long long)(y0 + r) * g_pitch + x0 + c));
                    }
                }
#pragma unroll
                for (int u = 0; u < NB4; ++u) {
                    const int k = k0 + u * nth + tid;
                    if (k < NC * TH_) {
                        const int r = k / NC, c = (k - r * NC) * 4;
                        *reinterpret_cast<float4*>(gs + r * kWgTileW + c) = q[u];
                    }
                }
            }
        } else {
            for (int k = tid; k < kWgTileW * TH_; k += nth) {
                const int r = k / kWgTileW, c = k - r * kWgTileW;
                gs[k] = (x0 + c < W && y0 + r < H) ? g[(long long)(y0 + r) * g_pitch + x0 + c] : 0.f;
            }
        }
        const int sx0 = x0 - rx, sy0 = y0 - ry;
        const int epc = x_dt == IMCL_F32 ? 4 : 8;                     // elements per 16 bytes
        if (vec && sx0 >= 0 && sy0 >= 0 && round_up(sx0 + XW, epc) <= W && sy0 + XH <= H) {
            // whole x region inside, whole 16-byte chunks too: aligned loads, each element
            // to its column
            const int a0 = sx0 - sx0 % epc;
            const int nch = (sx0 + XW - a0 + epc - 1) / epc;
            const char* xb = static_cast<const char*>(x);
            const int esz = x_dt == IMCL_F32 ? 4 : 2;
            constexpr int NB16 = 4;    // 16-byte loads in flight per thread
            for (int k0 = 0; k0 < nch * XH; k0 += NB16 * nth) {
                uint4 q[NB16];
#pragma unroll
                for (int u = 0; u < NB16; ++u) {
                    const int k = k0 + u * nth + tid;
                    if (k < nch * XH) {
                        const int r = k / nch, a = a0 + (k - r * nch) * epc;
                        q[u] = __ldg(reinterpret_cast<const uint4*>(xb + ((long long)(sy0 + r) * x_pitch + a) * esz));
                    }
                }
#pragma unroll
                for (int u = 0; u < NB16; ++u) {
                    const int k = k0 + u * nth + tid;
                    if (k < nch * XH) {
                        const int r = k / nch, a = a0 + (k - r * nch) * epc;
                        float v[8];
                        if (x_dt == IMCL_F32) {
                            v[0] = __uint_as_float(q[u].x); v[1] = __uint_as_float(q[u].y);
                            v[2] = __uint_as_float(q[u].z); v[3] = __uint_as_float(q[u].w);
                            v[4] = v[5] = v[6] = v[7] = 0.f;
                        } else {
                            const uint32_t w[4] = {q[u].x, q[u].y, q[u].z, q[u].w};
                            if (x_dt == IMCL_F16) unpack_words<__half, 8>(w, v);
                            else unpack_words<__nv_bfloat16, 8>(w, v);
                        }
                        float* row = xs + r * XW;
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const int c = a + e - sx0;
                            if (e < epc && c >= 0 && c < XW) row[c] = v[e];
                        }
                    }
                }
            }
        } else {
            for (int k = tid; k < XW * XH; k += nth) {
                const int r = k / XW, c = k - r * XW;
                const int gx = sx0 + c, gy = sy0 + r;
                float v;
                if (gx >= 0 && gx < W && gy >= 0 && gy < H) v = load_px_f32(x, x_dt, (long long)gy * x_pitch + gx);
                else if (border == IMCL_BORDER_CONSTANT) v = bvf;
                else v = load_px_f32(x, x_dt, (long long)clampi(gy, 0, H - 1) * x_pitch + clampi(gx, 0, W - 1));
                xs[k] = v;
            }
        }
        __syncthreads();
        if (active) wgrad_accumulate<KW>(gs, kWgTileW, xs, XW, kWgTileW, TH_, kh, j0, lt, T, acc);
    }
    // combine the threads of each tap-row group in a fixed order (the staging area is free)
    wgrad_combine<KW>(acc, active, wsm, kh, T, partials + (long long)blockIdx.x * KW * kh, tid, nth);
}

// The same reduction with both operands staged by TMA (f32 x and g, 16-byte aligned
// rows) into a double-buffered ring: persistent CTAs prefetch their next tile while they
// reduce the current one.  The x region starts at column x0 - PADX, PADX = rx rounded up
// to 4 (TMA x coordinates must be 16-byte aligned), so reads start D = PADX - rx columns
// in.  TMA zero-fills outside the image, which is g's rule; x tiles at the image's edge
// are patched to the boundary rule in shared memory.  Waits are bounded (a timeout
// records IMCL_DEVERR_TIMEOUT and the CTA leaves).
template <int KW>
struct WgTma {
    static constexpr int TH = 32;                                          // tile rows
    static constexpr int MIN_CTAS = KW <= 5 ? 3 : 2;
    static constexpr int RX = (KW - 1) / 2;
    static constexpr int PADX = (RX + 3) / 4 * 4;
    static constexpr int D = PADX - RX;
    static constexpr int XQ = WgCfg<KW>::XQ + (D > 0 ? 1 : 0);
    static constexpr int XW = kWgTileW - kWgLx + 4 * XQ;                    // x region width (box)
};

template <int KW>
__host__ __device__ constexpr int wgrad_tma_stage_bytes(int kh) {
    return round_up(kWgTileW * WgTma<KW>::TH * 4, 128) + round_up(WgTma<KW>::XW * (WgTma<KW>::TH + kh - 1) * 4, 128);
}

template <int KW>
__global__ void __launch_bounds__(256, WgTma<KW>::MIN_CTAS)
    k_wgrad_tma(const __grid_constant__ CUtensorMap gmap, const __grid_constant__ CUtensorMap xmap, int W, int H,
                int kh, int border, float bvf, float* partials, int* status) {
    extern __shared__ __align__(128) uint8_t wsm8[];
    using TM = WgTma<KW>;
    constexpr int JR = WgCfg<KW>::JR, TH = TM::TH, TW = kWgTileW, XW = TM::XW;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int ry = (kh - 1) / 2, XH = TH + kh - 1;
    const int g_bytes = TW * TH * 4, x_bytes = XW * XH * 4;
    const int stage = wgrad_tma_stage_bytes<KW>(kh);
    uint64_t* bar = reinterpret_cast<uint64_t*>(wsm8);
    auto gbuf = [&](int s) { return reinterpret_cast<float*>(wsm8 + 128 + s * stage); };
    auto xbuf = [&](int s) { return reinterpret_cast<float*>(wsm8 + 128 + s * stage + round_up(g_bytes, 128)); };
    const int G = (kh + JR - 1) / JR, T = nth / G;
    const int grp = tid / T, lt = tid - grp * T;
    const bool active = grp < G;
    const int j0 = grp * JR;
    float acc[JR][KW];
#pragma unroll
    for (int jr = 0; jr < JR; ++jr)
#pragma unroll
        for (int i = 0; i < KW; ++i) acc[jr][i] = 0.f;
    const int tiles_x = (W + TW - 1) / TW, tiles_y = (H + TH - 1) / TH, ntiles = tiles_x * tiles_y;
    auto issue = [&](int t, int s) {
        const int x0 = (t % tiles_x) * TW, y0 = (t / tiles_x) * TH;
        mbar_arrive_expect_tx(&bar[s], (uint32_t)(g_bytes + x_bytes));
        tma_load_2d(gbuf(s), &gmap, x0, y0, &bar[s]);
        tma_load_2d(xbuf(s), &xmap, x0 - TM::PADX, y0 - ry, &bar[s]);
    };
    int t = blockIdx.x, s = 0;
    uint32_t parity = 0;
    if (tid == 0) {
        prefetch_tmap(&gmap);
        prefetch_tmap(&xmap);
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0 && t < ntiles) issue(t, 0);
    bool failed = false;
    for (; t < ntiles; t += gridDim.x) {
        const int x0 = (t % tiles_x) * TW, y0 = (t / tiles_x) * TH;
        const int tn = t + gridDim.x;
        const bool prefetch = tn < ntiles;
        if (tid == 0 && prefetch) {
            fence_proxy_async_smem();     // stage s^1 was released by the barrier ending the last tile
            issue(tn, s ^ 1);
        }
        const bool ok = mbar_wait(&bar[s], (parity >> s) & 1u, status);
        parity ^= (1u << s);
        if (__syncthreads_or(!ok)) {
            if (tid == 0 && prefetch) mbar_wait(&bar[s ^ 1], (parity >> (s ^ 1)) & 1u, nullptr);
            failed = true;
            break;
        }
        float* xs = xbuf(s);
        const int gx0 = x0 - TM::PADX, gy0 = y0 - ry;
        if (!tile_inside(gx0, gy0, XW, XH, W, H)) patch_tile<float>(xs, XW, XH, gx0, gy0, W, H, border, bvf, tid, nth);
        if (active) wgrad_accumulate<KW, TM::D>(gbuf(s), TW, xs, XW, TW, TH, kh, j0, lt, T, acc);
        __syncthreads();              // stage s may be refilled
        s ^= 1;
    }
    if (failed) return;
    // combine the threads of each tap-row group in a fixed order (the ring is idle now)
    wgrad_combine<KW>(acc, active, reinterpret_cast<float*>(wsm8 + 128), kh, T,
                      partials + (long long)blockIdx.x * KW * kh, tid, nth);
}

// out[tap] = (accumulate ? out[tap] : 0) + sum over nparts partial sums, as a fixed tree.
__global__ void __launch_bounds__(256)
    k_wgrad_finalize(const float* partials, int nparts, int ntaps, float* out, int accumulate) {
    __shared__ float sh[256];
    const int tap = blockIdx.x, tid = threadIdx.x;
    float s = 0.f;
    for (int p = tid; p < nparts; p += 256) s += partials[(long long)p * ntaps + tap];
    sh[tid] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (tid < w) sh[tid] += sh[tid + w];
        __syncthreads();
    }
    if (tid == 0) out[tap] = accumulate ? out[tap] + sh[0] : sh[0];
}

// flipped copies of device taps (and a single 1.0 tap) into dst
__global__ void k_flip_taps(const float* src, int kw, int kh, float* dst, float* one) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < kw * kh) dst[k] = src[kw * kh - 1 - k];
    if (k == 0 && one) *one = 1.f;
}

// ------------------------------------------------------------------ Harris elementwise steps
// products of the gradients: P = (Ix^2, Iy^2, Ix Iy), planes of pitch `pitch`
__global__ void k_harris_products(const float* ix, const float* iy, float* p0, float* p1, float* p2, long long pitch,
                                  int W, int H) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= W) return;
    for (int y = blockIdx.y; y < H; y += gridDim.y) {
        const long long o = (long long)y * pitch + x;
        const float a = ix[o], b = iy[o];
        p0[o] = a * a;
        p1[o] = b * b;
        p2[o] = a * b;
    }
}

// dR/dS: gSxx = gR (Syy - 2k tr), gSyy = gR (Sxx - 2k tr), gSxy = -2 gR Sxy (in place)
__global__ void k_harris_gs(const float* gR, long long gR_pitch, float* s0, float* s1, float* s2, long long pitch,
                            int W, int H, float k) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= W) return;
    for (int y = blockIdx.y; y < H; y += gridDim.y) {
        const long long o = (long long)y * pitch + x;
        const float g = gR[(long long)y * gR_pitch + x];
        const float sxx = s0[o], syy = s1[o], sxy = s2[o], tr = sxx + syy;
        s0[o] = g * (syy - 2.f * k * tr);
        s1[o] = g * (sxx - 2.f * k * tr);
        s2[o] = -2.f * g * sxy;
    }
}

// chain rule through the products: gIx = 2 Ix gPxx + Iy gPxy, gIy = 2 Iy gPyy + Ix gPxy
__global__ void k_harris_gi(const float* ix, const float* iy, const float* gp0, const float* gp1, const float* gp2,
                            float* gix, float* giy, long long pitch, int W, int H) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= W) return;
    for (int y = blockIdx.y; y < H; y += gridDim.y) {
        const long long o = (long long)y * pitch + x;
        const float a = ix[o], b = iy[o], pxx = gp0[o], pyy = gp1[o], pxy = gp2[o];
        gix[o] = __fmaf_rn(2.f * a, pxx, b * pxy);
        giy[o] = __fmaf_rn(2.f * b, pyy, a * pxy);
    }
}

// dst += src (planes)
__global__ void k_add_plane(float* dst, long long dst_pitch, const float* src, long long src_pitch, int W, int H) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= W) return;
    for (int y = blockIdx.y; y < H; y += gridDim.y) {
        dst[(long long)y * dst_pitch + x] += src[(long long)y * src_pitch + x];
    }
}

}  // namespace imcl
