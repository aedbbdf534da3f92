// sepbwd_kernels.cuh -- the separable adjoint (§6 separable benchmark, backward) in one
// persistent tile kernel, for equal row and column radii R.
//
// Forward (per stage, the border rule on the stage's input):
//   t(q) = sum_i r_i x_b(qx + i - R, qy),   y(p) = sum_j c_j t_b(px, py + j - R).
// Given g = dL/dy, one tile of TW x TH outputs stages g (zero outside the image) and x
// (under the forward's rule) over the tile plus R rows and P >= R columns on each side
// (P a multiple of 4, so that rows of the staged region start on 16-byte boundaries),
// then forms in shared memory
//   dt on the tile rows and halo columns: the zero-border correlation of g with the
//      flipped column taps, plus (clamp rule) the folds of clamped rows into rows 0, H-1;
//   t  on the tile columns and R halo rows (constant rule: the constant on rows outside);
// and for each group of 4 pixels of the tile
//   dx   = the zero-border correlation of dt with the flipped row taps, plus the folds of
//          clamped columns into columns 0 and W-1 (clamp rule);
//   drow[i] += dt(s) x_b(sx + i - R, sy);   dcol[j] += g(p) t_b(px, py + j - R).
// Every pass works on groups of 4 columns with 16-byte shared-memory loads.  With f32
// operands on 16-byte aligned rows (TMA = true) the staged regions arrive by 2D TMA into
// a two-stage mbarrier ring, the next tile's while the current one computes; the
// zero fill outside the image is g's border, and x's rule is patched in shared memory.
// The tap sums stay in registers across a CTA's tiles and are reduced per CTA into
// partial sums, which a second launch adds up in a fixed order.  g and x are read once (plus halos) and dx
// written once: 12 bytes per pixel for f32 images.
#pragma once

#include "backward_kernels.cuh"   // load_px_f32

namespace imcl {

constexpr int kSbTileW = 64, kSbTileH = 32, kSbMaxR = 8;

template <int R>
struct SbTaps {
    float r[2 * R + 1];
    float c[2 * R + 1];
};

struct SbArgs {
    const float* g;          // upstream gradient (f32), pitch in floats
    long long gp;
    const void* x;           // forward input, pitch in elements
    long long xp;
    int x_dt;
    float* dx;               // input gradient (f32) or nullptr
    long long dxp;
    const float* rdev;       // device taps, or nullptr for the launch parameters
    const float* cdev;
    float* prow;             // per-CTA partial sums [gridDim.x][2R+1]
    float* pcol;
    int W, H, border;
    float bvx;               // the constant as a pixel of x's type (x outside the image)
    float bvt;               // the constant as f32 (t on rows outside the image)
    int tiles_x, ntiles;
    int vec;                 // g and x are f32 with 16-byte aligned rows
};

template <int R>
struct SbGeo {
    static constexpr int NT = 2 * R + 1, TW = kSbTileW, TH = kSbTileH;
    static constexpr int P = (R + 3) / 4 * 4;           // staged halo columns per side
    static constexpr int RW = TW + 2 * P, RH = TH + 2 * R;
    static constexpr int NV = (2 * P + 4) / 4;          // float4s covering [c, c + 2P + 4)
    static constexpr int PLANE_B = (RH * RW * 4 + 127) / 128 * 128;        // a staged plane, bytes
    static constexpr int REST = TH * RW + RH * TW + 2 * NT;                 // dt, t, taps (floats)
};

// Dynamic shared memory of the kernel: barriers (128 bytes), then (TMA: two) stages of
// g and x (each plane 128-byte aligned), then dt, t and the taps.
template <int R, bool TMA>
__host__ __device__ constexpr int sb_smem_bytes() {
    return 128 + (TMA ? 2 : 1) * 2 * SbGeo<R>::PLANE_B + SbGeo<R>::REST * 4;
}

__device__ __forceinline__ void ld4(const float* p, float* v) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}

template <int R, bool TMA>
__global__ void __launch_bounds__(256, 3)
    k_sep_bwd_fused(const SbArgs a, const __grid_constant__ SbTaps<R> tp, const __grid_constant__ CUtensorMap gmap,
                    const __grid_constant__ CUtensorMap xmap, int* status) {
    using G = SbGeo<R>;
    constexpr int NT = G::NT, TW = G::TW, TH = G::TH, P = G::P, RW = G::RW, RH = G::RH, NV = G::NV;
    constexpr int NSTAGE = TMA ? 2 : 1;
    constexpr int PB = G::PLANE_B;
    extern __shared__ __align__(128) uint8_t sbraw[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(sbraw);
    uint8_t* stages = sbraw + 128;
    // stage k: g at stages + 2 k PB (RH x RW, zero outside; column c is x0 - P + c), x at + PB
    float* dts = reinterpret_cast<float*>(stages + NSTAGE * 2 * PB);   // TH x RW: dt, same columns
    float* ts = dts + TH * RW;          // RH x TW: t, tile columns, rows y0 - R ..
    float* wr = ts + RH * TW;
    float* wc = wr + NT;
    const int tid = threadIdx.x;
    if (tid < NT) {
        wr[tid] = a.rdev ? a.rdev[tid] : tp.r[tid];
        wc[tid] = a.cdev ? a.cdev[tid] : tp.c[tid];
    }
    const int W = a.W, H = a.H;
    const bool clamp = a.border == IMCL_BORDER_CLAMP;
    float accr[NT], accc[NT];
#pragma unroll
    for (int k = 0; k < NT; ++k) { accr[k] = 0.f; accc[k] = 0.f; }

    int s = 0;
    uint32_t parity = 0;
    if constexpr (TMA) {
        if (tid == 0) {
            prefetch_tmap(&gmap);
            prefetch_tmap(&xmap);
            mbar_init(&bar[0], 1);
            mbar_init(&bar[1], 1);
            fence_mbar_init();
        }
        __syncthreads();
        const int t0 = blockIdx.x;
        if (tid == 0 && t0 < a.ntiles) {
            const int x0 = (t0 % a.tiles_x) * TW, y0 = (t0 / a.tiles_x) * TH;
            mbar_arrive_expect_tx(&bar[0], (uint32_t)(2 * RH * RW * 4));
            tma_load_2d(stages, &gmap, x0 - P, y0 - R, &bar[0]);
            tma_load_2d(stages + PB, &xmap, x0 - P, y0 - R, &bar[0]);
        }
    }

    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const int x0 = (t % a.tiles_x) * TW, y0 = (t / a.tiles_x) * TH;
        const int gx0 = x0 - P, gy0 = y0 - R;
        float* gs = reinterpret_cast<float*>(stages + s * 2 * PB);
        float* xs = reinterpret_cast<float*>(stages + s * 2 * PB + PB);
        __syncthreads();   // the previous tile's reads (and the taps) are done
        // ---- stage g and x over [gx0, gx0 + RW) x [gy0, gy0 + RH)
        if constexpr (TMA) {
            const int tn = t + gridDim.x;
            const bool prefetch = tn < a.ntiles;
            if (tid == 0 && prefetch) {
                const int nx0 = (tn % a.tiles_x) * TW, ny0 = (tn / a.tiles_x) * TH;
                uint8_t* ng = stages + (s ^ 1) * 2 * PB;
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&bar[s ^ 1], (uint32_t)(2 * RH * RW * 4));
                tma_load_2d(ng, &gmap, nx0 - P, ny0 - R, &bar[s ^ 1]);
                tma_load_2d(ng + PB, &xmap, nx0 - P, ny0 - R, &bar[s ^ 1]);
            }
            const bool ok = mbar_wait(&bar[s], (parity >> s) & 1u, status);
            parity ^= (1u << s);
            if (__syncthreads_or(!ok)) {
                if (tid == 0 && prefetch) mbar_wait(&bar[s ^ 1], (parity >> (s ^ 1)) & 1u, nullptr);
                return;
            }
            // g: the TMA zero fill is its border; x: the forward's rule
            if (!tile_inside(gx0, gy0, RW, RH, W, H))
                patch_tile<float>(xs, RW, RH, gx0, gy0, W, H, a.border, a.bvx, tid, 256);
        } else if (a.vec && gx0 >= 0 && gy0 >= 0 && gx0 + RW <= W && gy0 + RH <= H) {
            const float* xf = static_cast<const float*>(a.x);
            for (int i = tid; i < RH * (RW / 4); i += 256) {
                const int r = i / (RW / 4), c = (i - r * (RW / 4)) * 4;
                const long long gy = gy0 + r;
                *reinterpret_cast<float4*>(gs + r * RW + c) =
                    __ldg(reinterpret_cast<const float4*>(a.g + gy * a.gp + gx0 + c));
                *reinterpret_cast<float4*>(xs + r * RW + c) =
                    __ldg(reinterpret_cast<const float4*>(xf + gy * a.xp + gx0 + c));
            }
        } else {
            for (int i = tid; i < RH * RW; i += 256) {
                const int r = i / RW, c = i - r * RW;
                const int gy = gy0 + r, gx = gx0 + c;
                const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
                gs[i] = in ? __ldg(a.g + (long long)gy * a.gp + gx) : 0.f;
                float xv;
                if (in) xv = load_px_f32(a.x, a.x_dt, (long long)gy * a.xp + gx);
                else if (!clamp) xv = a.bvx;
                else xv = load_px_f32(a.x, a.x_dt, (long long)clampi(gy, 0, H - 1) * a.xp + clampi(gx, 0, W - 1));
                xs[i] = xv;
            }
        }
        if constexpr (!TMA) __syncthreads();
        // ---- dt on the tile rows, all staged columns, 4 at a time
        for (int i = tid; i < TH * (RW / 4); i += 256) {
            const int r = i / (RW / 4), c = (i - r * (RW / 4)) * 4;
            const int qy = y0 + r;
            float v[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                float s[4];
                ld4(gs + (r + 2 * R - j) * RW + c, s);
#pragma unroll
                for (int e = 0; e < 4; ++e) v[e] = __fmaf_rn(wc[j], s[e], v[e]);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int qx = gx0 + c + e;
                if (qx < 0 || qx >= W || qy >= H) {
                    v[e] = 0.f;
                } else if (clamp && (qy == 0 || qy == H - 1)) {
                    // rows py whose tap j was clamped onto row 0 (py + j - R < 0) or row H-1
                    if (qy == 0)
                        for (int j = 0; j < NT; ++j)
                            for (int py = 0; py < R - j && py < H; ++py) v[e] += wc[j] * gs[(py - gy0) * RW + c + e];
                    if (qy == H - 1)
                        for (int j = 0; j < NT; ++j)
                            for (int py = max(H + R - j, 0); py < H; ++py) v[e] += wc[j] * gs[(py - gy0) * RW + c + e];
                }
            }
            *reinterpret_cast<float4*>(dts + r * RW + c) = make_float4(v[0], v[1], v[2], v[3]);
        }
        // ---- t on rows y0 - R .. (RH) x the tile's columns (the forward's row pass)
        for (int i = tid; i < RH * (TW / 4); i += 256) {
            const int r = i / (TW / 4), c = (i - r * (TW / 4)) * 4;
            const int gy = gy0 + r;
            float v[4];
            if (!clamp && (gy < 0 || gy >= H)) {
#pragma unroll
                for (int e = 0; e < 4; ++e) v[e] = a.bvt;
            } else {
                float s[4 * NV];
#pragma unroll
                for (int q = 0; q < NV; ++q) ld4(xs + r * RW + c + 4 * q, s + 4 * q);
#pragma unroll
                for (int e = 0; e < 4; ++e) v[e] = 0.f;
                // x(x0 + c + e + k - R) is staged column c + e + k + P - R
#pragma unroll
                for (int k = 0; k < NT; ++k)
#pragma unroll
                    for (int e = 0; e < 4; ++e) v[e] = __fmaf_rn(wr[k], s[e + k + P - R], v[e]);
            }
            *reinterpret_cast<float4*>(ts + r * TW + c) = make_float4(v[0], v[1], v[2], v[3]);
        }
        __syncthreads();
        // ---- per group of 4 pixels of the tile: dx, and the tap sums
        for (int i = tid; i < TH * (TW / 4); i += 256) {
            const int r = i / (TW / 4), c = (i - r * (TW / 4)) * 4;
            const int sy = y0 + r, sx = x0 + c;
            if (sy >= H || sx >= W) continue;
            const int nv = min(4, W - sx);        // pixels of the group inside the image
            float d[4 * NV], xv[4 * NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                ld4(dts + r * RW + c + 4 * q, d + 4 * q);
                ld4(xs + (r + R) * RW + c + 4 * q, xv + 4 * q);
            }
            if (a.dx) {
                float v[4] = {0.f, 0.f, 0.f, 0.f};
                // dt(sx + e + R - k) is at column c + e + 2R - k + P - R
#pragma unroll
                for (int k = 0; k < NT; ++k)
#pragma unroll
                    for (int e = 0; e < 4; ++e) v[e] = __fmaf_rn(wr[k], d[e + 2 * R - k + P - R], v[e]);
                if (clamp && (sx == 0 || sx + 3 >= W - 1)) {
                    const float* drw = dts + r * RW;
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int px = sx + e;
                        // columns qx whose tap k was clamped onto column 0 (qx + k - R < 0) or W-1
                        if (px == 0)
                            for (int k = 0; k < NT; ++k)
                                for (int qx = 0; qx < R - k && qx < W; ++qx) v[e] += wr[k] * drw[qx - gx0];
                        if (px == W - 1)
                            for (int k = 0; k < NT; ++k)
                                for (int qx = max(W + R - k, 0); qx < W; ++qx) v[e] += wr[k] * drw[qx - gx0];
                    }
                }
                float* o = a.dx + (long long)sy * a.dxp + sx;
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (e < nv) o[e] = v[e];
            }
            float gv[4];
            ld4(gs + (r + R) * RW + c + P, gv);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (e >= nv) { gv[e] = 0.f; d[e + P] = 0.f; }
            }
#pragma unroll
            for (int k = 0; k < NT; ++k) {
                float tv[4];
                ld4(ts + (r + k) * TW + c, tv);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    accr[k] = __fmaf_rn(d[e + P], xv[e + k + P - R], accr[k]);
                    accc[k] = __fmaf_rn(gv[e], tv[e], accc[k]);
                }
            }
        }
        if constexpr (TMA) s ^= 1;
    }

    // CTA sums of the tap gradients: warps, then the 8 warp sums in a fixed order
    __syncthreads();
    float* red = reinterpret_cast<float*>(stages);   // 8 warps x 2 NT (the staging buffers are free now)
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int k = 0; k < NT; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            accr[k] += __shfl_xor_sync(0xffffffffu, accr[k], o);
            accc[k] += __shfl_xor_sync(0xffffffffu, accc[k], o);
        }
        if (lane == 0) {
            red[warp * 2 * NT + k] = accr[k];
            red[warp * 2 * NT + NT + k] = accc[k];
        }
    }
    __syncthreads();
    if (tid < 2 * NT) {
        float s = 0.f;
        for (int w = 0; w < 8; ++w) s += red[w * 2 * NT + tid];
        if (tid < NT) a.prow[(long long)blockIdx.x * NT + tid] = s;
        else a.pcol[(long long)blockIdx.x * NT + tid - NT] = s;
    }
}

}  // namespace imcl
