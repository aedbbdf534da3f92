// harris_bwd_kernels.cuh -- the Harris adjoint as one tile kernel.
//
// Forward (clamped rule on each stage's input; o a tap offset):
//   Ix(p) = sum_o Sx[o] I(b(p+o)),  Iy likewise;  P = (Ix^2, Iy^2, Ix Iy)
//   S_c(p) = sum_o G[o] P_c(b(p+o));  R = Sxx Syy - Sxy^2 - k (Sxx + Syy)^2
// Backward for an upstream gradient gR, one stage at a time in reverse:
//   gS = (gR (Syy - 2k tr), gR (Sxx - 2k tr), -2 gR Sxy)
//   gP_c(q) = sum_{p, o: b(p+o) = q} G[o] gS_c(p);   dG[o] = sum_p sum_c gS_c(p) P_c(b(p+o))
//   gIx = 2 Ix gPxx + Iy gPxy,  gIy = 2 Iy gPyy + Ix gPxy
//   dI(q) = sum_{p, o: b(p+o) = q} Sx[o] gIx(p) + Sy[o] gIy(p)
//   dSx[o] = sum_p gIx(p) I(b(p+o)),  dSy[o] likewise
// A CTA owns a TB x TB tile of dI and recomputes what it needs on shrinking halos:
// I on halo 2 + 2RW, (Ix, Iy, P) on 1 + 2RW (taken at the clamped position outside the
// image, as the window reads them), gS on 1 + RW (zero outside), (gP, gI) on 1 (zero
// outside), dI on the tile.  Inside the image the adjoint sums are the plain
// correlations with reversed offsets (b(p+o) = q with p = q - o); on the image's first
// and last rows and columns they also collect the offsets that were clamped onto q (the
// transpose of the clamp), added by explicit loops there.  Tap gradients are per-thread
// sums over the CTA's tiles, combined in a fixed order into per-CTA partials (then
// reduced by k_wgrad_finalize): deterministic.
#pragma once

#include "tile_common.cuh"

namespace imcl {

constexpr int kHbTile = 32;                       // output tile side

// taps as kernel parameters (host taps): window, Sobel x, Sobel y
template <int WK>
struct HbTaps {
    float g[WK * WK];
    float sx[9];
    float sy[9];
};

template <int WK>
struct HbGeo {
    static constexpr int RW = (WK - 1) / 2;
    static constexpr int TB = kHbTile;
    static constexpr int HI = 2 + 2 * RW, HP = 1 + 2 * RW, HS = 1 + RW, HG = 1;
    static constexpr int WI = TB + 2 * HI;                                  // I region rows
    static constexpr int XI = HI;                                           // I region's left halo
    static constexpr int WIX = TB + 2 * XI;                                 // I region columns
    static constexpr int WP = TB + 2 * HP;                                  // P region side
    static constexpr int WS = TB + 2 * HS;                                  // gS region side
    static constexpr int WG = TB + 2 * HG;                                  // gI region side
    static constexpr int NSI = (WS + 3) / 4;                                // 4-wide items per gS row
    static constexpr int NGI = (WG + 3) / 4;                                // 4-wide items per gI row
    // row pitches (floats): odd, so that threads walking down a column of items (the
    // mapping of steps 3 to 5) touch distinct banks
    static constexpr int PPI = WIX;
    static constexpr int PPP = (4 * NSI + 2 * RW) | 1;
    static constexpr int PPS = ((4 * NGI + 2 * RW) > 4 * NSI ? (4 * NGI + 2 * RW) : 4 * NSI) | 1;
    static constexpr int PPG = (4 * NGI) | 1;
    static constexpr int NTAP = WK * WK + 18;                               // window, Sobel x, Sobel y
    // shared memory (floats): taps, I, Ix Iy Pxx Pyy Pxy, gSxx gSyy gSxy, gIx gIy
    static constexpr int O_TAP = 0;
    static constexpr int O_I = round_up(NTAP, 4);
    static constexpr int O_X = O_I + PPI * WI;                              // after the I rows
    static constexpr int PLANE_P = PPP * WP;
    static constexpr int O_S = O_X + 5 * PLANE_P;
    static constexpr int PLANE_S = PPS * WS;
    static constexpr int O_G = O_S + 3 * PLANE_S;
    static constexpr int PLANE_G = PPG * WG;
    static constexpr int TOTAL = O_G + 2 * PLANE_G;
};

template <int WK>
__global__ void __launch_bounds__(256, 2)
    k_harris_bwd_fused(const float* __restrict__ I, long long i_pitch, const float* __restrict__ gR, long long g_pitch,
                       float* dI, long long d_pitch, int W, int H, float k, const float* sx_dev, const float* sy_dev,
                       const float* gw_dev, const __grid_constant__ HbTaps<WK> tp, float* part_w, float* part_sx,
                       float* part_sy) {
    using G = HbGeo<WK>;
    constexpr int RW = G::RW, TB = G::TB, HI = G::HI, HP = G::HP, HS = G::HS, XI = G::XI;
    extern __shared__ __align__(16) float hsm[];
    float* taps = hsm + G::O_TAP;                 // window (WK*WK), Sobel x (9), Sobel y (9)
    float* Is = hsm + G::O_I;
    float* Ixs = hsm + G::O_X;
    float* Iys = Ixs + G::PLANE_P;
    float* Ps = Iys + G::PLANE_P;                 // Pxx, Pyy, Pxy planes
    float* gSs = hsm + G::O_S;                    // gSxx, gSyy, gSxy planes
    float* gIs = hsm + G::O_G;                    // gIx, gIy planes
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int q = tid; q < G::NTAP; q += nth) {
        float v;
        if (q < WK * WK) v = gw_dev ? gw_dev[q] : tp.g[q];
        else if (q < WK * WK + 9) v = sx_dev ? sx_dev[q - WK * WK] : tp.sx[q - WK * WK];
        else v = sy_dev ? sy_dev[q - WK * WK - 9] : tp.sy[q - WK * WK - 9];
        taps[q] = v;
    }
    const float* gw = taps;
    const float* sxw = taps + WK * WK;
    const float* syw = taps + WK * WK + 9;

    float aw[WK * WK], asx[9], asy[9];            // this thread's tap-gradient sums
#pragma unroll
    for (int q = 0; q < WK * WK; ++q) aw[q] = 0.f;
#pragma unroll
    for (int q = 0; q < 9; ++q) { asx[q] = 0.f; asy[q] = 0.f; }

    const int tiles_x = (W + TB - 1) / TB, tiles_y = (H + TB - 1) / TB;
    for (int t = blockIdx.x; t < tiles_x * tiles_y; t += gridDim.x) {
        const int x0 = (t % tiles_x) * TB, y0 = (t / tiles_x) * TB;
        const bool border_tile = x0 - HI < 0 || y0 - HI < 0 || x0 + TB + HI > W || y0 + TB + HI > H;
        __syncthreads();   // taps staged / the previous tile's planes are no longer read
        // (1) I on the I region (rows from y0 - HI, columns from x0 - XI), at clamped positions
        for (int q = tid; q < G::WI * G::WIX; q += nth) {
            const int r = q / G::WIX, c = q - r * G::WIX;
            const int gy = clampi(y0 - HI + r, 0, H - 1), gx = clampi(x0 - XI + c, 0, W - 1);
            Is[r * G::PPI + c] = I[(long long)gy * i_pitch + gx];
        }
        __syncthreads();
        // (2) Ix, Iy and the products on the P region, each at its clamped pixel
        for (int q = tid; q < G::WP * G::WP; q += nth) {
            const int r = q / G::WP, c = q - r * G::WP;
            int ir = r + (HI - HP), ic = c + (XI - HP);       // I-region coordinates of the pixel
            if (border_tile) {
                ir = clampi(y0 - HP + r, 0, H - 1) - (y0 - HI);
                ic = clampi(x0 - HP + c, 0, W - 1) - (x0 - XI);
            }
            float ix = 0.f, iy = 0.f;
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const float u = Is[(ir - 1 + j) * G::PPI + ic - 1 + i];
                    ix = __fmaf_rn(sxw[j * 3 + i], u, ix);
                    iy = __fmaf_rn(syw[j * 3 + i], u, iy);
                }
            const int o = r * G::PPP + c;
            Ixs[o] = ix;
            Iys[o] = iy;
            Ps[o] = ix * ix;
            Ps[G::PLANE_P + o] = iy * iy;
            Ps[2 * G::PLANE_P + o] = ix * iy;
        }
        __syncthreads();
        // (3) window sums and gS on the gS region, 4 columns per item (zero outside)
        for (int it = tid; it < G::WS * G::NSI; it += nth) {
            const int c0 = (it / G::WS) * 4, r = it - (c0 / 4) * G::WS;   // rows fastest
            float s[3][4];
#pragma unroll
            for (int ch = 0; ch < 3; ++ch)
#pragma unroll
                for (int e = 0; e < 4; ++e) s[ch][e] = 0.f;
#pragma unroll
            for (int j = 0; j < WK; ++j) {
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    // P-region row r + j, columns c0 .. c0 + 3 + 2RW (offset (i - RW, j - RW))
                    const float* pr = Ps + ch * G::PLANE_P + (r + j) * G::PPP + c0;
                    float v[4 + 2 * RW];
#pragma unroll
                    for (int q = 0; q < 4 + 2 * RW; ++q) v[q] = pr[q];
#pragma unroll
                    for (int i = 0; i < WK; ++i) {
                        const float w = gw[j * WK + i];
#pragma unroll
                        for (int e = 0; e < 4; ++e) s[ch][e] = __fmaf_rn(w, v[e + i], s[ch][e]);
                    }
                }
            }
            const int gy = y0 - HS + r;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int gx = x0 - HS + c0 + e;
                float gxx = 0.f, gyy = 0.f, gxy = 0.f;
                if (c0 + e < G::WS && gx >= 0 && gx < W && gy >= 0 && gy < H) {
                    const float g = gR[(long long)gy * g_pitch + gx];
                    const float tr = s[0][e] + s[1][e];
                    gxx = g * (s[1][e] - 2.f * k * tr);
                    gyy = g * (s[0][e] - 2.f * k * tr);
                    gxy = -2.f * g * s[2][e];
                }
                const int o = r * G::PPS + c0 + e;
                gSs[o] = gxx;
                gSs[G::PLANE_S + o] = gyy;
                gSs[2 * G::PLANE_S + o] = gxy;
            }
        }
        __syncthreads();
        // (4) window-tap gradient: dG[o] += sum_c gS_c(p) P_c(b(p + o)) over the tile's pixels
        for (int it = tid; it < TB * (TB / 4); it += nth) {
            const int tx0 = (it / TB) * 4, ty = it - (tx0 / 4) * TB;     // rows fastest
            if (y0 + ty >= H) continue;
            float g[3][4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const bool in = x0 + tx0 + e < W;
                const int o = (ty + HS) * G::PPS + tx0 + e + HS;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) g[ch][e] = in ? gSs[ch * G::PLANE_S + o] : 0.f;
            }
#pragma unroll
            for (int j = 0; j < WK; ++j) {
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    const float* pr = Ps + ch * G::PLANE_P + (ty + HP + j - RW) * G::PPP + tx0 + HP - RW;
                    float v[4 + 2 * RW];
#pragma unroll
                    for (int q = 0; q < 4 + 2 * RW; ++q) v[q] = pr[q];
#pragma unroll
                    for (int i = 0; i < WK; ++i)
#pragma unroll
                        for (int e = 0; e < 4; ++e) aw[j * WK + i] = __fmaf_rn(g[ch][e], v[e + i], aw[j * WK + i]);
                }
            }
        }
        // (5) gP (window adjoint, with the clamp folds on the image's edges) and gI on the
        //     gI region, 4 columns per item (zero outside)
        for (int it = tid; it < G::WG * G::NGI; it += nth) {
            const int c0 = (it / G::WG) * 4, r = it - (c0 / 4) * G::WG;   // rows fastest
            float gp[3][4];
#pragma unroll
            for (int ch = 0; ch < 3; ++ch)
#pragma unroll
                for (int e = 0; e < 4; ++e) gp[ch][e] = 0.f;
#pragma unroll
            for (int j = 0; j < WK; ++j) {
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    // gS at q - o: gS-region row r + 2RW - j, columns c0 + e + 2RW - i
                    const float* sr = gSs + ch * G::PLANE_S + (r + 2 * RW - j) * G::PPS + c0;
                    float v[4 + 2 * RW];
#pragma unroll
                    for (int q = 0; q < 4 + 2 * RW; ++q) v[q] = sr[q];
#pragma unroll
                    for (int i = 0; i < WK; ++i) {
                        const float w = gw[j * WK + i];
#pragma unroll
                        for (int e = 0; e < 4; ++e) gp[ch][e] = __fmaf_rn(w, v[e + 2 * RW - i], gp[ch][e]);
                    }
                }
            }
            const int gy = y0 - 1 + r;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int gx = x0 - 1 + c0 + e;
                float gix = 0.f, giy = 0.f;
                if (c0 + e < G::WG && gx >= 0 && gx < W && gy >= 0 && gy < H) {
                    if (gx == 0 || gy == 0 || gx == W - 1 || gy == H - 1) {
                        // offsets clamped onto this edge pixel: p + o outside, b(p + o) = q
                        for (int py = max(gy - RW, 0); py <= min(gy + RW, H - 1); ++py)
                            for (int px = max(gx - RW, 0); px <= min(gx + RW, W - 1); ++px)
                                for (int j = 0; j < WK; ++j)
                                    for (int i = 0; i < WK; ++i) {
                                        const int qy = py + j - RW, qx = px + i - RW;
                                        if (qx >= 0 && qx < W && qy >= 0 && qy < H) continue;
                                        if (clampi(qx, 0, W - 1) != gx || clampi(qy, 0, H - 1) != gy) continue;
                                        const int o = (py - (y0 - HS)) * G::PPS + px - (x0 - HS);
                                        const float w = gw[j * WK + i];
#pragma unroll
                                        for (int ch = 0; ch < 3; ++ch)
                                            gp[ch][e] = __fmaf_rn(w, gSs[ch * G::PLANE_S + o], gp[ch][e]);
                                    }
                    }
                    const int op = (r + HP - 1) * G::PPP + c0 + e + HP - 1;
                    const float ix = Ixs[op], iy = Iys[op];
                    gix = 2.f * ix * gp[0][e] + iy * gp[2][e];
                    giy = 2.f * iy * gp[1][e] + ix * gp[2][e];
                }
                const int o = r * G::PPG + c0 + e;
                gIs[o] = gix;
                gIs[G::PLANE_G + o] = giy;
            }
        }
        __syncthreads();
        // (6) dI on the tile (Sobel adjoint with the clamp folds) and the Sobel tap gradients
        for (int q = tid; q < TB * TB; q += nth) {
            const int ty = q / TB, tx = q - ty * TB;
            const int gy = y0 + ty, gx = x0 + tx;
            if (gy >= H || gx >= W) continue;
            float acc = 0.f;
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    // gI at q - o: gI-region (ty + 1 - (j - 1), tx + 1 - (i - 1))
                    const int o = (ty + 2 - j) * G::PPG + tx + 2 - i;
                    acc = __fmaf_rn(sxw[j * 3 + i], gIs[o], acc);
                    acc = __fmaf_rn(syw[j * 3 + i], gIs[G::PLANE_G + o], acc);
                }
            if (gx == 0 || gy == 0 || gx == W - 1 || gy == H - 1) {
                for (int py = max(gy - 1, 0); py <= min(gy + 1, H - 1); ++py)
                    for (int px = max(gx - 1, 0); px <= min(gx + 1, W - 1); ++px)
                        for (int j = 0; j < 3; ++j)
                            for (int i = 0; i < 3; ++i) {
                                const int qy = py + j - 1, qx = px + i - 1;
                                if (qx >= 0 && qx < W && qy >= 0 && qy < H) continue;
                                if (clampi(qx, 0, W - 1) != gx || clampi(qy, 0, H - 1) != gy) continue;
                                const int o = (py - (y0 - 1)) * G::PPG + px - (x0 - 1);
                                acc = __fmaf_rn(sxw[j * 3 + i], gIs[o], acc);
                                acc = __fmaf_rn(syw[j * 3 + i], gIs[G::PLANE_G + o], acc);
                            }
            }
            if (dI) dI[(long long)gy * d_pitch + gx] = acc;
            const int og = (ty + 1) * G::PPG + tx + 1;
            const float gix = gIs[og], giy = gIs[G::PLANE_G + og];
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const float u = Is[(ty + HI + j - 1) * G::PPI + tx + XI + i - 1];   // I(b(p + o))
                    asx[j * 3 + i] = __fmaf_rn(gix, u, asx[j * 3 + i]);
                    asy[j * 3 + i] = __fmaf_rn(giy, u, asy[j * 3 + i]);
                }
        }
    }
    // combine the threads' tap sums in a fixed order into this CTA's partials
    __syncthreads();
    float* red = hsm;                             // nth x NTAP
#pragma unroll
    for (int q = 0; q < WK * WK; ++q) red[tid * G::NTAP + q] = aw[q];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        red[tid * G::NTAP + WK * WK + q] = asx[q];
        red[tid * G::NTAP + WK * WK + 9 + q] = asy[q];
    }
    __syncthreads();
    for (int q = tid; q < G::NTAP; q += nth) {
        float sum = 0.f;
        for (int r = 0; r < nth; ++r) sum += red[r * G::NTAP + q];
        if (q < WK * WK) part_w[(long long)blockIdx.x * WK * WK + q] = sum;
        else if (q < WK * WK + 9) part_sx[(long long)blockIdx.x * 9 + q - WK * WK] = sum;
        else part_sy[(long long)blockIdx.x * 9 + q - WK * WK - 9] = sum;
    }
}

}  // namespace imcl
