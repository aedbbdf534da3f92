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
// A CTA owns a TW x TH tile of dI and recomputes what it needs on shrinking halos:
// I on halo 2 + 2RW, (Ix, Iy, P) on 1 + 2RW (taken at the clamped position outside the
// image, as the window reads them), gS on 1 + RW (zero outside), (gP, gI) on 1 (zero
// outside), dI on the tile.  Inside the image the adjoint sums are the plain
// correlations with reversed offsets (b(p+o) = q with p = q - o); on the image's first
// and last rows and columns they also collect the offsets that were clamped onto q (the
// transpose of the clamp), added by explicit loops there.
//
// The two window passes and the window-gradient pass work on items of one channel x
// 4 rows x 4 columns: each row of the input plane read (16-byte loads, quad-aligned
// columns) feeds up to four output rows from registers.  Items run columns fastest and
// the quad pitches of those planes are odd, so the eight lanes of a quarter warp read
// distinct bank quads.  The channel-mixing steps (gS from the window sums, gI from gP)
// are separate element-wise passes.  Tap gradients are per-thread sums over the CTA's
// tiles, combined in a fixed order into per-CTA partials (then reduced by
// k_wgrad_finalize): deterministic.
#pragma once

#include "tile_common.cuh"

namespace imcl {

constexpr int kHbTileW = 64, kHbTileH = 32;       // output tile (columns, rows)

// taps as kernel parameters (host taps): window, Sobel x, Sobel y
template <int WK>
struct HbTaps {
    float g[WK * WK];
    float sx[9];
    float sy[9];
};

__host__ __device__ constexpr int hb_max(int a, int b) { return a > b ? a : b; }
// a quad pitch (multiple of 4 floats) with an odd number of quads
__host__ __device__ constexpr int hb_odd_quads(int v) { return (round_up(v, 4) / 4) % 2 ? round_up(v, 4) : round_up(v, 4) + 4; }

template <int WK>
struct HbGeo {
    static constexpr int RW = (WK - 1) / 2;
    static constexpr int TW = kHbTileW, TH = kHbTileH;
    static constexpr int HI = 2 + 2 * RW, HP = 1 + 2 * RW, HS = 1 + RW;
    // regions (rows x columns): I, P (and Ix, Iy), gS, gI; each starts at its halo
    static constexpr int RI = TH + 2 * HI, CI = TW + 2 * HI;
    static constexpr int RP = TH + 2 * HP, CP = TW + 2 * HP;
    static constexpr int RS = TH + 2 * HS, CS = TW + 2 * HS;
    static constexpr int RG = TH + 2, CG = TW + 2;
    // item grids (rows x 4 columns) of the window pass (gS region, PYS rows), its adjoint
    // (gI region, 4 rows), the window-gradient pass (tile, PYT rows), and the 4-row column
    // items of the Sobel passes; item heights chosen so the item counts of the long passes
    // fill the CTA's threads in whole rounds (702 of 768, 459 of 512, 768 of 768 slots)
    static constexpr int PYS = 3, PYT = 2;
    static constexpr int NRS = (RS + PYS - 1) / PYS, NCS = (CS + 3) / 4;
    static constexpr int NRG = (RG + 3) / 4, NCG = (CG + 3) / 4;
    static constexpr int NRT = TH / PYT, NCT = TW / 4;
    static constexpr int NRP = (RP + 3) / 4;
    // float4 loads per item row: window passes (4 + 2RW columns from the item's quad),
    // window gradient (4 + 2RW columns from HP - RW past it)
    static constexpr int NV = (4 + 2 * RW + 3) / 4;
    static constexpr int OFF4 = HP - RW;
    static constexpr int NV4 = (OFF4 + 4 + 2 * RW + 3) / 4;
    // stored rows and pitches (floats), each covering every index its passes touch
    static constexpr int SRI = hb_max(RI, 4 * NRP + 2);
    static constexpr int PPI = CI;
    static constexpr int SRP = hb_max(hb_max(RP, 4 * NRP), hb_max(PYS * NRS + 2 * RW, 4 * NRG));
    static constexpr int PPP = hb_odd_quads(hb_max(hb_max(CP, 4 * NCG), hb_max(4 * (NCS - 1) + 4 * NV, 4 * (NCT - 1) + 4 * NV4)));
    static constexpr int SRS = hb_max(PYS * NRS, 4 * NRG + 2 * RW);
    static constexpr int PPS = hb_odd_quads(hb_max(4 * NCS, 4 * (NCG - 1) + 4 * NV));
    static constexpr int PPG = round_up(CG, 4);                          // quads, for (5b)
    static constexpr int NTAP = WK * WK + 18;                               // window, Sobel x, Sobel y
    // shared memory (floats): taps, I, Pxx Pyy Pxy (later gPxx gPyy gPxy),
    // gSxx gSyy gSxy (first the window sums), Ix Iy (later gIx gIy)
    static constexpr int O_TAP = 0;
    static constexpr int O_I = round_up(NTAP, 4);
    static constexpr int PLANE_P = PPP * SRP;
    static constexpr int O_P = round_up(O_I + PPI * SRI, 4);
    static constexpr int PLANE_S = PPS * SRS;
    static constexpr int O_S = O_P + 3 * PLANE_P;
    static constexpr int PLANE_G = PPG * RG;
    static constexpr int O_G = O_S + 3 * PLANE_S;
    static constexpr int TOTAL = O_G + 2 * PLANE_G;
    static_assert(PLANE_P % 4 == 0 && PLANE_S % 4 == 0 && PLANE_G % 4 == 0, "quad-aligned planes");
};

constexpr int kHbThreads = 256;                   // threads per CTA (the launch uses exactly this)

// The transpose of the clamp at an image-edge pixel q = (gx, gy) for a correlation of
// radius R: every source u outside the image that the clamp maps onto q, and each offset
// o = (i - R, j - R) whose output p = u - o lies inside the image; f(j, i, py, px) gets
// the tap and p.  (Along x, b(u) = gx exactly for u = gx, and for u < 0 when gx = 0 and
// u > W - 1 when gx = W - 1; likewise along y.)
template <int R, typename F>
__device__ __forceinline__ void hb_clamp_fold(int gx, int gy, int W, int H, F&& f) {
    const int ux0 = gx == 0 ? -R : gx, ux1 = gx == W - 1 ? W - 1 + R : gx;
    const int uy0 = gy == 0 ? -R : gy, uy1 = gy == H - 1 ? H - 1 + R : gy;
    for (int uy = uy0; uy <= uy1; ++uy)
        for (int ux = ux0; ux <= ux1; ++ux) {
            if (ux >= 0 && ux < W && uy >= 0 && uy < H) continue;
            for (int j = 0; j < 2 * R + 1; ++j) {
                const int py = uy - (j - R);
                if (py < 0 || py >= H) continue;
                for (int i = 0; i < 2 * R + 1; ++i) {
                    const int px = ux - (i - R);
                    if (px >= 0 && px < W) f(j, i, py, px);
                }
            }
        }
}

// Store the products at P-region pixel (r, c), and Ix, Iy where the gI region covers it
template <int WK>
__device__ __forceinline__ void hb_store_p(float* Ps, float* gIs, int r, int c, float ix, float iy) {
    using G = HbGeo<WK>;
    const int o = r * G::PPP + c;
    Ps[o] = ix * ix;
    Ps[G::PLANE_P + o] = iy * iy;
    Ps[2 * G::PLANE_P + o] = ix * iy;
    const int gr = r - (G::HP - 1), gc = c - (G::HP - 1);          // gI-region coordinates
    if (gr >= 0 && gr < G::RG && gc >= 0 && gc < G::CG) {
        gIs[gr * G::PPG + gc] = ix;
        gIs[G::PLANE_G + gr * G::PPG + gc] = iy;
    }
}

template <int WK>
__global__ void __launch_bounds__(kHbThreads, 2)
    k_harris_bwd_fused(const float* __restrict__ I, long long i_pitch, const float* __restrict__ gR, long long g_pitch,
                       float* dI, long long d_pitch, int W, int H, float k, const float* sx_dev, const float* sy_dev,
                       const float* gw_dev, const __grid_constant__ HbTaps<WK> tp, float* part_w, float* part_sx,
                       float* part_sy) {
    using G = HbGeo<WK>;
    constexpr int RW = G::RW, TW = G::TW, TH = G::TH, HI = G::HI, HP = G::HP, HS = G::HS;
    extern __shared__ __align__(16) float hsm[];
    float* taps = hsm + G::O_TAP;                 // window (WK*WK), Sobel x (9), Sobel y (9)
    float* Is = hsm + G::O_I;
    float* Ps = hsm + G::O_P;                     // Pxx, Pyy, Pxy planes; later gP
    float* gSs = hsm + G::O_S;                    // window sums, then gSxx, gSyy, gSxy planes
    float* gIs = hsm + G::O_G;                    // Ix, Iy planes; later gIx, gIy
    const int tid = threadIdx.x;
    constexpr int nth = kHbThreads;
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

    const int tiles_x = (W + TW - 1) / TW, tiles_y = (H + TH - 1) / TH;
    // Tiles whose halo leaves the image take the slower clamped paths.  They lie in tile
    // row 0 and rows ryb.., tile column 0 and columns cxb.. (TH, TW > HI); the CTAs take
    // tiles round-robin in the order border rows, then the border columns of the other
    // rows, then the interior, so each gets about the same share of border tiles (a
    // static order: the tap-gradient partials stay reproducible).
    int ryb = tiles_y, cxb = tiles_x;
    while (ryb > 1 && (ryb - 1) * TH + TH + HI > H) --ryb;
    while (cxb > 1 && (cxb - 1) * TW + TW + HI > W) --cxb;
    const int nbr = 1 + tiles_y - ryb, nbc = 1 + tiles_x - cxb, nic = cxb - 1;
    for (int t = blockIdx.x; t < tiles_x * tiles_y; t += gridDim.x) {
        int tx, ty;
        if (t < nbr * tiles_x) {
            const int rr = t / tiles_x;
            ty = rr == 0 ? 0 : ryb + rr - 1;
            tx = t - rr * tiles_x;
        } else if (t < nbr * tiles_x + (ryb - 1) * nbc) {
            const int o = t - nbr * tiles_x, cc = o % nbc;
            ty = 1 + o / nbc;
            tx = cc == 0 ? 0 : cxb + cc - 1;
        } else {
            const int o = t - nbr * tiles_x - (ryb - 1) * nbc;
            ty = 1 + o / nic;
            tx = 1 + o % nic;
        }
        const int x0 = tx * TW, y0 = ty * TH;
        const bool border_tile = x0 - HI < 0 || y0 - HI < 0 || x0 + TW + HI > W || y0 + TH + HI > H;
        __syncthreads();   // taps staged / the previous tile's planes are no longer read
        // (1) I on the I region (rows from y0 - HI, columns from x0 - HI), at clamped positions
        //     (all of a thread's loads issued before its first store)
        {
            constexpr int N = G::RI * G::CI, NQ = (N + kHbThreads - 1) / kHbThreads;
            float v[NQ];
#pragma unroll
            for (int n = 0; n < NQ; ++n) {
                const int q = tid + n * kHbThreads, r = q / G::CI, c = q - r * G::CI;
                const int gy = clampi(y0 - HI + r, 0, H - 1), gx = clampi(x0 - HI + c, 0, W - 1);
                v[n] = q < N ? I[(long long)gy * i_pitch + gx] : 0.f;
            }
#pragma unroll
            for (int n = 0; n < NQ; ++n) {
                const int q = tid + n * kHbThreads, r = q / G::CI, c = q - r * G::CI;
                if (q < N) Is[r * G::PPI + c] = v[n];
            }
        }
        __syncthreads();
        // (2) Ix, Iy and the products on the P region, each at its clamped pixel; Ix and
        //     Iy also into the gI planes where the gI region covers the pixel
        if (border_tile) {
            for (int q = tid; q < G::RP * G::CP; q += nth) {
                const int r = q / G::CP, c = q - r * G::CP;
                const int ir = clampi(y0 - HP + r, 0, H - 1) - (y0 - HI);
                const int ic = clampi(x0 - HP + c, 0, W - 1) - (x0 - HI);
                float ix = 0.f, iy = 0.f;
#pragma unroll
                for (int j = 0; j < 3; ++j)
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        const float u = Is[(ir - 1 + j) * G::PPI + ic - 1 + i];
                        ix = __fmaf_rn(sxw[j * 3 + i], u, ix);
                        iy = __fmaf_rn(syw[j * 3 + i], u, iy);
                    }
                hb_store_p<WK>(Ps, gIs, r, c, ix, iy);
            }
        } else {
            // columns fastest, 4 rows per item: the I-region rows r0 .. r0 + 5 around them
            for (int q = tid; q < G::NRP * G::CP; q += nth) {
                const int r0 = (q / G::CP) * 4, c = q - (r0 / 4) * G::CP;
                float u[6][3];
#pragma unroll
                for (int jj = 0; jj < 6; ++jj)
#pragma unroll
                    for (int i = 0; i < 3; ++i) u[jj][i] = Is[(r0 + jj + (HI - HP) - 1) * G::PPI + c + (HI - HP) - 1 + i];
#pragma unroll
                for (int py = 0; py < 4; ++py) {
                    if (r0 + py >= G::RP) break;
                    float ix = 0.f, iy = 0.f;
#pragma unroll
                    for (int j = 0; j < 3; ++j)
#pragma unroll
                        for (int i = 0; i < 3; ++i) {
                            ix = __fmaf_rn(sxw[j * 3 + i], u[py + j][i], ix);
                            iy = __fmaf_rn(syw[j * 3 + i], u[py + j][i], iy);
                        }
                    hb_store_p<WK>(Ps, gIs, r0 + py, c, ix, iy);
                }
            }
        }
        __syncthreads();
        // (3) window sums S_c on the gS region: items of one channel x PYS rows x 4 columns,
        //     P rows r0 .. r0 + PYS - 1 + 2RW each feeding the item rows it lies under
        {
            float wr[WK * WK];
#pragma unroll
            for (int q = 0; q < WK * WK; ++q) wr[q] = gw[q];
            for (int it = tid; it < 3 * G::NRS * G::NCS; it += nth) {
                const int ch = it / (G::NRS * G::NCS), rem = it - ch * (G::NRS * G::NCS);
                const int r0 = (rem / G::NCS) * G::PYS, c0 = (rem % G::NCS) * 4;
                float s[G::PYS][4];
#pragma unroll
                for (int py = 0; py < G::PYS; ++py)
#pragma unroll
                    for (int e = 0; e < 4; ++e) s[py][e] = 0.f;
                const float* pr = Ps + ch * G::PLANE_P + r0 * G::PPP + c0;
#pragma unroll
                for (int jr = 0; jr < WK + G::PYS - 1; ++jr) {
                    float v[4 * G::NV];
#pragma unroll
                    for (int q = 0; q < G::NV; ++q) {
                        const float4 f = *reinterpret_cast<const float4*>(pr + jr * G::PPP + 4 * q);
                        v[4 * q] = f.x; v[4 * q + 1] = f.y; v[4 * q + 2] = f.z; v[4 * q + 3] = f.w;
                    }
#pragma unroll
                    for (int py = 0; py < G::PYS; ++py) {
                        const int j = jr - py;                 // window row of this P row for item row py
                        if (j < 0 || j >= WK) continue;
#pragma unroll
                        for (int i = 0; i < WK; ++i)
#pragma unroll
                            for (int e = 0; e < 4; ++e) s[py][e] = __fmaf_rn(wr[j * WK + i], v[e + i], s[py][e]);
                    }
                }
                float* sr = gSs + ch * G::PLANE_S + r0 * G::PPS + c0;
#pragma unroll
                for (int py = 0; py < G::PYS; ++py)
                    *reinterpret_cast<float4*>(sr + py * G::PPS) = make_float4(s[py][0], s[py][1], s[py][2], s[py][3]);
            }
        }
        __syncthreads();
        // (3b) gS from the window sums and gR, in place (zero outside the image), one quad
        //     of columns per item; all of a thread's gR loads issued first
        {
            constexpr int N = G::RS * G::NCS, NQ = (N + kHbThreads - 1) / kHbThreads;
            float gv[NQ][4];
#pragma unroll
            for (int n = 0; n < NQ; ++n) {
                const int q = tid + n * kHbThreads, r = q / G::NCS, c = (q - r * G::NCS) * 4;
                const int gy = y0 - HS + r, gx = x0 - HS + c;
                const bool row_in = q < N && gy >= 0 && gy < H;
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    gv[n][e] = row_in && gx + e >= 0 && gx + e < W && c + e < G::CS ? gR[(long long)gy * g_pitch + gx + e] : 0.f;
            }
#pragma unroll
            for (int n = 0; n < NQ; ++n) {
                const int q = tid + n * kHbThreads, r = q / G::NCS, c = (q - r * G::NCS) * 4;
                if (q >= N) continue;
                float* o = gSs + r * G::PPS + c;
                const float4 sxx = *reinterpret_cast<const float4*>(o);
                const float4 syy = *reinterpret_cast<const float4*>(o + G::PLANE_S);
                const float4 sxy = *reinterpret_cast<const float4*>(o + 2 * G::PLANE_S);
                const float a[4] = {sxx.x, sxx.y, sxx.z, sxx.w}, b[4] = {syy.x, syy.y, syy.z, syy.w};
                const float d[4] = {sxy.x, sxy.y, sxy.z, sxy.w};
                const int gy = y0 - HS + r, gx = x0 - HS + c;
                float gxx[4], gyy[4], gxy[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const bool in = gy >= 0 && gy < H && gx + e >= 0 && gx + e < W;
                    const float g = gv[n][e], tr = a[e] + b[e];
                    gxx[e] = in ? g * (b[e] - 2.f * k * tr) : 0.f;
                    gyy[e] = in ? g * (a[e] - 2.f * k * tr) : 0.f;
                    gxy[e] = in ? -2.f * g * d[e] : 0.f;
                }
                *reinterpret_cast<float4*>(o) = make_float4(gxx[0], gxx[1], gxx[2], gxx[3]);
                *reinterpret_cast<float4*>(o + G::PLANE_S) = make_float4(gyy[0], gyy[1], gyy[2], gyy[3]);
                *reinterpret_cast<float4*>(o + 2 * G::PLANE_S) = make_float4(gxy[0], gxy[1], gxy[2], gxy[3]);
            }
        }
        __syncthreads();
        // (4) window-tap gradient: dG[o] += gS_c(p) P_c(b(p + o)) over the tile's pixels
        //     (gS is zero outside the image), items of one channel x PYT rows x 4 columns
        for (int it = tid; it < 3 * G::NRT * G::NCT; it += nth) {
            const int ch = it / (G::NRT * G::NCT), rem = it - ch * (G::NRT * G::NCT);
            const int r0 = (rem / G::NCT) * G::PYT, c0 = (rem % G::NCT) * 4;
            float g[G::PYT][4];
#pragma unroll
            for (int py = 0; py < G::PYT; ++py)
#pragma unroll
                for (int e = 0; e < 4; ++e) g[py][e] = gSs[ch * G::PLANE_S + (r0 + py + HS) * G::PPS + c0 + e + HS];
            const float* pr = Ps + ch * G::PLANE_P + (r0 + G::OFF4) * G::PPP + c0;
#pragma unroll
            for (int jr = 0; jr < WK + G::PYT - 1; ++jr) {
                float v[4 * G::NV4];
#pragma unroll
                for (int q = 0; q < G::NV4; ++q) {
                    const float4 f = *reinterpret_cast<const float4*>(pr + jr * G::PPP + 4 * q);
                    v[4 * q] = f.x; v[4 * q + 1] = f.y; v[4 * q + 2] = f.z; v[4 * q + 3] = f.w;
                }
#pragma unroll
                for (int py = 0; py < G::PYT; ++py) {
                    const int j = jr - py;
                    if (j < 0 || j >= WK) continue;
#pragma unroll
                    for (int i = 0; i < WK; ++i)
#pragma unroll
                        for (int e = 0; e < 4; ++e) aw[j * WK + i] = __fmaf_rn(g[py][e], v[e + i + G::OFF4], aw[j * WK + i]);
                }
            }
        }
        __syncthreads();   // P is no longer read: (5) writes gP over it
        // (5) gP_c on the gI region (window adjoint; the clamp folds follow in (5b)), items
        //     of one channel x 4 rows x 4 columns over gS rows r0 .. r0 + 3 + 2RW
        {
            float wr[WK * WK];
#pragma unroll
            for (int q = 0; q < WK * WK; ++q) wr[q] = gw[q];
            for (int it = tid; it < 3 * G::NRG * G::NCG; it += nth) {
                const int ch = it / (G::NRG * G::NCG), rem = it - ch * (G::NRG * G::NCG);
                const int r0 = (rem / G::NCG) * 4, c0 = (rem % G::NCG) * 4;
                float gp[4][4];
#pragma unroll
                for (int py = 0; py < 4; ++py)
#pragma unroll
                    for (int e = 0; e < 4; ++e) gp[py][e] = 0.f;
                const float* gs = gSs + ch * G::PLANE_S;
#pragma unroll
                for (int jr = 0; jr < WK + 3; ++jr) {
                    float v[4 * G::NV];
#pragma unroll
                    for (int q = 0; q < G::NV; ++q) {
                        const float4 f = *reinterpret_cast<const float4*>(gs + (r0 + jr) * G::PPS + c0 + 4 * q);
                        v[4 * q] = f.x; v[4 * q + 1] = f.y; v[4 * q + 2] = f.z; v[4 * q + 3] = f.w;
                    }
#pragma unroll
                    for (int py = 0; py < 4; ++py) {
                        const int j = py + 2 * RW - jr;        // gS at q - o: row r0 + py + 2RW - j
                        if (j < 0 || j >= WK) continue;
#pragma unroll
                        for (int i = 0; i < WK; ++i)
#pragma unroll
                            for (int e = 0; e < 4; ++e) gp[py][e] = __fmaf_rn(wr[j * WK + i], v[e + 2 * RW - i], gp[py][e]);
                    }
                }
                float* gq = Ps + ch * G::PLANE_P + r0 * G::PPP + c0;
#pragma unroll
                for (int py = 0; py < 4; ++py)
                    *reinterpret_cast<float4*>(gq + py * G::PPP) = make_float4(gp[py][0], gp[py][1], gp[py][2], gp[py][3]);
            }
        }
        __syncthreads();
        // (5b) gI from gP and (Ix, Iy), in place over Ix, Iy (zero outside the image), one
        //     quad of columns per item; on the image's edges gP first collects the window
        //     offsets clamped onto the pixel
        for (int q = tid; q < G::RG * G::NCG; q += kHbThreads) {
            const int r = q / G::NCG, c = (q - r * G::NCG) * 4;
            const int gy = y0 - 1 + r, gx = x0 - 1 + c;
            float* o = gIs + r * G::PPG + c;
            const float* op = Ps + r * G::PPP + c;
            const float4 vx = *reinterpret_cast<const float4*>(o), vy = *reinterpret_cast<const float4*>(o + G::PLANE_G);
            const float4 vxx = *reinterpret_cast<const float4*>(op);
            const float4 vyy = *reinterpret_cast<const float4*>(op + G::PLANE_P);
            const float4 vxy = *reinterpret_cast<const float4*>(op + 2 * G::PLANE_P);
            const float ix[4] = {vx.x, vx.y, vx.z, vx.w}, iy[4] = {vy.x, vy.y, vy.z, vy.w};
            float gxx[4] = {vxx.x, vxx.y, vxx.z, vxx.w}, gyy[4] = {vyy.x, vyy.y, vyy.z, vyy.w};
            float gxy[4] = {vxy.x, vxy.y, vxy.z, vxy.w};
            float gix[4], giy[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int px = gx + e;
                const bool in = c + e < G::CG && px >= 0 && px < W && gy >= 0 && gy < H;
                if (in && border_tile && (px == 0 || gy == 0 || px == W - 1 || gy == H - 1))
                    hb_clamp_fold<RW>(px, gy, W, H, [&](int j, int i, int sy, int sx) {
                        const int os = (sy - (y0 - HS)) * G::PPS + sx - (x0 - HS);
                        const float w = gw[j * WK + i];
                        gxx[e] = __fmaf_rn(w, gSs[os], gxx[e]);
                        gyy[e] = __fmaf_rn(w, gSs[G::PLANE_S + os], gyy[e]);
                        gxy[e] = __fmaf_rn(w, gSs[2 * G::PLANE_S + os], gxy[e]);
                    });
                gix[e] = in ? 2.f * ix[e] * gxx[e] + iy[e] * gxy[e] : 0.f;
                giy[e] = in ? 2.f * iy[e] * gyy[e] + ix[e] * gxy[e] : 0.f;
            }
            *reinterpret_cast<float4*>(o) = make_float4(gix[0], gix[1], gix[2], gix[3]);
            *reinterpret_cast<float4*>(o + G::PLANE_G) = make_float4(giy[0], giy[1], giy[2], giy[3]);
        }
        __syncthreads();
        // (6) dI on the tile (Sobel adjoint with the clamp folds) and the Sobel tap
        //     gradients: columns fastest, 4 rows per item over gI rows r0 .. r0 + 5
        for (int q = tid; q < (TH / 4) * TW; q += nth) {
            const int r0 = (q / TW) * 4, tx = q - (r0 / 4) * TW;
            const int gx = x0 + tx;
            if (gx >= W || y0 + r0 >= H) continue;
            float gc[2][4];                       // gIx, gIy at the item's pixels
            {
                float ga[6][3], gb[6][3];
#pragma unroll
                for (int jj = 0; jj < 6; ++jj)
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        ga[jj][i] = gIs[(r0 + jj) * G::PPG + tx + i];
                        gb[jj][i] = gIs[G::PLANE_G + (r0 + jj) * G::PPG + tx + i];
                    }
#pragma unroll
                for (int py = 0; py < 4; ++py) {
                    const int gy = y0 + r0 + py;
                    gc[0][py] = ga[py + 1][1];
                    gc[1][py] = gb[py + 1][1];
                    if (gy >= H) continue;
                    float acc = 0.f;
#pragma unroll
                    for (int j = 0; j < 3; ++j)
#pragma unroll
                        for (int i = 0; i < 3; ++i) {
                            // gI at q - o: gI-region (ty + 1 - (j - 1), tx + 1 - (i - 1))
                            acc = __fmaf_rn(sxw[j * 3 + i], ga[py + 2 - j][2 - i], acc);
                            acc = __fmaf_rn(syw[j * 3 + i], gb[py + 2 - j][2 - i], acc);
                        }
                    if (border_tile && (gx == 0 || gy == 0 || gx == W - 1 || gy == H - 1))
                        hb_clamp_fold<1>(gx, gy, W, H, [&](int j, int i, int py2, int px2) {
                            const int o = (py2 - (y0 - 1)) * G::PPG + px2 - (x0 - 1);
                            acc = __fmaf_rn(sxw[j * 3 + i], gIs[o], acc);
                            acc = __fmaf_rn(syw[j * 3 + i], gIs[G::PLANE_G + o], acc);
                        });
                    if (dI) dI[(long long)gy * d_pitch + gx] = acc;
                }
            }
            float u[6][3];                        // I(b(p + o)) rows around the item
#pragma unroll
            for (int jj = 0; jj < 6; ++jj)
#pragma unroll
                for (int i = 0; i < 3; ++i) u[jj][i] = Is[(r0 + jj + HI - 1) * G::PPI + tx + HI - 1 + i];
#pragma unroll
            for (int py = 0; py < 4; ++py) {
                if (y0 + r0 + py >= H) break;
#pragma unroll
                for (int j = 0; j < 3; ++j)
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        asx[j * 3 + i] = __fmaf_rn(gc[0][py], u[py + j][i], asx[j * 3 + i]);
                        asy[j * 3 + i] = __fmaf_rn(gc[1][py], u[py + j][i], asy[j * 3 + i]);
                    }
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
