// harris_kernels.cuh -- Harris corner response (§6 corner-detection benchmark; the paper
// runs a Sobel kernel and a Harris kernel, Tables 4 and 5).  Clamped boundary on every
// stage's input:
//   Ix = Sx (*) I,  Iy = Sy (*) I                       3x3 correlations
//   Pxx = Ix^2, Pyy = Iy^2, Pxy = Ix Iy
//   Sc = G (*) Pc                                       WK x WK window, c in {xx, yy, xy}
//   R = Sxx Syy - Sxy^2 - k (Sxx + Syy)^2
//
//  * k_harris_sobel_plain + k_harris_resp_plain: the untuned two-kernel form (Ix, Iy in
//    a caller workspace; one pixel per thread; clamped global loads; rolled loops).
//  * k_harris_fused: one kernel per tile.  The image tile plus a (WK/2 + 1)-pixel halo
//    is staged in shared memory (TMA ring or cooperative loads) and patched to the clamp
//    rule; the three products are formed for the tile plus the window halo, each at
//    the clamped position of its pixel (so a product outside the image equals the
//    product at the nearest pixel inside, which is what the clamped window reads); the
//    window sums run on a register-blocked PX x PY layout over the three planes and the
//    response is formed in registers: one HBM read and one write per pixel.
#pragma once

#include "tile_common.cuh"

namespace imcl {

// Window tap (j, i) of a WK x WK window reads offset (i - WK/2, j - WK/2): centred for
// odd WK, offsets {-1, 0} for the 2x2 block.  Window-pass geometry: the product buffer's
// column c holds region column c (image column x0 - WK/2 + c), so a thread's segment
// starts at its own first output column, 16-byte aligned, and holds exactly the
// PX + WK - 1 products it needs (rounded up to whole float4s).
template <int WK>
struct HarrisWindowGeo {
    static constexpr int PX = 4;
    static constexpr int WLO = WK / 2;
    static constexpr int VB = 4;
    static constexpr int SEG = round_up(PX + WK - 1, 4);
    static constexpr int LO = 0;
    static constexpr int USED = PX + WK - 1;
};

// taps of the Harris operator as they travel in the launch parameters
template <int WK>
struct HarrisTaps {
    float sx[9];
    float sy[9];
    float g[WK * WK];
};

// ------------------------------------------------------------------ plain, unfused
__global__ void __launch_bounds__(256)
    k_harris_sobel_plain(const ConvArgs a, const __grid_constant__ HarrisTaps<7> tp) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= a.W) return;
    const float* in = static_cast<const float*>(a.in);
    const float* sx = a.taps_dev ? static_cast<const float*>(a.taps_dev) : tp.sx;
    const float* sy = a.taps2_dev ? static_cast<const float*>(a.taps2_dev) : tp.sy;
    for (int y = blockIdx.y * blockDim.y + threadIdx.y; y < a.H; y += gridDim.y * blockDim.y) {
        float gx = 0.f, gy = 0.f;
#pragma unroll 1
        for (int j = 0; j < 3; ++j) {
            const int yy = clampi(y + j - 1, 0, a.H - 1);
#pragma unroll 1
            for (int i = 0; i < 3; ++i) {
                const float v = in[(long long)yy * a.in_pitch + clampi(x + i - 1, 0, a.W - 1)];
                gx = __fmaf_rn(sx[j * 3 + i], v, gx);
                gy = __fmaf_rn(sy[j * 3 + i], v, gy);
            }
        }
        float* ix = static_cast<float*>(a.work);
        ix[(long long)y * a.W + x] = gx;
        ix[(long long)a.W * a.H + (long long)y * a.W + x] = gy;
    }
}

__global__ void __launch_bounds__(256)
    k_harris_resp_plain(const ConvArgs a, const __grid_constant__ HarrisTaps<7> tp) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= a.W) return;
    const float* ix = static_cast<const float*>(a.work);
    const float* iy = ix + (long long)a.W * a.H;
    // a.kw: the (odd) side run; a.kh: the caller's side, the stride of device taps (an
    // even window runs with a zero last row and column)
    const float* gd = static_cast<const float*>(a.taps3_dev);
    const int wk = a.kw, rw = wk / 2, src = a.kh;   // tap j reads offset j - wk/2
    for (int y = blockIdx.y * blockDim.y + threadIdx.y; y < a.H; y += gridDim.y * blockDim.y) {
        float sxx = 0.f, syy = 0.f, sxy = 0.f;
#pragma unroll 1
        for (int j = 0; j < wk; ++j) {
            const int yy = clampi(y + j - rw, 0, a.H - 1);
#pragma unroll 1
            for (int i = 0; i < wk; ++i) {
                const long long o = (long long)yy * a.W + clampi(x + i - rw, 0, a.W - 1);
                const float w = gd ? ((j < src && i < src) ? gd[j * src + i] : 0.f) : tp.g[j * wk + i];
                const float gx = ix[o], gy = iy[o];
                sxx = __fmaf_rn(w, gx * gx, sxx);
                syy = __fmaf_rn(w, gy * gy, syy);
                sxy = __fmaf_rn(w, gx * gy, sxy);
            }
        }
        const float tr = sxx + syy;
        static_cast<float*>(a.out)[(long long)y * a.out_pitch + x] = sxx * syy - sxy * sxy - a.hk * tr * tr;
    }
}

// ------------------------------------------------------------------ fused
template <int WK, int PY, int LOAD, int FILT>
__global__ void __launch_bounds__(256, 2)
    k_harris_fused(const ConvArgs a, const __grid_constant__ HarrisTaps<WK> tp,
                   const __grid_constant__ CUtensorMap tmap) {
    constexpr int PX = 4;
    constexpr int WLO = WK / 2;                        // window rows / columns before the pixel
    constexpr int HALO = WLO + 1;                      // input rows/cols before the tile
    constexpr int PADI = 4;                            // staged input halo columns (16 B)
    static_assert(HALO <= PADI && WK - WLO <= PADI, "window too large for the staged halo");
    using GW = HarrisWindowGeo<WK>;                   // window pass: region column == buffer column
    extern __shared__ __align__(128) uint8_t smem[];

    const int tid = threadIdx.x, nth = blockDim.x;
    const int bx = a.bx, by = a.by;
    const int TW = bx * PX, TH = by * PY;
    const int SW = TW + 2 * PADI, SH = TH + WK + 1;
    const int NG = (TW + WK - 1 + 3) / 4;              // product groups of 4 columns per row
    const int PH = TH + WK - 1, PW = 4 * NG;
    const int stage_bytes = round_up(SW * SH * 4, 128);
    constexpr int kStages = LOAD == IMCL_LOAD_TMA ? 2 : 1;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    float* pbuf = reinterpret_cast<float*>(smem + 128 + kStages * stage_bytes);   // 3 planes PH x PW
    float* wsm = pbuf + 3 * PH * PW;                                               // 18 + WK*WK taps
    const int plane = PH * PW;

    if constexpr (FILT == IMCL_FILT_SMEM) {
        const float* sx = a.taps_dev ? static_cast<const float*>(a.taps_dev) : tp.sx;
        const float* sy = a.taps2_dev ? static_cast<const float*>(a.taps2_dev) : tp.sy;
        const float* gd = static_cast<const float*>(a.taps3_dev);
        const int src = a.kh;   // the caller's window side (device taps' stride)
        for (int i = tid; i < 18 + WK * WK; i += nth) {
            float v;
            if (i < 9) v = sx[i];
            else if (i < 18) v = sy[i - 9];
            else if (!gd) v = tp.g[i - 18];
            else {
                const int j = (i - 18) / WK, c = (i - 18) % WK;
                v = (j < src && c < src) ? gd[j * src + c] : 0.f;
            }
            wsm[i] = v;
        }
    }
    const float *sxw, *syw, *gw;
    if constexpr (FILT == IMCL_FILT_SMEM) { sxw = wsm; syw = wsm + 9; gw = wsm + 18; }
    else { sxw = tp.sx; syw = tp.sy; gw = tp.g; }

    const float* in = static_cast<const float*>(a.in);
    float* out = static_cast<float*>(a.out);
    const int ntiles = a.tiles_x * a.tiles_y;
    int t = blockIdx.x;
    int s = 0;
    uint32_t parity = 0;
    if constexpr (LOAD == IMCL_LOAD_TMA) {
        if (tid == 0) {
            prefetch_tmap(&tmap);
            mbar_init(&bar[0], 1);
            mbar_init(&bar[1], 1);
            fence_mbar_init();
        }
        __syncthreads();
        if (tid == 0 && t < ntiles) {
            const int tx0 = (t % a.tiles_x) * TW, ty0 = (t / a.tiles_x) * TH;
            mbar_arrive_expect_tx(&bar[0], (uint32_t)(SW * SH * 4));
            tma_load_2d(smem + 128, &tmap, tx0 - PADI, ty0 - HALO, &bar[0]);
        }
    } else {
        __syncthreads();
    }

    for (; t < ntiles; t += gridDim.x) {
        const int x0 = (t % a.tiles_x) * TW, y0 = (t / a.tiles_x) * TH;
        const int gx0 = x0 - PADI, gy0 = y0 - HALO;
        float* st = reinterpret_cast<float*>(smem + 128 + s * stage_bytes);
        if constexpr (LOAD == IMCL_LOAD_TMA) {
            const int tn = t + gridDim.x;
            const bool prefetch = tn < ntiles;
            if (tid == 0 && prefetch) {
                const int nx0 = (tn % a.tiles_x) * TW, ny0 = (tn / a.tiles_x) * TH;
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&bar[s ^ 1], (uint32_t)(SW * SH * 4));
                tma_load_2d(smem + 128 + (s ^ 1) * stage_bytes, &tmap, nx0 - PADI, ny0 - HALO, &bar[s ^ 1]);
            }
            const bool ok = mbar_wait(&bar[s], (parity >> s) & 1u, a.status);
            parity ^= (1u << s);
            if (__syncthreads_or(!ok)) {
                if (tid == 0 && prefetch) mbar_wait(&bar[s ^ 1], (parity >> (s ^ 1)) & 1u, nullptr);
                return;
            }
            if (!tile_inside(gx0, gy0, SW, SH, a.W, a.H))
                patch_tile<float>(st, SW, SH, gx0, gy0, a.W, a.H, IMCL_BORDER_CLAMP, 0.f, tid, nth);
        } else {
            coop_load_tile<float>(st, in, a.in_pitch, SW, SH, gx0, gy0, a.W, a.H, IMCL_BORDER_CLAMP, 0.f,
                                  a.vec_in != 0, tid, nth);
            __syncthreads();
        }

        // products for the (TW + WK - 1) x (TH + WK - 1) window region, 4 columns per item.
        // Product column pc (region-local, 0 = image column x0 - WLO) lives at pbuf column
        // pc, so a group of 4 is one aligned float4 per plane.  Each product is taken at
        // the clamped position of its pixel.
        const bool interior = x0 - WLO >= 0 && y0 - WLO >= 0 && x0 - WLO + 4 * NG <= a.W &&
                              y0 - WLO + PH <= a.H;
        for (int it = tid; it < PH * NG; it += nth) {
            const int pr = it / NG, pc0 = (it - pr * NG) * 4;
            float gx[4], gy[4];
            if (interior) {
                // input column of region column pc is pc + PADI - WLO; the Sobel reads -1..+1
                const float* r0 = st + pr * SW + pc0;   // aligned chunk holding column pc0 + PADI-WLO-1
#pragma unroll
                for (int e = 0; e < 4; ++e) { gx[e] = 0.f; gy[e] = 0.f; }
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    float v[8];
                    const float4 c0 = *reinterpret_cast<const float4*>(r0 + j * SW);
                    const float4 c1 = *reinterpret_cast<const float4*>(r0 + j * SW + 4);
                    v[0] = c0.x; v[1] = c0.y; v[2] = c0.z; v[3] = c0.w;
                    v[4] = c1.x; v[5] = c1.y; v[6] = c1.z; v[7] = c1.w;
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        const float wx = sxw[j * 3 + i], wy = syw[j * 3 + i];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float u = v[PADI - WLO - 1 + e + i];
                            gx[e] = __fmaf_rn(wx, u, gx[e]);
                            gy[e] = __fmaf_rn(wy, u, gy[e]);
                        }
                    }
                }
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    // clamped pixel of this product, in input-tile coordinates
                    const int px = clampi(x0 - WLO + pc0 + e, 0, a.W - 1) - gx0;
                    const int py = clampi(y0 - WLO + pr, 0, a.H - 1) - gy0;
                    float ax = 0.f, ay = 0.f;
                    if (px >= 1 && px < SW - 1 && py >= 1 && py < SH - 1) {
#pragma unroll
                        for (int j = 0; j < 3; ++j)
#pragma unroll
                            for (int i = 0; i < 3; ++i) {
                                const float u = st[(py - 1 + j) * SW + px - 1 + i];
                                ax = __fmaf_rn(sxw[j * 3 + i], u, ax);
                                ay = __fmaf_rn(syw[j * 3 + i], u, ay);
                            }
                    } else {
                        dev_fail(a.status, DEVERR_BOUNDS);   // geometry guarantees this never runs
                    }
                    gx[e] = ax;
                    gy[e] = ay;
                }
            }
            float* p = pbuf + pr * PW + pc0;
            *reinterpret_cast<float4*>(p) =
                make_float4(gx[0] * gx[0], gx[1] * gx[1], gx[2] * gx[2], gx[3] * gx[3]);
            *reinterpret_cast<float4*>(p + plane) =
                make_float4(gy[0] * gy[0], gy[1] * gy[1], gy[2] * gy[2], gy[3] * gy[3]);
            *reinterpret_cast<float4*>(p + 2 * plane) =
                make_float4(gx[0] * gy[0], gx[1] * gy[1], gx[2] * gy[2], gx[3] * gy[3]);
        }
        __syncthreads();

        // window sums on PX x PY blocks, then the response
        {
            const int tx = tid % bx, ty = tid / bx;
            float axx[PY][PX], ayy[PY][PX], axy[PY][PX];
#pragma unroll
            for (int oy = 0; oy < PY; ++oy)
#pragma unroll
                for (int ox = 0; ox < PX; ++ox) { axx[oy][ox] = 0.f; ayy[oy][ox] = 0.f; axy[oy][ox] = 0.f; }
#pragma unroll
            for (int yy = 0; yy < PY + WK - 1; ++yy) {
                float sxx[GW::SEG], syy[GW::SEG], sxy[GW::SEG];
                const float* rp = pbuf + (ty * PY + yy) * PW + tx * PX;
                load_seg_smem<float, GW>(rp, sxx);
                load_seg_smem<float, GW>(rp + plane, syy);
                load_seg_smem<float, GW>(rp + 2 * plane, sxy);
                fma_row_blocked<GW, WK, PX, PY, 0>(yy, sxx, axx, gw);
                fma_row_blocked<GW, WK, PX, PY, 0>(yy, syy, ayy, gw);
                fma_row_blocked<GW, WK, PX, PY, 0>(yy, sxy, axy, gw);
            }
#pragma unroll
            for (int oy = 0; oy < PY; ++oy) {
                float r[PX];
#pragma unroll
                for (int ox = 0; ox < PX; ++ox) {
                    const float tr = axx[oy][ox] + ayy[oy][ox];
                    r[ox] = axx[oy][ox] * ayy[oy][ox] - axy[oy][ox] * axy[oy][ox] - a.hk * tr * tr;
                }
                store_block_row<float, PX>(out, a.out_pitch, x0 + tx * PX, y0 + ty * PY + oy, a.W, a.H,
                                           a.vec_out != 0, r);
            }
        }
        __syncthreads();
        if constexpr (LOAD == IMCL_LOAD_TMA) s ^= 1;
    }
}

// ------------------------------------------------------------------ host launchers
// Host taps into the launch parameters; the window (c.kh x c.kh, the caller's side)
// goes into the top-left of the c.kw x c.kw table, zeros elsewhere.
template <int WK>
inline void fill_harris_taps(HarrisTaps<WK>& tp, const ConvCall& c) {
    memset(&tp, 0, sizeof tp);
    if (c.taps_mem != IMCL_MEM_HOST) return;
    memcpy(tp.sx, c.taps, 9 * sizeof(float));
    memcpy(tp.sy, c.taps2, 9 * sizeof(float));
    const float* g = static_cast<const float*>(c.taps3);
    for (int j = 0; j < c.kh; ++j)
        for (int i = 0; i < c.kh; ++i) tp.g[j * c.kw + i] = g[j * c.kh + i];
}

imcl_status launch_harris_plain(const ConvCall& c, const imcl_variant& v, cudaStream_t s);

template <int WK, int PY, int LOAD, int FILT>
imcl_status launch_harris_fused(const ConvCall& c, const imcl_variant& v, cudaStream_t s) {
    constexpr int PX = 4, PADI = 4;
    const int bx = v.bx, by = v.by, nth = bx * by;
    if (bx <= 0 || by <= 0 || nth > 256 || nth % 32 != 0)
        return fail(IMCL_ERR_UNSUPPORTED, "fused harris: bx*by must be a multiple of 32, at most 256");
    if (c.kw != WK) return fail(IMCL_ERR_UNSUPPORTED, "fused harris: window side mismatch");
    if (c.taps_mem == IMCL_MEM_DEVICE && FILT != IMCL_FILT_SMEM)
        return fail(IMCL_ERR_UNSUPPORTED, "device-resident taps need a FILT_SMEM variant");
    const int TW = bx * PX, TH = by * PY;
    const int SW = TW + 2 * PADI, SH = TH + WK + 1;
    if (LOAD == IMCL_LOAD_TMA && (SW > 256 || SH > 256))
        return fail(IMCL_ERR_UNSUPPORTED, "fused harris: TMA box larger than 256 in a dimension");
    const int PH = TH + WK - 1, PW = 4 * ((TW + WK - 1 + 3) / 4);
    const int stage_bytes = round_up(SW * SH * 4, 128);
    const int nstage = LOAD == IMCL_LOAD_TMA ? 2 : 1;
    const int smem = 128 + nstage * stage_bytes + 3 * PH * PW * 4 + (18 + WK * WK) * 4;
    if (smem > c.dev->max_smem_optin) return fail(IMCL_ERR_UNSUPPORTED, "fused harris: tile too large for shared memory");
    auto kfn = k_harris_fused<WK, PY, LOAD, FILT>;
    imcl_status st = set_smem_limit((const void*)kfn, smem);
    if (st != IMCL_OK) return st;
    ConvArgs a = make_conv_args(c, v, 16, 16);
    a.tiles_x = (c.W + TW - 1) / TW;
    a.tiles_y = (c.H + TH - 1) / TH;
    const int ntiles = a.tiles_x * a.tiles_y;
    CUtensorMap tmap;
    memset(&tmap, 0, sizeof(tmap));
    if (LOAD == IMCL_LOAD_TMA) {
        if ((reinterpret_cast<uintptr_t>(c.in) & 15) || (c.in_pitch_b & 15))
            return fail(IMCL_ERR_ALIGN, "TMA staging needs a 16-byte aligned input and pitch");
        st = encode_tmap_2d(&tmap, IMCL_F32, c.in, c.W, c.H, c.in_pitch_b, SW, SH);
        if (st != IMCL_OK) return st;
    }
    HarrisTaps<WK> tp;
    fill_harris_taps(tp, c);
    int grid = ntiles;
    if (v.persistent || LOAD == IMCL_LOAD_TMA) {
        const int occ = cached_occupancy((const void*)kfn, nth, smem);
        if (occ <= 0) return fail(IMCL_ERR_UNSUPPORTED, "fused harris: kernel cannot be resident");
        const int slots = occ * c.dev->sm_count;
        grid = ntiles < slots ? ntiles : slots;
    }
    kfn<<<grid, nth, smem, s>>>(a, tp, tmap);
    return cuda_fail(cudaGetLastError(), "harris fused launch");
}

template <int WK, int PY, int LOAD, int FILT>
inline ConvEntry harris_entry(int bx, int by, int persistent) {
    imcl_variant v{};
    v.kind = IMCL_KIND_TILED;
    v.bx = bx;
    v.by = by;
    v.px = 4;
    v.py = PY;
    v.load = LOAD;
    v.filt = FILT;
    v.map = IMCL_MAP_BLOCKED;
    v.unroll = 1;
    v.persistent = persistent;
    return ConvEntry{IMCL_F32, IMCL_F32, WK, v, &launch_harris_fused<WK, PY, LOAD, FILT>};
}

}  // namespace imcl
