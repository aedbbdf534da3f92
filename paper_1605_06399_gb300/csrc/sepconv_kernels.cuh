// sepconv_kernels.cuh -- separable correlation (§6 separable convolution benchmark).
//
//   t(x, y)   = sum_i row[i] * in(b(x + i - rr, y))        row pass, boundary rule on in
//   out(x, y) = sum_j col[j] * t(x, b(y + j - rc))         column pass, boundary rule on t
//
// The paper runs the two passes as two kernels (Table 2: R and C) and notes (§7) that
// fusing them with the intermediate kept in on-chip memory is what its language could
// not express.  Here:
//  * k_sep_row_plain / k_sep_col_plain: the untuned two-kernel form (one pixel per
//    thread, clamped global loads, rolled loops, t in a caller workspace in f32);
//  * k_sepconv_fused: one kernel.  A CTA stages its input tile plus R halo rows and PAD
//    halo columns (TMA double-buffered ring, cooperative loads, or the L1 path), runs
//    the row pass for the TH + 2R rows the column pass needs into an f32 buffer in
//    shared memory, then the column pass from that buffer, and writes the tile once:
//    one HBM read and one write per pixel.
// Row and column tap counts may differ: both are zero-padded (exactly neutral) to the
// kernel's radius R = max(rr, rc).  The UNROLL_PACKED form does both passes with f32x2
// FMAs over adjacent column pairs.
#pragma once

#include "tile_common.cuh"

namespace imcl {

// ------------------------------------------------------------------ plain, unfused
template <typename Tin>
__global__ void __launch_bounds__(256)
    k_sep_row_plain(const ConvArgs a, const __grid_constant__ TapsParam<float, 2 * 33> tp) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= a.W) return;
    const Tin* in = static_cast<const Tin*>(a.in);
    const float* row = a.taps_dev ? static_cast<const float*>(a.taps_dev) : tp.w;
    const float bv = to_acc(border_pixel<Tin>(a));
    const int rr = (a.kw - 1) / 2;
    for (int y = blockIdx.y * blockDim.y + threadIdx.y; y < a.H; y += gridDim.y * blockDim.y) {
        float acc = 0.f;
#pragma unroll 1
        for (int i = 0; i < a.kw; ++i) {
            const int gx = x + i - rr;
            float v;
            if (gx >= 0 && gx < a.W) v = to_acc(in[(long long)y * a.in_pitch + gx]);
            else if (a.border == IMCL_BORDER_CONSTANT) v = bv;
            else v = to_acc(in[(long long)y * a.in_pitch + clampi(gx, 0, a.W - 1)]);
            acc = __fmaf_rn(row[i], v, acc);
        }
        static_cast<float*>(a.work)[(long long)y * a.W + x] = acc;
    }
}

template <typename Tout>
__global__ void __launch_bounds__(256)
    k_sep_col_plain(const ConvArgs a, const __grid_constant__ TapsParam<float, 2 * 33> tp) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= a.W) return;
    const float* t = static_cast<const float*>(a.work);
    const float* col = a.taps2_dev ? static_cast<const float*>(a.taps2_dev) : tp.w + 33;
    const int rc = (a.kh - 1) / 2;
    for (int y = blockIdx.y * blockDim.y + threadIdx.y; y < a.H; y += gridDim.y * blockDim.y) {
        float acc = 0.f;
#pragma unroll 1
        for (int j = 0; j < a.kh; ++j) {
            const int gy = y + j - rc;
            float v;
            if (gy >= 0 && gy < a.H) v = t[(long long)gy * a.W + x];
            else if (a.border == IMCL_BORDER_CONSTANT) v = a.bv_f;
            else v = t[(long long)clampi(gy, 0, a.H - 1) * a.W + x];
            acc = __fmaf_rn(col[j], v, acc);
        }
        static_cast<Tout*>(a.out)[(long long)y * a.out_pitch + x] = Store<Tout, float>::cvt(acc);
    }
}

// ------------------------------------------------------------------ fused
// t[ox] = sum_i w[i] * seg[LO + ox + i] for ox < N, as scalar FMAs or as packed f32x2
// FMAs over the column pairs (2p, 2p + 1); each lane keeps the scalar operation order.
// The packed form takes its taps duplicated, (w, w) per tap.
template <int N, int NT, int LO, int UNR, typename W>
__device__ __forceinline__ void row_taps(const float* seg, const W* w, float* t) {
    if constexpr (UNR == IMCL_UNROLL_PACKED) {
        static_assert(N % 2 == 0, "packed rows need an even width");
        float2 sp[N + NT - 2];
#pragma unroll
        for (int k = 0; k < N + NT - 2; ++k) sp[k] = make_float2(seg[LO + k], seg[LO + k + 1]);
        float2 t2[N / 2];
#pragma unroll
        for (int p = 0; p < N / 2; ++p) t2[p] = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < NT; ++i) {
#pragma unroll
            for (int p = 0; p < N / 2; ++p) t2[p] = mad2(w[i], sp[2 * p + i], t2[p]);
        }
#pragma unroll
        for (int p = 0; p < N / 2; ++p) {
            t[2 * p] = t2[p].x;
            t[2 * p + 1] = t2[p].y;
        }
    } else {
#pragma unroll
        for (int ox = 0; ox < N; ++ox) t[ox] = 0.f;
#pragma unroll
        for (int i = 0; i < NT; ++i) {
            const float wi = w[i];
#pragma unroll
            for (int ox = 0; ox < N; ++ox) t[ox] = __fmaf_rn(wi, seg[LO + ox + i], t[ox]);
        }
    }
}

// acc[ox] += w * t[ox] for ox < N (scalar, or packed over column pairs with w = (w, w)).
template <int N, int UNR, typename W>
__device__ __forceinline__ void axpy_row(const W w, const float* t, float* acc) {
    if constexpr (UNR == IMCL_UNROLL_PACKED) {
        const float2 w2 = w;
#pragma unroll
        for (int p = 0; p < N / 2; ++p) {
            const float2 r = mad2(w2, make_float2(t[2 * p], t[2 * p + 1]), make_float2(acc[2 * p], acc[2 * p + 1]));
            acc[2 * p] = r.x;
            acc[2 * p + 1] = r.y;
        }
    } else {
#pragma unroll
        for (int ox = 0; ox < N; ++ox) acc[ox] = __fmaf_rn(w, t[ox], acc[ox]);
    }
}

// MODE 0: the row pass result goes through a shared f32 buffer (rows computed once);
// MODE 1: each thread keeps the row pass of its own PY + 2R input rows in registers
// (halo rows computed by the threads above and below as well, no buffer, one barrier
// less), for small radii.
template <typename Tin, typename Tout, int R, int PX, int PY, int LOAD, int FILT, int MODE, int UNR>
__global__ void __launch_bounds__(256, MODE == 1 ? 3 : 1)
    k_sepconv_fused(const ConvArgs a, const __grid_constant__ TapsParamFor<float, 2 * (2 * R + 1), UNR> tp,
                    const __grid_constant__ CUtensorMap tmap) {
    constexpr int NT = 2 * R + 1;
    using G = TileGeo<Tin, NT, PX>;      // staging geometry (PAD)
    using GR = TileGeo<Tin, NT, 8>;      // row pass: 8 outputs per work item, same PAD
    static_assert(PX == 4, "the t buffer is written and read as float4");
    static_assert(G::PAD == GR::PAD, "row pass and staging must agree on the halo");
    extern __shared__ __align__(128) uint8_t smem[];

    const int tid = threadIdx.x, nth = blockDim.x;
    const int bx = a.bx, by = a.by;
    const int TW = bx * PX, TH = by * PY;
    const int SW = TW + 2 * G::PAD, SH = TH + 2 * R;
    const int stage_bytes = round_up(SW * SH * G::SZ, 128);
    constexpr int kStages = LOAD == IMCL_LOAD_TMA ? 2 : (LOAD == IMCL_LOAD_SMEM ? 1 : 0);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    float* tbuf = reinterpret_cast<float*>(smem + 128 + kStages * stage_bytes);
    using W = typename std::remove_cv<typename std::remove_reference<decltype(tp.w[0])>::type>::type;
    W* wsm = reinterpret_cast<W*>(tbuf + (MODE == 0 ? SH * TW : 0));

    const Tin* in = static_cast<const Tin*>(a.in);
    Tout* out = static_cast<Tout*>(a.out);
    const Tin bv_t = border_pixel<Tin>(a);
    const float bv = to_acc(bv_t);

    if constexpr (FILT == IMCL_FILT_SMEM) {
        if (a.taps_dev) {
            const int orr = R - (a.kw - 1) / 2, orc = R - (a.kh - 1) / 2;
            const float* rd = static_cast<const float*>(a.taps_dev);
            const float* cd = static_cast<const float*>(a.taps2_dev);
            for (int i = tid; i < NT; i += nth) {
                const float r = (i >= orr && i < orr + a.kw) ? rd[i - orr] : 0.f;
                const float c = (i >= orc && i < orc + a.kh) ? cd[i - orc] : 0.f;
                if constexpr (UNR == IMCL_UNROLL_PACKED) {
                    wsm[i] = make_float2(r, r);
                    wsm[NT + i] = make_float2(c, c);
                } else {
                    wsm[i] = r;
                    wsm[NT + i] = c;
                }
            }
        } else {
            for (int i = tid; i < 2 * NT; i += nth) wsm[i] = tp.w[i];
        }
    }
    const W* rw;
    if constexpr (FILT == IMCL_FILT_SMEM) rw = wsm; else rw = tp.w;
    const W* cw = rw + NT;

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
            mbar_arrive_expect_tx(&bar[0], (uint32_t)(SW * SH * G::SZ));
            tma_load_2d(smem + 128, &tmap, tx0 - G::PAD, ty0 - R, &bar[0]);
        }
    } else {
        __syncthreads();
    }

    for (; t < ntiles; t += gridDim.x) {
        const int x0 = (t % a.tiles_x) * TW, y0 = (t / a.tiles_x) * TH;
        const int gx0 = x0 - G::PAD, gy0 = y0 - R;
        Tin* st = reinterpret_cast<Tin*>(smem + 128 + s * stage_bytes);

        if constexpr (LOAD == IMCL_LOAD_TMA) {
            const int tn = t + gridDim.x;
            const bool prefetch = tn < ntiles;
            if (tid == 0 && prefetch) {
                const int nx0 = (tn % a.tiles_x) * TW, ny0 = (tn / a.tiles_x) * TH;
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&bar[s ^ 1], (uint32_t)(SW * SH * G::SZ));
                tma_load_2d(smem + 128 + (s ^ 1) * stage_bytes, &tmap, nx0 - G::PAD, ny0 - R, &bar[s ^ 1]);
            }
            const bool ok = mbar_wait(&bar[s], (parity >> s) & 1u, a.status);
            parity ^= (1u << s);
            if (__syncthreads_or(!ok)) {
                if (tid == 0 && prefetch) mbar_wait(&bar[s ^ 1], (parity >> (s ^ 1)) & 1u, nullptr);
                return;
            }
            if (!tile_inside(gx0, gy0, SW, SH, a.W, a.H))
                patch_tile<Tin>(st, SW, SH, gx0, gy0, a.W, a.H, a.border, bv_t, tid, nth);
        } else if constexpr (LOAD == IMCL_LOAD_SMEM) {
            coop_load_tile<Tin>(st, in, a.in_pitch, SW, SH, gx0, gy0, a.W, a.H, a.border, bv_t, a.vec_in != 0,
                                tid, nth);
            __syncthreads();
        }

        if constexpr (MODE == 1) {
            const int tx = tid % bx, ty = tid / bx;
            float acc[PY][PX];
#pragma unroll
            for (int oy = 0; oy < PY; ++oy)
#pragma unroll
                for (int ox = 0; ox < PX; ++ox) acc[oy][ox] = 0.f;
#pragma unroll
            for (int yy = 0; yy < PY + 2 * R; ++yy) {
                const int row = ty * PY + yy;
                const int gy = gy0 + row;
                float t4[PX];
                if (a.border == IMCL_BORDER_CONSTANT && (gy < 0 || gy >= a.H)) {
#pragma unroll
                    for (int ox = 0; ox < PX; ++ox) t4[ox] = a.bv_f;   // t is padded with the constant
                } else {
                    float seg[G::SEG];
                    if constexpr (LOAD == IMCL_LOAD_GLOBAL)
                        load_seg_global<Tin, G>(in, a.in_pitch, gy, x0 + tx * PX - G::PAD, a.W, a.H, a.border, bv,
                                                a.vec_in != 0, seg);
                    else
                        load_seg_smem<Tin, G>(st + row * SW + tx * PX, seg);
                    row_taps<PX, NT, G::LO, UNR>(seg, rw, t4);
                }
#pragma unroll
                for (int oy = 0; oy < PY; ++oy) {
                    const int j = yy - oy;
                    if (j >= 0 && j < NT) axpy_row<PX, UNR>(cw[j], t4, acc[oy]);
                }
            }
#pragma unroll
            for (int oy = 0; oy < PY; ++oy)
                store_block_row<Tout, PX>(out, a.out_pitch, x0 + tx * PX, y0 + ty * PY + oy, a.W, a.H,
                                          a.vec_out != 0, acc[oy]);
        } else {
            // row pass: t for the SH staged rows and TW columns, 8 columns per work item; a
            // thread keeps one column segment and steps down the rows
            {
                const int nseg = TW / 8, rstep = nth / nseg;
                const int c0 = (tid % nseg) * 8;
                for (int row = tid / nseg; row < SH; row += rstep) {
                    const int gy = gy0 + row;
                    float r8[8];
                    if (a.border == IMCL_BORDER_CONSTANT && (gy < 0 || gy >= a.H)) {
    #pragma unroll
                        for (int ox = 0; ox < 8; ++ox) r8[ox] = a.bv_f;   // t is padded with the constant
                    } else {
                        float seg[GR::SEG];
                        if constexpr (LOAD == IMCL_LOAD_GLOBAL)
                            load_seg_global<Tin, GR>(in, a.in_pitch, gy, x0 + c0 - GR::PAD, a.W, a.H, a.border, bv,
                                                     a.vec_in != 0, seg);
                        else
                            load_seg_smem<Tin, GR>(st + row * SW + c0, seg);
                        row_taps<8, NT, GR::LO, UNR>(seg, rw, r8);
                    }
                    float* tp = tbuf + row * TW + c0;
                    *reinterpret_cast<float4*>(tp) = make_float4(r8[0], r8[1], r8[2], r8[3]);
                    *reinterpret_cast<float4*>(tp + 4) = make_float4(r8[4], r8[5], r8[6], r8[7]);
                }
            }
            __syncthreads();

            // column pass: PX x PY block per thread, sliding down the t buffer
            {
                const int tx = tid % bx, ty = tid / bx;
                float acc[PY][PX];
    #pragma unroll
                for (int oy = 0; oy < PY; ++oy)
    #pragma unroll
                    for (int ox = 0; ox < PX; ++ox) acc[oy][ox] = 0.f;
    #pragma unroll
                for (int yy = 0; yy < PY + 2 * R; ++yy) {
                    const float4 v = *reinterpret_cast<const float4*>(tbuf + (ty * PY + yy) * TW + tx * PX);
                    const float tv[4] = {v.x, v.y, v.z, v.w};
    #pragma unroll
                    for (int oy = 0; oy < PY; ++oy) {
                        const int j = yy - oy;
                        if (j >= 0 && j < NT) axpy_row<PX, UNR>(cw[j], tv, acc[oy]);
                    }
                }
    #pragma unroll
                for (int oy = 0; oy < PY; ++oy)
                    store_block_row<Tout, PX>(out, a.out_pitch, x0 + tx * PX, y0 + ty * PY + oy, a.W, a.H,
                                              a.vec_out != 0, acc[oy]);
            }
        }
        __syncthreads();   // t buffer and stage s may be refilled
        if constexpr (LOAD == IMCL_LOAD_TMA) s ^= 1;
    }
}

// ------------------------------------------------------------------ host launchers
template <typename W>
inline void fill_sep_taps(W* w, int R, const ConvCall& c) {
    const int NT = 2 * R + 1;
    for (int i = 0; i < 2 * NT; ++i) set_tap(w[i], 0.f);
    if (c.taps_mem != IMCL_MEM_HOST) return;
    const float* row = static_cast<const float*>(c.taps);
    const float* col = static_cast<const float*>(c.taps2);
    const int orr = R - (c.kw - 1) / 2, orc = R - (c.kh - 1) / 2;
    for (int i = 0; i < c.kw; ++i) set_tap(w[orr + i], row[i]);
    for (int j = 0; j < c.kh; ++j) set_tap(w[NT + orc + j], col[j]);
}

template <typename Tin, typename Tout>
imcl_status launch_sep_plain(const ConvCall& c, const imcl_variant& v, cudaStream_t s) {
    const size_t need = (size_t)c.W * c.H * sizeof(float);
    if (!c.workspace || c.ws_bytes < need)
        return fail(IMCL_ERR_INVALID, "the unfused separable kernels need a workspace of width*height*4 bytes");
    const int bx = v.bx > 0 ? v.bx : 16, by = v.by > 0 ? v.by : 16;
    if (bx * by > 256) return fail(IMCL_ERR_UNSUPPORTED, "plain kernel: bx*by must be <= 256");
    ConvArgs a = make_conv_args(c, v, 1, 1);
    TapsParam<float, 66> tp;
    for (int i = 0; i < 66; ++i) tp.w[i] = 0.f;
    if (c.taps_mem == IMCL_MEM_HOST) {
        for (int i = 0; i < c.kw; ++i) tp.w[i] = static_cast<const float*>(c.taps)[i];
        for (int j = 0; j < c.kh; ++j) tp.w[33 + j] = static_cast<const float*>(c.taps2)[j];
    }
    dim3 grid = grid_2d(c.W, c.H, bx, by), block(bx, by);
    k_sep_row_plain<Tin><<<grid, block, 0, s>>>(a, tp);
    k_sep_col_plain<Tout><<<grid, block, 0, s>>>(a, tp);
    return cuda_fail(cudaGetLastError(), "sepconv plain launch");
}

template <typename Tin, typename Tout, int R, int PX, int PY, int LOAD, int FILT, int MODE, int UNR>
imcl_status launch_sep_fused(const ConvCall& c, const imcl_variant& v, cudaStream_t s) {
    constexpr int NT = 2 * R + 1;
    using G = TileGeo<Tin, NT, PX>;
    const int bx = v.bx, by = v.by, nth = bx * by;
    if (bx <= 0 || by <= 0 || nth > 256 || nth % 32 != 0)
        return fail(IMCL_ERR_UNSUPPORTED, "fused sepconv: bx*by must be a multiple of 32, at most 256");
    if ((bx * PX) % G::CV != 0) return fail(IMCL_ERR_UNSUPPORTED, "fused sepconv: bx*px must be a multiple of 16 bytes");
    if ((bx * PX) % 8 != 0 || nth % ((bx * PX) / 8) != 0)
        return fail(IMCL_ERR_UNSUPPORTED, "fused sepconv: the row pass needs tile widths of 8 columns per thread group");
    if (std::max(1, (std::max(c.kw, c.kh) - 1) / 2) != R)
        return fail(IMCL_ERR_UNSUPPORTED, "fused sepconv: radius mismatch");
    if (c.taps_mem == IMCL_MEM_DEVICE && FILT != IMCL_FILT_SMEM)
        return fail(IMCL_ERR_UNSUPPORTED, "device-resident taps need a FILT_SMEM variant");
    const int TW = bx * PX, TH = by * PY;
    const int SW = TW + 2 * G::PAD, SH = TH + 2 * R;
    if (LOAD == IMCL_LOAD_TMA && (SW > 256 || SH > 256))
        return fail(IMCL_ERR_UNSUPPORTED, "fused sepconv: TMA box larger than 256 in a dimension");
    const int stage_bytes = round_up(SW * SH * G::SZ, 128);
    const int nstage = LOAD == IMCL_LOAD_TMA ? 2 : (LOAD == IMCL_LOAD_SMEM ? 1 : 0);
    using TP = TapsParamFor<float, 2 * NT, UNR>;
    const int smem = 128 + nstage * stage_bytes + (MODE == 0 ? SH * TW * 4 : 0) + (int)sizeof(TP);
    if (smem > c.dev->max_smem_optin) return fail(IMCL_ERR_UNSUPPORTED, "fused sepconv: tile too large for shared memory");
    auto kfn = k_sepconv_fused<Tin, Tout, R, PX, PY, LOAD, FILT, MODE, UNR>;
    imcl_status st = set_smem_limit((const void*)kfn, smem);
    if (st != IMCL_OK) return st;
    // the L1-path row pass reads GR::VB-pixel vectors straight from global memory
    using GR = TileGeo<Tin, NT, 8>;
    const int in_align = (LOAD == IMCL_LOAD_GLOBAL) ? GR::VB * GR::SZ : 16;
    ConvArgs a = make_conv_args(c, v, in_align, PX * (int)sizeof(Tout) > 16 ? 16 : PX * (int)sizeof(Tout));
    a.tiles_x = (c.W + TW - 1) / TW;
    a.tiles_y = (c.H + TH - 1) / TH;
    const int ntiles = a.tiles_x * a.tiles_y;
    CUtensorMap tmap;
    memset(&tmap, 0, sizeof(tmap));
    if (LOAD == IMCL_LOAD_TMA) {
        if ((reinterpret_cast<uintptr_t>(c.in) & 15) || (c.in_pitch_b & 15))
            return fail(IMCL_ERR_ALIGN, "TMA staging needs a 16-byte aligned input and pitch");
        st = encode_tmap_2d(&tmap, c.in_dtype, c.in, c.W, c.H, c.in_pitch_b, SW, SH);
        if (st != IMCL_OK) return st;
    }
    TP tp;
    fill_sep_taps(tp.w, R, c);
    int grid = ntiles;
    if (v.persistent || LOAD == IMCL_LOAD_TMA) {
        const int occ = cached_occupancy((const void*)kfn, nth, smem);
        if (occ <= 0) return fail(IMCL_ERR_UNSUPPORTED, "fused sepconv: kernel cannot be resident");
        const int slots = occ * c.dev->sm_count;
        grid = ntiles < slots ? ntiles : slots;
    }
    kfn<<<grid, nth, smem, s>>>(a, tp, tmap);
    return cuda_fail(cudaGetLastError(), "sepconv fused launch");
}

template <typename Tin, typename Tout, int R, int PX, int PY, int LOAD, int FILT, int MODE = 0,
          int UNR = IMCL_UNROLL_FULL>
inline ConvEntry sep_entry(int bx, int by, int persistent) {
    imcl_variant v{};
    v.kind = IMCL_KIND_TILED;
    v.bx = bx;
    v.by = by;
    v.px = PX;
    v.py = PY;
    v.load = LOAD;
    v.filt = FILT;
    v.map = MODE == 1 ? IMCL_MAP_REGISTER : IMCL_MAP_BLOCKED;
    v.unroll = UNR;
    v.persistent = persistent;
    return ConvEntry{DtypeOf<Tin>::v, DtypeOf<Tout>::v, R, v,
                     &launch_sep_fused<Tin, Tout, R, PX, PY, LOAD, FILT, MODE, UNR>};
}

}  // namespace imcl
