// conv2d_kernels.cuh -- non-separable correlation kernels (§6 non-separable convolution).
//
//   out(x, y) = sum_{j<K, i<K} w[j][i] * in(b(x + i - R, y + j - R)),   R = (K-1)/2
//
// b() is the boundary rule of §5 / Fig. 3 (clamp each coordinate, or a constant).
//
// Two kernel families:
//  * k_conv2d_plain: the untuned baseline, i.e. what naive code generation gives (§5.1):
//    one pixel per thread, 16x16 blocks, every tap read straight from global memory
//    with the boundary rule applied per read, taps read per use, rolled loops.
//  * k_conv2d_tiled: the tuned family.  A CTA owns a TW x TH output tile
//    (TW = bx*PX, TH = by*PY: work-group size x thread coarsening, Table 1).  The input
//    tile plus a halo of R rows and PAD >= R columns is staged in shared memory (the
//    "local memory" transform of §5.2, Fig. 5) either by a 2D TMA copy into a
//    double-buffered ring driven by an mbarrier (LOAD_TMA, persistent CTAs prefetch the
//    next tile while computing this one), or by cooperative 16-byte loads (LOAD_SMEM);
//    LOAD_GLOBAL skips shared memory and reads through the L1/texture path (the "image
//    memory" option).  Each thread computes a PX x PY register block, walking the PY+K-1
//    input rows once and reusing every loaded row segment for all output rows and taps
//    that need it.  Taps come from the launch's parameter space (FILT_PARAM, the
//    constant bank, §5.2 "constant memory") or from shared memory (FILT_SMEM).
//
// TMA fills out-of-image parts of the box with zeros; tiles that touch the border are
// then patched in shared memory (clamp: copy the nearest in-image pixel; constant: write
// the constant), so the compute loop never branches on the border.
#pragma once

#include "tile_common.cuh"

namespace imcl {

// ------------------------------------------------------------------ plain kernel
template <typename Tin, typename Tout, bool DEV_TAPS>
__global__ void __launch_bounds__(256)
    k_conv2d_plain(const ConvArgs a, const __grid_constant__ TapsParam<typename AccOf<Tin>::type, kMaxK * kMaxK> tp) {
    using Acc = typename AccOf<Tin>::type;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= a.W) return;
    const Tin* in = static_cast<const Tin*>(a.in);
    const Acc* taps = DEV_TAPS ? static_cast<const Acc*>(a.taps_dev) : tp.w;
    const int rx = (a.kw - 1) / 2, ry = (a.kh - 1) / 2;
    const Acc bv = to_acc(border_pixel<Tin>(a));
    for (int y = blockIdx.y * blockDim.y + threadIdx.y; y < a.H; y += gridDim.y * blockDim.y) {
        Acc acc = 0;
#pragma unroll 1
        for (int j = 0; j < a.kh; ++j) {
            const int gy = y + j - ry;
#pragma unroll 1
            for (int i = 0; i < a.kw; ++i) {
                const int gx = x + i - rx;
                Acc v;
                if (gx >= 0 && gx < a.W && gy >= 0 && gy < a.H) {
                    v = to_acc(in[(long long)gy * a.in_pitch + gx]);
                } else if (a.border == IMCL_BORDER_CONSTANT) {
                    v = bv;
                } else {
                    v = to_acc(in[(long long)clampi(gy, 0, a.H - 1) * a.in_pitch + clampi(gx, 0, a.W - 1)]);
                }
                acc = mad(taps[j * a.kw + i], v, acc);
            }
        }
        static_cast<Tout*>(a.out)[(long long)y * a.out_pitch + x] = Store<Tout, Acc>::cvt(acc);
    }
}

// ------------------------------------------------------------------ tiled kernel
// FACC: integer (u8) pixels and taps accumulated with f32 FMAs.  Every product and
// partial sum is an integer of magnitude at most sum |w| * 255; while that stays below
// 2^24 all of them are exact in f32, so the int32 result is bit-identical to integer
// accumulation (the launcher checks the bound) at the FP32 pipe's rate, which is twice
// the int32 multiply-add rate.
template <typename Tin, bool FACC>
using TiledAcc = typename std::conditional<FACC, float, typename AccOf<Tin>::type>::type;

template <typename Tin, typename Tout, int K, int PX, int PY, int LOAD, int FILT, int MAP, bool FACC = false>
__global__ void __launch_bounds__(256, 2)
    k_conv2d_tiled(const ConvArgs a, const __grid_constant__ TapsParam<TiledAcc<Tin, FACC>, K * K> tp,
                   const __grid_constant__ CUtensorMap tmap) {
    using Acc = TiledAcc<Tin, FACC>;
    using G = TileGeo<Tin, K, PX>;
    constexpr int R = G::R;
    extern __shared__ __align__(128) uint8_t smem[];

    const int tid = threadIdx.x, nth = blockDim.x;
    const int bx = a.bx, by = a.by;
    const int tx = tid % bx, ty = tid / bx;
    const int TW = bx * PX, TH = by * PY;
    const int SW = TW + 2 * G::PAD, SH = TH + K - 1;
    const int stage_bytes = round_up(SW * SH * G::SZ, 128);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    Tin* stage0 = reinterpret_cast<Tin*>(smem + 128);
    constexpr int kStages = LOAD == IMCL_LOAD_TMA ? 2 : (LOAD == IMCL_LOAD_SMEM ? 1 : 0);
    Acc* wsm = reinterpret_cast<Acc*>(smem + 128 + kStages * stage_bytes);

    const Tin* in = static_cast<const Tin*>(a.in);
    Tout* out = static_cast<Tout*>(a.out);
    const Tin bv_t = border_pixel<Tin>(a);
    const Acc bv = to_acc(bv_t);

    if constexpr (FILT == IMCL_FILT_SMEM) {
        const Acc* src = a.taps_dev ? static_cast<const Acc*>(a.taps_dev) : tp.w;
        for (int i = tid; i < K * K; i += nth) wsm[i] = src[i];
    }
    const Acc* wp;
    if constexpr (FILT == IMCL_FILT_SMEM) wp = wsm; else wp = tp.w;

    const int ntiles = a.tiles_x * a.tiles_y;
    int t = blockIdx.x;
    int s = 0;
    uint32_t parity = 0;   // bit s: phase to wait for on stage s

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
            tma_load_2d(stage0, &tmap, tx0 - G::PAD, ty0 - R, &bar[0]);
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
                // stage s^1 was released by the barrier that ended the previous iteration
                Tin* nst = reinterpret_cast<Tin*>(smem + 128 + (s ^ 1) * stage_bytes);
                const int nx0 = (tn % a.tiles_x) * TW, ny0 = (tn / a.tiles_x) * TH;
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&bar[s ^ 1], (uint32_t)(SW * SH * G::SZ));
                tma_load_2d(nst, &tmap, nx0 - G::PAD, ny0 - R, &bar[s ^ 1]);
            }
            const bool ok = mbar_wait(&bar[s], (parity >> s) & 1u, a.status);
            parity ^= (1u << s);
            if (__syncthreads_or(!ok)) {
                // give the prefetch issued above a bounded chance to land before exiting
                if (tid == 0 && prefetch) mbar_wait(&bar[s ^ 1], (parity >> (s ^ 1)) & 1u, nullptr);
                return;
            }
            if (!tile_inside(gx0, gy0, SW, SH, a.W, a.H))
                patch_tile<Tin>(st, SW, SH, gx0, gy0, a.W, a.H, a.border, bv_t, tid, nth);
        } else if constexpr (LOAD == IMCL_LOAD_SMEM) {
            coop_load_tile<Tin>(st, in, a.in_pitch, SW, SH, gx0, gy0, a.W, a.H, a.border, bv_t,
                                a.vec_in != 0, tid, nth);
            __syncthreads();
        }

        Acc acc[PY][PX];
#pragma unroll
        for (int oy = 0; oy < PY; ++oy)
#pragma unroll
            for (int ox = 0; ox < PX; ++ox) acc[oy][ox] = Acc(0);

        if constexpr (MAP == IMCL_MAP_BLOCKED) {
            const int r0 = ty * PY;   // first input row of the thread's block (tile-local)
#pragma unroll
            for (int yy = 0; yy < PY + K - 1; ++yy) {
                Acc seg[G::SEG];
                if constexpr (LOAD == IMCL_LOAD_GLOBAL) {
                    load_seg_global<Tin, G>(in, a.in_pitch, y0 + r0 + yy - R, x0 + tx * PX - G::PAD, a.W,
                                            a.H, a.border, bv, a.vec_in != 0, seg);
                } else {
                    load_seg_smem<Tin, G>(st + (r0 + yy) * SW + tx * PX, seg);
                }
                fma_row_blocked<G, K, PX, PY, FILT>(yy, seg, acc, wp);
            }
#pragma unroll
            for (int oy = 0; oy < PY; ++oy)
                store_block_row<Tout, PX>(out, a.out_pitch, x0 + tx * PX, y0 + r0 + oy, a.W, a.H,
                                          a.vec_out != 0, acc[oy]);
        } else {
            // MAP_INTERLEAVED: output rows ty, ty + by, ty + 2 by, ... (no vertical reuse)
#pragma unroll
            for (int oy = 0; oy < PY; ++oy) {
                const int r0 = ty + oy * by;
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    Acc seg[G::SEG];
                    if constexpr (LOAD == IMCL_LOAD_GLOBAL) {
                        load_seg_global<Tin, G>(in, a.in_pitch, y0 + r0 + j - R, x0 + tx * PX - G::PAD,
                                                a.W, a.H, a.border, bv, a.vec_in != 0, seg);
                    } else {
                        load_seg_smem<Tin, G>(st + (r0 + j) * SW + tx * PX, seg);
                    }
#pragma unroll
                    for (int i = 0; i < K; ++i) {
                        const Acc w = wp[j * K + i];
#pragma unroll
                        for (int ox = 0; ox < PX; ++ox)
                            acc[oy][ox] = mad(w, seg[G::LO + ox + i], acc[oy][ox]);
                    }
                }
            }
#pragma unroll
            for (int oy = 0; oy < PY; ++oy)
                store_block_row<Tout, PX>(out, a.out_pitch, x0 + tx * PX, y0 + ty + oy * by, a.W, a.H,
                                          a.vec_out != 0, acc[oy]);
        }

        if constexpr (LOAD != IMCL_LOAD_GLOBAL) __syncthreads();   // stage s may be refilled
        if constexpr (LOAD == IMCL_LOAD_TMA) s ^= 1;
    }
}

// ------------------------------------------------------------------ host launchers
template <typename Acc, int N>
inline void fill_taps(TapsParam<Acc, N>& tp, const ConvCall& c) {
    for (int i = 0; i < N; ++i) tp.w[i] = Acc(0);
    if (c.taps_mem == IMCL_MEM_HOST) {
        const Acc* src = static_cast<const Acc*>(c.taps);
        for (int i = 0; i < c.kw * c.kh && i < N; ++i) tp.w[i] = src[i];
    }
}

template <typename Tin, typename Tout>
imcl_status launch_conv_plain(const ConvCall& c, const imcl_variant& v, cudaStream_t s) {
    using Acc = typename AccOf<Tin>::type;
    const int bx = v.bx > 0 ? v.bx : 16, by = v.by > 0 ? v.by : 16;
    if (bx * by > 256 || bx * by <= 0) return fail(IMCL_ERR_UNSUPPORTED, "plain kernel: bx*by must be <= 256");
    ConvArgs a = make_conv_args(c, v, 1, 1);
    TapsParam<Acc, kMaxK * kMaxK> tp;
    fill_taps(tp, c);
    dim3 grid = grid_2d(c.W, c.H, bx, by), block(bx, by);
    if (c.taps_mem == IMCL_MEM_DEVICE)
        k_conv2d_plain<Tin, Tout, true><<<grid, block, 0, s>>>(a, tp);
    else
        k_conv2d_plain<Tin, Tout, false><<<grid, block, 0, s>>>(a, tp);
    return cuda_fail(cudaGetLastError(), "conv2d plain launch");
}

template <typename Tin, typename Tout, int K, int PX, int PY, int LOAD, int FILT, int MAP, bool FACC = false>
imcl_status launch_conv_tiled(const ConvCall& c, const imcl_variant& v, cudaStream_t s) {
    using Acc = TiledAcc<Tin, FACC>;
    using G = TileGeo<Tin, K, PX>;
    if constexpr (FACC) {
        static_assert(std::is_same<Tin, uint8_t>::value, "f32 accumulation of integer taps: u8 images only");
        // exact only while sum |w| * 255 < 2^24; otherwise the integer-accumulating twin
        if (c.taps_mem != IMCL_MEM_HOST || c.kw != K || c.kh != K)
            return fail(IMCL_ERR_UNSUPPORTED, "f32-accumulating u8 conv2d takes host taps of its side");
        int64_t l1 = 0;
        for (int i = 0; i < K * K; ++i) {
            const int64_t w = static_cast<const int32_t*>(c.taps)[i];
            l1 += w < 0 ? -w : w;
        }
        if (l1 * 255 >= (int64_t(1) << 24)) return launch_conv_tiled<Tin, Tout, K, PX, PY, LOAD, FILT, MAP, false>(c, v, s);
    }
    const int bx = v.bx, by = v.by;
    const int nth = bx * by;
    if (bx <= 0 || by <= 0 || nth > 256 || nth % 32 != 0)
        return fail(IMCL_ERR_UNSUPPORTED, "tiled conv2d: bx*by must be a multiple of 32, at most 256");
    if ((bx * PX) % G::CV != 0) return fail(IMCL_ERR_UNSUPPORTED, "tiled conv2d: bx*px must be a multiple of 16 bytes");
    const int TW = bx * PX, TH = by * PY;
    const int SW = TW + 2 * G::PAD, SH = TH + K - 1;
    if (LOAD == IMCL_LOAD_TMA && (SW > 256 || SH > 256))
        return fail(IMCL_ERR_UNSUPPORTED, "tiled conv2d: TMA box larger than 256 in a dimension");
    if (c.kw != K || c.kh != K) return fail(IMCL_ERR_UNSUPPORTED, "tiled conv2d: filter side mismatch");
    if (c.taps_mem == IMCL_MEM_DEVICE && FILT != IMCL_FILT_SMEM)
        return fail(IMCL_ERR_UNSUPPORTED, "device-resident taps need a FILT_SMEM variant");
    const int stage_bytes = round_up(SW * SH * G::SZ, 128);
    const int nstage = LOAD == IMCL_LOAD_TMA ? 2 : (LOAD == IMCL_LOAD_SMEM ? 1 : 0);
    const int smem = 128 + nstage * stage_bytes + (FILT == IMCL_FILT_SMEM ? K * K * (int)sizeof(Acc) : 0);
    if (smem > c.dev->max_smem_optin) return fail(IMCL_ERR_UNSUPPORTED, "tiled conv2d: tile too large for shared memory");

    auto kfn = k_conv2d_tiled<Tin, Tout, K, PX, PY, LOAD, FILT, MAP, FACC>;
    imcl_status st = set_smem_limit((const void*)kfn, smem);
    if (st != IMCL_OK) return st;
    const int in_align = (LOAD == IMCL_LOAD_GLOBAL) ? G::VB * G::SZ : 16;
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
    TapsParam<Acc, K * K> tp;
    if constexpr (FACC) {
        for (int i = 0; i < K * K; ++i) tp.w[i] = (float)static_cast<const int32_t*>(c.taps)[i];
    } else {
        fill_taps(tp, c);
    }
    int grid = ntiles;
    if (v.persistent || LOAD == IMCL_LOAD_TMA) {
        const int occ = cached_occupancy((const void*)kfn, nth, smem);
        if (occ <= 0) return fail(IMCL_ERR_UNSUPPORTED, "tiled conv2d: kernel cannot be resident");
        const int slots = occ * c.dev->sm_count;
        grid = ntiles < slots ? ntiles : slots;
    }
    kfn<<<grid, nth, smem, s>>>(a, tp, tmap);
    return cuda_fail(cudaGetLastError(), "conv2d tiled launch");
}

template <typename Tin, typename Tout, int K, int PX, int PY, int LOAD, int FILT, int MAP, bool FACC = false>
inline ConvEntry conv_entry(int bx, int by, int persistent) {
    imcl_variant v{};
    v.kind = IMCL_KIND_TILED;
    v.bx = bx;
    v.by = by;
    v.px = PX;
    v.py = PY;
    v.load = LOAD;
    v.filt = FILT;
    v.map = MAP;
    v.unroll = FACC ? IMCL_UNROLL_F32_EXACT : IMCL_UNROLL_FULL;
    v.persistent = persistent;
    return ConvEntry{DtypeOf<Tin>::v, DtypeOf<Tout>::v, K, v,
                     &launch_conv_tiled<Tin, Tout, K, PX, PY, LOAD, FILT, MAP, FACC>};
}

}  // namespace imcl
