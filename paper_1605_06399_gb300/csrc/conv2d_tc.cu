// conv2d_tc.cu -- the tensor-core variant of the non-separable correlation for large
// filters (sides 9..15): a banded-Toeplitz formulation on tcgen05 MMAs with the image
// operand and the accumulator in tensor memory.  Compiled once per side with
// -DIMCL_TC_K=K.
//
// The correlation y(x, y) = sum_{j,i} w[j][i] in(x + i - R, y + j - R) of §6's
// non-separable benchmark is, for one filter row j and a block of 16 output columns, a
// product of the input rows with a banded Toeplitz matrix T_j (32 x 16, T_j[k][n] =
// w[j][k - n - 8 + R] inside the band, 0 outside):
//
//     P_j[r][n] = sum_k A[r][k] T_j[k][n],   A[r][k] = in(x0 - 8 + k, y0 - R + r)
//     y(x0 + n, y0 + m) = sum_j P_j[m + j][n].
//
// The filter rows are split into G = 2 groups of J = (K + 1) / 2 rows.  One MMA of a
// group multiplies 128 staged rows (shifted down by g J rows) with the J Toeplitz
// matrices of the group side by side (N = 16 J columns), so both groups accumulate into
// one 128 x 16 J tile D[m][(j', n)] = sum_g P_{gJ+j'}[m + gJ][n] in tensor memory.  The
// epilogue adds the J lane-shifted column blocks, y(x0 + n, y0 + m) =
// sum_{j'} D[m + j'][(j', n)], with warp shuffles (and a small shared-memory exchange
// across the four lane quarters), giving 129 - J output rows per 128-row MMA tile.
//
// The image operand A lives in tensor memory: each converter warp writes, for its
// quarter of the 128 lanes, the rows of both groups (lane m holds staged row m + g J of
// copy g), so the MMAs read only the Toeplitz operand B from shared memory.  Reading A
// from shared memory as well (128 x 32 bytes per MMA) kept an earlier form of this
// kernel at the shared-memory bandwidth.
//
// Precision.  f16 / bf16 images are exact MMA operands; the taps are split into a high
// and a low part of the same type (f16 taps are scaled by a power of two first so both
// parts stay normal), and A T_hi and A T_lo accumulate into the same columns: each
// product carries about 2^-17 relative error.  f32 images use the tf32 kind with both
// operands split into tf32 high and low parts (x = x_hi + x_lo, truncated so that each
// part is exactly a tf32 value) and three MMAs, x_hi w_hi + x_hi w_lo + x_lo w_hi: a
// relative error below 3 * 2^-20 per product, the dropped x_lo w_lo term included.  Both
// stay inside the 1e-5 scaled tolerance of the f32 results.
//
// Pipeline (one persistent CTA per SM, 704 threads, work units = a band of 129 - J
// output rows x a segment of 16 NB columns):
//   warp 0       TMA producer: 16-column slabs of the 128 + J staged rows, one row-major
//                2D box each, into a ring of eight staging slots (zero fill outside;
//                the ring is deep because a box takes a few microseconds to land);
//   warp 1       allocates the tensor memory and issues the MMAs (one thread): block b
//                of a unit reads A slabs b and b + 1 (the 32-column K window);
//   warps 2-5    converters, one per tensor-memory lane quarter: staging slot -> A slab
//                in tensor memory, with the boundary rule outside the image and, for
//                f32, the tf32 high and low parts;
//   warps 6-21   epilogue, four warps per lane quarter (4 output columns each): tensor
//                memory -> shifted sums -> global stores, while the MMAs of the next
//                blocks fill the other accumulator buffers.
// Every wait is bounded (the device status word records a timeout); the tensor memory
// is released on every path.
#include "conv2d_kernels.cuh"
#include "tcgen05.cuh"

#if !defined(IMCL_TC_K)
#error "compile with -DIMCL_TC_K=<odd side 9..15>"
#endif

#define IMCL_CAT2(a, b) a##b
#define IMCL_CAT(a, b) IMCL_CAT2(a, b)
#define IMCL_TC_REG_NAME IMCL_CAT(register_conv_tc_k, IMCL_TC_K)

namespace imcl {

template <typename Tin, int K>
struct TcGeo {
    static constexpr bool F32 = std::is_same<Tin, float>::value;
    static constexpr int R = (K - 1) / 2;
    static constexpr int J = (K + 1) / 2;          // filter rows per group
    static constexpr int G = 2;                    // groups, G J >= K
    static constexpr int N1 = 16 * J;              // accumulator columns: (quarter ch, row j', column n')
    static constexpr int N2 = 2 * N1;              // B rows: the high tap set, then the low one
    static constexpr int BH = 129 - J;             // output rows per band
    static constexpr int AR = 128 + J;             // staged rows: image rows y0 - R ..
    static constexpr int ESZ = (int)sizeof(Tin);
    static constexpr int CE = 16 / ESZ;            // elements per 16-byte chunk (B layout)
    static constexpr int KCH = 32 / CE;            // chunks of the 32-element K window
    static constexpr int KSTEP = F32 ? 8 : 16;     // K of one MMA
    static constexpr int NKS = 32 / KSTEP;         // MMAs along K per group and operand pair
    static constexpr int LBO_B = N2 * 16;
    static constexpr int BBYTES = G * KCH * LBO_B;
    static constexpr int SS = 8;                   // staging ring depth: TMA boxes in flight
    static constexpr int STAGE = (AR * 16 * ESZ + 127) / 128 * 128;
    // tensor memory: an A ring of ST slabs, then the accumulator buffers
    static constexpr int ST = 4;                   // A slabs in tensor memory
    static constexpr int SCOL = 16 * ESZ / 4;      // 32-bit columns of 16 elements (16 or 8)
    static constexpr int NCOPY = F32 ? 4 : 2;      // copies per slab: (hi, lo) x group, or group
    static constexpr int ACOLS = NCOPY * SCOL;     // columns of one A slab
    static constexpr int TMEM_COLS = 512;
    static constexpr int NBUF0 = (TMEM_COLS - ST * ACOLS) / N1;
    static constexpr int NBUF = NBUF0 > 4 ? 4 : NBUF0;   // accumulator buffers
    static constexpr int ACC0 = ST * ACOLS;        // first accumulator column
    static constexpr int NEPI = 16;                // epilogue warps (four per lane quarter)
    static constexpr int NCONV = 4;                // converter warps (one per lane quarter)
    static constexpr int NT = J * (J - 1) / 2;     // exchange entries per warp
    static constexpr int XBYTES = 2 * NEPI * NT * 4 * 4;
    static constexpr int THREADS = 32 * (2 + NCONV + NEPI);
    static_assert(G * J >= K && N1 <= 256 && NBUF >= 2, "tensor tile shape");
    static_assert(R <= 7, "the 32-column window holds 16 outputs' taps for R <= 7");
    // shared-memory layout (bytes from the 1024-aligned base)
    static constexpr int OFF_STAGE = 0;
    static constexpr int OFF_B = OFF_STAGE + SS * STAGE;
    static constexpr int OFF_X = OFF_B + BBYTES;
    static constexpr int OFF_BAR = OFF_X + XBYTES;
    static constexpr int NBAR = 2 * SS + 2 * ST + 2 * NBUF + 2 + 1;   // sfull, sempty; ready, empty; tfull, tempty; xready; done
    static constexpr int SMEM = OFF_BAR + NBAR * 8 + 16 + 1024;
    static_assert(SMEM <= 232448, "shared memory per CTA");
};

struct TcArgs {
    ConvArgs a;
    int nb;            // 16-column blocks per unit
    int nsegs, units;  // segments per band, units in the grid
};

__device__ __forceinline__ uint32_t tf32_part(float v) { return __float_as_uint(v) & 0xFFFFE000u; }

// A wait every lane of the warp takes; all lanes see the same outcome, so a timeout never
// splits the warp before its warp-wide instructions.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, int* status) {
    return __all_sync(0xffffffffu, mbar_wait(bar, parity, status));
}

__device__ __forceinline__ void mbar_arrive1(uint64_t* bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
                 : "memory");
}

template <typename Tin, typename Tout, int K>
__global__ void __launch_bounds__(TcGeo<Tin, K>::THREADS, 1)
    k_conv2d_tc(const TcArgs ta, const __grid_constant__ TapsParam<float, K * K> tp,
                const __grid_constant__ CUtensorMap tmap) {
    using G = TcGeo<Tin, K>;
    constexpr int R = G::R, J = G::J, ST = G::ST, SS = G::SS, NBUF = G::NBUF;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // TMA destinations want 128-byte aligned shared addresses: align the base to 1024
    uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const ConvArgs& a = ta.a;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    uint8_t* stage = smem + G::OFF_STAGE;
    uint8_t* bmat = smem + G::OFF_B;
    float* xch = reinterpret_cast<float*>(smem + G::OFF_X);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + G::OFF_BAR);
    uint64_t* sfull = bars;                 // a staging slot holds its TMA box
    uint64_t* sempty = sfull + SS;          // the converters have read it
    uint64_t* ready = sempty + SS;          // an A slab is written to tensor memory
    uint64_t* empty = ready + ST;           // the MMAs reading an A slab have completed
    uint64_t* tfull = empty + ST;           // an accumulator buffer holds a finished block
    uint64_t* tempty = tfull + NBUF;        // the epilogue has read it
    uint64_t* xready = tempty + NBUF;       // the epilogue's cross-quarter rows are written
    uint64_t* done = xready + 2;
    uint32_t* tmem_word = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_word + 1);

    if (tid == 0) {
        for (int i = 0; i < SS; ++i) {
            mbar_init(&sfull[i], 1);
            mbar_init(&sempty[i], G::NCONV);
        }
        for (int i = 0; i < ST; ++i) {
            mbar_init(&ready[i], G::NCONV);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < NBUF; ++i) {
            mbar_init(&tfull[i], 1);
            mbar_init(&tempty[i], G::NEPI);
        }
        for (int i = 0; i < 2; ++i) mbar_init(&xready[i], G::NEPI);
        mbar_init(done, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(tmem_word, G::TMEM_COLS);
        tmem_relinquish();
    }

    // The Toeplitz operand B[(g, chunk c)][row][e], K-major, rows = half * N1 + within:
    // within = ch * 4 J + j' * 4 + n' holds output column n = 4 ch + n' of filter row
    // g J + j', so each epilogue warp (column quarter ch) reads 4 J consecutive
    // accumulator columns.
    const float* taps = a.taps_dev ? static_cast<const float*>(a.taps_dev) : tp.w;
    float scale = 1.f, inv_scale = 1.f;
    if constexpr (std::is_same<Tin, __half>::value) {
        // f16 taps: a power of two that puts the largest tap in [2^13, 2^14)
        float wmax = 0.f;
        for (int i = 0; i < K * K; ++i) wmax = fmaxf(wmax, fabsf(taps[i]));
        if (wmax > 0.f) {
            int e;
            frexpf(wmax, &e);
            scale = ldexpf(1.f, 14 - e);
            inv_scale = ldexpf(1.f, e - 14);
        }
    }
    constexpr int BELEMS = G::G * G::KCH * G::N2 * G::CE;
    for (int idx = tid; idx < BELEMS; idx += blockDim.x) {
        const int e = idx % G::CE;
        const int row = (idx / G::CE) % G::N2;
        const int gc = idx / (G::CE * G::N2);          // g * KCH + c
        const int g = gc / G::KCH, c = gc % G::KCH;
        const int k = c * G::CE + e;
        const int half = row / G::N1, within = row % G::N1;
        const int ch = within / (4 * J), jj = (within % (4 * J)) / 4, n = 4 * ch + within % 4;
        const int j = g * J + jj, i = k - n - (8 - R);
        const float w = (j < K && i >= 0 && i < K) ? taps[j * K + i] : 0.f;
        uint8_t* dst = bmat + gc * G::LBO_B + row * 16;
        if constexpr (G::F32) {
            const uint32_t hi = tf32_part(w);
            const uint32_t lo = tf32_part(w - __uint_as_float(hi));
            reinterpret_cast<uint32_t*>(dst)[e] = half ? lo : hi;
        } else {
            const float ws = w * scale;
            const Tin hi = Store<Tin, float>::cvt(ws);
            const Tin lo = Store<Tin, float>::cvt(ws - to_acc(hi));
            reinterpret_cast<Tin*>(dst)[e] = half ? lo : hi;
        }
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_word;

    const int W = a.W, H = a.H;
    const int nb_full = ta.nb;
    auto unit_geo = [&](int u, int& x0, int& y0, int& nbu) {
        const int band = u / ta.nsegs, seg = u % ta.nsegs;
        y0 = band * G::BH;
        x0 = seg * 16 * nb_full;
        const int rem = (W - x0 + 15) / 16;
        nbu = rem < nb_full ? rem : nb_full;
    };

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            prefetch_tmap(&tmap);
            uint32_t p = 0;
            for (int u = blockIdx.x; u < ta.units && !*abort_flag; u += gridDim.x) {
                int x0, y0, nbu;
                unit_geo(u, x0, y0, nbu);
                for (int sl = 0; sl <= nbu; ++sl, ++p) {
                    const int slot = p % SS;
                    if (p >= (uint32_t)SS && !mbar_wait(&sempty[slot], ((p / SS) - 1) & 1, a.status)) {
                        *abort_flag = 1;
                        break;
                    }
                    // one row-major box: 16 columns x AR rows
                    mbar_arrive_expect_tx(&sfull[slot], G::AR * 16 * G::ESZ);
                    tma_load_2d(stage + slot * G::STAGE, &tmap, x0 - 8 + 16 * sl, y0 - R, &sfull[slot]);
                }
            }
            // wait (bounded) for the copies still in flight
            const uint32_t first = p > (uint32_t)SS ? p - SS : 0;
            for (uint32_t q = first; q < p; ++q) mbar_wait(&sfull[q % SS], (q / SS) & 1, a.status);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issue
        if (lane == 0) {
            constexpr uint32_t fmt = G::F32 ? UMMA_TF32 : (std::is_same<Tin, __half>::value ? UMMA_F16 : UMMA_BF16);
            const uint32_t idesc = umma_idesc(fmt, 128, G::N1);
            const uint32_t b_s = smem_u32(bmat);
            uint32_t p = 0, q = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < ta.units && ok && !*abort_flag; u += gridDim.x) {
                int x0, y0, nbu;
                unit_geo(u, x0, y0, nbu);
                if (!mbar_wait(&ready[p % ST], (p / ST) & 1, a.status)) { ok = false; break; }
                for (int b = 0; b < nbu; ++b, ++q) {
                    const uint32_t pn = p + b + 1;
                    if (!mbar_wait(&ready[pn % ST], (pn / ST) & 1, a.status)) { ok = false; break; }
                    const int buf = q % NBUF;
                    if (q >= (uint32_t)NBUF && !mbar_wait(&tempty[buf], ((q / NBUF) - 1) & 1, a.status)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem_base + G::ACC0 + buf * G::N1;
#pragma unroll
                    for (int g = 0; g < G::G; ++g) {
#pragma unroll
                        for (int ks = 0; ks < G::NKS; ++ks) {
                            // K step ks: slab b + ks (16-bit) or columns 8 (ks % 2) of slab b + ks / 2 (f32)
                            const int sidx = G::F32 ? b + ks / 2 : b + ks;
                            const uint32_t a0 = tmem_base + ((p + sidx) % ST) * G::ACOLS + (G::F32 ? (ks % 2) * 8 : 0);
                            const uint32_t boff = b_s + (g * G::KCH + ks * 2) * G::LBO_B;
                            const uint64_t b_hi = umma_smem_desc(boff, G::LBO_B, 128);
                            const uint64_t b_lo = umma_smem_desc(boff + G::N1 * 16, G::LBO_B, 128);
                            const uint32_t acc = (g | ks) != 0;
                            if constexpr (G::F32) {
                                const uint32_t a_h = a0 + g * G::SCOL, a_l = a0 + (2 + g) * G::SCOL;
                                umma_tf32_ta(d, a_h, b_hi, idesc, acc);
                                umma_tf32_ta(d, a_h, b_lo, idesc, 1u);
                                umma_tf32_ta(d, a_l, b_hi, idesc, 1u);
                            } else {
                                const uint32_t a_g = a0 + g * G::SCOL;
                                umma_f16_ta(d, a_g, b_hi, idesc, acc);
                                umma_f16_ta(d, a_g, b_lo, idesc, 1u);
                            }
                        }
                    }
                    umma_commit(&tfull[buf]);
                    umma_commit(&empty[(p + b) % ST]);
                }
                if (!ok) break;
                umma_commit(&empty[(p + nbu) % ST]);
                p += nbu + 1;
            }
            if (!ok) *abort_flag = 1;
            umma_commit(done);
            mbar_wait(done, 0, a.status);
        }
    } else if (warp < 2 + G::NCONV) {
        // ------------------------------------------------------------ converters
        // staging slot (row-major, 16 elements a row) -> A slab in tensor memory: lane m of
        // this warp's quarter gets staged row m + g J as copy g (f32: copies g and 2 + g
        // hold the tf32 high and low parts), with the boundary rule outside the image
        const int cq = warp & 3;
        const int m = 32 * cq + lane;
        const uint32_t tq = tmem_base + ((uint32_t)(32 * cq) << 16);
        const Tin bv = border_pixel<Tin>(a);
        const Tin* in = static_cast<const Tin*>(a.in);
        uint32_t p = 0;
        for (int u = blockIdx.x; u < ta.units && !__any_sync(0xffffffffu, *abort_flag); u += gridDim.x) {
            int x0, y0, nbu;
            unit_geo(u, x0, y0, nbu);
            for (int sl = 0; sl <= nbu; ++sl, ++p) {
                const int slot = p % ST, ss = p % SS;
                if (!warp_wait(&sfull[ss], (p / SS) & 1, a.status) ||
                    (p >= (uint32_t)ST && !warp_wait(&empty[slot], ((p / ST) - 1) & 1, a.status))) {
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const int xs = x0 - 8 + 16 * sl, ys = y0 - R;
                const bool inside = xs >= 0 && xs + 16 <= W && ys >= 0 && ys + G::AR <= H;
                const uint8_t* st = stage + ss * G::STAGE;
#pragma unroll
                for (int g = 0; g < G::G; ++g) {
                    const int r = m + g * J;
                    uint4 raw[G::ESZ];   // the row's 16 elements: 4 (f32) or 2 (16-bit) chunks
#pragma unroll
                    for (int c = 0; c < G::ESZ; ++c) raw[c] = *reinterpret_cast<const uint4*>(st + r * 16 * G::ESZ + c * 16);
                    Tin* e = reinterpret_cast<Tin*>(raw);
                    if (!inside) {
                        const int gy = ys + r;
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            const int gx = xs + q;
                            if (gx < 0 || gx >= W || gy < 0 || gy >= H)
                                e[q] = a.border == IMCL_BORDER_CONSTANT
                                           ? bv
                                           : in[(long long)clampi(gy, 0, H - 1) * a.in_pitch + clampi(gx, 0, W - 1)];
                        }
                    }
                    const uint32_t* wv = reinterpret_cast<const uint32_t*>(raw);
                    if constexpr (G::F32) {
#pragma unroll
                        for (int hf = 0; hf < 2; ++hf) {   // two halves of 8 columns keep the registers low
                            uint32_t h[8], l[8];
#pragma unroll
                            for (int q = 0; q < 8; ++q) {
                                const float x = __uint_as_float(wv[8 * hf + q]);
                                h[q] = tf32_part(x);
                                l[q] = tf32_part(x - __uint_as_float(h[q]));
                            }
                            tmem_st8(tq + slot * G::ACOLS + g * G::SCOL + 8 * hf, h);
                            tmem_st8(tq + slot * G::ACOLS + (2 + g) * G::SCOL + 8 * hf, l);
                        }
                    } else {
                        tmem_st8(tq + slot * G::ACOLS + g * G::SCOL, wv);
                    }
                }
                tmem_wait_st();
                fence_proxy_async_smem();   // the staging slot is refilled by TMA after this
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive1(&ready[slot]);
                    mbar_arrive1(&sempty[ss]);
                }
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int ew = warp - 2 - G::NCONV;      // epilogue warp 0..15
        const int eq = warp & 3, ch = ew >> 2;   // TMEM lane quarter, output column quarter
        const int xi = ch * 4 + eq;              // exchange slot of (column quarter, lane quarter)
        const int m = 32 * eq + lane;            // accumulator row of this thread
        Tout* out = static_cast<Tout*>(a.out);
        uint32_t q = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < ta.units && ok && !__any_sync(0xffffffffu, *abort_flag); u += gridDim.x) {
            int x0, y0, nbu;
            unit_geo(u, x0, y0, nbu);
            for (int b = 0; b < nbu; ++b, ++q) {
                const int buf = q % NBUF, xb = q & 1;
                if (!warp_wait(&tfull[buf], (q / NBUF) & 1, a.status)) { ok = false; break; }
                tc_fence_after();
                float v[4 * J];   // v[4 j' + n']: filter row j', output column 4 ch + n'
                tmem_ld4xJ<J>(tmem_base + ((uint32_t)(32 * eq) << 16) + G::ACC0 + buf * G::N1 + ch * 4 * J, v);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive1(&tempty[buf]);
                float acc[4] = {v[0], v[1], v[2], v[3]};
                float4* xw = reinterpret_cast<float4*>(xch) + (xb * G::NEPI + xi) * G::NT;
#pragma unroll
                for (int jj = 1; jj < J; ++jj) {
                    if (lane < jj)   // rows the warp of the next lane quarter needs
                        xw[jj * (jj - 1) / 2 + lane] = make_float4(v[4 * jj], v[4 * jj + 1], v[4 * jj + 2], v[4 * jj + 3]);
                    const bool mine = lane + jj < 32;
#pragma unroll
                    for (int n = 0; n < 4; ++n) {
                        const float t = __shfl_down_sync(0xffffffffu, v[4 * jj + n], jj);
                        if (mine) acc[n] += t;
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive1(&xready[xb]);
                if (!warp_wait(&xready[xb], (q / 2) & 1, a.status)) { ok = false; break; }
                if (eq < 3) {   // rows m + j' past this quarter: the next quarter's first lanes
                    const float4* xn = reinterpret_cast<const float4*>(xch) + (xb * G::NEPI + xi + 1) * G::NT;
#pragma unroll
                    for (int jj = 1; jj < J; ++jj) {
                        if (lane + jj >= 32) {
                            const float4 t = xn[jj * (jj - 1) / 2 + lane + jj - 32];
                            acc[0] += t.x;
                            acc[1] += t.y;
                            acc[2] += t.z;
                            acc[3] += t.w;
                        }
                    }
                }
                if constexpr (std::is_same<Tin, __half>::value) {
#pragma unroll
                    for (int n = 0; n < 4; ++n) acc[n] *= inv_scale;
                }
                const int gy = y0 + m, gx = x0 + 16 * b + 4 * ch;
                if (m < G::BH && gy < H) store_block_row<Tout, 4>(out, a.out_pitch, gx, gy, W, H, a.vec_out, acc);
            }
        }
        if (!ok) *abort_flag = 1;
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, G::TMEM_COLS);
    }
}

template <typename Tin, typename Tout, int K>
imcl_status launch_conv_tc(const ConvCall& c, const imcl_variant& v, cudaStream_t s) {
    using G = TcGeo<Tin, K>;
    if (c.kw != K || c.kh != K) return fail(IMCL_ERR_UNSUPPORTED, "tensor-core conv2d: filter side mismatch");
    if ((reinterpret_cast<uintptr_t>(c.in) & 15) || (c.in_pitch_b & 15))
        return fail(IMCL_ERR_ALIGN, "tensor-core conv2d: TMA staging needs a 16-byte aligned input and pitch");
    const int nb = v.bx > 0 ? v.bx : 8;
    if (nb > 64) return fail(IMCL_ERR_UNSUPPORTED, "tensor-core conv2d: at most 64 column blocks per unit");
    // at least half of the SM's shared memory, so one CTA (and one tensor-memory
    // allocation of 512 columns) per SM
    const int smem = G::SMEM > 116 * 1024 ? G::SMEM : 116 * 1024;
    if (smem > c.dev->max_smem_optin) return fail(IMCL_ERR_UNSUPPORTED, "tensor-core conv2d: shared memory");
    auto kfn = k_conv2d_tc<Tin, Tout, K>;
    imcl_status st = set_smem_limit((const void*)kfn, smem);
    if (st != IMCL_OK) return st;
    CUtensorMap tmap;
    memset(&tmap, 0, sizeof tmap);
    st = encode_tmap_2d(&tmap, c.in_dtype, c.in, c.W, c.H, c.in_pitch_b, 16, G::AR);   // one slab per box
    if (st != IMCL_OK) return st;
    TcArgs ta;
    ta.a = make_conv_args(c, v, 16, 16);
    ta.nb = nb;
    ta.nsegs = (c.W + 16 * nb - 1) / (16 * nb);
    const long long units = (long long)ta.nsegs * ((c.H + G::BH - 1) / G::BH);
    if (units > (1ll << 30)) return fail(IMCL_ERR_UNSUPPORTED, "tensor-core conv2d: image too large");
    ta.units = (int)units;
    TapsParam<float, K * K> tp;
    for (int i = 0; i < K * K; ++i) tp.w[i] = 0.f;
    if (c.taps_mem == IMCL_MEM_HOST)
        for (int i = 0; i < K * K; ++i) tp.w[i] = static_cast<const float*>(c.taps)[i];
    const int grid = ta.units < c.dev->sm_count ? ta.units : c.dev->sm_count;
    kfn<<<grid, G::THREADS, smem, s>>>(ta, tp, tmap);
    return cuda_fail(cudaGetLastError(), "tensor-core conv2d launch");
}

template <typename Tin, typename Tout>
static ConvEntry tc_entry() {
    imcl_variant v{};
    v.kind = IMCL_KIND_TENSOR;
    v.bx = 8;    // 16-column blocks per work unit
    v.by = 1;
    v.px = 16;
    v.py = TcGeo<Tin, IMCL_TC_K>::BH;
    v.load = IMCL_LOAD_TMA;
    v.filt = IMCL_FILT_SMEM;
    v.map = IMCL_MAP_BLOCKED;
    v.unroll = 1;
    v.persistent = 1;
    return ConvEntry{DtypeOf<Tin>::v, DtypeOf<Tout>::v, IMCL_TC_K, v, &launch_conv_tc<Tin, Tout, IMCL_TC_K>};
}

void IMCL_TC_REG_NAME(std::vector<ConvEntry>& t) {
    t.push_back(tc_entry<float, float>());
    t.push_back(tc_entry<__half, float>());
    t.push_back(tc_entry<__half, __half>());
    t.push_back(tc_entry<__nv_bfloat16, float>());
    t.push_back(tc_entry<__nv_bfloat16, __nv_bfloat16>());
}

}  // namespace imcl
