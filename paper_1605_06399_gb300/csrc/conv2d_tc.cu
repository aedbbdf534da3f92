// conv2d_tc.cu -- the tensor-core variant of the non-separable correlation for large
// filters (sides 9..15): a banded-Toeplitz formulation on tcgen05 MMAs with the
// accumulator in tensor memory.  Compiled once per side with -DIMCL_TC_K=K.
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
// group multiplies the 128 staged rows, shifted down by g J rows, with the J Toeplitz
// matrices of the group side by side (N = 16 J columns), so all groups accumulate into
// one 128 x 16 J tile D[m][(j', n)] = sum_g P_{gJ+j'}[m + gJ][n] in tensor memory.  The
// epilogue adds the J lane-shifted column blocks, y(x0 + n, y0 + m) =
// sum_{j'} D[m + j'][(j', n)], with warp shuffles (and a small shared-memory exchange
// across the four lane quarters), giving 129 - J output rows per 128-row MMA tile.
// Grouping keeps N at 16 J, so each MMA reads its 128 x 32-byte A slice once for at
// least 80 columns of products (shared-memory bandwidth, not the tensor pipe, bounds an
// N = 16 Toeplitz MMA).
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
// Pipeline (one persistent CTA per SM, 384 threads, work units = a band of 129 - J
// output rows x a segment of 16 NB columns):
//   warp 0       TMA producer: 16-column slabs of the 128 + J staged rows, one row-major
//                2D box each, into a ring of eight staging slots (zero fill outside;
//                the ring is deep because a box takes a few microseconds to land);
//   warp 1       allocates the tensor memory and issues the MMAs (one thread): block b
//                of a unit reads operand slabs b and b + 1 (the 32-column K window);
//   warps 2-3    converters: copy a staging slot into the chunk-major operand layout of
//                the MMAs, applying the boundary rule outside the image and, for f32,
//                writing the tf32 high and low parts;
//   warps 4-11   epilogue, two warps per tensor-memory lane quarter (8 output columns
//                each): one load of all J column groups, shifted sums, global stores.
//                The accumulator has four buffers, so the MMAs of the next blocks
//                overlap the epilogue of this one.
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
    static constexpr int N1 = 16 * J;              // accumulator columns: (half ch, row j', column n')
    static constexpr int N2 = 2 * N1;              // B rows: the high tap set, then the low one
    static constexpr int BH = 129 - J;             // output rows per band
    static constexpr int AR = 128 + J;             // staged rows: image rows y0 - R ..
    static constexpr int ARP = (AR + 7) / 8 * 8;   // rows per chunk column (whole core matrices)
    static constexpr int CE = 16 / (int)sizeof(Tin);   // elements per 16-byte chunk
    static constexpr int CPS = 16 / CE;                // chunk columns per 16-column slab
    // chunk columns are 2 (f32) or 4 (16-bit) rows more than whole core matrices apart, so
    // the converters' 16-byte stores of neighbouring rows and chunks fall in distinct banks
    static constexpr int PADR = F32 ? 2 : 4;
    static constexpr int LBO_A = (ARP + PADR) * 16;    // bytes between chunk columns
    static constexpr int SLAB = CPS * LBO_A;           // bytes of one slab (one operand copy)
    static constexpr int KCH = 32 / CE;                // chunks of the 32-element K window
    static constexpr int KSTEP = F32 ? 8 : 16;         // K of one MMA
    static constexpr int NKS = 32 / KSTEP;             // MMAs along K per group and operand pair
    static constexpr int LBO_B = N2 * 16;
    static constexpr int BBYTES = G * KCH * LBO_B;
    static constexpr int S = 4;                        // operand slab ring depth
    static constexpr int SS = 8;                       // staging ring depth: TMA boxes in flight
    static constexpr int STAGE = (AR * 16 * (int)sizeof(Tin) + 127) / 128 * 128;
    static constexpr int NCOPY = F32 ? 2 : 1;          // hi (and lo) copies of a slab
    static constexpr int NBUF = 4;                     // accumulator buffers
    static constexpr int NEPI = 8;                     // epilogue warps
    static constexpr int NT = J * (J - 1) / 2;         // exchange entries per warp
    static constexpr int XBYTES = 2 * NEPI * NT * 8 * 4;
    static constexpr int TMEM_COLS = 512;
    static constexpr int THREADS = 32 * (4 + NEPI);
    static_assert(G * J >= K && N1 <= 256 && NBUF * N1 <= TMEM_COLS, "tensor tile shape");
    static_assert(R <= 7, "the 32-column window holds 16 outputs' taps for R <= 7");
    // shared-memory layout (bytes from the 1024-aligned base)
    static constexpr int OFF_STAGE = 0;
    static constexpr int OFF_A = OFF_STAGE + SS * STAGE;
    static constexpr int OFF_B = OFF_A + NCOPY * S * SLAB;
    static constexpr int OFF_X = OFF_B + BBYTES;
    static constexpr int OFF_BAR = OFF_X + XBYTES;
    static constexpr int NBAR = 2 * SS + 2 * S + 2 * NBUF + 2 + 1;   // sfull, sempty; ready, empty; tfull, tempty; xready; done
    static constexpr int SMEM = OFF_BAR + NBAR * 8 + 16 + 1024;
    static_assert(SMEM <= 232448, "shared memory per CTA");
};

struct TcArgs {
    ConvArgs a;
    int nb;            // 16-column blocks per unit
    int nsegs, units;  // segments per band, units in the grid
};

// The chunk (CE elements) of a slab's chunk column c, row r: byte c LBO_A + r 16.
template <typename G>
__device__ __forceinline__ int slab_off(int c, int r) { return c * G::LBO_A + r * 16; }

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
    constexpr int R = G::R, J = G::J, S = G::S, NBUF = G::NBUF;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // TMA destinations want 128-byte aligned shared addresses: align the base to 1024
    uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const ConvArgs& a = ta.a;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    uint8_t* stage = smem + G::OFF_STAGE;
    uint8_t* a_hi = smem + G::OFF_A;
    uint8_t* a_lo = smem + G::OFF_A + S * G::SLAB;   // f32 only
    uint8_t* bmat = smem + G::OFF_B;
    float* xch = reinterpret_cast<float*>(smem + G::OFF_X);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + G::OFF_BAR);
    uint64_t* sfull = bars;                 // a staging slot holds its TMA box
    uint64_t* sempty = sfull + G::SS;       // the converters have read it
    uint64_t* ready = sempty + G::SS;       // an operand slab is written
    uint64_t* empty = ready + S;            // the MMAs reading an operand slab have completed
    uint64_t* tfull = empty + S;
    uint64_t* tempty = tfull + NBUF;
    uint64_t* xready = tempty + NBUF;
    uint64_t* done = xready + 2;
    uint32_t* tmem_word = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_word + 1);

    if (tid == 0) {
        for (int i = 0; i < G::SS; ++i) {
            mbar_init(&sfull[i], 1);
            mbar_init(&sempty[i], 2);
        }
        for (int i = 0; i < S; ++i) {
            mbar_init(&ready[i], 2);
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
    // within = ch * 8 J + j' * 8 + n' holds output column n = 8 ch + n' of filter row
    // g J + j', so each epilogue warp (column half ch) reads 8 J consecutive accumulator
    // columns.
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
        const int ch = within / (8 * J), jj = (within % (8 * J)) / 8, n = 8 * ch + within % 8;
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
                    const int slot = p % G::SS;
                    if (p >= (uint32_t)G::SS && !mbar_wait(&sempty[slot], ((p / G::SS) - 1) & 1, a.status)) {
                        *abort_flag = 1;
                        break;
                    }
                    // one row-major box: 16 columns x AR rows
                    mbar_arrive_expect_tx(&sfull[slot], G::AR * 16 * (int)sizeof(Tin));
                    tma_load_2d(stage + slot * G::STAGE, &tmap, x0 - 8 + 16 * sl, y0 - R, &sfull[slot]);
                }
            }
            // wait (bounded) for the copies still in flight
            const uint32_t first = p > (uint32_t)G::SS ? p - G::SS : 0;
            for (uint32_t q = first; q < p; ++q) mbar_wait(&sfull[q % G::SS], (q / G::SS) & 1, a.status);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issue
        if (lane == 0) {
            constexpr uint32_t fmt = G::F32 ? UMMA_TF32 : (std::is_same<Tin, __half>::value ? UMMA_F16 : UMMA_BF16);
            const uint32_t idesc = umma_idesc(fmt, 128, G::N1);
            const uint32_t a_hi_s = smem_u32(a_hi), a_lo_s = smem_u32(a_lo), b_s = smem_u32(bmat);
            uint32_t p = 0, q = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < ta.units && ok && !*abort_flag; u += gridDim.x) {
                int x0, y0, nbu;
                unit_geo(u, x0, y0, nbu);
                if (!mbar_wait(&ready[p % S], (p / S) & 1, a.status)) { ok = false; break; }
                for (int b = 0; b < nbu; ++b, ++q) {
                    const uint32_t pn = p + b + 1;
                    if (!mbar_wait(&ready[pn % S], (pn / S) & 1, a.status)) { ok = false; break; }
                    const int buf = q % NBUF;
                    if (q >= (uint32_t)NBUF && !mbar_wait(&tempty[buf], ((q / NBUF) - 1) & 1, a.status)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem_base + buf * G::N1;
#pragma unroll
                    for (int g = 0; g < G::G; ++g) {
#pragma unroll
                        for (int ks = 0; ks < G::NKS; ++ks) {
                            const int sidx = G::F32 ? b + ks / 2 : b + ks;
                            const int chunk0 = G::F32 ? (ks % 2) * 2 : 0;
                            const uint32_t slot = (p + sidx) % S;
                            const uint32_t aoff = slot * G::SLAB + chunk0 * G::LBO_A + g * J * 16;
                            const uint32_t boff = b_s + (g * G::KCH + ks * 2) * G::LBO_B;
                            const uint64_t b_hi = umma_smem_desc(boff, G::LBO_B, 128);
                            const uint64_t b_lo = umma_smem_desc(boff + G::N1 * 16, G::LBO_B, 128);
                            const uint64_t a_h = umma_smem_desc(a_hi_s + aoff, G::LBO_A, 128);
                            const uint32_t acc = (g | ks) != 0;
                            if constexpr (G::F32) {
                                const uint64_t a_l = umma_smem_desc(a_lo_s + aoff, G::LBO_A, 128);
                                umma_tf32(d, a_h, b_hi, idesc, acc);
                                umma_tf32(d, a_h, b_lo, idesc, 1u);
                                umma_tf32(d, a_l, b_hi, idesc, 1u);
                            } else {
                                umma_f16(d, a_h, b_hi, idesc, acc);
                                umma_f16(d, a_h, b_lo, idesc, 1u);
                            }
                        }
                    }
                    umma_commit(&tfull[buf]);
                    umma_commit(&empty[(p + b) % S]);
                }
                if (!ok) break;
                umma_commit(&empty[(p + nbu) % S]);
                p += nbu + 1;
            }
            if (!ok) *abort_flag = 1;
            umma_commit(done);
            mbar_wait(done, 0, a.status);
        }
    } else if (warp < 4) {
        // ------------------------------------------------------------ converters
        // staging slot (row-major, 16 elements a row) -> operand slab (chunk-major), with
        // the boundary rule on pixels outside the image and, for f32, the tf32 split
        const int ct = tid - 64;
        const Tin bv = border_pixel<Tin>(a);
        const Tin* in = static_cast<const Tin*>(a.in);
        uint32_t p = 0;
        for (int u = blockIdx.x; u < ta.units && !__any_sync(0xffffffffu, *abort_flag); u += gridDim.x) {
            int x0, y0, nbu;
            unit_geo(u, x0, y0, nbu);
            for (int sl = 0; sl <= nbu; ++sl, ++p) {
                const int slot = p % S, ss = p % G::SS;
                if (!warp_wait(&sfull[ss], (p / G::SS) & 1, a.status) ||
                    (p >= (uint32_t)S && !warp_wait(&empty[slot], ((p / S) - 1) & 1, a.status))) {
                    *abort_flag = 1;
                    break;
                }
                const int xs = x0 - 8 + 16 * sl, ys = y0 - R;
                const bool inside = xs >= 0 && xs + 16 <= W && ys >= 0 && ys + G::AR <= H;
                const uint8_t* st = stage + ss * G::STAGE;
                uint8_t* hi = a_hi + slot * G::SLAB;
                // four 16-byte chunks per thread in flight: loads first, then the conversions
                constexpr int TOT = G::CPS * G::AR;
                for (int i0 = ct; i0 < TOT; i0 += 4 * 64) {
                    uint4 raw[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        if (i0 + 64 * t < TOT) raw[t] = *reinterpret_cast<const uint4*>(st + (i0 + 64 * t) * 16);
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int idx = i0 + 64 * t;
                        if (idx >= TOT) break;
                        const int r = idx / G::CPS, c = idx % G::CPS;
                        if (!inside) {
                            Tin* e = reinterpret_cast<Tin*>(&raw[t]);
                            const int gy = ys + r;
#pragma unroll
                            for (int q = 0; q < G::CE; ++q) {
                                const int gx = xs + G::CE * c + q;
                                if (gx < 0 || gx >= W || gy < 0 || gy >= H)
                                    e[q] = a.border == IMCL_BORDER_CONSTANT
                                               ? bv
                                               : in[(long long)clampi(gy, 0, H - 1) * a.in_pitch + clampi(gx, 0, W - 1)];
                            }
                        }
                        if constexpr (G::F32) {
                            const uint4 v = raw[t];
                            uint4 h, l;
                            h.x = tf32_part(__uint_as_float(v.x));
                            h.y = tf32_part(__uint_as_float(v.y));
                            h.z = tf32_part(__uint_as_float(v.z));
                            h.w = tf32_part(__uint_as_float(v.w));
                            l.x = tf32_part(__uint_as_float(v.x) - __uint_as_float(h.x));
                            l.y = tf32_part(__uint_as_float(v.y) - __uint_as_float(h.y));
                            l.z = tf32_part(__uint_as_float(v.z) - __uint_as_float(h.z));
                            l.w = tf32_part(__uint_as_float(v.w) - __uint_as_float(h.w));
                            *reinterpret_cast<uint4*>(hi + slab_off<G>(c, r)) = h;
                            *reinterpret_cast<uint4*>(a_lo + slot * G::SLAB + slab_off<G>(c, r)) = l;
                        } else {
                            *reinterpret_cast<uint4*>(hi + slab_off<G>(c, r)) = raw[t];
                        }
                    }
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive1(&ready[slot]);
                    mbar_arrive1(&sempty[ss]);
                }
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int ew = warp - 4;                 // epilogue warp 0..7
        const int eq = ew & 3, ch = ew >> 2;     // TMEM lane quarter, column half
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
                float v[8 * J];
                tmem_ld8xJ<J>(tmem_base + ((uint32_t)(32 * eq) << 16) + buf * G::N1 + ch * 8 * J, v);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive1(&tempty[buf]);
                float acc[8];
#pragma unroll
                for (int n = 0; n < 8; ++n) acc[n] = v[n];
                float* xw = xch + (xb * G::NEPI + ew) * G::NT * 8;
#pragma unroll
                for (int jj = 1; jj < J; ++jj) {
                    if (lane < jj) {   // rows the warp of the next lane quarter needs
                        float4* dst = reinterpret_cast<float4*>(xw + (jj * (jj - 1) / 2 + lane) * 8);
                        dst[0] = make_float4(v[8 * jj], v[8 * jj + 1], v[8 * jj + 2], v[8 * jj + 3]);
                        dst[1] = make_float4(v[8 * jj + 4], v[8 * jj + 5], v[8 * jj + 6], v[8 * jj + 7]);
                    }
                    const bool mine = lane + jj < 32;
#pragma unroll
                    for (int n = 0; n < 8; ++n) {
                        const float t = __shfl_down_sync(0xffffffffu, v[8 * jj + n], jj);
                        if (mine) acc[n] += t;
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive1(&xready[xb]);
                if (!warp_wait(&xready[xb], (q / 2) & 1, a.status)) { ok = false; break; }
                if (eq < 3) {   // rows m + j' past this quarter: the next quarter's first lanes
                    const float* xn = xch + (xb * G::NEPI + ew + 1) * G::NT * 8;
#pragma unroll
                    for (int jj = 1; jj < J; ++jj) {
                        if (lane + jj >= 32) {
                            const float4* src = reinterpret_cast<const float4*>(xn + (jj * (jj - 1) / 2 + lane + jj - 32) * 8);
                            const float4 t0 = src[0], t1 = src[1];
                            acc[0] += t0.x;
                            acc[1] += t0.y;
                            acc[2] += t0.z;
                            acc[3] += t0.w;
                            acc[4] += t1.x;
                            acc[5] += t1.y;
                            acc[6] += t1.z;
                            acc[7] += t1.w;
                        }
                    }
                }
                if constexpr (std::is_same<Tin, __half>::value) {
#pragma unroll
                    for (int n = 0; n < 8; ++n) acc[n] *= inv_scale;
                }
                const int gy = y0 + m, gx = x0 + 16 * b + 8 * ch;
                if (m < G::BH && gy < H) store_block_row<Tout, 8>(out, a.out_pitch, gx, gy, W, H, a.vec_out, acc);
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
