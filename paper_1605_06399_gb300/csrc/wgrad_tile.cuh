// wgrad_tile.cuh -- the register-blocked tap-gradient reduction over one staged tile,
// shared by the stand-alone tap-gradient kernel and the ragged batch's backward tiles.
//
//   dw[j][i] += sum_p g(p) x(p + (i - rx, j - ry))   over the tile's pixels p
//
// g is staged as th rows of gsw floats; x as the matching region, its row 0 / column 0
// holding the tile's offset (-rx, -ry), rows of xsw >= wg_xpitch<KW>(tw) floats.  The
// tile splits into 4 x 8 pixel blocks; a thread owns JR consecutive tap rows (j0 ..) and
// all KW columns of them (JR x KW accumulators) and walks blocks lt, lt + T, ...: the
// block's 32 g values stay in registers while the 8 + JR - 1 x rows it meets stream
// through, each feeding every (block row, tap row) pair it serves.  Neighbouring lanes
// take neighbouring blocks, so their 16-byte shared-memory loads are contiguous.
// Per-thread sums run in a fixed order; wgrad_combine adds the threads of each tap-row
// group in a fixed order, so results are deterministic.
#pragma once

#include "tile_common.cuh"

namespace imcl {

constexpr int kWgLx = 4, kWgLy = 8;           // pixels of a thread's block (x, y)

template <int KW>
struct WgCfg {
    // tap rows per thread: JR x KW accumulators (at most 48; 20 for the short rows, whose
    // kernels run three CTAs per SM)
    static constexpr int JR = KW > 15 ? 1 : (KW <= 5 ? 4 : (48 / KW < 8 ? 48 / KW : 8));
    static constexpr int XQ = (kWgLx + KW - 1 + 3) / 4;                    // float4s per x row
};

// x row pitch (floats) a tile of width tw needs: every block's float4 reads stay in the row
template <int KW>
__host__ __device__ constexpr int wg_xpitch(int tw) { return tw - kWgLx + 4 * WgCfg<KW>::XQ; }

// Accumulate the blocks lt, lt + T, ... of a tw x th tile (tw % 4 == 0, th % 8 == 0, gs,
// xs, gsw and xsw 16-byte aligned) into acc, for tap rows j0 .. j0 + JR - 1 (< kh).  D:
// the x region starts D columns further left than the tile's offset -rx (an aligned
// staging origin); a row's reads then start D columns in, loaded from the aligned column
// before them.
template <int KW, int D = 0, int JR = WgCfg<KW>::JR>
__device__ __forceinline__ void wgrad_accumulate(const float* gs, int gsw, const float* xs, int xsw, int tw, int th,
                                                 int kh, int j0, int lt, int T, float (&acc)[JR][KW]) {
    constexpr int XQ = WgCfg<KW>::XQ + (D > 0 ? 1 : 0), LX = kWgLx, LY = kWgLy;
    static_assert(D >= 0 && D < 4, "staging offset within one float4");
    const int BX = tw / LX, NB = BX * (th / LY);
    for (int b = lt; b < NB; b += T) {
        const int by = b / BX, bxx = b - by * BX;
        const int px0 = bxx * LX, py0 = by * LY;
        float gv[LY][LX];
#pragma unroll
        for (int yy = 0; yy < LY; ++yy) {
            const float4 q = *reinterpret_cast<const float4*>(gs + (py0 + yy) * gsw + px0);
            gv[yy][0] = q.x; gv[yy][1] = q.y; gv[yy][2] = q.z; gv[yy][3] = q.w;
        }
        // x row (py0 + r + j0) serves block row yy = r - jr for each tap row jr
#pragma unroll
        for (int r = 0; r < LY + JR - 1; ++r) {
            const bool row_used = r < LY || j0 + (r - LY + 1) < kh;   // some jr < kh with yy = r - jr < LY
            if (row_used) {
                float xv[4 * XQ];
                const float* xr = xs + (py0 + r + j0) * xsw + px0;
#pragma unroll
                for (int q = 0; q < XQ; ++q) {
                    const float4 v = *reinterpret_cast<const float4*>(xr + 4 * q);
                    xv[4 * q] = v.x; xv[4 * q + 1] = v.y; xv[4 * q + 2] = v.z; xv[4 * q + 3] = v.w;
                }
#pragma unroll
                for (int jr = 0; jr < JR; ++jr) {
                    const int yy = r - jr;
                    if (yy >= 0 && yy < LY && j0 + jr < kh) {
#pragma unroll
                        for (int i = 0; i < KW; ++i)
#pragma unroll
                            for (int p = 0; p < LX; ++p) acc[jr][i] = __fmaf_rn(gv[yy][p], xv[D + p + i], acc[jr][i]);
                    }
                }
            }
        }
    }
}

// out[j * KW + i] = sum over the T threads of tap-row group j / JR, in thread order.  red:
// nth * JR * KW floats of shared memory that nothing else uses now.  Ends synchronised.
template <int KW, int JR = WgCfg<KW>::JR>
__device__ void wgrad_combine(const float (&acc)[JR][KW], bool active, float* red, int kh, int T, float* out, int tid,
                              int nth) {
    __syncthreads();
#pragma unroll
    for (int jr = 0; jr < JR; ++jr)
#pragma unroll
        for (int i = 0; i < KW; ++i) red[tid * JR * KW + jr * KW + i] = active ? acc[jr][i] : 0.f;
    __syncthreads();
    for (int q = tid; q < KW * kh; q += nth) {
        const int j = q / KW, i = q - j * KW;
        const int gq = j / JR, jr = j - gq * JR;
        float sum = 0.f;
        for (int r = 0; r < T; ++r) sum += red[(gq * T + r) * JR * KW + jr * KW + i];
        out[q] = sum;
    }
    __syncthreads();
}

// The same sums as wgrad_combine, for kernels that combine once per tile: each tap's T
// partial sums are split over S lanes of one warp (S a power of two, at most 32, as many
// as the block has threads for), each lane adding every S-th of them in order, and the S
// lane sums are added in a fixed shuffle tree.  The order depends only on T, S and the
// block size, so results stay deterministic.  Ends synchronised.
template <int KW, int JR = WgCfg<KW>::JR>
__device__ void wgrad_combine_wide(const float (&acc)[JR][KW], bool active, float* red, int kh, int T, float* out,
                                   int tid, int nth) {
    __syncthreads();
#pragma unroll
    for (int jr = 0; jr < JR; ++jr)
#pragma unroll
        for (int i = 0; i < KW; ++i) red[tid * JR * KW + jr * KW + i] = active ? acc[jr][i] : 0.f;
    __syncthreads();
    const int nq = KW * kh;
    int S = 1;
    while (S < 32 && S * 2 * nq <= nth) S *= 2;
    for (int base = 0; base < nq * S; base += nth) {          // uniform trip count
        const int idx = base + tid, q = idx / S, sub = idx - q * S;
        float sum = 0.f;
        if (q < nq) {
            const int j = q / KW, i = q - j * KW;
            const int gq = j / JR, jr = j - gq * JR;
            for (int r = sub; r < T; r += S) sum += red[(gq * T + r) * JR * KW + jr * KW + i];
        }
        for (int o = S >> 1; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (q < nq && sub == 0) out[q] = sum;
    }
    __syncthreads();
}

}  // namespace imcl
