/*
 * imagecl_oracle.c -- plain CPU oracle for the per-pixel stencil operators.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU
 * baseline call this code; the CUDA library never does, and the two share no source.
 *
 * Every function is the definition written out as loops, accumulating in double
 * (floating point) or int64 (integers).  OpenMP splits independent output rows across
 * threads; each output is still summed by one thread in a fixed order.
 *
 * Conventions (from the paper's language description, §5):
 *  - One logical thread per output pixel (idx, idy) = (x, y); x is the contiguous axis
 *    and images are row-major, x fastest (§5.1: images become 1D arrays).
 *  - Listing 1 reads in[idx + i][idy + j] with no filter flip: the operators are
 *    correlations.  For an odd side K the taps are centred: offset = tap - (K-1)/2.
 *  - Filters are row-major, w[j*kw + i] with j the row (dy) and i the column (dx).
 *  - Boundary conditions (§5, Fig. 3): clamped (out-of-image reads return the closest
 *    pixel inside, each coordinate clamped on its own) or constant (out-of-image
 *    reads return a constant).
 *  - Multi-stage operators apply the boundary rule to each stage's own input.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_BORDER_CLAMP 0
#define ORA_BORDER_CONSTANT 1

/* Threads the parallel loops use (1 without OpenMP). */
int ora_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int64_t clampi(int64_t v, int64_t lo, int64_t hi) {
    return v < lo ? lo : (v > hi ? hi : v);
}

/* Read x at (qx, qy) under the boundary rule of §5 (Fig. 3). */
static double read_f64(const double *x, int64_t W, int64_t H, int64_t qx, int64_t qy,
                       int border, double bv) {
    if (qx >= 0 && qx < W && qy >= 0 && qy < H) return x[qy * W + qx];
    if (border == ORA_BORDER_CONSTANT) return bv;
    return x[clampi(qy, 0, H - 1) * W + clampi(qx, 0, W - 1)];
}

/*
 * Non-separable correlation (Listing 1 generalised to weighted taps; the
 * non-separable convolution benchmark of §6):
 *   out(x, y) = sum_{j<kh} sum_{i<kw} w[j][i] * in(x + i - rx, y + j - ry)
 * with rx = (kw-1)/2, ry = (kh-1)/2 and the boundary rule applied to `in`.
 * Output rows [y0, y1) only; out holds (y1 - y0) * W values.
 */
int ora_conv2d_f64(const double *x, int64_t W, int64_t H, const double *w, int kw, int kh,
                   int border, double bv, int64_t y0, int64_t y1, double *out) {
    if (!x || !w || !out || W <= 0 || H <= 0 || kw <= 0 || kh <= 0) return 1;
    if (y0 < 0 || y1 > H || y0 > y1) return 1;
    const int rx = (kw - 1) / 2, ry = (kh - 1) / 2;
#pragma omp parallel for schedule(static)
    for (int64_t py = y0; py < y1; ++py) {
        for (int64_t px = 0; px < W; ++px) {
            double s = 0.0;
            for (int j = 0; j < kh; ++j)
                for (int i = 0; i < kw; ++i)
                    s += w[j * kw + i] * read_f64(x, W, H, px + i - rx, py + j - ry, border, bv);
            out[(py - y0) * W + px] = s;
        }
    }
    return 0;
}

/*
 * The same correlation on integer pixels and taps: exact int64 accumulation, then the
 * result is wrapped to int32 (two's complement, mod 2^32).  The constant border value
 * is an integer here.
 */
int ora_conv2d_i64(const int64_t *x, int64_t W, int64_t H, const int64_t *w, int kw, int kh,
                   int border, int64_t bv, int64_t y0, int64_t y1, int32_t *out) {
    if (!x || !w || !out || W <= 0 || H <= 0 || kw <= 0 || kh <= 0) return 1;
    if (y0 < 0 || y1 > H || y0 > y1) return 1;
    const int rx = (kw - 1) / 2, ry = (kh - 1) / 2;
#pragma omp parallel for schedule(static)
    for (int64_t py = y0; py < y1; ++py) {
        for (int64_t px = 0; px < W; ++px) {
            int64_t s = 0;
            for (int j = 0; j < kh; ++j)
                for (int i = 0; i < kw; ++i) {
                    int64_t qx = px + i - rx, qy = py + j - ry, v;
                    if (qx >= 0 && qx < W && qy >= 0 && qy < H) v = x[qy * W + qx];
                    else if (border == ORA_BORDER_CONSTANT) v = bv;
                    else v = x[clampi(qy, 0, H - 1) * W + clampi(qx, 0, W - 1)];
                    s += w[j * kw + i] * v;
                }
            out[(py - y0) * W + px] = (int32_t)(uint32_t)(uint64_t)s;
        }
    }
    return 0;
}

/*
 * Separable correlation (the separable convolution benchmark of §6, a row pass then a
 * column pass, §7 discusses keeping the intermediate on chip):
 *   t(x, y)   = sum_i row[i] * in(x + i - rr, y)          (boundary rule on in)
 *   out(x, y) = sum_j col[j] * t(x, y + j - rc)           (boundary rule on t)
 * Output rows [y0, y1).  t is formed for every row the column pass reads.
 */
int ora_sepconv_f64(const double *x, int64_t W, int64_t H, const double *row, int nr,
                    const double *col, int nc, int border, double bv, int64_t y0, int64_t y1,
                    double *out) {
    if (!x || !row || !col || !out || W <= 0 || H <= 0 || nr <= 0 || nc <= 0) return 1;
    if (y0 < 0 || y1 > H || y0 > y1) return 1;
    if (y0 == y1) return 0;
    const int rr = (nr - 1) / 2, rc = (nc - 1) / 2;
    /* rows of t that the column pass can read inside the image */
    const int64_t t0 = clampi(y0 - rc, 0, H - 1), t1 = clampi(y1 - 1 + rc, 0, H - 1) + 1;
    double *t = (double *)malloc(sizeof(double) * (size_t)((t1 - t0) * W));
    if (!t) return 2;
#pragma omp parallel for schedule(static)
    for (int64_t ty = t0; ty < t1; ++ty)
        for (int64_t px = 0; px < W; ++px) {
            double s = 0.0;
            for (int i = 0; i < nr; ++i)
                s += row[i] * read_f64(x, W, H, px + i - rr, ty, border, bv);
            t[(ty - t0) * W + px] = s;
        }
#pragma omp parallel for schedule(static)
    for (int64_t py = y0; py < y1; ++py)
        for (int64_t px = 0; px < W; ++px) {
            double s = 0.0;
            for (int j = 0; j < nc; ++j) {
                int64_t qy = py + j - rc;
                double v;
                if (qy >= 0 && qy < H) v = t[(qy - t0) * W + px];
                else if (border == ORA_BORDER_CONSTANT) v = bv;
                else v = t[(clampi(qy, 0, H - 1) - t0) * W + px];
                s += col[j] * v;
            }
            out[(py - y0) * W + px] = s;
        }
    free(t);
    return 0;
}

/*
 * Harris corner response (the corner-detection benchmark of §6: a Sobel stage then a
 * Harris stage, Tables 4 and 5), clamped boundary on each stage's input:
 *   Ix = Sx (*) I,  Iy = Sy (*) I                          (3x3 correlations)
 *   Pxx = Ix*Ix,  Pyy = Iy*Iy,  Pxy = Ix*Iy
 *   Sc = G (*) Pc  for c in {xx, yy, xy}                  (wk x wk window)
 *   R = Sxx*Syy - Sxy*Sxy - k*(Sxx + Syy)^2
 * Window tap (j, i) reads the product at offset (i - wk/2, j - wk/2) (integer division):
 * centred for odd wk; for even wk (the 2x2 "block" of the Harris benchmark) the anchor is
 * the lower-right of the four central taps, offsets {-1, 0} for wk = 2.
 * Output rows [y0, y1) of R.  If `inter` is not NULL it receives, for those rows,
 * 8 planes [Ix, Iy, Pxx, Pyy, Pxy, Sxx, Syy, Sxy], each (y1 - y0) * W.
 */
static void sobel_at(const double *I, int64_t W, int64_t H, const double *sx,
                     const double *sy, int64_t px, int64_t py, double *ix, double *iy) {
    double gx = 0.0, gy = 0.0;
    for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) {
            double v = I[clampi(py + j - 1, 0, H - 1) * W + clampi(px + i - 1, 0, W - 1)];
            gx += sx[j * 3 + i] * v;
            gy += sy[j * 3 + i] * v;
        }
    *ix = gx;
    *iy = gy;
}

int ora_harris_f64(const double *I, int64_t W, int64_t H, const double *sx, const double *sy,
                   const double *win, int wk, double k, int64_t y0, int64_t y1, double *R,
                   double *inter) {
    if (!I || !sx || !sy || !win || !R || W <= 0 || H <= 0 || wk <= 0) return 1;
    if (y0 < 0 || y1 > H || y0 > y1) return 1;
    if (y0 == y1) return 0;
    const int rw = wk / 2;   /* anchor: odd wk centred, even wk offsets -wk/2 .. wk/2-1 */
    const int64_t p0 = clampi(y0 - rw, 0, H - 1), p1 = clampi(y1 - 1 + rw, 0, H - 1) + 1;
    const int64_t np = (p1 - p0) * W;
    double *P = (double *)malloc(sizeof(double) * (size_t)(3 * np + 2 * np));
    if (!P) return 2;
    double *Pxx = P, *Pyy = P + np, *Pxy = P + 2 * np, *Ix = P + 3 * np, *Iy = P + 4 * np;
#pragma omp parallel for schedule(static)
    for (int64_t py = p0; py < p1; ++py)
        for (int64_t px = 0; px < W; ++px) {
            double gx, gy;
            sobel_at(I, W, H, sx, sy, px, py, &gx, &gy);
            int64_t o = (py - p0) * W + px;
            Ix[o] = gx;
            Iy[o] = gy;
            Pxx[o] = gx * gx;
            Pyy[o] = gy * gy;
            Pxy[o] = gx * gy;
        }
    const int64_t nb = (y1 - y0) * W;
#pragma omp parallel for schedule(static)
    for (int64_t py = y0; py < y1; ++py)
        for (int64_t px = 0; px < W; ++px) {
            double sxx = 0.0, syy = 0.0, sxy = 0.0;
            for (int j = 0; j < wk; ++j)
                for (int i = 0; i < wk; ++i) {
                    int64_t qy = clampi(py + j - rw, 0, H - 1), qx = clampi(px + i - rw, 0, W - 1);
                    int64_t o = (qy - p0) * W + qx;
                    double g = win[j * wk + i];
                    sxx += g * Pxx[o];
                    syy += g * Pyy[o];
                    sxy += g * Pxy[o];
                }
            double tr = sxx + syy;
            int64_t o = (py - y0) * W + px;
            R[o] = sxx * syy - sxy * sxy - k * tr * tr;
            if (inter) {
                int64_t q = (py - p0) * W + px;
                inter[0 * nb + o] = Ix[q];
                inter[1 * nb + o] = Iy[q];
                inter[2 * nb + o] = Pxx[q];
                inter[3 * nb + o] = Pyy[q];
                inter[4 * nb + o] = Pxy[q];
                inter[5 * nb + o] = sxx;
                inter[6 * nb + o] = syy;
                inter[7 * nb + o] = sxy;
            }
        }
    free(P);
    return 0;
}

/* ------------------------------------------------------------------------ adjoints
 * The backward passes are the transposes of the forward maps, written as explicit
 * scatter loops: for every output p and tap o, the forward read in(b(p + o)) with
 * weight w[o]; so the input gradient receives w[o] * g[p] at b(p + o), and the weight
 * gradient receives g[p] * in(b(p + o)).  With the clamped rule b() is the clamp, so
 * taps that fell outside the image scatter onto the edge pixels.  Under the constant
 * rule an outside read has no input to flow back to (the constant is not a variable).
 * Serial loops: the scatter order is fixed.
 */

/* Adjoint of ora_conv2d_f64 over the whole image.  dx (W*H) and dw (kh*kw) may be
 * NULL; when given they are overwritten. */
int ora_conv2d_bwd_f64(const double *x, int64_t W, int64_t H, const double *w, int kw, int kh,
                       int border, double bv, const double *g, double *dx, double *dw) {
    if (!x || !w || !g || W <= 0 || H <= 0 || kw <= 0 || kh <= 0) return 1;
    const int rx = (kw - 1) / 2, ry = (kh - 1) / 2;
    if (dx) memset(dx, 0, sizeof(double) * (size_t)(W * H));
    if (dw) memset(dw, 0, sizeof(double) * (size_t)(kw * kh));
    for (int64_t py = 0; py < H; ++py)
        for (int64_t px = 0; px < W; ++px) {
            const double gp = g[py * W + px];
            for (int j = 0; j < kh; ++j)
                for (int i = 0; i < kw; ++i) {
                    int64_t qx = px + i - rx, qy = py + j - ry;
                    int inside = qx >= 0 && qx < W && qy >= 0 && qy < H;
                    if (!inside && border == ORA_BORDER_CONSTANT) {
                        if (dw) dw[j * kw + i] += gp * bv;
                        continue;
                    }
                    qx = clampi(qx, 0, W - 1);
                    qy = clampi(qy, 0, H - 1);
                    if (dx) dx[qy * W + qx] += w[j * kw + i] * gp;
                    if (dw) dw[j * kw + i] += gp * x[qy * W + qx];
                }
        }
    return 0;
}

/* Adjoint of ora_sepconv_f64 (whole image): the column pass is undone first, giving
 * dt and dcol, then the row pass, giving dx and drow.  Outputs may be NULL. */
int ora_sepconv_bwd_f64(const double *x, int64_t W, int64_t H, const double *row, int nr,
                        const double *col, int nc, int border, double bv, const double *g,
                        double *dx, double *drow, double *dcol) {
    if (!x || !row || !col || !g || W <= 0 || H <= 0 || nr <= 0 || nc <= 0) return 1;
    const int rr = (nr - 1) / 2, rc = (nc - 1) / 2;
    const int64_t n = W * H;
    double *t = (double *)malloc(sizeof(double) * (size_t)n);
    double *dt = (double *)calloc((size_t)n, sizeof(double));
    if (!t || !dt) { free(t); free(dt); return 2; }
    /* the row pass t of the forward, recomputed */
    for (int64_t py = 0; py < H; ++py)
        for (int64_t px = 0; px < W; ++px) {
            double s = 0.0;
            for (int i = 0; i < nr; ++i) s += row[i] * read_f64(x, W, H, px + i - rr, py, border, bv);
            t[py * W + px] = s;
        }
    if (drow) memset(drow, 0, sizeof(double) * (size_t)nr);
    if (dcol) memset(dcol, 0, sizeof(double) * (size_t)nc);
    if (dx) memset(dx, 0, sizeof(double) * (size_t)n);
    /* column pass: out(p) = sum_j col[j] t(px, b(py + j - rc)) */
    for (int64_t py = 0; py < H; ++py)
        for (int64_t px = 0; px < W; ++px) {
            const double gp = g[py * W + px];
            for (int j = 0; j < nc; ++j) {
                int64_t qy = py + j - rc;
                if ((qy < 0 || qy >= H) && border == ORA_BORDER_CONSTANT) {
                    if (dcol) dcol[j] += gp * bv;
                    continue;
                }
                qy = clampi(qy, 0, H - 1);
                dt[qy * W + px] += col[j] * gp;
                if (dcol) dcol[j] += gp * t[qy * W + px];
            }
        }
    /* row pass: t(p) = sum_i row[i] x(b(px + i - rr), py) */
    for (int64_t py = 0; py < H; ++py)
        for (int64_t px = 0; px < W; ++px) {
            const double gp = dt[py * W + px];
            for (int i = 0; i < nr; ++i) {
                int64_t qx = px + i - rr;
                if ((qx < 0 || qx >= W) && border == ORA_BORDER_CONSTANT) {
                    if (drow) drow[i] += gp * bv;
                    continue;
                }
                qx = clampi(qx, 0, W - 1);
                if (dx) dx[py * W + qx] += row[i] * gp;
                if (drow) drow[i] += gp * x[py * W + qx];
            }
        }
    free(t);
    free(dt);
    return 0;
}

/* Adjoint of ora_harris_f64 (whole image, clamped rule), by the chain rule taken one
 * stage at a time in reverse:
 *   gSxx = gR (Syy - 2k tr),  gSyy = gR (Sxx - 2k tr),  gSxy = -2 gR Sxy
 *   window adjoint: gPc(b(p+o)) += G[o] gSc(p);  dwin[o] += sum_c gSc(p) Pc(b(p+o))
 *   gIx = 2 Ix gPxx + Iy gPxy,  gIy = 2 Iy gPyy + Ix gPxy
 *   Sobel adjoint: dI(b(p+o)) += Sx[o] gIx(p) + Sy[o] gIy(p);
 *                  dsx[o] += gIx(p) I(b(p+o)),  dsy[o] += gIy(p) I(b(p+o))
 * Outputs may be NULL. */
int ora_harris_bwd_f64(const double *I, int64_t W, int64_t H, const double *sx, const double *sy,
                       const double *win, int wk, double k, const double *gR, double *dI,
                       double *dsx, double *dsy, double *dwin) {
    if (!I || !sx || !sy || !win || !gR || W <= 0 || H <= 0 || wk <= 0) return 1;
    const int rw = wk / 2;   /* anchor: odd wk centred, even wk offsets -wk/2 .. wk/2-1 */
    const int64_t n = W * H;
    double *inter = (double *)malloc(sizeof(double) * (size_t)(8 * n));
    double *R = (double *)malloc(sizeof(double) * (size_t)n);
    double *gP = (double *)calloc((size_t)(3 * n), sizeof(double));
    double *gI = (double *)malloc(sizeof(double) * (size_t)(2 * n));
    if (!inter || !R || !gP || !gI) { free(inter); free(R); free(gP); free(gI); return 2; }
    ora_harris_f64(I, W, H, sx, sy, win, wk, k, 0, H, R, inter);
    const double *Ix = inter, *Iy = inter + n, *Pxx = inter + 2 * n, *Pyy = inter + 3 * n,
                 *Pxy = inter + 4 * n, *Sxx = inter + 5 * n, *Syy = inter + 6 * n,
                 *Sxy = inter + 7 * n;
    if (dwin) memset(dwin, 0, sizeof(double) * (size_t)(wk * wk));
    if (dsx) memset(dsx, 0, sizeof(double) * 9);
    if (dsy) memset(dsy, 0, sizeof(double) * 9);
    if (dI) memset(dI, 0, sizeof(double) * (size_t)n);
    for (int64_t py = 0; py < H; ++py)
        for (int64_t px = 0; px < W; ++px) {
            const int64_t p = py * W + px;
            const double tr = Sxx[p] + Syy[p];
            const double gsxx = gR[p] * (Syy[p] - 2.0 * k * tr);
            const double gsyy = gR[p] * (Sxx[p] - 2.0 * k * tr);
            const double gsxy = -2.0 * gR[p] * Sxy[p];
            for (int j = 0; j < wk; ++j)
                for (int i = 0; i < wk; ++i) {
                    const int64_t q = clampi(py + j - rw, 0, H - 1) * W + clampi(px + i - rw, 0, W - 1);
                    const double g = win[j * wk + i];
                    gP[q] += g * gsxx;
                    gP[n + q] += g * gsyy;
                    gP[2 * n + q] += g * gsxy;
                    if (dwin) dwin[j * wk + i] += gsxx * Pxx[q] + gsyy * Pyy[q] + gsxy * Pxy[q];
                }
        }
    for (int64_t p = 0; p < n; ++p) {
        gI[p] = 2.0 * Ix[p] * gP[p] + Iy[p] * gP[2 * n + p];
        gI[n + p] = 2.0 * Iy[p] * gP[n + p] + Ix[p] * gP[2 * n + p];
    }
    for (int64_t py = 0; py < H; ++py)
        for (int64_t px = 0; px < W; ++px) {
            const int64_t p = py * W + px;
            for (int j = 0; j < 3; ++j)
                for (int i = 0; i < 3; ++i) {
                    const int64_t q = clampi(py + j - 1, 0, H - 1) * W + clampi(px + i - 1, 0, W - 1);
                    if (dI) dI[q] += sx[j * 3 + i] * gI[p] + sy[j * 3 + i] * gI[n + p];
                    if (dsx) dsx[j * 3 + i] += gI[p] * I[q];
                    if (dsy) dsy[j * 3 + i] += gI[n + p] * I[q];
                }
        }
    free(inter);
    free(R);
    free(gP);
    free(gI);
    return 0;
}
