/*
 * FP64 CPU oracle for one-level 2D DWT pansharpening, written from
 * Al-Oraiqat, Bashkov, Babkov, Titarenko, "Fusion of multispectral satellite
 * imagery using a cluster of graphics processing unit" (arXiv:1803.00737).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this library.  The product (the CUDA
 * library and its Python binding) never calls, links or imports it, and this
 * file shares no code, header or table with the product.
 *
 * What it computes, in the paper's order and notation (Sec. 2):
 *   - 1D forward Haar transform, Eq. 1-2; 1D forward Daubechies-4 transform,
 *     Eq. 3-6 (with the periodic wrap of Eq. 5-6), coefficients Eq. 7-10;
 *   - 1D inverse Haar transform, Eq. 11-12; 1D inverse Daubechies-4 transform,
 *     Eq. 13-16 with the t/u tables defined after Eq. 16;
 *   - 2D transform: 1D transform of every row, then of every column; inverse:
 *     columns first, then rows (Sec. 2, the paragraph after the step list);
 *   - fusion (Sec. 2 step list): forward 2D DWT of PAN, replace the
 *     approximation (LL, top-left H/2 x W/2 quadrant) by the MS band, inverse
 *     2D DWT; once per MS band.
 * Each 1D equation is written as a list of taps (input index, weight) for one
 * output index.  The whole-vector transforms, the point-wise evaluator and the
 * adjoints all read that one list, so every path states each equation once.
 *
 * Readings where the paper is garbled or silent (each pinned by a test):
 *   R1  g of Eq. 9-10 as printed fails perfect reconstruction; the oracle uses
 *       the quadrature mirror g = [h3, -h2, h1, -h0] of the h of Eq. 7-8.  The
 *       printed g is kept (oracle_d4_g_printed) only for the pin showing it
 *       fails.
 *   R2  Index ranges: Eq. 1 i in [0, N/2); Eq. 3-4 cover i in [0, N/2-2] and
 *       Eq. 5-6 give i = N/2-1; Eq. 15-16 cover i in [0, N/2-2]; in Eq. 13-14
 *       "(N-1)k" is the index 0 for k = 0 and N-1 for k = 1; "u_i, g_i" after
 *       Eq. 16 means h_i, g_i.
 *   R3  LL replacement gain (silent): LL <- gain * MS with gain = DC gain of
 *       the 2D low-pass, 1 for Haar (2x2 mean), 2 for D4 (sum h = sqrt 2 per
 *       axis).  The gain is an argument here so other readings can be tested.
 *   R4  MS pixel (i, j) replaces LL coefficient (i, j) with no shift.
 *   R5  Periodic wrap over the whole image, never per tile.
 *   R6  uint8 output: clamp to [0, 255], then round half to even.
 *   R7  ERGAS and QNR are not defined in the paper (Sec. 4, Table 3): the
 *       definitions used are stated at oracle_ergas and oracle_qnr.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_HAAR 0
#define ORACLE_D4 1

/* ---------------------------------------------------------------- coeffs */

/* Eq. 7-8: h_i = (1 + 2i + sqrt3) / (4 sqrt2), h_{i+2} = (3 - 2i - sqrt3) / (4 sqrt2),
 * i in {0, 1}.  Reading R1: g_k = (-1)^k h_{3-k}. */
static void d4_coeffs(double h[4], double g[4]) {
    const double r3 = sqrt(3.0), den = 4.0 * sqrt(2.0);
    for (int i = 0; i < 2; ++i) {
        h[i] = (1.0 + 2.0 * i + r3) / den;
        h[i + 2] = (3.0 - 2.0 * i - r3) / den;
    }
    g[0] = h[3];
    g[1] = -h[2];
    g[2] = h[1];
    g[3] = -h[0];
}

void oracle_d4_h(double out[4]) {
    double h[4], g[4];
    d4_coeffs(h, g);
    memcpy(out, h, sizeof h);
}

void oracle_d4_g(double out[4]) {
    double h[4], g[4];
    d4_coeffs(h, g);
    memcpy(out, g, sizeof g);
}

/* Eq. 9-10 exactly as printed: g_i = (2i + sqrt3 - 3)/(4 sqrt2),
 * g_{i+2} = (sqrt3 - 1 - 2i)/(4 sqrt2).  Used only by the pin that shows why
 * reading R1 is needed. */
void oracle_d4_g_printed(double out[4]) {
    const double r3 = sqrt(3.0), den = 4.0 * sqrt(2.0);
    for (int i = 0; i < 2; ++i) {
        out[i] = (2.0 * i + r3 - 3.0) / den;
        out[i + 2] = (r3 - 1.0 - 2.0 * i) / den;
    }
}

/* A wavelet as used by the oracle: which family, and its filters (D4 only). */
typedef struct {
    int kind;
    double h[4], g[4];
} wavelet_t;

static wavelet_t make_wavelet(int kind, const double *g_override) {
    wavelet_t w;
    memset(&w, 0, sizeof w);
    w.kind = kind;
    if (kind == ORACLE_D4) {
        d4_coeffs(w.h, w.g);
        if (g_override) memcpy(w.g, g_override, sizeof w.g);
    }
    return w;
}

/* ------------------------------------------------------------ 1D taps */

/* Taps of one output of the 1D forward transform of a length-N vector s laid
 * out as [approximation (N/2) | detail (N/2)].  Writes input indices and
 * weights; returns the number of taps. */
static int fwd1d_taps(const wavelet_t *w, long N, long o, long idx[4], double wt[4]) {
    const long half = N / 2;
    const int detail = o >= half;
    const long i = detail ? o - half : o;
    if (w->kind == ORACLE_HAAR) {
        /* Eq. 1: s'_i = (s_2i + s_2i+1) / 2;  Eq. 2: s'_{N/2+i} = (s_2i - s_2i+1) / 2 */
        idx[0] = 2 * i;
        wt[0] = 0.5;
        idx[1] = 2 * i + 1;
        wt[1] = detail ? -0.5 : 0.5;
        return 2;
    }
    const double *c = detail ? w->g : w->h;
    if (i <= half - 2) {
        /* Eq. 3 (h) / Eq. 4 (g): sum_k s_{2i+k} c_k, k in [0, 3] */
        for (int k = 0; k < 4; ++k) {
            idx[k] = 2 * i + k;
            wt[k] = c[k];
        }
        return 4;
    }
    /* Eq. 5 (h) / Eq. 6 (g), i = N/2 - 1: sum_m s_{N-2+m} c_m + sum_m s_m c_{2+m}, m in [0, 1] */
    for (int m = 0; m < 2; ++m) {
        idx[m] = N - 2 + m;
        wt[m] = c[m];
        idx[2 + m] = m;
        wt[2 + m] = c[2 + m];
    }
    return 4;
}

/* Taps of output n of the 1D inverse transform of c = [approx | detail]. */
static int inv1d_taps(const wavelet_t *w, long N, long n, long idx[4], double wt[4]) {
    const long half = N / 2;
    if (w->kind == ORACLE_HAAR) {
        /* Eq. 11: s_2i = s'_i + s'_{N/2+i};  Eq. 12: s_2i+1 = s'_i - s'_{N/2+i} */
        const long i = n / 2;
        idx[0] = i;
        wt[0] = 1.0;
        idx[1] = half + i;
        wt[1] = (n % 2 == 0) ? 1.0 : -1.0;
        return 2;
    }
    /* Tables after Eq. 16: t = (h2, g2, h0, g0), u = (h3, g3, h1, g1). */
    const double t[4] = {w->h[2], w->g[2], w->h[0], w->g[0]};
    const double u[4] = {w->h[3], w->g[3], w->h[1], w->g[1]};
    const double *v = (n % 2 == 0) ? t : u;
    if (n < 2) {
        /* Eq. 13 (n = 0, table t) / Eq. 14 (n = 1, table u):
         * sum_k s'_{N/2-1+k} v_{3k} + sum_k s'_{(N-1)k} v_{2-k}, k in [0, 1] */
        for (int k = 0; k < 2; ++k) {
            idx[k] = half - 1 + k;
            wt[k] = v[3 * k];
            idx[2 + k] = (N - 1) * k;
            wt[2 + k] = v[2 - k];
        }
        return 4;
    }
    /* Eq. 15 (n = 2 + 2i, table t) / Eq. 16 (n = 3 + 2i, table u):
     * sum_k s'_{i+k} v_{2k} + sum_k s'_{i+N/2+k} v_{1+2k}, k in [0, 1] */
    const long i = (n - 2) / 2;
    for (int k = 0; k < 2; ++k) {
        idx[k] = i + k;
        wt[k] = v[2 * k];
        idx[2 + k] = i + half + k;
        wt[2 + k] = v[1 + 2 * k];
    }
    return 4;
}

/* ------------------------------------------------------- 1D transforms */

/* y = T x for a strided vector (x and y must not overlap). */
static void apply1d(int inverse, const wavelet_t *w, long N, const double *x, long xs, double *y,
                    long ys) {
    long idx[4];
    double wt[4];
    for (long o = 0; o < N; ++o) {
        const int nt = inverse ? inv1d_taps(w, N, o, idx, wt) : fwd1d_taps(w, N, o, idx, wt);
        double acc = 0.0;
        for (int k = 0; k < nt; ++k) acc += wt[k] * x[idx[k] * xs];
        y[o * ys] = acc;
    }
}

/* xbar += T^T ybar: every tap (o <- i, weight w) becomes (i <- o, weight w). */
static void apply1d_adjoint(int inverse, const wavelet_t *w, long N, const double *ybar, long ys,
                            double *xbar, long xs) {
    long idx[4];
    double wt[4];
    for (long i = 0; i < N; ++i) xbar[i * xs] = 0.0;
    for (long o = 0; o < N; ++o) {
        const int nt = inverse ? inv1d_taps(w, N, o, idx, wt) : fwd1d_taps(w, N, o, idx, wt);
        for (int k = 0; k < nt; ++k) xbar[idx[k] * xs] += wt[k] * ybar[o * ys];
    }
}

int oracle_dwt1d(int kind, long N, const double *x, double *y) {
    if (N < 2 || N % 2) return 1;
    wavelet_t w = make_wavelet(kind, NULL);
    apply1d(0, &w, N, x, 1, y, 1);
    return 0;
}

int oracle_idwt1d(int kind, long N, const double *x, double *y) {
    if (N < 2 || N % 2) return 1;
    wavelet_t w = make_wavelet(kind, NULL);
    apply1d(1, &w, N, x, 1, y, 1);
    return 0;
}

/* Same as oracle_dwt1d / oracle_idwt1d but with an explicit D4 g (pins only). */
int oracle_dwt1d_g(long N, const double *g, const double *x, double *y) {
    if (N < 2 || N % 2) return 1;
    wavelet_t w = make_wavelet(ORACLE_D4, g);
    apply1d(0, &w, N, x, 1, y, 1);
    return 0;
}

int oracle_idwt1d_g(long N, const double *g, const double *x, double *y) {
    if (N < 2 || N % 2) return 1;
    wavelet_t w = make_wavelet(ORACLE_D4, g);
    apply1d(1, &w, N, x, 1, y, 1);
    return 0;
}

/* ------------------------------------------------------- 2D transforms */

/* One pass of a 1D map over every row (axis 1) or every column (axis 0) of
 * an H x W image, in place.  adjoint selects T^T instead of T. */
static void pass2d(int inverse, int adjoint, const wavelet_t *w, double *img, long H, long W,
                   int axis) {
    const long lines = axis == 1 ? H : W;
    const long N = axis == 1 ? W : H;
    const long stride = axis == 1 ? 1 : W;
#pragma omp parallel
    {
        double *src = (double *)malloc(sizeof(double) * N);
        double *dst = (double *)malloc(sizeof(double) * N);
#pragma omp for schedule(static)
        for (long l = 0; l < lines; ++l) {
            double *base = axis == 1 ? img + l * W : img + l;
            for (long k = 0; k < N; ++k) src[k] = base[k * stride];
            if (adjoint)
                apply1d_adjoint(inverse, w, N, src, 1, dst, 1);
            else
                apply1d(inverse, w, N, src, 1, dst, 1);
            for (long k = 0; k < N; ++k) base[k * stride] = dst[k];
        }
        free(src);
        free(dst);
    }
}

/* Forward 2D DWT (rows, then columns), in place. */
static void dwt2(const wavelet_t *w, double *img, long H, long W) {
    pass2d(0, 0, w, img, H, W, 1);
    pass2d(0, 0, w, img, H, W, 0);
}

/* Inverse 2D DWT (columns, then rows), in place. */
static void idwt2(const wavelet_t *w, double *img, long H, long W) {
    pass2d(1, 0, w, img, H, W, 0);
    pass2d(1, 0, w, img, H, W, 1);
}

static int check_shape(int kind, long H, long W) {
    if (kind != ORACLE_HAAR && kind != ORACLE_D4) return 1;
    if (H < 2 || W < 2 || H % 2 || W % 2) return 1;
    return 0;
}

int oracle_dwt2(int kind, long H, long W, const double *x, double *y) {
    if (check_shape(kind, H, W)) return 1;
    wavelet_t w = make_wavelet(kind, NULL);
    memcpy(y, x, sizeof(double) * H * W);
    dwt2(&w, y, H, W);
    return 0;
}

int oracle_idwt2(int kind, long H, long W, const double *x, double *y) {
    if (check_shape(kind, H, W)) return 1;
    wavelet_t w = make_wavelet(kind, NULL);
    memcpy(y, x, sizeof(double) * H * W);
    idwt2(&w, y, H, W);
    return 0;
}

/* ------------------------------------------------------------- fusion */

/* Reading R3: the DC gain of the 2D low-pass of each wavelet. */
double oracle_default_gain(int kind) { return kind == ORACLE_D4 ? 2.0 : 1.0; }

/* Fusion, Sec. 2 step list, for each of the B bands:
 *   X = DWT2(PAN);  X[i][j] <- gain * MS_b[i][j] for i < H/2, j < W/2;  F_b = IDWT2(X).
 * pan: H x W; ms: B arrays of H/2 x W/2; out: B x H x W.  All FP64, row-major. */
int oracle_fuse(int kind, long H, long W, int B, double gain, const double *pan,
                const double *const *ms, double *out) {
    if (check_shape(kind, H, W) || B < 1) return 1;
    wavelet_t w = make_wavelet(kind, NULL);
    const long H2 = H / 2, W2 = W / 2, n = H * W;
    double *X = (double *)malloc(sizeof(double) * n);
    if (!X) return 2;
    memcpy(X, pan, sizeof(double) * n);
    dwt2(&w, X, H, W);
    for (int b = 0; b < B; ++b) {
        double *Y = out + (long)b * n;
        memcpy(Y, X, sizeof(double) * n);
        for (long i = 0; i < H2; ++i)
            for (long j = 0; j < W2; ++j) Y[i * W + j] = gain * ms[b][i * W2 + j];
        idwt2(&w, Y, H, W);
    }
    free(X);
    return 0;
}

/* Adjoint of the fusion map (PAN, MS_1..MS_B) -> (F_1..F_B), built by
 * transposing each step of oracle_fuse in reverse order:
 *   Ybar_b = IDWT2^T(gF_b)                       (rows^T, then columns^T)
 *   gMS_b  = gain * Ybar_b[LL];  Ybar_b[LL] <- 0  (transpose of the swap)
 *   gPAN   = sum_b DWT2^T(Ybar_b)                (columns^T, then rows^T)
 * grad_out: B x H x W; grad_pan: H x W; grad_ms: B arrays of H/2 x W/2. */
int oracle_fuse_adjoint(int kind, long H, long W, int B, double gain, const double *grad_out,
                        double *grad_pan, double *const *grad_ms) {
    if (check_shape(kind, H, W) || B < 1) return 1;
    wavelet_t w = make_wavelet(kind, NULL);
    const long H2 = H / 2, W2 = W / 2, n = H * W;
    double *Y = (double *)malloc(sizeof(double) * n);
    if (!Y) return 2;
    memset(grad_pan, 0, sizeof(double) * n);
    for (int b = 0; b < B; ++b) {
        memcpy(Y, grad_out + (long)b * n, sizeof(double) * n);
        pass2d(1, 1, &w, Y, H, W, 1);
        pass2d(1, 1, &w, Y, H, W, 0);
        for (long i = 0; i < H2; ++i)
            for (long j = 0; j < W2; ++j) {
                grad_ms[b][i * W2 + j] = gain * Y[i * W + j];
                Y[i * W + j] = 0.0;
            }
        pass2d(0, 1, &w, Y, H, W, 0);
        pass2d(0, 1, &w, Y, H, W, 1);
        for (long k = 0; k < n; ++k) grad_pan[k] += Y[k];
    }
    free(Y);
    return 0;
}

/* --------------------------------------------- point-wise evaluation */

/* The same fusion evaluated lazily for one output pixel: each stage asks only
 * for the inputs its taps name.  Used to check sampled pixels of images too
 * large for the whole-image oracle.  Indices are those of the whole image, so
 * the wrap of Eq. 5-6 and Eq. 13-14 is the whole image's. */
typedef struct {
    const wavelet_t *w;
    long H, W;
    double gain;
    const double *pan;
    const uint8_t *pan_u8;
    const double *ms;
    const uint8_t *ms_u8;
} point_ctx;

static double pan_at(const point_ctx *c, long y, long x) {
    return c->pan ? c->pan[y * c->W + x] : (double)c->pan_u8[y * c->W + x];
}

static double ms_at(const point_ctx *c, long i, long j) {
    const long W2 = c->W / 2;
    return c->ms ? c->ms[i * W2 + j] : (double)c->ms_u8[i * W2 + j];
}

/* Row pass of the forward transform: output k of row y. */
static double row_fwd(const point_ctx *c, long y, long k) {
    long idx[4];
    double wt[4], acc = 0.0;
    const int nt = fwd1d_taps(c->w, c->W, k, idx, wt);
    for (int t = 0; t < nt; ++t) acc += wt[t] * pan_at(c, y, idx[t]);
    return acc;
}

/* Column pass of the forward transform, then the LL swap: coefficient (i, k). */
static double coeff_swapped(const point_ctx *c, long i, long k) {
    if (i < c->H / 2 && k < c->W / 2) return c->gain * ms_at(c, i, k);
    long idx[4];
    double wt[4], acc = 0.0;
    const int nt = fwd1d_taps(c->w, c->H, i, idx, wt);
    for (int t = 0; t < nt; ++t) acc += wt[t] * row_fwd(c, idx[t], k);
    return acc;
}

/* Column pass of the inverse transform: value (y, k). */
static double col_inv(const point_ctx *c, long y, long k) {
    long idx[4];
    double wt[4], acc = 0.0;
    const int nt = inv1d_taps(c->w, c->H, y, idx, wt);
    for (int t = 0; t < nt; ++t) acc += wt[t] * coeff_swapped(c, idx[t], k);
    return acc;
}

/* Row pass of the inverse transform: fused value (y, x). */
static double row_inv(const point_ctx *c, long y, long x) {
    long idx[4];
    double wt[4], acc = 0.0;
    const int nt = inv1d_taps(c->w, c->W, x, idx, wt);
    for (int t = 0; t < nt; ++t) acc += wt[t] * col_inv(c, y, idx[t]);
    return acc;
}

/* Fused values of one band at n sampled pixels (ys[k], xs[k]).  Exactly one of
 * pan/pan_u8 and one of ms/ms_u8 is non-NULL. */
int oracle_fuse_points(int kind, long H, long W, double gain, const double *pan,
                       const uint8_t *pan_u8, const double *ms, const uint8_t *ms_u8, long n,
                       const long *ys, const long *xs, double *out) {
    if (check_shape(kind, H, W)) return 1;
    if (!pan == !pan_u8 || !ms == !ms_u8) return 1;
    wavelet_t w = make_wavelet(kind, NULL);
    point_ctx c = {&w, H, W, gain, pan, pan_u8, ms, ms_u8};
#pragma omp parallel for schedule(dynamic, 16)
    for (long k = 0; k < n; ++k) out[k] = row_inv(&c, ys[k], xs[k]);
    return 0;
}

/* Coefficients of the forward 2D transform (rows, then columns) at n sampled
 * indices (is[k], js[k]) of the H x W coefficient image, from the same tap
 * lists (for images too large for the whole-image oracle). */
int oracle_dwt2_points(int kind, long H, long W, const double *img, const uint8_t *img_u8, long n,
                       const long *is, const long *js, double *out) {
    if (check_shape(kind, H, W)) return 1;
    if (!img == !img_u8) return 1;
    wavelet_t w = make_wavelet(kind, NULL);
    point_ctx c = {&w, H, W, 0.0, img, img_u8, NULL, NULL};
#pragma omp parallel for schedule(dynamic, 16)
    for (long k = 0; k < n; ++k) {
        long idx[4];
        double wt[4], acc = 0.0;
        const int nt = fwd1d_taps(c.w, H, is[k], idx, wt);
        for (int t = 0; t < nt; ++t) acc += wt[t] * row_fwd(&c, idx[t], js[k]);
        out[k] = acc;
    }
    return 0;
}

/* ------------------------------------- point-wise evaluation of the adjoint */

/* Users of input index i under a 1D map: the outputs o whose tap list names i,
 * each with the summed weight of those taps.  The transposed map at i is
 * sum over users (o, w) of w * ybar[o].  Each output of the forward map reads
 * inputs 2a .. 2a+3 (mod N) of its half-index a, and each output n of the
 * inverse map reads coefficients of half-index (n-2)/2 .. n/2 (mod N/2), so
 * the outputs that can name i lie within a few places of it; those candidates
 * are filtered by their own tap lists, and no equation is restated here.
 * Returns the number of users (at most 8). */
static int users1d(int inverse, const wavelet_t *w, long N, long i, long o_out[8], double wt_out[8]) {
    const long half = N / 2;
    long cand[16];
    int nc = 0;
    if (!inverse) {
        /* forward outputs: approximation a and detail half + a, a near i / 2 */
        for (long d = -2; d <= 1; ++d) {
            const long a = ((i / 2 + d) % half + half) % half;
            cand[nc++] = a;
            cand[nc++] = half + a;
        }
    } else {
        /* inverse outputs near twice the half-index of coefficient i */
        const long a = i % half;
        for (long d = -2; d <= 5; ++d) cand[nc++] = ((2 * a + d) % N + N) % N;
    }
    int nu = 0;
    for (int c = 0; c < nc; ++c) {
        int dup = 0;
        for (int k = 0; k < c; ++k) dup |= cand[k] == cand[c];
        if (dup) continue;
        long idx[4];
        double wt[4], acc = 0.0;
        int hit = 0;
        const int nt = inverse ? inv1d_taps(w, N, cand[c], idx, wt) : fwd1d_taps(w, N, cand[c], idx, wt);
        for (int t = 0; t < nt; ++t)
            if (idx[t] == i) {
                acc += wt[t];
                hit = 1;
            }
        if (hit) {
            o_out[nu] = cand[c];
            wt_out[nu] = acc;
            ++nu;
        }
    }
    return nu;
}

/* The output gradient of one band is given on a periodic window of the image:
 * g[r][s] = gF(y, x) for y = (gy0 + r) mod H, r < hg, and x = (gx0 + s) mod W,
 * s < wg (gy0 = gx0 = 0, hg = H, wg = W for the whole image).  A read outside
 * the window gives NaN, which propagates into the evaluated value. */
typedef struct {
    const wavelet_t *w;
    long H, W;
    double gain;
    const double *g; /* B planes of hg x wg */
    long gy0, gx0, hg, wg;
} adj_ctx;

static double gout_at(const adj_ctx *c, int b, long y, long x) {
    const long r = ((y - c->gy0) % c->H + c->H) % c->H;
    const long s = ((x - c->gx0) % c->W + c->W) % c->W;
    if (r >= c->hg || s >= c->wg) return NAN;
    return c->g[((long)b * c->hg + r) * c->wg + s];
}

/* Transpose of the inverse row pass (Eq. 11-16 along a row): value (y, k). */
static double adj_row_inv(const adj_ctx *c, int b, long y, long k) {
    long o[8];
    double wt[8], acc = 0.0;
    const int nu = users1d(1, c->w, c->W, k, o, wt);
    for (int t = 0; t < nu; ++t) acc += wt[t] * gout_at(c, b, y, o[t]);
    return acc;
}

/* Transpose of the inverse column pass: coefficient (i, k) of Ybar_b. */
static double adj_col_inv(const adj_ctx *c, int b, long i, long k) {
    long o[8];
    double wt[8], acc = 0.0;
    const int nu = users1d(1, c->w, c->H, i, o, wt);
    for (int t = 0; t < nu; ++t) acc += wt[t] * adj_row_inv(c, b, o[t], k);
    return acc;
}

/* Transpose of the LL swap: the LL quadrant of Ybar_b goes to MS, the rest on. */
static double adj_swapped(const adj_ctx *c, int b, long i, long k) {
    if (i < c->H / 2 && k < c->W / 2) return 0.0;
    return adj_col_inv(c, b, i, k);
}

/* Transpose of the forward column pass (Eq. 1-6 along a column): value (r, k). */
static double adj_col_fwd(const adj_ctx *c, int b, long r, long k) {
    long o[8];
    double wt[8], acc = 0.0;
    const int nu = users1d(0, c->w, c->H, r, o, wt);
    for (int t = 0; t < nu; ++t) acc += wt[t] * adj_swapped(c, b, o[t], k);
    return acc;
}

/* Transpose of the forward row pass: this band's share of grad PAN (y, x). */
static double adj_row_fwd(const adj_ctx *c, int b, long y, long x) {
    long o[8];
    double wt[8], acc = 0.0;
    const int nu = users1d(0, c->w, c->W, x, o, wt);
    for (int t = 0; t < nu; ++t) acc += wt[t] * adj_col_fwd(c, b, y, o[t]);
    return acc;
}

/* The adjoint of the fusion (the map oracle_fuse_adjoint applies to whole
 * images) evaluated lazily at sampled outputs:
 *   grad_pan at n pixels (ys[k], xs[k]):  sum_b DWT2^T(Ybar_b, LL zeroed)
 *   grad_ms of every band at nm MS pixels (is[k], js[k]):  gain * Ybar_b[LL]
 * with Ybar_b = IDWT2^T(gF_b).  Each transposed pass sums over the users of an
 * index, taken from the same tap lists as the forward maps.  g: B planes of
 * the output gradient on the periodic window (gy0, gx0, hg, wg) described at
 * gout_at; out_ms: B x nm.  A value needing gradient outside the window is NaN. */
int oracle_fuse_adjoint_points(int kind, long H, long W, int B, double gain, const double *g, long gy0,
                               long gx0, long hg, long wg, long n, const long *ys, const long *xs,
                               double *out_pan, long nm, const long *is, const long *js,
                               double *out_ms) {
    if (check_shape(kind, H, W) || B < 1) return 1;
    if (hg < 1 || wg < 1 || hg > H || wg > W) return 1;
    wavelet_t w = make_wavelet(kind, NULL);
    adj_ctx c = {&w, H, W, gain, g, gy0, gx0, hg, wg};
#pragma omp parallel for schedule(dynamic, 16)
    for (long k = 0; k < n; ++k) {
        double acc = 0.0;
        for (int b = 0; b < B; ++b) acc += adj_row_fwd(&c, b, ys[k], xs[k]);
        out_pan[k] = acc;
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (long k = 0; k < nm; ++k)
        for (int b = 0; b < B; ++b) out_ms[(long)b * nm + k] = gain * adj_col_inv(&c, b, is[k], js[k]);
    return 0;
}

/* ------------------------------------------------------ uint8 output */

/* Reading R6: clamp to [0, 255], then round half to even. */
void oracle_to_u8(long n, const double *x, uint8_t *y) {
    for (long k = 0; k < n; ++k) {
        double v = x[k];
        if (!(v > 0.0)) v = 0.0;
        if (v > 255.0) v = 255.0;
        y[k] = (uint8_t)nearbyint(v);
    }
}

/* ------------------------------------------------------------ metrics */

/* Images given to the metrics are either FP64 or uint8 (the 8-bit product);
 * every value is read as a double. */
#define ORACLE_F64 0
#define ORACLE_U8 1

static double img_at(const void *base, int type, long idx) {
    return type == ORACLE_U8 ? (double)((const uint8_t *)base)[idx] : ((const double *)base)[idx];
}

static const void *img_plane(const void *base, int type, long offset) {
    return type == ORACLE_U8 ? (const void *)((const uint8_t *)base + offset)
                             : (const void *)((const double *)base + offset);
}

/* ERGAS (Sec. 4, Table 3; the paper gives no formula).  Definition used:
 *   ERGAS = 100 * (d_h / d_l) * sqrt( (1/B) sum_b RMSE_b^2 / mu_b^2 ),
 * d_h / d_l = 1/2 (PAN is twice the MS resolution per side, Sec. 2), the
 * reference for band b is MS_b repeated 2 x 2 to PAN size, RMSE_b is taken
 * over all H x W pixels and mu_b is the mean of that reference.
 * fused: B x H x W; ms: B arrays of H/2 x W/2. */
double oracle_ergas_t(long H, long W, int B, const void *fused, int ftype, const void *const *ms,
                      int mtype) {
    const long W2 = W / 2, n = H * W;
    double acc = 0.0;
    for (int b = 0; b < B; ++b) {
        double se = 0.0, sum = 0.0;
        for (long y = 0; y < H; ++y)
            for (long x = 0; x < W; ++x) {
                const double ref = img_at(ms[b], mtype, (y / 2) * W2 + x / 2);
                const double d = img_at(fused, ftype, (long)b * n + y * W + x) - ref;
                se += d * d;
                sum += ref;
            }
        const double mse = se / (double)n, mu = sum / (double)n;
        acc += mse / (mu * mu);
    }
    return 100.0 * 0.5 * sqrt(acc / (double)B);
}

double oracle_ergas(long H, long W, int B, const double *fused, const double *const *ms) {
    return oracle_ergas_t(H, W, B, fused, ORACLE_F64, (const void *const *)ms, ORACLE_F64);
}

/* Universal image quality index of Wang and Bovik on one window:
 *   Q = 4 s_xy mu_x mu_y / ((s_x^2 + s_y^2) (mu_x^2 + mu_y^2)),
 * population (co)variances.  A zero denominator gives 1 if the two windows are
 * identical and 0 otherwise.  (x0, y0 index the window's top-left pixel.) */
static double q_window(const void *x, int xt, const void *y, int yt, long stride, long off,
                       long win) {
    const double n = (double)(win * win);
    double mx = 0.0, my = 0.0;
    for (long r = 0; r < win; ++r)
        for (long s = 0; s < win; ++s) {
            mx += img_at(x, xt, off + r * stride + s);
            my += img_at(y, yt, off + r * stride + s);
        }
    mx /= n;
    my /= n;
    double vx = 0.0, vy = 0.0, cxy = 0.0;
    int same = 1;
    for (long r = 0; r < win; ++r)
        for (long s = 0; s < win; ++s) {
            const double a = img_at(x, xt, off + r * stride + s);
            const double b = img_at(y, yt, off + r * stride + s);
            vx += (a - mx) * (a - mx);
            vy += (b - my) * (b - my);
            cxy += (a - mx) * (b - my);
            if (a != b) same = 0;
        }
    vx /= n;
    vy /= n;
    cxy /= n;
    const double den = (vx + vy) * (mx * mx + my * my);
    if (den == 0.0) return same ? 1.0 : 0.0;
    return 4.0 * cxy * mx * my / den;
}

/* Q averaged over the non-overlapping win x win windows of two h x w images
 * (windows at multiples of win; a ragged right/bottom edge is dropped).
 * Windows are evaluated in parallel into a per-window array and summed in
 * window order.  Returns NAN if no full window fits. */
double oracle_q_index_t(long h, long w, const void *x, int xt, const void *y, int yt, long win) {
    const long ny = h / win, nx = w / win;
    if (ny < 1 || nx < 1) return NAN;
    double *q = (double *)malloc(sizeof(double) * ny * nx);
    if (!q) return NAN;
#pragma omp parallel for schedule(static)
    for (long k = 0; k < ny * nx; ++k) {
        const long wy = k / nx, wx = k % nx;
        q[k] = q_window(x, xt, y, yt, w, wy * win * w + wx * win, win);
    }
    double acc = 0.0;
    for (long k = 0; k < ny * nx; ++k) acc += q[k];
    free(q);
    return acc / (double)(ny * nx);
}

double oracle_q_index(long h, long w, const double *x, const double *y, long win) {
    return oracle_q_index_t(h, w, x, ORACLE_F64, y, ORACLE_F64, win);
}

/* QNR (Sec. 4, Table 3; the paper gives no formula).  Definition used, with
 * alpha = beta = 1 and p = q = 1:
 *   D_lambda = mean over ordered pairs l != r of |Q(F_l, F_r) - Q(MS_l, MS_r)|
 *   D_s      = mean over l of |Q(F_l, PAN) - Q(MS_l, PAN~)|,
 *              PAN~ = 2 x 2 block mean of PAN (PAN brought to MS size)
 *   QNR      = (1 - D_lambda) (1 - D_s)
 * Q is oracle_q_index with win x win windows, at PAN size for F and PAN and at
 * MS size for MS and PAN~.  B = 1 gives D_lambda = 0.
 * fused: B x H x W (ftype); ms: B arrays of H/2 x W/2 (mtype); pan: H x W (ptype). */
int oracle_qnr_t(long H, long W, int B, const void *fused, int ftype, const void *const *ms,
                 int mtype, const void *pan, int ptype, long win, double *qnr, double *d_lambda,
                 double *d_s) {
    const long H2 = H / 2, W2 = W / 2, n = H * W;
    if (H / win < 1 || W / win < 1 || H2 / win < 1 || W2 / win < 1 || B < 1) return 1;
    double *pan_lo = (double *)malloc(sizeof(double) * H2 * W2);
    if (!pan_lo) return 2;
    for (long i = 0; i < H2; ++i)
        for (long j = 0; j < W2; ++j)
            pan_lo[i * W2 + j] =
                (img_at(pan, ptype, (2 * i) * W + 2 * j) + img_at(pan, ptype, (2 * i) * W + 2 * j + 1) +
                 img_at(pan, ptype, (2 * i + 1) * W + 2 * j) +
                 img_at(pan, ptype, (2 * i + 1) * W + 2 * j + 1)) /
                4.0;
    double dl = 0.0;
    if (B > 1) {
        for (int l = 0; l < B; ++l)
            for (int r = 0; r < B; ++r) {
                if (l == r) continue;
                const double qf = oracle_q_index_t(H, W, img_plane(fused, ftype, (long)l * n), ftype,
                                                   img_plane(fused, ftype, (long)r * n), ftype, win);
                const double qm = oracle_q_index_t(H2, W2, ms[l], mtype, ms[r], mtype, win);
                dl += fabs(qf - qm);
            }
        dl /= (double)(B * (B - 1));
    }
    double ds = 0.0;
    for (int l = 0; l < B; ++l) {
        const double qf =
            oracle_q_index_t(H, W, img_plane(fused, ftype, (long)l * n), ftype, pan, ptype, win);
        const double qm = oracle_q_index_t(H2, W2, ms[l], mtype, pan_lo, ORACLE_F64, win);
        ds += fabs(qf - qm);
    }
    ds /= (double)B;
    free(pan_lo);
    *d_lambda = dl;
    *d_s = ds;
    *qnr = (1.0 - dl) * (1.0 - ds);
    return 0;
}

int oracle_qnr(long H, long W, int B, const double *fused, const double *const *ms,
               const double *pan, long win, double *qnr, double *d_lambda, double *d_s) {
    return oracle_qnr_t(H, W, B, fused, ORACLE_F64, (const void *const *)ms, ORACLE_F64, pan,
                        ORACLE_F64, win, qnr, d_lambda, d_s);
}

/* ------------------------------------------------------------ threads */

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
