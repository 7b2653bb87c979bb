/*
 * FP64 reverse mode of the oracle estimator: gradients of a loss
 * L(u, v) with respect to both input frames and the 5x5 pre-filter weights,
 * given dL/du and dL/dv.
 *
 * TEST INFRASTRUCTURE ONLY (see ofv_oracle.c).  The paper has no adjoint;
 * this is the plain chain rule through the forward steps of ofv_oracle.c,
 * written step by step in reverse order, with every intermediate recomputed
 * or stored in full arrays.  Local normalization (NR > 0) is not
 * differentiated (returns 3).
 *
 * Forward recap (ofv_oracle.c):
 *   I = raw * s (s = 1/(2^bits - 1) or 1);  J = w (*) I (5x5 correlation,
 *   clamp-to-edge) or J = I;  P^0 = J, P^{l+1} = reduce(P^l);
 *   stage k (level l, iteration t): V0 = 0 (first stage), 2*bilinear(V^{k-1},
 *   x/2, y/2) (t = 0), or V^{k-1};  V^k = solve(window sums of products);
 *   (u, v) = V^{last}.
 * Derivatives at a bilinear cell boundary use the cell floor() picks; a
 * guarded pixel (V = V0) passes its gradient straight to V0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "ofv_oracle.h"

static inline int cl(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Bilinear sample of P at (px, py) with clamp-to-edge taps (same positions
   and weights as orc_bilinear), returning the value and its derivatives
   with respect to px and py. */
static double bil_d(const double *P, int H, int W, double px, double py, double *dpx, double *dpy, int *xa, int *xb,
                    int *ya, int *yb, double *fx, double *fy)
{
    double fx0 = floor(px), fy0 = floor(py);
    if (!(fx0 >= -2.0)) fx0 = -2.0;
    if (fx0 > W + 1.0) fx0 = W + 1.0;
    if (!(fy0 >= -2.0)) fy0 = -2.0;
    if (fy0 > H + 1.0) fy0 = H + 1.0;
    const int x0 = (int)fx0, y0 = (int)fy0;
    *fx = px - floor(px);
    *fy = py - floor(py);
    *xa = cl(x0, 0, W - 1);
    *xb = cl(x0 + 1, 0, W - 1);
    *ya = cl(y0, 0, H - 1);
    *yb = cl(y0 + 1, 0, H - 1);
    const double p00 = P[(int64_t)*ya * W + *xa], p01 = P[(int64_t)*ya * W + *xb];
    const double p10 = P[(int64_t)*yb * W + *xa], p11 = P[(int64_t)*yb * W + *xb];
    const double a = *fx, b = *fy;
    *dpx = (1.0 - b) * (p01 - p00) + b * (p11 - p10);
    *dpy = ((1.0 - a) * p10 + a * p11) - ((1.0 - a) * p00 + a * p01);
    return (1.0 - b) * ((1.0 - a) * p00 + a * p01) + b * ((1.0 - a) * p10 + a * p11);
}

/* Transpose of the bilinear sample: add g times the tap weights into gP. */
static void bil_scatter(double *gP, int W, int xa, int xb, int ya, int yb, double fx, double fy, double g)
{
    gP[(int64_t)ya * W + xa] += g * (1.0 - fx) * (1.0 - fy);
    gP[(int64_t)ya * W + xb] += g * fx * (1.0 - fy);
    gP[(int64_t)yb * W + xa] += g * (1.0 - fx) * fy;
    gP[(int64_t)yb * W + xb] += g * fx * fy;
}

/* Transpose of the central differences Dx, Dy (clamp-to-edge) added into gP. */
static void central_diff_T(int H, int W, const double *gDx, const double *gDy, double *gP)
{
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            const double gx = 0.5 * gDx[(int64_t)i * W + j], gy = 0.5 * gDy[(int64_t)i * W + j];
            gP[(int64_t)i * W + cl(j + 1, 0, W - 1)] += gx;
            gP[(int64_t)i * W + cl(j - 1, 0, W - 1)] -= gx;
            gP[(int64_t)cl(i + 1, 0, H - 1) * W + j] += gy;
            gP[(int64_t)cl(i - 1, 0, H - 1) * W + j] -= gy;
        }
}

/* Adjoint of one Gauss-Newton stage at one level (direct form of Eq. 2's
   linearisation).  Inputs: level images P1, P2, the stage input field
   (u0, v0), the stage output gradient (gu, gv).  Adds into gP1, gP2 and
   writes the gradient of the stage input field into (gu0, gv0). */
static int stage_adjoint(int H, int W, const double *P1, const double *P2, const double *u0, const double *v0,
                         int kr, double eps_rel, double eps_abs, const double *gu, const double *gv, double *gP1,
                         double *gP2, double *gu0, double *gv0)
{
    const int64_t N = (int64_t)H * W;
    double *buf = (double *)calloc((size_t)N * 26, sizeof(double));
    if (!buf) return 1;
    double *D1x = buf, *D1y = buf + N, *D2x = buf + 2 * N, *D2y = buf + 3 * N;
    double *pr[5], *S[5], *gS[5], *gpr[5];
    for (int c = 0; c < 5; ++c) {
        pr[c] = buf + (4 + c) * N;
        S[c] = buf + (9 + c) * N;
        gS[c] = buf + (14 + c) * N;
        gpr[c] = buf + (19 + c) * N;
    }
    double *gD1x = buf + 24 * N, *gD1y = buf + 25 * N;
    double *gD2x = (double *)calloc((size_t)N * 2, sizeof(double));
    if (!gD2x) {
        free(buf);
        return 1;
    }
    double *gD2y = gD2x + N;
    orc_central_diff(H, W, P1, D1x, D1y);
    orc_central_diff(H, W, P2, D2x, D2y);

    /* forward: products and window sums */
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            const int64_t k = (int64_t)i * W + j;
            const double uk = u0[k], vk = v0[k];
            const double p1x = j - 0.5 * uk, p1y = i - 0.5 * vk, p2x = j + 0.5 * uk, p2y = i + 0.5 * vk;
            const double A = orc_bilinear(P1, H, W, p1x, p1y), B = orc_bilinear(P2, H, W, p2x, p2y);
            const double Gx = 0.5 * (orc_bilinear(D1x, H, W, p1x, p1y) + orc_bilinear(D2x, H, W, p2x, p2y));
            const double Gy = 0.5 * (orc_bilinear(D1y, H, W, p1x, p1y) + orc_bilinear(D2y, H, W, p2x, p2y));
            const double r = Gx * uk + Gy * vk - (B - A);
            pr[0][k] = Gx * Gx;
            pr[1][k] = Gx * Gy;
            pr[2][k] = Gy * Gy;
            pr[3][k] = Gx * r;
            pr[4][k] = Gy * r;
        }
    for (int c = 0; c < 5; ++c) orc_box_sum(H, W, pr[c], kr, S[c]);

    /* adjoint of the guarded solve: V = H^-1 b, so g_b = H^-1 gV = lambda
       and g_H = -lambda V^T (symmetrised for the three entries of H) */
    for (int64_t m = 0; m < N; ++m) {
        const double a = S[0][m], b = S[1][m], c = S[2][m];
        const double tr = a + c, det = a * c - b * b;
        gu0[m] = 0.0;
        gv0[m] = 0.0;
        if (!(tr > eps_abs) || det <= eps_rel * tr * tr) {
            gu0[m] = gu[m];
            gv0[m] = gv[m];
            continue;
        }
        const double Vx = (c * S[3][m] - b * S[4][m]) / det, Vy = (a * S[4][m] - b * S[3][m]) / det;
        const double lx = (c * gu[m] - b * gv[m]) / det, ly = (a * gv[m] - b * gu[m]) / det;
        gS[0][m] = -lx * Vx;
        gS[1][m] = -(lx * Vy + ly * Vx);
        gS[2][m] = -ly * Vy;
        gS[3][m] = lx;
        gS[4][m] = ly;
    }
    /* adjoint of the window sums: the same (symmetric, truncated) box sum */
    for (int c = 0; c < 5; ++c) orc_box_sum(H, W, gS[c], kr, gpr[c]);

    /* adjoint of products, residual, gradients and warps */
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            const int64_t k = (int64_t)i * W + j;
            const double uk = u0[k], vk = v0[k];
            const double p1x = j - 0.5 * uk, p1y = i - 0.5 * vk, p2x = j + 0.5 * uk, p2y = i + 0.5 * vk;
            int xa1, xb1, ya1, yb1, xa2, xb2, ya2, yb2;
            double fx1, fy1, fx2, fy2;
            double dA_x, dA_y, dB_x, dB_y, d1xx, d1xy, d1yx, d1yy, d2xx, d2xy, d2yx, d2yy;
            const double A = bil_d(P1, H, W, p1x, p1y, &dA_x, &dA_y, &xa1, &xb1, &ya1, &yb1, &fx1, &fy1);
            const double B = bil_d(P2, H, W, p2x, p2y, &dB_x, &dB_y, &xa2, &xb2, &ya2, &yb2, &fx2, &fy2);
            const double g1x = bil_d(D1x, H, W, p1x, p1y, &d1xx, &d1xy, &xa1, &xb1, &ya1, &yb1, &fx1, &fy1);
            const double g1y = bil_d(D1y, H, W, p1x, p1y, &d1yx, &d1yy, &xa1, &xb1, &ya1, &yb1, &fx1, &fy1);
            const double g2x = bil_d(D2x, H, W, p2x, p2y, &d2xx, &d2xy, &xa2, &xb2, &ya2, &yb2, &fx2, &fy2);
            const double g2y = bil_d(D2y, H, W, p2x, p2y, &d2yx, &d2yy, &xa2, &xb2, &ya2, &yb2, &fx2, &fy2);
            const double Gx = 0.5 * (g1x + g2x), Gy = 0.5 * (g1y + g2y);
            const double It = B - A;
            const double r = Gx * uk + Gy * vk - It;
            const double q0 = gpr[0][k], q1 = gpr[1][k], q2 = gpr[2][k], q3 = gpr[3][k], q4 = gpr[4][k];
            const double gr = Gx * q3 + Gy * q4;
            const double gGx = 2.0 * Gx * q0 + Gy * q1 + r * q3 + uk * gr;
            const double gGy = Gx * q1 + 2.0 * Gy * q2 + r * q4 + vk * gr;
            const double gIt = -gr;
            const double gA = -gIt, gB = gIt;
            const double gg1x = 0.5 * gGx, gg2x = 0.5 * gGx, gg1y = 0.5 * gGy, gg2y = 0.5 * gGy;
            /* field: direct term of r, then the positions p1 = k - V0/2, p2 = k + V0/2 */
            const double dp1x = gA * dA_x + gg1x * d1xx + gg1y * d1yx;
            const double dp1y = gA * dA_y + gg1x * d1xy + gg1y * d1yy;
            const double dp2x = gB * dB_x + gg2x * d2xx + gg2y * d2yx;
            const double dp2y = gB * dB_y + gg2x * d2xy + gg2y * d2yy;
            gu0[k] += Gx * gr - 0.5 * dp1x + 0.5 * dp2x;
            gv0[k] += Gy * gr - 0.5 * dp1y + 0.5 * dp2y;
            /* images: value taps and gradient-image taps */
            bil_scatter(gP1, W, xa1, xb1, ya1, yb1, fx1, fy1, gA);
            bil_scatter(gP2, W, xa2, xb2, ya2, yb2, fx2, fy2, gB);
            bil_scatter(gD1x, W, xa1, xb1, ya1, yb1, fx1, fy1, gg1x);
            bil_scatter(gD1y, W, xa1, xb1, ya1, yb1, fx1, fy1, gg1y);
            bil_scatter(gD2x, W, xa2, xb2, ya2, yb2, fx2, fy2, gg2x);
            bil_scatter(gD2y, W, xa2, xb2, ya2, yb2, fx2, fy2, gg2y);
        }
    central_diff_T(H, W, gD1x, gD1y, gP1);
    central_diff_T(H, W, gD2x, gD2y, gP2);
    free(buf);
    free(gD2x);
    return 0;
}

/* Transpose of orc_upsample: (gu, gv) on the fine H x W grid to the coarse
   Hc x Wc grid (added into guc, gvc). */
static void upsample_T(int Hc, int Wc, int H, int W, const double *gu, const double *gv, double *guc, double *gvc)
{
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double dx, dy, fx, fy;
            int xa, xb, ya, yb;
            (void)bil_d(guc, Hc, Wc, 0.5 * j, 0.5 * i, &dx, &dy, &xa, &xb, &ya, &yb, &fx, &fy);
            bil_scatter(guc, Wc, xa, xb, ya, yb, fx, fy, 2.0 * gu[(int64_t)i * W + j]);
            bil_scatter(gvc, Wc, xa, xb, ya, yb, fx, fy, 2.0 * gv[(int64_t)i * W + j]);
        }
}

/* Transpose of orc_reduce: gradient of level l+1 (Hc x Wc) added into
   level l (H x W). */
static void reduce_T(int H, int W, const double *gc, double *g)
{
    static const double c[5] = {1.0 / 16, 4.0 / 16, 6.0 / 16, 4.0 / 16, 1.0 / 16};
    const int Hc = (H + 1) / 2, Wc = (W + 1) / 2;
    for (int i = 0; i < Hc; ++i)
        for (int j = 0; j < Wc; ++j) {
            const double v = gc[(int64_t)i * Wc + j];
            for (int a = -2; a <= 2; ++a)
                for (int b = -2; b <= 2; ++b)
                    g[(int64_t)cl(2 * i + a, 0, H - 1) * W + cl(2 * j + b, 0, W - 1)] += c[a + 2] * c[b + 2] * v;
        }
}

/* Adjoint of the local normalization of Sec. 2 (step 1, orc_normalize):
   J(m) = (I(m) - mu(m)) / s(m), s = sqrt(var(m) + eps_n^2), where mu(m) and
   var(m) are the mean and variance of I over the in-image part B(m) of the
   (2NR+1)^2 box centred on m, of n(m) pixels.  By the chain rule, with
   a = dL/dJ and var = sum_B I^2 / n - mu^2,
     dL/dI(k) = a(k) / s(k)
                - sum_{m : k in B(m)} a(m) [1 / (s(m) n(m))
                                            + J(m) (I(k) - mu(m)) / (s(m)^2 n(m))],
   and k lies in B(m) exactly when m lies in B(k).  gI receives dL/dI. */
static int normalize_T(int H, int W, const double *I, int nr, double eps_n, const double *gJ, double *gI)
{
    const int64_t N = (int64_t)H * W;
    double *mu = (double *)malloc(sizeof(double) * N), *sd = (double *)malloc(sizeof(double) * N);
    double *cnt = (double *)malloc(sizeof(double) * N);
    if (!mu || !sd || !cnt) { free(mu); free(sd); free(cnt); return 1; }
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double sum = 0.0;
            int n = 0;
            for (int a = -nr; a <= nr; ++a)
                for (int b = -nr; b <= nr; ++b) {
                    const int ii = i + a, jj = j + b;
                    if (ii < 0 || ii >= H || jj < 0 || jj >= W) continue;
                    sum += I[(int64_t)ii * W + jj];
                    ++n;
                }
            const double m = sum / n;
            double q = 0.0;
            for (int a = -nr; a <= nr; ++a)
                for (int b = -nr; b <= nr; ++b) {
                    const int ii = i + a, jj = j + b;
                    if (ii < 0 || ii >= H || jj < 0 || jj >= W) continue;
                    const double d = I[(int64_t)ii * W + jj] - m;
                    q += d * d;
                }
            mu[(int64_t)i * W + j] = m;
            sd[(int64_t)i * W + j] = sqrt(q / n + eps_n * eps_n);
            cnt[(int64_t)i * W + j] = (double)n;
        }
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            const int64_t k = (int64_t)i * W + j;
            double g = gJ[k] / sd[k];
            for (int a = -nr; a <= nr; ++a)
                for (int b = -nr; b <= nr; ++b) {
                    const int ii = i + a, jj = j + b;
                    if (ii < 0 || ii >= H || jj < 0 || jj >= W) continue;
                    const int64_t m = (int64_t)ii * W + jj;
                    const double Jm = (I[m] - mu[m]) / sd[m];
                    g -= gJ[m] / (sd[m] * cnt[m]) + gJ[m] * Jm * (I[k] - mu[m]) / (sd[m] * sd[m] * cnt[m]);
                }
            gI[k] = g;
        }
    free(mu); free(sd); free(cnt);
    return 0;
}

/* Gradients of L with respect to raw1, raw2 (H x W) and, when the
   pre-filter is on, its 25 weights (gw25, nullable), given gu = dL/du and
   gv = dL/dv.  u, v (nullable) receive the forward field.  Returns 0, 3 for
   an estimator variant (it covers the direct form, box window, from V = 0,
   no mask), 2 for bad parameters, 1 when out of memory. */
int orc_flow_grad(int H, int W, const double *raw1, const double *raw2, const orc_params *p, const double *gu,
                  const double *gv, double *g1, double *g2, double *gw25, double *u, double *v)
{
    if (H < 1 || W < 1 || p->psl < 0 || p->psl > 15 || p->kr < 0 || p->it < 1) return 2;
    /* the reverse mode covers the direct form with the uniform box, from V = 0 */
    if (p->increment_form || p->win_sigma > 0.0 || p->u_init || p->v_init || p->mask) return 3;
    const int L = p->psl + 1, S = L * p->it;
    int Hs[16], Ws[16];
    orc_level_sizes(H, W, p->psl, Hs, Ws);
    const int64_t N = (int64_t)H * W;
    int rc = 0;
    double *I1 = (double *)malloc(sizeof(double) * N), *I2 = (double *)malloc(sizeof(double) * N);
    double *pyr1[16] = {0}, *pyr2[16] = {0}, *gp1[16] = {0}, *gp2[16] = {0};
    double **V = (double **)calloc((size_t)S * 2, sizeof(double *));     /* stage outputs u, v */
    double **V0 = (double **)calloc((size_t)S * 2, sizeof(double *));    /* stage inputs u, v */
    double *gu_c = (double *)calloc((size_t)N, sizeof(double)), *gv_c = (double *)calloc((size_t)N, sizeof(double));
    double *gu_n = (double *)calloc((size_t)N, sizeof(double)), *gv_n = (double *)calloc((size_t)N, sizeof(double));
    double *t = (double *)malloc(sizeof(double) * N);
    double *N1 = NULL, *N2 = NULL;
    if (!I1 || !I2 || !V || !V0 || !gu_c || !gv_c || !gu_n || !gv_n || !t) { rc = 1; goto done; }
    for (int l = 0; l < L; ++l) {
        const int64_t n = (int64_t)Hs[l] * Ws[l];
        pyr1[l] = (double *)malloc(sizeof(double) * n);
        pyr2[l] = (double *)malloc(sizeof(double) * n);
        gp1[l] = (double *)calloc((size_t)n, sizeof(double));
        gp2[l] = (double *)calloc((size_t)n, sizeof(double));
        if (!pyr1[l] || !pyr2[l] || !gp1[l] || !gp2[l]) { rc = 1; goto done; }
    }
    for (int s = 0; s < S; ++s) {
        const int l = L - 1 - s / p->it;
        const int64_t n = (int64_t)Hs[l] * Ws[l];
        for (int k = 0; k < 2; ++k) {
            V[2 * s + k] = (double *)malloc(sizeof(double) * n);
            V0[2 * s + k] = (double *)calloc((size_t)n, sizeof(double));
            if (!V[2 * s + k] || !V0[2 * s + k]) { rc = 1; goto done; }
        }
    }

    /* forward, keeping every stage's input and output field; I1, I2 hold the
       scaled frames, N1, N2 the normalized ones (the pre-filter's input) */
    orc_scale(N, raw1, p->bits, I1);
    orc_scale(N, raw2, p->bits, I2);
    if (p->nr > 0) {
        N1 = (double *)malloc(sizeof(double) * N);
        N2 = (double *)malloc(sizeof(double) * N);
        if (!N1 || !N2) { rc = 1; goto done; }
        orc_normalize(H, W, I1, p->nr, p->eps_n, N1);
        orc_normalize(H, W, I2, p->nr, p->eps_n, N2);
    }
    const double *F1 = p->nr > 0 ? N1 : I1, *F2 = p->nr > 0 ? N2 : I2;
    if (p->prefilter) {
        orc_prefilter(H, W, F1, p->w25, pyr1[0]);
        orc_prefilter(H, W, F2, p->w25, pyr2[0]);
    } else {
        memcpy(pyr1[0], F1, sizeof(double) * N);
        memcpy(pyr2[0], F2, sizeof(double) * N);
    }
    for (int l = 1; l < L; ++l) {
        orc_reduce(Hs[l - 1], Ws[l - 1], pyr1[l - 1], pyr1[l]);
        orc_reduce(Hs[l - 1], Ws[l - 1], pyr2[l - 1], pyr2[l]);
    }
    for (int s = 0; s < S; ++s) {
        const int l = L - 1 - s / p->it, it = s % p->it;
        if (s > 0 && it == 0)
            orc_upsample(Hs[l + 1], Ws[l + 1], V[2 * (s - 1)], V[2 * (s - 1) + 1], Hs[l], Ws[l], V0[2 * s],
                         V0[2 * s + 1]);
        else if (s > 0) {
            memcpy(V0[2 * s], V[2 * (s - 1)], sizeof(double) * (size_t)Hs[l] * Ws[l]);
            memcpy(V0[2 * s + 1], V[2 * (s - 1) + 1], sizeof(double) * (size_t)Hs[l] * Ws[l]);
        }
        if (orc_iterate(Hs[l], Ws[l], pyr1[l], pyr2[l], V0[2 * s], V0[2 * s + 1], p->kr, 0.0, p->eps_rel, p->eps_abs, 0, NULL,
                        V[2 * s], V[2 * s + 1], NULL, NULL)) { rc = 1; goto done; }
    }
    if (u) memcpy(u, V[2 * (S - 1)], sizeof(double) * N);
    if (v) memcpy(v, V[2 * (S - 1) + 1], sizeof(double) * N);

    /* reverse */
    memcpy(gu_c, gu, sizeof(double) * N);
    memcpy(gv_c, gv, sizeof(double) * N);
    for (int s = S - 1; s >= 0; --s) {
        const int l = L - 1 - s / p->it, it = s % p->it;
        const int64_t n = (int64_t)Hs[l] * Ws[l];
        if (stage_adjoint(Hs[l], Ws[l], pyr1[l], pyr2[l], V0[2 * s], V0[2 * s + 1], p->kr, p->eps_rel, p->eps_abs,
                          gu_c, gv_c, gp1[l], gp2[l], gu_n, gv_n)) { rc = 1; goto done; }
        if (s == 0) break;
        if (it > 0) {
            memcpy(gu_c, gu_n, sizeof(double) * n);
            memcpy(gv_c, gv_n, sizeof(double) * n);
        } else {
            const int64_t nc = (int64_t)Hs[l + 1] * Ws[l + 1];
            memset(gu_c, 0, sizeof(double) * nc);
            memset(gv_c, 0, sizeof(double) * nc);
            upsample_T(Hs[l + 1], Ws[l + 1], Hs[l], Ws[l], gu_n, gv_n, gu_c, gv_c);
        }
    }
    for (int l = L - 1; l >= 1; --l) {
        reduce_T(Hs[l - 1], Ws[l - 1], gp1[l], gp1[l - 1]);
        reduce_T(Hs[l - 1], Ws[l - 1], gp2[l], gp2[l - 1]);
    }
    /* pre-filter: J(i,j) = sum w[a][b] F(i+a, j+b) (clamped), F the
       normalized frame (or the scaled one when NR = 0); then the
       normalization adjoint and the input scale */
    for (int f = 0; f < 2; ++f) {
        const double *gJ = f ? gp2[0] : gp1[0];
        const double *I = f ? F2 : F1;
        double *gI = p->nr > 0 ? t : (f ? g2 : g1);
        if (p->prefilter) {
            memset(gI, 0, sizeof(double) * N);
            for (int i = 0; i < H; ++i)
                for (int j = 0; j < W; ++j) {
                    const double g = gJ[(int64_t)i * W + j];
                    for (int a = -2; a <= 2; ++a)
                        for (int b = -2; b <= 2; ++b) {
                            const int64_t src = (int64_t)cl(i + a, 0, H - 1) * W + cl(j + b, 0, W - 1);
                            gI[src] += p->w25[(a + 2) * 5 + (b + 2)] * g;
                            if (gw25) gw25[(a + 2) * 5 + (b + 2)] += g * I[src];
                        }
                }
        } else {
            memcpy(gI, gJ, sizeof(double) * N);
        }
        if (p->nr > 0) {
            gI = f ? g2 : g1;
            if (normalize_T(H, W, f ? I2 : I1, p->nr, p->eps_n, t, gI)) { rc = 1; goto done; }
        }
        if (p->bits > 0) {
            const double sc = 1.0 / (double)((1ULL << p->bits) - 1ULL);
            for (int64_t k = 0; k < N; ++k) gI[k] *= sc;
        }
    }

done:
    free(N1); free(N2);
    for (int l = 0; l < 16; ++l) { free(pyr1[l]); free(pyr2[l]); free(gp1[l]); free(gp2[l]); }
    if (V) for (int s = 0; s < 2 * S; ++s) free(V[s]);
    if (V0) for (int s = 0; s < 2 * S; ++s) free(V0[s]);
    free(V); free(V0); free(I1); free(I2); free(gu_c); free(gv_c); free(gu_n); free(gv_n); free(t);
    return rc;
}
