/*
 * FP64 CPU oracle of the dense optical-flow velocimetry estimator
 * (Pimienta & Aider, "High Resolution and High-Speed Live Optical Flow
 * Velocimetry", arXiv 2509.25924).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the estimator computes.  Only the tests, the smoke check
 * and the benchmark's CPU-baseline leg may call it; the estimator itself never
 * does.  It shares no source, header, table or helper with the CUDA path.
 *
 * Everything is double precision.  Window sums are direct (every tap of the
 * (2KR+1)^2 box is added), the pyramid filter is applied as its full 5x5
 * kernel, and each step is a separate pass over whole images, in the order of
 * the paper's six-step pipeline (Sec. 2, enumerated list):
 *   1. local intensity normalization          -> orc_normalize
 *   2. Gaussian-pyramid sub-sampling          -> orc_reduce
 *   3. per-pixel LK estimate by Gauss-Newton  -> orc_iterate (Eq. 2)
 *   4. up-sampling and projection             -> orc_upsample
 *   5. steps 3-4 from the coarsest level down -> orc_flow
 *   6. the dense field at full resolution     -> orc_flow outputs
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - window N(m): square (2KR+1)^2 box of uniform weight, truncated at the
 *     image border (terms outside the image count zero); as a variant, the
 *     same box with Gaussian weights exp(-(a^2 + b^2) / (2 sigma^2)) of the
 *     offset (a, b) from the centre (orc_params.win_sigma > 0);
 *   - the warp of Eq. 2 is applied per pixel with the current field V0(k) and
 *     the 2x2 system is solved for V(m) directly:
 *       H V = sum_k G_k (G_k . V0(k) - It_k)
 *     (equal to the increment form V0 + H^-1 sum G (-It) when V0 is constant
 *     over the window; orc_params.increment_form selects the latter);
 *   - image gradients are central differences of the level image, sampled
 *     bilinearly at the warped points and averaged over the two frames;
 *   - interpolation is bilinear with clamp-to-edge taps;
 *   - the pyramid kernel is Burt-Adelson's 5-tap [1 4 6 4 1]/16 with
 *     clamp-to-edge and even-sample decimation, sizes ceil(n/2);
 *   - levels = PSL + 1; the coarse field is carried to the next finer level
 *     as 2 * bilinear(V, x/2, y/2);
 *   - normalization: zero mean, unit deviation over the (2NR+1)^2 box,
 *     I~ = (I - mu) / sqrt(sigma^2 + eps_n^2), eps_n = 1e-2 (parity unpinned);
 *   - guard: if Sxx + Syy <= eps_abs or det <= eps_rel (Sxx + Syy)^2 the
 *     pixel keeps V0(m) (parity unpinned);
 *   - warm start (a variant for time-resolved sequences): the coarsest level
 *     starts from a given level-0 field sampled at the pixels that level
 *     keeps, V_L(i, j) = V(2^L i, 2^L j) / 2^L, instead of from zero;
 *   - region mask (a variant; masked regions such as a model and its shadow,
 *     Sec. 7): the products of a masked pixel are left out of every window
 *     sum (weight 0) at every level, the level-l mask being the level-0 mask
 *     at (2^l i, 2^l j); the output of a masked pixel is NaN (no vector).
 *
 * Build: gcc -O2 -fPIC -shared -fopenmp -ffp-contract=off ofv_oracle.c -lm
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "ofv_oracle.h"

#ifdef _OPENMP
#include <omp.h>
#endif

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static inline int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Pixel value at row i, column j, with clamp-to-edge. */
static inline double at(const double *P, int H, int W, int i, int j)
{
    return P[(int64_t)clampi(i, 0, H - 1) * W + clampi(j, 0, W - 1)];
}

/* ------------------------------------------------------------------ */
/* Step 0: input scaling.  Integer counts of a bits-deep sensor map to    */
/* [0, 1] by raw / (2^bits - 1); bits == 0 means already intensities.     */
/* ------------------------------------------------------------------ */
void orc_scale(int64_t n, const double *raw, int bits, double *out)
{
    double full = bits > 0 ? (double)((1ULL << bits) - 1ULL) : 1.0;
    for (int64_t k = 0; k < n; ++k) out[k] = bits > 0 ? raw[k] / full : raw[k];
}

/* ------------------------------------------------------------------ */
/* Step 1: local pixel-centred intensity normalization of radius NR      */
/* (Sec. 2, pre-processing).  Mean and variance over the in-image part of  */
/* the (2NR+1)^2 box centred on the pixel.                                */
/* ------------------------------------------------------------------ */
void orc_normalize(int H, int W, const double *I, int nr, double eps_n, double *out)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < H; ++i) {
        for (int j = 0; j < W; ++j) {
            double s = 0.0;
            int cnt = 0;
            for (int a = -nr; a <= nr; ++a)
                for (int b = -nr; b <= nr; ++b) {
                    int ii = i + a, jj = j + b;
                    if (ii < 0 || ii >= H || jj < 0 || jj >= W) continue;
                    s += I[(int64_t)ii * W + jj];
                    ++cnt;
                }
            double mu = s / cnt;
            double q = 0.0;
            for (int a = -nr; a <= nr; ++a)
                for (int b = -nr; b <= nr; ++b) {
                    int ii = i + a, jj = j + b;
                    if (ii < 0 || ii >= H || jj < 0 || jj >= W) continue;
                    double d = I[(int64_t)ii * W + jj] - mu;
                    q += d * d;
                }
            double var = q / cnt;
            out[(int64_t)i * W + j] = (I[(int64_t)i * W + j] - mu) / sqrt(var + eps_n * eps_n);
        }
    }
}

/* Optional learnable pre-filter: 5x5 correlation, clamp-to-edge.
   out(i,j) = sum_{a,b=-2..2} w[(a+2)*5 + (b+2)] * I(i+a, j+b). */
void orc_prefilter(int H, int W, const double *I, const double *w25, double *out)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double s = 0.0;
            for (int a = -2; a <= 2; ++a)
                for (int b = -2; b <= 2; ++b)
                    s += w25[(a + 2) * 5 + (b + 2)] * at(I, H, W, i + a, j + b);
            out[(int64_t)i * W + j] = s;
        }
}

/* ------------------------------------------------------------------ */
/* Step 2: one Burt-Adelson reduction (Sec. 2: each sub-level halves both  */
/* dimensions).  out is ceil(H/2) x ceil(W/2):                             */
/*   out(i,j) = sum_{a,b=-2..2} c_a c_b P(2i+a, 2j+b),  c = [1 4 6 4 1]/16  */
/* ------------------------------------------------------------------ */
void orc_reduce(int H, int W, const double *P, double *out)
{
    static const double c[5] = {1.0 / 16, 4.0 / 16, 6.0 / 16, 4.0 / 16, 1.0 / 16};
    int Hc = (H + 1) / 2, Wc = (W + 1) / 2;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < Hc; ++i)
        for (int j = 0; j < Wc; ++j) {
            double s = 0.0;
            for (int a = -2; a <= 2; ++a)
                for (int b = -2; b <= 2; ++b)
                    s += c[a + 2] * c[b + 2] * at(P, H, W, 2 * i + a, 2 * j + b);
            out[(int64_t)i * Wc + j] = s;
        }
}

/* Bilinear sample of P at (px, py) = (column, row), clamp-to-edge taps. */
double orc_bilinear(const double *P, int H, int W, double px, double py)
{
    double fx0 = floor(px), fy0 = floor(py);
    /* far outside the image every tap clamps to the same edge pixel, so the
       position can be limited without changing the value */
    if (!(fx0 >= -2.0)) fx0 = -2.0;
    if (fx0 > W + 1.0) fx0 = W + 1.0;
    if (!(fy0 >= -2.0)) fy0 = -2.0;
    if (fy0 > H + 1.0) fy0 = H + 1.0;
    int x0 = (int)fx0, y0 = (int)fy0;
    double fx = px - floor(px), fy = py - floor(py);
    double p00 = at(P, H, W, y0, x0), p01 = at(P, H, W, y0, x0 + 1);
    double p10 = at(P, H, W, y0 + 1, x0), p11 = at(P, H, W, y0 + 1, x0 + 1);
    return (1.0 - fy) * ((1.0 - fx) * p00 + fx * p01) + fy * ((1.0 - fx) * p10 + fx * p11);
}

/* Central differences of a level image, clamp-to-edge:
   Dx(i,j) = (P(i,j+1) - P(i,j-1)) / 2,  Dy(i,j) = (P(i+1,j) - P(i-1,j)) / 2. */
void orc_central_diff(int H, int W, const double *P, double *Dx, double *Dy)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            Dx[(int64_t)i * W + j] = 0.5 * (at(P, H, W, i, j + 1) - at(P, H, W, i, j - 1));
            Dy[(int64_t)i * W + j] = 0.5 * (at(P, H, W, i + 1, j) - at(P, H, W, i - 1, j));
        }
}

/* Window sum over the (2KR+1)^2 box centred on each pixel, truncated at the
   border (taps outside the image are absent), summed tap by tap. */
void orc_box_sum(int H, int W, const double *in, int kr, double *out)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double s = 0.0;
            for (int a = -kr; a <= kr; ++a) {
                int ii = i + a;
                if (ii < 0 || ii >= H) continue;
                for (int b = -kr; b <= kr; ++b) {
                    int jj = j + b;
                    if (jj < 0 || jj >= W) continue;
                    s += in[(int64_t)ii * W + jj];
                }
            }
            out[(int64_t)i * W + j] = s;
        }
}

/* Window sum with Gaussian weights: out(i,j) = sum over the in-image taps
   (i+a, j+b), |a|, |b| <= KR, of exp(-(a^2 + b^2) / (2 sigma^2)) in(i+a, j+b).
   sigma <= 0 gives the uniform box (orc_box_sum). */
void orc_window_sum(int H, int W, const double *in, int kr, double sigma, double *out)
{
    if (!(sigma > 0.0)) {
        orc_box_sum(H, W, in, kr, out);
        return;
    }
    const double c = 1.0 / (2.0 * sigma * sigma);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double s = 0.0;
            for (int a = -kr; a <= kr; ++a) {
                int ii = i + a;
                if (ii < 0 || ii >= H) continue;
                for (int b = -kr; b <= kr; ++b) {
                    int jj = j + b;
                    if (jj < 0 || jj >= W) continue;
                    s += exp(-(double)(a * a + b * b) * c) * in[(int64_t)ii * W + jj];
                }
            }
            out[(int64_t)i * W + j] = s;
        }
}

/* Region mask at level `level`: the level-0 mask (H x W) at the pixels that
   level keeps, (2^level i, 2^level j), as 0 / 1. */
void orc_decimate_mask(int H, int W, const unsigned char *mask, int level, unsigned char *out)
{
    int Hs[16], Ws[16];
    orc_level_sizes(H, W, level, Hs, Ws);
    const int f = 1 << level;
    for (int i = 0; i < Hs[level]; ++i)
        for (int j = 0; j < Ws[level]; ++j)
            out[(int64_t)i * Ws[level] + j] = mask[(int64_t)(f * i) * W + (int64_t)f * j] ? 1 : 0;
}

/* Warm start: the level-`level` field taken from a level-0 field (H x W) at
   the pixels that level keeps (even-sample decimation `level` times puts
   level pixel i at level-0 pixel 2^level i), in level units (/ 2^level). */
void orc_decimate_field(int H, int W, const double *u, const double *v, int level, double *uc, double *vc)
{
    int Hs[16], Ws[16];
    orc_level_sizes(H, W, level, Hs, Ws);
    const int f = 1 << level;
    for (int i = 0; i < Hs[level]; ++i)
        for (int j = 0; j < Ws[level]; ++j) {
            const int64_t src = (int64_t)(f * i) * W + (int64_t)f * j;
            uc[(int64_t)i * Ws[level] + j] = u[src] / f;
            vc[(int64_t)i * Ws[level] + j] = v[src] / f;
        }
}

/* ------------------------------------------------------------------ */
/* Step 4: carry the field of level l+1 (Hc x Wc) to level l (H x W):     */
/* coarse pixel i sits at fine 2i, so V_l(x, y) = 2 V_{l+1}(x/2, y/2),    */
/* sampled bilinearly with clamp-to-edge.                                 */
/* ------------------------------------------------------------------ */
void orc_upsample(int Hc, int Wc, const double *uc, const double *vc, int H, int W,
                  double *u, double *v)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            u[(int64_t)i * W + j] = 2.0 * orc_bilinear(uc, Hc, Wc, 0.5 * j, 0.5 * i);
            v[(int64_t)i * W + j] = 2.0 * orc_bilinear(vc, Hc, Wc, 0.5 * j, 0.5 * i);
        }
}

/* ------------------------------------------------------------------ */
/* Step 3: one Gauss-Newton iteration of the symmetric SSD of Eq. 2 at one */
/* level.  V0 = (u0, v0) is the current field (per pixel).                 */
/*   p1 = k - V0(k)/2,  p2 = k + V0(k)/2                                   */
/*   A = P1(p1), B = P2(p2), g1 = (Dx P1, Dy P1)(p1), g2 = (Dx P2, Dy P2)(p2)*/
/*   G = (g1 + g2)/2, It = B - A, r = G . V0(k) - It                       */
/* Linearising A(V) - B(V) about V0 gives -It - G.(V - V0); setting the    */
/* gradient of the summed square to zero gives H V = sum G r with           */
/* H = sum G G^T over N(m), solved per pixel by Cramer's rule.              */
/* Optional outputs: ndet = det / (Sxx + Syy)^2 (0 when the trace is       */
/* below eps_abs) and guarded = 1 where V0(m) was kept.                    */
/* ------------------------------------------------------------------ */
int orc_iterate(int H, int W, const double *P1, const double *P2, const double *u0,
                const double *v0, int kr, double win_sigma, double eps_rel, double eps_abs,
                int increment_form, const unsigned char *mask, double *u, double *v, double *ndet,
                unsigned char *guarded)
{
    int64_t N = (int64_t)H * W;
    double *buf = (double *)malloc(sizeof(double) * (size_t)N * 14);
    if (!buf) return 1;
    double *D1x = buf, *D1y = buf + N, *D2x = buf + 2 * N, *D2y = buf + 3 * N;
    double *Gxx = buf + 4 * N, *Gxy = buf + 5 * N, *Gyy = buf + 6 * N;
    double *Gxr = buf + 7 * N, *Gyr = buf + 8 * N;
    double *Sxx = buf + 9 * N, *Sxy = buf + 10 * N, *Syy = buf + 11 * N;
    double *Sxr = buf + 12 * N, *Syr = buf + 13 * N;

    orc_central_diff(H, W, P1, D1x, D1y);
    orc_central_diff(H, W, P2, D2x, D2y);

    /* warp, gradients, residual and the five products at every pixel k */
#pragma omp parallel for schedule(static)
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            int64_t k = (int64_t)i * W + j;
            double uk = u0[k], vk = v0[k];
            double p1x = j - 0.5 * uk, p1y = i - 0.5 * vk;
            double p2x = j + 0.5 * uk, p2y = i + 0.5 * vk;
            double A = orc_bilinear(P1, H, W, p1x, p1y);
            double B = orc_bilinear(P2, H, W, p2x, p2y);
            double g1x = orc_bilinear(D1x, H, W, p1x, p1y);
            double g1y = orc_bilinear(D1y, H, W, p1x, p1y);
            double g2x = orc_bilinear(D2x, H, W, p2x, p2y);
            double g2y = orc_bilinear(D2y, H, W, p2x, p2y);
            double Gx = 0.5 * (g1x + g2x), Gy = 0.5 * (g1y + g2y);
            double It = B - A;
            double r = increment_form ? -It : (Gx * uk + Gy * vk - It);
            double w = (mask && !mask[k]) ? 0.0 : 1.0;  /* masked pixels leave the window sums */
            Gxx[k] = w * Gx * Gx;
            Gxy[k] = w * Gx * Gy;
            Gyy[k] = w * Gy * Gy;
            Gxr[k] = w * Gx * r;
            Gyr[k] = w * Gy * r;
        }

    /* window sums over N(m) */
    orc_window_sum(H, W, Gxx, kr, win_sigma, Sxx);
    orc_window_sum(H, W, Gxy, kr, win_sigma, Sxy);
    orc_window_sum(H, W, Gyy, kr, win_sigma, Syy);
    orc_window_sum(H, W, Gxr, kr, win_sigma, Sxr);
    orc_window_sum(H, W, Gyr, kr, win_sigma, Syr);

    /* guarded 2x2 solve per pixel */
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < N; ++m) {
        double a = Sxx[m], b = Sxy[m], c = Syy[m];
        double tr = a + c;
        double det = a * c - b * b;
        int keep = 0;
        if (!(tr > eps_abs)) keep = 1;
        else if (det <= eps_rel * tr * tr) keep = 1;
        if (ndet) ndet[m] = tr > eps_abs ? det / (tr * tr) : 0.0;
        if (guarded) guarded[m] = (unsigned char)keep;
        if (keep) {
            u[m] = u0[m];
            v[m] = v0[m];
        } else {
            double du = (c * Sxr[m] - b * Syr[m]) / det;
            double dv = (a * Syr[m] - b * Sxr[m]) / det;
            u[m] = increment_form ? u0[m] + du : du;
            v[m] = increment_form ? v0[m] + dv : dv;
        }
    }
    free(buf);
    return 0;
}

/* Ingest one frame: scale, then normalize (NR > 0), then pre-filter. */
static int ingest(int H, int W, const double *raw, const orc_params *p, double *out)
{
    int64_t N = (int64_t)H * W;
    double *t = (double *)malloc(sizeof(double) * (size_t)N);
    if (!t) return 1;
    orc_scale(N, raw, p->bits, out);
    if (p->nr > 0) {
        orc_normalize(H, W, out, p->nr, p->eps_n, t);
        memcpy(out, t, sizeof(double) * (size_t)N);
    }
    if (p->prefilter) {
        orc_prefilter(H, W, out, p->w25, t);
        memcpy(out, t, sizeof(double) * (size_t)N);
    }
    free(t);
    return 0;
}

void orc_level_sizes(int H, int W, int psl, int *Hs, int *Ws)
{
    Hs[0] = H;
    Ws[0] = W;
    for (int l = 1; l <= psl; ++l) {
        Hs[l] = (Hs[l - 1] + 1) / 2;
        Ws[l] = (Ws[l - 1] + 1) / 2;
    }
}

/* Level-0 input images after ingest (for per-step comparisons). */
int orc_ingest(int H, int W, const double *raw, const orc_params *p, double *out)
{
    return ingest(H, W, raw, p, out);
}

/* ------------------------------------------------------------------ */
/* Steps 1-6: the whole estimator on one pair.  raw1/raw2 hold the input   */
/* samples (integer counts as doubles when bits > 0).  u, v (H x W) receive */
/* the displacement in px/frame at each pixel (u along columns, v along    */
/* rows).  ndet (nullable) receives det/(Sxx+Syy)^2 of the last iteration  */
/* at level 0; guard0 (nullable) receives, per pixel, a bit mask of the    */
/* level-0 iterations whose guard kept V0.  Returns 0 on success.           */
/* ------------------------------------------------------------------ */
int orc_flow(int H, int W, const double *raw1, const double *raw2, const orc_params *p,
             double *u, double *v, double *ndet, unsigned char *guard0)
{
    if (H < 1 || W < 1 || p->psl < 0 || p->psl > 15 || p->kr < 0 || p->it < 1) return 2;
    int L = p->psl + 1;
    int Hs[16], Ws[16];
    orc_level_sizes(H, W, p->psl, Hs, Ws);
    int64_t N = (int64_t)H * W;
    double *pyr1[16], *pyr2[16];
    int rc = 0;
    for (int l = 0; l < L; ++l) {
        int64_t n = (int64_t)Hs[l] * Ws[l];
        pyr1[l] = (double *)malloc(sizeof(double) * (size_t)n);
        pyr2[l] = (double *)malloc(sizeof(double) * (size_t)n);
    }
    double *cu = (double *)calloc((size_t)N, sizeof(double));
    double *cv = (double *)calloc((size_t)N, sizeof(double));
    double *nu = (double *)malloc(sizeof(double) * (size_t)N);
    double *nv = (double *)malloc(sizeof(double) * (size_t)N);
    unsigned char *g = (unsigned char *)malloc((size_t)N);
    unsigned char *lm = p->mask ? (unsigned char *)malloc((size_t)N) : NULL;
    if (!cu || !cv || !nu || !nv || !g || (p->mask && !lm)) { rc = 1; goto done; }
    for (int l = 0; l < L; ++l)
        if (!pyr1[l] || !pyr2[l]) { rc = 1; goto done; }

    /* steps 1-2: ingest and pyramid */
    if (ingest(H, W, raw1, p, pyr1[0]) || ingest(H, W, raw2, p, pyr2[0])) { rc = 1; goto done; }
    for (int l = 1; l < L; ++l) {
        orc_reduce(Hs[l - 1], Ws[l - 1], pyr1[l - 1], pyr1[l]);
        orc_reduce(Hs[l - 1], Ws[l - 1], pyr2[l - 1], pyr2[l]);
    }
    if (guard0) memset(guard0, 0, (size_t)N);

    /* steps 3-5: coarse to fine; the coarsest level starts from V = 0, or
       from the decimated initial field (warm start) */
    for (int l = L - 1; l >= 0; --l) {
        int h = Hs[l], w = Ws[l];
        int64_t n = (int64_t)h * w;
        if (l == L - 1 && p->u_init && p->v_init) {
            orc_decimate_field(H, W, p->u_init, p->v_init, l, cu, cv);
        } else if (l == L - 1) {
            memset(cu, 0, sizeof(double) * (size_t)n);
            memset(cv, 0, sizeof(double) * (size_t)n);
        } else {
            /* cu/cv hold the level l+1 field */
            orc_upsample(Hs[l + 1], Ws[l + 1], cu, cv, h, w, nu, nv);
            memcpy(cu, nu, sizeof(double) * (size_t)n);
            memcpy(cv, nv, sizeof(double) * (size_t)n);
        }
        if (lm) orc_decimate_mask(H, W, p->mask, l, lm);
        for (int t = 0; t < p->it; ++t) {
            int last = (l == 0 && t == p->it - 1);
            if (orc_iterate(h, w, pyr1[l], pyr2[l], cu, cv, p->kr, p->win_sigma, p->eps_rel, p->eps_abs,
                            p->increment_form, lm, nu, nv, last ? ndet : NULL, g)) {
                rc = 1;
                goto done;
            }
            if (l == 0 && guard0 && t < 8)
                for (int64_t m = 0; m < n; ++m) guard0[m] |= (unsigned char)(g[m] << t);
            memcpy(cu, nu, sizeof(double) * (size_t)n);
            memcpy(cv, nv, sizeof(double) * (size_t)n);
        }
    }
    /* step 6: the level-0 field; no vector at masked pixels */
    memcpy(u, cu, sizeof(double) * (size_t)N);
    memcpy(v, cv, sizeof(double) * (size_t)N);
    if (p->mask)
        for (int64_t m = 0; m < N; ++m)
            if (!p->mask[m]) u[m] = v[m] = NAN;

done:
    for (int l = 0; l < L; ++l) { free(pyr1[l]); free(pyr2[l]); }
    free(cu); free(cv); free(nu); free(nv); free(g); free(lm);
    return rc;
}

/* Pyramid of one frame after ingest: level l written at out + offset_l,
   offsets packed level after level (sizes from orc_level_sizes). */
int orc_pyramid(int H, int W, const double *raw, const orc_params *p, double *out)
{
    int Hs[16], Ws[16];
    if (p->psl < 0 || p->psl > 15) return 2;
    orc_level_sizes(H, W, p->psl, Hs, Ws);
    if (ingest(H, W, raw, p, out)) return 1;
    double *prev = out;
    for (int l = 1; l <= p->psl; ++l) {
        double *cur = prev + (int64_t)Hs[l - 1] * Ws[l - 1];
        orc_reduce(Hs[l - 1], Ws[l - 1], prev, cur);
        prev = cur;
    }
    return 0;
}

/* ---- quantities derived from a field (Sec. 7) --------------------------- */

/* d f / d x along a row of n samples at unit spacing: central differences
   inside, one-sided differences at the two ends (0 for n = 1). */
static double row_derivative(const double *f, int n, int j, int step)
{
    if (n < 2) return 0.0;
    if (j == 0) return f[step] - f[0];
    if (j == n - 1) return f[(int64_t)(n - 1) * step] - f[(int64_t)(n - 2) * step];
    return 0.5 * (f[(int64_t)(j + 1) * step] - f[(int64_t)(j - 1) * step]);
}

/* Out-of-plane vorticity of the field (u along columns x, v along rows y):
   omega = dv/dx - du/dy (Sec. 7: computed from the instantaneous 2D field). */
void orc_vorticity(int H, int W, const double *u, const double *v, double *omega)
{
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            const double dvdx = row_derivative(v + (int64_t)i * W, W, j, 1);
            const double dudy = row_derivative(u + j, H, i, W);
            omega[(int64_t)i * W + j] = dvdx - dudy;
        }
}

/* Recirculation area of Eq. 6 in pixels: the number of pixels of the region
   (mask[k] != 0, or every pixel when mask is NULL) where u < 0, i.e. where
   the Heaviside function H(-u) is 1. */
int64_t orc_recirculation_count(int H, int W, const double *u, const unsigned char *mask)
{
    int64_t c = 0;
    for (int64_t k = 0; k < (int64_t)H * W; ++k)
        if ((mask == NULL || mask[k] != 0) && u[k] < 0.0) ++c;
    return c;
}
