/*
 * Seeded synthetic PIV image generator.
 *
 * This module produces the inputs that both the FP64 oracle and the CUDA
 * estimator consume: particle images of analytically displaced particles,
 * and the analytic displacement fields themselves.  It contains none of the
 * estimator's arithmetic (no pyramid, warp, gradient, window sum or solve).
 *
 * Conventions
 *   - Pixel (i, j) is row i, column j; its centre is at (x, y) = (j, i) and it
 *     covers [j-1/2, j+1/2] x [i-1/2, i+1/2].
 *   - A displacement field d(x, y) = (dx, dy) is given in px/frame and is
 *     attributed to the midpoint between the two exposures: a particle whose
 *     midpoint is p is drawn at p - d(p)/2 in frame 1 and at p + d(p)/2 in
 *     frame 2 (symmetric formulation, Eq. 2).
 *   - Particles are Gaussian blobs whose diameter is read as the FWHM,
 *     FWHM = 2 sqrt(2 ln 2) sigma (Sec. 4.2).  The pixel value is the blob's
 *     average over the pixel footprint (product of erf differences).
 *   - Random numbers come from a counter-based generator: the splitmix64
 *     finaliser of Steele, Lea and Flood (OOPSLA 2014) applied to a
 *     (seed, stream, index) counter, so every draw is reproducible and
 *     independent of thread count.
 *
 * Build: gcc -O2 -fPIC -shared -fopenmp -ffp-contract=off synth.c -lm
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* counter-based random numbers                                        */
/* ------------------------------------------------------------------ */
static inline uint64_t mix64(uint64_t z)
{
    z += 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static inline uint64_t ctr_hash(uint64_t seed, uint64_t stream, uint64_t i)
{
    return mix64(mix64(seed ^ mix64(stream * 0xd1b54a32d192ed03ULL)) ^ i);
}

/* uniform double in [0, 1) */
static inline double ctr_u01(uint64_t seed, uint64_t stream, uint64_t i)
{
    return (double)(ctr_hash(seed, stream, i) >> 11) * 0x1.0p-53;
}

/* standard normal by Box-Muller from two uniforms of the same counter */
static inline double ctr_normal(uint64_t seed, uint64_t stream, uint64_t i)
{
    double u1 = ctr_u01(seed, stream, 2 * i);
    double u2 = ctr_u01(seed, stream, 2 * i + 1);
    if (u1 < 1e-300) u1 = 1e-300;
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

void syn_uniform(uint64_t seed, uint64_t stream, int64_t n, double lo, double hi, double *out)
{
    for (int64_t i = 0; i < n; ++i)
        out[i] = lo + (hi - lo) * ctr_u01(seed, stream, (uint64_t)i);
}

void syn_normal(uint64_t seed, uint64_t stream, int64_t n, double *out)
{
    for (int64_t i = 0; i < n; ++i)
        out[i] = ctr_normal(seed, stream, (uint64_t)i);
}

/* ------------------------------------------------------------------ */
/* analytic displacement fields                                        */
/* ------------------------------------------------------------------ */
typedef struct {
    /* uniform translation */
    double ux, uy;
    /* Rankine vortex: centre, core radius R, peak azimuthal displacement
       dmax reached at r = R (Sec. 4.1 box: u_theta = G/(2 pi M R) * {r/R, R/r},
       with G/(2 pi M R) chosen equal to dmax).  Off when R <= 0. */
    double rk_cx, rk_cy, rk_R, rk_dmax;
    /* stream-function turbulence psi = sum_n A_n cos(k_n . x + phi_n);
       u = d psi / dy, v = - d psi / dx.  Off when turb_n == 0. */
    int64_t turb_n;
    const double *turb_kx, *turb_ky, *turb_amp, *turb_phase;
    /* potential flow round a cylinder of radius cyl_a centred at
       (cyl_cx, cyl_cy) with free stream cyl_uinf along +x.  Off when a <= 0 */
    double cyl_cx, cyl_cy, cyl_a, cyl_uinf;
    /* Lamb-Oseen vortices: u_theta = G/(2 pi r) (1 - exp(-r^2/rc^2)) */
    int64_t lo_n;
    const double *lo_x, *lo_y, *lo_gamma;
    double lo_rc;
    /* overall multiplier applied to the sum of all parts */
    double scale;
    /* when grid_h > 0 the field is instead the bilinear interpolation
       (clamp-to-edge) of displacements sampled at every pixel centre of a
       grid_h x grid_w grid (used to advect long particle streams cheaply) */
    int64_t grid_h, grid_w;
    const double *grid_u, *grid_v;
} syn_field;

static void grid_at(const syn_field *f, double x, double y, double *dx, double *dy)
{
    double fx0 = floor(x), fy0 = floor(y);
    double fx = x - fx0, fy = y - fy0;
    int64_t x0 = (int64_t)fx0, y0 = (int64_t)fy0;
    int64_t xa = x0 < 0 ? 0 : (x0 > f->grid_w - 1 ? f->grid_w - 1 : x0);
    int64_t xb = x0 + 1 < 0 ? 0 : (x0 + 1 > f->grid_w - 1 ? f->grid_w - 1 : x0 + 1);
    int64_t ya = y0 < 0 ? 0 : (y0 > f->grid_h - 1 ? f->grid_h - 1 : y0);
    int64_t yb = y0 + 1 < 0 ? 0 : (y0 + 1 > f->grid_h - 1 ? f->grid_h - 1 : y0 + 1);
    const double *U = f->grid_u, *V = f->grid_v;
    int64_t W = f->grid_w;
    *dx = (1 - fy) * ((1 - fx) * U[ya * W + xa] + fx * U[ya * W + xb]) +
          fy * ((1 - fx) * U[yb * W + xa] + fx * U[yb * W + xb]);
    *dy = (1 - fy) * ((1 - fx) * V[ya * W + xa] + fx * V[ya * W + xb]) +
          fy * ((1 - fx) * V[yb * W + xa] + fx * V[yb * W + xb]);
}

/* Rankine displacement at midpoint (x, y).  A particle at radius r turns by
   phi(r) = u_theta(r) / r about the centre; frame 1 and frame 2 hold it at
   -phi/2 and +phi/2.  The chord joining them has its midpoint at radius
   rho = r cos(phi/2) and length 2 r sin(phi/2), tangential.  Given the
   midpoint radius rho, r is found by fixed-point iteration. */
static void rankine_at(const syn_field *f, double x, double y, double *dx, double *dy)
{
    double X = x - f->rk_cx, Y = y - f->rk_cy;
    double rho = sqrt(X * X + Y * Y);
    if (rho <= 0.0) { *dx = 0.0; *dy = 0.0; return; }
    double R = f->rk_R, D = f->rk_dmax;
    double r = rho;
    double phi = 0.0;
    for (int it = 0; it < 60; ++it) {
        double ut = (r <= R) ? D * (r / R) : D * (R / r);
        phi = ut / r;
        double rn = rho / cos(0.5 * phi);
        if (fabs(rn - r) < 1e-15 * (1.0 + r)) { r = rn; break; }
        r = rn;
    }
    {
        double ut = (r <= R) ? D * (r / R) : D * (R / r);
        phi = ut / r;
    }
    double mag = 2.0 * r * sin(0.5 * phi);
    /* tangential unit vector for a positive rotation (x toward y) */
    *dx = -mag * (Y / rho);
    *dy = mag * (X / rho);
}

void syn_field_eval(const syn_field *f, int64_t n, const double *x, const double *y,
                    double *dx, double *dy)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double px = x[i], py = y[i];
        if (f->grid_h > 0) {
            double gx, gy;
            grid_at(f, px, py, &gx, &gy);
            dx[i] = f->scale * gx;
            dy[i] = f->scale * gy;
            continue;
        }
        double sx = f->ux, sy = f->uy;
        if (f->rk_R > 0.0) {
            double ax, ay;
            rankine_at(f, px, py, &ax, &ay);
            sx += ax; sy += ay;
        }
        for (int64_t m = 0; m < f->turb_n; ++m) {
            double s = sin(f->turb_kx[m] * px + f->turb_ky[m] * py + f->turb_phase[m]);
            /* psi = A cos(theta): d psi/dy = -A ky sin, -d psi/dx = A kx sin */
            sx += -f->turb_amp[m] * f->turb_ky[m] * s;
            sy += f->turb_amp[m] * f->turb_kx[m] * s;
        }
        if (f->cyl_a > 0.0) {
            /* complex velocity u - i v = U (1 - a^2 / z^2) */
            double zx = px - f->cyl_cx, zy = py - f->cyl_cy;
            double r2 = zx * zx + zy * zy;
            if (r2 > 0.0) {
                /* 1/z^2 = conj(z)^2 / |z|^4 */
                double re = (zx * zx - zy * zy) / (r2 * r2);
                double im = (-2.0 * zx * zy) / (r2 * r2);
                double a2 = f->cyl_a * f->cyl_a;
                double wre = f->cyl_uinf * (1.0 - a2 * re);
                double wim = f->cyl_uinf * (-a2 * im);
                sx += wre;
                sy += -wim;
            }
        }
        for (int64_t m = 0; m < f->lo_n; ++m) {
            double X = px - f->lo_x[m], Y = py - f->lo_y[m];
            double r2 = X * X + Y * Y;
            if (r2 <= 0.0) continue;
            double rc2 = f->lo_rc * f->lo_rc;
            /* u_theta / r = G/(2 pi r^2) (1 - exp(-r^2/rc^2)) */
            double w = f->lo_gamma[m] / (6.283185307179586 * r2) * (1.0 - exp(-r2 / rc2));
            sx += -w * Y;
            sy += w * X;
        }
        dx[i] = f->scale * sx;
        dy[i] = f->scale * sy;
    }
}

/* ------------------------------------------------------------------ */
/* particles                                                           */
/* ------------------------------------------------------------------ */

/* Seeded particle set: midpoint positions uniform over [x0,x1) x [y0,y1),
   FWHM diameter uniform in [dmin, dmax], peak intensity uniform in
   [amin, amax].  sigma = diameter / (2 sqrt(2 ln 2)). */
void syn_particles(uint64_t seed, int64_t n, double x0, double x1, double y0, double y1,
                   double dmin, double dmax, double amin, double amax,
                   double *x, double *y, double *sigma, double *amp)
{
    const double fwhm_per_sigma = 2.0 * sqrt(2.0 * log(2.0));
    for (int64_t i = 0; i < n; ++i) {
        x[i] = x0 + (x1 - x0) * ctr_u01(seed, 1, (uint64_t)i);
        y[i] = y0 + (y1 - y0) * ctr_u01(seed, 2, (uint64_t)i);
        double d = dmin + (dmax - dmin) * ctr_u01(seed, 3, (uint64_t)i);
        sigma[i] = d / fwhm_per_sigma;
        amp[i] = amin + (amax - amin) * ctr_u01(seed, 4, (uint64_t)i);
    }
}

/* Accumulate n pixel-integrated Gaussian blobs into rows [r0, r1) of img
   (H x W, row-major).  The average over pixel [j-1/2, j+1/2] x [i-1/2, i+1/2]
   of amp * exp(-|X - p|^2 / (2 sigma^2)) is amp * (pi/2) sigma^2 * Ex(j) * Ey(i)
   with Ex(j) = erf((j+1/2-x)/(sqrt2 sigma)) - erf((j-1/2-x)/(sqrt2 sigma)).
   Each pixel receives its contributions in particle order. */
static void render_rows(int H, int W, int r0, int r1, int64_t n, const double *x,
                        const double *y, const double *sigma, const double *amp, double *img)
{
    double ex[64], ey[64];
    for (int64_t p = 0; p < n; ++p) {
        double s = sigma[p];
        int rad = (int)ceil(4.0 * s + 1.0);
        if (rad > 31) rad = 31;
        int jc = (int)floor(x[p] + 0.5), ic = (int)floor(y[p] + 0.5);
        int j0 = jc - rad, j1 = jc + rad, i0 = ic - rad, i1 = ic + rad;
        if (i0 < r0) i0 = r0;
        if (i1 > r1 - 1) i1 = r1 - 1;
        if (j0 < 0) j0 = 0;
        if (j1 > W - 1) j1 = W - 1;
        if (j1 < j0 || i1 < i0) continue;
        double inv = 1.0 / (sqrt(2.0) * s);
        /* adjacent pixels share a boundary: one erf per pixel edge */
        double lo = erf((j0 - 0.5 - x[p]) * inv);
        for (int j = j0; j <= j1; ++j) {
            double hi = erf((j + 0.5 - x[p]) * inv);
            ex[j - j0] = hi - lo;
            lo = hi;
        }
        lo = erf((i0 - 0.5 - y[p]) * inv);
        for (int i = i0; i <= i1; ++i) {
            double hi = erf((i + 0.5 - y[p]) * inv);
            ey[i - i0] = hi - lo;
            lo = hi;
        }
        /* amp * (pi/2) sigma^2 */
        double a = amp[p] * 1.5707963267948966 * s * s;
        for (int i = i0; i <= i1; ++i) {
            double wy = a * ey[i - i0];
            double *row = img + (int64_t)i * W;
            for (int j = j0; j <= j1; ++j) row[j] += wy * ex[j - j0];
        }
    }
    (void)H;
}

/* Accumulate n blobs into the whole image; threads own bands of rows, so the
   result does not depend on the thread count. */
void syn_render(int H, int W, int64_t n, const double *x, const double *y,
                const double *sigma, const double *amp, double *img)
{
    int nb = 1;
#ifdef _OPENMP
    nb = omp_get_max_threads();
#endif
    if (nb > H) nb = H;
    if (nb < 1) nb = 1;
#pragma omp parallel for schedule(static, 1)
    for (int b = 0; b < nb; ++b) {
        int r0 = (int)((int64_t)H * b / nb), r1 = (int)((int64_t)H * (b + 1) / nb);
        render_rows(H, W, r0, r1, n, x, y, sigma, amp, img);
    }
}

/* Turn an accumulated image into a frame: add Gaussian noise of standard
   deviation noise_sigma (full scale = 1) drawn from counter stream
   (seed, stream), clip to [0, 1], then
     out_kind 0: float32 in [0, 1];
     out_kind 1: uint16 = round(I * (2^bits - 1));
     out_kind 2: uint8  = round(I * (2^bits - 1)). */
void syn_finalize(int H, int W, const double *img, double noise_sigma, uint64_t seed,
                  uint64_t stream, int bits, int out_kind, void *out)
{
    int64_t N = (int64_t)H * W;
    double full = (double)((1u << bits) - 1u);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < N; ++k) {
        double v = img[k];
        if (noise_sigma > 0.0) v += noise_sigma * ctr_normal(seed, stream, (uint64_t)k);
        if (v < 0.0) v = 0.0;
        if (v > 1.0) v = 1.0;
        if (out_kind == 0) {
            ((float *)out)[k] = (float)v;
        } else if (out_kind == 1) {
            ((uint16_t *)out)[k] = (uint16_t)floor(v * full + 0.5);
        } else {
            ((uint8_t *)out)[k] = (uint8_t)floor(v * full + 0.5);
        }
    }
}

/* Frame positions of particles with midpoints (x, y): frame 1 at p - d/2,
   frame 2 at p + d/2. */
void syn_pair_positions(const syn_field *f, int64_t n, const double *x, const double *y,
                        double *x1, double *y1, double *x2, double *y2)
{
    double *dx = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *dy = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    syn_field_eval(f, n, x, y, dx, dy);
    for (int64_t i = 0; i < n; ++i) {
        x1[i] = x[i] - 0.5 * dx[i];
        y1[i] = y[i] - 0.5 * dy[i];
        x2[i] = x[i] + 0.5 * dx[i];
        y2[i] = y[i] + 0.5 * dy[i];
    }
    free(dx);
    free(dy);
}

/* Time-resolved sequence of n_frames frames of a steady field.  Particle
   positions start at (x, y) (frame 0) and advance by the explicit midpoint
   rule X' = X + d(X + d(X)/2), so that the displacement between consecutive
   frames is the field at the chord midpoint to second order.  A particle
   leaving the extended domain [-margin, W+margin) x [-margin, H+margin) is
   wrapped to the opposite side; with margin larger than the blob radius plus
   the largest displacement it is invisible in both frames of that pair.
   Frames are written to out (n_frames x H x W of the out_kind element type).
   Frame f's noise uses counter stream (noise_seed, f).  Frames are rendered
   in parallel, chunk by chunk. */
int syn_stream(int H, int W, int n_frames, int64_t n, const double *x0, const double *y0,
               const double *sigma, const double *amp, const syn_field *f, double margin,
               double noise_sigma, uint64_t noise_seed, int bits, int out_kind, void *out)
{
    int nt = 1;
#ifdef _OPENMP
    nt = omp_get_max_threads();
#endif
    if (nt < 1) nt = 1;
    int64_t N = (int64_t)H * W;
    size_t esz = out_kind == 0 ? 4 : (out_kind == 1 ? 2 : 1);
    double *px = (double *)malloc(sizeof(double) * (size_t)n * (size_t)nt);
    double *py = (double *)malloc(sizeof(double) * (size_t)n * (size_t)nt);
    double *cx = (double *)malloc(sizeof(double) * (size_t)n);
    double *cy = (double *)malloc(sizeof(double) * (size_t)n);
    double *img = (double *)malloc(sizeof(double) * (size_t)N * (size_t)nt);
    if (!px || !py || !cx || !cy || !img) {
        free(px); free(py); free(cx); free(cy); free(img);
        return 1;
    }
    memcpy(cx, x0, sizeof(double) * (size_t)n);
    memcpy(cy, y0, sizeof(double) * (size_t)n);
    double ext_w = W + 2.0 * margin, ext_h = H + 2.0 * margin;
    double *dx = (double *)malloc(sizeof(double) * (size_t)n);
    double *dy = (double *)malloc(sizeof(double) * (size_t)n);
    double *mx = (double *)malloc(sizeof(double) * (size_t)n);
    double *my = (double *)malloc(sizeof(double) * (size_t)n);
    for (int f0 = 0; f0 < n_frames; f0 += nt) {
        int cnt = n_frames - f0 < nt ? n_frames - f0 : nt;
        for (int c = 0; c < cnt; ++c) {
            memcpy(px + (size_t)c * n, cx, sizeof(double) * (size_t)n);
            memcpy(py + (size_t)c * n, cy, sizeof(double) * (size_t)n);
            /* advance to the next frame */
            syn_field_eval(f, n, cx, cy, dx, dy);
            for (int64_t i = 0; i < n; ++i) {
                mx[i] = cx[i] + 0.5 * dx[i];
                my[i] = cy[i] + 0.5 * dy[i];
            }
            syn_field_eval(f, n, mx, my, dx, dy);
            for (int64_t i = 0; i < n; ++i) {
                double nx = cx[i] + dx[i], ny = cy[i] + dy[i];
                if (nx < -margin) nx += ext_w;
                else if (nx >= W + margin) nx -= ext_w;
                if (ny < -margin) ny += ext_h;
                else if (ny >= H + margin) ny -= ext_h;
                cx[i] = nx;
                cy[i] = ny;
            }
        }
#pragma omp parallel for schedule(dynamic, 1)
        for (int c = 0; c < cnt; ++c) {
            double *im = img + (size_t)c * (size_t)N;
            memset(im, 0, sizeof(double) * (size_t)N);
            render_rows(H, W, 0, H, n, px + (size_t)c * n, py + (size_t)c * n, sigma, amp, im);
        }
        for (int c = 0; c < cnt; ++c) {
            syn_finalize(H, W, img + (size_t)c * (size_t)N, noise_sigma, noise_seed,
                         (uint64_t)(f0 + c), bits, out_kind,
                         (char *)out + (size_t)(f0 + c) * (size_t)N * esz);
        }
    }
    free(px); free(py); free(cx); free(cy); free(img);
    free(dx); free(dy); free(mx); free(my);
    return 0;
}
