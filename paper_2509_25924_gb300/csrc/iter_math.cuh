// Per-pixel arithmetic of one Gauss-Newton iteration of the symmetric SSD
// (Eq. 2), shared by the fused and the plain kernels.
//
// For pixel k with current field V0(k):
//   p1 = k - V0/2, p2 = k + V0/2 (symmetric midpoint warp, Eq. 2)
//   A = P1(p1), B = P2(p2)                 bilinear, clamp-to-edge
//   g1 = (Dx P1, Dy P1)(p1), g2 likewise   central differences sampled bilinearly
//   G = (g1 + g2) / 2, It = B - A, r = G . V0 - It (r = -It in the
//   increment form)
//   products: Gx^2, Gx Gy, Gy^2, Gx r, Gy r
// and for pixel m, with S the window sums of the products over N(m):
//   H = [[Sxx, Sxy], [Sxy, Syy]], V(m) = H^-1 (Sxr, Syr) by Cramer's rule
//   (V0(m) + H^-1 (Sxr, Syr) in the increment form), unless
//   Sxx + Syy <= eps_abs or det <= eps_rel (Sxx + Syy)^2, where V0(m) is
//   kept.  The window sums weigh tap (a, b) by wg[|a|] wg[|b|] with the
//   Gaussian window, by 1 with the box.
#pragma once
#include "ofv_common.cuh"

namespace ofv {

struct Sample { float val, gx, gy; };

// Bilinear value and gradient of the level image P at (x + d.x, y + d.y).
// The integer pixel and the fraction are taken from the offset d alone, so
// the fraction keeps full precision at any image coordinate.
//
// Clamp-to-edge makes a tap column c < 0 read column 0 and c > W-1 read W-1.
// For x0 = floor(px) < 0 both bilinear taps sit on column 0, which is the
// same as x0 = 0 with fraction 0; for x0 >= W-1 both sit on column W-1, the
// same as x0 = W-2 with fraction 1.  After that remap the two taps are
// x0 and x0+1 inside the image and their central differences need columns
// x0-1 .. x0+2 (clamped); rows likewise.  12 loads per sample.
template <typename T>
__device__ __forceinline__ Sample sample_level(const T *__restrict__ P, int H, int W, int pitch,
                                               int x, int y, float dx, float dy)
{
    const float lim_x = (float)(W + 4), lim_y = (float)(H + 4);
    dx = fminf(fmaxf(dx, -lim_x), lim_x);  // NaN-safe: fmaxf(NaN, a) = a
    dy = fminf(fmaxf(dy, -lim_y), lim_y);
    const float flx = floorf(dx), fly = floorf(dy);
    float fx = dx - flx, fy = dy - fly;
    int x0 = x + (int)flx, y0 = y + (int)fly;
    if (x0 < 0) { x0 = 0; fx = 0.f; }
    if (x0 > W - 2) { x0 = W - 2; fx = 1.f; }
    if (y0 < 0) { y0 = 0; fy = 0.f; }
    if (y0 > H - 2) { y0 = H - 2; fy = 1.f; }
    const int xm = max(x0 - 1, 0), xp = min(x0 + 2, W - 1);
    const int ym = max(y0 - 1, 0), yp = min(y0 + 2, H - 1);
    const T *r0 = P + (int64_t)y0 * pitch;
    const T *r1 = r0 + pitch;
    const T *rm = P + (int64_t)ym * pitch;
    const T *rp = P + (int64_t)yp * pitch;
    const float q00 = ld_store(r0 + xm), q01 = ld_store(r0 + x0), q02 = ld_store(r0 + x0 + 1), q03 = ld_store(r0 + xp);
    const float q10 = ld_store(r1 + xm), q11 = ld_store(r1 + x0), q12 = ld_store(r1 + x0 + 1), q13 = ld_store(r1 + xp);
    const float e0 = ld_store(rm + x0), e1 = ld_store(rm + x0 + 1);
    const float e2 = ld_store(rp + x0), e3 = ld_store(rp + x0 + 1);
    const float wx0 = 1.f - fx, wy0 = 1.f - fy;
    Sample s;
    s.val = wy0 * (wx0 * q01 + fx * q02) + fy * (wx0 * q11 + fx * q12);
    // Dx at the four taps
    const float dxa0 = 0.5f * (q02 - q00), dxb0 = 0.5f * (q03 - q01);
    const float dxa1 = 0.5f * (q12 - q10), dxb1 = 0.5f * (q13 - q11);
    s.gx = wy0 * (wx0 * dxa0 + fx * dxb0) + fy * (wx0 * dxa1 + fx * dxb1);
    // Dy at the four taps
    const float dya0 = 0.5f * (q11 - e0), dyb0 = 0.5f * (q12 - e1);
    const float dya1 = 0.5f * (e2 - q01), dyb1 = 0.5f * (e3 - q02);
    s.gy = wy0 * (wx0 * dya0 + fx * dyb0) + fy * (wx0 * dya1 + fx * dyb1);
    return s;
}

// V0 at pixel (x, y) of the current level.
template <int MODE>
__device__ __forceinline__ float2 fetch_v0(const IterArgs &a, int x, int y)
{
    if (MODE == V0_ZERO) return make_float2(0.f, 0.f);
    if (MODE == V0_SAME) return __ldg(a.V0 + (int64_t)y * a.vpitch + x);
    // V0_UP: coarse pixel i sits at fine 2i; V = 2 * bilinear(Vc, x/2, y/2)
    const int cx = x >> 1, cy = y >> 1;
    const float fx = (x & 1) ? 0.5f : 0.f, fy = (y & 1) ? 0.5f : 0.f;
    const int cx1 = min(cx + 1, a.Wc - 1), cy1 = min(cy + 1, a.Hc - 1);
    const int cxa = min(cx, a.Wc - 1), cya = min(cy, a.Hc - 1);
    const float2 v00 = __ldg(a.Vc + (int64_t)cya * a.vcpitch + cxa);
    const float2 v01 = __ldg(a.Vc + (int64_t)cya * a.vcpitch + cx1);
    const float2 v10 = __ldg(a.Vc + (int64_t)cy1 * a.vcpitch + cxa);
    const float2 v11 = __ldg(a.Vc + (int64_t)cy1 * a.vcpitch + cx1);
    const float wx0 = 1.f - fx, wy0 = 1.f - fy;
    float2 r;
    r.x = 2.f * (wy0 * (wx0 * v00.x + fx * v01.x) + fy * (wx0 * v10.x + fx * v11.x));
    r.y = 2.f * (wy0 * (wx0 * v00.y + fx * v01.y) + fy * (wx0 * v10.y + fx * v11.y));
    return r;
}

// The five products at pixel (x, y) given V0 there.
template <typename T>
__device__ __forceinline__ void pixel_products(const IterArgs &a, int x, int y, float2 V0, float p[5])
{
    const T *P1 = static_cast<const T *>(a.P1);
    const T *P2 = static_cast<const T *>(a.P2);
    const float hx = 0.5f * V0.x, hy = 0.5f * V0.y;
    const Sample s1 = sample_level(P1, a.H, a.W, a.pitch, x, y, -hx, -hy);
    const Sample s2 = sample_level(P2, a.H, a.W, a.pitch, x, y, hx, hy);
    const float Gx = 0.5f * (s1.gx + s2.gx), Gy = 0.5f * (s1.gy + s2.gy);
    const float It = s2.val - s1.val;
    const float r = a.inc ? -It : Gx * V0.x + Gy * V0.y - It;
    p[0] = Gx * Gx;
    p[1] = Gx * Gy;
    p[2] = Gy * Gy;
    p[3] = Gx * r;
    p[4] = Gy * r;
}

// Guarded Cramer solve of [[Sxx, Sxy], [Sxy, Syy]] X = (Sxr, Syr); V = X,
// or V0 + X in the increment form.
__device__ __forceinline__ float2 solve2(const float S[5], float2 V0, float eps_rel, float eps_abs, int inc)
{
    const float a = S[0], b = S[1], c = S[2];
    const float tr = a + c;
    const float det = a * c - b * b;
    if (!(tr > eps_abs) || det <= eps_rel * tr * tr) return V0;
    const float2 X = make_float2((c * S[3] - b * S[4]) / det, (a * S[4] - b * S[3]) / det);
    return inc ? make_float2(V0.x + X.x, V0.y + X.y) : X;
}

// Window weight of tap offset t = 0 .. 2 kr along one axis.
__device__ __forceinline__ float win_weight(const IterArgs &a, int t)
{
    return a.gauss ? a.wg[abs(t - a.kr)] : 1.f;
}

}  // namespace ofv
