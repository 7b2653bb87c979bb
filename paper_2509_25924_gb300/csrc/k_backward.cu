// Adjoint (reverse mode) of the estimator: gradients of a loss with respect
// to both input frames and the 5x5 pre-filter weights, given dL/du, dL/dv.
// The paper has no adjoint; this is the chain rule through the steps of
// Sec. 2 in reverse order.  Per Gauss-Newton stage (level l, iteration t):
//   forward again: products at every pixel, window sums S;
//   solve:   V = H^-1 b  =>  lambda = H^-1 gV, gH = -lambda V^T, gb = lambda
//            (a guarded pixel, V = V0, passes gV to V0 unchanged);
//   sums:    the adjoint of a truncated box sum is the same box sum;
//   products, residual r = G.V0 - It, G = (g1 + g2)/2, It = B - A:
//            gradients of the five products to G, r, and on to the samples;
//   samples: bilinear samples of the level images and of their central
//            differences at p1 = k - V0/2, p2 = k + V0/2: scatter to the image
//            taps (atomics) and differentiate with respect to the position,
//            which gives the gradient of V0 (clamped taps: zero slope beyond
//            the border);
//   then the up-sampling (scatter to the coarse field), the pyramid
//   reductions (scatter) and the pre-filter (transpose and weight
//   gradient).  Float atomics make the summation order, and so the last bits,
//   vary from run to run.
#include <cstring>

#include "iter_math.cuh"
#include "k_bw_block.cuh"
#include "ofv_handle.h"

namespace ofv {

// V0 of a stage written as a plane: zero, same (copy of the previous stage
// output) or the x2 up-sampled coarse field.
__global__ void k_bw_v0(IterArgs a, int mode, float2 *out)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.W || y >= a.H) return;
    float2 v = make_float2(0.f, 0.f);
    if (mode == V0_SAME) v = fetch_v0<V0_SAME>(a, x, y);
    else if (mode == V0_UP) v = fetch_v0<V0_UP>(a, x, y);
    out[(int64_t)y * a.vpitch + x] = v;
}

// Forward products of a stage (V0 from a.V0, pitch a.vpitch).
template <typename T>
__global__ void k_bw_products(IterArgs a, Planes5 out)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.W || y >= a.H) return;
    float p[5];
    pixel_products<T>(a, x, y, fetch_v0<V0_SAME>(a, x, y), p);
    const int64_t o = (int64_t)y * out.pitch + x;
#pragma unroll
    for (int c = 0; c < 5; ++c) out.p[c][o] = p[c];
}

// Truncated box sums along rows (dir 0) or columns (dir 1), five planes.
__global__ void k_bw_box(Planes5 in, Planes5 out, int H, int W, int kr, int dir)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= W || y >= H) return;
    const int64_t o = (int64_t)y * in.pitch + x;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        float s = 0.f;
        if (dir == 0) {
            const int j0 = max(x - kr, 0), j1 = min(x + kr, W - 1);
            const float *row = in.p[c] + (int64_t)y * in.pitch;
            for (int j = j0; j <= j1; ++j) s += row[j];
        } else {
            const int i0 = max(y - kr, 0), i1 = min(y + kr, H - 1);
            for (int i = i0; i <= i1; ++i) s += in.p[c][(int64_t)i * in.pitch + x];
        }
        out.p[c][o] = s;
    }
}

// Adjoint of the guarded 2x2 solve.  S holds the window sums; gV the
// gradient of the stage output (pitch vpitch).  Writes gS (five planes) and
// the direct part of the gradient of V0 (guarded pixels) into gV0.
__global__ void k_bw_solve(Planes5 S, const float2 *gV, int vpitch, int H, int W, float eps_rel, float eps_abs,
                           Planes5 gS, float2 *gV0)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= W || y >= H) return;
    const int64_t o = (int64_t)y * S.pitch + x;
    const int64_t ov = (int64_t)y * vpitch + x;
    const float a = S.p[0][o], b = S.p[1][o], c = S.p[2][o], sxr = S.p[3][o], syr = S.p[4][o];
    const float tr = a + c, det = a * c - b * b;
    const float2 g = gV[ov];
    float r[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    float2 direct = make_float2(0.f, 0.f);
    if (!(tr > eps_abs) || det <= eps_rel * tr * tr) {
        direct = g;
    } else {
        const float inv = 1.f / det;
        const float Vx = (c * sxr - b * syr) * inv, Vy = (a * syr - b * sxr) * inv;
        const float lx = (c * g.x - b * g.y) * inv, ly = (a * g.y - b * g.x) * inv;
        r[0] = -lx * Vx;
        r[1] = -(lx * Vy + ly * Vx);
        r[2] = -ly * Vy;
        r[3] = lx;
        r[4] = ly;
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) gS.p[k][o] = r[k];
    gV0[ov] = direct;
}

template <typename T>
__device__ __forceinline__ float ldp(const T *P, int pitch, int y, int x) { return ld_store(P + (int64_t)y * pitch + x); }

// Image-gradient scatter straight to global memory (float atomics).
struct ScatterGlobal {
    float *g;
    int pitch;
    __device__ __forceinline__ void operator()(int y, int x, float v) const { atomicAdd(g + (int64_t)y * pitch + x, v); }
};

// Value, gradient and position derivatives of one bilinear sample at
// (x + dx, y + dy) with clamp-to-edge taps, and the scatter of (gval, ggx,
// ggy) into the image gradient through add(row, column, value).  Returns
// through dpx, dpy the derivative of gval*val + ggx*gx + ggy*gy w.r.t. the
// position.
template <typename T, typename Scatter>
__device__ __forceinline__ void sample_adj(const T *P, int H, int W, int pitch, int x, int y, float dx, float dy,
                                           float gval, float ggx, float ggy, const Scatter &add, float &dpx,
                                           float &dpy)
{
    const float lim_x = (float)(W + 4), lim_y = (float)(H + 4);
    dx = fminf(fmaxf(dx, -lim_x), lim_x);
    dy = fminf(fmaxf(dy, -lim_y), lim_y);
    const float flx = floorf(dx), fly = floorf(dy);
    const float fx = dx - flx, fy = dy - fly;
    const int x0 = x + (int)flx, y0 = y + (int)fly;
    const int xa = clampi(x0, 0, W - 1), xb = clampi(x0 + 1, 0, W - 1);
    const int ya = clampi(y0, 0, H - 1), yb = clampi(y0 + 1, 0, H - 1);
    const int xam = clampi(xa - 1, 0, W - 1), xap = clampi(xa + 1, 0, W - 1);
    const int xbm = clampi(xb - 1, 0, W - 1), xbp = clampi(xb + 1, 0, W - 1);
    const int yam = clampi(ya - 1, 0, H - 1), yap = clampi(ya + 1, 0, H - 1);
    const int ybm = clampi(yb - 1, 0, H - 1), ybp = clampi(yb + 1, 0, H - 1);
    const float p00 = ldp(P, pitch, ya, xa), p01 = ldp(P, pitch, ya, xb);
    const float p10 = ldp(P, pitch, yb, xa), p11 = ldp(P, pitch, yb, xb);
    const float dx00 = 0.5f * (ldp(P, pitch, ya, xap) - ldp(P, pitch, ya, xam));
    const float dx01 = 0.5f * (ldp(P, pitch, ya, xbp) - ldp(P, pitch, ya, xbm));
    const float dx10 = 0.5f * (ldp(P, pitch, yb, xap) - ldp(P, pitch, yb, xam));
    const float dx11 = 0.5f * (ldp(P, pitch, yb, xbp) - ldp(P, pitch, yb, xbm));
    const float dy00 = 0.5f * (ldp(P, pitch, yap, xa) - ldp(P, pitch, yam, xa));
    const float dy01 = 0.5f * (ldp(P, pitch, yap, xb) - ldp(P, pitch, yam, xb));
    const float dy10 = 0.5f * (ldp(P, pitch, ybp, xa) - ldp(P, pitch, ybm, xa));
    const float dy11 = 0.5f * (ldp(P, pitch, ybp, xb) - ldp(P, pitch, ybm, xb));
    const float wx0 = 1.f - fx, wy0 = 1.f - fy;
    auto ddx = [&](float q00, float q01, float q10, float q11) { return wy0 * (q01 - q00) + fy * (q11 - q10); };
    auto ddy = [&](float q00, float q01, float q10, float q11) {
        return (wx0 * q10 + fx * q11) - (wx0 * q00 + fx * q01);
    };
    dpx = gval * ddx(p00, p01, p10, p11) + ggx * ddx(dx00, dx01, dx10, dx11) + ggy * ddx(dy00, dy01, dy10, dy11);
    dpy = gval * ddy(p00, p01, p10, p11) + ggx * ddy(dx00, dx01, dx10, dx11) + ggy * ddy(dy00, dy01, dy10, dy11);
    const float w[4] = {wx0 * wy0, fx * wy0, wx0 * fy, fx * fy};
    const int ty[4] = {ya, ya, yb, yb}, tx[4] = {xa, xb, xa, xb};
    const int txm[4] = {xam, xbm, xam, xbm}, txp[4] = {xap, xbp, xap, xbp};
    const int tym[4] = {yam, yam, ybm, ybm}, typ[4] = {yap, yap, ybp, ybp};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (gval != 0.f) add(ty[k], tx[k], gval * w[k]);
        const float gdx = 0.5f * ggx * w[k], gdy = 0.5f * ggy * w[k];
        if (gdx != 0.f) {
            add(ty[k], txp[k], gdx);
            add(ty[k], txm[k], -gdx);
        }
        if (gdy != 0.f) {
            add(typ[k], tx[k], gdy);
            add(tym[k], tx[k], -gdy);
        }
    }
}

// Adjoint of the products, the residual, the averaged gradient and the two
// warped samples at pixel (x, y); adds into gV0 and, through add1 and add2,
// into the level-image gradients.
template <typename T, typename Scatter>
__device__ __forceinline__ void samples_adjoint_pixel(const IterArgs &a, const Planes5 &gprod, float2 *gV0, int x,
                                                      int y, const Scatter &add1, const Scatter &add2)
{
    const T *P1 = static_cast<const T *>(a.P1);
    const T *P2 = static_cast<const T *>(a.P2);
    const float2 V0 = fetch_v0<V0_SAME>(a, x, y);
    const float hx = 0.5f * V0.x, hy = 0.5f * V0.y;
    const Sample s1 = sample_level(P1, a.H, a.W, a.pitch, x, y, -hx, -hy);
    const Sample s2 = sample_level(P2, a.H, a.W, a.pitch, x, y, hx, hy);
    const float Gx = 0.5f * (s1.gx + s2.gx), Gy = 0.5f * (s1.gy + s2.gy);
    const float It = s2.val - s1.val;
    const float r = Gx * V0.x + Gy * V0.y - It;
    const int64_t o = (int64_t)y * gprod.pitch + x;
    const float q0 = gprod.p[0][o], q1 = gprod.p[1][o], q2 = gprod.p[2][o], q3 = gprod.p[3][o], q4 = gprod.p[4][o];
    const float gr = Gx * q3 + Gy * q4;
    const float gGx = 2.f * Gx * q0 + Gy * q1 + r * q3 + V0.x * gr;
    const float gGy = Gx * q1 + 2.f * Gy * q2 + r * q4 + V0.y * gr;
    const float gA = gr, gB = -gr;  // It = B - A, gIt = -gr
    float d1x, d1y, d2x, d2y;
    sample_adj(P1, a.H, a.W, a.pitch, x, y, -hx, -hy, gA, 0.5f * gGx, 0.5f * gGy, add1, d1x, d1y);
    sample_adj(P2, a.H, a.W, a.pitch, x, y, hx, hy, gB, 0.5f * gGx, 0.5f * gGy, add2, d2x, d2y);
    float2 g = gV0[(int64_t)y * a.vpitch + x];
    g.x += Gx * gr - 0.5f * d1x + 0.5f * d2x;
    g.y += Gy * gr - 0.5f * d1y + 0.5f * d2y;
    gV0[(int64_t)y * a.vpitch + x] = g;
}

// One pixel per thread, scatter to global memory (window radii > 10).
template <typename T>
__global__ void k_bw_samples(IterArgs a, Planes5 gprod, float2 *gV0, float *gP1, float *gP2, int gpitch)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.W || y >= a.H) return;
    samples_adjoint_pixel<T>(a, gprod, gV0, x, y, ScatterGlobal{gP1, gpitch}, ScatterGlobal{gP2, gpitch});
}

// A 32 x 32 tile of pixels per CTA.  The image-gradient scatter lands in a
// shared-memory window around the tile (margin REACH + 2, which holds every
// tap of a warp up to REACH px) and reaches global memory once per window
// element; taps outside the window (larger warps) go to global memory
// directly.  Windows of neighbouring tiles overlap, so the final adds are
// atomic too.
constexpr int kSampTS = 32, kSampM = kBlockReach + 2, kSampWW = kSampTS + 2 * kSampM;

struct ScatterWindow {
    float (*win)[kSampWW + 1];
    float *g;
    int pitch, wx0, wy0;
    __device__ __forceinline__ void operator()(int y, int x, float v) const
    {
        const int r = y - wy0, c = x - wx0;
        if ((unsigned)r < (unsigned)kSampWW && (unsigned)c < (unsigned)kSampWW)
            atomicAdd(&win[r][c], v);
        else
            atomicAdd(g + (int64_t)y * pitch + x, v);
    }
};

template <typename T>
__global__ void __launch_bounds__(256) k_bw_samples_tile(IterArgs a, Planes5 gprod, float2 *gV0, float *gP1,
                                                         float *gP2, int gpitch)
{
    __shared__ float acc[2][kSampWW][kSampWW + 1];
    const int tid = threadIdx.x;
    const int tx0 = blockIdx.x * kSampTS, ty0 = blockIdx.y * kSampTS;
    const int wx0 = tx0 - kSampM, wy0 = ty0 - kSampM;
    float *flat = &acc[0][0][0];
    for (int i = tid; i < 2 * kSampWW * (kSampWW + 1); i += 256) flat[i] = 0.f;
    __syncthreads();
    const ScatterWindow s1{acc[0], gP1, gpitch, wx0, wy0}, s2{acc[1], gP2, gpitch, wx0, wy0};
    for (int i = tid; i < kSampTS * kSampTS; i += 256) {
        const int y = ty0 + i / kSampTS, x = tx0 + i % kSampTS;
        if (y < a.H && x < a.W) samples_adjoint_pixel<T>(a, gprod, gV0, x, y, s1, s2);
    }
    __syncthreads();
    for (int i = tid; i < 2 * kSampWW * kSampWW; i += 256) {
        const int f = i / (kSampWW * kSampWW), rem = i - f * kSampWW * kSampWW;
        const int r = rem / kSampWW, c = rem - r * kSampWW;
        const int y = wy0 + r, x = wx0 + c;
        const float v = acc[f][r][c];
        if (v != 0.f && y >= 0 && y < a.H && x >= 0 && x < a.W) atomicAdd((f ? gP2 : gP1) + (int64_t)y * gpitch + x, v);
    }
}

// Transpose of the x2 up-sampling: scatter 2 * w * gV0(fine) to the coarse
// taps (gc zeroed beforehand).
__global__ void k_bw_upsample_T(const float2 *gV0, int vpitch, int H, int W, float2 *gc, int cpitch, int Hc, int Wc)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= W || y >= H) return;
    const float2 g = gV0[(int64_t)y * vpitch + x];
    const int cx = x >> 1, cy = y >> 1;
    const float fx = (x & 1) ? 0.5f : 0.f, fy = (y & 1) ? 0.5f : 0.f;
    const int xa = min(cx, Wc - 1), xb = min(cx + 1, Wc - 1), ya = min(cy, Hc - 1), yb = min(cy + 1, Hc - 1);
    const float w[4] = {(1.f - fx) * (1.f - fy), fx * (1.f - fy), (1.f - fx) * fy, fx * fy};
    const int ty[4] = {ya, ya, yb, yb}, tx[4] = {xa, xb, xa, xb};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (w[k] == 0.f) continue;
        float *p = reinterpret_cast<float *>(gc + (int64_t)ty[k] * cpitch + tx[k]);
        atomicAdd(p, 2.f * w[k] * g.x);
        atomicAdd(p + 1, 2.f * w[k] * g.y);
    }
}

// Transpose of one pyramid reduction: level l+1 gradient (Hc x Wc) added
// into level l (H x W), both dense with their pitches.
__global__ void k_bw_reduce_T(const float *gc, int cpitch, int Hc, int Wc, float *g, int pitch, int H, int W)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= Hc || j >= Wc) return;
    const float c[5] = {0.0625f, 0.25f, 0.375f, 0.25f, 0.0625f};
    const float v = gc[(int64_t)i * cpitch + j];
    if (v == 0.f) return;
#pragma unroll
    for (int a = 0; a < 5; ++a)
#pragma unroll
        for (int b = 0; b < 5; ++b)
            atomicAdd(g + (int64_t)clampi(2 * i + a - 2, 0, H - 1) * pitch + clampi(2 * j + b - 2, 0, W - 1),
                      c[a] * c[b] * v);
}

// Pre-filter transpose and weight gradient, then the input scaling:
// gI(src) += w[a][b] * gJ(i,j) for src = clamp(i+a, j+b); gw[a][b] +=
// gJ(i,j) * I(src).  The frame values I come from the raw input (scaled).
template <typename TI>
__device__ __forceinline__ float ld_raw(const TI *p) { return (float)__ldg(p); }

template <typename TI>
__global__ void k_bw_prefilter(const float *gJ, int pitch, int H, int W, const TI *raw, float scale, const float *w25,
                               float *gI, float *gw)
{
    __shared__ float sw[25][8];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    const int lane = threadIdx.x + threadIdx.y * blockDim.x;
    float acc[25];
#pragma unroll
    for (int k = 0; k < 25; ++k) acc[k] = 0.f;
    if (i < H && j < W) {
        const float g = gJ[(int64_t)i * pitch + j];
        if (g != 0.f) {
#pragma unroll
            for (int a = 0; a < 5; ++a)
#pragma unroll
                for (int b = 0; b < 5; ++b) {
                    const int64_t src = (int64_t)clampi(i + a - 2, 0, H - 1) * W + clampi(j + b - 2, 0, W - 1);
                    atomicAdd(gI + src, __ldg(w25 + a * 5 + b) * g * scale);
                    acc[a * 5 + b] = g * ld_raw(raw + src) * scale;
                }
        }
    }
    // block reduction of the weight gradient: warp shuffles, then one atomic per warp
#pragma unroll
    for (int k = 0; k < 25; ++k) {
        float v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((lane & 31) == 0) sw[k][lane >> 5] = v;
    }
    __syncthreads();
    if (lane < 25) {
        float s = 0.f;
        for (int k = 0; k < (int)(blockDim.x * blockDim.y + 31) / 32; ++k) s += sw[lane][k];
        atomicAdd(gw + lane, s);
    }
}

// Without a pre-filter: gI = scale * gJ (dense output).
__global__ void k_bw_copy_scaled(const float *gJ, int pitch, int H, int W, float scale, float *gI)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= H || j >= W) return;
    gI[(int64_t)i * W + j] = scale * gJ[(int64_t)i * pitch + j];
}

// ---------------------------------------------------------------------------
// Adjoint of the local normalization (Sec. 2 step 1).  Forward:
// J(m) = (I(m) - mu(m)) / s(m), s = sqrt(var + eps_n^2), mu and var over the
// in-image part B(m) of the (2NR+1)^2 box, n(m) pixels.  With a = dL/dJ:
//   dL/dI(k) = a(k)/s(k) - A(k) - I(k) B(k) + C(k),
// where A, B, C are the truncated box sums of alpha = a / (s n),
// beta = a J / (s^2 n) and beta mu (B(m) holds k exactly when B(k) holds m).
// Planes here are dense H x W floats.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int box_count(int i, int j, int H, int W, int nr)
{
    return (min(i + nr, H - 1) - max(i - nr, 0) + 1) * (min(j + nr, W - 1) - max(j - nr, 0) + 1);
}

// Per pixel: mu, s and the normalized value J of the scaled input I = raw *
// scale (mean, then the centred variance, as the forward ingest).
template <typename TI>
__global__ void k_bw_norm_stats(const TI *raw, float scale, int H, int W, int nr, float eps_n, float *J, float *mu,
                                float *sd)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= H || j >= W) return;
    const int i0 = max(i - nr, 0), i1 = min(i + nr, H - 1), j0 = max(j - nr, 0), j1 = min(j + nr, W - 1);
    float sum = 0.f;
    for (int ii = i0; ii <= i1; ++ii)
        for (int jj = j0; jj <= j1; ++jj) sum += ld_raw(raw + (int64_t)ii * W + jj) * scale;
    const float n = (float)((i1 - i0 + 1) * (j1 - j0 + 1));
    const float m = sum / n;
    float q = 0.f;
    for (int ii = i0; ii <= i1; ++ii)
        for (int jj = j0; jj <= j1; ++jj) {
            const float d = ld_raw(raw + (int64_t)ii * W + jj) * scale - m;
            q = fmaf(d, d, q);
        }
    const float sv = sqrtf(q / n + eps_n * eps_n);
    const int64_t k = (int64_t)i * W + j;
    mu[k] = m;
    sd[k] = sv;
    J[k] = (ld_raw(raw + k) * scale - m) / sv;
}

// alpha = a / (s n), beta = a J / (s^2 n), gamma = beta mu.
__global__ void k_bw_norm_coef(const float *a, const float *J, const float *mu, const float *sd, int H, int W, int nr,
                               float *alpha, float *beta, float *gamma)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= H || j >= W) return;
    const int64_t k = (int64_t)i * W + j;
    const float sn = sd[k] * (float)box_count(i, j, H, W, nr);
    const float al = a[k] / sn;
    const float be = al * J[k] / sd[k];
    alpha[k] = al;
    beta[k] = be;
    gamma[k] = be * mu[k];
}

// Truncated box sums of radius nr of three planes along rows (dir 0) or
// columns (dir 1).
__global__ void k_bw_box3(const float *x0, const float *x1, const float *x2, int H, int W, int nr, int dir, float *y0,
                          float *y1, float *y2)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= H || j >= W) return;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    if (dir == 0) {
        const int64_t r = (int64_t)i * W;
        for (int jj = max(j - nr, 0); jj <= min(j + nr, W - 1); ++jj) {
            s0 += x0[r + jj];
            s1 += x1[r + jj];
            s2 += x2[r + jj];
        }
    } else {
        for (int ii = max(i - nr, 0); ii <= min(i + nr, H - 1); ++ii) {
            const int64_t o = (int64_t)ii * W + j;
            s0 += x0[o];
            s1 += x1[o];
            s2 += x2[o];
        }
    }
    const int64_t k = (int64_t)i * W + j;
    y0[k] = s0;
    y1[k] = s1;
    y2[k] = s2;
}

// dL/draw = scale (a/s - A - I B + C), I = raw * scale.
template <typename TI>
__global__ void k_bw_norm_out(const float *a, const float *sd, const TI *raw, float scale, const float *A,
                              const float *B, const float *C, int H, int W, float *gI)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= H || j >= W) return;
    const int64_t k = (int64_t)i * W + j;
    const float I = ld_raw(raw + k) * scale;
    gI[k] = scale * (a[k] / sd[k] - A[k] - I * B[k] + C[k]);
}

// Dense planar (gu, gv) into an interleaved field of pitch vpitch.
__global__ void k_bw_pack(const float *gu, const float *gv, int H, int W, float2 *out, int vpitch)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= W || y >= H) return;
    const int64_t i = (int64_t)y * W + x;
    out[(int64_t)y * vpitch + x] = make_float2(__ldg(gu + i), __ldg(gv + i));
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static dim3 grid2(int W, int H) { return dim3((W + 31) / 32, (H + 7) / 8); }

cudaError_t bw_pack(const float *gu, const float *gv, int H, int W, float2 *out, int vpitch, cudaStream_t s)
{
    k_bw_pack<<<grid2(W, H), dim3(32, 8), 0, s>>>(gu, gv, H, W, out, vpitch);
    return cudaGetLastError();
}

cudaError_t bw_v0(const IterArgs &a, int mode, float2 *out, cudaStream_t s)
{
    k_bw_v0<<<grid2(a.W, a.H), dim3(32, 8), 0, s>>>(a, mode, out);
    return cudaGetLastError();
}

namespace {
cudaError_t box_tile(int kr, Planes5 in, Planes5 out, int H, int W, cudaStream_t s)
{
    switch (kr) {
#define OFV_BOX_CASE(K) \
    case K: return run_bw_box_tile<K>(in, out, H, W, s);
    OFV_BOX_CASE(1) OFV_BOX_CASE(2) OFV_BOX_CASE(3) OFV_BOX_CASE(4) OFV_BOX_CASE(5)
    OFV_BOX_CASE(6) OFV_BOX_CASE(7) OFV_BOX_CASE(8) OFV_BOX_CASE(9) OFV_BOX_CASE(10)
#undef OFV_BOX_CASE
    default: return cudaErrorInvalidValue;
    }
}
}  // namespace

// One stage of the adjoint.  Window radii 1..10: the solve adjoint from the
// window sums the forward pass kept (Sk; gS into B, direct part of gV0), the
// box-sum adjoint tile by tile (gS -> gprod in A), the samples adjoint with
// the scatter accumulated per tile in shared memory.  Larger radii: one
// pixel per thread throughout.
cudaError_t bw_stage(const IterArgs &a, int store, Planes5 Sk, Planes5 A, Planes5 B, const float2 *gV, float2 *gV0,
                     float *gP1, float *gP2, int gpitch, cudaStream_t s)
{
    const dim3 g = grid2(a.W, a.H), b(32, 8);
    if (block_supports(a.kr)) {
        k_bw_solve<<<g, b, 0, s>>>(Sk, gV, a.vpitch, a.H, a.W, a.eps_rel, a.eps_abs, B, gV0);
        cudaError_t e = box_tile(a.kr, B, A, a.H, a.W, s);
        if (e != cudaSuccess) return e;
        const dim3 gt((a.W + kSampTS - 1) / kSampTS, (a.H + kSampTS - 1) / kSampTS);
        switch (store) {
        case ST_F16: k_bw_samples_tile<__half><<<gt, 256, 0, s>>>(a, A, gV0, gP1, gP2, gpitch); break;
        case ST_BF16: k_bw_samples_tile<__nv_bfloat16><<<gt, 256, 0, s>>>(a, A, gV0, gP1, gP2, gpitch); break;
        default: k_bw_samples_tile<float><<<gt, 256, 0, s>>>(a, A, gV0, gP1, gP2, gpitch); break;
        }
        return cudaGetLastError();
    }
    switch (store) {
    case ST_F16: k_bw_products<__half><<<g, b, 0, s>>>(a, A); break;
    case ST_BF16: k_bw_products<__nv_bfloat16><<<g, b, 0, s>>>(a, A); break;
    default: k_bw_products<float><<<g, b, 0, s>>>(a, A); break;
    }
    k_bw_box<<<g, b, 0, s>>>(A, B, a.H, a.W, a.kr, 0);
    k_bw_box<<<g, b, 0, s>>>(B, A, a.H, a.W, a.kr, 1);
    k_bw_solve<<<g, b, 0, s>>>(A, gV, a.vpitch, a.H, a.W, a.eps_rel, a.eps_abs, B, gV0);
    k_bw_box<<<g, b, 0, s>>>(B, A, a.H, a.W, a.kr, 0);
    k_bw_box<<<g, b, 0, s>>>(A, B, a.H, a.W, a.kr, 1);
    switch (store) {
    case ST_F16: k_bw_samples<__half><<<g, b, 0, s>>>(a, B, gV0, gP1, gP2, gpitch); break;
    case ST_BF16: k_bw_samples<__nv_bfloat16><<<g, b, 0, s>>>(a, B, gV0, gP1, gP2, gpitch); break;
    default: k_bw_samples<float><<<g, b, 0, s>>>(a, B, gV0, gP1, gP2, gpitch); break;
    }
    return cudaGetLastError();
}

cudaError_t bw_upsample_T(const float2 *gV0, int vpitch, int H, int W, float2 *gc, int cpitch, int Hc, int Wc,
                          cudaStream_t s)
{
    k_bw_upsample_T<<<grid2(W, H), dim3(32, 8), 0, s>>>(gV0, vpitch, H, W, gc, cpitch, Hc, Wc);
    return cudaGetLastError();
}

cudaError_t bw_reduce_T(const float *gc, int cpitch, int Hc, int Wc, float *g, int pitch, int H, int W, cudaStream_t s)
{
    k_bw_reduce_T<<<grid2(Wc, Hc), dim3(32, 8), 0, s>>>(gc, cpitch, Hc, Wc, g, pitch, H, W);
    return cudaGetLastError();
}

// Reverse of ingest with local normalization: J (pyramid level 0) = pre-filter
// (optional) of the normalized frame N; gJ -> gN (pre-filter transpose, weight
// gradient against N) -> gI through the normalization adjoint.  t[0..9]:
// dense H x W scratch planes.
template <typename TI>
cudaError_t bw_input_norm_t(const float *gJ, int pitch, int H, int W, const TI *raw, float scale, int nr, float eps_n,
                            const float *w25, int prefilter, float *gI, float *gw, float *const *t, cudaStream_t s)
{
    const dim3 g = grid2(W, H), b(32, 8);
    float *N = t[0], *mu = t[1], *sd = t[2], *gN = t[3];
    k_bw_norm_stats<TI><<<g, b, 0, s>>>(raw, scale, H, W, nr, eps_n, N, mu, sd);
    if (prefilter) {
        cudaError_t e = cudaMemsetAsync(gN, 0, (size_t)H * W * sizeof(float), s);
        if (e != cudaSuccess) return e;
        k_bw_prefilter<float><<<g, b, 0, s>>>(gJ, pitch, H, W, N, 1.f, w25, gN, gw);
    } else {
        k_bw_copy_scaled<<<g, b, 0, s>>>(gJ, pitch, H, W, 1.f, gN);
    }
    k_bw_norm_coef<<<g, b, 0, s>>>(gN, N, mu, sd, H, W, nr, t[4], t[5], t[6]);
    k_bw_box3<<<g, b, 0, s>>>(t[4], t[5], t[6], H, W, nr, 0, t[7], t[8], t[9]);
    k_bw_box3<<<g, b, 0, s>>>(t[7], t[8], t[9], H, W, nr, 1, t[4], t[5], t[6]);
    k_bw_norm_out<TI><<<g, b, 0, s>>>(gN, sd, raw, scale, t[4], t[5], t[6], H, W, gI);
    return cudaGetLastError();
}

cudaError_t bw_input_norm(const float *gJ, int pitch, int H, int W, const void *raw, int in_type, float scale, int nr,
                          float eps_n, const float *w25, int prefilter, float *gI, float *gw, float *const *t,
                          cudaStream_t s)
{
    switch (in_type) {
    case IN_U8: return bw_input_norm_t(gJ, pitch, H, W, static_cast<const uint8_t *>(raw), scale, nr, eps_n, w25,
                                       prefilter, gI, gw, t, s);
    case IN_U16: return bw_input_norm_t(gJ, pitch, H, W, static_cast<const uint16_t *>(raw), scale, nr, eps_n, w25,
                                        prefilter, gI, gw, t, s);
    default: return bw_input_norm_t(gJ, pitch, H, W, static_cast<const float *>(raw), scale, nr, eps_n, w25,
                                    prefilter, gI, gw, t, s);
    }
}

cudaError_t bw_input(const float *gJ, int pitch, int H, int W, const void *raw, int in_type, float scale,
                     const float *w25, int prefilter, float *gI, float *gw, cudaStream_t s)
{
    const dim3 g = grid2(W, H), b(32, 8);
    if (!prefilter) {
        k_bw_copy_scaled<<<g, b, 0, s>>>(gJ, pitch, H, W, scale, gI);
        return cudaGetLastError();
    }
    switch (in_type) {
    case IN_U8: k_bw_prefilter<uint8_t><<<g, b, 0, s>>>(gJ, pitch, H, W, static_cast<const uint8_t *>(raw), scale, w25, gI, gw); break;
    case IN_U16: k_bw_prefilter<uint16_t><<<g, b, 0, s>>>(gJ, pitch, H, W, static_cast<const uint16_t *>(raw), scale, w25, gI, gw); break;
    default: k_bw_prefilter<float><<<g, b, 0, s>>>(gJ, pitch, H, W, static_cast<const float *>(raw), scale, w25, gI, gw); break;
    }
    return cudaGetLastError();
}

}  // namespace ofv

namespace {

using namespace ofv;

struct BwDevGuard {
    int prev = -1;
    bool ok = true;
    explicit BwDevGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~BwDevGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Carve the reverse-mode workspace; returns its size (nothing written when
// base is null).
struct BwLayout {
    float2 *Vst[kMaxLevels * 64];
    float *Sst[kMaxLevels * 64];  // five window-sum planes per stage (block path)
    float2 *V0in[kMaxLevels];
    Planes5 A, B;
    float2 *gV, *gV0;
    float *gP1[kMaxLevels], *gP2[kMaxLevels];
    float *gw_scratch;
};

size_t bw_layout(const ofv_handle *h, char *base, BwLayout *o)
{
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *p = base ? base + off : nullptr;
        off = align_up(off + bytes, 256);
        return p;
    };
    const int L = h->L, IT = h->p.iterations;
    for (int s = 0; s < L * IT; ++s) {
        const int l = L - 1 - s / IT;
        o->Vst[s] = reinterpret_cast<float2 *>(take((size_t)h->Hs[l] * h->pitch[l] * sizeof(float2)));
        o->Sst[s] = block_supports(h->p.kernel_radius)
                        ? reinterpret_cast<float *>(take(5 * (size_t)h->Hs[l] * h->pitch[l] * sizeof(float)))
                        : nullptr;
    }
    for (int l = 0; l < L; ++l)
        o->V0in[l] = reinterpret_cast<float2 *>(take((size_t)h->Hs[l] * h->pitch[l] * sizeof(float2)));
    const size_t plane = (size_t)h->Hs[0] * h->pitch[0];
    for (int c = 0; c < 5; ++c) {
        o->A.p[c] = reinterpret_cast<float *>(take(plane * sizeof(float)));
        o->B.p[c] = reinterpret_cast<float *>(take(plane * sizeof(float)));
    }
    o->gV = reinterpret_cast<float2 *>(take(plane * sizeof(float2)));
    o->gV0 = reinterpret_cast<float2 *>(take(plane * sizeof(float2)));
    for (int l = 0; l < L; ++l) {
        o->gP1[l] = reinterpret_cast<float *>(take((size_t)h->Hs[l] * h->pitch[l] * sizeof(float)));
        o->gP2[l] = reinterpret_cast<float *>(take((size_t)h->Hs[l] * h->pitch[l] * sizeof(float)));
    }
    o->gw_scratch = reinterpret_cast<float *>(take(32 * sizeof(float)));
    return off;
}

#define BW_TRY(expr, what)                                 \
    do {                                                   \
        cudaError_t e_ = (expr);                           \
        if (e_ != cudaSuccess) return cuda_fail_msg(e_, what); \
    } while (0)

}  // namespace

extern "C" ofv_status ofv_backward(ofv_handle *h, const void *I1, const void *I2, const float *gu, const float *gv,
                                   float *gI1, float *gI2, float *gw25, ofv_stream_t stream)
{
    if (!h) return fail_msg(OFV_ERR_INVALID_ARG, "ofv_backward: handle is NULL");
    if (!I1 || !I2 || !gu || !gv || !gI1 || !gI2)
        return fail_msg(OFV_ERR_INVALID_ARG, "ofv_backward: I1, I2, gu, gv, gI1 and gI2 must be non-NULL");
    if (gI1 == gI2) return fail_msg(OFV_ERR_INVALID_ARG, "ofv_backward: gI1 and gI2 must be distinct buffers");
    const ofv_params &p = h->p;
    if (p.window != OFV_WINDOW_BOX || p.increment_form || h->mask_on)
        return fail_msg(OFV_ERR_UNSUPPORTED,
                        "ofv_backward: covers the direct form with the uniform box window and no region mask only");
    if (p.iterations * h->L > kMaxLevels * 64)
        return fail_msg(OFV_ERR_UNSUPPORTED, "ofv_backward: too many stages");
    BwDevGuard g(h->device);
    if (!g.ok) return fail_msg(OFV_ERR_CUDA, "ofv_backward: cannot select the handle's device");
    {
        cudaError_t e = cudaPeekAtLastError();
        if (e != cudaSuccess) {
            cudaGetLastError();
            return cuda_fail_msg(e, "error pending before ofv_backward");
        }
    }
    if (tma_expired(h)) return fail_msg(OFV_ERR_TIMEOUT, "ofv_backward: a TMA copy of an earlier launch did not complete");
    cudaStream_t s = (cudaStream_t)stream;
    BwLayout w;
    const size_t need = bw_layout(h, nullptr, &w);
    if (need > h->bw_bytes) {
        if (h->bw_arena) {
            BW_TRY(cudaStreamSynchronize(s), "ofv_backward: waiting before growing the workspace");
            cudaFree(h->bw_arena);
            h->bw_arena = nullptr;
            h->bw_bytes = 0;
        }
        if (dev_alloc(&h->bw_arena, need) != cudaSuccess) {
            cudaGetLastError();
            h->bw_arena = nullptr;
            return fail_msg(OFV_ERR_ALLOC, "ofv_backward: cudaMalloc of %zu bytes failed", need);
        }
        h->bw_bytes = need;
    }
    bw_layout(h, static_cast<char *>(h->bw_arena), &w);

    // forward again (steps 1-5), keeping every stage's input and output field
    const void *fr[2] = {I1, I2};
    const int slots[2] = {0, 1};
    ofv_status st = handle_pyramids(h, fr, slots, 2, s);
    if (st != OFV_OK) return st;
    h->last_s1 = 0;
    h->last_s2 = 1;
    const int L = h->L, IT = p.iterations, S = L * IT;
    auto stage_args = [&](int sidx) {
        const int l = L - 1 - sidx / IT, t = sidx % IT;
        IterArgs a;
        memset(&a, 0, sizeof a);
        a.P1 = h->lvl[0][l];
        a.P2 = h->lvl[1][l];
        a.H = h->Hs[l];
        a.W = h->Ws[l];
        a.pitch = h->pitch[l];
        a.vpitch = h->pitch[l];
        a.kr = p.kernel_radius;
        a.eps_rel = p.det_rel_eps;
        a.eps_abs = p.det_abs_eps;
        a.V0 = t == 0 ? w.V0in[l] : w.Vst[sidx - 1];
        return a;
    };
    for (int sidx = 0; sidx < S; ++sidx) {
        const int l = L - 1 - sidx / IT, t = sidx % IT;
        IterArgs a = stage_args(sidx);
        if (t == 0) {
            IterArgs b = a;
            int mode = V0_ZERO;
            if (sidx > 0) {
                mode = V0_UP;
                b.Vc = w.Vst[sidx - 1];
                b.Hc = h->Hs[l + 1];
                b.Wc = h->Ws[l + 1];
                b.vcpitch = h->pitch[l + 1];
            }
            BW_TRY(bw_v0(b, mode, w.V0in[l], s), "ofv_backward: stage input field");
        }
        a.Vout = w.Vst[sidx];
        if (w.Sst[sidx]) {  // keep the window sums for the solve adjoint
            a.s_out = w.Sst[sidx];
            a.s_plane = (size_t)h->Hs[l] * h->pitch[l];
            a.s_pitch = h->pitch[l];
        }
        cudaError_t e = block_supports(p.kernel_radius) ? launch_iter_block(&a, 1, p.storage, V0_SAME, s)
                                                        : launch_iter_fused(a, p.storage, V0_SAME, s);
        BW_TRY(e, "ofv_backward: forward iteration");
    }

    // reverse
    for (int l = 0; l < L; ++l) {
        BW_TRY(cudaMemsetAsync(w.gP1[l], 0, (size_t)h->Hs[l] * h->pitch[l] * sizeof(float), s), "ofv_backward: memset");
        BW_TRY(cudaMemsetAsync(w.gP2[l], 0, (size_t)h->Hs[l] * h->pitch[l] * sizeof(float), s), "ofv_backward: memset");
    }
    BW_TRY(bw_pack(gu, gv, h->H, h->W, w.gV, h->pitch[0], s), "ofv_backward: packing dL/dV");
    float2 *gV = w.gV, *gV0 = w.gV0;
    for (int sidx = S - 1; sidx >= 0; --sidx) {
        const int l = L - 1 - sidx / IT, t = sidx % IT;
        IterArgs a = stage_args(sidx);
        Planes5 A = w.A, B = w.B, Sk = {};
        A.pitch = B.pitch = Sk.pitch = h->pitch[l];
        if (w.Sst[sidx])
            for (int c = 0; c < 5; ++c) Sk.p[c] = w.Sst[sidx] + c * (size_t)h->Hs[l] * h->pitch[l];
        BW_TRY(bw_stage(a, p.storage, Sk, A, B, gV, gV0, w.gP1[l], w.gP2[l], h->pitch[l], s),
               "ofv_backward: stage adjoint");
        if (sidx == 0) break;
        if (t > 0) {
            float2 *tmp = gV;
            gV = gV0;
            gV0 = tmp;
        } else {
            BW_TRY(cudaMemsetAsync(gV, 0, (size_t)h->Hs[l + 1] * h->pitch[l + 1] * sizeof(float2), s),
                   "ofv_backward: memset");
            BW_TRY(bw_upsample_T(gV0, h->pitch[l], h->Hs[l], h->Ws[l], gV, h->pitch[l + 1], h->Hs[l + 1], h->Ws[l + 1], s),
                   "ofv_backward: up-sampling adjoint");
        }
    }
    for (int l = L - 1; l >= 1; --l) {
        BW_TRY(bw_reduce_T(w.gP1[l], h->pitch[l], h->Hs[l], h->Ws[l], w.gP1[l - 1], h->pitch[l - 1], h->Hs[l - 1],
                           h->Ws[l - 1], s),
               "ofv_backward: reduce adjoint");
        BW_TRY(bw_reduce_T(w.gP2[l], h->pitch[l], h->Hs[l], h->Ws[l], w.gP2[l - 1], h->pitch[l - 1], h->Hs[l - 1],
                           h->Ws[l - 1], s),
               "ofv_backward: reduce adjoint");
    }
    const float scale = p.input == OFV_IN_F32 ? 1.0f : 1.0f / (float)((1u << p.bit_depth) - 1u);
    float *gw = gw25 ? gw25 : w.gw_scratch;
    const size_t nbytes = (size_t)h->H * h->W * sizeof(float);
    if (p.prefilter) {
        BW_TRY(cudaMemsetAsync(gI1, 0, nbytes, s), "ofv_backward: memset");
        BW_TRY(cudaMemsetAsync(gI2, 0, nbytes, s), "ofv_backward: memset");
        BW_TRY(cudaMemsetAsync(gw, 0, 25 * sizeof(float), s), "ofv_backward: memset");
    } else if (gw25) {
        BW_TRY(cudaMemsetAsync(gw25, 0, 25 * sizeof(float), s), "ofv_backward: memset");
    }
    if (p.norm_radius > 0) {
        // the ten level-0 planes of A and B are free now: dense H x W scratch
        float *t[10];
        for (int c = 0; c < 5; ++c) {
            t[c] = w.A.p[c];
            t[5 + c] = w.B.p[c];
        }
        BW_TRY(bw_input_norm(w.gP1[0], h->pitch[0], h->H, h->W, I1, p.input, scale, p.norm_radius, p.norm_eps,
                             h->w25, p.prefilter, gI1, gw, t, s),
               "ofv_backward: normalization adjoint");
        BW_TRY(bw_input_norm(w.gP2[0], h->pitch[0], h->H, h->W, I2, p.input, scale, p.norm_radius, p.norm_eps,
                             h->w25, p.prefilter, gI2, gw, t, s),
               "ofv_backward: normalization adjoint");
        return OFV_OK;
    }
    BW_TRY(bw_input(w.gP1[0], h->pitch[0], h->H, h->W, I1, p.input, scale, h->w25, p.prefilter, gI1, gw, s),
           "ofv_backward: input adjoint");
    BW_TRY(bw_input(w.gP2[0], h->pitch[0], h->H, h->W, I2, p.input, scale, h->w25, p.prefilter, gI2, gw, s),
           "ofv_backward: input adjoint");
    return OFV_OK;
}
