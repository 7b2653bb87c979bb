// Plain multi-kernel form of one Gauss-Newton iteration, kept beside the
// fused kernel for comparison.  Same arithmetic (Eq. 2, Sec. 2 step 3), split
// into simple one-thread-per-pixel kernels that pass the five product planes
// and their row sums through device memory:
//   [up-sample V0]  ->  products (5 planes)  ->  row sums  ->  column sums + solve
#include "iter_math.cuh"

namespace ofv {

// V0 = 2 * bilinear(Vc, x/2, y/2) written as a plane (Sec. 2 step 4).
__global__ void __launch_bounds__(256) k_plain_upsample(IterArgs a, float2 *out)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.W || y >= a.H) return;
    out[(int64_t)y * a.vpitch + x] = fetch_v0<V0_UP>(a, x, y);
}

template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_plain_products(IterArgs a, PlainBufs b)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.W || y >= a.H) return;
    const float2 V0 = fetch_v0<MODE>(a, x, y);
    float p[5];
    pixel_products<T>(a, x, y, V0, p);
    if (a.mask && !a.mask[(int64_t)y * a.W + x]) p[0] = p[1] = p[2] = p[3] = p[4] = 0.f;
    const int64_t o = (int64_t)y * a.pitch + x;
#pragma unroll
    for (int c = 0; c < 5; ++c) b.prod[c * b.plane + o] = p[c];
}

// Row sums over columns x-KR .. x+KR that lie inside the image (weighted
// with the Gaussian window).
__global__ void __launch_bounds__(256) k_plain_rowsum(IterArgs a, PlainBufs b)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.W || y >= a.H) return;
    const int j0 = max(x - a.kr, 0), j1 = min(x + a.kr, a.W - 1);
    const int64_t o = (int64_t)y * a.pitch;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        const float *row = b.prod + c * b.plane + o;
        float s = 0.f;
        if (a.gauss)
            for (int j = j0; j <= j1; ++j) s = fmaf(win_weight(a, j - x + a.kr), row[j], s);
        else
            for (int j = j0; j <= j1; ++j) s += row[j];
        b.hsum[c * b.plane + o + x] = s;
    }
}

// Column sums over rows y-KR .. y+KR inside the image, then the solve.
template <bool PLANAR>
__global__ void __launch_bounds__(256) k_plain_colsum_solve(IterArgs a, PlainBufs b, int mode)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.W || y >= a.H) return;
    const int i0 = max(y - a.kr, 0), i1 = min(y + a.kr, a.H - 1);
    float S[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        const float *col = b.hsum + c * b.plane + x;
        float s = 0.f;
        if (a.gauss)
            for (int i = i0; i <= i1; ++i) s = fmaf(win_weight(a, i - y + a.kr), col[(int64_t)i * a.pitch], s);
        else
            for (int i = i0; i <= i1; ++i) s += col[(int64_t)i * a.pitch];
        S[c] = s;
    }
    float2 V0 = make_float2(0.f, 0.f);
    if (mode == V0_SAME) V0 = a.V0[(int64_t)y * a.vpitch + x];
    else if (mode == V0_UP) V0 = b.vtmp[(int64_t)y * a.vpitch + x];
    float2 V = solve2(S, V0, a.eps_rel, a.eps_abs, a.inc);
    if (PLANAR && a.mask && !a.mask[(int64_t)y * a.W + x]) V = make_float2(no_vector(), no_vector());
    if (PLANAR) {
        a.u_out[(int64_t)y * a.W + x] = V.x;
        a.v_out[(int64_t)y * a.W + x] = V.y;
    } else {
        a.Vout[(int64_t)y * a.vpitch + x] = V;
    }
}

template <typename T>
static cudaError_t plain_t(const IterArgs &a0, const PlainBufs &b, int mode, cudaStream_t s)
{
    dim3 blk(32, 8);
    dim3 grd((a0.W + 31) / 32, (a0.H + 7) / 8);
    IterArgs a = a0;
    if (mode == V0_UP) {
        k_plain_upsample<<<grd, blk, 0, s>>>(a, b.vtmp);
        IterArgs as = a;
        as.V0 = b.vtmp;  // the products read the up-sampled plane like a same-level field
        k_plain_products<T, V0_SAME><<<grd, blk, 0, s>>>(as, b);
    } else if (mode == V0_SAME) {
        k_plain_products<T, V0_SAME><<<grd, blk, 0, s>>>(a, b);
    } else {
        k_plain_products<T, V0_ZERO><<<grd, blk, 0, s>>>(a, b);
    }
    k_plain_rowsum<<<grd, blk, 0, s>>>(a, b);
    if (a.u_out) k_plain_colsum_solve<true><<<grd, blk, 0, s>>>(a, b, mode);
    else k_plain_colsum_solve<false><<<grd, blk, 0, s>>>(a, b, mode);
    return cudaGetLastError();
}

cudaError_t launch_iter_plain(const IterArgs &a, const PlainBufs &b, int store, int mode,
                              cudaStream_t s)
{
    switch (store) {
    case ST_F16: return plain_t<__half>(a, b, mode, s);
    case ST_BF16: return plain_t<__nv_bfloat16>(a, b, mode, s);
    default: return plain_t<float>(a, b, mode, s);
    }
}

}  // namespace ofv
