// Fused Gauss-Newton iteration: symmetric warp + gradients + products,
// separable window sums and the per-pixel 2x2 solve in one kernel
// (Sec. 2 step 3, Eq. 2; window N(m) of radius KR).
//
// One CTA owns a TX x TY tile of output pixels.  It computes the five
// products on the tile plus a KR halo into shared memory, sums them along
// rows (2KR+1 taps), then along columns, solves, and writes V.  Products of
// halo pixels outside the image are zero, which truncates the window at the
// border.  The field V0 of the previous iteration (or the up-sampled coarse
// field, or zero) is read per pixel; image samples are gathered through the
// read-only path because the warp reach is data dependent.
#include "iter_math.cuh"

namespace ofv {

constexpr int kTX = 32, kTY = 32, kThreads = 256;

inline size_t fused_smem_bytes(int kr)
{
    const int RW = kTX + 2 * kr, RH = kTY + 2 * kr;
    return sizeof(float) * (size_t)(5 * RH * RW + 5 * RH * kTX) + sizeof(float2) * kTX * kTY;
}

template <typename T, int MODE, bool PLANAR>
__global__ void __launch_bounds__(kThreads) k_iter_fused(IterArgs a)
{
    extern __shared__ float4 smem_f4[];
    float *smem = reinterpret_cast<float *>(smem_f4);
    const int kr = a.kr;
    const int RW = kTX + 2 * kr, RH = kTY + 2 * kr;
    const int RN = RH * RW;
    float *prod = smem;                                      // [5][RH][RW]
    float *hs = prod + 5 * RN;                               // [5][RH][kTX]
    float2 *v0c = reinterpret_cast<float2 *>(hs + 5 * RH * kTX);  // [kTY][kTX]
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;

    // phase 1: products on tile + halo
    for (int idx = threadIdx.x; idx < RN; idx += kThreads) {
        const int ry = idx / RW, rx = idx - ry * RW;
        const int gy = y0 - kr + ry, gx = x0 - kr + rx;
        float p[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        if (gy >= 0 && gy < a.H && gx >= 0 && gx < a.W) {
            const float2 V0 = fetch_v0<MODE>(a, gx, gy);
            pixel_products<T>(a, gx, gy, V0, p);
            if (a.mask && !a.mask[(int64_t)gy * a.W + gx]) p[0] = p[1] = p[2] = p[3] = p[4] = 0.f;
            const int cy = ry - kr, cx = rx - kr;
            if (cy >= 0 && cy < kTY && cx >= 0 && cx < kTX) v0c[cy * kTX + cx] = V0;
        }
#pragma unroll
        for (int c = 0; c < 5; ++c) prod[c * RN + idx] = p[c];
    }
    __syncthreads();

    // phase 2: row sums of 2KR+1 taps (weighted with the Gaussian window)
    const int taps = 2 * kr + 1;
    for (int idx = threadIdx.x; idx < RH * kTX; idx += kThreads) {
        const int ry = idx / kTX, ox = idx - ry * kTX;
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            const float *row = prod + c * RN + ry * RW + ox;
            float s = 0.f;
            if (a.gauss)
                for (int t = 0; t < taps; ++t) s = fmaf(win_weight(a, t), row[t], s);
            else
                for (int t = 0; t < taps; ++t) s += row[t];
            hs[c * RH * kTX + idx] = s;
        }
    }
    __syncthreads();

    // phase 3: column sums, solve, write
    for (int idx = threadIdx.x; idx < kTY * kTX; idx += kThreads) {
        const int oy = idx / kTX, ox = idx - oy * kTX;
        const int gy = y0 + oy, gx = x0 + ox;
        if (gy >= a.H || gx >= a.W) continue;
        float S[5];
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            const float *col = hs + c * RH * kTX + oy * kTX + ox;
            float s = 0.f;
            if (a.gauss)
                for (int t = 0; t < taps; ++t) s = fmaf(win_weight(a, t), col[t * kTX], s);
            else
                for (int t = 0; t < taps; ++t) s += col[t * kTX];
            S[c] = s;
        }
        float2 V = solve2(S, v0c[idx], a.eps_rel, a.eps_abs, a.inc);
        if (PLANAR && a.mask && !a.mask[(int64_t)gy * a.W + gx]) V = make_float2(no_vector(), no_vector());
        if (PLANAR) {
            a.u_out[(int64_t)gy * a.W + gx] = V.x;
            a.v_out[(int64_t)gy * a.W + gx] = V.y;
        } else {
            a.Vout[(int64_t)gy * a.vpitch + gx] = V;
        }
    }
}

template <typename T, int MODE, bool PLANAR>
static cudaError_t run(const IterArgs &a, cudaStream_t s)
{
    const size_t smem = fused_smem_bytes(a.kr);
    auto kern = k_iter_fused<T, MODE, PLANAR>;
    // raise the dynamic shared-memory limit once per device and instantiation
    static size_t granted[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || granted[dev] < smem) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) granted[dev] = smem;
    }
    dim3 grd((a.W + kTX - 1) / kTX, (a.H + kTY - 1) / kTY);
    kern<<<grd, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t dispatch_mode(const IterArgs &a, int mode, cudaStream_t s)
{
    const bool planar = a.u_out != nullptr;
    switch (mode) {
    case V0_ZERO: return planar ? run<T, V0_ZERO, true>(a, s) : run<T, V0_ZERO, false>(a, s);
    case V0_SAME: return planar ? run<T, V0_SAME, true>(a, s) : run<T, V0_SAME, false>(a, s);
    default: return planar ? run<T, V0_UP, true>(a, s) : run<T, V0_UP, false>(a, s);
    }
}

cudaError_t launch_iter_fused(const IterArgs &a, int store, int mode, cudaStream_t s)
{
    switch (store) {
    case ST_F16: return dispatch_mode<__half>(a, mode, s);
    case ST_BF16: return dispatch_mode<__nv_bfloat16>(a, mode, s);
    default: return dispatch_mode<float>(a, mode, s);
    }
}

size_t fused_smem_for_kr(int kr) { return fused_smem_bytes(kr); }

}  // namespace ofv
