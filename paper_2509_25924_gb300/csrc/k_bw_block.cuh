// Reverse mode on the block kernel's machinery (window radii 1..10).
//
// Per Gauss-Newton stage the adjoint needs the forward window sums S: the
// forward pass that the reverse mode recomputes keeps them (five planes per
// stage, written by the solve epilogue), so the guard decisions are those of
// the forward pass, and an elementwise kernel applies the solve adjoint:
//   V = H^-1 b  =>  lambda = H^-1 gV,
//   gS = (-lambda_x V_x, -(lambda_x V_y + lambda_y V_x), -lambda_y V_y, lambda_x, lambda_y),
// and a guarded pixel (V = V0) passes gV to V0.  k_bw_box_tile applies the
// adjoint of the truncated box sums, which is the same truncated box sum,
// tile by tile in shared memory.
#pragma once
#include "k_block.cuh"

namespace ofv {

struct Planes5 {
    float *p[5];
    int pitch;  // elements
};

// Truncated (2KR+1)^2 box sums of five planes, one TS x TS output tile per
// CTA: the (TS+2KR)^2 input region (zero outside the image) in shared
// memory, then the forward kernel's horizontal and vertical passes.
template <int KR>
__global__ void __launch_bounds__(BlockShape<KR>::NT, BlockShape<KR>::MINB) k_bw_box_tile(Planes5 in, Planes5 out, int H, int W)
{
    using BS = BlockShape<KR>;
    constexpr int TS = BS::TS, NT = BS::NT, RW = BS::RW, RWP = BS::RWP, PLANE = RW * RWP;
    extern __shared__ __align__(128) float4 smem_f4[];
    float *pl = reinterpret_cast<float *>(smem_f4);
    const int tid = threadIdx.x;
    const int tx0 = blockIdx.x * TS, ty0 = blockIdx.y * TS;
    for (int idx = tid; idx < RW * RW; idx += NT) {
        const int ry = idx / RW, rx = idx - ry * RW;
        const int gy = ty0 - KR + ry, gx = tx0 - KR + rx;
        const bool in_img = gy >= 0 && gy < H && gx >= 0 && gx < W;
        const int64_t o = (int64_t)gy * in.pitch + gx;
#pragma unroll
        for (int c = 0; c < 5; ++c) pl[c * PLANE + ry * RWP + rx] = in_img ? in.p[c][o] : 0.f;
    }
    __syncthreads();
    for (int t = tid; t < 5 * RW; t += NT) {
        const int c = t / RW, row = t - c * RW;
        window_sums_inplace<KR, TS>(pl + c * PLANE + row * RWP, 1);
    }
    __syncthreads();
    for (int t = tid; t < 5 * TS; t += NT) {
        const int c = t / TS, col = t - c * TS;
        window_sums_inplace<KR, TS>(pl + c * PLANE + col, RWP);
    }
    __syncthreads();
    for (int idx = tid; idx < TS * TS; idx += NT) {
        const int oy = idx / TS, ox = idx - oy * TS;
        const int gy = ty0 + oy, gx = tx0 + ox;
        if (gy >= H || gx >= W) continue;
        const int64_t o = (int64_t)gy * out.pitch + gx;
#pragma unroll
        for (int c = 0; c < 5; ++c) out.p[c][o] = pl[c * PLANE + oy * RWP + ox];
    }
}

template <int KR>
cudaError_t run_bw_box_tile(Planes5 in, Planes5 out, int H, int W, cudaStream_t s)
{
    using BS = BlockShape<KR>;
    constexpr size_t smem = sizeof(float) * 5 * BS::RW * BS::RWP;
    static bool granted[64];  // shared-memory opt-in done, per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !granted[dev]) {
        e = cudaFuncSetAttribute(k_bw_box_tile<KR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) granted[dev] = true;
    }
    k_bw_box_tile<KR><<<dim3((W + BS::TS - 1) / BS::TS, (H + BS::TS - 1) / BS::TS), BS::NT, smem, s>>>(in, out, H, W);
    return cudaGetLastError();
}

}  // namespace ofv
