// Quantities derived from the displacement fields in real time (Sec. 7):
// the out-of-plane vorticity, the recirculation area of Eq. 6 and point
// probes (time series of the field at chosen points).
//
//   omega = dv/dx - du/dy, the derivatives by second-order central
//   differences inside the field and first-order one-sided differences on
//   its first and last column / row (the usual finite-difference gradient);
//   RA = sum over the region of H(-u), H(-u) = 1 where u < 0, counted in
//   pixels (the caller multiplies by the pixel area dx dz).
//
// Both run over n fields of a sequence in one launch (blockIdx.z = field).
#include <cstdint>

#include "../../include/ofv.h"
#include "ofv_common.cuh"
#include "ofv_handle.h"

namespace ofv {

// d f / d x at column j of a row (finite-difference gradient, unit spacing).
__device__ __forceinline__ float ddx_row(const float *row, int j, int W)
{
    if (W < 2) return 0.f;
    if (j == 0) return row[1] - row[0];
    if (j == W - 1) return row[W - 1] - row[W - 2];
    return 0.5f * (row[j + 1] - row[j - 1]);
}

__device__ __forceinline__ float vort_at(const float *uf, const float *vf, int H, int W, int i, int j)
{
    const float dvdx = ddx_row(vf + (size_t)i * W, j, W);
    float dudy = 0.f;
    if (H >= 2) {
        if (i == 0) dudy = uf[(size_t)W + j] - uf[j];
        else if (i == H - 1) dudy = uf[(size_t)(H - 1) * W + j] - uf[(size_t)(H - 2) * W + j];
        else dudy = 0.5f * (uf[(size_t)(i + 1) * W + j] - uf[(size_t)(i - 1) * W + j]);
    }
    return dvdx - dudy;
}

// Four pixels per thread: 16-byte loads and stores where the four pixels
// and their neighbours are inside the field and the rows are 16-byte
// aligned (W % 4 == 0, field stride % 4 == 0, base pointers aligned);
// the general form elsewhere.
__global__ void __launch_bounds__(256) k_vorticity(int H, int W, const float *u, const float *v, size_t stride,
                                                   float *omega, int vec)
{
    const int W4 = (W + 3) / 4;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (t >= W4) return;
    const int j0 = 4 * t;
    const size_t f = (size_t)blockIdx.z * stride;
    const float *uf = u + f, *vf = v + f;
    float *of = omega + f;
    if (vec && i > 0 && i < H - 1 && j0 > 0 && j0 + 4 < W) {
        const float *vr = vf + (size_t)i * W;
        const float4 vc = __ldg(reinterpret_cast<const float4 *>(vr + j0));
        const float vl = __ldg(vr + j0 - 1), vrr = __ldg(vr + j0 + 4);
        const float4 ua = __ldg(reinterpret_cast<const float4 *>(uf + (size_t)(i - 1) * W + j0));
        const float4 ub = __ldg(reinterpret_cast<const float4 *>(uf + (size_t)(i + 1) * W + j0));
        float4 o;
        o.x = 0.5f * (vc.y - vl) - 0.5f * (ub.x - ua.x);
        o.y = 0.5f * (vc.z - vc.x) - 0.5f * (ub.y - ua.y);
        o.z = 0.5f * (vc.w - vc.y) - 0.5f * (ub.z - ua.z);
        o.w = 0.5f * (vrr - vc.z) - 0.5f * (ub.w - ua.w);
        *reinterpret_cast<float4 *>(of + (size_t)i * W + j0) = o;
        return;
    }
    for (int j = j0; j < j0 + 4 && j < W; ++j) of[(size_t)i * W + j] = vort_at(uf, vf, H, W, i, j);
}

// Count of u < 0 inside the region (mask != 0, or everywhere) per field:
// four pixels per step (16-byte loads when vec), a warp reduction, one
// atomic per warp.
__global__ void __launch_bounds__(256) k_recirc_count(int64_t N, const float *u, size_t stride, const uint8_t *mask,
                                                      unsigned long long *counts, int vec)
{
    const float *uf = u + (size_t)blockIdx.y * stride;
    unsigned long long c = 0;
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    if (vec) {
        const int64_t N4 = N / 4;
        for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N4; k += step) {
            const float4 x = __ldg(reinterpret_cast<const float4 *>(uf) + k);
            unsigned m = 0xffffffffu;
            if (mask) m = __ldg(reinterpret_cast<const unsigned *>(mask) + k);
            c += ((m & 0xffu) && x.x < 0.f) + ((m & 0xff00u) && x.y < 0.f) + ((m & 0xff0000u) && x.z < 0.f) +
                 ((m & 0xff000000u) && x.w < 0.f);
        }
    } else {
        for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += step) {
            const bool in = mask == nullptr || mask[k] != 0;
            c += (in && __ldg(uf + k) < 0.f) ? 1ull : 0ull;
        }
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(counts + blockIdx.y, c);
}

// Point probes: the field of every one of n fields at npts points (x, y) in
// pixel coordinates, bilinear with clamp-to-edge taps (the interpolation of
// the estimator).  One thread per (point, field).
__global__ void __launch_bounds__(256) k_probe(int H, int W, const float *u, const float *v, size_t stride, int npts,
                                               const float2 *xy, float2 *out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npts) return;
    const size_t f = (size_t)blockIdx.y * stride;
    const float2 p = __ldg(xy + k);
    const float flx = floorf(p.x), fly = floorf(p.y);
    const float fx = p.x - flx, fy = p.y - fly;
    const int x0 = (int)fminf(fmaxf(flx, -1.f), (float)W), y0 = (int)fminf(fmaxf(fly, -1.f), (float)H);
    const int xa = min(max(x0, 0), W - 1), xb = min(max(x0 + 1, 0), W - 1);
    const int ya = min(max(y0, 0), H - 1), yb = min(max(y0 + 1, 0), H - 1);
    const float *uf = u + f, *vf = v + f;
    auto bil = [&](const float *g) {
        const float a = __ldg(g + (size_t)ya * W + xa), b = __ldg(g + (size_t)ya * W + xb);
        const float c = __ldg(g + (size_t)yb * W + xa), d = __ldg(g + (size_t)yb * W + xb);
        return (1.f - fy) * ((1.f - fx) * a + fx * b) + fy * ((1.f - fx) * c + fx * d);
    };
    out[(size_t)blockIdx.y * npts + k] = make_float2(bil(uf), bil(vf));
}

}  // namespace ofv

using namespace ofv;

extern "C" {

ofv_status ofv_vorticity(int H, int W, int n, const float *u, const float *v, size_t field_stride, float *omega,
                         ofv_stream_t s)
{
    if (!u || !v || !omega) return fail_msg(OFV_ERR_INVALID_ARG, "ofv_vorticity: u, v and omega must be non-NULL");
    if (H < 1 || W < 1 || n < 1 || n > 65535)
        return fail_msg(OFV_ERR_SHAPE, "ofv_vorticity: H=%d W=%d n=%d (n at most 65535)", H, W, n);
    if (field_stride < (size_t)H * W)
        return fail_msg(OFV_ERR_INVALID_ARG, "ofv_vorticity: field_stride=%zu is smaller than one field", field_stride);
    if (H > 65535) return fail_msg(OFV_ERR_SHAPE, "ofv_vorticity: H=%d above 65535", H);
    const int vec = W % 4 == 0 && field_stride % 4 == 0 && ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(v) |
                                                              reinterpret_cast<uintptr_t>(omega)) & 15u) == 0;
    const dim3 g(((W + 3) / 4 + 255) / 256, H, n);
    k_vorticity<<<g, 256, 0, (cudaStream_t)s>>>(H, W, u, v, field_stride, omega, vec);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? OFV_OK : cuda_fail_msg(e, "ofv_vorticity launch");
}

ofv_status ofv_recirculation_area(int H, int W, int n, const float *u, size_t field_stride, const uint8_t *mask,
                                  unsigned long long *counts, ofv_stream_t s)
{
    if (!u || !counts) return fail_msg(OFV_ERR_INVALID_ARG, "ofv_recirculation_area: u and counts must be non-NULL");
    if (H < 1 || W < 1 || n < 1 || n > 65535)
        return fail_msg(OFV_ERR_SHAPE, "ofv_recirculation_area: H=%d W=%d n=%d (n at most 65535)", H, W, n);
    if (field_stride < (size_t)H * W)
        return fail_msg(OFV_ERR_INVALID_ARG, "ofv_recirculation_area: field_stride=%zu is smaller than one field",
                        field_stride);
    cudaStream_t cs = (cudaStream_t)s;
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * (size_t)n, cs);
    if (e != cudaSuccess) return cuda_fail_msg(e, "ofv_recirculation_area: clearing the counts");
    const int64_t N = (int64_t)H * W;
    const int vec = N % 4 == 0 && field_stride % 4 == 0 &&
                    ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(mask)) & 15u) == 0;
    int blocks = (int)(((vec ? N / 4 : N) + 255) / 256);
    if (blocks > 512) blocks = 512;
    k_recirc_count<<<dim3(blocks, n), 256, 0, cs>>>(N, u, field_stride, mask, counts, vec);
    e = cudaGetLastError();
    return e == cudaSuccess ? OFV_OK : cuda_fail_msg(e, "ofv_recirculation_area launch");
}

ofv_status ofv_probe(int H, int W, int n, const float *u, const float *v, size_t field_stride, int npts,
                     const float *xy, float *out, ofv_stream_t s)
{
    if (!u || !v || !xy || !out) return fail_msg(OFV_ERR_INVALID_ARG, "ofv_probe: u, v, xy and out must be non-NULL");
    if (H < 1 || W < 1 || n < 1 || n > 65535 || npts < 1)
        return fail_msg(OFV_ERR_SHAPE, "ofv_probe: H=%d W=%d n=%d npts=%d (n at most 65535)", H, W, n, npts);
    if (field_stride < (size_t)H * W)
        return fail_msg(OFV_ERR_INVALID_ARG, "ofv_probe: field_stride=%zu is smaller than one field", field_stride);
    if ((reinterpret_cast<uintptr_t>(xy) | reinterpret_cast<uintptr_t>(out)) & 7u)
        return fail_msg(OFV_ERR_INVALID_ARG, "ofv_probe: xy and out must be 8-byte aligned");
    k_probe<<<dim3((npts + 255) / 256, n), 256, 0, (cudaStream_t)s>>>(H, W, u, v, field_stride, npts,
                                                                     reinterpret_cast<const float2 *>(xy),
                                                                     reinterpret_cast<float2 *>(out));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? OFV_OK : cuda_fail_msg(e, "ofv_probe launch");
}

}  // extern "C"
