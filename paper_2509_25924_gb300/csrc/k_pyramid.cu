// Ingest (scale, local normalization, optional 5x5 pre-filter) and
// Burt-Adelson pyramid reduction kernels.
//
// Sec. 2 of the paper: step 1 is a local, pixel-centred intensity
// normalization of radius NR; step 2 builds a Gaussian pyramid in which each
// sub-level halves both image dimensions (Burt & Adelson's reduction).
#include "ofv_common.cuh"

namespace ofv {

template <typename TI>
__device__ __forceinline__ float ld_in(const TI *p);
template <> __device__ __forceinline__ float ld_in<uint8_t>(const uint8_t *p) { return (float)__ldg(p); }
template <> __device__ __forceinline__ float ld_in<uint16_t>(const uint16_t *p) { return (float)__ldg(p); }
template <> __device__ __forceinline__ float ld_in<float>(const float *p) { return __ldg(p); }

struct IngestPair { IngestArgs f[kMaxFramesPerLaunch]; float scale; };

// Scaled intensity I = raw * scale (scale = 1/(2^bits - 1), or 1 for FP32
// input), then, for NR > 0, (I - mu) / sqrt(var + eps_n^2) with mu and var
// taken over the in-image part of the (2NR+1)^2 box.  Writes level 0 in the
// storage type, or FP32 scratch when a pre-filter follows.
template <typename TI, typename TS>
__global__ void __launch_bounds__(256) k_ingest(IngestPair p)
{
    const IngestArgs &a = p.f[blockIdx.z];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= a.H || j >= a.W) return;
    const TI *raw = static_cast<const TI *>(a.raw);
    const float sc = p.scale;
    float val = ld_in(raw + (int64_t)i * a.W + j) * sc;
    if (a.nr > 0) {
        const int i0 = max(i - a.nr, 0), i1 = min(i + a.nr, a.H - 1);
        const int j0 = max(j - a.nr, 0), j1 = min(j + a.nr, a.W - 1);
        const float inv_n = 1.0f / (float)((i1 - i0 + 1) * (j1 - j0 + 1));
        float s = 0.f;
        for (int ii = i0; ii <= i1; ++ii)
            for (int jj = j0; jj <= j1; ++jj) s += ld_in(raw + (int64_t)ii * a.W + jj) * sc;
        const float mu = s * inv_n;
        float q = 0.f;
        for (int ii = i0; ii <= i1; ++ii)
            for (int jj = j0; jj <= j1; ++jj) {
                const float d = ld_in(raw + (int64_t)ii * a.W + jj) * sc - mu;
                q = fmaf(d, d, q);
            }
        const float var = q * inv_n;
        val = (val - mu) * rsqrtf(var + a.eps_n * a.eps_n);
    }
    if (a.prefilter)
        a.tmp[(int64_t)i * a.pitch + j] = val;
    else
        st_store(static_cast<TS *>(a.out) + (int64_t)i * a.pitch + j, val);
}

// 5x5 correlation with clamp-to-edge: out(i,j) = sum w[a][b] I(i+a-2, j+b-2).
template <typename TS>
__global__ void __launch_bounds__(256) k_prefilter(IngestPair p)
{
    const IngestArgs &a = p.f[blockIdx.z];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= a.H || j >= a.W) return;
    float s = 0.f;
#pragma unroll
    for (int r = 0; r < 5; ++r) {
        const float *row = a.tmp + (int64_t)clampi(i + r - 2, 0, a.H - 1) * a.pitch;
#pragma unroll
        for (int c = 0; c < 5; ++c) s = fmaf(__ldg(a.w25 + r * 5 + c), __ldg(row + clampi(j + c - 2, 0, a.W - 1)), s);
    }
    st_store(static_cast<TS *>(a.out) + (int64_t)i * a.pitch + j, s);
}

template <typename TS>
static cudaError_t ingest_t(const IngestPair &p, int nframes, cudaStream_t s)
{
    const IngestArgs &a = p.f[0];
    dim3 blk(32, 8);
    dim3 grd((a.W + 31) / 32, (a.H + 7) / 8, nframes);
    switch (a.in_type) {
    case IN_U8: k_ingest<uint8_t, TS><<<grd, blk, 0, s>>>(p); break;
    case IN_U16: k_ingest<uint16_t, TS><<<grd, blk, 0, s>>>(p); break;
    default: k_ingest<float, TS><<<grd, blk, 0, s>>>(p); break;
    }
    if (a.prefilter) k_prefilter<TS><<<grd, blk, 0, s>>>(p);
    return cudaGetLastError();
}

// Ingest nframes (1 .. kMaxFramesPerLaunch) frames in one launch
// (gridDim.z = nframes).
cudaError_t launch_ingest_frames(const IngestArgs *f, int nframes, int store, cudaStream_t s)
{
    if (nframes < 1 || nframes > kMaxFramesPerLaunch) return cudaErrorInvalidValue;
    IngestPair p;
    for (int k = 0; k < nframes; ++k) p.f[k] = f[k];
    p.scale = f[0].in_type == IN_F32 ? 1.0f : 1.0f / (float)((1u << f[0].bits) - 1u);
    switch (store) {
    case ST_F16: return ingest_t<__half>(p, nframes, s);
    case ST_BF16: return ingest_t<__nv_bfloat16>(p, nframes, s);
    default: return ingest_t<float>(p, nframes, s);
    }
}

// ---------------------------------------------------------------------------
// Pyramid reduction: out(i,j) = sum_{a,b=-2..2} c_a c_b P(2i+a, 2j+b),
// c = [1 4 6 4 1]/16, clamp-to-edge, out size ceil(H/2) x ceil(W/2).
// ---------------------------------------------------------------------------
struct ReducePair { ReduceArgs f[kMaxFramesPerLaunch]; };

template <typename TS>
__global__ void __launch_bounds__(256) k_reduce(ReducePair p)
{
    const ReduceArgs &a = p.f[blockIdx.z];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= a.Hd || j >= a.Wd) return;
    const TS *src = static_cast<const TS *>(a.src);
    const float c[5] = {0.0625f, 0.25f, 0.375f, 0.25f, 0.0625f};
    int cols[5];
#pragma unroll
    for (int b = 0; b < 5; ++b) cols[b] = clampi(2 * j + b - 2, 0, a.Ws - 1);
    float acc = 0.f;
#pragma unroll
    for (int r = 0; r < 5; ++r) {
        const TS *row = src + (int64_t)clampi(2 * i + r - 2, 0, a.Hs - 1) * a.spitch;
        float h = 0.f;
#pragma unroll
        for (int b = 0; b < 5; ++b) h = fmaf(c[b], ld_store(row + cols[b]), h);
        acc = fmaf(c[r], h, acc);
    }
    st_store(static_cast<TS *>(a.dst) + (int64_t)i * a.dpitch + j, acc);
}

// Reduce one level of nframes (1 .. kMaxFramesPerLaunch) frames in one launch.
cudaError_t launch_reduce_frames(const ReduceArgs *f, int nframes, int store, cudaStream_t s)
{
    if (nframes < 1 || nframes > kMaxFramesPerLaunch) return cudaErrorInvalidValue;
    ReducePair p;
    for (int k = 0; k < nframes; ++k) p.f[k] = f[k];
    dim3 blk(32, 8);
    dim3 grd((f[0].Wd + 31) / 32, (f[0].Hd + 7) / 8, nframes);
    switch (store) {
    case ST_F16: k_reduce<__half><<<grd, blk, 0, s>>>(p); break;
    case ST_BF16: k_reduce<__nv_bfloat16><<<grd, blk, 0, s>>>(p); break;
    default: k_reduce<float><<<grd, blk, 0, s>>>(p); break;
    }
    return cudaGetLastError();
}

// Dense FP32 copy of a stored level (inspection).
template <typename TS>
__global__ void k_read_level(const TS *src, int H, int W, int pitch, float *dst)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= H || j >= W) return;
    dst[(int64_t)i * W + j] = ld_store(src + (int64_t)i * pitch + j);
}

cudaError_t launch_read_level(const void *src, int H, int W, int pitch, int store, float *dst,
                              cudaStream_t s)
{
    dim3 blk(32, 8);
    dim3 grd((W + 31) / 32, (H + 7) / 8);
    switch (store) {
    case ST_F16: k_read_level<<<grd, blk, 0, s>>>(static_cast<const __half *>(src), H, W, pitch, dst); break;
    case ST_BF16: k_read_level<<<grd, blk, 0, s>>>(static_cast<const __nv_bfloat16 *>(src), H, W, pitch, dst); break;
    default: k_read_level<<<grd, blk, 0, s>>>(static_cast<const float *>(src), H, W, pitch, dst); break;
    }
    return cudaGetLastError();
}

}  // namespace ofv
