// Ingest (scale, local normalization, optional 5x5 pre-filter) and
// Burt-Adelson pyramid reduction kernels.
//
// Sec. 2 of the paper: step 1 is a local, pixel-centred intensity
// normalization of radius NR; step 2 builds a Gaussian pyramid in which each
// sub-level halves both image dimensions (Burt & Adelson's reduction).
#include <algorithm>

#include "ofv_common.cuh"

namespace ofv {

template <typename TI>
__device__ __forceinline__ float ld_in(const TI *p);
template <> __device__ __forceinline__ float ld_in<uint8_t>(const uint8_t *p) { return (float)__ldg(p); }
template <> __device__ __forceinline__ float ld_in<uint16_t>(const uint16_t *p) { return (float)__ldg(p); }
template <> __device__ __forceinline__ float ld_in<float>(const float *p) { return __ldg(p); }

// The frames of one launch: a few passed by value, or any number in device
// memory (the batched entry point); blockIdx.z selects the frame.
struct IngestPair {
    IngestArgs f[kMaxFramesPerLaunch];
    float scale;
    __device__ __forceinline__ const IngestArgs &get(int k) const { return f[k]; }
};
struct IngestList {
    const IngestArgs *f;
    float scale;
    __device__ __forceinline__ const IngestArgs &get(int k) const { return f[k]; }
};

// Scaled intensity I = raw * scale (scale = 1/(2^bits - 1), or 1 for FP32
// input), then, for NR > 0, (I - mu) / sqrt(var + eps_n^2) with mu and var
// taken over the in-image part of the (2NR+1)^2 box.  Writes level 0 in the
// storage type, or FP32 scratch when a pre-filter follows.  With NR > 0 it
// serves only NR > 16 (k_ingest_norm below covers 1 .. 16, with the mean
// from separable sums: the two agree to FP32 rounding).
template <typename TI, typename TS, typename FR>
__global__ void __launch_bounds__(256) k_ingest(const __grid_constant__ FR p)
{
    const IngestArgs &a = p.get(blockIdx.z);
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

// The same with the boxes in shared memory: a CTA of 32 x 8 threads stages
// a 32 x 32 block (four rows per thread) and the NR halo (scaled values,
// zero outside the image, so the boxes are truncated there).  The mean comes from separable sums:
// row sums over 2NR+1 columns for every staged row, then 2NR+1 of them down
// each output column.  The variance is the centred sum of (I - mu)^2 over
// the in-image box (E[I^2] - mu^2 cancels too many digits where the box is
// flat), with the loop unrolled for NR 1 .. 4 (template NRC) and the box
// bounds tested only for pixels within NR of the border.
template <int NRC, typename TI, typename TS, typename FR>
__device__ __forceinline__ void ingest_norm_tile(const FR &p)
{
    extern __shared__ float tile[];  // (32 + 2 NR) rows of (32 + 2 NR), then (32 + 2 NR) x 32 row sums
    const IngestArgs &a = p.get(blockIdx.z);
    const int nr = NRC > 0 ? NRC : a.nr, K = 2 * nr + 1;
    const int TW = 32 + 2 * nr, TH = 32 + 2 * nr;
    float *rs = tile + TH * TW;
    const int bx0 = blockIdx.x * 32, by0 = blockIdx.y * 32;
    if (bx0 >= a.W || by0 >= a.H) return;  // the whole CTA lies outside this frame
    const int x0 = bx0 - nr, y0 = by0 - nr;
    const TI *raw = static_cast<const TI *>(a.raw);
    const float sc = p.scale;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    for (int t = tid; t < TW * TH; t += 256) {
        const int r = t / TW, c = t - r * TW;
        const int gy = y0 + r, gx = x0 + c;
        tile[t] = (gy >= 0 && gy < a.H && gx >= 0 && gx < a.W) ? ld_in(raw + (int64_t)gy * a.W + gx) * sc : 0.f;
    }
    __syncthreads();
    for (int t = tid; t < TH * 32; t += 256) {
        const float *row = tile + (t >> 5) * TW + (t & 31);
        float s1 = 0.f;
        if constexpr (NRC > 0) {
#pragma unroll
            for (int k = 0; k < 2 * NRC + 1; ++k) s1 += row[k];
        } else {
            for (int k = 0; k < K; ++k) s1 += row[k];
        }
        rs[t] = s1;
    }
    __syncthreads();
    const int j = bx0 + threadIdx.x;
    if (j >= a.W) return;
    const int j0 = max(j - nr, 0), j1 = min(j + nr, a.W - 1);
#pragma unroll 1
    for (int ly = threadIdx.y; ly < 32; ly += 8) {
        const int i = by0 + ly;
        if (i >= a.H) break;
        const int i0 = max(i - nr, 0), i1 = min(i + nr, a.H - 1);
        const float inv_n = 1.0f / (float)((i1 - i0 + 1) * (j1 - j0 + 1));
        float s1 = 0.f;
        if constexpr (NRC > 0) {
#pragma unroll
            for (int k = 0; k < 2 * NRC + 1; ++k) s1 += rs[(ly + k) * 32 + threadIdx.x];
        } else {
            for (int k = 0; k < K; ++k) s1 += rs[(ly + k) * 32 + threadIdx.x];
        }
        const float mu = s1 * inv_n;
        float q = 0.f;
        const float *box = tile + ly * TW + threadIdx.x;  // staged (i - nr, j - nr)
        if (NRC > 0 && i - nr >= 0 && i + nr < a.H && j - nr >= 0 && j + nr < a.W) {
#pragma unroll
            for (int r = 0; r < 2 * NRC + 1; ++r)
#pragma unroll
                for (int c = 0; c < 2 * NRC + 1; ++c) {
                    const float d = box[r * TW + c] - mu;
                    q = fmaf(d, d, q);
                }
        } else {
            for (int ii = i0; ii <= i1; ++ii) {
                const float *row = tile + (ii - y0) * TW;
                for (int jj = j0; jj <= j1; ++jj) {
                    const float d = row[jj - x0] - mu;
                    q = fmaf(d, d, q);
                }
            }
        }
        const float var = q * inv_n;
        const float val = (tile[(ly + nr) * TW + threadIdx.x + nr] - mu) * rsqrtf(var + a.eps_n * a.eps_n);
        if (a.prefilter)
            a.tmp[(int64_t)i * a.pitch + j] = val;
        else
            st_store(static_cast<TS *>(a.out) + (int64_t)i * a.pitch + j, val);
    }
}

template <typename TI, typename TS, typename FR>
__global__ void __launch_bounds__(256) k_ingest_norm(const __grid_constant__ FR p)
{
    switch (p.get(blockIdx.z).nr) {
    case 1: ingest_norm_tile<1, TI, TS>(p); break;
    case 2: ingest_norm_tile<2, TI, TS>(p); break;
    case 3: ingest_norm_tile<3, TI, TS>(p); break;
    case 4: ingest_norm_tile<4, TI, TS>(p); break;
    default: ingest_norm_tile<0, TI, TS>(p); break;
    }
}

// Ingest without normalization or pre-filter (the common case): I = raw *
// scale stored directly, eight pixels per thread with 16-byte stores (rows
// of W % 8 == 0 pixels, 16-byte aligned input).
template <typename TI> struct Raw8;
template <> struct Raw8<uint8_t> { using V = uint2; };
template <> struct Raw8<uint16_t> { using V = uint4; };

__device__ __forceinline__ void unpack8(uint2 r, float sc, float f[8])
{
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        f[k] = (float)((r.x >> (8 * k)) & 0xffu) * sc;
        f[4 + k] = (float)((r.y >> (8 * k)) & 0xffu) * sc;
    }
}
__device__ __forceinline__ void unpack8(uint4 r, float sc, float f[8])
{
    const unsigned w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        f[2 * k] = (float)(w[k] & 0xffffu) * sc;
        f[2 * k + 1] = (float)(w[k] >> 16) * sc;
    }
}

__device__ __forceinline__ void store8(float *d, const float f[8])
{
    reinterpret_cast<float4 *>(d)[0] = make_float4(f[0], f[1], f[2], f[3]);
    reinterpret_cast<float4 *>(d)[1] = make_float4(f[4], f[5], f[6], f[7]);
}
__device__ __forceinline__ void store8(__half *d, const float f[8])
{
    __half2 h[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) h[k] = __floats2half2_rn(f[2 * k], f[2 * k + 1]);
    *reinterpret_cast<uint4 *>(d) = *reinterpret_cast<const uint4 *>(h);
}
__device__ __forceinline__ void store8(__nv_bfloat16 *d, const float f[8])
{
    __nv_bfloat162 h[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) h[k] = __floats2bfloat162_rn(f[2 * k], f[2 * k + 1]);
    *reinterpret_cast<uint4 *>(d) = *reinterpret_cast<const uint4 *>(h);
}

template <typename TI, typename TS, typename FR>
__global__ void __launch_bounds__(256) k_ingest8(const __grid_constant__ FR p)
{
    const IngestArgs &a = p.get(blockIdx.z);
    const int W8 = a.W >> 3;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)W8 * a.H) return;
    const int i = (int)(t / W8), j = (int)(t - (int64_t)i * W8) * 8;
    float f[8];
    const TI *src = static_cast<const TI *>(a.raw) + (int64_t)i * a.W + j;
    if constexpr (sizeof(TI) == 4) {
        const float4 x0 = __ldg(reinterpret_cast<const float4 *>(src));
        const float4 x1 = __ldg(reinterpret_cast<const float4 *>(src) + 1);
        f[0] = x0.x; f[1] = x0.y; f[2] = x0.z; f[3] = x0.w;
        f[4] = x1.x; f[5] = x1.y; f[6] = x1.z; f[7] = x1.w;
    } else {
        unpack8(__ldg(reinterpret_cast<const typename Raw8<TI>::V *>(src)), p.scale, f);
    }
    store8(static_cast<TS *>(a.out) + (int64_t)i * a.pitch + j, f);
}

// 5x5 correlation with clamp-to-edge: out(i,j) = sum w[a][b] I(i+a-2, j+b-2).
template <typename TS, typename FR>
__global__ void __launch_bounds__(256) k_prefilter(const __grid_constant__ FR p)
{
    const IngestArgs &a = p.get(blockIdx.z);
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

// f: the frames on the host (sizes, types and alignment decide the form and
// the grid, which covers the largest frame); p: the same frames as the
// kernels read them.
template <typename TS, typename FR>
static cudaError_t ingest_t(const FR &p, const IngestArgs *f, int nframes, cudaStream_t s)
{
    const IngestArgs &a = f[0];
    bool vec = a.nr == 0 && !a.prefilter;
    int64_t n8 = 0;
    int H = 0, W = 0;
    for (int k = 0; k < nframes; ++k) {
        vec = vec && f[k].W % 8 == 0 && (reinterpret_cast<uintptr_t>(f[k].raw) & 15u) == 0;
        n8 = std::max<int64_t>(n8, (int64_t)(f[k].W / 8) * f[k].H);
        H = std::max(H, f[k].H);
        W = std::max(W, f[k].W);
    }
    if (vec) {
        dim3 grd((unsigned)((n8 + 255) / 256), 1, nframes);
        switch (a.in_type) {
        case IN_U8: k_ingest8<uint8_t, TS, FR><<<grd, 256, 0, s>>>(p); break;
        case IN_U16: k_ingest8<uint16_t, TS, FR><<<grd, 256, 0, s>>>(p); break;
        default: k_ingest8<float, TS, FR><<<grd, 256, 0, s>>>(p); break;
        }
        return cudaGetLastError();
    }
    dim3 blk(32, 8);
    dim3 grd((W + 31) / 32, (H + 7) / 8, nframes);
    if (a.nr > 0 && a.nr <= 16) {
        const size_t smem = sizeof(float) * (size_t)(32 + 2 * a.nr) * (32 + 2 * a.nr + 32);
        const dim3 grdn((W + 31) / 32, (H + 31) / 32, nframes);
        switch (a.in_type) {
        case IN_U8: k_ingest_norm<uint8_t, TS, FR><<<grdn, blk, smem, s>>>(p); break;
        case IN_U16: k_ingest_norm<uint16_t, TS, FR><<<grdn, blk, smem, s>>>(p); break;
        default: k_ingest_norm<float, TS, FR><<<grdn, blk, smem, s>>>(p); break;
        }
    } else {
        switch (a.in_type) {
        case IN_U8: k_ingest<uint8_t, TS, FR><<<grd, blk, 0, s>>>(p); break;
        case IN_U16: k_ingest<uint16_t, TS, FR><<<grd, blk, 0, s>>>(p); break;
        default: k_ingest<float, TS, FR><<<grd, blk, 0, s>>>(p); break;
        }
    }
    if (a.prefilter) k_prefilter<TS, FR><<<grd, blk, 0, s>>>(p);
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
    case ST_F16: return ingest_t<__half>(p, f, nframes, s);
    case ST_BF16: return ingest_t<__nv_bfloat16>(p, f, nframes, s);
    default: return ingest_t<float>(p, f, nframes, s);
    }
}

// Any number of frames (of any sizes) in one launch: f on the host, dev_f
// the same descriptors in device memory (kept until the launch has run).
cudaError_t launch_ingest_list(const IngestArgs *f, const IngestArgs *dev_f, int nframes, int store, cudaStream_t s)
{
    if (nframes < 1 || nframes > 65535) return cudaErrorInvalidValue;
    IngestList p{dev_f, f[0].in_type == IN_F32 ? 1.0f : 1.0f / (float)((1u << f[0].bits) - 1u)};
    switch (store) {
    case ST_F16: return ingest_t<__half>(p, f, nframes, s);
    case ST_BF16: return ingest_t<__nv_bfloat16>(p, f, nframes, s);
    default: return ingest_t<float>(p, f, nframes, s);
    }
}

// ---------------------------------------------------------------------------
// Pyramid reduction: out(i,j) = sum_{a,b=-2..2} c_a c_b P(2i+a, 2j+b),
// c = [1 4 6 4 1]/16, clamp-to-edge, out size ceil(H/2) x ceil(W/2).
// ---------------------------------------------------------------------------
struct ReducePair {
    ReduceArgs f[kMaxFramesPerLaunch];
    __device__ __forceinline__ const ReduceArgs &get(int k) const { return f[k]; }
};
struct ReduceList {
    const ReduceArgs *f;
    __device__ __forceinline__ const ReduceArgs &get(int k) const { return f[k]; }
};

// Two horizontally adjacent outputs j = 2t, 2t+1 per thread: they share
// input columns 4t-2 .. 4t+4 (7 loads per row instead of 10), loaded as
// 8-byte pairs for FP32 storage away from the left and right borders.  Each
// output is accumulated in the same order as the one-output form.
template <typename TS>
__device__ __forceinline__ void load7(const TS *row, int c0, int Ws, bool inside, float v[7])
{
#pragma unroll
    for (int k = 0; k < 7; ++k) v[k] = ld_store(row + (inside ? c0 + k : clampi(c0 + k, 0, Ws - 1)));
}
template <>
__device__ __forceinline__ void load7<float>(const float *row, int c0, int Ws, bool inside, float v[7])
{
    if (inside) {  // c0 even, row 8-byte aligned
        const float2 a = __ldg(reinterpret_cast<const float2 *>(row + c0));
        const float2 b = __ldg(reinterpret_cast<const float2 *>(row + c0 + 2));
        const float2 c = __ldg(reinterpret_cast<const float2 *>(row + c0 + 4));
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y; v[4] = c.x; v[5] = c.y;
        v[6] = __ldg(row + c0 + 6);
        return;
    }
#pragma unroll
    for (int k = 0; k < 7; ++k) v[k] = __ldg(row + clampi(c0 + k, 0, Ws - 1));
}

template <typename TS, typename FR>
__global__ void __launch_bounds__(256) k_reduce(const __grid_constant__ FR p)
{
    const ReduceArgs &a = p.get(blockIdx.z);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    const int j0 = 2 * t;
    if (i >= a.Hd || j0 >= a.Wd) return;
    const TS *src = static_cast<const TS *>(a.src);
    const float c[5] = {0.0625f, 0.25f, 0.375f, 0.25f, 0.0625f};
    const int c0 = 2 * j0 - 2;  // first input column of output j0
    const bool inside = c0 >= 0 && c0 + 6 <= a.Ws - 1;
    float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
    for (int r = 0; r < 5; ++r) {
        const TS *row = src + (int64_t)clampi(2 * i + r - 2, 0, a.Hs - 1) * a.spitch;
        float v[7];
        load7<TS>(row, c0, a.Ws, inside, v);
        float h0 = 0.f, h1 = 0.f;
#pragma unroll
        for (int b = 0; b < 5; ++b) {
            h0 = fmaf(c[b], v[b], h0);
            h1 = fmaf(c[b], v[b + 2], h1);
        }
        acc0 = fmaf(c[r], h0, acc0);
        acc1 = fmaf(c[r], h1, acc1);
    }
    TS *dst = static_cast<TS *>(a.dst) + (int64_t)i * a.dpitch;
    st_store(dst + j0, acc0);
    if (j0 + 1 < a.Wd) st_store(dst + j0 + 1, acc1);
}

// The grid covers the largest output of the frames (each exits outside its own).
template <typename FR>
static cudaError_t reduce_t(const FR &p, const ReduceArgs *f, int nframes, int store, cudaStream_t s)
{
    int Hd = 0, Wd = 0;
    for (int k = 0; k < nframes; ++k) {
        Hd = std::max(Hd, f[k].Hd);
        Wd = std::max(Wd, f[k].Wd);
    }
    dim3 blk(32, 8);
    dim3 grd(((Wd + 1) / 2 + 31) / 32, (Hd + 7) / 8, nframes);
    switch (store) {
    case ST_F16: k_reduce<__half, FR><<<grd, blk, 0, s>>>(p); break;
    case ST_BF16: k_reduce<__nv_bfloat16, FR><<<grd, blk, 0, s>>>(p); break;
    default: k_reduce<float, FR><<<grd, blk, 0, s>>>(p); break;
    }
    return cudaGetLastError();
}

// Reduce one level of nframes (1 .. kMaxFramesPerLaunch) frames in one launch.
cudaError_t launch_reduce_frames(const ReduceArgs *f, int nframes, int store, cudaStream_t s)
{
    if (nframes < 1 || nframes > kMaxFramesPerLaunch) return cudaErrorInvalidValue;
    ReducePair p;
    for (int k = 0; k < nframes; ++k) p.f[k] = f[k];
    return reduce_t(p, f, nframes, store, s);
}

// Any number of frames (of any sizes) in one launch (see launch_ingest_list).
cudaError_t launch_reduce_list(const ReduceArgs *f, const ReduceArgs *dev_f, int nframes, int store, cudaStream_t s)
{
    if (nframes < 1 || nframes > 65535) return cudaErrorInvalidValue;
    return reduce_t(ReduceList{dev_f}, f, nframes, store, s);
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

// Warm start (a variant for time-resolved sequences): the coarsest level's
// starting field taken from an earlier level-0 field at the pixels that
// level keeps, V_L(i, j) = V(2^L i, 2^L j) / 2^L.  Division by a power of two
// is exact.  One launch for up to kMaxPairsPerLaunch fields (blockIdx.z).
struct SeedPack {
    SeedArgs a[kMaxPairsPerLaunch];
};

__global__ void __launch_bounds__(256) k_seed_field(const __grid_constant__ SeedPack p)
{
    const SeedArgs &a = p.a[blockIdx.z];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= a.W) return;
    const float sc = 1.f / (float)(1 << a.level);
    for (int i = blockIdx.y; i < a.H; i += gridDim.y) {
        const int64_t src = ((int64_t)i * a.W0 << a.level) + ((int64_t)j << a.level);
        a.out[(int64_t)i * a.vpitch + j] = make_float2(__ldg(a.u + src) * sc, __ldg(a.v + src) * sc);
    }
}

// Region mask (a variant; masked regions of Sec. 7 such as a model and its
// shadow): level l keeps the level-0 mask at (2^l i, 2^l j), as 0 / 1.
__global__ void __launch_bounds__(256) k_mask_level(const uint8_t *__restrict__ mask, int W0, int level,
                                                    uint8_t *__restrict__ out, int H, int W)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= W) return;
    for (int i = blockIdx.y; i < H; i += gridDim.y)
        out[(int64_t)i * W + j] = __ldg(mask + ((int64_t)i * W0 << level) + ((int64_t)j << level)) != 0 ? 1 : 0;
}

cudaError_t launch_mask_levels(const uint8_t *mask, int W, uint8_t *const *out, const int *Hs, const int *Ws, int L,
                               cudaStream_t s)
{
    for (int l = 0; l < L; ++l) {
        k_mask_level<<<dim3((Ws[l] + 255) / 256, Hs[l] < 65535 ? Hs[l] : 65535), 256, 0, s>>>(mask, W, l, out[l], Hs[l],
                                                                                             Ws[l]);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_seed_fields(const SeedArgs *a, int n, cudaStream_t s)
{
    if (n < 1 || n > kMaxPairsPerLaunch) return cudaErrorInvalidValue;
    SeedPack p;
    int H = 0, W = 0;
    for (int k = 0; k < n; ++k) {
        p.a[k] = a[k];
        H = a[k].H > H ? a[k].H : H;
        W = a[k].W > W ? a[k].W : W;
    }
    k_seed_field<<<dim3((W + 255) / 256, H < 65535 ? H : 65535, n), 256, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace ofv
