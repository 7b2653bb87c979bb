// Definitions of the block kernels' host launchers for one level storage
// type T and variant flag VAR, for window radii 1..10.  Each k_block_*.cu
// translation unit instantiates one (T, VAR) pair, so the instantiations
// compile in parallel.
#pragma once
#include "k_block.cuh"

namespace ofv {

template <typename T, int KR, bool VAR>
cudaError_t run_block(const BlockParams &p, dim3 grid, int dev, cudaStream_t s)
{
    static size_t granted[64] = {};  // dynamic shared memory raised per device
    constexpr size_t smem = block_smem_bytes<T, KR>();
    auto kern = k_iter_block<T, KR, VAR>;
    if (dev < 0 || dev >= 64 || granted[dev] < smem) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) granted[dev] = smem;
    }
    kern<<<grid, BlockShape<KR>::NT, smem, s>>>(p);
    return cudaGetLastError();
}

// KS = kr + 16 shape for the radii and shapes instantiated here: every
// radius with its default shape; the alternative shapes without the
// estimator variants.  0 when not instantiated.
template <bool VAR>
constexpr int ks_of(int kr, int shape)
{
    return (kr < 1 || kr > kBlockMaxKR || shape < 0 || shape > 1 || (VAR && shape != 0)) ? 0 : kr + 16 * shape;
}

#define OFV_KS_CASES(X)                                                                                    \
    X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10)                                                      \
    OFV_KS_ALT(X, 17) OFV_KS_ALT(X, 18) OFV_KS_ALT(X, 19) OFV_KS_ALT(X, 20) OFV_KS_ALT(X, 21)                \
    OFV_KS_ALT(X, 22) OFV_KS_ALT(X, 23) OFV_KS_ALT(X, 24) OFV_KS_ALT(X, 25) OFV_KS_ALT(X, 26)

// nrows: tile rows of the launch from p.by0 on (0: to the bottom of the level)
template <typename T, bool VAR>
cudaError_t launch_block_t(const BlockParams &p, int kr, int npairs, cudaStream_t s, int nrows, int shape)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const IterArgs &a = p.a[0];
    switch (ks_of<VAR>(kr, shape)) {
#define OFV_KS_ALT(X, K) \
    case K:              \
        if constexpr (!VAR) { X##_BODY(K) } else { break; }
#define OFV_BLOCK_CASE(K) case K: OFV_BLOCK_CASE_BODY(K)
#define OFV_BLOCK_CASE_BODY(K)                                                                             \
    {                                                                                                      \
        constexpr int TS = BlockShape<K>::TS;                                                              \
        const int nby = nrows > 0 ? nrows : (a.H + TS - 1) / TS - p.by0;                                   \
        return run_block<T, K, VAR>(p, dim3((a.W + TS - 1) / TS, nby, npairs), dev, s);                    \
    }
    OFV_KS_CASES(OFV_BLOCK_CASE)
#undef OFV_BLOCK_CASE
#undef OFV_BLOCK_CASE_BODY
#undef OFV_KS_ALT
    default: break;
    }
    return cudaErrorInvalidValue;
}

template <typename T, int KR, bool VAR>
cudaError_t run_queue(const QueueParams &q, int ctas, int dev, cudaStream_t s)
{
    static size_t granted[64] = {};
    constexpr size_t smem = block_smem_bytes<T, KR>();
    auto kern = k_iter_queue<T, KR, VAR>;
    if (dev < 0 || dev >= 64 || granted[dev] < smem) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) granted[dev] = smem;
    }
    kern<<<ctas, BlockShape<KR>::NT, smem, s>>>(q);
    return cudaGetLastError();
}

template <typename T, int KR, bool VAR>
int queue_occupancy_kr()
{
    constexpr size_t smem = block_smem_bytes<T, KR>();
    cudaFuncSetAttribute(k_iter_queue<T, KR, VAR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_iter_queue<T, KR, VAR>, BlockShape<KR>::NT, smem) !=
        cudaSuccess)
        return 0;
    return n;
}

// Persistent batched launch with ctas CTAs (at most the resident count).
template <typename T, bool VAR>
cudaError_t launch_queue_t(const QueueParams &q, int kr, int ctas, cudaStream_t s, int shape)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    switch (ks_of<VAR>(kr, shape)) {
#define OFV_KS_ALT(X, K) \
    case K:              \
        if constexpr (!VAR) { X##_BODY(K) } else { break; }
#define OFV_QUEUE_CASE(K) case K: OFV_QUEUE_CASE_BODY(K)
// the persistent kernel's own thread count: KS | 32 (see BlockShape)
#define OFV_QUEUE_CASE_BODY(K) return run_queue<T, (K) | 32, VAR>(q, ctas, dev, s);
    OFV_KS_CASES(OFV_QUEUE_CASE)
#undef OFV_QUEUE_CASE
#undef OFV_QUEUE_CASE_BODY
#undef OFV_KS_ALT
    default: break;
    }
    return cudaErrorInvalidValue;
}

// Resident CTAs per SM of the persistent kernel.
template <typename T, bool VAR>
int queue_occupancy_t(int kr, int shape)
{
    switch (ks_of<VAR>(kr, shape)) {
#define OFV_KS_ALT(X, K) \
    case K:              \
        if constexpr (!VAR) { X##_BODY(K) } else { break; }
#define OFV_OCC_CASE(K) case K: OFV_OCC_CASE_BODY(K)
#define OFV_OCC_CASE_BODY(K) return queue_occupancy_kr<T, (K) | 32, VAR>();
    OFV_KS_CASES(OFV_OCC_CASE)
#undef OFV_OCC_CASE
#undef OFV_OCC_CASE_BODY
#undef OFV_KS_ALT
    default: break;
    }
    return 0;
}

#define OFV_INSTANTIATE_BLOCK_LAUNCHERS(T, VAR)                                                     \
    template cudaError_t launch_block_t<T, VAR>(const BlockParams &, int, int, cudaStream_t, int, int); \
    template cudaError_t launch_queue_t<T, VAR>(const QueueParams &, int, int, cudaStream_t, int);      \
    template int queue_occupancy_t<T, VAR>(int, int);

}  // namespace ofv
