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

// nrows: tile rows of the launch from p.by0 on (0: to the bottom of the level)
template <typename T, bool VAR>
cudaError_t launch_block_t(const BlockParams &p, int kr, int npairs, cudaStream_t s, int nrows)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const IterArgs &a = p.a[0];
    switch (kr) {
#define OFV_BLOCK_CASE(K)                                                                                  \
    case K: {                                                                                              \
        constexpr int TS = BlockShape<K>::TS;                                                              \
        const int nby = nrows > 0 ? nrows : (a.H + TS - 1) / TS - p.by0;                                   \
        return run_block<T, K, VAR>(p, dim3((a.W + TS - 1) / TS, nby, npairs), dev, s);                    \
    }
    OFV_BLOCK_CASE(1) OFV_BLOCK_CASE(2) OFV_BLOCK_CASE(3) OFV_BLOCK_CASE(4) OFV_BLOCK_CASE(5)
    OFV_BLOCK_CASE(6) OFV_BLOCK_CASE(7) OFV_BLOCK_CASE(8) OFV_BLOCK_CASE(9) OFV_BLOCK_CASE(10)
#undef OFV_BLOCK_CASE
    default: return cudaErrorInvalidValue;
    }
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
cudaError_t launch_queue_t(const QueueParams &q, int kr, int ctas, cudaStream_t s)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    switch (kr) {
#define OFV_QUEUE_CASE(K) \
    case K: return run_queue<T, K, VAR>(q, ctas, dev, s);
    OFV_QUEUE_CASE(1) OFV_QUEUE_CASE(2) OFV_QUEUE_CASE(3) OFV_QUEUE_CASE(4) OFV_QUEUE_CASE(5)
    OFV_QUEUE_CASE(6) OFV_QUEUE_CASE(7) OFV_QUEUE_CASE(8) OFV_QUEUE_CASE(9) OFV_QUEUE_CASE(10)
#undef OFV_QUEUE_CASE
    default: return cudaErrorInvalidValue;
    }
}

// Resident CTAs per SM of the persistent kernel.
template <typename T, bool VAR>
int queue_occupancy_t(int kr)
{
    switch (kr) {
#define OFV_OCC_CASE(K) \
    case K: return queue_occupancy_kr<T, K, VAR>();
    OFV_OCC_CASE(1) OFV_OCC_CASE(2) OFV_OCC_CASE(3) OFV_OCC_CASE(4) OFV_OCC_CASE(5)
    OFV_OCC_CASE(6) OFV_OCC_CASE(7) OFV_OCC_CASE(8) OFV_OCC_CASE(9) OFV_OCC_CASE(10)
#undef OFV_OCC_CASE
    default: return 0;
    }
}

#define OFV_INSTANTIATE_BLOCK_LAUNCHERS(T, VAR)                                                     \
    template cudaError_t launch_block_t<T, VAR>(const BlockParams &, int, int, cudaStream_t, int); \
    template cudaError_t launch_queue_t<T, VAR>(const QueueParams &, int, int, cudaStream_t);      \
    template int queue_occupancy_t<T, VAR>(int);

}  // namespace ofv
