// Block-tiled iteration kernel instantiated for float level storage, window
// radii 1..10.
#include "k_block.cuh"
#include "k_bw_block.cuh"

namespace ofv {

namespace {
size_t g_granted_f32[64][kBlockMaxKR + 1];

template <int KR>
cudaError_t run_f32(const BlockParams &p, dim3 grid, int dev, cudaStream_t s)
{
    constexpr size_t smem = block_smem_bytes<float, KR>();
    auto kern = k_iter_block<float, KR>;
    if (dev < 0 || dev >= 64 || g_granted_f32[dev][KR] < smem) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) g_granted_f32[dev][KR] = smem;
    }
    kern<<<grid, BlockShape<KR>::NT, smem, s>>>(p);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_block_f32(const BlockParams &p, int kr, int npairs, cudaStream_t s)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const IterArgs &a = p.a[0];
    switch (kr) {
#define OFV_BLOCK_CASE(K)                                                                          \
    case K: {                                                                                      \
        constexpr int TS = BlockShape<K>::TS;                                                      \
        return run_f32<K>(p, dim3((a.W + TS - 1) / TS, (a.H + TS - 1) / TS, npairs), dev, s);     \
    }
    OFV_BLOCK_CASE(1) OFV_BLOCK_CASE(2) OFV_BLOCK_CASE(3) OFV_BLOCK_CASE(4) OFV_BLOCK_CASE(5)
    OFV_BLOCK_CASE(6) OFV_BLOCK_CASE(7) OFV_BLOCK_CASE(8) OFV_BLOCK_CASE(9) OFV_BLOCK_CASE(10)
#undef OFV_BLOCK_CASE
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ofv

namespace ofv {

namespace {
size_t g_qgranted_f32[64][kBlockMaxKR + 1];

template <int KR>
cudaError_t runq_f32(const QueueParams &q, int ctas, int dev, cudaStream_t s)
{
    constexpr size_t smem = block_smem_bytes<float, KR>();
    auto kern = k_iter_queue<float, KR>;
    if (dev < 0 || dev >= 64 || g_qgranted_f32[dev][KR] < smem) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) g_qgranted_f32[dev][KR] = smem;
    }
    kern<<<ctas, BlockShape<KR>::NT, smem, s>>>(q);
    return cudaGetLastError();
}

template <int KR>
int occq_f32()
{
    constexpr size_t smem = block_smem_bytes<float, KR>();
    cudaFuncSetAttribute(k_iter_queue<float, KR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_iter_queue<float, KR>, BlockShape<KR>::NT, smem) != cudaSuccess)
        return 0;
    return n;
}
}  // namespace

// Persistent batched launch with ctas CTAs (at most the resident count).
cudaError_t launch_queue_f32(const QueueParams &q, int kr, int ctas, cudaStream_t s)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    switch (kr) {
#define OFV_QUEUE_CASE(K) \
    case K: return runq_f32<K>(q, ctas, dev, s);
    OFV_QUEUE_CASE(1) OFV_QUEUE_CASE(2) OFV_QUEUE_CASE(3) OFV_QUEUE_CASE(4) OFV_QUEUE_CASE(5)
    OFV_QUEUE_CASE(6) OFV_QUEUE_CASE(7) OFV_QUEUE_CASE(8) OFV_QUEUE_CASE(9) OFV_QUEUE_CASE(10)
#undef OFV_QUEUE_CASE
    default: return cudaErrorInvalidValue;
    }
}

// Resident CTAs per SM of the persistent kernel.
int queue_occupancy_f32(int kr)
{
    switch (kr) {
#define OFV_OCC_CASE(K) \
    case K: return occq_f32<K>();
    OFV_OCC_CASE(1) OFV_OCC_CASE(2) OFV_OCC_CASE(3) OFV_OCC_CASE(4) OFV_OCC_CASE(5)
    OFV_OCC_CASE(6) OFV_OCC_CASE(7) OFV_OCC_CASE(8) OFV_OCC_CASE(9) OFV_OCC_CASE(10)
#undef OFV_OCC_CASE
    default: return 0;
    }
}

// Output tile edge of the block kernel for radius kr.
int block_tile_size(int kr)
{
    return kr <= 5 ? BlockShape<5>::TS : BlockShape<10>::TS;
}

}  // namespace ofv

namespace ofv {

// Reverse-mode stage kernel (window sums again, solve adjoint) for this storage.
cudaError_t launch_bw_stage_S_f32(const BwStageParams &q, cudaStream_t s)
{
    switch (q.a.kr) {
#define OFV_BW_CASE(K) \
    case K: return run_bw_stage_S<float, K>(q, s);
    OFV_BW_CASE(1) OFV_BW_CASE(2) OFV_BW_CASE(3) OFV_BW_CASE(4) OFV_BW_CASE(5)
    OFV_BW_CASE(6) OFV_BW_CASE(7) OFV_BW_CASE(8) OFV_BW_CASE(9) OFV_BW_CASE(10)
#undef OFV_BW_CASE
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ofv
