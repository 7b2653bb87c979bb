// Host launcher of the block-tiled iteration kernel.
#include "k_block.cuh"

namespace ofv {

cudaError_t launch_block_f32(const BlockParams &p, int kr, int npairs, cudaStream_t s);
cudaError_t launch_block_f16(const BlockParams &p, int kr, int npairs, cudaStream_t s);
cudaError_t launch_block_bf16(const BlockParams &p, int kr, int npairs, cudaStream_t s);

bool block_supports(int kr) { return kr >= 1 && kr <= kBlockMaxKR; }

cudaError_t launch_iter_block(const IterArgs *a, int npairs, int store, int mode, cudaStream_t s)
{
    if (npairs < 1 || npairs > kBlockMaxBatch || !block_supports(a[0].kr)) return cudaErrorInvalidValue;
    BlockParams p;
    for (int k = 0; k < npairs; ++k) p.a[k] = a[k];
    p.mode = mode;
    switch (store) {
    case ST_F16: return launch_block_f16(p, a[0].kr, npairs, s);
    case ST_BF16: return launch_block_bf16(p, a[0].kr, npairs, s);
    default: return launch_block_f32(p, a[0].kr, npairs, s);
    }
}

}  // namespace ofv
