// Block-tiled iteration kernels for __nv_bfloat16 level storage, window radii 1..10:
// the estimator as read from Sec. 2 (no variant code), the persistent batched
// form and the reverse-mode stage kernel.
#include "k_block_inst.cuh"
#include "k_bw_block.cuh"

namespace ofv {

OFV_INSTANTIATE_BLOCK_LAUNCHERS(__nv_bfloat16, false)

// Reverse-mode stage kernel (window sums again, solve adjoint) for this storage.
cudaError_t launch_bw_stage_S_bf16(const BwStageParams &q, cudaStream_t s)
{
    switch (q.a.kr) {
#define OFV_BW_CASE(K) \
    case K: return run_bw_stage_S<__nv_bfloat16, K>(q, s);
    OFV_BW_CASE(1) OFV_BW_CASE(2) OFV_BW_CASE(3) OFV_BW_CASE(4) OFV_BW_CASE(5)
    OFV_BW_CASE(6) OFV_BW_CASE(7) OFV_BW_CASE(8) OFV_BW_CASE(9) OFV_BW_CASE(10)
#undef OFV_BW_CASE
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ofv
