// Block-tiled iteration kernels for __half level storage, window radii 1..10:
// the estimator as read from Sec. 2 (no variant code) and the persistent
// batched form.
#include "k_block_inst.cuh"

namespace ofv {

OFV_INSTANTIATE_BLOCK_LAUNCHERS(__half, false)

}  // namespace ofv
