// Block-tiled iteration kernels for float level storage, window radii 1..10,
// with the estimator variants (increment form, Gaussian window).
#include "k_block_inst.cuh"

namespace ofv {

OFV_INSTANTIATE_BLOCK_LAUNCHERS(float, true)

}  // namespace ofv
