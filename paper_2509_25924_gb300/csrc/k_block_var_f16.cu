// Block-tiled iteration kernels for __half level storage, window radii 1..10,
// with the estimator variants (increment form, Gaussian window).
#include "k_block_inst.cuh"

namespace ofv {

OFV_INSTANTIATE_BLOCK_LAUNCHERS(__half, true)

}  // namespace ofv
