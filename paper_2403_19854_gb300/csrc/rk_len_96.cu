// Pass kernels for lines of 96 nodes, both precisions.
#include "rk_launch.cuh"

namespace rk {
RK_INSTANTIATE_LENGTH(96)
}  // namespace rk
