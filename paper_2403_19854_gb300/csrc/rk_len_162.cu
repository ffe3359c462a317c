// Pass kernels for lines of 162 nodes, both precisions.
#include "rk_launch.cuh"

namespace rk {
RK_INSTANTIATE_LENGTH(162)
}  // namespace rk
