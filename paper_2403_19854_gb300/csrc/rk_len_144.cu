// Pass kernels for lines of 144 nodes, both precisions.
#include "rk_launch.cuh"

namespace rk {
RK_INSTANTIATE_LENGTH(144)
}  // namespace rk
