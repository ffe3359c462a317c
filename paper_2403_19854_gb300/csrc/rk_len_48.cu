// Pass kernels for lines of 48 nodes, both precisions.
#include "rk_launch.cuh"

namespace rk {
RK_INSTANTIATE_LENGTH(48)
}  // namespace rk
