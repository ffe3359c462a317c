// Pass kernels for lines of 16 nodes, both precisions.
#include "rk_launch.cuh"

namespace rk {
RK_INSTANTIATE_LENGTH(16)
}  // namespace rk
