// Pass kernels for lines of 100 nodes, both precisions.
#include "rk_launch.cuh"

namespace rk {
RK_INSTANTIATE_LENGTH(100)
}  // namespace rk
