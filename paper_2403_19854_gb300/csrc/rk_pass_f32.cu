// Axis-pass kernels (SPLIT / MERGE along x, y, z) instantiated for float.
#include "rk_launch.cuh"

namespace rk {
template cudaError_t launch_split<float>(int, int, const PassArgs<float>&, cudaStream_t);
template cudaError_t launch_merge<float>(int, int, const PassArgs<float>&, cudaStream_t);
}  // namespace rk
