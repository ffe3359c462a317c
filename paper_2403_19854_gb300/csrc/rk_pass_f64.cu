// Axis-pass kernels (SPLIT / MERGE along x, y, z) instantiated for double.
#include "rk_launch.cuh"

namespace rk {
template cudaError_t launch_split<double>(int, int, const PassArgs<double>&, cudaStream_t);
template cudaError_t launch_merge<double>(int, int, const PassArgs<double>&, cudaStream_t);
}  // namespace rk
