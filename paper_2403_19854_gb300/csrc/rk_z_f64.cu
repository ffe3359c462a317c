// Fused z-pass kernels (Alg. 2 pointwise stage, Alg. 3, Alg. 4) instantiated for double.
#include "rk_launch.cuh"

namespace rk {
template cudaError_t launch_z<double>(int, int, const ZArgs<double>&, cudaStream_t);
}  // namespace rk
