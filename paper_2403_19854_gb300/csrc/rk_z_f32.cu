// Fused z-pass kernels (Alg. 2 pointwise stage, Alg. 3, Alg. 4) instantiated for float.
#include "rk_launch.cuh"

namespace rk {
template cudaError_t launch_z<float>(int, int, const ZArgs<float>&, cudaStream_t);
}  // namespace rk
