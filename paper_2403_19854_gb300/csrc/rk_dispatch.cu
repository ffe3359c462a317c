// Run-time selection of the pass kernels by line length; the kernels themselves
// are instantiated in rk_len_<N>.cu.
#include "rk_launch.cuh"

namespace rk {

RK_FOR_EACH_LENGTH(RK_DECLARE_LENGTH)

template <typename T>
cudaError_t launch_split(int axis, int n, const PassArgs<T>& a, cudaStream_t s, const TileMaps* maps,
                         const PointwiseArgs<T>* pw) {
  switch (n) {
#define RK_CASE(N) \
  case N: return split_n<T, N>(axis, a, s, maps, pw);
    RK_FOR_EACH_LENGTH(RK_CASE)
#undef RK_CASE
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_merge(int axis, int n, const PassArgs<T>& a, cudaStream_t s, const TileMaps* maps) {
  switch (n) {
#define RK_CASE(N) \
  case N: return merge_n<T, N>(axis, a, s, maps);
    RK_FOR_EACH_LENGTH(RK_CASE)
#undef RK_CASE
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_z(int mode, int n, const ZArgs<T>& a, cudaStream_t s) {
  switch (n) {
#define RK_CASE(N) \
  case N: return z_n<T, N>(mode, a, s);
    RK_FOR_EACH_LENGTH(RK_CASE)
#undef RK_CASE
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_px(int c2r, int n, const PxArgs<T>& a, cudaStream_t s) {
  switch (n) {
#define RK_CASE(N) \
  case N: return px_n<T, N>(c2r, a, s);
    RK_FOR_EACH_LENGTH(RK_CASE)
#undef RK_CASE
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_pfft(int mode, int n, const PfftArgs<T>& a, cudaStream_t s) {
  switch (n) {
#define RK_CASE(N) \
  case N: return pfft_n<T, N>(mode, a, s);
    RK_FOR_EACH_LENGTH(RK_CASE)
#undef RK_CASE
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_split<float>(int, int, const PassArgs<float>&, cudaStream_t, const TileMaps*,
                                        const PointwiseArgs<float>*);
template cudaError_t launch_split<double>(int, int, const PassArgs<double>&, cudaStream_t, const TileMaps*,
                                         const PointwiseArgs<double>*);
template cudaError_t launch_merge<float>(int, int, const PassArgs<float>&, cudaStream_t, const TileMaps*);
template cudaError_t launch_merge<double>(int, int, const PassArgs<double>&, cudaStream_t, const TileMaps*);
template cudaError_t launch_z<float>(int, int, const ZArgs<float>&, cudaStream_t);
template cudaError_t launch_z<double>(int, int, const ZArgs<double>&, cudaStream_t);
template cudaError_t launch_px<float>(int, int, const PxArgs<float>&, cudaStream_t);
template cudaError_t launch_px<double>(int, int, const PxArgs<double>&, cudaStream_t);
template cudaError_t launch_pfft<float>(int, int, const PfftArgs<float>&, cudaStream_t);
template cudaError_t launch_pfft<double>(int, int, const PfftArgs<double>&, cudaStream_t);

}  // namespace rk
