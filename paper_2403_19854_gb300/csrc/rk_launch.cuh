// rk_launch.cuh -- launch configuration of the pass kernels; included by the
// per-precision translation units, which instantiate it for float and double.
#pragma once

#include <algorithm>

#include "rk_internal.cuh"
#include "rk_zpass_tma.cuh"

namespace rk {

// Node pairs per block (strided passes), x-pass threads per block, node pairs per
// block of the fused z pass.  Rows of 2L values: 128 bytes per line position.
template <typename T>
struct Cfg;
template <>
struct Cfg<float> {
  static constexpr int L = 16;
  static constexpr int XTHREADS = 128;
  static constexpr int LZ = z_pairs<float>();
};
template <>
struct Cfg<double> {
  static constexpr int L = 8;
  static constexpr int XTHREADS = 128;
  static constexpr int LZ = z_pairs<double>();
};

template <typename K>
inline cudaError_t set_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, int N>
cudaError_t split_n(int axis, const PassArgs<T>& a, cudaStream_t s) {
  if (axis == 0) {
    constexpr int LX = Cfg<T>::XTHREADS / LineShape<N>::P;
    using X = XPass<T, N, LX>;
    const long long npairs = ((long long)a.ny * a.nz) / 2;
    const unsigned nb = (unsigned)((npairs + LX - 1) / LX);
    auto k = k_x_split<T, N, LX>;
    cudaError_t e = set_smem(k, X::SMEM);
    if (e != cudaSuccess) return e;
    count_launch();
    k<<<nb, X::THREADS, X::SMEM, s>>>(a);
  } else {
    constexpr int L = Cfg<T>::L;
    using S = Strided<T, N, L>;
    dim3 grid((unsigned)((a.nx / 2 + L - 1) / L), (unsigned)(axis == 1 ? a.nz : a.ny));
    auto k = k_strided_split<T, N, L>;
    cudaError_t e = set_smem(k, S::SMEM);
    if (e != cudaSuccess) return e;
    count_launch();
    k<<<grid, S::THREADS, S::SMEM, s>>>(a);
  }
  return cudaGetLastError();
}

template <typename T, int N>
cudaError_t merge_n(int axis, const PassArgs<T>& a, cudaStream_t s) {
  if (axis == 0) {
    constexpr int LX = Cfg<T>::XTHREADS / LineShape<N>::P;
    using X = XPass<T, N, LX>;
    const long long npairs = ((long long)a.ny * a.nz) / 2;
    const unsigned nb = (unsigned)((npairs + LX - 1) / LX);
    auto k = k_x_merge<T, N, LX>;
    cudaError_t e = set_smem(k, X::SMEM);
    if (e != cudaSuccess) return e;
    count_launch();
    k<<<nb, X::THREADS, X::SMEM, s>>>(a);
  } else {
    constexpr int L = Cfg<T>::L;
    using S = Strided<T, N, L>;
    dim3 grid((unsigned)((a.nx / 2 + L - 1) / L), (unsigned)(axis == 1 ? a.nz : a.ny));
    auto k = k_strided_merge<T, N, L>;
    cudaError_t e = set_smem(k, S::SMEM);
    if (e != cudaSuccess) return e;
    count_launch();
    k<<<grid, S::THREADS, S::SMEM, s>>>(a);
  }
  return cudaGetLastError();
}

inline int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
  }
  return n;
}

// persistent TMA-pipelined Z_STIFF: two resident blocks per SM
template <typename T, int N>
cudaError_t z_stiff_tma(const ZArgs<T>& a, cudaStream_t s) {
  constexpr int L = Cfg<T>::LZ;
  using Z = ZTma<T, N, L>;
  const long long npen = (long long)((a.nx / 2 + L - 1) / L) * a.ny;
  const long long nb = std::min<long long>(npen, 2LL * sm_count());
  auto k = k_z_stiff_tma<T, N, L>;
  cudaError_t e = set_smem(k, Z::SMEM);
  if (e != cudaSuccess) return e;
  count_launch();
  k<<<(unsigned)nb, Z::THREADS, Z::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int N, int MODE>
cudaError_t z_n_mode(const ZArgs<T>& a, cudaStream_t s) {
  if (MODE == Z_STIFF && a.use_tma && a.cidx) return z_stiff_tma<T, N>(a, s);
  constexpr int L = Cfg<T>::LZ;
  using Z = ZPass<T, N, L, MODE>;
  dim3 grid((unsigned)((a.nx / 2 + L - 1) / L), (unsigned)a.ny);
  auto k = k_z_fused<T, N, L, MODE>;
  cudaError_t e = set_smem(k, Z::SMEM);
  if (e != cudaSuccess) return e;
  count_launch();
  k<<<grid, Z::THREADS, Z::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int N>
cudaError_t z_n(int mode, const ZArgs<T>& a, cudaStream_t s) {
  switch (mode) {
    case Z_STIFF: return z_n_mode<T, N, Z_STIFF>(a, s);
    case Z_EVAL_U: return z_n_mode<T, N, Z_EVAL_U>(a, s);
    case Z_TRANSPOSE_U: return z_n_mode<T, N, Z_TRANSPOSE_U>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

#define RK_FOR_EACH_LENGTH(X) X(8) X(16) X(32) X(64) X(96) X(128) X(256)

template <typename T>
cudaError_t launch_split(int axis, int n, const PassArgs<T>& a, cudaStream_t s) {
  switch (n) {
#define RK_CASE(N) \
  case N: return split_n<T, N>(axis, a, s);
    RK_FOR_EACH_LENGTH(RK_CASE)
#undef RK_CASE
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_merge(int axis, int n, const PassArgs<T>& a, cudaStream_t s) {
  switch (n) {
#define RK_CASE(N) \
  case N: return merge_n<T, N>(axis, a, s);
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

}  // namespace rk
