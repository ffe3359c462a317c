// rk_launch.cuh -- launch configuration of the pass kernels; included by the
// per-precision translation units, which instantiate it for float and double.
#pragma once

#include <algorithm>

#include "rk_internal.cuh"

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
  // static plus dynamic shared memory above 48 KB needs the opt-in; the kernels
  // here use less than 16 KB of static shared memory
  if (bytes <= 32 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Persistent strided pass: as many blocks as fit on the device at once (the
// occupancy of the kernel is queried on first use), each looping over tiles of
// 2L x values times one index of the other axis.  a16: every row of every input
// starts on a 16-byte boundary (16-byte async copies), else per-element copies.
template <typename T, int N, bool MERGE, int PW = 0>
cudaError_t launch_strided(int axis, const PassArgs<T>& a, cudaStream_t s, const TileMaps* maps,
                           const PointwiseArgs<T>* pw = nullptr) {
  constexpr int L = Cfg<T>::L;
  using S = Strided<T, N, L>;
  static int resident = 0;  // blocks per SM of this kernel (first device used)
  static int sms = 0;
  auto occupancy = [&](auto kernel) -> cudaError_t {
    cudaError_t e = set_smem(kernel, S::SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0, nb = 0, nsm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, S::THREADS, S::SMEM)) != cudaSuccess) return e;
    sms = nsm;
    resident = nb > 0 ? nb : 1;
    return cudaSuccess;
  };
  if (!resident) {
    cudaError_t e;
    if constexpr (MERGE)
      e = occupancy(k_strided_merge<T, N, L>);
    else
      e = occupancy(k_strided_split<T, N, L, PW>);
    if (e != cudaSuccess) return e;
  }
  const int nbx = (a.nx + S::ROW - 1) / S::ROW;
  const long long ntiles = (long long)nbx * (axis == 1 ? a.nz : a.ny);
  bool a16 = (a.line_stride * (long long)sizeof(T)) % 16 == 0 && (a.other_stride * (long long)sizeof(T)) % 16 == 0;
  for (int i = 0; i < kMaxIn; ++i)
    if (a.in[i] && (reinterpret_cast<uintptr_t>(a.in[i]) % 16) != 0) a16 = false;
  const long long cap = (long long)resident * sms;
  const unsigned grid = (unsigned)(ntiles < cap ? ntiles : cap);
  static const TileMaps none = {};
  static const PointwiseArgs<T> no_pw = {};
  count_launch();
  if constexpr (MERGE)
    k_strided_merge<T, N, L><<<grid, S::THREADS, S::SMEM, s>>>(a, nbx, ntiles, a16 ? 1 : 0, maps ? *maps : none,
                                                               maps ? axis : 0);
  else
    k_strided_split<T, N, L, PW><<<grid, S::THREADS, S::SMEM, s>>>(a, nbx, ntiles, a16 ? 1 : 0, maps ? *maps : none,
                                                                   maps ? axis : 0, pw ? *pw : no_pw);
  return cudaGetLastError();
}

// x split: rows arrive by bulk async copies when the pass carries the fused CG
// direction update (two fields, r and p, per row: 0.099 -> 0.072 ms at 256^3),
// a row is a whole number of 16-byte units and every field starts on a 16-byte
// boundary.  With one field per row (plain split, and the merge pass) per-thread
// loads measured faster (0.060 vs 0.069 ms), so those keep them.
template <typename T, int N, int LX>
bool x_bulk_setup(PassArgs<T>& b) {
  using X = XPass<T, N, LX>;
  bool ok = X::BULK && b.n_groups == 1 && b.cg_r;
  auto aligned = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) % 16) == 0; };
  for (int i = 0; i < kMaxIn; ++i)
    if (b.in[i] && !aligned(b.in[i])) ok = false;
  if ((b.cg_r && !aligned(b.cg_r)) || (b.cg_p && !aligned(b.cg_p))) ok = false;
  b.xbulk = ok ? 1 : 0;
  return ok;
}

template <typename T, int N>
cudaError_t split_n(int axis, const PassArgs<T>& a, cudaStream_t s, const TileMaps* maps, const PointwiseArgs<T>* pw) {
  if (axis == 0) {
    constexpr int LX = Cfg<T>::XTHREADS / LineShape<N>::P;
    using X = XPass<T, N, LX>;
    const long long npairs = ((long long)a.ny * a.nz + 1) / 2;  // an odd last row pairs with zeros
    const unsigned nb = (unsigned)((npairs + LX - 1) / LX);
    PassArgs<T> b = a;
    if (x_bulk_setup<T, N, LX>(b)) {
      auto k = k_x_split<T, N, LX, true>;
      cudaError_t e = set_smem(k, X::SMEM_FEED);
      if (e != cudaSuccess) return e;
      count_launch();
      k<<<nb, X::THREADS, X::SMEM_FEED, s>>>(b);
    } else {
      auto k = k_x_split<T, N, LX, false>;
      cudaError_t e = set_smem(k, X::SMEM);
      if (e != cudaSuccess) return e;
      count_launch();
      k<<<nb, X::THREADS, X::SMEM, s>>>(b);
    }
  } else {
    if (pw && pw->s == 4) return launch_strided<T, N, false, 4>(axis, a, s, maps, pw);
    if (pw && pw->s == 10) return launch_strided<T, N, false, 10>(axis, a, s, maps, pw);
    return launch_strided<T, N, false>(axis, a, s, maps);
  }
  return cudaGetLastError();
}

template <typename T, int N>
cudaError_t merge_n(int axis, const PassArgs<T>& a, cudaStream_t s, const TileMaps* maps) {
  if (axis == 0) {
    constexpr int LX = Cfg<T>::XTHREADS / LineShape<N>::P;
    using X = XPass<T, N, LX>;
    const long long npairs = ((long long)a.ny * a.nz + 1) / 2;  // an odd last row pairs with zeros
    const unsigned nb = (unsigned)((npairs + LX - 1) / LX);
    auto aligned = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) % 16) == 0; };
    const bool fed = X::MERGE_BULK && a.cg_p && a.out_mask && a.n_groups == 1 && aligned(a.cg_p) && aligned(a.out_mask);
    if constexpr (sizeof(T) == 4 && X::FIVE && X::SMEM >= X::TILE) {
      if (fed && a.g_begin[1] - a.g_begin[0] == 2 && aligned(a.in[a.term_io[a.g_begin[0]]]) &&
          aligned(a.in[a.term_io[a.g_begin[0] + 1]])) {
        auto k = k_x_merge_fed2<T, N, LX>;
        cudaError_t e = set_smem(k, X::SMEM_MERGE_FEED);
        if (e != cudaSuccess) return e;
        count_launch();
        k<<<nb, X::THREADS, X::SMEM_MERGE_FEED, s>>>(a);
        return cudaGetLastError();
      }
    }
    if (fed) {
      auto k = k_x_merge<T, N, LX, true>;
      cudaError_t e = set_smem(k, X::SMEM_MERGE_FEED);
      if (e != cudaSuccess) return e;
      count_launch();
      k<<<nb, X::THREADS, X::SMEM_MERGE_FEED, s>>>(a);
    } else {
      auto k = k_x_merge<T, N, LX, false>;
      cudaError_t e = set_smem(k, X::SMEM);
      if (e != cudaSuccess) return e;
      count_launch();
      k<<<nb, X::THREADS, X::SMEM, s>>>(a);
    }
  } else {
    return launch_strided<T, N, true>(axis, a, s, maps);
  }
  return cudaGetLastError();
}

template <typename T, int N, int MODE>
cudaError_t z_n_mode(const ZArgs<T>& a, cudaStream_t s) {
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

// spectral preconditioner passes (rk_precond.cuh)
template <typename T, int N>
cudaError_t px_n(int c2r, const PxArgs<T>& a, cudaStream_t s) {
  constexpr int LX = Cfg<T>::XTHREADS / LineShape<N>::P;
  using X = XPass<T, N, LX>;
  const long long npairs = ((long long)a.ny * a.nz) / 2;
  const unsigned nb = (unsigned)((npairs + LX - 1) / LX);
  auto k = c2r ? k_px_c2r<T, N, LX> : k_px_r2c<T, N, LX>;
  cudaError_t e = set_smem(k, X::SMEM);
  if (e != cudaSuccess) return e;
  count_launch();
  k<<<nb, X::THREADS, X::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int N, int MODE>
cudaError_t pfft_n_mode(const PfftArgs<T>& a, cudaStream_t s) {
  constexpr int L = Cfg<T>::L;
  using S = Strided<T, N, L>;
  auto kernel = k_pfft<T, N, L, MODE>;
  static int resident = 0;
  static int sms = 0;
  if (!resident) {
    cudaError_t e = set_smem(kernel, S::SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0, nb = 0, nsm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, S::THREADS, S::SMEM)) != cudaSuccess) return e;
    sms = nsm;
    resident = nb > 0 ? nb : 1;
  }
  const int nbx = (a.ncols + L - 1) / L;
  const long long ntiles = (long long)nbx * a.nother;
  const long long cap = (long long)resident * sms;
  count_launch();
  kernel<<<(unsigned)(ntiles < cap ? ntiles : cap), S::THREADS, S::SMEM, s>>>(a, nbx, ntiles);
  return cudaGetLastError();
}

template <typename T, int N>
cudaError_t pfft_n(int mode, const PfftArgs<T>& a, cudaStream_t s) {
  switch (mode) {
    case PF_FWD: return pfft_n_mode<T, N, PF_FWD>(a, s);
    case PF_SYM: return pfft_n_mode<T, N, PF_SYM>(a, s);
    case PF_INV: return pfft_n_mode<T, N, PF_INV>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

// One translation unit per line length instantiates split_n, merge_n and z_n for
// both precisions (rk_len_<N>.cu); rk_dispatch.cu selects them at run time.
#define RK_FOR_EACH_LENGTH(X) X(8) X(16) X(32) X(36) X(48) X(64) X(72) X(96) X(100) X(128) X(144) X(162) X(256)

#define RK_DECLARE_LENGTH(N)                                                                  \
  extern template cudaError_t split_n<float, N>(int, const PassArgs<float>&, cudaStream_t, const TileMaps*,             \
                                               const PointwiseArgs<float>*);   \
  extern template cudaError_t split_n<double, N>(int, const PassArgs<double>&, cudaStream_t, const TileMaps*,           \
                                                const PointwiseArgs<double>*); \
  extern template cudaError_t merge_n<float, N>(int, const PassArgs<float>&, cudaStream_t, const TileMaps*);   \
  extern template cudaError_t merge_n<double, N>(int, const PassArgs<double>&, cudaStream_t, const TileMaps*); \
  extern template cudaError_t z_n<float, N>(int, const ZArgs<float>&, cudaStream_t);          \
  extern template cudaError_t z_n<double, N>(int, const ZArgs<double>&, cudaStream_t);        \
  extern template cudaError_t px_n<float, N>(int, const PxArgs<float>&, cudaStream_t);        \
  extern template cudaError_t px_n<double, N>(int, const PxArgs<double>&, cudaStream_t);      \
  extern template cudaError_t pfft_n<float, N>(int, const PfftArgs<float>&, cudaStream_t);    \
  extern template cudaError_t pfft_n<double, N>(int, const PfftArgs<double>&, cudaStream_t);

#define RK_INSTANTIATE_LENGTH(N)                                                       \
  template cudaError_t split_n<float, N>(int, const PassArgs<float>&, cudaStream_t, const TileMaps*,             \
                                               const PointwiseArgs<float>*);   \
  template cudaError_t split_n<double, N>(int, const PassArgs<double>&, cudaStream_t, const TileMaps*,           \
                                                const PointwiseArgs<double>*); \
  template cudaError_t merge_n<float, N>(int, const PassArgs<float>&, cudaStream_t, const TileMaps*);   \
  template cudaError_t merge_n<double, N>(int, const PassArgs<double>&, cudaStream_t, const TileMaps*); \
  template cudaError_t z_n<float, N>(int, const ZArgs<float>&, cudaStream_t);          \
  template cudaError_t z_n<double, N>(int, const ZArgs<double>&, cudaStream_t);        \
  template cudaError_t px_n<float, N>(int, const PxArgs<float>&, cudaStream_t);        \
  template cudaError_t px_n<double, N>(int, const PxArgs<double>&, cudaStream_t);      \
  template cudaError_t pfft_n<float, N>(int, const PfftArgs<float>&, cudaStream_t);    \
  template cudaError_t pfft_n<double, N>(int, const PfftArgs<double>&, cudaStream_t);

}  // namespace rk
