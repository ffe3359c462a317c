// rk_vec.cu -- per-node moment solve of Alg. 1 and the vector kernels of the
// conjugate-gradient driver (Alg. 5).
#include "rk_internal.cuh"
#include "rk_moment.cuh"

namespace rk {

std::atomic<long long> g_launches{0};

bool supported_length(int n) {
  switch (n) {
    case 8: case 16: case 32: case 64: case 96: case 128: case 256: return true;
    default: return false;
  }
}

cudaError_t launch_moment_solve(const MomentArgs& a, cudaStream_t s) {
  const long long nb = (a.nbox + 127) / 128;
  const unsigned grid = (unsigned)(nb < 152 * 64 ? nb : 152 * 64);
  count_launch();
  k_moment_solve<<<grid, 128, 0, s>>>(a);
  return cudaGetLastError();
}

// ----------------------------------------------------------- reductions
// Fixed grid and fixed combination order: results are bit-reproducible.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[kRedThreads / 32];
  v = warp_sum(v);
  const int w = threadIdx.x / 32, ln = threadIdx.x % 32;
  if (ln == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = (ln < kRedThreads / 32) ? sh[ln] : 0.0;
    r = warp_sum(r);
  }
  __syncthreads();
  return r;  // valid in thread 0
}

template <typename Ta, typename Tb>
__global__ void __launch_bounds__(kRedThreads) k_dot(const Ta* __restrict__ a, const Tb* __restrict__ b, long long n,
                                                    double* __restrict__ part) {
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * kRedThreads + threadIdx.x; i < n; i += (long long)kRedBlocks * kRedThreads)
    acc += (double)a[i] * (double)b[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__device__ __forceinline__ double reduce_partials(const double* part) {
  double v = 0.0;
  for (int i = threadIdx.x; i < kRedBlocks; i += kRedThreads) v += part[i];
  return block_sum(v);
}

__global__ void __launch_bounds__(kRedThreads) k_reduce_to(const double* part, double* out) {
  const double v = reduce_partials(part);
  if (threadIdx.x == 0) *out = v;
}

template <typename Ta, typename Tb>
cudaError_t launch_dot(const Ta* a, const Tb* b, long long n, double* partials, double* out, cudaStream_t s) {
  count_launch();
  k_dot<Ta, Tb><<<kRedBlocks, kRedThreads, 0, s>>>(a, b, n, partials);
  count_launch();
  k_reduce_to<<<1, kRedThreads, 0, s>>>(partials, out);
  return cudaGetLastError();
}
template cudaError_t launch_dot<double, double>(const double*, const double*, long long, double*, double*, cudaStream_t);
template cudaError_t launch_dot<float, float>(const float*, const float*, long long, double*, double*, cudaStream_t);

// rr = sum(partials); alpha = beta = 0
__global__ void k_cg_init(const double* part, CGState* st) {
  const double v = reduce_partials(part);
  if (threadIdx.x == 0) {
    st->rr = v;
    st->alpha = 0.0;
    st->beta = 0.0;
    st->flag = 0;
  }
}
cudaError_t launch_cg_init(const double* partials, CGState* st, cudaStream_t s) {
  count_launch();
  k_cg_init<<<1, kRedThreads, 0, s>>>(partials, st);
  return cudaGetLastError();
}

// pAp = sum(partials); alpha = rr / pAp  (0 and flag on breakdown or rr == 0)
__global__ void k_cg_alpha(const double* part, CGState* st) {
  const double v = reduce_partials(part);
  if (threadIdx.x == 0) {
    st->pAp = v;
    double al = 0.0;
    if (st->rr > 0.0) {
      if (v > 0.0 && isfinite(v))
        al = st->rr / v;
      else
        st->flag = 1;
    }
    st->alpha = al;
  }
}
cudaError_t launch_cg_alpha(const double* partials, CGState* st, cudaStream_t s) {
  count_launch();
  k_cg_alpha<<<1, kRedThreads, 0, s>>>(partials, st);
  return cudaGetLastError();
}

// x += alpha p, r -= alpha Ap, partial r.r
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_cg_xr(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
                                                      const T* __restrict__ Ap, const CGState* st, long long n,
                                                      double* __restrict__ part) {
  const T al = (T)st->alpha;
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * kRedThreads + threadIdx.x; i < n; i += (long long)kRedBlocks * kRedThreads) {
    x[i] += al * p[i];
    const T ri = r[i] - al * Ap[i];
    r[i] = ri;
    acc += (double)ri * (double)ri;
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}
template <typename T>
cudaError_t launch_cg_xr(T* x, T* r, const T* p, const T* Ap, CGState* st, long long n, double* partials,
                         cudaStream_t s) {
  count_launch();
  k_cg_xr<T><<<kRedBlocks, kRedThreads, 0, s>>>(x, r, p, Ap, st, n, partials);
  return cudaGetLastError();
}
template cudaError_t launch_cg_xr<double>(double*, double*, const double*, const double*, CGState*, long long,
                                          double*, cudaStream_t);
template cudaError_t launch_cg_xr<float>(float*, float*, const float*, const float*, CGState*, long long, double*,
                                         cudaStream_t);

// rr_new = sum(partials); beta = rr_new / rr; rr = rr_new
__global__ void k_cg_beta(const double* part, CGState* st) {
  const double v = reduce_partials(part);
  if (threadIdx.x == 0) {
    st->rr_new = v;
    st->beta = (st->rr > 0.0) ? v / st->rr : 0.0;
    st->rr = v;
  }
}
cudaError_t launch_cg_beta(const double* partials, CGState* st, cudaStream_t s) {
  count_launch();
  k_cg_beta<<<1, kRedThreads, 0, s>>>(partials, st);
  return cudaGetLastError();
}

template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_cg_p(T* __restrict__ p, const T* __restrict__ r, const CGState* st,
                                                     long long n) {
  const T be = (T)st->beta;
  for (long long i = (long long)blockIdx.x * kRedThreads + threadIdx.x; i < n; i += (long long)kRedBlocks * kRedThreads)
    p[i] = r[i] + be * p[i];
}
template <typename T>
cudaError_t launch_cg_p(T* p, const T* r, const CGState* st, long long n, cudaStream_t s) {
  count_launch();
  k_cg_p<T><<<kRedBlocks, kRedThreads, 0, s>>>(p, r, st, n);
  return cudaGetLastError();
}
template cudaError_t launch_cg_p<double>(double*, const double*, const CGState*, long long, cudaStream_t);
template cudaError_t launch_cg_p<float>(float*, const float*, const CGState*, long long, cudaStream_t);

// ------------------------------------------------------------ elementwise
#define RK_GRID_LOOP(i, n)                                                             \
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (n); \
       i += (long long)gridDim.x * blockDim.x)

static inline unsigned ew_grid(long long n) {
  const long long b = (n + 255) / 256;
  return (unsigned)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

__global__ void k_dirichlet_d0(double* d0, const double* g, const uint8_t* cg, long long n) {
  RK_GRID_LOOP(i, n) d0[i] = cg[i] ? g[i] : 0.0;
}
cudaError_t launch_dirichlet_d0(double* d0, const double* g, const uint8_t* chi_gamma, long long n, cudaStream_t s) {
  count_launch();
  k_dirichlet_d0<<<ew_grid(n), 256, 0, s>>>(d0, g, chi_gamma, n);
  return cudaGetLastError();
}

__global__ void k_masked_diff(double* F, const double* a, const double* b, const uint8_t* m, long long n) {
  RK_GRID_LOOP(i, n) F[i] = m[i] ? a[i] - b[i] : 0.0;
}
cudaError_t launch_masked_diff(double* F, const double* a, const double* b, const uint8_t* mask, long long n,
                               cudaStream_t s) {
  count_launch();
  k_masked_diff<<<ew_grid(n), 256, 0, s>>>(F, a, b, mask, n);
  return cudaGetLastError();
}

__global__ void k_to_f32(float* y, const double* x, double sc, long long n) {
  RK_GRID_LOOP(i, n) y[i] = (float)(x[i] * sc);
}
cudaError_t launch_to_f32(float* y, const double* x, double scale, long long n, cudaStream_t s) {
  count_launch();
  k_to_f32<<<ew_grid(n), 256, 0, s>>>(y, x, scale, n);
  return cudaGetLastError();
}

__global__ void k_acc_f32(double* x, const float* c, double sc, long long n) {
  RK_GRID_LOOP(i, n) x[i] += sc * (double)c[i];
}
cudaError_t launch_acc_f32(double* x, const float* c, double scale, long long n, cudaStream_t s) {
  count_launch();
  k_acc_f32<<<ew_grid(n), 256, 0, s>>>(x, c, scale, n);
  return cudaGetLastError();
}

__global__ void k_add(double* d, const double* a, const double* b, long long n) {
  RK_GRID_LOOP(i, n) d[i] = a[i] + b[i];
}
cudaError_t launch_add(double* d, const double* a, const double* b, long long n, cudaStream_t s) {
  count_launch();
  k_add<<<ew_grid(n), 256, 0, s>>>(d, a, b, n);
  return cudaGetLastError();
}

__global__ void k_sub(double* d, const double* a, const double* b, long long n) {
  RK_GRID_LOOP(i, n) d[i] = a[i] - b[i];
}
cudaError_t launch_sub(double* out, const double* a, const double* b, long long n, cudaStream_t s) {
  count_launch();
  k_sub<<<ew_grid(n), 256, 0, s>>>(out, a, b, n);
  return cudaGetLastError();
}

__global__ void k_mask(double* o, const double* a, const uint8_t* m, long long n) {
  RK_GRID_LOOP(i, n) o[i] = m[i] ? a[i] : 0.0;
}
cudaError_t launch_mask(double* out, const double* a, const uint8_t* mask, long long n, cudaStream_t s) {
  count_launch();
  k_mask<<<ew_grid(n), 256, 0, s>>>(out, a, mask, n);
  return cudaGetLastError();
}

__global__ void k_mul(double* a, const double* b, long long n) {
  RK_GRID_LOOP(i, n) a[i] *= b[i];
}
cudaError_t launch_mul(double* a, const double* b, long long n, cudaStream_t s) {
  count_launch();
  k_mul<<<ew_grid(n), 256, 0, s>>>(a, b, n);
  return cudaGetLastError();
}

__global__ void k_u8_to_f64(double* o, const uint8_t* m, long long n) {
  RK_GRID_LOOP(i, n) o[i] = m[i] ? 1.0 : 0.0;
}
cudaError_t launch_u8_to_f64(double* out, const uint8_t* m, long long n, cudaStream_t s) {
  count_launch();
  k_u8_to_f64<<<ew_grid(n), 256, 0, s>>>(out, m, n);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_fill(T* p, T v, long long n) {
  RK_GRID_LOOP(i, n) p[i] = v;
}
template <typename T>
cudaError_t launch_fill(T* p, T v, long long n, cudaStream_t s) {
  count_launch();
  k_fill<T><<<ew_grid(n), 256, 0, s>>>(p, v, n);
  return cudaGetLastError();
}
template cudaError_t launch_fill<double>(double*, double, long long, cudaStream_t);
template cudaError_t launch_fill<float>(float*, float, long long, cudaStream_t);

template <typename T>
__global__ void k_copy(T* d, const T* s, long long n) {
  RK_GRID_LOOP(i, n) d[i] = s[i];
}
template <typename T>
cudaError_t launch_copy(T* dst, const T* src, long long n, cudaStream_t s) {
  count_launch();
  k_copy<T><<<ew_grid(n), 256, 0, s>>>(dst, src, n);
  return cudaGetLastError();
}
template cudaError_t launch_copy<double>(double*, const double*, long long, cudaStream_t);
template cudaError_t launch_copy<float>(float*, const float*, long long, cudaStream_t);

}  // namespace rk
