// rk_internal.cuh -- declarations shared by the kernel translation units and the
// host library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>

#include "rk_passes.cuh"

namespace rk {

// Number of kernels launched by the library in this process.
extern std::atomic<long long> g_launches;
inline void count_launch(int k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// Line lengths with instantiated FFT kernels.
bool supported_length(int n);

// axis: 0 = x (contiguous lines), 1 = y, 2 = z (strided lines)
template <typename T>
cudaError_t launch_split(int axis, int n, const PassArgs<T>& a, cudaStream_t s);
template <typename T>
cudaError_t launch_merge(int axis, int n, const PassArgs<T>& a, cudaStream_t s);
template <typename T>
cudaError_t launch_z(int mode, int n, const ZArgs<T>& a, cudaStream_t s);

// ------------------------------------------------------------- set-up kernel
constexpr int kMaxS = 10;
struct MomentArgs {
  const double* mom;            // moment fields [n_mom][nbox]
  int n_mom;
  int s;
  signed char pq[kMaxS][kMaxS]; // moment field of M_pq
  const uint8_t* chi;
  double inv_a[3];              // 1 / a_k
  const double* V;
  double* b64;                  // [4][s][nbox]
  float* b32;                   // [4][s][nbox]
  double* chiV64;
  float* chiV32;
  long long nbox;
  unsigned long long* n_singular;
  unsigned long long* first_singular;
};
cudaError_t launch_moment_solve(const MomentArgs& a, cudaStream_t s);

// ------------------------------------------------------------ CG kernels
struct CGState {
  double rr;      // r.r of the current iterate
  double pAp;
  double alpha;
  double beta;
  double rr_new;
  int flag;       // 1: breakdown (p^T A p <= 0 or not finite)
  int pad;
};

constexpr int kRedBlocks = 608;  // 4 x 152 SMs; fixed so reductions are deterministic
constexpr int kRedThreads = 256;

template <typename Ta, typename Tb>
cudaError_t launch_dot(const Ta* a, const Tb* b, long long n, double* partials, double* out, cudaStream_t s);
cudaError_t launch_cg_alpha(const double* partials, CGState* st, cudaStream_t s);
template <typename T>
cudaError_t launch_cg_xr(T* x, T* r, const T* p, const T* Ap, CGState* st, long long n, double* partials,
                         cudaStream_t s);
cudaError_t launch_cg_beta(const double* partials, CGState* st, cudaStream_t s);
template <typename T>
cudaError_t launch_cg_p(T* p, const T* r, const CGState* st, long long n, cudaStream_t s);
cudaError_t launch_cg_init(const double* partials, CGState* st, cudaStream_t s);

// elementwise helpers (double unless noted)
cudaError_t launch_dirichlet_d0(double* d0, const double* g, const uint8_t* chi_gamma, long long n, cudaStream_t s);
// F = mask o (a - b)
cudaError_t launch_masked_diff(double* F, const double* a, const double* b, const uint8_t* mask, long long n,
                               cudaStream_t s);
// y = x (double) ; y32 = (float)(x * scale)
cudaError_t launch_to_f32(float* y, const double* x, double scale, long long n, cudaStream_t s);
// x64 += scale * (double)x32
cudaError_t launch_acc_f32(double* x, const float* c, double scale, long long n, cudaStream_t s);
// d = d0 + x
cudaError_t launch_add(double* d, const double* a, const double* b, long long n, cudaStream_t s);
// out = mask o a
cudaError_t launch_mask(double* out, const double* a, const uint8_t* mask, long long n, cudaStream_t s);
// out = a - b
cudaError_t launch_sub(double* out, const double* a, const double* b, long long n, cudaStream_t s);
// a *= b (elementwise)
cudaError_t launch_mul(double* a, const double* b, long long n, cudaStream_t s);
// u8 -> double
cudaError_t launch_u8_to_f64(double* out, const uint8_t* m, long long n, cudaStream_t s);
template <typename T>
cudaError_t launch_fill(T* p, T v, long long n, cudaStream_t s);
template <typename T>
cudaError_t launch_copy(T* dst, const T* src, long long n, cudaStream_t s);

}  // namespace rk
