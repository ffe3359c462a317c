// rk_internal.cuh -- declarations shared by the kernel translation units and the
// host library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>

#include "rk_passes.cuh"
#include "rk_precond.cuh"
#include "rk_zcorr.cuh"

namespace rk {

// Number of kernels launched by the library in this process.
extern std::atomic<long long> g_launches;
inline void count_launch(int k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// Node pairs per block of the fused z pass (tile width 2L values, 64 bytes).
template <typename T>
constexpr int z_pairs() {
  return sizeof(T) == 4 ? 8 : 4;
}

// Line lengths with instantiated FFT kernels.
bool supported_length(int n);

// axis: 0 = x (contiguous lines), 1 = y, 2 = z (strided lines)
template <typename T>
// pw (z SPLIT of Alg. 2 only): apply the pointwise stage to each tile written
cudaError_t launch_split(int axis, int n, const PassArgs<T>& a, cudaStream_t s, const TileMaps* maps = nullptr,
                         const PointwiseArgs<T>* pw = nullptr);
template <typename T>
cudaError_t launch_merge(int axis, int n, const PassArgs<T>& a, cudaStream_t s, const TileMaps* maps = nullptr);
template <typename T>
cudaError_t launch_z(int mode, int n, const ZArgs<T>& a, cudaStream_t s);

// ------------------------------------------------------------- set-up kernel
constexpr int kMaxS = 10;
struct MomentArgs {
  const double* mom;            // moment fields [n_mom][nbox]
  int n_mom;
  int s;
  int dim;                      // 3, or 2 (no z axis: b^z = 0)
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
// set-up of the masks: chi and chi_gamma to 0/1 in place, chi_omega, the count of
// chi nodes (scratch bytes 0..7) and the Eq. 66 gap check (bytes 8..11: 1 when the
// gap along one of the dim axes is narrower than reach); scratch holds
// 16 + n0 + n1 + n2 bytes and is cleared by the call
cudaError_t launch_setup_masks(uint8_t* chi, uint8_t* gam, uint8_t* omg, const int n[3], int dim, int reach,
                               uint8_t* scratch, cudaStream_t s);

// ------------------------------------------------- coefficient compression
// out = 1 where every node within +-r along `axis` (periodic) has in = 1.
cudaError_t launch_erode(uint8_t* out, const uint8_t* in, int axis, int r, const int n[3], cudaStream_t s);
// cls = 0 (chi = 0), 1 (regular: eroded and V == vreg), 2 (irregular)
cudaError_t launch_classify(uint8_t* cls, const uint8_t* chi, const uint8_t* eroded, const double* V, double vreg,
                            long long n, cudaStream_t s);
// 4-node groups g (nodes 4g .. 4g + 3): gcls = 0 all regular, 1 all outside chi,
// 2 other; bit g of regbits / outbits (one word per 32 groups) marks 0 / 1
cudaError_t launch_group_class(uint8_t* gcls, uint32_t* regbits, uint32_t* outbits, const int* cidx, long long ngroups,
                               cudaStream_t s);
// ordered indices of the entries with cls == 2 (offsets from launch_count_irregular
// and launch_scan_counts over the same array)
cudaError_t launch_list_compact(const uint8_t* cls, const int* offsets, long long n, int* list, cudaStream_t s);
constexpr int kScanBlock = 1024;  // nodes per compaction block
// per-block counts of class 2 -> counts[nblk]
cudaError_t launch_count_irregular(const uint8_t* cls, long long n, int* counts, cudaStream_t s);
// exclusive scan of counts (single block, in place); total -> *total
cudaError_t launch_scan_counts(int* counts, int nblk, int* total, cudaStream_t s);
// cidx = -1 / 0 / 1 + compact index; table rows [ncoef][n_irr] filled from b (families 1..3) and chiV
template <typename T>
cudaError_t launch_compact(const uint8_t* cls, const int* offsets, long long n, int* cidx, const T* b, int s,
                           const T* chiV, T* tab, long long n_irr, cudaStream_t st);
// out[j] = src[j * stride + idx] for j < count
cudaError_t launch_gather(double* out, const double* src, long long stride, long long idx, int count, cudaStream_t s);

// --------------------------------------------- pointwise stage of Alg. 2
// In place over the s fields D_p (z-pass outputs of the forward chain):
//   A^k = sum_q b^k_q D_q (Eq. 90),  g_p = chi V sum_k b^k_p A^k (Eq. 91),
// with the coefficients of a node from breg (cidx = 0), from row cidx - 1 of ctab
// (cidx > 0), or g = 0 off chi (cidx = -1).
template <typename T>
cudaError_t launch_pointwise_stiff(const PointwiseArgs<T>& a, cudaStream_t s);
// Alg. 3 without a z axis (2D): u = mask o sum_p b^0_p o D_p over the s fields D[p]
template <typename T>
cudaError_t launch_eval_u_fields(T* u, T* const* D, const T* b0, int s, const uint8_t* mask, long long n,
                                 cudaStream_t st);
// Alg. 4 without a z axis (2D): D[p] = w o b^0_p o y with w = wfield (or 1) times
// wmask (or 1)
template <typename T>
cudaError_t launch_transpose_u_fields(T* const* D, const T* y, const T* b0, int s, const T* wfield,
                                      const uint8_t* wmask, long long n, cudaStream_t st);
// the pointwise stage on the listed 4-node groups only (after a z SPLIT with diag)
template <typename T>
cudaError_t launch_pointwise_groups(const PointwiseArgs<T>& a, const int* list, long long count, cudaStream_t s);

// ------------------------------------- z axis: regular part + local corrections
// G_g += reflected z-convolutions of delta over the correction windows (rk_zcorr.cuh)
template <typename T>
cudaError_t launch_zcorr(const ZCorrArgs<T>& a, cudaStream_t s);
// need = dil && cidx != 0;  out = !in
cudaError_t launch_zwin_need(uint8_t* need, const uint8_t* dil, const int* cidx, long long n, cudaStream_t s);
cudaError_t launch_u8_not(uint8_t* out, const uint8_t* in, long long n, cudaStream_t s);
// per z-line need nodes and the positions within r of one (8 words per line each),
// and flags (1: chi node, 2: need node)
cudaError_t launch_zwin_mark(const uint8_t* need, const uint8_t* chi, const int n[3], int r, uint32_t* mk,
                             uint32_t* nk, uint8_t* flags, cudaStream_t s);
// records per group of kZGW lines: fill = 0 counts them into counts[group]; fill = 1
// writes them from the exclusive offsets in counts
cudaError_t launch_zwin_groups(int fill, const uint32_t* mk, const uint8_t* flags, const int n[3], int chunk,
                               int* counts, ZWin* out, cudaStream_t s);

// ------------------------------------------------------------ CG kernels

constexpr int kRedBlocks = 608;  // 4 x 152 SMs; fixed so reductions are deterministic
constexpr int kRedThreads = 256;

template <typename Ta, typename Tb>
cudaError_t launch_dot(const Ta* a, const Tb* b, long long n, double* partials, double* out, cudaStream_t s);
// rr = sum(partials), alpha = beta = 0, flag cleared; pcg selects who forms r.z
// (without preconditioner rz = rr)
cudaError_t launch_cg_init(const double* partials, CGState* st, int pcg, cudaStream_t s);
// rr = sum(partials) after a residual replacement, leaving beta and the search
// direction as they are (rz too without preconditioner)
cudaError_t launch_cg_set_rr(const double* partials, CGState* st, cudaStream_t s);
// x += alpha p, r -= alpha Ap; the last block sets rr_new and rr, and without
// preconditioner also beta = rr_new / rr and rz = rr_new
template <typename T>
cudaError_t launch_cg_xr_fused(T* x, T* r, const T* p, const T* Ap, CGState* st, long long n, double* partials,
                               unsigned* counter, cudaStream_t s);

// spectral preconditioner passes (rk_precond.cuh): x R2C / C2R and the complex
// y / z passes, dispatched by line length
template <typename T>
cudaError_t launch_px(int c2r, int n, const PxArgs<T>& a, cudaStream_t s);
template <typename T>
cudaError_t launch_pfft(int mode, int n, const PfftArgs<T>& a, cudaStream_t s);
// the multiplier table of the z SYM pass, computed in FP64
template <typename T>
cudaError_t launch_symbol_table(const SymbolArgs<double>& y, T* tab, int nxp, int ny, int nz, cudaStream_t s);

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
// nonlinear reaction terms (kind 0: c u^3, 1: c sinh u, 2: c exp u)
cudaError_t launch_nl_apply(double* Nu, const double* u, const uint8_t* chi, int kind, double c, long long n,
                            cudaStream_t s);
// g_p = chi V (sum_k a_k b^k_p) N_u for p < s (b = [4][s][n]; the gradient-type force, Eq. B.10)
cudaError_t launch_grad_g(double* const* g, const double* b, const double* chiV, const double* Nu, const double a[3],
                          int s, long long n, cudaStream_t st);
// out2 = {sum_chi V w N(u + alpha w), sum_chi V w^2 N'(u + alpha w)}; partials2 holds 2 x kRedBlocks
cudaError_t launch_nl_line(const double* u, const double* w, const double* V, const uint8_t* chi, int kind, double c,
                           double alpha, long long n, double* partials2, double* out2, cudaStream_t s);
// y = a x + b y
cudaError_t launch_axpby(double* y, double a, const double* x, double b, long long n, cudaStream_t s);
// d += dt (f - Kd) / ml where mask (forward Euler with lumped mass)
cudaError_t launch_explicit_step(double* d, const double* f, const double* Kd, const double* ml, const uint8_t* mask,
                                 double dt, long long n, cudaStream_t s);
template <typename T>
cudaError_t launch_fill(T* p, T v, long long n, cudaStream_t s);
template <typename T>
cudaError_t launch_copy(T* dst, const T* src, long long n, cudaStream_t s);

}  // namespace rk
