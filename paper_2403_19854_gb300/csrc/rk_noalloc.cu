// rk_noalloc.cu -- rk_apply_K_noalloc: the FP64 stiffness action of rk_apply_K
// for callers that must not allocate device memory.
//
// Who needs it: code embedded in a host application that owns every byte of
// device memory through its own pool or arena (and forbids other allocations),
// and latency-critical loops in which a cudaMalloc / cudaFree -- which can
// synchronise the whole device and stall other streams -- is not acceptable.
// The caller passes the inputs and the output; the intermediate fields of the
// five passes and the per-axis tables live in one file-scope device array of
// fixed size (RK_NOALLOC_MAX_DOUBLES doubles, about 16.8 MB), which every GPU
// that loads this library holds until the process exits, next to two small
// arrays for the status flags and the axis projections of chi.
#include <algorithm>
#include <cstring>

#include "fcrkpm.h"
#include "rk_internal.cuh"

namespace rk {
namespace {

constexpr long long kTableDoubles = 8192;  // per-axis multiplier rows and twiddles
static_assert(RK_NOALLOC_MAX_DOUBLES > kTableDoubles, "scratch too small");
constexpr int kMaxSide = 1024;             // box side covered by the projection array

static __device__ __align__(256) double g_noalloc_scratch[RK_NOALLOC_MAX_DOUBLES];
// [0]: a bounded wait for an input tile gave up; [1]: chi violates the gap of Eq. 66
static __device__ __align__(16) int g_noalloc_flags[4];
// occupied node indices of chi along x, y, z (n0 + n1 + n2 bytes)
static __device__ __align__(16) uint8_t g_noalloc_proj[3 * kMaxSide];

// Device address of a file-scope array for the current device: the host-side
// name is only a stand-in.  Looked up on every call (no allocation), so it also
// holds after a device reset or on another device.
template <typename P, typename Sym>
cudaError_t symbol_address(P** out, const Sym& sym) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, sym);
  if (e != cudaSuccess) return e;
  *out = static_cast<P*>(p);
  return cudaSuccess;
}

// An array the kernels may read or write in place: device (or managed) memory of
// the current device, aligned to 16 bytes.
bool device_array_ok(const void* p, int dev) {
  if (!p || reinterpret_cast<uintptr_t>(p) % 16 != 0) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

// proj[i] = 1 (x), proj[n0 + j] = 1 (y), proj[n0 + n1 + k] = 1 (z) for every node
// (i, j, k) of chi; each block gathers its nodes in shared memory first.
__global__ void k_noalloc_project(const uint8_t* chi, int n0, int n1, int n2, long long nbox, uint8_t* proj) {
  __shared__ uint8_t loc[3 * kMaxSide];
  const int np = n0 + n1 + n2;
  for (int t = threadIdx.x; t < np; t += blockDim.x) loc[t] = 0;
  __syncthreads();
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < nbox;
       idx += (long long)gridDim.x * blockDim.x) {
    if (!chi[idx]) continue;
    const long long jk = idx / n0;
    loc[idx - jk * n0] = 1;
    loc[n0 + (int)(jk % n1)] = 1;
    loc[n0 + n1 + (int)(jk / n1)] = 1;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < np; t += blockDim.x)
    if (loc[t]) proj[t] = 1;
}

// Eq. 66 in discrete form (as rk_setup checks it): along each axis the occupied
// indices must leave a circular run of at least `reach` empty ones; flag = 1 if
// not.  One thread per axis.
__global__ void k_noalloc_gap(const uint8_t* proj, int n0, int n1, int n2, int reach, int* flag) {
  const int ax = threadIdx.x;
  if (ax >= 3) return;
  const int n = ax == 0 ? n0 : (ax == 1 ? n1 : n2);
  const uint8_t* occ = proj + (ax == 0 ? 0 : (ax == 1 ? n0 : n0 + n1));
  int best = 0, run = 0;
  bool any = false;
  for (int t = 0; t < 2 * n; ++t) {
    if (occ[t % n]) {
      any = true;
      run = 0;
    } else {
      run = min(run + 1, n);
      best = max(best, run);
    }
  }
  if (any && best < reach) *flag = 1;
}

// f = NaN when a pass recorded a wait that gave up
__global__ void k_noalloc_poison(double* f, long long nbox, const int* flag) {
  if (!*(volatile const int*)flag) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nbox; i += (long long)gridDim.x * blockDim.x)
    f[i] = __longlong_as_double(0x7ff8000000000000LL);
}

__device__ double noalloc_profile(double z) {  // Eq. 7, zero for z >= 1
  z = fabs(z);
  if (z >= 1.0) return 0.0;
  if (z <= 0.5) return 2.0 / 3.0 - 4.0 * z * z + 4.0 * z * z * z;
  const double t = 1.0 - z;
  return (4.0 / 3.0) * t * t * t;
}

// Spectral multiplier rows (m = 0..mmax, divided by n) and twiddles of one axis,
// computed on the device so no host buffer or copy is needed.
__global__ void k_noalloc_tables(double* coef, cpx<double>* tw, int n, double a_tilde, int reach, int mmax) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    for (int m = 0; m <= mmax; ++m) {
      double acc = (m == 0) ? noalloc_profile(0.0) : 0.0;
      for (int o = 1; o <= reach; ++o) {
        const double xi = (double)o / a_tilde;
        double t = noalloc_profile(xi);
        for (int q = 0; q < m; ++q) t *= xi;
        double sn, cs;
        sincospi(2.0 * (double)(((long long)o * k) % n) / (double)n, &sn, &cs);
        acc += (m % 2 == 0) ? 2.0 * t * cs : -2.0 * t * sn;
      }
      coef[(long long)m * n + k] = acc / (double)n;
    }
    double sn, cs;
    sincospi(2.0 * (double)k / (double)n, &sn, &cs);
    tw[k] = cmk(cs, -sn);
  }
}

// status of a rejected call (the message documents the reason at the call site)
rk_status nf(rk_status s, const char* /*reason*/) { return s; }

}  // namespace
}  // namespace rk

using namespace rk;

extern "C" rk_status rk_apply_K_noalloc(const rk_grid* grid, int32_t degree, double a_tilde, const uint8_t* chi,
                                        const double* chiV, const double* b, const double* d, double* f,
                                        void* stream) {
  if (!grid || !chi || !chiV || !b || !d || !f) return nf(RK_ERR_INVALID_ARG, "NULL argument");
  if (degree != 1 && degree != 2) return nf(RK_ERR_INVALID_ARG, "degree must be 1 or 2");
  if (!(a_tilde > 0.5 && a_tilde < 16.0)) return nf(RK_ERR_INVALID_ARG, "a_tilde out of range");
  for (int k = 0; k < 3; ++k)
    if (!supported_length(grid->n[k])) return nf(RK_ERR_UNSUPPORTED, "box side not built");
  if (grid->n[0] % 2 != 0 || ((long long)grid->n[1] * grid->n[2]) % 2 != 0)
    return nf(RK_ERR_UNSUPPORTED, "n[0] and n[1]*n[2] must be even");
  const int s = degree == 1 ? 4 : 10;
  const int nX = degree + 1;
  const int nY = degree == 1 ? 3 : 6;
  const long long nbox = (long long)grid->n[0] * grid->n[1] * grid->n[2];
  const long long need = (long long)(nX + 2 * nY) * nbox + kTableDoubles;
  if (need > RK_NOALLOC_MAX_DOUBLES)
    return nf(RK_ERR_UNSUPPORTED, "box too large for the fixed scratch of rk_apply_K_noalloc");
  int reach = 0;
  while (reach < 64) {
    const double z = (double)(reach + 1) / a_tilde;
    if (!(z < 1.0)) break;
    ++reach;
  }
  long long tab_need = 0;
  for (int k = 0; k < 3; ++k) tab_need += (long long)(2 * degree + 1) * grid->n[k] + 2LL * grid->n[k];
  if (tab_need > kTableDoubles) return nf(RK_ERR_UNSUPPORTED, "tables exceed the fixed scratch");
  for (int k = 0; k < 3; ++k)
    if (grid->n[k] > kMaxSide) return nf(RK_ERR_UNSUPPORTED, "box side beyond the projection array");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nf(RK_ERR_CUDA, "cudaGetDevice failed");
  const void* arrays[5] = {chi, chiV, b, d, f};
  for (const void* p : arrays)
    if (!device_array_ok(p, dev))
      return nf(RK_ERR_INVALID_ARG, "arrays must be 16-byte aligned device memory of the current device");
  cudaStream_t st = (cudaStream_t)stream;
  double* base = nullptr;
  int* flags = nullptr;
  uint8_t* proj = nullptr;
  if (symbol_address(&base, g_noalloc_scratch) != cudaSuccess || symbol_address(&flags, g_noalloc_flags) != cudaSuccess ||
      symbol_address(&proj, g_noalloc_proj) != cudaSuccess)
    return nf(RK_ERR_CUDA, "cudaGetSymbolAddress failed");

  // the gap of Eq. 66, checked on the device before anything else is queued
  if (cudaMemsetAsync(flags, 0, 4 * sizeof(int), st) != cudaSuccess ||
      cudaMemsetAsync(proj, 0, 3 * kMaxSide, st) != cudaSuccess)
    return nf(RK_ERR_CUDA, "clearing the flags failed");
  {
    const long long blocks = std::min<long long>((nbox + 255) / 256, 4 * 152);
    count_launch(2);
    k_noalloc_project<<<(unsigned)blocks, 256, 0, st>>>(chi, grid->n[0], grid->n[1], grid->n[2], nbox, proj);
    k_noalloc_gap<<<1, 32, 0, st>>>(proj, grid->n[0], grid->n[1], grid->n[2], reach, flags + 1);
    int gap_bad = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&gap_bad, flags + 1, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return nf(RK_ERR_CUDA, "gap check failed");
    if (gap_bad) return nf(RK_ERR_UNSUPPORTED, "gap of chi narrower than the support (Eq. 66)");
  }

  // scratch layout: [tables | x outputs | y outputs | z outputs]
  double* coef[3];
  cpx<double>* tw[3];
  double* q = base;
  for (int k = 0; k < 3; ++k) {
    coef[k] = q;
    q += (size_t)(2 * degree + 1) * grid->n[k];
    tw[k] = reinterpret_cast<cpx<double>*>(q);
    q += 2 * (size_t)grid->n[k];
  }
  double* fields = base + kTableDoubles;
  auto fld = [&](int i) { return fields + (size_t)i * nbox; };
  for (int k = 0; k < 3; ++k) {
    count_launch();
    k_noalloc_tables<<<(grid->n[k] + 127) / 128, 128, 0, st>>>(coef[k], tw[k], grid->n[k], a_tilde, reach, degree);
  }
  if (cudaGetLastError() != cudaSuccess) return nf(RK_ERR_CUDA, "table kernel launch failed");

  // basis exponents in the order [1, x, y, z, x^2, xy, xz, y^2, yz, z^2] (Eq. 4)
  static const int al[10][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0},
                                {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1}, {0, 0, 2}};
  int ymx[6], ymy[6], ny = 0;
  int zmz[6][3], zp[6][3], zn[6] = {0, 0, 0, 0, 0, 0};
  for (int p = 0; p < s; ++p) {
    int g = -1;
    for (int t = 0; t < ny; ++t)
      if (ymx[t] == al[p][0] && ymy[t] == al[p][1]) g = t;
    if (g < 0) {
      g = ny++;
      ymx[g] = al[p][0];
      ymy[g] = al[p][1];
    }
    zmz[g][zn[g]] = al[p][2];
    zp[g][zn[g]] = p;
    ++zn[g];
  }
  auto base_args = [&](int axis) {
    PassArgs<double> a;
    memset(&a, 0, sizeof(a));
    a.err = flags;                 // a bounded wait that gives up sets flags[0]
    a.coef_rows = degree + 1;      // the rows the table kernel fills
    a.coef = coef[axis];
    a.tw = tw[axis];
    a.nx = grid->n[0];
    a.ny = grid->n[1];
    a.nz = grid->n[2];
    if (axis == 1) {
      a.line_stride = grid->n[0];
      a.other_stride = (long long)grid->n[0] * grid->n[1];
    } else if (axis == 2) {
      a.line_stride = (long long)grid->n[0] * grid->n[1];
      a.other_stride = grid->n[0];
    }
    return a;
  };
  // x pass: chi o d -> X_m
  PassArgs<double> ax = base_args(0);
  ax.in[0] = d;
  ax.in_mask = chi;
  ax.n_groups = 1;
  for (int m = 0; m < nX; ++m) {
    ax.out[m] = fld(m);
    ax.term_io[m] = m;
    ax.term_m[m] = m;
  }
  ax.g_begin[1] = nX;
  if (launch_split<double>(0, grid->n[0], ax, st) != cudaSuccess) return nf(RK_ERR_CUDA, "x pass failed");
  // y pass: X_mx -> Y_(mx,my)
  PassArgs<double> ay = base_args(1);
  ay.n_groups = nX;
  int t = 0;
  for (int mx = 0; mx < nX; ++mx) {
    ay.in[mx] = fld(mx);
    ay.g_io[mx] = mx;
    ay.g_begin[mx] = t;
    for (int g = 0; g < ny; ++g)
      if (ymx[g] == mx) {
        ay.out[g] = fld(nX + g);
        ay.term_io[t] = g;
        ay.term_m[t] = ymy[g];
        ++t;
      }
  }
  ay.g_begin[nX] = t;
  if (launch_split<double>(1, grid->n[1], ay, st) != cudaSuccess) return nf(RK_ERR_CUDA, "y pass failed");
  // fused z pass of Alg. 2
  ZArgs<double> az;
  memset(&az, 0, sizeof(az));
  az.n_groups = ny;
  t = 0;
  for (int g = 0; g < ny; ++g) {
    az.g_begin[g] = t;
    for (int j = 0; j < zn[g]; ++j) {
      az.term_mz[t] = zmz[g][j];
      az.term_p[t] = zp[g][j];
      ++t;
    }
    az.in[g] = fld(nX + g);
    az.out[g] = fld(nX + ny + g);
  }
  az.g_begin[ny] = t;
  az.b = b;
  az.s = s;
  az.wfield = chiV;
  az.coef = coef[2];
  az.tw = tw[2];
  az.nx = grid->n[0];
  az.ny = grid->n[1];
  az.nz = grid->n[2];
  az.nbox = nbox;
  if (launch_z<double>(Z_STIFF, grid->n[2], az, st) != cudaSuccess) return nf(RK_ERR_CUDA, "z pass failed");
  // reflected y pass: Z_(mx,my) -> X_mx
  PassArgs<double> ry = base_args(1);
  ry.reflect = 1;
  ry.n_groups = nX;
  t = 0;
  for (int mx = 0; mx < nX; ++mx) {
    ry.out[mx] = fld(mx);
    ry.g_io[mx] = mx;
    ry.g_begin[mx] = t;
    for (int g = 0; g < ny; ++g)
      if (ymx[g] == mx) {
        ry.in[g] = fld(nX + ny + g);
        ry.term_io[t] = g;
        ry.term_m[t] = ymy[g];
        ++t;
      }
  }
  ry.g_begin[nX] = t;
  if (launch_merge<double>(1, grid->n[1], ry, st) != cudaSuccess) return nf(RK_ERR_CUDA, "y merge failed");
  // reflected x pass: X_m -> f, masked by chi
  PassArgs<double> rx = base_args(0);
  rx.reflect = 1;
  rx.out_mask = chi;
  rx.n_groups = 1;
  rx.out[0] = f;
  for (int m = 0; m < nX; ++m) {
    rx.in[m] = fld(m);
    rx.term_io[m] = m;
    rx.term_m[m] = m;
  }
  rx.g_begin[1] = nX;
  if (launch_merge<double>(0, grid->n[0], rx, st) != cudaSuccess) return nf(RK_ERR_CUDA, "x merge failed");
  count_launch();
  k_noalloc_poison<<<(unsigned)std::min<long long>((nbox + 255) / 256, 4 * 152), 256, 0, st>>>(f, nbox, flags);
  if (cudaGetLastError() != cudaSuccess) return nf(RK_ERR_CUDA, "status kernel launch failed");
  return RK_OK;
}
