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
// that loads this library holds until the process exits.
#include <cstring>
#include <mutex>

#include "fcrkpm.h"
#include "rk_internal.cuh"

namespace rk {
namespace {

constexpr long long kTableDoubles = 8192;  // per-axis multiplier rows and twiddles
static_assert(RK_NOALLOC_MAX_DOUBLES > kTableDoubles, "scratch too small");

static __device__ __align__(256) double g_noalloc_scratch[RK_NOALLOC_MAX_DOUBLES];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
double* g_addr[kMaxDevices] = {};

// Device address of the scratch array for the current device (the host-side name
// is only a stand-in).  Looked up once per device, with that device current.
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
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
  cudaStream_t st = (cudaStream_t)stream;
  double* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return nf(RK_ERR_CUDA, "cudaGetSymbolAddress failed");

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
  return RK_OK;
}
