// rk_api.cu -- host side of the FC-RKPM library: the C ABI declared in
// include/fcrkpm.h.  Owns the handle (tables, coefficient fields, workspaces),
// sequences the axis passes into the operators of Alg. 1-4 and runs the
// conjugate-gradient driver of Alg. 5 (plain FP64, or FP32 inner solves inside
// FP64 iterative refinement).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "fcrkpm.h"
#include "rk_internal.cuh"

using namespace rk;

namespace {

thread_local std::string g_err;

rk_status fail(rk_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

rk_status cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? RK_ERR_OOM : RK_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define RK_CK(...)                                               \
  do {                                                           \
    cudaError_t e_ = (__VA_ARGS__);                              \
    if (e_ != cudaSuccess) return cuda_fail(e_, #__VA_ARGS__);   \
  } while (0)

#define RK_TRY(call)                     \
  do {                                   \
    rk_status s_ = (call);               \
    if (s_ != RK_OK) return s_;          \
  } while (0)

// Eq. 7 with z >= 1 -> 0; second branch in the factored form (4/3)(1 - z)^3.
double kernel_profile(double z) {
  z = std::fabs(z);
  if (z >= 1.0) return 0.0;
  if (z <= 0.5) return 2.0 / 3.0 - 4.0 * z * z + 4.0 * z * z * z;
  const double t = 1.0 - z;
  return (4.0 / 3.0) * t * t * t;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Monomial exponents of the basis (Eq. 4 in 3D), graded order; in 2D (dim = 2) the
// monomials free of z, in the same order ([1, x, y] / [1, x, y, x^2, xy, y^2]: the
// paper states the method in 2D), in 1D those free of y and z ([1, x] / [1, x, x^2],
// Sec. 6.1.1).  Returns s.
int basis_exponents(int degree, int dim, int alpha[][3]) {
  static const int e[10][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0},
                               {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1}, {0, 0, 2}};
  const int n3 = degree == 1 ? 4 : 10;
  int s = 0;
  for (int p = 0; p < n3; ++p) {
    if ((dim < 3 && e[p][2] != 0) || (dim < 2 && e[p][1] != 0)) continue;
    for (int k = 0; k < 3; ++k) alpha[s][k] = e[p][k];
    ++s;
  }
  return s;
}

// Structure of the forward / reflected chains for the basis of the handle:
// x-pass outputs m_x in [0, deg]; y-pass outputs = groups (m_x, m_y); z terms (m_z, p).
struct Chain {
  int deg = 1, s = 4;
  int alpha[10][3];
  int nX = 0;
  int nY = 0;
  int ymx[kMaxIn], ymy[kMaxIn];
  std::vector<std::pair<int, int>> zterms[kMaxIn];  // (m_z, p)
  void build(int degree, int dim) {
    deg = degree;
    s = basis_exponents(degree, dim, alpha);
    nX = deg + 1;
    nY = 0;
    for (int p = 0; p < s; ++p) {
      int g = -1;
      for (int q = 0; q < nY; ++q)
        if (ymx[q] == alpha[p][0] && ymy[q] == alpha[p][1]) g = q;
      if (g < 0) {
        g = nY++;
        ymx[g] = alpha[p][0];
        ymy[g] = alpha[p][1];
        zterms[g].clear();
      }
      zterms[g].push_back({alpha[p][2], p});
    }
  }
};

}  // namespace

// --------------------------------------------------------------------- handle
struct rk_handle {
  int n[3];
  int dim = 3;  // 2 when n[2] == 1: no z axis (no z kernel factor, monomial or gradient); 1 when n[1] == n[2] == 1
  double h[3];
  double a_tilde;
  int degree, s;
  int reach;
  long long nbox;
  long long n_omega;
  int device;
  Chain chain;
  // inputs and coefficient fields (device)
  uint8_t* chi = nullptr;
  uint8_t* chi_gamma = nullptr;
  uint8_t* chi_omega = nullptr;
  double* V = nullptr;
  double* chiV64 = nullptr;
  float* chiV32 = nullptr;
  double* b64 = nullptr;  // [4][s][nbox]
  float* b32 = nullptr;
  // per-axis tables (device): spectral multipliers [2deg+1][n] and twiddles [n]
  double* coef64[3] = {nullptr, nullptr, nullptr};
  float* coef32[3] = {nullptr, nullptr, nullptr};
  cpx<double>* tw64[3] = {nullptr, nullptr, nullptr};
  cpx<float>* tw32[3] = {nullptr, nullptr, nullptr};
  // compressed coefficients of the pointwise stage: node class / index, table of
  // the irregular nodes, interior values
  int* cidx = nullptr;
  double* ctab64 = nullptr;
  float* ctab32 = nullptr;
  long long n_irr = 0;
  double breg64[31] = {};
  float breg32[31] = {};
  // Regular nodes see a support symmetric about them, so their odd moments vanish
  // and b^k_q = 0 for q != 1+k: there g_{1+k} = c_k D_{1+k}, c_k = chi V (b^k_{1+k})^2,
  // and every other g_p = 0.  The z table then carries, at row zrow_scaled[k], c_k
  // times the row of D_{1+k}, so the z SPLIT of Alg. 2 writes the regular nodes'
  // g directly (diag_reg; zrows rows in the z table).
  bool diag_reg = false;
  // bit g: nodes 4g .. 4g + 3 all regular / all outside chi (one spare word at the
  // end); pw_list: the other groups, in order
  uint32_t* regbits = nullptr;
  uint32_t* outbits = nullptr;
  int* pw_list = nullptr;
  long long pw_count = 0;
  int zrow_scaled[3] = {-1, -1, -1};
  int zrows = 0;
  double inv_c[3] = {0.0, 0.0, 0.0};
  // z axis of Alg. 2 as its regular part plus local corrections (rk_zcorr.cuh):
  // zreg_row[g] is the row of the z table holding c n |T^|^2 for group g (-1: the
  // group has no gradient basis function, its regular part is 0); zwin lists the
  // correction windows
  bool zcorr = false;
  int zreg_row[kMaxIn];
  ZWin* zwin = nullptr;
  long long nzwin = 0;
  uint32_t* zbits = nullptr;  // per z-line: need bits (8 words), then marked bits (8 words per line)
  double ztab[3][2 * kZMaxReach + 1] = {};  // T_m(o) along z, m <= degree
  double creg[10] = {};                     // c_p of a regular node
  // workspaces of the operator chains: X outputs, Y outputs, z-pass outputs
  double* ws64 = nullptr;
  float* ws32 = nullptr;
  // solver vectors (allocated on first solve)
  double* sv64 = nullptr;  // x, r, p, Ap, F, d0, t0, t1
  float* sv32 = nullptr;   // x, r, p, Ap, z
  double* partials = nullptr;
  double* xpartials = nullptr;  // one partial p.Ap per block of the x MERGE pass
  unsigned* counters2 = nullptr;  // [0]: x MERGE blocks done, [1]: update blocks done
  double* dscal = nullptr;   // scratch scalars (device)
  CGState* cg = nullptr;     // device CG state
  double* hscal = nullptr;   // pinned host scalars
  // TMA tensor maps of the workspace fields for the strided passes: [axis-1][field]
  std::vector<CUtensorMap> tmaps32[2], tmaps64[2];
  int* err_host = nullptr;   // mapped pinned word: a bounded device wait gave up
  int* err_dev = nullptr;    // its device address
  int short_wait = 0;        // rk_debug_short_waits: first waits for input tiles give up at once
  // spectral preconditioner: half spectra (per handle, rows of nxp complex); the
  // per-axis symbol factors, the symbol parameters and the multiplier tables live
  // in the set-up handle and are shared with its clones
  cpx<float>* spec32 = nullptr;
  cpx<double>* spec64 = nullptr;
  int nxp = 0;
  double* symc64[3] = {nullptr, nullptr, nullptr};
  bool pc_ready = false;
  SymbolArgs<double> sym64;
  float* mult32 = nullptr;   // z SYM multiplier tables (owned by the set-up handle)
  double* mult64 = nullptr;
  // transient and nonlinear solvers (Appendices B, C): 5 FP64 and 1 FP32 scratch
  // fields and 2 x 608 reduction partials, on first use
  double* trans64 = nullptr;
  float* trans32 = nullptr;
  double* part2 = nullptr;
  double* mlumped = nullptr;  // M^l, computed once (Alg. C.2)
  // staging of host arrays
  double* stage[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  unsigned long long* counters = nullptr;  // singular count, first singular
  long long n_singular = 0, first_singular = -1;
  std::vector<void*> owned;
  const rk_handle* parent = nullptr;  // set for clones: domain arrays belong to the parent
  cudaStream_t bstream = nullptr;     // stream of this handle inside rk_solve_batched
  cudaEvent_t bevent = nullptr;
  cudaGraphExec_t chunk_graph = nullptr;  // captured chunk of FP32 CG iterations
  int chunk_len = 0;
  long long chunk_kernels = 0;
  // per-class kernel timing with CUDA events (rk_profile_enable)
  struct Pend {
    int cls;
    cudaEvent_t a, b;
  };
  bool prof_on = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<Pend> pend;
  double prof_ms[2 * RK_PROF_CLASSES] = {};  // [FP32 classes | FP64 classes]
  long long prof_n[2 * RK_PROF_CLASSES] = {};

  template <typename T>
  rk_status alloc(T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    owned.push_back(q);
    *p = (T*)q;
    return RK_OK;
  }
  double* v64(int i) { return sv64 + (size_t)i * nbox; }
  float* v32(int i) { return sv32 + (size_t)i * nbox; }
  template <typename T>
  T* ws(int i);
};
template <>
double* rk_handle::ws<double>(int i) { return ws64 + (size_t)i * nbox; }
template <>
float* rk_handle::ws<float>(int i) { return ws32 + (size_t)i * nbox; }

namespace {

cudaEvent_t prof_event(rk_handle* h) {
  if (!h->ev_pool.empty()) {
    cudaEvent_t e = h->ev_pool.back();
    h->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Resolve the recorded event pairs into per-class milliseconds.
void prof_flush(rk_handle* h) {
  for (auto& p : h->pend) {
    cudaEventSynchronize(p.b);
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      h->prof_ms[p.cls] += ms;
      h->prof_n[p.cls] += 1;
    }
    h->ev_pool.push_back(p.a);
    h->ev_pool.push_back(p.b);
  }
  h->pend.clear();
}

// Times the launches issued during its lifetime on stream s when profiling is on.
struct ProfScope {
  rk_handle* h;
  int cls;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  ProfScope(rk_handle* h_, int cls_, cudaStream_t s_) : h(h_), cls(cls_), s(s_) {
    if (h->prof_on) {
      a = prof_event(h);
      cudaEventRecord(a, s);
    }
  }
  ~ProfScope() {
    if (!a) return;
    cudaEvent_t b = prof_event(h);
    cudaEventRecord(b, s);
    h->pend.push_back({cls, a, b});
    if (h->pend.size() >= 2048) prof_flush(h);
  }
};

template <typename T>
constexpr int prof_cls(int c) {
  return c + (sizeof(T) == 8 ? RK_PROF_CLASSES : 0);
}

const char* const kProfNames[RK_PROF_CLASSES] = {"x_split", "y_split", "z_split", "stiff_pointwise", "z_eval_u",
                                                 "z_transpose_u", "y_merge", "x_merge", "moment_solve", "cg_vector",
                                                 "z_merge", "precond"};

template <typename T>
const T* coef_of(const rk_handle* h, int axis);
template <>
const double* coef_of<double>(const rk_handle* h, int axis) { return h->coef64[axis]; }
template <>
const float* coef_of<float>(const rk_handle* h, int axis) { return h->coef32[axis]; }
template <typename T>
const cpx<T>* tw_of(const rk_handle* h, int axis);
template <>
const cpx<double>* tw_of<double>(const rk_handle* h, int axis) { return h->tw64[axis]; }
template <>
const cpx<float>* tw_of<float>(const rk_handle* h, int axis) { return h->tw32[axis]; }
template <typename T>
const T* bfields(const rk_handle* h);
template <>
const double* bfields<double>(const rk_handle* h) { return h->b64; }
template <>
const float* bfields<float>(const rk_handle* h) { return h->b32; }
template <typename T>
const T* ctab_of(const rk_handle* h);
template <>
const double* ctab_of<double>(const rk_handle* h) { return h->ctab64; }
template <>
const float* ctab_of<float>(const rk_handle* h) { return h->ctab32; }
template <typename T>
T breg_of(const rk_handle* h, int j);
template <>
double breg_of<double>(const rk_handle* h, int j) { return h->breg64[j]; }
template <>
float breg_of<float>(const rk_handle* h, int j) { return h->breg32[j]; }

template <typename T>
const T* chiV(const rk_handle* h);
template <>
const double* chiV<double>(const rk_handle* h) { return h->chiV64; }
template <>
const float* chiV<float>(const rk_handle* h) { return h->chiV32; }

template <typename T>
PassArgs<T> pass_base(const rk_handle* h, int axis) {
  PassArgs<T> a;
  memset(&a, 0, sizeof(a));
  a.err = h->err_dev;
  a.short_wait = h->short_wait;
  a.coef_rows = 2 * h->degree + 1;
  a.coef = coef_of<T>(h, axis);
  a.tw = tw_of<T>(h, axis);
  a.nx = h->n[0];
  a.ny = h->n[1];
  a.nz = h->n[2];
  if (axis == 1) {
    a.line_stride = h->n[0];
    a.other_stride = (long long)h->n[0] * h->n[1];
  } else if (axis == 2) {
    a.line_stride = (long long)h->n[0] * h->n[1];
    a.other_stride = h->n[0];
  }
  return a;
}

template <typename T>
const std::vector<CUtensorMap>& tmaps_of(const rk_handle* h, int axis);
template <>
const std::vector<CUtensorMap>& tmaps_of<float>(const rk_handle* h, int axis) { return h->tmaps32[axis - 1]; }
template <>
const std::vector<CUtensorMap>& tmaps_of<double>(const rk_handle* h, int axis) { return h->tmaps64[axis - 1]; }

// Tensor maps of the inputs of a strided pass when every input is a whole
// workspace field with an encoded map (else false: the pass uses cp.async).
template <typename T>
bool tile_maps_for(rk_handle* h, int axis, const PassArgs<T>& a, TileMaps* tm) {
  if (axis == 0) return false;
  const std::vector<CUtensorMap>& maps = tmaps_of<T>(h, axis);
  if (maps.empty()) return false;
  const T* ws = h->ws<T>(0);
  for (int i = 0; i < kMaxIn; ++i) {
    if (!a.in[i]) continue;
    if (i >= kMaxTma || a.in[i] < ws) return false;
    const long long off = a.in[i] - ws;
    if (off % h->nbox || off / h->nbox >= (long long)maps.size()) return false;
    tm->m[i] = maps[(size_t)(off / h->nbox)];
  }
  return true;
}

// pw: the z SPLIT of Alg. 2 also applies the pointwise stage to the regular nodes
template <typename T>
rk_status run_split(rk_handle* h, int axis, const PassArgs<T>& a, cudaStream_t s,
                    const PointwiseArgs<T>* pw = nullptr, int prof = -1) {
  ProfScope ps(h, prof_cls<T>(prof >= 0 ? prof : (axis == 0 ? RK_PROF_X_SPLIT : (axis == 1 ? RK_PROF_Y_SPLIT : RK_PROF_Z_SPLIT))),
               s);
  TileMaps tm;
  const bool use = tile_maps_for<T>(h, axis, a, &tm);
  cudaError_t e = launch_split<T>(axis, h->n[axis], a, s, use ? &tm : nullptr, pw);
  return e == cudaSuccess ? RK_OK : cuda_fail(e, "split pass");
}
template <typename T>
rk_status run_merge(rk_handle* h, int axis, const PassArgs<T>& a, cudaStream_t s) {
  ProfScope ps(h, prof_cls<T>(axis == 0 ? RK_PROF_X_MERGE : (axis == 1 ? RK_PROF_Y_MERGE : RK_PROF_Z_MERGE)), s);
  TileMaps tm;
  const bool use = tile_maps_for<T>(h, axis, a, &tm);
  cudaError_t e = launch_merge<T>(axis, h->n[axis], a, s, use ? &tm : nullptr);
  return e == cudaSuccess ? RK_OK : cuda_fail(e, "merge pass");
}

// Workspace layout of the operator chains: [0, nX) x-pass outputs, [nX, nX+nY)
// y-pass outputs, [nX+nY, nX+2nY) z-pass outputs, [nX+2nY, nX+2nY+s) the fields
// D_p / g_p of the z axis of Alg. 2.
inline int ws_fields(const Chain& c) { return c.nX + 2 * c.nY + c.s; }

// CG step fused into the x passes of A p: p = r + beta p before the x SPLIT uses
// it, p . Ap (and alpha) after the x MERGE writes Ap.
template <typename T>
struct CGFuse {
  T* p;
  const T* r;
};

// forward chain, x and y passes: E_{mx,my} = conv_x conv_y (mask o d)   (Alg. 2 line 1-2)
template <typename T>
rk_status chain_forward_xy(rk_handle* h, const T* d, const uint8_t* in_mask, cudaStream_t s,
                           const CGFuse<T>* fuse = nullptr) {
  const Chain& c = h->chain;
  PassArgs<T> ax = pass_base<T>(h, 0);
  ax.in[0] = d;
  ax.in_mask = in_mask;
  if (fuse) {
    ax.cg_p = fuse->p;
    ax.cg_r = fuse->r;
    ax.cg = h->cg;
  }
  ax.n_groups = 1;
  ax.g_io[0] = 0;
  ax.g_begin[0] = 0;
  for (int m = 0; m < c.nX; ++m) {
    ax.out[m] = h->ws<T>(m);
    ax.term_io[m] = m;
    ax.term_m[m] = m;
  }
  ax.g_begin[1] = c.nX;
  RK_TRY(run_split<T>(h, 0, ax, s));
  if (h->dim == 1) return RK_OK;  // 1D: the x outputs are the D_p
  PassArgs<T> ay = pass_base<T>(h, 1);
  ay.n_groups = c.nX;
  int q = 0;
  for (int mx = 0; mx < c.nX; ++mx) {
    ay.in[mx] = h->ws<T>(mx);
    ay.g_io[mx] = mx;
    ay.g_begin[mx] = q;
    for (int g = 0; g < c.nY; ++g)
      if (c.ymx[g] == mx) {
        ay.out[g] = h->ws<T>(c.nX + g);
        ay.term_io[q] = g;
        ay.term_m[q] = c.ymy[g];
        ++q;
      }
  }
  ay.g_begin[c.nX] = q;
  return run_split<T>(h, 1, ay, s);
}

// reflected chain, y and x passes: f = out_mask o sum conv_x(Hbar) conv_y(Hbar) G   (Alg. 2 last line)
// G_g in workspace field gin + g (default: the z-pass outputs; in 2D the fields of
// the y-pass outputs, which hold g_p there)
template <typename T>
rk_status chain_reflect_yx(rk_handle* h, T* f, const uint8_t* out_mask, cudaStream_t s,
                           const CGFuse<T>* fuse = nullptr, int gin = -1) {
  const Chain& c = h->chain;
  if (gin < 0) gin = c.nX + c.nY;
  PassArgs<T> ay = pass_base<T>(h, 1);
  ay.reflect = 1;
  ay.n_groups = c.nX;
  int q = 0;
  for (int mx = 0; mx < c.nX; ++mx) {
    ay.out[mx] = h->ws<T>(mx);
    ay.g_io[mx] = mx;
    ay.g_begin[mx] = q;
    for (int g = 0; g < c.nY; ++g)
      if (c.ymx[g] == mx) {
        ay.in[g] = h->ws<T>(gin + g);
        ay.term_io[q] = g;
        ay.term_m[q] = c.ymy[g];
        ++q;
      }
  }
  ay.g_begin[c.nX] = q;
  if (h->dim > 1) RK_TRY(run_merge<T>(h, 1, ay, s));  // 1D: the g_p already sit in the x fields
  PassArgs<T> ax = pass_base<T>(h, 0);
  ax.reflect = 1;
  ax.out_mask = out_mask;
  if (fuse) {
    ax.cg_p = fuse->p;
    ax.cg = h->cg;
    ax.partials = h->xpartials;
    ax.counter = h->counters2;
  }
  ax.n_groups = 1;
  ax.out[0] = f;
  ax.g_io[0] = 0;
  ax.g_begin[0] = 0;
  for (int m = 0; m < c.nX; ++m) {
    ax.in[m] = h->ws<T>(m);
    ax.term_io[m] = m;
    ax.term_m[m] = m;
  }
  ax.g_begin[1] = c.nX;
  return run_merge<T>(h, 0, ax, s);
}

template <typename T>
ZArgs<T> z_base(const rk_handle* h) {
  ZArgs<T> a;
  memset(&a, 0, sizeof(a));
  const Chain& c = h->chain;
  a.n_groups = c.nY;
  int q = 0;
  for (int g = 0; g < c.nY; ++g) {
    a.g_begin[g] = q;
    for (auto& t : c.zterms[g]) {
      a.term_mz[q] = t.first;
      a.term_p[q] = t.second;
      ++q;
    }
  }
  a.g_begin[c.nY] = q;
  a.b = bfields<T>(h);
  a.s = h->s;
  a.coef = coef_of<T>(h, 2);
  a.tw = tw_of<T>(h, 2);
  a.nx = h->n[0];
  a.ny = h->n[1];
  a.nz = h->n[2];
  a.nbox = h->nbox;
  return a;
}

template <typename T>
rk_status run_z(rk_handle* h, int mode, const ZArgs<T>& a, cudaStream_t s) {
  ProfScope ps(h, prof_cls<T>(mode == Z_STIFF ? RK_PROF_Z_STIFF : (mode == Z_EVAL_U ? RK_PROF_Z_EVAL_U : RK_PROF_Z_TRANSPOSE_U)), s);
  cudaError_t e = launch_z<T>(mode, h->n[2], a, s);
  return e == cudaSuccess ? RK_OK : cuda_fail(e, "z pass");
}

// Alg. 2: f = out_mask o K (in_mask o d).  The z axis runs as three kernels: a
// SPLIT along z (E_(ax,ay) -> D_p, p = 1..s), the pointwise stage of Eq. 90-91 in
// place (D_p -> g_p), and a reflected MERGE along z (g_p -> G_(ax,ay)).
// p -> workspace field of D_p in 2D: the y-pass output of the group of p (each
// group (m_x, m_y) holds one basis function there)
inline int field_2d(const Chain& c, int p) {
  for (int g = 0; g < c.nY; ++g)
    if (c.zterms[g][0].second == p) return c.nX + g;
  return -1;
}
// Workspace field of D_p / g_p on a box without a z axis: the y-pass output of p
// in 2D, the x-pass output of p (m = alpha_x(p)) in 1D.
inline int field_low(const rk_handle* h, int p) {
  return h->dim == 1 ? h->chain.alpha[p][0] : field_2d(h->chain, p);
}

template <typename T>
PointwiseArgs<T> pointwise_base(const rk_handle* h) {
  PointwiseArgs<T> pw;
  memset(&pw, 0, sizeof(pw));
  pw.s = h->s;
  pw.cidx = h->cidx;
  pw.ctab = ctab_of<T>(h);
  pw.n_irr = h->n_irr;
  for (int j = 0; j < 3 * h->s + 1; ++j) pw.breg[j] = breg_of<T>(h, j);
  pw.nbox = h->nbox;
  return pw;
}

template <typename T>
ZCorrArgs<T> zcorr_args(const rk_handle* h);

// reflected z MERGE of Alg. 2: G_g = sum_{p in g} conv_z(g_p, Tbar_{alpha_z(p)}) from
// the fields g_p (workspace nX + 2 nY + p) into the z outputs (nX + nY + g)
template <typename T>
rk_status reflect_z(rk_handle* h, cudaStream_t s) {
  const Chain& c = h->chain;
  const int dbase = c.nX + 2 * c.nY;
  PassArgs<T> rz = pass_base<T>(h, 2);
  rz.reflect = 1;
  rz.n_groups = c.nY;
  int q = 0;
  for (int g = 0; g < c.nY; ++g) {
    rz.out[g] = h->ws<T>(c.nX + c.nY + g);
    rz.g_io[g] = g;
    rz.g_begin[g] = q;
    for (auto& t : c.zterms[g]) {
      rz.in[t.second] = h->ws<T>(dbase + t.second);
      rz.term_io[q] = t.second;
      rz.term_m[q] = t.first;
      ++q;
    }
  }
  rz.g_begin[c.nY] = q;
  return run_merge<T>(h, 2, rz, s);
}

template <typename T>
rk_status op_K(rk_handle* h, const T* d, T* f, const uint8_t* in_mask, const uint8_t* out_mask, cudaStream_t s,
               const CGFuse<T>* fuse = nullptr) {
  const Chain& c = h->chain;
  RK_TRY(chain_forward_xy<T>(h, d, in_mask, s, fuse));
  if (h->dim < 3) {
    // no z axis: the y outputs (2D) or x outputs (1D) are the D_p; the pointwise
    // stage in place, then the reflected passes read the g_p from the same fields
    PointwiseArgs<T> pw = pointwise_base<T>(h);
    for (int p = 0; p < h->s; ++p) pw.D[p] = h->ws<T>(field_low(h, p));
    {
      ProfScope ps(h, prof_cls<T>(RK_PROF_Z_STIFF), s);
      cudaError_t e = launch_pointwise_stiff<T>(pw, s);
      if (e != cudaSuccess) return cuda_fail(e, "pointwise stage");
    }
    return chain_reflect_yx<T>(h, f, out_mask, s, fuse, c.nX);
  }
  const int dbase = c.nX + 2 * c.nY;  // D_p / g_p fields
  PassArgs<T> az = pass_base<T>(h, 2);
  az.n_groups = c.nY;
  int q = 0;
  for (int g = 0; g < c.nY; ++g) {
    az.in[g] = h->ws<T>(c.nX + g);
    az.g_io[g] = g;
    az.g_begin[g] = q;
    for (auto& t : c.zterms[g]) {
      az.out[t.second] = h->ws<T>(dbase + t.second);
      az.term_io[q] = t.second;
      az.term_m[q] = t.first;
      ++q;
    }
  }
  az.g_begin[c.nY] = q;
  if (h->zcorr) {
    // the z axis as its regular part -- one spectral pass, E_g -> G_g with the
    // multiplier c n |T^|^2 of the group's gradient basis function (none: G_g = 0)
    // -- and the local corrections of the non-regular nodes (rk_zcorr.cuh)
    // Every group has one multiplier at most, so the pass is split-shaped (one
    // transform in, one product, one transform out per group) and runs on the
    // split kernel, which holds no accumulator and keeps three blocks per SM; the
    // outputs of the groups without a multiplier are set to 0.
    PassArgs<T> rg = pass_base<T>(h, 2);
    rg.coef_rows = h->zrows;
    int ng = 0;
    for (int g = 0; g < c.nY; ++g) {
      T* out = h->ws<T>(c.nX + c.nY + g);
      if (h->zreg_row[g] < 0) {
        RK_CK(cudaMemsetAsync(out, 0, sizeof(T) * (size_t)h->nbox, s));
        continue;
      }
      rg.in[ng] = h->ws<T>(c.nX + g);
      rg.out[ng] = out;
      rg.g_io[ng] = ng;
      rg.g_begin[ng] = ng;
      rg.term_io[ng] = ng;
      rg.term_m[ng] = h->zreg_row[g];
      ++ng;
    }
    rg.n_groups = ng;
    rg.g_begin[ng] = ng;
    if (ng > 0) RK_TRY(run_split<T>(h, 2, rg, s, nullptr, RK_PROF_Z_MERGE));
    {
      ProfScope ps(h, prof_cls<T>(RK_PROF_Z_STIFF), s);
      cudaError_t e = launch_zcorr<T>(zcorr_args<T>(h), s);
      if (e != cudaSuccess) return cuda_fail(e, "z corrections");
    }
    return chain_reflect_yx<T>(h, f, out_mask, s, fuse);
  }
  PointwiseArgs<T> pw = pointwise_base<T>(h);
  for (int p = 0; p < h->s; ++p) pw.D[p] = h->ws<T>(dbase + p);
  if (h->n[0] % 4 == 0 && h->diag_reg) {
    // with diagonal interior coefficients the z SPLIT writes g_x, g_y, g_z of the
    // regular nodes directly (scaled multiplier rows) and 0 for the other g_p of the
    // regular and outside groups; the boundary groups follow in a short kernel
    for (int qq = 0; qq < q; ++qq)
      for (int k = 0; k < 3; ++k)
        if (az.term_io[qq] == 1 + k) az.term_m[qq] = h->zrow_scaled[k];
    az.coef_rows = h->zrows;
    pw.diag = 1;
    pw.regbits = h->regbits;
    pw.outbits = h->outbits;
    for (int k = 0; k < 3; ++k) pw.inv_c[k] = (T)h->inv_c[k];
    RK_TRY(run_split<T>(h, 2, az, s, &pw));
    ProfScope ps(h, prof_cls<T>(RK_PROF_Z_STIFF), s);
    cudaError_t e = launch_pointwise_groups<T>(pw, h->pw_list, h->pw_count, s);
    if (e != cudaSuccess) return cuda_fail(e, "pointwise stage");
  } else {
    RK_TRY(run_split<T>(h, 2, az, s));
    ProfScope ps(h, prof_cls<T>(RK_PROF_Z_STIFF), s);
    cudaError_t e = launch_pointwise_stiff<T>(pw, s);
    if (e != cudaSuccess) return cuda_fail(e, "pointwise stage");
  }
  RK_TRY(reflect_z<T>(h, s));
  return chain_reflect_yx<T>(h, f, out_mask, s, fuse);
}

// The reflected chain of Alg. 2 applied to fields g_p held where the pointwise
// stage leaves them (3D: workspace field nX + 2 nY + p; 2D: the y-pass output of
// p): f = out_mask o sum_p conv(g_p, Hbar^a_p).  With g_p = chi V sum_k b^k_p N^k
// this is B^T N, the gradient-type force of Eq. B.10.
template <typename T>
rk_status op_BT(rk_handle* h, T* f, const uint8_t* out_mask, cudaStream_t s) {
  if (h->dim < 3) return chain_reflect_yx<T>(h, f, out_mask, s, nullptr, h->chain.nX);
  RK_TRY(reflect_z<T>(h, s));
  return chain_reflect_yx<T>(h, f, out_mask, s);
}

// workspace field of g_p for op_BT
inline int g_field(const rk_handle* h, int p) {
  const Chain& c = h->chain;
  return h->dim < 3 ? field_low(h, p) : c.nX + 2 * c.nY + p;
}

// Alg. 3: u = chi o sum_p b^0_p o conv(chi o d, H^a_p)
template <typename T>
rk_status op_U(rk_handle* h, const T* d, T* u, cudaStream_t s) {
  RK_TRY(chain_forward_xy<T>(h, d, h->chi, s));
  if (h->dim < 3) {
    T* D[10];
    for (int p = 0; p < h->s; ++p) D[p] = h->ws<T>(field_low(h, p));
    ProfScope ps(h, prof_cls<T>(RK_PROF_Z_EVAL_U), s);
    cudaError_t e = launch_eval_u_fields<T>(u, D, bfields<T>(h), h->s, h->chi, h->nbox, s);
    return e == cudaSuccess ? RK_OK : cuda_fail(e, "u^h");
  }
  ZArgs<T> z = z_base<T>(h);
  for (int g = 0; g < h->chain.nY; ++g) z.in[g] = h->ws<T>(h->chain.nX + g);
  z.out1 = u;
  z.mask = h->chi;
  return run_z<T>(h, Z_EVAL_U, z, s);
}

// Alg. 4 (wfield = chi V) and the transpose of Alg. 3 (wmask = chi):
// w = chi o sum_p conv(weight o b^0_p o y, Hbar^a_p)
template <typename T>
rk_status op_UT(rk_handle* h, const T* y, T* w, const T* wfield, const uint8_t* wmask, cudaStream_t s) {
  if (h->dim < 3) {
    T* D[10];
    for (int p = 0; p < h->s; ++p) D[p] = h->ws<T>(field_low(h, p));
    {
      ProfScope ps(h, prof_cls<T>(RK_PROF_Z_TRANSPOSE_U), s);
      cudaError_t e = launch_transpose_u_fields<T>(D, y, bfields<T>(h), h->s, wfield, wmask, h->nbox, s);
      if (e != cudaSuccess) return cuda_fail(e, "transpose of u^h");
    }
    return chain_reflect_yx<T>(h, w, h->chi, s, nullptr, h->chain.nX);
  }
  ZArgs<T> z = z_base<T>(h);
  z.in1 = y;
  z.wfield = wfield;
  z.mask = wmask;
  for (int g = 0; g < h->chain.nY; ++g) z.out[g] = h->ws<T>(h->chain.nX + h->chain.nY + g);
  RK_TRY(run_z<T>(h, Z_TRANSPOSE_U, z, s));
  return chain_reflect_yx<T>(h, w, h->chi, s);
}

// ------------------------------------------------------------- staging
struct Staged {
  const void* user;
  void* dev;
  size_t bytes;
  bool host;
};

rk_status stage_in(rk_handle* h, int slot, const void* p, size_t bytes, cudaStream_t s, Staged* out) {
  out->user = p;
  out->bytes = bytes;
  out->host = p && !is_device_ptr(p);
  if (!p) {
    out->dev = nullptr;
    return RK_OK;
  }
  if (!out->host) {
    if (((uintptr_t)p) & 15) return fail(RK_ERR_INVALID_ARG, "device array not 16-byte aligned");
    out->dev = const_cast<void*>(p);
    return RK_OK;
  }
  if (!h->stage[slot]) RK_TRY(h->alloc(&h->stage[slot], (size_t)h->nbox));
  out->dev = h->stage[slot];
  RK_CK(cudaMemcpyAsync(out->dev, p, bytes, cudaMemcpyHostToDevice, s));
  return RK_OK;
}

rk_status stage_out_prepare(rk_handle* h, int slot, void* p, size_t bytes, Staged* out) {
  out->user = p;
  out->bytes = bytes;
  out->host = p && !is_device_ptr(p);
  if (!p) {
    out->dev = nullptr;
    return RK_OK;
  }
  if (!out->host) {
    if (((uintptr_t)p) & 15) return fail(RK_ERR_INVALID_ARG, "device array not 16-byte aligned");
    out->dev = p;
    return RK_OK;
  }
  if (!h->stage[slot]) RK_TRY(h->alloc(&h->stage[slot], (size_t)h->nbox));
  out->dev = h->stage[slot];
  return RK_OK;
}

rk_status stage_out_finish(const Staged& st, cudaStream_t s) {
  if (st.host && st.user) RK_CK(cudaMemcpyAsync(const_cast<void*>(st.user), st.dev, st.bytes, cudaMemcpyDeviceToHost, s));
  return RK_OK;
}

bool any_host(std::initializer_list<const Staged*> l) {
  for (auto* p : l)
    if (p->host) return true;
  return false;
}

// ------------------------------------------------------------ tables
// Spectral multipliers of one axis: for m in [0, mmax], the DFT (Eq. 30) of the
// wrapped table T_m(o) = (o/a~)^m phi(|o|/a~), o = -r..r (Eq. 68, 77), divided by n
// (the 1/n of Eq. 31).  Even m: real spectrum; odd m: imaginary (stored as its
// imaginary part).
void axis_tables(int n, double a_tilde, int reach, int mmax, std::vector<double>& coef,
                 std::vector<cpx<double>>& tw) {
  coef.assign((size_t)(mmax + 1) * n, 0.0);
  std::vector<double> T((size_t)(mmax + 1) * (reach + 1));
  for (int m = 0; m <= mmax; ++m)
    for (int o = 0; o <= reach; ++o) {
      const double xi = (double)o / a_tilde;
      T[(size_t)m * (reach + 1) + o] = std::pow(xi, m) * kernel_profile(xi);
    }
  for (int m = 0; m <= mmax; ++m)
    for (int k = 0; k < n; ++k) {
      double acc = 0.0;
      if (m % 2 == 0) {
        acc = T[(size_t)m * (reach + 1) + 0];
        for (int o = 1; o <= reach; ++o) acc += 2.0 * T[(size_t)m * (reach + 1) + o] * trig::cos2pi((long long)o * k, n);
      } else {
        for (int o = 1; o <= reach; ++o) acc -= 2.0 * T[(size_t)m * (reach + 1) + o] * trig::sin2pi((long long)o * k, n);
      }
      coef[(size_t)m * n + k] = acc / (double)n;
    }
  tw.resize(n);
  for (int m = 0; m < n; ++m) tw[m] = cmk(trig::cos2pi(m, n), -trig::sin2pi(m, n));
}

template <typename T>
void to_device_async(T* dst, const std::vector<T>& src, cudaStream_t s) {
  cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s);
}

// ------------------------------------------------------------------ TMA maps
// Tensor maps of every workspace field for the strided y and z passes: 3D
// x-fastest fields, box {2L, n_y, 1} (y) or {2L, 1, n_z} (z), 128-byte rows.
// Left empty (the passes then copy tiles with cp.async) when the driver entry
// point is unavailable or a field does not meet TMA's alignment rules (row pitch
// a multiple of 16 bytes, line length at most 256).
template <typename T>
void encode_ws_maps(rk_handle* h, std::vector<CUtensorMap>* out, PFN_cuTensorMapEncodeTiled_v12000 enc) {
  const int nf = ws_fields(h->chain);
  constexpr int ROW = 128 / (int)sizeof(T);
  for (int axis = 1; axis <= 2; ++axis) {
    std::vector<CUtensorMap>& maps = out[axis - 1];
    maps.clear();
    cuuint64_t dims[3] = {(cuuint64_t)h->n[0], (cuuint64_t)h->n[1], (cuuint64_t)h->n[2]};
    cuuint64_t strides[2] = {(cuuint64_t)h->n[0] * sizeof(T), (cuuint64_t)h->n[0] * h->n[1] * sizeof(T)};
    cuuint32_t box[3] = {(cuuint32_t)ROW, axis == 1 ? (cuuint32_t)h->n[1] : 1u, axis == 2 ? (cuuint32_t)h->n[2] : 1u};
    cuuint32_t estr[3] = {1u, 1u, 1u};
    if (h->n[axis] > 256 || (strides[0] % 16) || (strides[1] % 16)) continue;
    std::vector<CUtensorMap> m((size_t)nf);
    bool ok = true;
    for (int f = 0; f < nf && ok; ++f) {
      CUresult r = enc(&m[(size_t)f], sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                       3, h->ws<T>(f), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      ok = r == CUDA_SUCCESS;
    }
    if (ok) maps.swap(m);
  }
}

rk_status setup_tma(rk_handle* h) {
  if (!h->err_host) {
    void* p = nullptr;
    RK_CK(cudaHostAlloc(&p, sizeof(int), cudaHostAllocMapped));
    h->err_host = (int*)p;
    *h->err_host = 0;
    void* d = nullptr;
    RK_CK(cudaHostGetDevicePointer(&d, p, 0));
    h->err_dev = (int*)d;
  }
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    return RK_OK;
  }
  auto enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  encode_ws_maps<float>(h, h->tmaps32, enc);
  encode_ws_maps<double>(h, h->tmaps64, enc);
  return RK_OK;
}

// RK_ERR_TIMEOUT if a bounded device wait gave up since the last check (the word
// is cleared).  Only meaningful once the work in question has completed.
rk_status check_device_flag(rk_handle* h) {
  if (!h->err_host || !*(volatile int*)h->err_host) return RK_OK;
  *(volatile int*)h->err_host = 0;
  return fail(RK_ERR_TIMEOUT, "a bounded wait for an input tile of a strided pass gave up");
}

// ------------------------------------------------------------------ solver
rk_status ensure_solver(rk_handle* h) {
  if (!h->sv64) RK_TRY(h->alloc(&h->sv64, (size_t)9 * h->nbox));
  if (!h->sv32) RK_TRY(h->alloc(&h->sv32, (size_t)5 * h->nbox));
  if (!h->partials) RK_TRY(h->alloc(&h->partials, (size_t)kRedBlocks));
  if (!h->xpartials) RK_TRY(h->alloc(&h->xpartials, (size_t)((long long)h->n[1] * h->n[2] / 2 + 1)));
  if (!h->counters2) {
    RK_TRY(h->alloc(&h->counters2, (size_t)2));
    RK_CK(cudaMemset(h->counters2, 0, 2 * sizeof(unsigned)));
  }
  if (!h->dscal) RK_TRY(h->alloc(&h->dscal, (size_t)8));
  if (!h->cg) RK_TRY(h->alloc(&h->cg, (size_t)1));
  if (!h->hscal) {
    void* p = nullptr;
    RK_CK(cudaMallocHost(&p, 16 * sizeof(double)));  // a CGState or a scalar
    h->hscal = (double*)p;
  }
  return RK_OK;
}

rk_status read_scalar(rk_handle* h, const double* dptr, double* out, cudaStream_t s) {
  RK_CK(cudaMemcpyAsync(h->hscal, dptr, sizeof(double), cudaMemcpyDeviceToHost, s));
  RK_CK(cudaStreamSynchronize(s));
  *out = h->hscal[0];
  return RK_OK;
}

rk_status norm2(rk_handle* h, const double* v, double* out, cudaStream_t s) {
  RK_CK(launch_dot<double, double>(v, v, h->nbox, h->partials, h->dscal, s));
  double r2 = 0.0;
  RK_TRY(read_scalar(h, h->dscal, &r2, s));
  RK_TRY(check_device_flag(h));
  *out = std::sqrt(std::max(r2, 0.0));
  return RK_OK;
}

// ----------------------------------------------------- spectral preconditioner
template <typename T>
T*& mult_of(rk_handle* h);
template <>
double*& mult_of<double>(rk_handle* h) { return h->mult64; }
template <>
float*& mult_of<float>(rk_handle* h) { return h->mult32; }
template <typename T>
cpx<T>*& spec_of(rk_handle* h);
template <>
cpx<double>*& spec_of<double>(rk_handle* h) { return h->spec64; }
template <>
cpx<float>*& spec_of<float>(rk_handle* h) { return h->spec32; }

// Symbol of the operator at regular nodes (see rk_precond.cuh): per-axis real
// factors c_m(k) of the table spectra T^_m (m <= degree; i per odd m applied via
// imag/sgn), the interior b^k_p and V, the shift 1e-3 lam(2 pi / n_x, 0, 0) and
// the 1/(n_x n_y n_z) of the unnormalised transforms.
rk_status ensure_precond(rk_handle* h) {
  if (h->pc_ready) return RK_OK;
  if (h->dim < 3) return fail(RK_ERR_UNSUPPORTED, "spectral preconditioner: three-dimensional boxes only");
  if (h->parent) {
    // a clone shares the parent's symbol (set up once, on the first use by either)
    rk_handle* par = const_cast<rk_handle*>(h->parent);
    RK_TRY(ensure_precond(par));
  } else {
    if (!(h->breg64[3 * h->s] > 0.0))
      return fail(RK_ERR_UNSUPPORTED, "spectral preconditioner: the domain has no regular node");
    for (int k = 0; k < 3; ++k)
      if (h->n[k] > 256) return fail(RK_ERR_UNSUPPORTED, "spectral preconditioner: box side above 256");
    int alpha[10][3];
    basis_exponents(h->degree, h->dim, alpha);
    std::vector<double> c[3];
    for (int ax = 0; ax < 3; ++ax) {
      const int n = h->n[ax];
      std::vector<double> coef;
      std::vector<cpx<double>> tw;
      axis_tables(n, h->a_tilde, h->reach, 2 * h->degree, coef, tw);
      c[ax].assign((size_t)(h->degree + 1) * n, 0.0);
      for (int m = 0; m <= h->degree; ++m)
        for (int k = 0; k < n; ++k) c[ax][(size_t)m * n + k] = (double)n * coef[(size_t)m * n + k];
      RK_TRY(h->alloc(&h->symc64[ax], c[ax].size()));
      RK_CK(cudaMemcpy(h->symc64[ax], c[ax].data(), c[ax].size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    SymbolArgs<double> y;
    memset(&y, 0, sizeof(y));
    for (int k = 0; k < 3; ++k) y.n[k] = h->n[k];
    y.s = h->s;
    for (int p = 0; p < h->s; ++p) {
      int odd = 0;
      for (int k = 0; k < 3; ++k) {
        y.alpha[p][k] = alpha[p][k];
        odd += alpha[p][k] % 2;
      }
      y.imag[p] = odd % 2;           // i^odd: 1, i, -1, -i
      y.sgn[p] = (odd % 4 < 2) ? 1.0 : -1.0;
      for (int k = 0; k < 3; ++k) y.b[k][p] = h->breg64[k * h->s + p];
    }
    y.vreg = h->breg64[3 * h->s];
    // lam at the first x frequency, in FP64 on the host
    double R[3] = {0, 0, 0}, I[3] = {0, 0, 0};
    for (int p = 0; p < h->s; ++p) {
      const double f = y.sgn[p] * c[0][(size_t)y.alpha[p][0] * h->n[0] + 1] * c[1][(size_t)y.alpha[p][1] * h->n[1]] *
                       c[2][(size_t)y.alpha[p][2] * h->n[2]];
      for (int k = 0; k < 3; ++k) (y.imag[p] ? I[k] : R[k]) += y.b[k][p] * f;
    }
    double lam1 = 0.0;
    for (int k = 0; k < 3; ++k) lam1 += R[k] * R[k] + I[k] * I[k];
    lam1 *= y.vreg;
    if (!(lam1 > 0.0)) return fail(RK_ERR_UNSUPPORTED, "spectral preconditioner: degenerate symbol");
    y.shift = 1e-3 * lam1;
    y.scale = 1.0 / ((double)h->n[0] * h->n[1] * h->n[2]);
    y.cx = h->symc64[0];
    y.cy = h->symc64[1];
    y.cz = h->symc64[2];
    h->sym64 = y;
  }
  h->nxp = (h->n[0] / 2 + 1 + 1) / 2 * 2;
  h->pc_ready = true;
  return RK_OK;
}

// z = M^{-1} r (rk_precond.cuh), five passes on stream s.  With fused CG state
// (rz_mode >= 0) the last pass also forms r.z and beta.
template <typename T>
rk_status apply_precond(rk_handle* h, const T* r, T* z, cudaStream_t s, int rz_mode) {
  RK_TRY(ensure_precond(h));
  cpx<T>*& S = spec_of<T>(h);
  if (!S) RK_TRY(h->alloc(&S, (size_t)h->nxp * h->n[1] * h->n[2]));
  ProfScope ps(h, prof_cls<T>(RK_PROF_PRECOND), s);
  PxArgs<T> px;
  memset(&px, 0, sizeof(px));
  px.in = r;
  px.S = S;
  px.nxp = h->nxp;
  px.tw = tw_of<T>(h, 0);
  px.nx = h->n[0];
  px.ny = h->n[1];
  px.nz = h->n[2];
  cudaError_t e = launch_px<T>(0, h->n[0], px, s);
  PfftArgs<T> py;
  memset(&py, 0, sizeof(py));
  py.S = S;
  py.ncols = h->nxp;
  py.line_stride = h->nxp;
  py.other_stride = (long long)h->nxp * h->n[1];
  py.nother = h->n[2];
  py.tw = tw_of<T>(h, 1);
  if (e == cudaSuccess) e = launch_pfft<T>(PF_FWD, h->n[1], py, s);
  PfftArgs<T> pz = py;
  pz.line_stride = (long long)h->nxp * h->n[1];
  pz.other_stride = h->nxp;
  pz.nother = h->n[1];
  pz.tw = tw_of<T>(h, 2);
  rk_handle* owner = h->parent ? const_cast<rk_handle*>(h->parent) : h;
  T*& mult = mult_of<T>(owner);
  if (!mult) {
    RK_TRY(owner->alloc(&mult, (size_t)owner->nxp * h->n[1] * h->n[2]));
    RK_CK(launch_symbol_table<T>(owner->sym64, mult, owner->nxp, h->n[1], h->n[2], s));
    // finished before any stream uses it: clones of the owner share the table and
    // may run on other streams (rk_solve_batched)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    RK_CK(cudaStreamIsCapturing(s, &cs));
    if (cs == cudaStreamCaptureStatusNone) RK_CK(cudaStreamSynchronize(s));
  }
  pz.mult = mult;
  if (e == cudaSuccess) e = launch_pfft<T>(PF_SYM, h->n[2], pz, s);
  if (e == cudaSuccess) e = launch_pfft<T>(PF_INV, h->n[1], py, s);
  px.in = nullptr;
  px.out = z;
  px.out_mask = h->chi_omega;
  if (rz_mode >= 0) {
    px.cg_r = r;
    px.cg = h->cg;
    px.partials = h->xpartials;
    px.counter = h->counters2;
    px.rz_mode = rz_mode;
  }
  if (e == cudaSuccess) e = launch_px<T>(1, h->n[0], px, s);
  return e == cudaSuccess ? RK_OK : cuda_fail(e, "preconditioner");
}

// CG on the masked operator A v = chi_Omega o K(chi_Omega o v) in precision T.
// On entry x holds the initial iterate and r = b - A x.  Stops when r.r <= rr_target.
// With pcg, z = M^{-1} r is formed after every update (z holds it) and the search
// direction follows z (PCG); else z is unused.
template <typename T>
rk_status cg_run(rk_handle* h, T* x, T* r, T* p, T* Ap, T* z, bool pcg, double rr_target, int max_iter,
                 int check_every, cudaStream_t s, int* iters, double* rr_final, int* matvecs) {
  const long long n = h->nbox;
  if (pcg)
    RK_CK(launch_fill<T>(p, (T)0, n, s));
  else
    RK_CK(launch_copy<T>(p, r, n, s));
  RK_CK(launch_dot<T, T>(r, r, n, h->partials, h->dscal, s));
  RK_CK(launch_cg_init(h->partials, h->cg, pcg ? 1 : 0, s));
  if (pcg) RK_TRY(apply_precond<T>(h, r, z, s, 2));
  int it = 0;
  double rr = 0.0;
  for (;;) {
    if (it % check_every == 0 || it >= max_iter) {
      RK_CK(cudaMemcpyAsync(h->hscal, h->cg, sizeof(CGState), cudaMemcpyDeviceToHost, s));
      RK_CK(cudaStreamSynchronize(s));
      RK_TRY(check_device_flag(h));
      CGState st;
      memcpy(&st, h->hscal, sizeof(CGState));
      rr = st.rr;
      if (st.flag) {
        *iters = it;
        *rr_final = rr;
        return fail(RK_ERR_BREAKDOWN, "CG breakdown (p^T A p <= 0, r^T z <= 0 or not finite)");
      }
      if (!(rr > rr_target) || it >= max_iter) break;
    }
    // one iteration: p = r + beta p (x pass prologue), Ap (p is zero off chi_Omega,
    // so only the output mask applies), p.Ap -> alpha (x pass epilogue), then
    // x += alpha p, r -= alpha Ap, r.r -> beta
    const CGFuse<T> fz{p, pcg ? z : r};
    RK_TRY(op_K<T>(h, p, Ap, nullptr, h->chi_omega, s, &fz));
    ++*matvecs;
    {
      ProfScope ps(h, prof_cls<T>(RK_PROF_CG_VECTOR), s);
      RK_CK(launch_cg_xr_fused<T>(x, r, p, Ap, h->cg, n, h->partials, h->counters2 + 1, s));
    }
    if (pcg) RK_TRY(apply_precond<T>(h, r, z, s, 0));
    ++it;
  }
  *iters = it;
  *rr_final = rr;
  return RK_OK;
}

// Mixed precision as a resumable job: one FP32 CG (FP32 K.u and vectors, FP64 dot
// products) whose recurrence residual is replaced by the true FP64 residual
// F - A64 x64 whenever it has dropped by the factor inner_tol since the last
// replacement, after the FP32 update accumulated since then is added to the FP64
// iterate.  The search direction is kept across replacements (the Krylov space is
// not lost).  rk_solve runs one job to completion; rk_solve_batched interleaves
// many, each on its own stream.
// A residual replacement is forced after this many FP32 iterations without one, so
// that a stagnating FP32 recurrence is noticed; kStallReplacements replacements in a
// row that do not halve the best FP64 residual hand the solve to FP64 CG.
constexpr int kMaxItersPerReplacement = 1000;
constexpr int kStallReplacements = 3;

struct MixedJob {
  rk_handle* h = nullptr;
  cudaStream_t s = nullptr;
  rk_solve_opts o;
  rk_solve_info* info = nullptr;
  const double* F = nullptr;
  double* x = nullptr;
  double fn = 0, target = 0, rn = 0, rmax = 0, best = 0;
  int stall = 0, it = 0, it_replaced = 0;
  bool done = false;
  bool use_graph = false;
  bool fp64_tail = false;  // the mixed iterations stalled: finish in FP64
  bool pcg = false;        // preconditioned (opts.precond)
};

// r64 = F - A64 x (FP64 operator), rn = |r64|
rk_status true_residual64(rk_handle* h, const double* F, const double* x, rk_solve_info* info, cudaStream_t s,
                          double* rn) {
  RK_TRY(op_K<double>(h, x, h->v64(3), h->chi_omega, h->chi_omega, s));
  info->matvec_f64++;
  RK_CK(launch_sub(h->v64(1), F, h->v64(3), h->nbox, s));
  return norm2(h, h->v64(1), rn, s);
}

// j.rn holds |F - A x| for the current x (r64 = h->v64(1) holds the residual)
rk_status mixed_start(MixedJob& j) {
  rk_handle* h = j.h;
  const long long n = h->nbox;
  j.pcg = j.o.precond != 0;
  RK_CK(launch_to_f32(h->v32(1), h->v64(1), 1.0, n, j.s));
  RK_CK(launch_fill<float>(h->v32(0), 0.0f, n, j.s));
  if (j.pcg)
    RK_CK(launch_fill<float>(h->v32(2), 0.0f, n, j.s));
  else
    RK_CK(launch_copy<float>(h->v32(2), h->v32(1), n, j.s));
  RK_CK(launch_dot<float, float>(h->v32(1), h->v32(1), n, h->partials, h->dscal, j.s));
  RK_CK(launch_cg_init(h->partials, h->cg, j.pcg ? 1 : 0, j.s));
  if (j.pcg) RK_TRY(apply_precond<float>(h, h->v32(1), h->v32(4), j.s, 2));
  j.rmax = j.best = j.rn;
  j.done = j.rn <= j.target;
  return RK_OK;
}

// one fused FP32 iteration: p = r + beta p, Ap, p.Ap -> alpha; x += alpha p, r -= alpha Ap, beta
rk_status mixed_iteration(MixedJob& j) {
  rk_handle* h = j.h;
  float* x32 = h->v32(0);
  float* r32 = h->v32(1);
  float* p32 = h->v32(2);
  float* Ap32 = h->v32(3);
  const CGFuse<float> fz{p32, j.pcg ? h->v32(4) : r32};
  RK_TRY(op_K<float>(h, p32, Ap32, nullptr, h->chi_omega, j.s, &fz));
  {
    ProfScope ps(h, prof_cls<float>(RK_PROF_CG_VECTOR), j.s);
    RK_CK(launch_cg_xr_fused<float>(x32, r32, p32, Ap32, h->cg, h->nbox, h->partials, h->counters2 + 1, j.s));
  }
  if (j.pcg) RK_TRY(apply_precond<float>(h, r32, h->v32(4), j.s, 0));
  return RK_OK;
}

// Issue up to check_every iterations (a replayed CUDA graph when use_graph) and an
// asynchronous copy of the CG scalars to the pinned host slot.
rk_status mixed_issue(MixedJob& j) {
  rk_handle* h = j.h;
  const int k = std::min(j.o.check_every, j.o.max_iter - j.it);
  if (k > 0) {
    if (j.use_graph && !h->prof_on && k == j.o.check_every) {
      if (!h->chunk_graph || h->chunk_len != k) {
        if (h->chunk_graph) cudaGraphExecDestroy(h->chunk_graph);
        h->chunk_graph = nullptr;
        // this chunk runs as ordinary launches (kernel attributes get set), then the
        // same k iterations are captured for the later chunks: the iterates do not
        // depend on whether the handle already held a graph
        for (int i = 0; i < k; ++i) RK_TRY(mixed_iteration(j));
        j.info->matvec_f32 += k;
        j.it += k;
        const long long l0 = g_launches.load();
        cudaGraph_t gr = nullptr;
        RK_CK(cudaStreamBeginCapture(j.s, cudaStreamCaptureModeThreadLocal));
        rk_status st = RK_OK;
        for (int i = 0; i < k && st == RK_OK; ++i) st = mixed_iteration(j);
        cudaError_t e = cudaStreamEndCapture(j.s, &gr);
        if (st != RK_OK) return st;
        if (e != cudaSuccess) return cuda_fail(e, "capture of CG iterations");
        h->chunk_kernels = g_launches.load() - l0;
        g_launches.fetch_sub(h->chunk_kernels);  // counted when the graph runs
        e = cudaGraphInstantiate(&h->chunk_graph, gr, 0);
        cudaGraphDestroy(gr);
        if (e != cudaSuccess) return cuda_fail(e, "graph instantiation");
        h->chunk_len = k;
        RK_CK(cudaMemcpyAsync(h->hscal, h->cg, sizeof(CGState), cudaMemcpyDeviceToHost, j.s));
        return RK_OK;
      }
      RK_CK(cudaGraphLaunch(h->chunk_graph, j.s));
      count_launch((int)h->chunk_kernels);
      j.info->matvec_f32 += k;
      j.it += k;
    } else {
      for (int i = 0; i < k; ++i) RK_TRY(mixed_iteration(j));
      j.info->matvec_f32 += k;
      j.it += k;
    }
  }
  RK_CK(cudaMemcpyAsync(h->hscal, h->cg, sizeof(CGState), cudaMemcpyDeviceToHost, j.s));
  return RK_OK;
}

// Wait for the scalars of the last issue; replace the residual when due.
rk_status mixed_check(MixedJob& j) {
  rk_handle* h = j.h;
  const long long n = h->nbox;
  RK_CK(cudaStreamSynchronize(j.s));
  RK_TRY(check_device_flag(h));
  CGState cs;
  memcpy(&cs, h->hscal, sizeof(CGState));
  const double rest = std::sqrt(std::max(cs.rr, 0.0));
  const bool cap = j.it >= j.o.max_iter;
  const bool due = j.it - j.it_replaced >= kMaxItersPerReplacement;
  if (!(cs.flag || rest <= j.o.inner_tol * j.rmax || rest <= 0.5 * j.target || cap || due)) return RK_OK;
  j.it_replaced = j.it;
  // residual replacement: x64 += x32, r64 = F - A64 x64, r32 = r64
  RK_CK(launch_acc_f32(j.x, h->v32(0), 1.0, n, j.s));
  RK_CK(launch_fill<float>(h->v32(0), 0.0f, n, j.s));
  RK_TRY(true_residual64(h, j.F, j.x, j.info, j.s, &j.rn));
  j.info->outer++;
  if (j.rn <= j.target || cap) {
    j.done = true;
    return RK_OK;
  }
  if (j.rn < 0.5 * j.best) {
    j.best = j.rn;
    j.stall = 0;
  } else {
    ++j.stall;
  }
  // the FP32 recurrence no longer reduces the FP64 residual, or the cap on
  // refinement steps is reached
  if (j.stall >= kStallReplacements || j.info->outer >= j.o.max_outer) {
    j.done = true;
    j.fp64_tail = true;
    return RK_OK;
  }
  RK_CK(launch_to_f32(h->v32(1), h->v64(1), 1.0, n, j.s));
  RK_CK(launch_dot<float, float>(h->v32(1), h->v32(1), n, h->partials, h->dscal, j.s));
  if (cs.flag) {  // restart the direction after a breakdown
    if (j.pcg)
      RK_CK(launch_fill<float>(h->v32(2), 0.0f, n, j.s));
    else
      RK_CK(launch_copy<float>(h->v32(2), h->v32(1), n, j.s));
    RK_CK(launch_cg_init(h->partials, h->cg, j.pcg ? 1 : 0, j.s));
    if (j.pcg) RK_TRY(apply_precond<float>(h, h->v32(1), h->v32(4), j.s, 2));
  } else {
    // only r is replaced: z, r.z and beta keep their recurrence values, so the next
    // direction stays conjugate; the next preconditioner application sees the true r
    RK_CK(launch_cg_set_rr(h->partials, h->cg, j.s));
  }
  j.rmax = j.rn;
  return RK_OK;
}

// FP64 CG with restarts from x (r64 = h->v64(1) holds F - A x, *rn its norm) until
// ||F - A x|| <= target or the iteration budget of o is spent; *total counts the
// iterations already done on entry and is advanced.
rk_status fp64_cg(rk_handle* h, const double* F, double* x, double target, const rk_solve_opts& o,
                  rk_solve_info* info, cudaStream_t s, double* rn, int* total) {
  for (int restart = 0; restart < 8 && *rn > target && *total < o.max_iter; ++restart) {
    int it = 0, mv = 0;
    double rr;
    rk_status st = cg_run<double>(h, x, h->v64(1), h->v64(2), h->v64(3), h->v64(8), o.precond != 0, target * target,
                                  o.max_iter - *total, o.check_every, s, &it, &rr, &mv);
    *total += it;
    info->fp64_iterations += it;
    info->matvec_f64 += mv;
    if (st != RK_OK) return st;
    RK_TRY(true_residual64(h, F, x, info, s, rn));
  }
  return RK_OK;
}

// After the mixed iterations: when the FP32 recurrence stopped reducing the FP64
// residual (the FP32 operator cannot resolve the lowest modes once eps_32 * kappa
// is near 1), finish with FP64 CG from the current iterate.
rk_status mixed_finish(MixedJob& j) {
  if (!j.fp64_tail || !j.o.fp64_finish || j.rn <= j.target) return RK_OK;
  return fp64_cg(j.h, j.F, j.x, j.target, j.o, j.info, j.s, &j.rn, &j.it);
}

// Solve A x = F (F already masked to chi_Omega) to ||F - A x|| <= tol ||F|| with the
// precision of opts; x holds the initial guess (masked) on entry.
rk_status solve_masked(rk_handle* h, const double* F, double* x, const rk_solve_opts& o, rk_solve_info* info,
                       cudaStream_t s) {
  const long long n = h->nbox;
  double* r64 = h->v64(1);
  double* p64 = h->v64(2);
  double* Ap64 = h->v64(3);
  double fn = 0.0;
  RK_TRY(norm2(h, F, &fn, s));
  info->f_norm = fn;
  if (!std::isfinite(fn))
    return fail(RK_ERR_INVALID_ARG, "right-hand side is not finite (NaN or Inf in r, g or the Neumann data)");
  if (fn == 0.0) {
    RK_CK(launch_fill<double>(x, 0.0, n, s));
    info->rel_residual = 0.0;
    return RK_OK;
  }
  const double target = o.tol * fn;
  double rn;
  int total = 0;
  if (o.precision == RK_PREC_FP64) {
    RK_TRY(true_residual64(h, F, x, info, s, &rn));
    RK_TRY(fp64_cg(h, F, x, target, o, info, s, &rn, &total));
  } else {
    MixedJob j;
    j.h = h;
    j.s = s;
    j.o = o;
    j.info = info;
    j.F = F;
    j.x = x;
    j.fn = fn;
    j.target = target;
    RK_TRY(true_residual64(h, F, x, info, s, &j.rn));
    RK_TRY(mixed_start(j));
    while (!j.done) {
      RK_TRY(mixed_issue(j));
      RK_TRY(mixed_check(j));
    }
    RK_TRY(mixed_finish(j));
    rn = j.rn;
    total = j.it;
  }
  info->iterations = total;
  info->rel_residual = rn / fn;
  if (!(rn <= target)) return fail(RK_ERR_NOT_CONVERGED, "tolerance not reached");  // also a NaN residual
  return RK_OK;
}

void fill_defaults(rk_solve_opts* o) {
  o->tol = 1e-10;
  o->max_iter = 200000;
  o->precision = RK_PREC_MIXED;
  o->inner_tol = 0.1;
  o->max_outer = 60;
  o->check_every = 25;
  o->x0_given = 0;
  o->fp64_finish = 1;
  o->precond = RK_PRECOND_NONE;
  o->reserved = 0;
}

rk_status check_opts(const rk_solve_opts& o) {
  if (!(o.tol > 0.0) || o.max_iter < 1 || (o.precision != RK_PREC_FP64 && o.precision != RK_PREC_MIXED) ||
      !(o.inner_tol > 0.0 && o.inner_tol < 1.0) || o.max_outer < 1 || o.check_every < 1 ||
      (o.fp64_finish != 0 && o.fp64_finish != 1) || (o.precond != RK_PRECOND_NONE && o.precond != RK_PRECOND_SPECTRAL))
    return fail(RK_ERR_INVALID_ARG, "invalid solve options");
  return RK_OK;
}

// The forward solve of Alg. 5: d = d_Gamma + x, x on chi_Omega.  Vectors in the
// handle: F = v64(4), d0 = v64(5).
// f^q of Alg. A.1 (Eq. A.4-A.5): chi o sum_p Hbar_p (*) (chi A b0_p q)
rk_status boundary_rhs(rk_handle* h, const double* q, const double* A, double* fq, cudaStream_t s) {
  return op_UT<double>(h, q, fq, A, h->chi, s);
}

// q, A (optional, both or neither): Neumann flux and boundary quadrature weights;
// then F also holds f^q (Eq. 25)
rk_status forward_solve(rk_handle* h, const double* r, const double* g, double* d, const rk_solve_opts& o,
                        rk_solve_info* info, cudaStream_t s, const double* q = nullptr, const double* A = nullptr) {
  const long long n = h->nbox;
  double* F = h->v64(4);
  double* d0 = h->v64(5);
  double* t0 = h->v64(6);
  double* x = h->v64(0);
  // d_Gamma = g on chi_gamma (Eq. 29)
  if (g)
    RK_CK(launch_dirichlet_d0(d0, g, h->chi_gamma, n, s));
  else
    RK_CK(launch_fill<double>(d0, 0.0, n, s));
  // f^r (Alg. 4), f^q (Alg. A.1) and F = chi_Omega o (f^r + f^q - K d_Gamma)
  RK_TRY(op_UT<double>(h, r, t0, h->chiV64, nullptr, s));
  if (q && A) {
    RK_TRY(boundary_rhs(h, q, A, h->v64(8), s));  // v64(8) is free until the CG starts
    RK_CK(launch_add(t0, t0, h->v64(8), n, s));
  }
  RK_TRY(op_K<double>(h, d0, F, h->chi, h->chi_omega, s));
  info->matvec_f64++;
  RK_CK(launch_masked_diff(F, t0, F, h->chi_omega, n, s));
  if (o.x0_given)
    RK_CK(launch_mask(x, d, h->chi_omega, n, s));
  else
    RK_CK(launch_fill<double>(x, 0.0, n, s));
  rk_status st = solve_masked(h, F, x, o, info, s);
  RK_CK(launch_add(d, d0, x, n, s));
  return st;
}

// ------------------------------------------------------ time-dependent terms
// Appendix C: f^m = M v (Alg. C.1, Eq. C.11-C.12) is the chain of Alg. 3 followed
// by that of Alg. 4: A^0 = sum_q b0_q (H_q (*) chi v), f^m = chi o sum_p Hbar_p (*)
// (chi V b0_p A^0).  The lumped mass (Alg. C.2, Eq. C.13) is Alg. 4 applied to 1.
template <typename T>
T* trans_scratch(rk_handle* h);
template <>
double* trans_scratch<double>(rk_handle* h) { return h->trans64; }
template <>
float* trans_scratch<float>(rk_handle* h) { return h->trans32; }

rk_status ensure_transient(rk_handle* h) {
  if (!h->trans64) RK_TRY(h->alloc(&h->trans64, (size_t)5 * h->nbox));
  if (!h->trans32) RK_TRY(h->alloc(&h->trans32, (size_t)h->nbox));
  if (!h->part2) RK_TRY(h->alloc(&h->part2, (size_t)2 * kRedBlocks));
  return RK_OK;
}

template <typename T>
rk_status op_M(rk_handle* h, const T* v, T* fm, cudaStream_t s) {
  RK_TRY(ensure_transient(h));
  T* a0 = trans_scratch<T>(h);  // scratch 0
  RK_TRY(op_U<T>(h, v, a0, s));
  return op_UT<T>(h, a0, fm, chiV<T>(h), nullptr, s);
}

rk_status lumped_mass(rk_handle* h, double* ml, cudaStream_t s) {
  RK_TRY(ensure_transient(h));
  double* one = h->trans64 + (size_t)4 * h->nbox;  // scratch 4
  RK_CK(launch_fill<double>(one, 1.0, h->nbox, s));
  return op_UT<double>(h, one, ml, h->chiV64, nullptr, s);
}

// Alg. C.3 with forward Euler: d += dt (M^l)^{-1} (f - K d) on chi_Omega, d = g on Gamma_g
rk_status transient_explicit(rk_handle* h, const double* f, const double* g, double dt, int n_steps, double* d,
                             cudaStream_t s) {
  RK_TRY(ensure_transient(h));
  const long long n = h->nbox;
  if (!h->mlumped) {
    RK_TRY(h->alloc(&h->mlumped, (size_t)n));
    RK_TRY(lumped_mass(h, h->mlumped, s));
  }
  const double* ml = h->mlumped;
  double* Kd = h->trans64 + (size_t)2 * n;
  if (g) RK_CK(launch_dirichlet_d0(h->trans64 + (size_t)3 * n, g, h->chi_gamma, n, s));
  // d = g on Gamma_g, 0 off chi (d keeps its free values)
  if (g) {
    RK_CK(launch_mask(d, d, h->chi_omega, n, s));
    RK_CK(launch_add(d, d, h->trans64 + (size_t)3 * n, n, s));
  } else {
    RK_CK(launch_mask(d, d, h->chi_omega, n, s));
  }
  for (int k = 0; k < n_steps; ++k) {
    RK_TRY(op_K<double>(h, d, Kd, h->chi, h->chi_omega, s));
    RK_CK(launch_explicit_step(d, f, Kd, ml, h->chi_omega, dt, n, s));
  }
  return RK_OK;
}

// Alg. C.4 with backward Euler: (M + dt K) d_{k+1} = M d_k + dt f, d = g on
// Gamma_g; each step solved by FP64 CG on the free nodes, A = chi_Omega o (M + dt K)
rk_status transient_implicit(rk_handle* h, const double* f, const double* g, double dt, int n_steps, double* d,
                             const rk_solve_opts& o, rk_solve_info* info, cudaStream_t s) {
  RK_TRY(ensure_transient(h));
  RK_TRY(ensure_solver(h));
  const long long n = h->nbox;
  double* x = h->v64(0);   // free part of d
  double* r = h->v64(1);
  double* p = h->v64(2);
  double* Ap = h->v64(3);
  double* b = h->v64(4);
  double* dG = h->v64(5);  // g on Gamma_g
  double* t = h->v64(6);
  double* t2 = h->trans64 + (size_t)1 * n;
  auto apply_A = [&](const double* v, double* out) -> rk_status {
    RK_TRY(op_M<double>(h, v, out, s));
    RK_TRY(op_K<double>(h, v, t2, h->chi_omega, h->chi_omega, s));
    RK_CK(launch_axpby(out, dt, t2, 1.0, n, s));
    RK_CK(launch_mask(out, out, h->chi_omega, n, s));
    info->matvec_f64++;
    return RK_OK;
  };
  auto dot = [&](const double* a, const double* c, double* out) -> rk_status {
    RK_CK(launch_dot<double, double>(a, c, n, h->partials, h->dscal, s));
    return read_scalar(h, h->dscal, out, s);
  };
  if (g)
    RK_CK(launch_dirichlet_d0(dG, g, h->chi_gamma, n, s));
  else
    RK_CK(launch_fill<double>(dG, 0.0, n, s));
  // dt K d_Gamma is the same every step
  double* KdG = h->trans64 + (size_t)2 * n;
  RK_TRY(op_K<double>(h, dG, KdG, h->chi, h->chi_omega, s));
  RK_CK(launch_mask(x, d, h->chi_omega, n, s));
  for (int step = 0; step < n_steps; ++step) {
    // b = chi_Omega o (M x_k + dt f - dt K d_Gamma)   (M d_Gamma cancels between sides)
    RK_TRY(op_M<double>(h, x, b, s));
    RK_CK(launch_axpby(b, dt, f, 1.0, n, s));
    RK_CK(launch_axpby(b, -dt, KdG, 1.0, n, s));
    RK_CK(launch_mask(b, b, h->chi_omega, n, s));
    double bn = 0.0;
    RK_TRY(dot(b, b, &bn));
    bn = std::sqrt(bn);
    if (bn == 0.0) {
      RK_CK(launch_fill<double>(x, 0.0, n, s));
      continue;
    }
    RK_TRY(apply_A(x, Ap));
    RK_CK(launch_sub(r, b, Ap, n, s));
    RK_CK(launch_copy<double>(p, r, n, s));
    double rr = 0.0;
    RK_TRY(dot(r, r, &rr));
    int it = 0;
    while (std::sqrt(rr) > o.tol * bn && it < o.max_iter) {
      RK_TRY(apply_A(p, Ap));
      double pAp = 0.0;
      RK_TRY(dot(p, Ap, &pAp));
      if (!(pAp > 0.0) || !std::isfinite(pAp)) return fail(RK_ERR_BREAKDOWN, "CG breakdown in the implicit step");
      const double al = rr / pAp;
      RK_CK(launch_axpby(x, al, p, 1.0, n, s));
      RK_CK(launch_axpby(r, -al, Ap, 1.0, n, s));
      double rr2 = 0.0;
      RK_TRY(dot(r, r, &rr2));
      RK_CK(launch_axpby(p, 1.0, r, rr2 / rr, n, s));
      rr = rr2;
      ++it;
    }
    info->iterations += it;
    info->outer++;
    // true residual of the step
    RK_TRY(apply_A(x, Ap));
    RK_CK(launch_sub(t, b, Ap, n, s));
    double tr = 0.0;
    RK_TRY(dot(t, t, &tr));
    info->rel_residual = std::max(info->rel_residual, std::sqrt(tr) / bn);
    if (!(std::sqrt(tr) <= 10.0 * o.tol * bn)) return fail(RK_ERR_NOT_CONVERGED, "implicit step not converged");
  }
  RK_CK(launch_add(d, x, dG, n, s));
  return RK_OK;
}

// ------------------------------------------------- nonlinear reaction terms
// Appendix B: f^N = chi o F^{-1}[sum_p F(chi V b0_p N_u) F(Hbar^a_p)] with
// N_u = N(u^h), u^h from Alg. 3 (Eq. B.4, B.9): the chain of Alg. 3, the
// pointwise nonlinearity, the chain of Alg. 4.
rk_status nonlinear_force(rk_handle* h, const double* d, int kind, double c, double* fN, cudaStream_t s) {
  RK_TRY(ensure_transient(h));
  double* u = h->trans64;
  double* Nu = h->trans64 + (size_t)1 * h->nbox;
  RK_TRY(op_U<double>(h, d, u, s));
  RK_CK(launch_nl_apply(Nu, u, h->chi, kind, c, h->nbox, s));
  return op_UT<double>(h, Nu, fN, h->chiV64, nullptr, s);
}

// Gradient-type force (Eq. B.5-B.8 in the form of Eq. B.10): N^k = a_k N(u^h) with
// a fixed direction a, f^N = chi o sum_p conv(chi V sum_k b^k_p N^k, Hbar^a_p) =
// B^T N -- u^h by Alg. 3, the fields g_p, then the reflected chain of Alg. 2.
rk_status nonlinear_grad_force(rk_handle* h, const double* d, int kind, double c, const double a[3], double* fN,
                               cudaStream_t s) {
  RK_TRY(ensure_transient(h));
  double* u = h->trans64;
  double* Nu = h->trans64 + (size_t)1 * h->nbox;
  RK_TRY(op_U<double>(h, d, u, s));
  RK_CK(launch_nl_apply(Nu, u, h->chi, kind, c, h->nbox, s));
  double* g[10];
  for (int p = 0; p < h->s; ++p) g[p] = h->ws<double>(g_field(h, p));
  RK_CK(launch_grad_g(g, h->b64, h->chiV64, Nu, a, h->s, h->nbox, s));
  return op_BT<double>(h, fN, h->chi, s);
}

// Essential boundary conditions imposed weakly by the penalty method (Sec. 2.4):
// the weak form gains beta * int_{Gamma_g} w (u - g) dGamma, with direct nodal
// quadrature on the boundary nodes (weights A, as Eq. A.2) and w, u the RK
// approximations at those nodes (u^h of Alg. 3).  Every chi node is free:
//   (K + beta U^T diag(A) U) d = f^r + beta U^T (A o g),
// with U the nodal interpolation of Alg. 3 and U^T its transpose (the chain of
// Alg. 4 with weights A).  The operator is symmetric positive definite for
// beta > 0 (K is positive semi-definite with the constants in its null space, and
// U^T diag(A) U is positive on them), so plain CG in FP64 solves it.
rk_status solve_penalty(rk_handle* h, const double* r, const double* g, const double* A, double beta, double* d,
                        const rk_solve_opts& o, rk_solve_info* info, cudaStream_t s) {
  RK_TRY(ensure_solver(h));
  const long long n = h->nbox;
  double* x = h->v64(0);
  double* res = h->v64(1);
  double* p = h->v64(2);
  double* Ap = h->v64(3);
  double* b = h->v64(4);
  double* t = h->v64(5);
  double* u = h->v64(6);
  // M v = chi o K (chi o v) + beta U^T (A o U v)
  auto apply = [&](const double* v, double* out) -> rk_status {
    RK_TRY(op_K<double>(h, v, out, h->chi, h->chi, s));
    RK_TRY(op_U<double>(h, v, u, s));
    RK_TRY(op_UT<double>(h, u, t, A, nullptr, s));
    RK_CK(launch_axpby(out, beta, t, 1.0, n, s));
    info->matvec_f64++;
    return RK_OK;
  };
  RK_TRY(op_UT<double>(h, r, b, h->chiV64, nullptr, s));  // f^r (Alg. 4)
  RK_TRY(op_UT<double>(h, g, t, A, nullptr, s));          // U^T (A o g)
  RK_CK(launch_axpby(b, beta, t, 1.0, n, s));
  double bn = 0.0;
  RK_TRY(norm2(h, b, &bn, s));
  info->f_norm = bn;
  if (!std::isfinite(bn)) return fail(RK_ERR_INVALID_ARG, "right-hand side is not finite");
  RK_CK(launch_fill<double>(x, 0.0, n, s));
  RK_CK(launch_copy<double>(res, b, n, s));
  RK_CK(launch_copy<double>(p, b, n, s));
  double rr = 0.0;
  RK_CK(launch_dot<double, double>(res, res, n, h->partials, h->dscal, s));
  RK_TRY(read_scalar(h, h->dscal, &rr, s));
  const double target = o.tol * bn;
  int it = 0;
  while (std::sqrt(rr) > target && it < o.max_iter) {
    RK_TRY(apply(p, Ap));
    double pAp = 0.0;
    RK_CK(launch_dot<double, double>(p, Ap, n, h->partials, h->dscal, s));
    RK_TRY(read_scalar(h, h->dscal, &pAp, s));
    if (!(pAp > 0.0) || !std::isfinite(pAp)) return fail(RK_ERR_BREAKDOWN, "penalty CG: p.Ap <= 0");
    const double alpha = rr / pAp;
    RK_CK(launch_axpby(x, alpha, p, 1.0, n, s));
    RK_CK(launch_axpby(res, -alpha, Ap, 1.0, n, s));
    double rr_new = 0.0;
    RK_CK(launch_dot<double, double>(res, res, n, h->partials, h->dscal, s));
    RK_TRY(read_scalar(h, h->dscal, &rr_new, s));
    RK_CK(launch_axpby(p, 1.0, res, rr_new / rr, n, s));
    rr = rr_new;
    ++it;
  }
  // the true residual of the final iterate
  RK_TRY(apply(x, Ap));
  RK_CK(launch_sub(res, b, Ap, n, s));
  double rn;
  RK_TRY(norm2(h, res, &rn, s));
  info->iterations = it;
  info->fp64_iterations = it;
  info->rel_residual = bn > 0.0 ? rn / bn : 0.0;
  RK_CK(launch_copy<double>(d, x, n, s));
  if (!(rn <= target)) return fail(RK_ERR_NOT_CONVERGED, "penalty CG: iteration cap reached");
  return RK_OK;
}

// Alg. B.3: K d + f^N(d) = f^r on the free nodes, d = g on Gamma_g, by nonlinear
// CG (Polak-Ribiere+) on the convex energy E = 1/2 d.K d + sum_S V_S F(u_S) - d.f^r
// (F' = N, nondecreasing).  The line search along p is Newton's method on
// phi'(alpha) = p.(K x - f^r) + alpha p.K p + sum_S V_S w_S N(u_S + alpha w_S),
// w = U p: after one K.p and one U.p per direction it needs only node sums.
rk_status solve_nonlinear(rk_handle* h, const double* r, const double* g, int kind, double c, double* d,
                          const rk_solve_opts& o, rk_solve_info* info, cudaStream_t s) {
  RK_TRY(ensure_solver(h));
  RK_TRY(ensure_transient(h));
  const long long n = h->nbox;
  double* x = h->v64(0);    // free part of d
  double* R = h->v64(1);    // gradient (residual) on chi_Omega
  double* p = h->v64(2);
  double* Kp = h->v64(3);
  double* F = h->v64(4);    // chi_Omega o f^r
  double* dG = h->v64(5);
  double* Kx = h->v64(6);   // chi_Omega o K (x + d_Gamma)
  double* Rn = h->v64(8);
  double* u = h->trans64 + (size_t)2 * n;  // u^h(x + d_Gamma)
  double* w = h->trans64 + (size_t)3 * n;  // U p
  double* fN = h->trans64 + (size_t)4 * n;
  auto dot = [&](const double* a, const double* b2, double* out) -> rk_status {
    RK_CK(launch_dot<double, double>(a, b2, n, h->partials, h->dscal, s));
    return read_scalar(h, h->dscal, out, s);
  };
  auto line = [&](double alpha, double* s0, double* s1) -> rk_status {
    RK_CK(launch_nl_line(u, w, h->V, h->chi, kind, c, alpha, n, h->part2, h->dscal, s));
    RK_CK(cudaMemcpyAsync(h->hscal, h->dscal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    RK_CK(cudaStreamSynchronize(s));
    *s0 = h->hscal[0];
    *s1 = h->hscal[1];
    return RK_OK;
  };
  // gradient R = chi_Omega o (K x + f^N - f^r) at the current u
  auto gradient = [&](double* out) -> rk_status {
    double* Nu = h->trans64 + (size_t)1 * n;
    RK_CK(launch_nl_apply(Nu, u, h->chi, kind, c, n, s));
    RK_TRY(op_UT<double>(h, Nu, fN, h->chiV64, nullptr, s));
    RK_CK(launch_add(out, Kx, fN, n, s));
    RK_CK(launch_sub(out, out, F, n, s));
    RK_CK(launch_mask(out, out, h->chi_omega, n, s));
    return RK_OK;
  };
  if (g)
    RK_CK(launch_dirichlet_d0(dG, g, h->chi_gamma, n, s));
  else
    RK_CK(launch_fill<double>(dG, 0.0, n, s));
  RK_TRY(op_UT<double>(h, r, F, h->chiV64, nullptr, s));
  RK_CK(launch_mask(F, F, h->chi_omega, n, s));
  RK_CK(launch_fill<double>(x, 0.0, n, s));
  RK_TRY(op_U<double>(h, dG, u, s));
  RK_TRY(op_K<double>(h, dG, Kx, h->chi, h->chi_omega, s));
  info->matvec_f64 += 1;
  RK_TRY(gradient(R));
  double rr0 = 0.0, rr = 0.0;
  RK_TRY(dot(R, R, &rr0));
  rr = rr0;
  info->f_norm = std::sqrt(rr0);
  const double target = o.tol * std::sqrt(rr0);
  RK_CK(launch_axpby(p, -1.0, R, 0.0, n, s));
  int it = 0;
  while (std::sqrt(rr) > target && it < o.max_iter) {
    RK_TRY(op_K<double>(h, p, Kp, h->chi_omega, h->chi_omega, s));
    RK_TRY(op_U<double>(h, p, w, s));
    info->matvec_f64 += 1;
    double pKp = 0.0, pKx = 0.0, pF = 0.0;
    RK_TRY(dot(p, Kp, &pKp));
    RK_TRY(dot(p, Kx, &pKx));
    RK_TRY(dot(p, F, &pF));
    const double c0 = pKx - pF;
    double alpha = 0.0;
    for (int k = 0; k < 40; ++k) {
      double s0 = 0.0, s1 = 0.0;
      RK_TRY(line(alpha, &s0, &s1));
      const double d1 = c0 + alpha * pKp + s0, d2 = pKp + s1;
      if (!(d2 > 0.0) || !std::isfinite(d1)) return fail(RK_ERR_BREAKDOWN, "nonlinear CG: line search failed");
      const double step = d1 / d2;
      alpha -= step;
      if (std::abs(step) <= 1e-15 * std::max(std::abs(alpha), 1e-300)) break;
    }
    RK_CK(launch_axpby(x, alpha, p, 1.0, n, s));
    RK_CK(launch_axpby(u, alpha, w, 1.0, n, s));
    RK_CK(launch_axpby(Kx, alpha, Kp, 1.0, n, s));
    RK_TRY(gradient(Rn));
    double rn_rn, rn_r;
    RK_TRY(dot(Rn, Rn, &rn_rn));
    RK_TRY(dot(Rn, R, &rn_r));
    const double beta = std::max(0.0, (rn_rn - rn_r) / rr);  // Polak-Ribiere+
    RK_CK(launch_axpby(p, -1.0, Rn, beta, n, s));
    double slope;
    RK_TRY(dot(p, Rn, &slope));
    if (!(slope < 0.0)) RK_CK(launch_axpby(p, -1.0, Rn, 0.0, n, s));  // not a descent direction: restart
    RK_CK(launch_copy<double>(R, Rn, n, s));
    rr = rn_rn;
    ++it;
  }
  info->iterations = it;
  info->rel_residual = rr0 > 0.0 ? std::sqrt(rr / rr0) : 0.0;
  RK_CK(launch_add(d, x, dG, n, s));
  if (!(std::sqrt(rr) <= target)) return fail(RK_ERR_NOT_CONVERGED, "nonlinear CG: tolerance not reached");
  return RK_OK;
}

// A node is regular when its whole support (+-reach on every axis) lies in chi and
// its V equals the V of the first such node: its moment matrix (Eq. 48) and hence
// b and chi V are then those of every other regular node.  Regular nodes are
// served from 3s+1 interior values, irregular ones from a compact table in node
// order.
rk_status compress_coefficients(rk_handle* h, cudaStream_t s) {
  const long long n = h->nbox;
  const int nblk = (int)((n + kScanBlock - 1) / kScanBlock);
  uint8_t* tmp = nullptr;
  int* counts = nullptr;
  cudaError_t e = cudaMalloc((void**)&tmp, (size_t)3 * n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&counts, sizeof(int) * ((size_t)nblk + 1));
  auto done = [&](rk_status st) {
    cudaFree(tmp);
    cudaFree(counts);
    return st;
  };
  if (e != cudaSuccess) return done(cuda_fail(e, "compression workspace"));
  uint8_t *ea = tmp, *eb = tmp + n, *cls = tmp + 2 * n;
  if ((e = launch_erode(ea, h->chi, 0, h->reach, h->n, s)) != cudaSuccess ||
      (e = launch_erode(eb, ea, 1, h->reach, h->n, s)) != cudaSuccess ||
      (e = launch_erode(ea, eb, 2, h->reach, h->n, s)) != cudaSuccess)
    return done(cuda_fail(e, "erode"));
  std::vector<uint8_t> er((size_t)n);
  if ((e = cudaMemcpyAsync(er.data(), ea, (size_t)n, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return done(cuda_fail(e, "copy eroded mask"));
  long long reg = -1;
  for (long long i = 0; i < n; ++i)
    if (er[(size_t)i]) {
      reg = i;
      break;
    }
  double vreg = std::nan("");
  if (reg >= 0 && (e = cudaMemcpy(&vreg, h->V + reg, sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return done(cuda_fail(e, "read V"));
  int total = 0;
  if ((e = launch_classify(cls, h->chi, ea, h->V, vreg, n, s)) != cudaSuccess ||
      (e = launch_count_irregular(cls, n, counts, s)) != cudaSuccess ||
      (e = launch_scan_counts(counts, nblk, counts + nblk, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&total, counts + nblk, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return done(cuda_fail(e, "classify"));
  h->n_irr = total;
  const int ncoef = 3 * h->s + 1;
  rk_status st;
  if ((st = h->alloc(&h->cidx, (size_t)n)) != RK_OK ||
      (st = h->alloc(&h->ctab64, (size_t)ctab_pitch<double>(h->s) * total)) != RK_OK ||
      (st = h->alloc(&h->ctab32, (size_t)ctab_pitch<float>(h->s) * total)) != RK_OK)
    return done(st);
  if ((e = launch_compact<double>(cls, counts, n, h->cidx, h->b64, h->s, h->chiV64, h->ctab64, total, s)) !=
          cudaSuccess ||
      (e = launch_compact<float>(cls, counts, n, h->cidx, h->b32, h->s, h->chiV32, h->ctab32, total, s)) !=
          cudaSuccess)
    return done(cuda_fail(e, "compact"));
  if (reg >= 0) {
    double* g = nullptr;
    if ((e = cudaMalloc((void**)&g, sizeof(double) * (size_t)ncoef)) != cudaSuccess) return done(cuda_fail(e, "gather"));
    e = launch_gather(g, h->b64 + (size_t)h->s * n, n, reg, 3 * h->s, s);
    if (e == cudaSuccess) e = launch_gather(g + 3 * h->s, h->chiV64, 0, reg, 1, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->breg64, g, sizeof(double) * ncoef, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(g);
    if (e != cudaSuccess) return done(cuda_fail(e, "gather"));
    for (int j = 0; j < ncoef; ++j) h->breg32[j] = (float)h->breg64[j];
  }
  return done(RK_OK);
}

// Regular-node fast path of the pointwise stage (see rk_handle::diag_reg).  The
// support of a regular node is symmetric about it, so its odd moments (Eq. 48)
// vanish and b^k_q = 0 for q != 1+k exactly; the computed values are the FFT
// rounding of those zeros and are set to 0 (a check rejects anything above 1e-8
// of the diagonal).  Then appends to the z table the rows c_k T_{alpha_z(1+k)}, at
// indices of the same parity as alpha_z(1+k) (odd rows are imaginary spectra,
// Eq. 55).
rk_status scale_regular_rows(rk_handle* h, cudaStream_t s) {
  const int S = h->s, mmax = 2 * h->degree;
  h->zrows = mmax + 1;
  h->diag_reg = false;
  if (h->dim < 3) return RK_OK;  // the fast path lives in the z pass
  if (!(h->breg64[3 * S] > 0.0)) return RK_OK;  // no regular node
  for (int k = 0; k < 3; ++k) {
    const double dk = h->breg64[k * S + 1 + k];
    if (!(std::fabs(dk) > 0.0)) return RK_OK;
    for (int q = 0; q < S; ++q)
      if (q != 1 + k && !(std::fabs(h->breg64[k * S + q]) <= 1e-8 * std::fabs(dk))) return RK_OK;
  }
  for (int k = 0; k < 3; ++k)
    for (int q = 0; q < S; ++q)
      if (q != 1 + k) {
        h->breg64[k * S + q] = 0.0;
        h->breg32[k * S + q] = 0.0f;
      }
  std::vector<double> coef;
  std::vector<cpx<double>> tw;
  axis_tables(h->n[2], h->a_tilde, h->reach, mmax, coef, tw);
  const int n = h->n[2];
  int next[2] = {mmax + 1 + ((mmax + 1) % 2), mmax + 1 + ((mmax + 2) % 2)};  // next free even, odd row
  int rows = mmax + 1;
  double c[3];
  for (int k = 0; k < 3; ++k) {
    const int mz = h->chain.alpha[1 + k][2];
    h->zrow_scaled[k] = next[mz & 1];
    next[mz & 1] += 2;
    rows = std::max(rows, h->zrow_scaled[k] + 1);
    c[k] = h->breg64[3 * S] * h->breg64[k * S + 1 + k] * h->breg64[k * S + 1 + k];
    h->inv_c[k] = 1.0 / c[k];
  }
  // rows of the regular part of the z axis (rk_zcorr.cuh): for the group holding
  // the gradient basis function p = 1 + k, the multiplier c_k n |T^_{alpha_z(p)}|^2
  // of the forward and the reflected convolution with the pointwise factor c_k
  // between them (coef holds T^/n; the inverse transform in between is unnormalised)
  const Chain& ch = h->chain;
  for (int g = 0; g < ch.nY; ++g) {
    h->zreg_row[g] = -1;
    for (auto& t : ch.zterms[g])
      if (t.second >= 1 && t.second <= 3) {
        h->zreg_row[g] = next[0];
        next[0] += 2;
        rows = std::max(rows, h->zreg_row[g] + 1);
      }
  }
  coef.resize((size_t)rows * n, 0.0);
  for (int k = 0; k < 3; ++k) {
    const int mz = h->chain.alpha[1 + k][2];
    for (int i = 0; i < n; ++i) coef[(size_t)h->zrow_scaled[k] * n + i] = c[k] * coef[(size_t)mz * n + i];
  }
  for (int g = 0; g < ch.nY; ++g) {
    if (h->zreg_row[g] < 0) continue;
    for (auto& t : ch.zterms[g])
      if (t.second >= 1 && t.second <= 3) {
        const int k = t.second - 1, mz = t.first;
        for (int i = 0; i < n; ++i) {
          const double cm = coef[(size_t)mz * n + i];
          coef[(size_t)h->zreg_row[g] * n + i] = c[k] * (double)n * cm * cm;
        }
      }
  }
  for (int p = 0; p < S; ++p) h->creg[p] = (p >= 1 && p <= 3) ? c[p - 1] : 0.0;
  std::vector<float> coef32(coef.begin(), coef.end());
  rk_status st;
  if ((st = h->alloc(&h->coef64[2], coef.size())) != RK_OK || (st = h->alloc(&h->coef32[2], coef.size())) != RK_OK)
    return st;
  if (h->nbox % 4 == 0) {
    const long long ng = h->nbox / 4;
    const size_t nwords = (size_t)((ng + 31) / 32) + 1;
    const int nblk = (int)((ng + kScanBlock - 1) / kScanBlock);
    uint8_t* gcls = nullptr;
    int* counts = nullptr;
    int total = 0;
    if ((st = h->alloc(&h->regbits, nwords)) != RK_OK || (st = h->alloc(&h->outbits, nwords)) != RK_OK) return st;
    cudaError_t er = cudaMalloc((void**)&gcls, (size_t)ng);
    if (er == cudaSuccess) er = cudaMalloc((void**)&counts, sizeof(int) * ((size_t)nblk + 1));
    if (er == cudaSuccess) er = cudaMemsetAsync(h->regbits, 0, nwords * sizeof(uint32_t), s);
    if (er == cudaSuccess) er = cudaMemsetAsync(h->outbits, 0, nwords * sizeof(uint32_t), s);
    if (er == cudaSuccess) er = launch_group_class(gcls, h->regbits, h->outbits, h->cidx, ng, s);
    if (er == cudaSuccess) er = launch_count_irregular(gcls, ng, counts, s);
    if (er == cudaSuccess) er = launch_scan_counts(counts, nblk, counts + nblk, s);
    if (er == cudaSuccess) er = cudaMemcpyAsync(&total, counts + nblk, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (er == cudaSuccess) er = cudaStreamSynchronize(s);
    if (er == cudaSuccess && (st = h->alloc(&h->pw_list, (size_t)total)) != RK_OK) er = cudaErrorMemoryAllocation;
    if (er == cudaSuccess) er = launch_list_compact(gcls, counts, ng, h->pw_list, s);
    if (er == cudaSuccess) er = cudaStreamSynchronize(s);
    cudaFree(gcls);
    cudaFree(counts);
    if (er != cudaSuccess) return cuda_fail(er, "group classes");
    h->pw_count = total;
  }
  cudaError_t e = cudaMemcpy(h->coef64[2], coef.data(), coef.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->coef32[2], coef32.data(), coef32.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "copy z table");
  h->zrows = rows;
  h->diag_reg = h->regbits != nullptr;
  return RK_OK;
}

// The z axis of Alg. 2 as its regular part plus local corrections (rk_zcorr.cuh):
// the correction windows of every z-line -- the positions within the reach of a
// node that is not regular but lies within the support of chi (box dilation of chi
// by the reach) -- and the real-space z tables T_m(o).  Needs the regular rows of
// scale_regular_rows; leaves h->zcorr false (the z axis then runs as split,
// pointwise stage and merge) for 2D boxes, boxes without regular nodes and
// supports or sides beyond the window kernel's limits.
rk_status build_zwindows(rk_handle* h, cudaStream_t s) {
  h->zcorr = false;
  if (h->dim != 3 || !h->diag_reg || h->n[2] > 256 || h->reach < 1 || h->reach > kZMaxReach) return RK_OK;
  // the kernel's compile-time basis structure must be the handle's
  const Chain& ch = h->chain;
  for (int g = 0; g < ch.nY; ++g)
    for (auto& t : ch.zterms[g]) {
      const int p = t.second;
      const bool ok = h->s == 4 ? (ZBasis<4>::grp(p) == g && ZBasis<4>::az(p) == t.first)
                                : (ZBasis<10>::grp(p) == g && ZBasis<10>::az(p) == t.first);
      if (!ok) return RK_OK;
    }
  const long long n = h->nbox;
  const long long nl = (long long)h->n[0] * h->n[1];
  const long long ng = (long long)((h->n[0] + kZGW - 1) / kZGW) * h->n[1];
  uint8_t* tmp = nullptr;
  int* counts = nullptr;
  if (!h->zbits) RK_TRY(h->alloc(&h->zbits, (size_t)16 * nl));
  uint32_t* nk = h->zbits;
  uint32_t* mk = h->zbits + (size_t)8 * nl;
  cudaError_t e = cudaMalloc((void**)&tmp, (size_t)3 * n + (size_t)nl);
  if (e == cudaSuccess) e = cudaMalloc((void**)&counts, sizeof(int) * ((size_t)ng + 1));
  auto done = [&](rk_status st) {
    cudaFree(tmp);
    cudaFree(counts);
    return st;
  };
  if (e != cudaSuccess) return done(cuda_fail(e, "window workspace"));
  uint8_t *a = tmp, *b = tmp + n, *need = tmp + 2 * n, *flags = tmp + 3 * n;
  // box dilation of chi by the reach = complement of the erosion of its complement
  if ((e = launch_u8_not(a, h->chi, n, s)) != cudaSuccess || (e = launch_erode(b, a, 0, h->reach, h->n, s)) != cudaSuccess ||
      (e = launch_erode(a, b, 1, h->reach, h->n, s)) != cudaSuccess ||
      (e = launch_erode(b, a, 2, h->reach, h->n, s)) != cudaSuccess || (e = launch_u8_not(a, b, n, s)) != cudaSuccess ||
      (e = launch_zwin_need(need, a, h->cidx, n, s)) != cudaSuccess ||
      (e = launch_zwin_mark(need, h->chi, h->n, h->reach, mk, nk, flags, s)) != cudaSuccess)
    return done(cuda_fail(e, "correction nodes"));
  int total = 0;
  const int chunk = zcorr_chunk(h->s);
  if ((e = launch_zwin_groups(0, mk, flags, h->n, chunk, counts, nullptr, s)) != cudaSuccess ||
      (e = launch_scan_counts(counts, (int)ng, counts + ng, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&total, counts + ng, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return done(cuda_fail(e, "correction windows"));
  rk_status st = h->alloc(&h->zwin, (size_t)std::max(total, 1));
  if (st != RK_OK) return done(st);
  if ((e = launch_zwin_groups(1, mk, flags, h->n, chunk, counts, h->zwin, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return done(cuda_fail(e, "correction windows"));
  h->nzwin = total;
  for (int m = 0; m <= h->degree; ++m)
    for (int o = -h->reach; o <= h->reach; ++o) {
      const double xi = (double)o / h->a_tilde;
      h->ztab[m][o + h->reach] = std::pow(xi, m) * kernel_profile(xi);
    }
  h->zcorr = true;
  return done(RK_OK);
}

template <typename T>
ZCorrArgs<T> zcorr_args(const rk_handle* hc) {
  rk_handle* h = const_cast<rk_handle*>(hc);  // the workspace fields are written through
  ZCorrArgs<T> a;
  memset(&a, 0, sizeof(a));
  const Chain& c = h->chain;
  a.nY = c.nY;
  a.s = h->s;
  for (int g = 0; g < c.nY; ++g) {
    a.E[g] = h->ws<T>(c.nX + g);
    a.G[g] = h->ws<T>(c.nX + c.nY + g);
  }
  a.cidx = h->cidx;
  a.ctab = ctab_of<T>(h);
  for (int p = 0; p < h->s; ++p) a.creg[p] = (T)h->creg[p];
  for (int m = 0; m <= h->degree; ++m)
    for (int j = 0; j <= 2 * h->reach; ++j) a.tab[m][j] = (T)h->ztab[m][j];  // rows of length 2r + 1
  a.r = h->reach;
  a.nx = h->n[0];
  a.ny = h->n[1];
  a.nz = h->n[2];
  a.win = h->zwin;
  a.nwin = h->nzwin;
  a.nbits = h->zbits;
  a.mbits = h->zbits + (size_t)8 * h->n[0] * h->n[1];
  return a;
}

// Vector-Jacobian product of the solve map (r, g) -> u^h for a cotangent e on the
// grid (already masked by chi): w = U^T e (transpose of Alg. 3), one adjoint solve
// A lambda = chi_Omega o w (A = chi_Omega K chi_Omega is symmetric), then
// e_r = chi V o U lambda and e_g = chi_gamma o (w - K lambda).  The map is linear,
// so nothing of the forward solve is needed.  e may alias e_g (it is consumed
// first).  Solver vectors 0, 3, 4, 6 are used as scratch.
rk_status vjp_core(rk_handle* h, const double* e, double* e_r, double* e_g, const rk_solve_opts& o,
                   rk_solve_info* inf, cudaStream_t s) {
  const long long n = h->nbox;
  double* w = h->v64(6);
  double* F = h->v64(4);
  double* lam = h->v64(0);
  RK_TRY(op_UT<double>(h, e, w, nullptr, h->chi, s));
  RK_CK(launch_mask(F, w, h->chi_omega, n, s));
  RK_CK(launch_fill<double>(lam, 0.0, n, s));
  rk_solve_info ainf;
  memset(&ainf, 0, sizeof(ainf));
  rk_status st = solve_masked(h, F, lam, o, &ainf, s);
  inf->iterations += ainf.iterations;
  inf->outer += ainf.outer;
  inf->matvec_f32 += ainf.matvec_f32;
  inf->matvec_f64 += ainf.matvec_f64;
  inf->rel_residual = std::max(inf->rel_residual, ainf.rel_residual);
  if (st != RK_OK) return st;
  // e_g = chi_gamma o (w - K lambda)
  double* Klam = h->v64(3);
  RK_TRY(op_K<double>(h, lam, Klam, h->chi, h->chi_gamma, s));
  RK_CK(launch_masked_diff(e_g, w, Klam, h->chi_gamma, n, s));
  // e_r = chi V o U lambda
  RK_TRY(op_U<double>(h, lam, e_r, s));
  RK_CK(launch_mul(e_r, h->chiV64, n, s));
  return RK_OK;
}

// Alg. 5 "Initialize" for the batched solve: d_Gamma, F = chi_Omega (f^r - K d_Gamma),
// x = 0, |F| and the first true residual; leaves a started mixed job.
rk_status prepare_mixed_job(rk_handle* h, const double* r, const double* g, const rk_solve_opts& o,
                            rk_solve_info* info, cudaStream_t s, MixedJob& j) {
  const long long n = h->nbox;
  double* F = h->v64(4);
  double* d0 = h->v64(5);
  double* t0 = h->v64(6);
  double* x = h->v64(0);
  if (g)
    RK_CK(launch_dirichlet_d0(d0, g, h->chi_gamma, n, s));
  else
    RK_CK(launch_fill<double>(d0, 0.0, n, s));
  RK_TRY(op_UT<double>(h, r, t0, h->chiV64, nullptr, s));
  RK_TRY(op_K<double>(h, d0, F, h->chi, h->chi_omega, s));
  info->matvec_f64++;
  RK_CK(launch_masked_diff(F, t0, F, h->chi_omega, n, s));
  RK_CK(launch_fill<double>(x, 0.0, n, s));
  double fn = 0.0;
  RK_TRY(norm2(h, F, &fn, s));
  info->f_norm = fn;
  if (!std::isfinite(fn))
    return fail(RK_ERR_INVALID_ARG, "right-hand side is not finite (NaN or Inf in r or g)");
  j.h = h;
  j.s = s;
  j.o = o;
  j.info = info;
  j.F = F;
  j.x = x;
  j.fn = fn;
  j.target = o.tol * fn;
  j.use_graph = true;
  RK_CK(launch_copy<double>(h->v64(1), F, n, s));
  j.rn = fn;  // x = 0: the residual is F
  if (fn == 0.0) {
    j.done = true;
    return RK_OK;
  }
  return mixed_start(j);
}

}  // namespace

// ======================================================================= ABI
extern "C" {

void rk_default_solve_opts(rk_solve_opts* opts) {
  if (opts) fill_defaults(opts);
}

int rk_supported_length(int n) { return supported_length(n) ? 1 : 0; }

const char* rk_status_string(rk_status s) {
  switch (s) {
    case RK_OK: return "RK_OK";
    case RK_ERR_INVALID_ARG: return "RK_ERR_INVALID_ARG";
    case RK_ERR_CUDA: return "RK_ERR_CUDA";
    case RK_ERR_OOM: return "RK_ERR_OOM";
    case RK_ERR_SINGULAR_MOMENT: return "RK_ERR_SINGULAR_MOMENT";
    case RK_ERR_NOT_CONVERGED: return "RK_ERR_NOT_CONVERGED";
    case RK_ERR_BREAKDOWN: return "RK_ERR_BREAKDOWN";
    case RK_ERR_TIMEOUT: return "RK_ERR_TIMEOUT";
    case RK_ERR_UNSUPPORTED: return "RK_ERR_UNSUPPORTED";
  }
  return "RK_ERR_UNKNOWN";
}

const char* rk_last_error_message(void) { return g_err.c_str(); }

rk_status rk_destroy(rk_handle* h) {
  if (!h) return RK_OK;
  prof_flush(h);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  if (h->chunk_graph) cudaGraphExecDestroy(h->chunk_graph);
  if (h->bevent) cudaEventDestroy(h->bevent);
  if (h->bstream) cudaStreamDestroy(h->bstream);
  for (void* p : h->owned) cudaFree(p);
  if (h->hscal) cudaFreeHost(h->hscal);
  if (h->err_host) cudaFreeHost(h->err_host);
  delete h;
  return RK_OK;
}

int64_t rk_kernel_launches(void) { return (int64_t)g_launches.load(); }

rk_status rk_profile_enable(rk_handle* h, int32_t enable) {
  if (!h) return fail(RK_ERR_INVALID_ARG, "handle is NULL");
  prof_flush(h);
  for (int c = 0; c < 2 * RK_PROF_CLASSES; ++c) {
    h->prof_ms[c] = 0.0;
    h->prof_n[c] = 0;
  }
  h->prof_on = enable != 0;
  return RK_OK;
}

rk_status rk_profile_read(rk_handle* h, double* ms, int64_t* launches, int32_t n_classes) {
  if (!h || n_classes < 0) return fail(RK_ERR_INVALID_ARG, "bad arguments");
  prof_flush(h);
  for (int c = 0; c < n_classes && c < 2 * RK_PROF_CLASSES; ++c) {
    if (ms) ms[c] = h->prof_ms[c];
    if (launches) launches[c] = h->prof_n[c];
  }
  return RK_OK;
}

const char* rk_profile_class_name(int32_t cls) {
  return (cls >= 0 && cls < RK_PROF_CLASSES) ? kProfNames[cls] : "";
}

rk_status rk_setup(const rk_grid* grid, const uint8_t* chi, const uint8_t* chi_gamma, const double* V,
                   int32_t degree, double a_tilde, void* stream, rk_handle** out) {
  g_err.clear();
  if (!out) return fail(RK_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!grid || !chi || !V) return fail(RK_ERR_INVALID_ARG, "grid, chi and V are required");
  if (degree != 1 && degree != 2) return fail(RK_ERR_INVALID_ARG, "degree must be 1 or 2");
  if (!(a_tilde > 0.5 && a_tilde < 16.0)) return fail(RK_ERR_INVALID_ARG, "a_tilde out of range");
  // a box one node thick in z is two-dimensional, one node thick in y and z one-dimensional
  const int dim = grid->n[2] == 1 ? (grid->n[1] == 1 ? 1 : 2) : 3;
  if (grid->n[2] > 1 && grid->n[1] == 1) return fail(RK_ERR_INVALID_ARG, "bad grid: n[1] == 1 < n[2]");
  for (int k = 0; k < 3; ++k) {
    if ((k < dim && grid->n[k] < 2) || grid->n[k] < 1 || !(grid->h[k] > 0.0))
      return fail(RK_ERR_INVALID_ARG, "bad grid");
    if (k < dim && !supported_length(grid->n[k]))
      return fail(RK_ERR_UNSUPPORTED, "box side " + std::to_string(grid->n[k]) + " not built");
  }
  if (grid->n[0] % 2 != 0 || (dim > 1 && ((long long)grid->n[1] * grid->n[2]) % 2 != 0))
    return fail(RK_ERR_UNSUPPORTED, "n[0] and n[1]*n[2] must be even");
  if (dim == 1 && grid->n[0] % 4 != 0)  // the pointwise stage reads 16-byte vectors of nodes
    return fail(RK_ERR_UNSUPPORTED, "a 1D box needs n[0] a multiple of 4");
  cudaStream_t s = (cudaStream_t)stream;
  rk_handle* h = new rk_handle();
  auto bail = [&](rk_status st) {
    rk_destroy(h);
    return st;
  };
  for (int k = 0; k < 3; ++k) {
    h->n[k] = grid->n[k];
    h->h[k] = grid->h[k];
  }
  h->a_tilde = a_tilde;
  h->degree = degree;
  h->dim = dim;
  h->nbox = (long long)grid->n[0] * grid->n[1] * grid->n[2];
  cudaGetDevice(&h->device);
  h->chain.build(degree, dim);
  h->s = h->chain.s;
  if (dim < 3)
    for (int p = 0; p < h->s; ++p)
      if (field_low(h, p) < 0) return bail(fail(RK_ERR_INVALID_ARG, "basis without a field of its own"));
  int reach = 0;
  while (kernel_profile((double)(reach + 1) / a_tilde) > 0.0) ++reach;
  h->reach = reach;
  for (int k = 0; k < dim; ++k)
    if (2 * reach + 1 > h->n[k]) return bail(fail(RK_ERR_UNSUPPORTED, "support wider than the box"));
  const long long n = h->nbox;

  // inputs to the device; host copy of chi for the gap check
  rk_status st;
  if ((st = h->alloc(&h->chi, n)) || (st = h->alloc(&h->chi_gamma, n)) || (st = h->alloc(&h->chi_omega, n)) ||
      (st = h->alloc(&h->V, n)) || (st = h->alloc(&h->chiV64, n)) || (st = h->alloc(&h->chiV32, n)) ||
      (st = h->alloc(&h->b64, (size_t)4 * h->s * n)) || (st = h->alloc(&h->b32, (size_t)4 * h->s * n)) ||
      (st = h->alloc(&h->ws64, (size_t)ws_fields(h->chain) * n)) ||
      (st = h->alloc(&h->ws32, (size_t)ws_fields(h->chain) * n)) || (st = h->alloc(&h->counters, 2)))
    return bail(st);
  if ((st = setup_tma(h)) != RK_OK) return bail(st);
  // inputs to the device; the masks are made 0/1, Omega counted and the gap of
  // Eq. 66 checked on the device, with one small read-back
  uint8_t* scr = nullptr;
  if ((st = h->alloc(&scr, (size_t)16 + h->n[0] + h->n[1] + h->n[2])) != RK_OK) return bail(st);
  cudaError_t e = cudaMemcpyAsync(h->chi, chi, n, cudaMemcpyDefault, s);
  if (e == cudaSuccess)
    e = chi_gamma ? cudaMemcpyAsync(h->chi_gamma, chi_gamma, n, cudaMemcpyDefault, s) : cudaMemsetAsync(h->chi_gamma, 0, n, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->V, V, n * sizeof(double), cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = launch_setup_masks(h->chi, h->chi_gamma, h->chi_omega, h->n, dim, reach, scr, s);
  unsigned char res[12];
  if (e == cudaSuccess) e = cudaMemcpyAsync(res, scr, sizeof(res), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bail(cuda_fail(e, "copy inputs"));
  unsigned long long nom = 0;
  int gap_narrow = 0;
  memcpy(&nom, res, sizeof(nom));
  memcpy(&gap_narrow, res + 8, sizeof(gap_narrow));
  h->n_omega = (long long)nom;
  if (gap_narrow)
    return bail(fail(RK_ERR_UNSUPPORTED, "gap between the domain and its periodic image is narrower than the support (Eq. 66)"));

  // per-axis tables for m in [0, 2 deg] (moments need 2 deg; the chains use <= deg)
  const int mmax = 2 * degree;
  for (int k = 0; k < dim; ++k) {
    std::vector<double> coef;
    std::vector<cpx<double>> tw;
    axis_tables(h->n[k], a_tilde, reach, mmax, coef, tw);
    std::vector<float> coef32(coef.begin(), coef.end());
    std::vector<cpx<float>> tw32(tw.size());
    for (size_t i = 0; i < tw.size(); ++i) tw32[i] = cmk((float)tw[i].x, (float)tw[i].y);
    if ((st = h->alloc(&h->coef64[k], coef.size())) || (st = h->alloc(&h->coef32[k], coef.size())) ||
        (st = h->alloc(&h->tw64[k], tw.size())) || (st = h->alloc(&h->tw32[k], tw.size())))
      return bail(st);
    e = cudaMemcpy(h->coef64[k], coef.data(), coef.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->coef32[k], coef32.data(), coef32.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->tw64[k], tw.data(), tw.size() * sizeof(cpx<double>), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->tw32[k], tw32.data(), tw32.size() * sizeof(cpx<float>), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bail(cuda_fail(e, "copy tables"));
  }

  // ---- Alg. 1: moment fields m_gamma = chi (*) prod_k T_{gamma_k}, |gamma| <= 2 deg
  const int D2 = 2 * degree;
  std::vector<std::pair<int, int>> ylist;      // (gx, gy)
  std::vector<std::array<int, 3>> zlist;       // (gx, gy, gz)
  for (int gx = 0; gx <= D2; ++gx)
    for (int gy = 0; gx + gy <= D2 && (dim > 1 || gy == 0); ++gy) ylist.push_back({gx, gy});
  std::vector<int> zbegin;
  for (auto& yg : ylist) {
    zbegin.push_back((int)zlist.size());
    for (int gz = 0; yg.first + yg.second + gz <= (dim == 3 ? D2 : yg.first + yg.second); ++gz)
      zlist.push_back({yg.first, yg.second, gz});
  }
  const int nXm = D2 + 1, nYm = (int)ylist.size(), nZm = (int)zlist.size();
  double* mws = nullptr;
  e = cudaMalloc((void**)&mws, sizeof(double) * (size_t)(1 + nXm + nYm + nZm) * n);
  if (e != cudaSuccess) return bail(cuda_fail(e, "set-up workspace"));
  auto mf = [&](int i) { return mws + (size_t)i * n; };
  auto run_setup = [&]() -> rk_status {
    RK_CK(launch_u8_to_f64(mf(0), h->chi, n, s));
    PassArgs<double> ax = pass_base<double>(h, 0);
    ax.in[0] = mf(0);
    ax.n_groups = 1;
    ax.g_io[0] = 0;
    ax.g_begin[0] = 0;
    for (int m = 0; m < nXm; ++m) {
      ax.out[m] = mf(1 + m);
      ax.term_io[m] = m;
      ax.term_m[m] = m;
    }
    ax.g_begin[1] = nXm;
    RK_TRY(run_split<double>(h, 0, ax, s));
    PassArgs<double> ay = pass_base<double>(h, 1);
    ay.n_groups = nXm;
    int q = 0;
    for (int gx = 0; gx < nXm; ++gx) {
      ay.in[gx] = mf(1 + gx);
      ay.g_io[gx] = gx;
      ay.g_begin[gx] = q;
      for (int yi = 0; yi < nYm; ++yi)
        if (ylist[yi].first == gx) {
          ay.out[yi] = mf(1 + nXm + yi);
          ay.term_io[q] = yi;
          ay.term_m[q] = ylist[yi].second;
          ++q;
        }
    }
    ay.g_begin[nXm] = q;
    if (dim > 1) RK_TRY(run_split<double>(h, 1, ay, s));
    PassArgs<double> az = pass_base<double>(h, 2);
    az.n_groups = nYm;
    q = 0;
    for (int yi = 0; yi < nYm; ++yi) {
      az.in[yi] = mf(1 + nXm + yi);
      az.g_io[yi] = yi;
      az.g_begin[yi] = q;
      for (int zi = zbegin[yi]; zi < (yi + 1 < nYm ? zbegin[yi + 1] : nZm); ++zi) {
        az.out[zi] = mf(1 + nXm + nYm + zi);
        az.term_io[q] = zi;
        az.term_m[q] = zlist[zi][2];
        ++q;
      }
    }
    az.g_begin[nYm] = q;
    // in 2D the y outputs are the moment fields (zlist = ylist with g_z = 0)
    if (dim == 3) RK_TRY(run_split<double>(h, 2, az, s));
    // per-node M^{-1} -> b (Eq. 83-85)
    MomentArgs ma;
    memset(&ma, 0, sizeof(ma));
    // 3D: the z outputs; 2D: the y outputs; 1D: the x outputs (zlist = (g_x, 0, 0) in g_x order)
    ma.mom = dim == 3 ? mf(1 + nXm + nYm) : (dim == 2 ? mf(1 + nXm) : mf(1));
    ma.n_mom = nZm;
    ma.s = h->s;
    ma.dim = dim;
    const Chain& c = h->chain;
    for (int p = 0; p < h->s; ++p)
      for (int qq = 0; qq < h->s; ++qq) {
        int gam[3] = {c.alpha[p][0] + c.alpha[qq][0], c.alpha[p][1] + c.alpha[qq][1], c.alpha[p][2] + c.alpha[qq][2]};
        int idx = -1;
        for (int zi = 0; zi < nZm; ++zi)
          if (zlist[zi][0] == gam[0] && zlist[zi][1] == gam[1] && zlist[zi][2] == gam[2]) idx = zi;
        ma.pq[p][qq] = (signed char)idx;
      }
    ma.chi = h->chi;
    for (int k = 0; k < 3; ++k) ma.inv_a[k] = 1.0 / (a_tilde * h->h[k]);
    ma.V = h->V;
    ma.b64 = h->b64;
    ma.b32 = h->b32;
    ma.chiV64 = h->chiV64;
    ma.chiV32 = h->chiV32;
    ma.nbox = n;
    ma.n_singular = h->counters;
    ma.first_singular = h->counters + 1;
    unsigned long long init[2] = {0ull, ~0ull};
    RK_CK(cudaMemcpyAsync(h->counters, init, sizeof(init), cudaMemcpyHostToDevice, s));
    {
      ProfScope ps(h, prof_cls<double>(RK_PROF_MOMENT_SOLVE), s);
      RK_CK(launch_moment_solve(ma, s));
    }
    unsigned long long res[2];
    RK_CK(cudaMemcpyAsync(res, h->counters, sizeof(res), cudaMemcpyDeviceToHost, s));
    RK_CK(cudaStreamSynchronize(s));
    h->n_singular = (long long)res[0];
    h->first_singular = res[0] ? (long long)res[1] : -1;
    return RK_OK;
  };
  st = run_setup();
  cudaFree(mws);
  if (st != RK_OK) return bail(st);
  if ((st = compress_coefficients(h, s)) != RK_OK) return bail(st);
  if ((st = scale_regular_rows(h, s)) != RK_OK) return bail(st);
  if ((st = build_zwindows(h, s)) != RK_OK) return bail(st);
  *out = h;
  if (h->n_singular)
    return fail(RK_ERR_SINGULAR_MOMENT,
                std::to_string(h->n_singular) + " singular moment matrices, first at " + std::to_string(h->first_singular));
  return RK_OK;
}

rk_status rk_clone(const rk_handle* parent, rk_handle** out) {
  if (!parent || !out) return fail(RK_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  rk_handle* h = new rk_handle(*parent);
  h->owned.clear();
  h->ev_pool.clear();
  h->pend.clear();
  h->prof_on = false;
  for (int c = 0; c < 2 * RK_PROF_CLASSES; ++c) {
    h->prof_ms[c] = 0.0;
    h->prof_n[c] = 0;
  }
  h->parent = parent->parent ? parent->parent : parent;
  h->ws64 = nullptr;
  h->ws32 = nullptr;
  h->sv64 = nullptr;
  h->sv32 = nullptr;
  h->partials = nullptr;
  h->xpartials = nullptr;
  h->counters2 = nullptr;
  h->dscal = nullptr;
  h->cg = nullptr;
  h->hscal = nullptr;
  for (auto& st : h->stage) st = nullptr;
  h->bstream = nullptr;
  h->bevent = nullptr;
  h->chunk_graph = nullptr;
  h->chunk_len = 0;
  h->err_host = nullptr;
  h->err_dev = nullptr;
  h->spec32 = nullptr;
  h->spec64 = nullptr;
  h->trans64 = nullptr;
  h->trans32 = nullptr;
  h->part2 = nullptr;
  h->mlumped = nullptr;
  for (int k = 0; k < 2; ++k) {
    h->tmaps32[k].clear();
    h->tmaps64[k].clear();
  }
  rk_status st;
  if ((st = h->alloc(&h->ws64, (size_t)ws_fields(h->chain) * h->nbox)) != RK_OK ||
      (st = h->alloc(&h->ws32, (size_t)ws_fields(h->chain) * h->nbox)) != RK_OK || (st = setup_tma(h)) != RK_OK) {
    rk_destroy(h);
    return st;
  }
  *out = h;
  return RK_OK;
}

rk_status rk_solve_batched(const rk_batch_item* items, int32_t n_items, const rk_solve_opts* opts,
                           rk_solve_info* infos, void* stream) {
  if (!items || n_items < 1) return fail(RK_ERR_INVALID_ARG, "no items");
  rk_solve_opts o;
  if (opts)
    o = *opts;
  else
    fill_defaults(&o);
  o.x0_given = 0;
  RK_TRY(check_opts(o));
  if (o.precision != RK_PREC_MIXED) return fail(RK_ERR_UNSUPPORTED, "batched solves run in mixed precision");
  for (int i = 0; i < n_items; ++i) {
    if (!items[i].h || !items[i].r || !items[i].d) return fail(RK_ERR_INVALID_ARG, "NULL item field");
    for (int k = 0; k < i; ++k)
      if (items[k].h == items[i].h) return fail(RK_ERR_INVALID_ARG, "items must use distinct handles (see rk_clone)");
  }
  cudaStream_t s = (cudaStream_t)stream;
  auto t0 = std::chrono::steady_clock::now();
  std::vector<rk_solve_info> inf((size_t)n_items);
  std::vector<MixedJob> jobs((size_t)n_items);
  std::vector<Staged> sd((size_t)n_items), su((size_t)n_items);
  cudaEvent_t fork = nullptr;
  RK_CK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
  RK_CK(cudaEventRecord(fork, s));
  rk_status first_err = RK_OK;
  for (int i = 0; i < n_items; ++i) {
    rk_handle* h = items[i].h;
    memset(&inf[i], 0, sizeof(rk_solve_info));
    RK_TRY(ensure_solver(h));
    if (!h->bstream) RK_CK(cudaStreamCreateWithFlags(&h->bstream, cudaStreamNonBlocking));
    if (!h->bevent) RK_CK(cudaEventCreateWithFlags(&h->bevent, cudaEventDisableTiming));
    RK_CK(cudaStreamWaitEvent(h->bstream, fork, 0));
    const size_t bytes = (size_t)h->nbox * 8;
    Staged sr, sg;
    RK_TRY(stage_in(h, 0, items[i].r, bytes, h->bstream, &sr));
    RK_TRY(stage_in(h, 1, items[i].g, bytes, h->bstream, &sg));
    RK_TRY(stage_out_prepare(h, 2, items[i].d, bytes, &sd[i]));
    RK_TRY(stage_out_prepare(h, 3, items[i].u, bytes, &su[i]));
    rk_status st = prepare_mixed_job(h, (const double*)sr.dev, (const double*)sg.dev, o, &inf[i], h->bstream, jobs[i]);
    if (st != RK_OK) {
      jobs[i].done = true;
      inf[i].status = st;
      if (first_err == RK_OK) first_err = st;
    }
  }
  // all jobs advance together: issue a chunk on every active stream, then check each
  for (;;) {
    bool any = false;
    for (auto& j : jobs)
      if (!j.done) {
        any = true;
        RK_TRY(mixed_issue(j));
      }
    if (!any) break;
    for (int i = 0; i < n_items; ++i)
      if (!jobs[i].done) RK_TRY(mixed_check(jobs[i]));
  }
  for (auto& j : jobs)
    if (j.h && inf[&j - jobs.data()].status == RK_OK) {
      rk_status st = mixed_finish(j);
      if (st != RK_OK) inf[&j - jobs.data()].status = st;
    }
  for (int i = 0; i < n_items; ++i) {
    rk_handle* h = items[i].h;
    MixedJob& j = jobs[i];
    inf[i].iterations = j.it;
    inf[i].rel_residual = j.fn > 0.0 ? j.rn / j.fn : 0.0;
    if (inf[i].status == RK_OK && !(j.rn <= j.target)) inf[i].status = RK_ERR_NOT_CONVERGED;
    RK_CK(launch_add((double*)sd[i].dev, h->v64(5), h->v64(0), h->nbox, h->bstream));
    if (su[i].dev) RK_TRY(op_U<double>(h, (const double*)sd[i].dev, (double*)su[i].dev, h->bstream));
    RK_TRY(stage_out_finish(sd[i], h->bstream));
    RK_TRY(stage_out_finish(su[i], h->bstream));
    RK_CK(cudaEventRecord(h->bevent, h->bstream));
    RK_CK(cudaStreamWaitEvent(s, h->bevent, 0));
    if (first_err == RK_OK && inf[i].status != RK_OK) first_err = (rk_status)inf[i].status;
  }
  RK_CK(cudaStreamSynchronize(s));
  cudaEventDestroy(fork);
  for (int i = 0; i < n_items; ++i)
    if (check_device_flag(items[i].h) != RK_OK && inf[i].status == RK_OK) {
      inf[i].status = RK_ERR_TIMEOUT;
      if (first_err == RK_OK) first_err = RK_ERR_TIMEOUT;
    }
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  for (int i = 0; i < n_items; ++i) {
    inf[i].solve_ms = ms;
    if (infos) infos[i] = inf[i];
  }
  if (first_err != RK_OK) return fail(first_err, "at least one batched solve failed (see infos)");
  return RK_OK;
}

rk_status rk_singular_nodes(const rk_handle* h, int64_t* count, int64_t* first) {
  if (!h) return fail(RK_ERR_INVALID_ARG, "handle is NULL");
  if (count) *count = h->n_singular;
  if (first) *first = h->first_singular;
  return RK_OK;
}

rk_status rk_get_shape(const rk_handle* h, int32_t n[3], int32_t* s, int64_t* n_omega) {
  if (!h) return fail(RK_ERR_INVALID_ARG, "handle is NULL");
  if (n)
    for (int k = 0; k < 3; ++k) n[k] = h->n[k];
  if (s) *s = h->s;
  if (n_omega) *n_omega = h->n_omega;
  return RK_OK;
}

rk_status rk_apply_K(rk_handle* h, const void* d, void* f, int32_t dtype, void* stream) {
  if (!h || !d || !f) return fail(RK_ERR_INVALID_ARG, "NULL argument");
  if (dtype != RK_F64 && dtype != RK_F32) return fail(RK_ERR_INVALID_ARG, "bad dtype");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)h->nbox * (dtype == RK_F64 ? 8 : 4);
  Staged sd, sf;
  RK_TRY(stage_in(h, 0, d, bytes, s, &sd));
  RK_TRY(stage_out_prepare(h, 1, f, bytes, &sf));
  if (dtype == RK_F64)
    RK_TRY(op_K<double>(h, (const double*)sd.dev, (double*)sf.dev, h->chi, h->chi, s));
  else
    RK_TRY(op_K<float>(h, (const float*)sd.dev, (float*)sf.dev, h->chi, h->chi, s));
  RK_TRY(stage_out_finish(sf, s));
  if (any_host({&sd, &sf})) {
    RK_CK(cudaStreamSynchronize(s));
    RK_TRY(check_device_flag(h));
  }
  return RK_OK;
}

rk_status rk_debug_short_waits(rk_handle* h, int32_t enable) {
  if (!h) return fail(RK_ERR_INVALID_ARG, "handle is NULL");
  if (enable != 0 && enable != 1) return fail(RK_ERR_INVALID_ARG, "enable must be 0 or 1");
  h->short_wait = enable;
  // a captured chunk of CG iterations holds the pass arguments it was captured with
  if (h->chunk_graph) cudaGraphExecDestroy(h->chunk_graph);
  h->chunk_graph = nullptr;
  h->chunk_len = 0;
  return RK_OK;
}

rk_status rk_apply_precond(rk_handle* h, const void* r, void* z, int32_t dtype, void* stream) {
  if (!h || !r || !z) return fail(RK_ERR_INVALID_ARG, "NULL argument");
  if (dtype != RK_F64 && dtype != RK_F32) return fail(RK_ERR_INVALID_ARG, "bad dtype");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)h->nbox * (dtype == RK_F64 ? 8 : 4);
  RK_TRY(ensure_solver(h));
  Staged sr, sz;
  RK_TRY(stage_in(h, 0, r, bytes, s, &sr));
  RK_TRY(stage_out_prepare(h, 1, z, bytes, &sz));
  if (dtype == RK_F64)
    RK_TRY(apply_precond<double>(h, (const double*)sr.dev, (double*)sz.dev, s, -1));
  else
    RK_TRY(apply_precond<float>(h, (const float*)sr.dev, (float*)sz.dev, s, -1));
  RK_TRY(stage_out_finish(sz, s));
  if (any_host({&sr, &sz})) RK_CK(cudaStreamSynchronize(s));
  return RK_OK;
}

rk_status rk_rhs(rk_handle* h, const double* r, double* fr, void* stream) {
  if (!h || !r || !fr) return fail(RK_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)h->nbox * 8;
  Staged a, b;
  RK_TRY(stage_in(h, 0, r, bytes, s, &a));
  RK_TRY(stage_out_prepare(h, 1, fr, bytes, &b));
  RK_TRY(op_UT<double>(h, (const double*)a.dev, (double*)b.dev, h->chiV64, nullptr, s));
  RK_TRY(stage_out_finish(b, s));
  if (any_host({&a, &b})) RK_CK(cudaStreamSynchronize(s));
  return RK_OK;
}

rk_status rk_eval_u(rk_handle* h, const double* d, double* u, void* stream) {
  if (!h || !d || !u) return fail(RK_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)h->nbox * 8;
  Staged a, b;
  RK_TRY(stage_in(h, 0, d, bytes, s, &a));
  RK_TRY(stage_out_prepare(h, 1, u, bytes, &b));
  RK_TRY(op_U<double>(h, (const double*)a.dev, (double*)b.dev, s));
  RK_TRY(stage_out_finish(b, s));
  if (any_host({&a, &b})) RK_CK(cudaStreamSynchronize(s));
  return RK_OK;
}

rk_status rk_eval_u_transpose(rk_handle* h, const double* ev, double* w, void* stream) {
  if (!h || !ev || !w) return fail(RK_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)h->nbox * 8;
  Staged a, b;
  RK_TRY(stage_in(h, 0, ev, bytes, s, &a));
  RK_TRY(stage_out_prepare(h, 1, w, bytes, &b));
  RK_TRY(op_UT<double>(h, (const double*)a.dev, (double*)b.dev, nullptr, h->chi, s));
  RK_TRY(stage_out_finish(b, s));
  if (any_host({&a, &b})) RK_CK(cudaStreamSynchronize(s));
  return RK_OK;
}

rk_status rk_get_b(rk_handle* h, double* b, void* stream) {
  if (!h || !b) return fail(RK_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  RK_CK(cudaMemcpyAsync(b, h->b64, sizeof(double) * (size_t)4 * h->s * h->nbox, cudaMemcpyDefault, s));
  if (!is_device_ptr(b)) RK_CK(cudaStreamSynchronize(s));
  return RK_OK;
}

}  // extern "C"

namespace {
// rk_solve and rk_solve_neumann: Alg. 5 with optional Neumann data (q, A)
rk_status solve_entry(rk_handle* h, const double* r, const double* g, const double* q, const double* A, double* d,
                      double* u, const rk_solve_opts* opts, rk_solve_info* info, void* stream) {
  if (!h || !r || !d) return fail(RK_ERR_INVALID_ARG, "NULL argument");
  rk_solve_opts o;
  if (opts)
    o = *opts;
  else
    fill_defaults(&o);
  RK_TRY(check_opts(o));
  rk_solve_info inf;
  memset(&inf, 0, sizeof(inf));
  cudaStream_t s = (cudaStream_t)stream;
  RK_TRY(ensure_solver(h));
  auto t0 = std::chrono::steady_clock::now();
  const size_t bytes = (size_t)h->nbox * 8;
  Staged sr, sg, sd, su;
  RK_TRY(stage_in(h, 0, r, bytes, s, &sr));
  RK_TRY(stage_in(h, 1, g, bytes, s, &sg));
  if (o.x0_given)
    RK_TRY(stage_in(h, 2, d, bytes, s, &sd));
  else
    RK_TRY(stage_out_prepare(h, 2, d, bytes, &sd));
  RK_TRY(stage_out_prepare(h, 3, u, bytes, &su));
  Staged sq, sa;
  RK_TRY(stage_in(h, 4, q, bytes, s, &sq));
  RK_TRY(stage_in(h, 5, A, bytes, s, &sa));
  rk_status st = forward_solve(h, (const double*)sr.dev, (const double*)sg.dev, (double*)sd.dev, o, &inf, s,
                               (const double*)sq.dev, (const double*)sa.dev);
  if (st == RK_OK || st == RK_ERR_NOT_CONVERGED || st == RK_ERR_BREAKDOWN) {
    if (su.dev) RK_TRY(op_U<double>(h, (const double*)sd.dev, (double*)su.dev, s));
    RK_TRY(stage_out_finish(sd, s));
    RK_TRY(stage_out_finish(su, s));
  }
  RK_CK(cudaStreamSynchronize(s));
  inf.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  inf.status = st;
  if (info) *info = inf;
  return st;
}
}  // namespace

extern "C" {

rk_status rk_solve(rk_handle* h, const double* r, const double* g, double* d, double* u, const rk_solve_opts* opts,
                   rk_solve_info* info, void* stream) {
  return solve_entry(h, r, g, nullptr, nullptr, d, u, opts, info, stream);
}

rk_status rk_solve_neumann(rk_handle* h, const double* r, const double* g, const double* q, const double* A, double* d,
                           double* u, const rk_solve_opts* opts, rk_solve_info* info, void* stream) {
  if (!q || !A) return fail(RK_ERR_INVALID_ARG, "NULL Neumann data");
  return solve_entry(h, r, g, q, A, d, u, opts, info, stream);
}

rk_status rk_apply_M(rk_handle* h, const void* v, void* fm, int32_t dtype, void* stream) {
  if (!h || !v || !fm) return fail(RK_ERR_INVALID_ARG, "NULL argument");
  if (dtype != RK_F64 && dtype != RK_F32) return fail(RK_ERR_INVALID_ARG, "bad dtype");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)h->nbox * (dtype == RK_F64 ? 8 : 4);
  Staged sv, sf;
  RK_TRY(stage_in(h, 0, v, bytes, s, &sv));
  RK_TRY(stage_out_prepare(h, 1, fm, bytes, &sf));
  if (dtype == RK_F64)
    RK_TRY(op_M<double>(h, (const double*)sv.dev, (double*)sf.dev, s));
  else
    RK_TRY(op_M<float>(h, (const float*)sv.dev, (float*)sf.dev, s));
  RK_TRY(stage_out_finish(sf, s));
  if (any_host({&sv, &sf})) RK_CK(cudaStreamSynchronize(s));
  return RK_OK;
}

rk_status rk_lumped_mass(rk_handle* h, double* ml, void* stream) {
  if (!h || !ml) return fail(RK_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  Staged sm;
  RK_TRY(stage_out_prepare(h, 1, ml, (size_t)h->nbox * 8, &sm));
  RK_TRY(lumped_mass(h, (double*)sm.dev, s));
  RK_TRY(stage_out_finish(sm, s));
  if (sm.host) RK_CK(cudaStreamSynchronize(s));
  return RK_OK;
}

rk_status rk_transient_explicit(rk_handle* h, const double* f, const double* g, double dt, int32_t n_steps, double* d,
                                void* stream) {
  if (!h || !f || !d || n_steps < 0 || !(dt > 0.0)) return fail(RK_ERR_INVALID_ARG, "bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)h->nbox * 8;
  Staged sf, sg, sd;
  RK_TRY(stage_in(h, 0, f, bytes, s, &sf));
  RK_TRY(stage_in(h, 1, g, bytes, s, &sg));
  RK_TRY(stage_in(h, 2, d, bytes, s, &sd));
  RK_TRY(transient_explicit(h, (const double*)sf.dev, (const double*)sg.dev, dt, n_steps, (double*)sd.dev, s));
  RK_TRY(stage_out_finish(sd, s));
  if (any_host({&sf, &sg, &sd})) RK_CK(cudaStreamSynchronize(s));
  return RK_OK;
}

rk_status rk_transient_implicit(rk_handle* h, const double* f, const double* g, double dt, int32_t n_steps, double* d,
                                const rk_solve_opts* opts, rk_solve_info* info, void* stream) {
  if (!h || !f || !d || n_steps < 0 || !(dt > 0.0)) return fail(RK_ERR_INVALID_ARG, "bad argument");
  rk_solve_opts o;
  if (opts)
    o = *opts;
  else
    fill_defaults(&o);
  RK_TRY(check_opts(o));
  rk_solve_info inf;
  memset(&inf, 0, sizeof(inf));
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)h->nbox * 8;
  Staged sf, sg, sd;
  RK_TRY(stage_in(h, 0, f, bytes, s, &sf));
  RK_TRY(stage_in(h, 1, g, bytes, s, &sg));
  RK_TRY(stage_in(h, 2, d, bytes, s, &sd));
  rk_status st = transient_implicit(h, (const double*)sf.dev, (const double*)sg.dev, dt, n_steps, (double*)sd.dev, o,
                                    &inf, s);
  if (st == RK_OK) RK_TRY(stage_out_finish(sd, s));
  RK_CK(cudaStreamSynchronize(s));
  inf.status = st;
  if (info) *info = inf;
  return st;
}

rk_status rk_nonlinear_force(rk_handle* h, const double* d, int32_t kind, double c, double* fN, void* stream) {
  if (!h || !d || !fN || kind < RK_NL_CUBIC || kind > RK_NL_EXP) return fail(RK_ERR_INVALID_ARG, "bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)h->nbox * 8;
  Staged sd, sf;
  RK_TRY(stage_in(h, 0, d, bytes, s, &sd));
  RK_TRY(stage_out_prepare(h, 1, fN, bytes, &sf));
  RK_TRY(nonlinear_force(h, (const double*)sd.dev, kind, c, (double*)sf.dev, s));
  RK_TRY(stage_out_finish(sf, s));
  if (any_host({&sd, &sf})) RK_CK(cudaStreamSynchronize(s));
  return RK_OK;
}

rk_status rk_solve_penalty(rk_handle* h, const double* r, const double* g, const double* A, double beta, double* d,
                           double* u, const rk_solve_opts* opts, rk_solve_info* info, void* stream) {
  if (!h || !r || !g || !A || !d || !(beta > 0.0) || !std::isfinite(beta)) return fail(RK_ERR_INVALID_ARG, "bad argument");
  rk_solve_opts o;
  if (opts)
    o = *opts;
  else
    fill_defaults(&o);
  RK_TRY(check_opts(o));
  rk_solve_info inf;
  memset(&inf, 0, sizeof(inf));
  cudaStream_t s = (cudaStream_t)stream;
  auto t0 = std::chrono::steady_clock::now();
  const size_t bytes = (size_t)h->nbox * 8;
  RK_TRY(ensure_solver(h));
  Staged sr, sg, sa, sd, su;
  RK_TRY(stage_in(h, 0, r, bytes, s, &sr));
  RK_TRY(stage_in(h, 1, g, bytes, s, &sg));
  RK_TRY(stage_in(h, 2, A, bytes, s, &sa));
  RK_TRY(stage_out_prepare(h, 3, d, bytes, &sd));
  rk_status st = solve_penalty(h, (const double*)sr.dev, (const double*)sg.dev, (const double*)sa.dev, beta,
                               (double*)sd.dev, o, &inf, s);
  if (st == RK_OK || st == RK_ERR_NOT_CONVERGED) {
    RK_TRY(stage_out_finish(sd, s));
    if (u) {
      RK_TRY(stage_out_prepare(h, 4, u, bytes, &su));
      RK_TRY(op_U<double>(h, (const double*)sd.dev, (double*)su.dev, s));
      RK_TRY(stage_out_finish(su, s));
    }
  }
  RK_CK(cudaStreamSynchronize(s));
  RK_TRY(check_device_flag(h));
  inf.status = st;
  inf.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = inf;
  return st;
}

rk_status rk_nonlinear_grad_force(rk_handle* h, const double* d, int32_t kind, double c, const double* a,
                                  double* fN, void* stream) {
  if (!h || !d || !a || !fN || kind < RK_NL_CUBIC || kind > RK_NL_EXP) return fail(RK_ERR_INVALID_ARG, "bad argument");
  const double av[3] = {a[0], h->dim > 1 ? a[1] : 0.0, h->dim == 3 ? a[2] : 0.0};
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)h->nbox * 8;
  Staged sd, sf;
  RK_TRY(stage_in(h, 0, d, bytes, s, &sd));
  RK_TRY(stage_out_prepare(h, 1, fN, bytes, &sf));
  RK_TRY(nonlinear_grad_force(h, (const double*)sd.dev, kind, c, av, (double*)sf.dev, s));
  RK_TRY(stage_out_finish(sf, s));
  if (any_host({&sd, &sf})) RK_CK(cudaStreamSynchronize(s));
  return RK_OK;
}

rk_status rk_solve_nonlinear(rk_handle* h, const double* r, const double* g, int32_t kind, double c, double* d,
                             double* u, const rk_solve_opts* opts, rk_solve_info* info, void* stream) {
  if (!h || !r || !d || kind < RK_NL_CUBIC || kind > RK_NL_EXP || !(c >= 0.0))
    return fail(RK_ERR_INVALID_ARG, "bad argument");
  rk_solve_opts o;
  if (opts)
    o = *opts;
  else
    fill_defaults(&o);
  RK_TRY(check_opts(o));
  rk_solve_info inf;
  memset(&inf, 0, sizeof(inf));
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)h->nbox * 8;
  auto t0 = std::chrono::steady_clock::now();
  Staged sr, sg, sd, su;
  RK_TRY(stage_in(h, 0, r, bytes, s, &sr));
  RK_TRY(stage_in(h, 1, g, bytes, s, &sg));
  RK_TRY(stage_out_prepare(h, 2, d, bytes, &sd));
  RK_TRY(stage_out_prepare(h, 3, u, bytes, &su));
  rk_status st = solve_nonlinear(h, (const double*)sr.dev, (const double*)sg.dev, kind, c, (double*)sd.dev, o, &inf, s);
  if (st == RK_OK || st == RK_ERR_NOT_CONVERGED) {
    if (su.dev) RK_TRY(op_U<double>(h, (const double*)sd.dev, (double*)su.dev, s));
    RK_TRY(stage_out_finish(sd, s));
    RK_TRY(stage_out_finish(su, s));
  }
  RK_CK(cudaStreamSynchronize(s));
  inf.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  inf.status = st;
  if (info) *info = inf;
  return st;
}

rk_status rk_boundary_rhs(rk_handle* h, const double* q, const double* A, double* fq, void* stream) {
  if (!h || !q || !A || !fq) return fail(RK_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)h->nbox * 8;
  Staged sq, sa, sf;
  RK_TRY(stage_in(h, 0, q, bytes, s, &sq));
  RK_TRY(stage_in(h, 1, A, bytes, s, &sa));
  RK_TRY(stage_out_prepare(h, 2, fq, bytes, &sf));
  RK_TRY(boundary_rhs(h, (const double*)sq.dev, (const double*)sa.dev, (double*)sf.dev, s));
  RK_TRY(stage_out_finish(sf, s));
  if (any_host({&sq, &sa, &sf})) RK_CK(cudaStreamSynchronize(s));
  return RK_OK;
}

rk_status rk_solve_adjoint(rk_handle* h, const double* r, const double* g, const double* u_target, double* dJ_dr,
                           double* dJ_dg, double* J, const rk_solve_opts* opts, rk_solve_info* info, void* stream) {
  if (!h || !r || !u_target || !dJ_dr || !dJ_dg) return fail(RK_ERR_INVALID_ARG, "NULL argument");
  rk_solve_opts o;
  if (opts)
    o = *opts;
  else
    fill_defaults(&o);
  o.x0_given = 0;
  RK_TRY(check_opts(o));
  rk_solve_info inf;
  memset(&inf, 0, sizeof(inf));
  cudaStream_t s = (cudaStream_t)stream;
  RK_TRY(ensure_solver(h));
  auto t0 = std::chrono::steady_clock::now();
  const long long n = h->nbox;
  const size_t bytes = (size_t)n * 8;
  Staged sr, sg, sut, sdr, sdg;
  RK_TRY(stage_in(h, 0, r, bytes, s, &sr));
  RK_TRY(stage_in(h, 1, g, bytes, s, &sg));
  RK_TRY(stage_in(h, 2, u_target, bytes, s, &sut));
  RK_TRY(stage_out_prepare(h, 3, dJ_dr, bytes, &sdr));
  RK_TRY(stage_out_prepare(h, 4, dJ_dg, bytes, &sdg));
  double* dvec = h->v64(7);
  double* uvec = (double*)sdr.dev;  // scratch until dJ/dr is written
  double* e = (double*)sdg.dev;     // scratch until dJ/dg is written
  // forward solve (recomputed from r, g)
  rk_status st = forward_solve(h, (const double*)sr.dev, (const double*)sg.dev, dvec, o, &inf, s);
  if (st != RK_OK) {
    inf.status = st;
    if (info) *info = inf;
    return st;
  }
  RK_TRY(op_U<double>(h, dvec, uvec, s));
  // e = chi o (u - u_target); J = 1/2 e.e
  RK_CK(launch_sub(e, uvec, (const double*)sut.dev, n, s));
  RK_CK(launch_mask(e, e, h->chi, n, s));
  double ee;
  RK_CK(launch_dot<double, double>(e, e, n, h->partials, h->dscal, s));
  RK_TRY(read_scalar(h, h->dscal, &ee, s));
  if (J) *J = 0.5 * ee;
  st = vjp_core(h, e, uvec, e, o, &inf, s);
  if (st != RK_OK) {
    inf.status = st;
    if (info) *info = inf;
    return st;
  }
  RK_TRY(stage_out_finish(sdr, s));
  RK_TRY(stage_out_finish(sdg, s));
  RK_CK(cudaStreamSynchronize(s));
  inf.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  inf.status = RK_OK;
  if (info) *info = inf;
  return RK_OK;
}

rk_status rk_solve_vjp(rk_handle* h, const double* u_bar, double* r_bar, double* g_bar, const rk_solve_opts* opts,
                       rk_solve_info* info, void* stream) {
  if (!h || !u_bar || !r_bar || !g_bar) return fail(RK_ERR_INVALID_ARG, "NULL argument");
  rk_solve_opts o;
  if (opts)
    o = *opts;
  else
    fill_defaults(&o);
  o.x0_given = 0;
  RK_TRY(check_opts(o));
  rk_solve_info inf;
  memset(&inf, 0, sizeof(inf));
  cudaStream_t s = (cudaStream_t)stream;
  RK_TRY(ensure_solver(h));
  auto t0 = std::chrono::steady_clock::now();
  const long long n = h->nbox;
  const size_t bytes = (size_t)n * 8;
  Staged su, sr, sg;
  RK_TRY(stage_in(h, 0, u_bar, bytes, s, &su));
  RK_TRY(stage_out_prepare(h, 3, r_bar, bytes, &sr));
  RK_TRY(stage_out_prepare(h, 4, g_bar, bytes, &sg));
  double* e = h->v64(7);
  RK_CK(launch_mask(e, (const double*)su.dev, h->chi, n, s));
  rk_status st = vjp_core(h, e, (double*)sr.dev, (double*)sg.dev, o, &inf, s);
  if (st == RK_OK) {
    RK_TRY(stage_out_finish(sr, s));
    RK_TRY(stage_out_finish(sg, s));
  }
  RK_CK(cudaStreamSynchronize(s));
  inf.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  inf.status = st;
  if (info) *info = inf;
  return st;
}

}  // extern "C"
