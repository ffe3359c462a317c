// rk_precond.cuh -- spectral preconditioner for the CG solve of Alg. 5 (an
// addition to the paper's plain CG, selected by rk_solve_opts.precond).
//
// M^{-1} r = chi_Omega o F^{-1}[ F(r) / lam~ ],  lam~(theta) = lam(theta) + shift,
// where lam is the symbol of the operator at regular nodes (whole support in chi,
// interior V): with the separable kernel tables T_m of each axis and the
// interior correction coefficients b^k_p,
//   D^_k(theta) = sum_p b^k_p  prod_axis T^_{alpha_axis(p)}(theta_axis)   (Eq. 44, 77)
//   lam(theta)  = V sum_k |D^_k(theta)|^2                                  (Eq. 26, DNI)
// i.e. K restricted to a periodic box full of regular nodes is the convolution
// whose eigenvalues are lam.  shift keeps the constant mode invertible.
//
// The 3D real FFT is done in five passes over one half spectrum S (complex,
// x frequencies 0..n_x/2 padded to an even row pitch):
//   x R2C   two real rows are one complex line; after the line FFT the two
//           spectra are separated with the Hermitian symmetry;
//   y FWD   complex lines along y, spectra stored at their frequency rows;
//   z SYM   complex lines along z: forward, times 1/(lam~ n_x n_y n_z), inverse;
//   y INV   frequency rows back to y;
//   x C2R   Hermitian completion of each row pair, inverse line FFT, chi_Omega
//           mask, and (inside CG) the product r.z with beta of the next step.
#pragma once

#include "rk_passes.cuh"

namespace rk {

enum PfftMode { PF_FWD = 0, PF_SYM = 1, PF_INV = 2 };

template <typename T>
struct SymbolArgs {
  const T* cx;       // [deg+1][n_x]: real factor of T^_m at each x frequency
  const T* cy;       // [deg+1][n_y]
  const T* cz;       // [deg+1][n_z]
  int n[3];
  int s;
  int alpha[10][3];  // basis exponents
  int imag[10];      // 1 when i^(odd exponents of p) is imaginary (T^_m is imaginary for odd m)
  T sgn[10];         // the sign of that power of i
  T b[3][10];        // b^x_p, b^y_p, b^z_p of a regular node
  T vreg;            // V of a regular node
  T shift;           // added to lam
  T scale;           // 1 / (n_x n_y n_z)
};

template <typename T>
struct PxArgs {
  const T* in;               // R2C: real field
  T* out;                    // C2R: real field
  cpx<T>* S;                 // half spectrum, rows of pitch nxp
  int nxp;
  const uint8_t* out_mask;   // C2R: chi_Omega (may be null)
  const cpx<T>* tw;          // x twiddles
  int nx, ny, nz;
  // C2R epilogue inside PCG: rz_new = r . z, then beta = rz_new / rz_prev, rz = rz_new.
  //   mode 0 (after an iteration): rz_prev = rz first;  2 (start): beta = 0,
  //   rz_prev = rz = rz_new.
  const T* cg_r;
  CGState* cg;
  double* partials;
  unsigned* counter;
  int rz_mode;
};

template <typename T>
struct PfftArgs {
  cpx<T>* S;                 // in place
  int ncols;                 // complex columns per row (nxp)
  long long line_stride;     // in complex elements
  long long other_stride;
  int nother;                // lines of the other axis
  const cpx<T>* tw;
  const T* mult;             // z SYM: 1 / (lam~ n_x n_y n_z) at [kz][ky][kx], rows of nxp
};

// lam~ (theta) at integer frequencies (kx, ky, kz), in FP64
RK_HD double symbol_value(const SymbolArgs<double>& y, int kx, int ky, int kz) {
  double R[3] = {0.0, 0.0, 0.0}, I[3] = {0.0, 0.0, 0.0};
  for (int p = 0; p < y.s; ++p) {
    const double f = y.sgn[p] * y.cx[y.alpha[p][0] * y.n[0] + kx] * y.cy[y.alpha[p][1] * y.n[1] + ky] *
                     y.cz[y.alpha[p][2] * y.n[2] + kz];
    for (int k = 0; k < 3; ++k) {
      if (y.imag[p])
        I[k] += y.b[k][p] * f;
      else
        R[k] += y.b[k][p] * f;
    }
  }
  return y.vreg * (R[0] * R[0] + I[0] * I[0] + R[1] * R[1] + I[1] * I[1] + R[2] * R[2] + I[2] * I[2]) + y.shift;
}

// ---------------------------------------------------------------- x R2C / C2R
template <typename T, int N, int LX>
__global__ void __launch_bounds__(XPass<T, N, LX>::THREADS) k_px_r2c(const PxArgs<T> a) {
  using X = XPass<T, N, LX>;
  using F = typename X::F;
  RK_DYN_SMEM(cpx<T>, sm);
  const int t = threadIdx.x % X::P, l = threadIdx.x / X::P;
  const long long q = (long long)blockIdx.x * LX + l;
  const long long npairs = ((long long)a.ny * a.nz) / 2;
  const bool ok = q < npairs;
  typename X::B buf{sm + (size_t)l * X::B::SIZE};
  cpx<T> v[X::R];
#pragma unroll
  for (int r = 0; r < X::R; ++r) {
    const int xp = F::nat_pos(t, r);
    v[r] = ok ? cmk(RK_LDG(a.in + 2 * q * N + xp), RK_LDG(a.in + (2 * q + 1) * N + xp)) : cmk((T)0, (T)0);
  }
  F::forward(v, t, buf, a.tw);
  // the spectrum Z = A + iB of the row pair in natural order, then A, B separated
  cpx<T>* z = sm + (size_t)l * X::B::SIZE;
  RK_SYNC();
#pragma unroll
  for (int r = 0; r < X::R; ++r) z[F::spec_idx(t, r)] = v[r];
  RK_SYNC();
  if (ok) {
    cpx<T>* s0 = a.S + (2 * q) * (long long)a.nxp;
    cpx<T>* s1 = s0 + a.nxp;
    for (int k = t; k < a.nxp; k += X::P) {
      cpx<T> A = cmk((T)0, (T)0), B = cmk((T)0, (T)0);
      if (k <= N / 2) {
        const cpx<T> zk = z[k], zm = z[(N - k) % N];
        A = cmk((T)0.5 * (zk.x + zm.x), (T)0.5 * (zk.y - zm.y));
        B = cmk((T)0.5 * (zk.y + zm.y), (T)0.5 * (zm.x - zk.x));
      }
      s0[k] = A;
      s1[k] = B;
    }
  }
}

template <typename T, int N, int LX>
__global__ void __launch_bounds__(XPass<T, N, LX>::THREADS) k_px_c2r(const PxArgs<T> a) {
  using X = XPass<T, N, LX>;
  using F = typename X::F;
  RK_DYN_SMEM(cpx<T>, sm);
  const int t = threadIdx.x % X::P, l = threadIdx.x / X::P;
  const long long q = (long long)blockIdx.x * LX + l;
  const long long npairs = ((long long)a.ny * a.nz) / 2;
  const bool ok = q < npairs;
  const long long r0 = 2 * q * N, r1 = r0 + N;
  typename X::B buf{sm + (size_t)l * X::B::SIZE};
  cpx<T> v[X::R];
  const cpx<T>* s0 = a.S + (2 * q) * (long long)a.nxp;
  const cpx<T>* s1 = s0 + a.nxp;
#pragma unroll
  for (int r = 0; r < X::R; ++r) {
    const int k = F::spec_idx(t, r);
    cpx<T> A = cmk((T)0, (T)0), B = cmk((T)0, (T)0);
    if (ok) {
      if (k <= N / 2) {
        A = s0[k];
        B = s1[k];
      } else {
        const cpx<T> a0 = s0[N - k], b0 = s1[N - k];
        A = cmk(a0.x, -a0.y);
        B = cmk(b0.x, -b0.y);
      }
    }
    v[r] = cmk(A.x - B.y, A.y + B.x);  // Z = A + iB
  }
  F::inverse(v, t, buf, a.tw);
  if (ok)
#pragma unroll
    for (int r = 0; r < X::R; ++r) {
      const int xp = F::nat_pos(t, r);
      const T m0 = a.out_mask ? (T)RK_LDG(a.out_mask + r0 + xp) : (T)1;
      const T m1 = a.out_mask ? (T)RK_LDG(a.out_mask + r1 + xp) : (T)1;
      v[r] = cmk(v[r].x * m0, v[r].y * m1);
      a.out[r0 + xp] = v[r].x;
      a.out[r1 + xp] = v[r].y;
    }
  if (a.cg) {
    DotAccPair<T> dot;
    if (ok)
#pragma unroll
      for (int r = 0; r < X::R; ++r) {
        const int xp = F::nat_pos(t, r);
        dot.add(cmk(a.cg_r[r0 + xp], a.cg_r[r1 + xp]), v[r]);
      }
    // fixed-order block and grid reduction as in cg_pap_reduce
    constexpr int THREADS = X::THREADS;
    constexpr int POW2 = THREADS >= 512 ? 512 : THREADS >= 256 ? 256 : THREADS >= 128 ? 128 : THREADS >= 64 ? 64 : 32;
    __shared__ double red[THREADS];
    __shared__ bool last;
    auto tree = [&]() {
      if (POW2 < THREADS) {
        if ((int)threadIdx.x < THREADS - POW2) red[threadIdx.x] += red[threadIdx.x + POW2];
        __syncthreads();
      }
      for (int o = POW2 / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
      }
    };
    red[threadIdx.x] = dot.value();
    __syncthreads();
    tree();
    if (threadIdx.x == 0) {
      a.partials[blockIdx.x] = red[0];
      __threadfence();
      last = atomicAdd(a.counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += THREADS) s += ((volatile double*)a.partials)[b];
    red[threadIdx.x] = s;
    __syncthreads();
    tree();
    if (threadIdx.x == 0) {
      const double rz = red[0];
      CGState* st = a.cg;
      if (a.rz_mode == 0) st->rz_prev = st->rz;
      if (a.rz_mode == 2) {
        st->beta = 0.0;
        st->rz_prev = rz;
      } else {
        st->beta = (st->rz_prev != 0.0 && isfinite(rz)) ? rz / st->rz_prev : 0.0;
      }
      if (!(rz > 0.0) || !isfinite(rz)) {
        if (st->rr > 0.0) st->flag = 1;  // M^{-1} is positive definite: r.z > 0 unless r = 0
      }
      st->rz = rz;
      *a.counter = 0u;
    }
  }
}

// ------------------------------------------------------ y / z complex passes
template <typename T, int N, int L, int MODE>
__global__ void __launch_bounds__(Strided<T, N, L>::THREADS, 2) k_pfft(const PfftArgs<T> a, const int nbx,
                                                                    const long long ntiles) {
  using S = Strided<T, N, L>;
  using F = typename S::F;
  RK_DYN_SMEM(unsigned char, smem);
  TileFeed<T, N, L> feed{reinterpret_cast<T*>(smem), nullptr, 0u, 0};
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smem + S::SMEM_TILE);
  const int l = threadIdx.x % L, t = threadIdx.x / L;
  InterleavedBuf<T, F::N1, F::N2> buf{sm + l, L};
  const T* Sf = reinterpret_cast<const T*>(a.S);
  const int nxf = 2 * a.ncols;  // floats per row of columns
  auto origin = [&](long long tile, int* c0) -> long long {
    *c0 = (int)(tile % nbx) * L;  // first complex column of the tile
    return (long long)*c0 + (tile / nbx) * a.other_stride;
  };
  auto prefetch = [&](long long tile) {
    int c0;
    const long long o = origin(tile, &c0);
    S::issue(feed.tile, Sf + 2 * o, nxf - 2 * c0, 2 * a.line_stride, true);
  };
  long long tile = blockIdx.x;
  if (tile < ntiles) prefetch(tile);
  cpx<T> v[S::R];
  for (; tile < ntiles; tile += gridDim.x) {
    int c0;
    const long long base = origin(tile, &c0) + l;
    const int col = c0 + l;
    const bool ok = col < a.ncols;
    cp_async_wait_all();
    RK_SYNC();
#pragma unroll
    for (int r = 0; r < S::R; ++r) v[r] = S::at(feed.tile, MODE == PF_INV ? F::spec_idx(t, r) : F::nat_pos(t, r), l);
    RK_SYNC();
    if (tile + gridDim.x < ntiles) prefetch(tile + gridDim.x);
    if (MODE == PF_FWD) {
      F::forward(v, t, buf, a.tw);
      if (ok)
#pragma unroll
        for (int r = 0; r < S::R; ++r) a.S[base + F::spec_idx(t, r) * a.line_stride] = v[r];
    } else if (MODE == PF_INV) {
      F::inverse(v, t, buf, a.tw);
      if (ok)
#pragma unroll
        for (int r = 0; r < S::R; ++r) a.S[base + F::nat_pos(t, r) * a.line_stride] = v[r];
    } else {
      F::forward(v, t, buf, a.tw);
      // the other index of the z pass is the y frequency; the table rows are [kz][ky]
      const long long mrow = (tile / nbx) * a.ncols + col;
#pragma unroll
      for (int r = 0; r < S::R; ++r) {
        const T m = ok ? RK_LDG(a.mult + mrow + (long long)F::spec_idx(t, r) * a.line_stride) : (T)0;
        v[r] = cscale(v[r], m);
      }
      F::inverse(v, t, buf, a.tw);
      if (ok)
#pragma unroll
        for (int r = 0; r < S::R; ++r) a.S[base + F::nat_pos(t, r) * a.line_stride] = v[r];
    }
  }
}

}  // namespace rk
