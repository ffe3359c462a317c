// rk_moment.cuh -- per-node moment solve of Alg. 1 (kernel body shared by the
// library build).
#pragma once

#include "rk_internal.cuh"

namespace rk {

// ---------------------------------------------------------------- Alg. 1 tail
// One thread per node: assemble M(x) from the moment fields (Eq. 48/80; M = I off
// chi), Cholesky factorisation in FP64, rows 1..1+dim of M^{-1} by two triangular
// solves, then b^0 = row 1, b^k = -(1/a_k) row (1+k) (Eq. 83-85, scaled basis;
// b^z = 0 in 2D).
// A pivot <= 1e-14 * trace(M) marks the node singular: its b are set to 0 and the
// node is counted.  The basis size S is a template parameter, so that the loops
// unroll and the packed factor stays in registers (with a run-time size it lived
// in local memory).
template <int S>
__global__ void __launch_bounds__(128) k_moment_solve(const MomentArgs a) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.nbox;
       i += (long long)gridDim.x * blockDim.x) {
    double L[S * (S + 1) / 2];  // packed lower triangle, row-major
    const bool in = a.chi[i] != 0;
    double tr = 0.0;
#pragma unroll
    for (int p = 0; p < S; ++p)
#pragma unroll
      for (int q = 0; q <= p; ++q) {
        double v = in ? a.mom[(long long)a.pq[p][q] * a.nbox + i] : (p == q ? 1.0 : 0.0);
        L[p * (p + 1) / 2 + q] = v;
        if (p == q) tr += fabs(v);
      }
    bool bad = false;
#pragma unroll
    for (int j = 0; j < S; ++j) {
      if (bad) continue;
      double d = L[j * (j + 1) / 2 + j];
#pragma unroll
      for (int k = 0; k < j; ++k) d -= L[j * (j + 1) / 2 + k] * L[j * (j + 1) / 2 + k];
      if (!(d > 1e-14 * tr)) {
        bad = true;
        continue;
      }
      const double l = sqrt(d);
      L[j * (j + 1) / 2 + j] = l;
#pragma unroll
      for (int r = j + 1; r < S; ++r) {
        double v = L[r * (r + 1) / 2 + j];
#pragma unroll
        for (int k = 0; k < j; ++k) v -= L[r * (r + 1) / 2 + k] * L[j * (j + 1) / 2 + k];
        L[r * (r + 1) / 2 + j] = v / l;
      }
    }
    if (bad) {
      atomicAdd(a.n_singular, 1ull);
      atomicMin(a.first_singular, (unsigned long long)i);
    }
#pragma unroll
    for (int row = 0; row < 4; ++row) {
      double x[S];
#pragma unroll
      for (int p = 0; p < S; ++p) x[p] = (p == row) ? 1.0 : 0.0;
      if (!bad && row <= a.dim) {  // b^k = 0 on an absent axis
#pragma unroll
        for (int p = 0; p < S; ++p) {
          double v = x[p];
#pragma unroll
          for (int k = 0; k < p; ++k) v -= L[p * (p + 1) / 2 + k] * x[k];
          x[p] = v / L[p * (p + 1) / 2 + p];
        }
#pragma unroll
        for (int p = S - 1; p >= 0; --p) {
          double v = x[p];
#pragma unroll
          for (int k = p + 1; k < S; ++k) v -= L[k * (k + 1) / 2 + p] * x[k];
          x[p] = v / L[p * (p + 1) / 2 + p];
        }
      } else {
#pragma unroll
        for (int p = 0; p < S; ++p) x[p] = 0.0;
      }
      const double sc = row == 0 ? 1.0 : -a.inv_a[row - 1];
#pragma unroll
      for (int p = 0; p < S; ++p) {
        const double v = sc * x[p];
        const long long o = ((long long)row * S + p) * a.nbox + i;
        a.b64[o] = v;
        if (a.b32) a.b32[o] = (float)v;
      }
    }
    const double cv = in ? a.V[i] : 0.0;
    a.chiV64[i] = cv;
    if (a.chiV32) a.chiV32[i] = (float)cv;
  }
}

}  // namespace rk
