// rk_pointwise.cuh -- the pointwise stage of Alg. 2 on one 16-byte vector of
// consecutive nodes, in place over the s fields D_p:
//   A^k = sum_q b^k_q D_q (Eq. 90),  g_p = chi V sum_k b^k_p A^k (Eq. 91),
// with the coefficients of a node from breg (cidx = 0), from row cidx - 1 of ctab
// (cidx > 0), or g = 0 off chi (cidx = -1).  Used by the stand-alone pointwise
// kernel and by the z SPLIT pass, which applies it to every tile right after
// writing the tile's D_p (the values then come back from L2, not HBM).
#pragma once

#include <cstring>
#include <type_traits>

#include "rk_common.cuh"

namespace rk {

template <typename T>
struct PointwiseArgs {
  T* D[10];
  int s;
  const int* cidx;   // per node: -1 outside chi, 0 regular, 1 + row of ctab
  const T* ctab;     // [n_irr][ctab_pitch<T>(s)]: b^x_p, b^y_p, b^z_p (s each), chi V, zero padding
  long long n_irr;
  T breg[31];        // the 3s+1 values of a regular node
  long long nbox;
  // diag (z SPLIT only): the regular nodes' b^k are diagonal and D_{1+k} arrive
  // scaled by c_k = chi V (b^k_{1+k})^2, i.e. already equal to their g_{1+k};
  // regbits: bit g set when nodes 4g .. 4g + 3 are all regular
  int diag;
  T inv_c[3];
  const uint32_t* regbits;
  const uint32_t* outbits;  // bit g set when nodes 4g .. 4g + 3 are all outside chi
};

// Row pitch of the table of irregular nodes: 3s+1 values padded to whole 16-byte
// vectors, so that a row is read with 16-byte loads.
template <typename T>
constexpr int ctab_pitch(int s) {
  return (3 * s + 1 + (int)(16 / sizeof(T)) - 1) / (int)(16 / sizeof(T)) * (int)(16 / sizeof(T));
}

template <typename T>
using Vec16 = typename std::conditional<sizeof(T) == 4, float4, double2>::type;

// br[CP] <- breg, zero padded; the caller synchronises before the first use
template <typename T, int S>
RK_DEV void pointwise_stage_breg(const PointwiseArgs<T>& a, T* br, int tid, int nthreads) {
  constexpr int NC = 3 * S + 1, CP = ctab_pitch<T>(S);
  for (int j = tid; j < CP; j += nthreads) br[j] = j < NC ? a.breg[j] : (T)0;
}

// The 3s+1 (padded) coefficients of a node of class c: its row of the table of
// irregular nodes (c > 0) or the shared interior values (16-byte loads).
template <typename T, int S>
RK_DEV void pointwise_coefs(const PointwiseArgs<T>& a, const T* br, int c, T* co) {
  constexpr int VEC = 16 / sizeof(T);
  constexpr int CP = ctab_pitch<T>(S);
  using V16 = Vec16<T>;
  if (c > 0) {
    const V16* src = reinterpret_cast<const V16*>(a.ctab + (long long)(c - 1) * CP);
#pragma unroll
    for (int k = 0; k < CP / VEC; ++k) {
      const V16 raw = __ldg(src + k);
      memcpy(co + k * VEC, &raw, 16);
    }
  } else {
#pragma unroll
    for (int k = 0; k < CP / VEC; ++k) {
      const V16 raw = reinterpret_cast<const V16*>(br)[k];
      memcpy(co + k * VEC, &raw, 16);
    }
  }
}

// Eq. 90-91 at one node: A^k = sum_q b^k_q d_q, g_p = chi V sum_k b^k_p A^k (0 off chi)
template <typename T, int S>
RK_DEV void pointwise_node(const T* co, int c, const T* d, T* g) {
  T A[3] = {(T)0, (T)0, (T)0};
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int q = 0; q < S; ++q) A[k] += co[k * S + q] * d[q];
  const T cv = c >= 0 ? co[3 * S] : (T)0;  // chi V; 0 outside chi
#pragma unroll
  for (int p = 0; p < S; ++p) g[p] = cv * (co[p] * A[0] + co[S + p] * A[1] + co[2 * S + p] * A[2]);
}

// Nodes i0 .. i0 + VEC - 1, i0 a multiple of VEC = 16 / sizeof(T).  L2ONLY: the D
// loads bypass L1 (ld.global.cg), as required when D was written earlier in the
// same kernel by other threads of the block.  With a.diag the scaling of D_x, D_y,
// D_z is undone first.
template <typename T, int S, bool L2ONLY>
RK_DEV void pointwise_vec(const PointwiseArgs<T>& a, const T* br, long long i0) {
  constexpr int VEC = 16 / sizeof(T);
  constexpr int CP = ctab_pitch<T>(S);
  using V16 = Vec16<T>;
  int ci[VEC];
  if (VEC == 4) {
    const int4 c4 = __ldg(reinterpret_cast<const int4*>(a.cidx + i0));
    ci[0] = c4.x;
    ci[1] = c4.y;
    ci[VEC > 2 ? 2 : 0] = c4.z;
    ci[VEC > 3 ? 3 : 0] = c4.w;
  } else {
    const int2 c2 = __ldg(reinterpret_cast<const int2*>(a.cidx + i0));
    ci[0] = c2.x;
    ci[1] = c2.y;
  }
  T d[S][VEC];
#pragma unroll
  for (int q = 0; q < S; ++q) {
    const V16* src = reinterpret_cast<const V16*>(a.D[q] + i0);
    const V16 raw = L2ONLY ? __ldcg(src) : *src;
    memcpy(d[q], &raw, 16);
  }
  if (a.diag)
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int e = 0; e < VEC; ++e) d[1 + k][e] *= a.inv_c[k];
  T g[S][VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) {
    T co[ctab_pitch<T>(S)];
    pointwise_coefs<T, S>(a, br, ci[e], co);
    T de[S], ge[S];
#pragma unroll
    for (int q = 0; q < S; ++q) de[q] = d[q][e];
    pointwise_node<T, S>(co, ci[e], de, ge);
#pragma unroll
    for (int p = 0; p < S; ++p) g[p][e] = ge[p];
  }
#pragma unroll
  for (int p = 0; p < S; ++p) {
    V16 raw;
    memcpy(&raw, g[p], 16);
    *reinterpret_cast<V16*>(a.D[p] + i0) = raw;
  }
}

}  // namespace rk
