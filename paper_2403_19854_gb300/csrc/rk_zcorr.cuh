// rk_zcorr.cuh -- the z axis of Alg. 2 split into its regular part and local
// corrections.
//
// Along z, Alg. 2 takes the y-pass outputs E_g (one per group g = (alpha_x,
// alpha_y)) to D_p = conv_z(E_g(p), T_{alpha_z(p)}) (Eq. 86), applies the pointwise
// stage g_p = chi V sum_k b^k_p A^k with A^k = sum_q b^k_q D_q (Eq. 90-91), and
// returns G_g = sum_{p in g} conv_z(g_p, Tbar_{alpha_z(p)}).  At a regular node
// (its whole support in chi, interior V) the odd moments vanish, b^k_q = 0 for
// q != 1+k, and the stage reduces to g_p = c_p D_p with c_{1+k} = chi V (b^k_{1+k})^2
// and c_p = 0 for the other p.  Writing g_p = c_p D_p + delta_p at every node, the
// part c_p D_p is a convolution of E_g(p) with T * Tbar scaled by c_p: one spectral
// multiplier c_p n |T^_{alpha_z}|^2 per group, applied by a z pass with one forward
// and one inverse transform per group (rk_passes.cuh, split kernel).  delta_p is
// zero at regular nodes and at nodes farther than the support from chi (where D
// vanishes), so it lives on the boundary layers; this file adds its reflected
// convolution to G by direct sums over the short z-windows around those nodes:
//   D_q(z)  = sum_{o=-r..r} T_{alpha_z(q)}(o) E_g(q)(z - o)          (Eq. 86 along z)
//   delta_p = g_p - c_p D_p                  (g from the node's coefficients; 0 off chi)
//   G_g(z) += sum_{p in g} sum_{o=-r..r} T_{alpha_z(p)}(o) delta_p(z + o)   (Eq. 91, 57)
// with T_m(o) = (o/a~)^m phi(|o|/a~) (Eq. 6-7, 77) and circular indices (Eq. 68).
// A line of the box without chi nodes has g = 0 everywhere, so its G is 0.
#pragma once

#include "rk_passes.cuh"
#include "rk_pointwise.cuh"

namespace rk {

// Lane layout of the correction kernel: a warp covers kZGW adjacent z-lines (x
// consecutive, so its loads and stores are coalesced) times kZW consecutive z,
// and walks its record kZW positions at a time.  A record spans at most
// zcorr_chunk(s) positions.
constexpr int kZGW = 4;
constexpr int kZW = 32 / kZGW;
constexpr int kZMaxReach = 4;  // supports up to a = 4.5h
constexpr RK_HD int zcorr_chunk(int s) { return s == 4 ? 32 : 16; }

// A record of the correction kernel for the group of kZGW z-lines starting at
// line0 (= x0 + n_x y, x0 a multiple of kZGW); lines of the group in `mask`.
// len > 0: output nodes z0 .. z0 + len - 1 (mod n_z, len <= zcorr_chunk(s)) of those lines
// get the correction.  len == 0: those lines hold no chi node; all their outputs
// are set to 0.
struct ZWin {
  int line0;
  short z0;
  short len;
  unsigned mask;
};

template <typename T>
struct ZCorrArgs {
  const T* E[6];        // z-axis inputs, one per group
  T* G[6];              // z-axis outputs, one per group (regular part on entry)
  int nY, s;
  const int* cidx;      // -1 outside chi, 0 regular, 1 + row of ctab
  const T* ctab;        // rows of the irregular nodes (b^x_p, b^y_p, b^z_p, chi V), pitch ctab_pitch<T>(s)
  T creg[10];           // c_p of a regular node (0 unless p = 1 + k)
  T tab[3][2 * kZMaxReach + 1];  // T_m(o), m = 0 .. 2, index o + r (row length 2r + 1)
  int r;
  int nx, ny, nz;
  const ZWin* win;
  long long nwin;
  const uint32_t* nbits;  // per line, 8 words: bit z set where delta may be nonzero (need)
  const uint32_t* mbits;  // per line, 8 words: bit z set within r of a need node (outputs)
};

// The z-axis structure of the basis (the group of each basis index p and its
// alpha_z) as compile-time tables, in the basis order [1, x, y, z, x^2, xy, xz,
// y^2, yz, z^2] with groups numbered by first appearance; set-up checks that the
// handle's chains match before it enables the corrections.
template <int S>
struct ZBasis;
template <>
struct ZBasis<4> {
  static constexpr int NY = 3;
  static constexpr RK_HD int grp(int p) { return p == 3 ? 0 : p; }
  static constexpr RK_HD int az(int p) { return p == 3 ? 1 : 0; }
};
template <>
struct ZBasis<10> {
  static constexpr int NY = 6;
  static constexpr RK_HD int grp(int p) {
    return p == 0 || p == 3 || p == 9 ? 0 : (p == 1 || p == 6 ? 1 : (p == 2 || p == 8 ? 2 : (p == 4 ? 3 : (p == 5 ? 4 : 5))));
  }
  static constexpr RK_HD int az(int p) { return p == 9 ? 2 : (p == 3 || p == 6 || p == 8 ? 1 : 0); }
};

// delta_p at node (line, zd) (0 at regular nodes); tb: T_m(o) for m <= 2 (shared
// memory).  The node class and the E values are loaded together, so a node costs
// one round trip to memory before its coefficient row.
template <typename T, int S, int R>
RK_DEV void zcorr_delta(const ZCorrArgs<T>& a, const T (*tb)[2 * R + 1], long long line, long long zs, int zd,
                        T* delta) {
  using B = ZBasis<S>;
  T ev[B::NY][2 * R + 1];
  const int c = __ldg(a.cidx + line + (long long)zd * zs);
#pragma unroll
  for (int g = 0; g < B::NY; ++g)
#pragma unroll
    for (int o = -R; o <= R; ++o) {
      int z = zd - o;
      z = z < 0 ? z + a.nz : (z >= a.nz ? z - a.nz : z);
      ev[g][o + R] = __ldg(a.E[g] + line + (long long)z * zs);
    }
#pragma unroll
  for (int p = 0; p < S; ++p) delta[p] = (T)0;
  if (c == 0) return;
  T D[S];
#pragma unroll
  for (int q = 0; q < S; ++q) {
    T acc = (T)0;
#pragma unroll
    for (int j = 0; j <= 2 * R; ++j) acc += tb[B::az(q)][j] * ev[B::grp(q)][j];
    D[q] = acc;
  }
  if (c > 0) {
    constexpr int CP = ctab_pitch<T>(S);
    T co[CP];
    const Vec16<T>* src = reinterpret_cast<const Vec16<T>*>(a.ctab + (long long)(c - 1) * CP);
#pragma unroll
    for (int k = 0; k < CP / (16 / (int)sizeof(T)); ++k) {
      const Vec16<T> raw = __ldg(src + k);
      memcpy(co + k * (16 / (int)sizeof(T)), &raw, 16);
    }
    T g[S];
    pointwise_node<T, S>(co, c, D, g);
#pragma unroll
    for (int p = 0; p < S; ++p) delta[p] = g[p] - a.creg[p] * D[p];
  } else {
#pragma unroll
    for (int p = 0; p < S; ++p) delta[p] = -a.creg[p] * D[p];
  }
}

template <typename T, int S>
constexpr int zcorr_warps() {
  return 4;
}

// One warp per record, WARPS records per block.  Per warp, shared memory holds
// delta on the positions z0 - R .. z0 + len + R - 1 a record needs: dl[t][p][xi].
// A lane computes delta only at its line's need nodes (zero elsewhere up to
// rounding) and updates only the outputs within r of one.
template <typename T, int S, int R, int WARPS>
__global__ void __launch_bounds__(32 * WARPS) k_zcorr(const ZCorrArgs<T> a) {
  using B = ZBasis<S>;
  constexpr int NPOS = zcorr_chunk(S) + 2 * R;
  __shared__ T dl[WARPS][NPOS][S][kZGW];
  __shared__ T tb[3][2 * R + 1];
  for (int i = threadIdx.x; i < 3 * (2 * R + 1); i += blockDim.x) tb[i / (2 * R + 1)][i % (2 * R + 1)] = a.tab[i / (2 * R + 1)][i % (2 * R + 1)];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int xi = lane % kZGW, zi = lane / kZGW;
  const long long zs = (long long)a.nx * a.ny;
  for (long long wi = (long long)blockIdx.x * WARPS + w; wi < a.nwin; wi += (long long)gridDim.x * WARPS) {
    const ZWin rec = a.win[wi];
    const bool active = (rec.mask >> xi) & 1u;
    const long long line = (long long)rec.line0 + xi;
    if (rec.len == 0) {
      if (active)
        for (int z = zi; z < a.nz; z += kZW)
#pragma unroll
          for (int g = 0; g < B::NY; ++g) a.G[g][line + (long long)z * zs] = (T)0;
      continue;
    }
    const uint32_t* nb = a.nbits + 8 * line;
    const uint32_t* mb = a.mbits + 8 * line;
    // delta at positions z0 - R + t, t < len + 2R
    for (int t = zi; t < rec.len + 2 * R; t += kZW) {
      T delta[S];
#pragma unroll
      for (int p = 0; p < S; ++p) delta[p] = (T)0;
      if (active) {
        int zd = rec.z0 - R + t;
        zd = zd < 0 ? zd + a.nz : (zd >= a.nz ? zd - a.nz : zd);
        if ((__ldg(nb + (zd >> 5)) >> (zd & 31)) & 1u) zcorr_delta<T, S, R>(a, tb, line, zs, zd, delta);
      }
#pragma unroll
      for (int p = 0; p < S; ++p) dl[w][t][p][xi] = delta[p];
    }
    __syncwarp();
    if (active)
      for (int zo = zi; zo < rec.len; zo += kZW) {
        int z = rec.z0 + zo;
        z = z >= a.nz ? z - a.nz : z;
        if (!((__ldg(mb + (z >> 5)) >> (z & 31)) & 1u)) continue;  // no need node within r
        const long long i = line + (long long)z * zs;
        T gv[B::NY];
#pragma unroll
        for (int g = 0; g < B::NY; ++g) gv[g] = a.G[g][i];
#pragma unroll
        for (int p = 0; p < S; ++p)
#pragma unroll
          for (int j = 0; j <= 2 * R; ++j) gv[B::grp(p)] += tb[B::az(p)][j] * dl[w][zo + j][p][xi];
#pragma unroll
        for (int g = 0; g < B::NY; ++g) a.G[g][i] = gv[g];
      }
    __syncwarp();
  }
}

// ------------------------------------------------------------ set-up
// Records of one group of kZGW lines (one thread per group): a zeroing record for
// its lines without chi nodes that are within the support of chi, and correction
// records over the union of the marked positions of its other lines, cut into
// runs of at most `chunk`.  FILL = 0 counts them into counts[group], FILL = 1 writes
// them from offset counts[group].
template <bool FILL>
__global__ void k_zwin_groups(const uint32_t* mk, const uint8_t* flags, int nx, int ny, int nz, int chunk, int* counts,
                              ZWin* out) {
  const int ngx = (nx + kZGW - 1) / kZGW;
  const long long ngroups = (long long)ngx * ny;
  for (long long G = (long long)blockIdx.x * blockDim.x + threadIdx.x; G < ngroups; G += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(G / ngx), x0 = (int)(G % ngx) * kZGW;
    const long long line0 = x0 + (long long)nx * y;
    uint32_t u[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    unsigned cmask = 0, zmask = 0;
    for (int xi = 0; xi < kZGW && x0 + xi < nx; ++xi) {
      const uint8_t f = flags[line0 + xi];
      if (!(f & 2)) continue;
      if (f & 1) {
        cmask |= 1u << xi;
        for (int k = 0; k < 8; ++k) u[k] |= mk[8 * (line0 + xi) + k];
      } else {
        zmask |= 1u << xi;
      }
    }
    int cnt = 0;
    int at = FILL ? counts[G] : 0;
    auto emit = [&](int z0, int len, unsigned mask) {
      if (FILL) {
        ZWin wv;
        wv.line0 = (int)line0;
        wv.z0 = (short)z0;
        wv.len = (short)len;
        wv.mask = mask;
        out[at++] = wv;
      }
      ++cnt;
    };
    auto marked = [&](int z) { return ((u[z >> 5] >> (z & 31)) & 1u) != 0; };
    if (zmask) emit(0, 0, zmask);
    if (cmask) {
      int s0 = -1;
      for (int z = 0; z < nz && s0 < 0; ++z)
        if (!marked(z)) s0 = z;
      if (s0 < 0) {
        for (int z0 = 0; z0 < nz; z0 += chunk) emit(z0, min(chunk, nz - z0), cmask);
      } else {
        int start = -1, len = 0;
        for (int t = 1; t <= nz; ++t) {
          const int z = (s0 + t) % nz;
          if (marked(z)) {
            if (start < 0) {
              start = z;
              len = 0;
            }
            ++len;
            if (len == chunk) {
              emit(start, len, cmask);
              start = -1;
            }
          } else if (start >= 0) {
            emit(start, len, cmask);
            start = -1;
          }
        }
        if (start >= 0) emit(start, len, cmask);
      }
    }
    if (!FILL) counts[G] = cnt;
  }
}

}  // namespace rk
