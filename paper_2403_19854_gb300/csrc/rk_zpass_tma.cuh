// rk_zpass_tma.cuh -- persistent fused z pass of Alg. 2 (Z_STIFF) with TMA input
// tiles.
//
// Each block owns a sequence of pencils (2L adjacent x, one y, all z).  The
// pencil's input fields E_(ax,ay) (outputs of the y pass) arrive as TMA boxes
// {2L, 1, N} into a double-buffered shared-memory stage; the tile after the one
// being transformed is always in flight, and the first tile of the next pencil is
// loaded while the current pencil runs its reflected chain.  The transforms,
// the pointwise stage (Eq. 90-91, compressed coefficients) and the outputs are
// those of k_z_fused<..., Z_STIFF>.
#pragma once

#include "rk_passes.cuh"
#include "rk_tma.cuh"

namespace rk {

template <typename T, int N, int L>
struct ZTma {
  using S = Strided<T, N, L>;
  using F = LineFFT<T, N>;
  static constexpr int P = F::P, R = F::R;
  static constexpr int THREADS = L * P;
  static constexpr int STAGES = 2;
  static constexpr size_t TILE = sizeof(T) * (size_t)N * 2 * L;  // bytes of one box
  static constexpr size_t OFF_BUF = STAGES * TILE;
  static constexpr size_t OFF_A = OFF_BUF + sizeof(cpx<T>) * (size_t)N * L;
  static constexpr size_t OFF_BREG = OFF_A + 3 * sizeof(cpx<T>) * (size_t)N * L;
  static constexpr size_t OFF_TW = OFF_BREG + 256;                  // N twiddles
  static constexpr size_t OFF_COEF = OFF_TW + sizeof(cpx<T>) * N;     // multiplier rows m = 0..2
  static constexpr size_t OFF_BAR = OFF_COEF + sizeof(T) * 3 * N;
  static constexpr size_t SMEM = OFF_BAR + 64;
  static_assert(TILE % 128 == 0, "TMA destinations must stay 128-byte aligned");
};

template <typename T, int N, int L>
__global__ void __launch_bounds__(ZTma<T, N, L>::THREADS) k_z_stiff_tma(const __grid_constant__ ZArgs<T> a) {
  using Z = ZTma<T, N, L>;
  using S = typename Z::S;
  using F = typename Z::F;
  using V2 = typename vec2<T>::type;
  extern __shared__ __align__(128) unsigned char zsm[];
  T* tiles = reinterpret_cast<T*>(zsm);
  cpx<T>* bufb = reinterpret_cast<cpx<T>*>(zsm + Z::OFF_BUF);
  cpx<T>* Acc = reinterpret_cast<cpx<T>*>(zsm + Z::OFF_A);
  T* breg_s = reinterpret_cast<T*>(zsm + Z::OFF_BREG);
  uint64_t* bars = reinterpret_cast<uint64_t*>(zsm + Z::OFF_BAR);
  cpx<T>* tw_s = reinterpret_cast<cpx<T>*>(zsm + Z::OFF_TW);
  T* coef_s = reinterpret_cast<T*>(zsm + Z::OFF_COEF);

  const int l = threadIdx.x % L, t = threadIdx.x / L;
  const int ntx = (a.nx / 2 + L - 1) / L;
  const long long npen = (long long)ntx * a.ny;
  const long long zs = (long long)a.nx * a.ny;
  const int nG = a.n_groups;
  if (threadIdx.x == 0) {
    for (int st = 0; st < Z::STAGES; ++st) mbar_init(&bars[st], 1);
    mbar_init_fence();
  }
  for (int j = threadIdx.x; j < 3 * a.s + 1; j += blockDim.x) breg_s[j] = a.breg[j];
  for (int j = threadIdx.x; j < N; j += blockDim.x) tw_s[j] = a.tw[j];
  const int mrows = a.s == 4 ? 2 : 3;  // z exponents used by the basis: 0..degree
  for (int j = threadIdx.x; j < mrows * N; j += blockDim.x) coef_s[j] = a.coef[j];
  __syncthreads();

  // k-th tile of this block: pencil blockIdx.x + (k / nG) gridDim.x, group k % nG
  auto issue = [&](long long k) {
    const long long pen = blockIdx.x + (k / nG) * (long long)gridDim.x;
    if (pen >= npen) return;
    const int g = (int)(k % nG), st = (int)(k % Z::STAGES);
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&bars[st], (uint32_t)Z::TILE);
    tma_load_3d(tiles + (size_t)st * (Z::TILE / sizeof(T)), &a.tmap[g], &bars[st], (int)(pen % ntx) * 2 * L,
                (int)(pen / ntx), 0);
  };
  long long k = 0;
  if (threadIdx.x == 0) issue(0);
  InterleavedBuf<T, F::N1, F::N2> buf{bufb + l, L};
  auto A = [&](int kk, int r) -> cpx<T>& { return Acc[((size_t)kk * N + F::nat_pos(t, r)) * L + l]; };
  bool failed = false;
  cpx<T> v[Z::R], w[Z::R];

  for (long long pen = blockIdx.x; pen < npen && !failed; pen += gridDim.x) {
    const int x = (int)(pen % ntx) * 2 * L + 2 * l;
    const bool ok = x < a.nx;
    const long long base = (long long)x + (pen / ntx) * a.nx;
    unsigned cls[(Z::R + 7) / 8] = {};  // 4 bits per register: 2 per node of the pair
    {
#pragma unroll
      for (int r = 0; r < Z::R; ++r) {
        int2 ci = make_int2(-1, -1);
        if (ok) ci = *reinterpret_cast<const int2*>(a.cidx + base + F::nat_pos(t, r) * zs);
        const unsigned c0 = ci.x < 0 ? 0u : (ci.x == 0 ? 1u : 2u);
        const unsigned c1 = ci.y < 0 ? 0u : (ci.y == 0 ? 1u : 2u);
        cls[r / 8] |= (c0 | (c1 << 2)) << (4 * (r % 8));
      }
    }
    // coefficient j (b^k_p at j = k s + p, chi V at j = 3s) of the node pair at off:
    // regular nodes take the interior value, irregular ones their table row
    auto ccoef = [&](int r, long long off, int j) -> cpx<T> {
      const unsigned code = (cls[r / 8] >> (4 * (r % 8))) & 15u;
      const T reg = breg_s[j];
      T v0 = (code & 3u) == 1u ? reg : (T)0;
      T v1 = (code >> 2) == 1u ? reg : (T)0;
      if ((code & 3u) == 2u) v0 = a.ctab[(long long)j * a.n_irr + (a.cidx[off] - 1)];
      if ((code >> 2) == 2u) v1 = a.ctab[(long long)j * a.n_irr + (a.cidx[off + 1] - 1)];
      return cmk(v0, v1);
    };
#pragma unroll
    for (int r = 0; r < Z::R; ++r) A(0, r) = A(1, r) = A(2, r) = cmk((T)0, (T)0);

    // forward chain: D_p = conv_z(E_(ax,ay), T_az), A^k += b^k_p D_p  (Eq. 90)
    for (int g = 0; g < nG; ++g) {
      if (threadIdx.x == 0) issue(k + 1);
      const int st = (int)(k % Z::STAGES);
      const bool okw = mbar_wait(&bars[st], (uint32_t)((k / Z::STAGES) & 1));
      if (__syncthreads_or(!okw)) {
        failed = true;
        break;
      }
      const T* tile = tiles + (size_t)st * (Z::TILE / sizeof(T));
#pragma unroll
      for (int r = 0; r < Z::R; ++r) {
        const V2 e = *reinterpret_cast<const V2*>(tile + (size_t)F::nat_pos(t, r) * 2 * L + 2 * l);
        v[r] = cmk(e.x, e.y);
      }
      ++k;
      F::forward(v, t, buf, tw_s);
      for (int q = a.g_begin[g]; q < a.g_begin[g + 1]; ++q) {
        const int mz = a.term_mz[q], p = a.term_p[q];
#pragma unroll
        for (int r = 0; r < Z::R; ++r) w[r] = spec_mul(v[r], coef_s, N, mz, F::spec_idx(t, r), 0);
        F::inverse(w, t, buf, tw_s);
#pragma unroll
        for (int r = 0; r < Z::R; ++r) {
          const long long off = base + F::nat_pos(t, r) * zs;
#pragma unroll
          for (int kk = 0; kk < 3; ++kk) {
            const cpx<T> bk = ccoef(r, off, kk * a.s + p);
            cpx<T>& Ak = A(kk, r);
            Ak = pfma(bk, w[r], Ak);
          }
        }
      }
    }
    if (failed) break;

    // reflected chain: G_(ax,ay) = sum_az conv_z(g_p, Tbar_az), g_p = chi V sum_k b^k_p A^k (Eq. 91)
    for (int g = 0; g < nG; ++g) {
      cpx<T> acc[Z::R];
#pragma unroll
      for (int r = 0; r < Z::R; ++r) acc[r] = cmk((T)0, (T)0);
      for (int q = a.g_begin[g]; q < a.g_begin[g + 1]; ++q) {
        const int mz = a.term_mz[q], p = a.term_p[q];
#pragma unroll
        for (int r = 0; r < Z::R; ++r) {
          const long long off = base + F::nat_pos(t, r) * zs;
          const cpx<T> cv = ccoef(r, off, 3 * a.s);
          cpx<T> sacc = cmk((T)0, (T)0);
#pragma unroll
          for (int kk = 0; kk < 3; ++kk) {
            const cpx<T> bk = ccoef(r, off, kk * a.s + p);
            const cpx<T> Ak = A(kk, r);
            sacc = pfma(bk, Ak, sacc);
          }
          v[r] = pmul(cv, sacc);
        }
        F::forward(v, t, buf, tw_s);
#pragma unroll
        for (int r = 0; r < Z::R; ++r) acc[r] = acc[r] + spec_mul(v[r], coef_s, N, mz, F::spec_idx(t, r), 1);
      }
      F::inverse(acc, t, buf, tw_s);
      if (ok)
#pragma unroll
        for (int r = 0; r < Z::R; ++r) S::store(a.out[g], base + F::nat_pos(t, r) * zs, acc[r]);
    }
  }
  if (failed && threadIdx.x == 0) {
    atomicExch(a.err, 1);
    // a prefetched tile may still be arriving: wait for it (bounded) before exit
    const int st = (int)(k % Z::STAGES);
    const long long pen = blockIdx.x + (k / nG) * (long long)gridDim.x;
    if (pen < npen) mbar_wait(&bars[st], (uint32_t)((k / Z::STAGES) & 1));
  }
}

}  // namespace rk
