// rk_passes.cuh -- axis passes of the FC-RKPM convolutions.
//
// Every convolving array of the method is a tensor product of 1D tables:
// H^a_p(x) = prod_k T^{(k)}_{alpha_k(p)}(x_k) with T_m(o) = (o/a~)^m phi(|o|/a~)
// (Eq. 6, 44, 77), and H_p H^a_q = prod_k T_{alpha_k(p)+alpha_k(q)} (Eq. 80).
// Its DFT (Eq. 30) is the product of the 1D DFTs, so each 3D fast convolution
// F^{-1}[F(a) o F(H)] of Eq. 34 factors into three 1D circular convolutions, one
// per axis, each done as forward FFT -> multiply -> inverse FFT along that axis.
// A pass applies one axis for several (input, table) pairs at once:
//   SPLIT: each input line is transformed once and convolved with several tables
//          (one output per table)                -- the forward chain of Alg. 1-3;
//   MERGE: several inputs, each with its table, are summed in the spectrum and
//          transformed back once                 -- the reflected chain of Alg. 2, 4.
// The z SPLIT of Alg. 2 also applies the pointwise stage between the two chains
// (A^k = sum_q b^k_q D_q, Eq. 90; C^k_p A^k, Eq. 91) to every tile it has just
// written, while the tile's values are still in L2.
//
// Data: real fields on the periodic box, x fastest (idx = i + nx*(j + ny*k)).
// Two real lines are packed into one complex line (re = line 0, im = line 1);
// the tables are real even/odd sequences, so convolution keeps the two apart.
//   x lines: pairs of consecutive rows (row r = j + ny*k), P threads per line;
//   y and z lines: pairs of adjacent x (a float2/double2 per node pair).
#pragma once

#include "rk_linefft.cuh"
#include "rk_pointwise.cuh"
#include "rk_tma.cuh"

namespace rk {

constexpr int kMaxIn = 16;   // input fields of one pass
constexpr int kMaxOut = 40;  // output fields (or terms) of one pass

// Spectral multiplier of table m at spectral index k:  coef[m*N + k] is real for
// even m (even table) and the imaginary part for odd m (odd table).  The 1/N of
// the inverse transform is included.  reflect selects H-bar (Eq. 55): (-1)^m.
template <typename T>
RK_HD cpx<T> spec_mul(cpx<T> v, const T* __restrict__ coef, int N, int m, int k, int reflect) {
  T c = coef[m * N + k];
  if (reflect && (m & 1)) c = -c;
  return (m & 1) ? ciscale(v, c) : cscale(v, c);
}

// Scalars of the conjugate-gradient recurrence, kept in device memory.
struct CGState {
  double rr;      // r.r of the current iterate (convergence)
  double pAp;
  double alpha;   // rz / pAp
  double beta;    // rz_new / rz_prev
  double rr_new;
  double rz;      // r.z (z = M^{-1} r; z = r without preconditioner, then rz = rr)
  double rz_prev;
  int flag;       // 1: breakdown (p^T A p <= 0, r.z <= 0 or not finite)
  int pcg;        // 1: z = M^{-1} r is formed by the preconditioner, which sets rz and beta
};
static_assert(sizeof(CGState) <= 16 * sizeof(double), "CGState must fit the pinned host slot");

template <typename T>
struct PassArgs {
  const T* in[kMaxIn];
  T* out[kMaxOut];
  int n_groups;
  int g_io[kMaxOut];          // SPLIT: input index of group g; MERGE: output index
  int g_begin[kMaxOut + 1];   // terms of group g
  int term_io[kMaxOut];       // SPLIT: output index of the term; MERGE: input index
  int term_m[kMaxOut];        // table (monomial power) of the term
  const T* coef;              // spectral multipliers of this axis, [mmax+1][N]
  const cpx<T>* tw;           // twiddles of this axis, [N]
  int reflect;
  int coef_rows;              // rows of coef (2 degree + 1); 0: not staged in shared memory
  const uint8_t* in_mask;     // optional: inputs multiplied by mask (x pass only)
  const uint8_t* out_mask;    // optional: outputs multiplied by mask (x pass only)
  int nx, ny, nz;
  long long line_stride;      // strided passes: element stride along the line
  long long other_stride;     // strided passes: stride of blockIdx.y
  // CG iteration fused into the x passes of A p (x SPLIT prologue, x MERGE epilogue):
  T* cg_p;                    // SPLIT: p, updated in place to r + beta p before use
                              // MERGE: p, for the product p . (A p) of the output
  const T* cg_r;              // SPLIT: r (prologue active when non-null)
  CGState* cg;                // beta (read); pAp, alpha, flag (written by the last MERGE block)
  double* partials;           // MERGE: one partial p.Ap per block
  unsigned* counter;          // MERGE: blocks finished (the last one reduces and resets it)
  int* err;                   // set to 1 when a bounded wait for an input tile gave up
  int xbulk;                  // x passes: rows arrive by bulk async copies (set by the launcher)
  int short_wait;             // 1: the first wait for each input tile gives up at once (tests
                              // of the time-out path; the copy still lands before the block
                              // returns); 0: waits of kWaitLimit polls
};

// ---------------------------------------------------------------- strided passes
// Block: L node pairs (2L adjacent x) times P threads per line; thread (t, l) with
// l = threadIdx.x % L fastest.  A tile is the N line positions x 2L values (128
// bytes per row) of one input field; it is copied into shared memory with
// cp.async while the block transforms the previous tile, so the loads of the
// next field (or of the next tile of the persistent loop) overlap the FFT work.

RK_DEV void cp_async16(void* smem, const void* gmem, int src_bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
RK_DEV void cp_async4(void* smem, const void* gmem, int src_bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
RK_DEV void cp_async8(void* smem, const void* gmem, int src_bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
RK_DEV void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
RK_DEV void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <typename T, int N, int L>
struct Strided {
  using F = LineFFT<T, N>;
  static constexpr int P = F::P, R = F::R;
  static constexpr int THREADS = L * P;
  // resident blocks per SM the register allocation must allow: the split pass
  // holds one line set per thread and gains from a third block, the merge pass
  // keeps an accumulator as well and spills at that register budget
  static constexpr int WARP_THREADS = (THREADS + 31) / 32 * 32;
  static constexpr int blocks_for(int threads_per_sm) {
    return threads_per_sm / WARP_THREADS > 2 ? threads_per_sm / WARP_THREADS : 2;
  }
  static constexpr int MIN_BLOCKS_SPLIT = blocks_for(sizeof(T) == 4 ? 768 : 384);
  static constexpr int MIN_BLOCKS_MERGE = blocks_for(sizeof(T) == 4 ? 512 : 384);
  static constexpr int ROW = 2 * L;                     // values per tile row
  static constexpr int C16 = ROW * (int)sizeof(T) / 16;  // 16-byte chunks per row
  static constexpr size_t SMEM_BUF = sizeof(cpx<T>) * (size_t)N * L;
  static constexpr size_t SMEM_TILE = sizeof(T) * (size_t)N * ROW;
  // FP32 split: the axis' multiplier rows (up to 5) and twiddles are copied to
  // shared memory once per block (the large shared-memory carve-out of these
  // kernels leaves little L1 for them; 2-3 % faster)
  static constexpr bool STAGE = sizeof(T) == 4;
  static constexpr int COEF_ROWS_MAX = 7;
  static constexpr size_t SMEM_CT = STAGE ? sizeof(T) * (size_t)COEF_ROWS_MAX * N + sizeof(cpx<T>) * (size_t)N : 0;
  static constexpr size_t SMEM = SMEM_BUF + SMEM_TILE + SMEM_CT;
  // copy coef / tw to shared memory; returns the pointers the block should use
  RK_DEV static void stage(const PassArgs<T>& a, unsigned char* smem, const T** coef, const cpx<T>** tw) {
    *coef = a.coef;
    *tw = a.tw;
    if (!STAGE || a.coef_rows <= 0 || a.coef_rows > COEF_ROWS_MAX) return;
    T* cs = reinterpret_cast<T*>(smem + SMEM_TILE + SMEM_BUF);
    cpx<T>* ts = reinterpret_cast<cpx<T>*>(cs + (size_t)COEF_ROWS_MAX * N);
    for (int i = threadIdx.x; i < a.coef_rows * N; i += THREADS) cs[i] = a.coef[i];
    for (int i = threadIdx.x; i < N; i += THREADS) ts[i] = a.tw[i];
    RK_SYNC();
    *coef = cs;
    *tw = ts;
  }

  // Copy rows src[x0 + j * line_stride + (0 .. nvalid-1)], j in [0, N), into tile
  // (zero-filled beyond nvalid).  a16: every row starts on a 16-byte boundary.
  RK_DEV static void issue(T* tile, const T* src, int nvalid, long long line_stride, bool a16) {
    if (a16) {
      for (int c = threadIdx.x; c < N * C16; c += THREADS) {
        const int j = c / C16, v0 = (c % C16) * (16 / (int)sizeof(T));
        const int bytes = max(0, min(16, (nvalid - v0) * (int)sizeof(T)));
        cp_async16(tile + j * ROW + v0, src + (long long)j * line_stride + (bytes > 0 ? v0 : 0), bytes);
      }
    } else {
      for (int c = threadIdx.x; c < N * ROW; c += THREADS) {
        const int j = c / ROW, v = c % ROW;
        const bool in = v < nvalid;
        const T* g = src + (long long)j * line_stride + (in ? v : 0);
        if (sizeof(T) == 4)
          cp_async4(tile + j * ROW + v, g, in ? 4 : 0);
        else
          cp_async8(tile + j * ROW + v, g, in ? 8 : 0);
      }
    }
    cp_async_commit();
  }
  RK_DEV static cpx<T> load(const T* p, long long off) {
    const typename vec2<T>::type v = RK_LDG(reinterpret_cast<const typename vec2<T>::type*>(p + off));
    return cmk(v.x, v.y);
  }
  RK_DEV static cpx<T> at(const T* tile, int row, int l) {
    return *reinterpret_cast<const cpx<T>*>(tile + row * ROW + 2 * l);
  }
  RK_DEV static void store(T* p, long long off, cpx<T> v) {
    typename vec2<T>::type w;
    w.x = v.x;
    w.y = v.y;
    *reinterpret_cast<typename vec2<T>::type*>(p + off) = w;
  }
};

// Tile feed of a strided pass.  tma_axis 1 or 2: the tiles are TMA boxes of the
// inputs' tensor maps ({2L, N, 1} at (x0, 0, other) along y, {2L, 1, N} at
// (x0, other, 0) along z), completed on one mbarrier; tma_axis 0: cp.async.
template <typename T, int N, int L>
struct TileFeed {
  using S = Strided<T, N, L>;
  T* tile;
  uint64_t* bar;
  uint32_t phase;
  int tma_axis;
  RK_DEV void init() {
    if (tma_axis) {
      if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_init_fence();
      }
      RK_SYNC();
    }
  }
  // start the copy of input `which` (pointer src = field + origin) of the tile at (x0, other)
  RK_DEV void issue(const TileMaps& maps, int which, const T* src, int x0, int other, int nx, long long line_stride,
                    bool a16) {
    if (tma_axis) {
      if (threadIdx.x == 0) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar, (uint32_t)S::SMEM_TILE);
        tma_load_3d(tile, &maps.m[which], bar, x0, tma_axis == 1 ? 0 : other, tma_axis == 1 ? other : 0);
      }
    } else {
      S::issue(tile, src, nx - x0, line_stride, a16);
    }
  }
  // wait for the tile; false (uniformly over the block) if the bounded wait gave up,
  // after which the caller returns
  RK_DEV bool wait(int* err, int short_wait) {
    bool ok = true;
    if (tma_axis) {
      ok = mbar_wait(bar, phase, short_wait ? 0u : kWaitLimit);
      phase ^= 1u;
    } else {
      cp_async_wait_all();
    }
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) flag_wait_error(err);
      if (tma_axis) mbar_wait(bar, phase ^ 1u);  // the copy still in flight, bounded
      return false;
    }
    return true;
  }
};

// PW > 0 (z SPLIT of Alg. 2, PW = s, diagonal interior coefficients): the
// multiplier rows of D_x, D_y, D_z carry c_k, so at regular nodes the pass writes
// g_x, g_y, g_z of Eq. 91 directly; it writes 0 for the other g_p of its regular
// 4-node groups and for every g_p of its groups outside chi (flags: a bit per
// group in pw.regbits / pw.outbits).  The remaining groups (boundary layers) are
// left to k_pointwise_groups.  Requires n_x to be a multiple of 4.
template <typename T, int N, int L, int PW>
__global__ void __launch_bounds__(Strided<T, N, L>::THREADS, Strided<T, N, L>::MIN_BLOCKS_SPLIT)
    k_strided_split(const PassArgs<T> a, const int nbx, const long long ntiles, const int a16,
                    const __grid_constant__ TileMaps maps, const int tma_axis,
                    const __grid_constant__ PointwiseArgs<T> pw) {
  using S = Strided<T, N, L>;
  using F = typename S::F;
  RK_DYN_SMEM(unsigned char, smem);
  __shared__ uint64_t bar;
  // per tile row: its all-regular / all-outside 4-node groups, a bit per group
  __shared__ uint8_t rflag[PW > 0 ? N : 1], oflag[PW > 0 ? N : 1];
  TileFeed<T, N, L> feed{reinterpret_cast<T*>(smem), &bar, 0u, tma_axis};
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smem + S::SMEM_TILE);
  const int l = threadIdx.x % L, t = threadIdx.x / L;
  InterleavedBuf<T, F::N1, F::N2> buf{sm + l, L};
  feed.init();
  auto prefetch = [&](long long tile, int g) {
    const int x0 = (int)(tile % nbx) * S::ROW;
    const long long by = tile / nbx;
    const int in = a.g_io[g];
    feed.issue(maps, in, a.in[in] + x0 + by * a.other_stride, x0, (int)by, a.nx, a.line_stride, a16 != 0);
  };
  long long tile = blockIdx.x;
  if (tile < ntiles) prefetch(tile, 0);
  const T* coef;
  const cpx<T>* tw;
  S::stage(a, smem, &coef, &tw);
  cpx<T> v[S::R], w[S::R];
  for (; tile < ntiles; tile += gridDim.x) {
    const int x0 = (int)(tile % nbx) * S::ROW;
    const long long base = x0 + (tile / nbx) * a.other_stride + 2 * l;
    const bool ok = x0 + 2 * l < a.nx;
    for (int g = 0; g < a.n_groups; ++g) {
      if (!feed.wait(a.err, a.short_wait)) return;  // (a block-wide barrier: the previous tile's flags are no longer read)
      if (PW > 0 && g == 0) {
        // the flag bytes of the tile rows: a row's ROW / 4 <= 8 groups start at bit
        // g0 = (tile origin + row * line_stride) / 4 and span at most two bytes (one
        // spare word ends the bit arrays)
        const uint8_t* rb = reinterpret_cast<const uint8_t*>(pw.regbits);
        const uint8_t* ob = reinterpret_cast<const uint8_t*>(pw.outbits);
        for (int row = threadIdx.x; row < N; row += S::THREADS) {
          const long long g0 = (base - 2 * l + row * a.line_stride) / 4;
          rflag[row] = (uint8_t)(((unsigned)__ldg(rb + g0 / 8) | ((unsigned)__ldg(rb + g0 / 8 + 1) << 8)) >> (g0 % 8));
          oflag[row] = (uint8_t)(((unsigned)__ldg(ob + g0 / 8) | ((unsigned)__ldg(ob + g0 / 8 + 1) << 8)) >> (g0 % 8));
        }
      }
#pragma unroll
      for (int r = 0; r < S::R; ++r) v[r] = S::at(feed.tile, F::nat_pos(t, r), l);
      RK_SYNC();  // the tile is free: fetch the next field (or the first of the next tile)
      if (g + 1 < a.n_groups)
        prefetch(tile, g + 1);
      else if (tile + gridDim.x < ntiles)
        prefetch(tile + gridDim.x, 0);
      F::forward(v, t, buf, tw);
      for (int q = a.g_begin[g]; q < a.g_begin[g + 1]; ++q) {
        const int m = a.term_m[q];
#pragma unroll
        for (int r = 0; r < S::R; ++r) w[r] = spec_mul(v[r], coef, N, m, F::spec_idx(t, r), a.reflect);
        F::inverse(w, t, buf, tw);
        const int p = a.term_io[q];
        T* out = a.out[p];
        // g_p = 0: every p outside chi; at regular nodes every p but x, y, z (the
        // node pair of this thread lies in group l / 2 of its tile row)
        const bool nongrad = p < 1 || p > 3;
        if (ok)
#pragma unroll
          for (int r = 0; r < S::R; ++r) {
            const int row = F::nat_pos(t, r);
            const bool zero = PW > 0 && (((oflag[row] | (nongrad ? rflag[row] : 0)) >> (l / 2)) & 1u);
            S::store(out, base + row * a.line_stride, zero ? cmk((T)0, (T)0) : w[r]);
          }
      }
    }
  }
}

template <typename T, int N, int L>
__global__ void __launch_bounds__(Strided<T, N, L>::THREADS, Strided<T, N, L>::MIN_BLOCKS_MERGE)
    k_strided_merge(const PassArgs<T> a, const int nbx, const long long ntiles, const int a16,
                    const __grid_constant__ TileMaps maps, const int tma_axis) {
  using S = Strided<T, N, L>;
  using F = typename S::F;
  RK_DYN_SMEM(unsigned char, smem);
  __shared__ uint64_t bar;
  TileFeed<T, N, L> feed{reinterpret_cast<T*>(smem), &bar, 0u, tma_axis};
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smem + S::SMEM_TILE);
  const int l = threadIdx.x % L, t = threadIdx.x / L;
  InterleavedBuf<T, F::N1, F::N2> buf{sm + l, L};
  feed.init();
  const int nterms = a.g_begin[a.n_groups];
  auto prefetch = [&](long long tile, int q) {
    const int x0 = (int)(tile % nbx) * S::ROW;
    const long long by = tile / nbx;
    const int in = a.term_io[q];
    feed.issue(maps, in, a.in[in] + x0 + by * a.other_stride, x0, (int)by, a.nx, a.line_stride, a16 != 0);
  };
  long long tile = blockIdx.x;
  if (tile < ntiles) prefetch(tile, 0);
  // multipliers and twiddles read through L1 (staging them in shared memory, as
  // the split pass does, measured slower here)
  const T* coef = a.coef;
  const cpx<T>* tw = a.tw;
  cpx<T> v[S::R], acc[S::R];
  for (; tile < ntiles; tile += gridDim.x) {
    const int x0 = (int)(tile % nbx) * S::ROW;
    const long long base = x0 + (tile / nbx) * a.other_stride + 2 * l;
    const bool ok = x0 + 2 * l < a.nx;
    for (int g = 0; g < a.n_groups; ++g) {
#pragma unroll
      for (int r = 0; r < S::R; ++r) acc[r] = cmk((T)0, (T)0);
      for (int q = a.g_begin[g]; q < a.g_begin[g + 1]; ++q) {
        const int m = a.term_m[q];
        if (!feed.wait(a.err, a.short_wait)) return;
#pragma unroll
        for (int r = 0; r < S::R; ++r) v[r] = S::at(feed.tile, F::nat_pos(t, r), l);
        RK_SYNC();
        if (q + 1 < nterms)
          prefetch(tile, q + 1);
        else if (tile + gridDim.x < ntiles)
          prefetch(tile + gridDim.x, 0);
        F::forward(v, t, buf, tw);
#pragma unroll
        for (int r = 0; r < S::R; ++r) acc[r] = acc[r] + spec_mul(v[r], coef, N, m, F::spec_idx(t, r), a.reflect);
      }
      F::inverse(acc, t, buf, tw);
      T* out = a.out[a.g_io[g]];
      if (ok)
#pragma unroll
        for (int r = 0; r < S::R; ++r) S::store(out, base + F::nat_pos(t, r) * a.line_stride, acc[r]);
    }
  }
}

// ------------------------------------------------------------------- x passes
// Block: LX pairs of rows times P threads per line; thread (t, l) with t fastest so
// that the P threads of a line read P consecutive x.
template <typename T, int N, int LX>
struct XPass {
  using F = LineFFT<T, N>;
  using B = PaddedBuf<T, F::N1, F::N2>;
  static constexpr int P = F::P, R = F::R;
  static constexpr int THREADS = LX * P;
  static constexpr size_t SMEM = (sizeof(cpx<T>) * (size_t)B::SIZE * LX + 127) / 128 * 128;
  // Row tiles of the bulk-copy feed: the block's 2 LX rows are contiguous in
  // memory; each row lands in shared memory with a 32-byte pad, so the two half
  // warps (rows 2l and 2l+2) read from disjoint bank halves.  Possible when a row
  // is a whole number of 16-byte units.
  static constexpr bool BULK = (N * sizeof(T)) % 16 == 0;
  static constexpr int ROWS = 2 * LX;
  static constexpr int PITCH = N + 32 / (int)sizeof(T);
  static constexpr size_t TILE = sizeof(T) * (size_t)ROWS * PITCH;
  static constexpr size_t SMEM_FEED = SMEM > 2 * TILE ? SMEM : 2 * TILE;
  // Bulk feed of the CG x merge: the block's rows of p (for p . Ap) and of the
  // output mask land in shared memory behind the transpose buffer while the block
  // transforms, so the epilogue reads neither from HBM.  Possible when a mask row
  // is a whole number of 16-byte units as well.
  static constexpr bool MERGE_BULK = BULK && N % 16 == 0;
  static constexpr size_t MASK_TILE = (size_t)ROWS * N;
  static constexpr size_t SMEM_MERGE_FEED = SMEM + TILE + MASK_TILE;
  // resident blocks per SM the register allocation must allow.  FP32 lines of at
  // most 12 values per thread, and N = 256: 5 blocks of 128 threads (102
  // registers; at N = 256 against 4 blocks: x split 64.2 -> 63.2 us, x merge
  // 82.1 -> 75.3 us); longer lines per thread keep the budget they need.
  static constexpr bool FIVE = sizeof(T) == 4 && (R <= 12 || N == 256);
  static constexpr int MIN_BLOCKS = FIVE ? 5 : (sizeof(T) == 4 ? 4 : 3);
  static constexpr int MIN_BLOCKS_MERGE = FIVE ? 5 : 1;
};

RK_DEV void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Bulk feed of the x passes: the rows [row0, row0 + rows) of up to two fields into
// row tiles, completion on one mbarrier (one transaction per call).
template <typename T, int N, int LX>
struct XFeed {
  using X = XPass<T, N, LX>;
  uint64_t* bar;
  uint32_t phase;
  RK_DEV void init() {
    if (threadIdx.x == 0) {
      mbar_init(bar, 1);
      mbar_init_fence();
    }
    RK_SYNC();
  }
  RK_DEV void issue(T* tileA, const T* srcA, T* tileB, const T* srcB, long long row0, int rows) {
    if (threadIdx.x < 32) {
      if (threadIdx.x == 0) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar, (uint32_t)(rows * N * sizeof(T) * (srcB ? 2 : 1)));
      }
      __syncwarp();
      for (int j = threadIdx.x; j < rows; j += 32) {
        bulk_g2s(tileA + j * X::PITCH, srcA + (row0 + j) * N, (uint32_t)(N * sizeof(T)), bar);
        if (srcB) bulk_g2s(tileB + j * X::PITCH, srcB + (row0 + j) * N, (uint32_t)(N * sizeof(T)), bar);
      }
    }
  }
  // false (uniformly) when the bounded wait gave up; the caller returns
  RK_DEV bool wait(int* err, int short_wait) {
    const bool ok = mbar_wait(bar, phase, short_wait ? 0u : kWaitLimit);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) flag_wait_error(err);
      mbar_wait(bar, phase ^ 1u);  // the copy still in flight, bounded
      return false;
    }
    return true;
  }
};

template <typename T>
RK_DEV T mask_of(const uint8_t* m, long long i) {
  return m ? (T)RK_LDG(m + i) : (T)1;
}

// The mask bytes of a block's 2*LX rows form one contiguous range (rows of
// consecutive pairs are consecutive); copy it to shared memory with 16-byte loads
// so the threads read their bytes from there.  Requires nx % 8 == 0 (the range
// then starts and ends on 16-byte boundaries of the mask array).
template <int N, int LX>
RK_DEV void stage_mask_rows(uint8_t* dst, const uint8_t* m, long long first_row, long long nrows_total) {
  const long long b0 = first_row * N;
  const long long nbytes = (long long)2 * LX * N;
  const long long avail = nrows_total * N - b0;
  const long long lim = nbytes < avail ? nbytes : avail;
  for (long long c = (long long)threadIdx.x * 16; c < lim; c += (long long)blockDim.x * 16) {
    if (c + 16 <= lim)
      *reinterpret_cast<uint4*>(dst + c) = RK_LDG(reinterpret_cast<const uint4*>(m + b0 + c));
    else  // the end of the array inside a 16-byte unit (a single row, 1D)
      for (long long b = c; b < lim; ++b) dst[b] = RK_LDG(m + b0 + b);
  }
  RK_SYNC();
}

// p . Ap of the x MERGE epilogue: block sum in a fixed tree order, one partial
// per block; the last block to finish sums the partials in block order (so the
// result is reproducible), sets pAp and alpha = rr / pAp (flag on breakdown) and
// resets the counter.
template <int THREADS, typename T>
__device__ __forceinline__ void cg_pap_reduce(double v, const PassArgs<T>& a) {
  // THREADS need not be a power of two (P = 6, 9, 10, 12 threads per line): the
  // top THREADS - POW2 values are folded onto the first ones before the tree.
  constexpr int POW2 = THREADS >= 512 ? 512 : THREADS >= 256 ? 256 : THREADS >= 128 ? 128 : THREADS >= 64 ? 64 : 32;
  static_assert(THREADS >= 32 && THREADS <= 1024 && THREADS < 2 * POW2, "block size");
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
  red[threadIdx.x] = v;
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
    const double pap = red[0];
    CGState* st = a.cg;
    st->pAp = pap;
    double al = 0.0;
    if (st->rz > 0.0) {
      if (pap > 0.0 && isfinite(pap))
        al = st->rz / pap;
      else
        st->flag = 1;
    }
    st->alpha = al;
    *a.counter = 0u;
  }
}

// The same reduction with warp shuffles for blocks of whole warps (fixed order as
// well: lanes in a butterfly, warps in index order, the partials in block order).
template <int THREADS, typename T>
__device__ __forceinline__ void cg_pap_reduce_warps(double v, const PassArgs<T>& a) {
  static_assert(THREADS % 32 == 0, "whole warps");
  constexpr int W = THREADS / 32;
  __shared__ double wsum[W];
  __shared__ bool last;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < W; ++w) s += wsum[w];
    a.partials[blockIdx.x] = s;
    __threadfence();
    last = atomicAdd(a.counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += THREADS) s += ((volatile double*)a.partials)[b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double pap = 0.0;
#pragma unroll
    for (int w = 0; w < W; ++w) pap += wsum[w];
    CGState* st = a.cg;
    st->pAp = pap;
    double al = 0.0;
    if (st->rz > 0.0) {
      if (pap > 0.0 && isfinite(pap))
        al = st->rz / pap;
      else
        st->flag = 1;
    }
    st->alpha = al;
    *a.counter = 0u;
  }
}

// FEED: the rows of r and p arrive by bulk async copies (the CG variant); a
// separate instantiation, so that the plain variant keeps the default shared
// memory carve-out (its twiddle and multiplier loads live in L1).
template <typename T, int N, int LX, bool FEED>
__global__ void __launch_bounds__(XPass<T, N, LX>::THREADS, XPass<T, N, LX>::MIN_BLOCKS)
    k_x_split(const PassArgs<T> a) {
  using X = XPass<T, N, LX>;
  using F = typename X::F;
  RK_DYN_SMEM(unsigned char, smem);
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smem);
  // the row tiles share the transpose buffer's memory: every tile read happens
  // before the forward transform, whose first barrier precedes any buffer write
  T* tileA = reinterpret_cast<T*>(smem);
  T* tileB = tileA + X::ROWS * X::PITCH;
  __shared__ uint64_t bar;
  const int t = threadIdx.x % X::P, l = threadIdx.x / X::P;
  const long long q = (long long)blockIdx.x * LX + l;  // row pair
  const long long nrows_all = (long long)a.ny * a.nz;
  const long long npairs = (nrows_all + 1) / 2;        // an odd last row pairs with a row of zeros
  const bool ok = q < npairs;
  const bool ok1 = 2 * q + 1 < nrows_all;
  const long long r0 = 2 * q * a.nx, r1 = r0 + a.nx;
  typename X::B buf{sm + (size_t)l * X::B::SIZE};
  cpx<T> v[X::R], w[X::R];
  const bool bulk = FEED && X::BULK && a.xbulk && a.n_groups == 1;
  const long long row0 = 2LL * blockIdx.x * LX;
  if (bulk) {
    XFeed<T, N, LX> feed{&bar, 0u};
    feed.init();
    const long long nrows = (long long)a.ny * a.nz;
    const int rows = (int)((nrows - row0) < X::ROWS ? (nrows - row0) : X::ROWS);
    feed.issue(tileA, a.cg_r ? a.cg_r : a.in[a.g_io[0]], tileB, a.cg_r ? a.cg_p : nullptr, row0, rows);
    if (!feed.wait(a.err, a.short_wait)) return;
  }
  const T* ra = tileA + (2 * l) * X::PITCH;  // this thread's rows in the tiles
  const T* rb = ra + X::PITCH;
  if (FEED && bulk && a.cg_r) {
    // the CG prologue from the row tiles, one group, outputs unmasked or masked
    const T be = (T)a.cg->beta;
    const T* pa = tileB + (2 * l) * X::PITCH;
#pragma unroll
    for (int r = 0; r < X::R; ++r) {
      const int xp = F::nat_pos(t, r);
      T p0 = (T)0, p1 = (T)0;
      if (ok) {
        p0 = ra[xp] + be * pa[xp];
        if (ok1) p1 = rb[xp] + be * pa[X::PITCH + xp];
        a.cg_p[r0 + xp] = p0;
        if (ok1) a.cg_p[r1 + xp] = p1;
      }
      v[r] = cmk(p0, p1);
    }
    F::forward(v, t, buf, a.tw);
    for (int qq = a.g_begin[0]; qq < a.g_begin[1]; ++qq) {
      const int m = a.term_m[qq];
#pragma unroll
      for (int r = 0; r < X::R; ++r) w[r] = spec_mul(v[r], a.coef, N, m, F::spec_idx(t, r), a.reflect);
      F::inverse(w, t, buf, a.tw);
      T* out = a.out[a.term_io[qq]];
      if (!ok) continue;
      if (a.out_mask) {
#pragma unroll
        for (int r = 0; r < X::R; ++r) {
          const int xp = F::nat_pos(t, r);
          out[r0 + xp] = w[r].x * (T)RK_LDG(a.out_mask + r0 + xp);
          if (ok1) out[r1 + xp] = w[r].y * (T)RK_LDG(a.out_mask + r1 + xp);
        }
      } else {
#pragma unroll
        for (int r = 0; r < X::R; ++r) {
          const int xp = F::nat_pos(t, r);
          out[r0 + xp] = w[r].x;
          if (ok1) out[r1 + xp] = w[r].y;
        }
      }
    }
    return;
  }
  for (int g = 0; g < a.n_groups; ++g) {
    const T* in = a.in[a.g_io[g]];
    if (a.cg_r) {
      // CG direction update fused into the load: p = r + beta p (Alg. 5, CG step)
      const T be = (T)a.cg->beta;
#pragma unroll
      for (int r = 0; r < X::R; ++r) {
        const int xp = F::nat_pos(t, r);
        T p0 = (T)0, p1 = (T)0;
        if (ok) {
          if (bulk) {
            p0 = ra[xp] + be * tileB[(2 * l) * X::PITCH + xp];
            if (ok1) p1 = rb[xp] + be * tileB[(2 * l + 1) * X::PITCH + xp];
          } else {
            p0 = a.cg_r[r0 + xp] + be * a.cg_p[r0 + xp];
            if (ok1) p1 = a.cg_r[r1 + xp] + be * a.cg_p[r1 + xp];
          }
          a.cg_p[r0 + xp] = p0;
          if (ok1) a.cg_p[r1 + xp] = p1;
        }
        v[r] = cmk(p0, p1);
      }
    } else if (a.in_mask && N % 8 == 0) {
      __shared__ __align__(16) uint8_t msk[2 * LX * N];
      stage_mask_rows<N, LX>(msk, a.in_mask, 2LL * blockIdx.x * LX, (long long)a.ny * a.nz);
#pragma unroll
      for (int r = 0; r < X::R; ++r) {
        const int xp = F::nat_pos(t, r);
        const T x0 = ok ? (bulk ? ra[xp] : RK_LDG(in + r0 + xp)) : (T)0;
        const T x1 = ok1 ? (bulk ? rb[xp] : RK_LDG(in + r1 + xp)) : (T)0;
        v[r] = cmk(x0 * (T)msk[(2 * l) * N + xp], ok1 ? x1 * (T)msk[(2 * l + 1) * N + xp] : (T)0);
      }
    } else {
#pragma unroll
      for (int r = 0; r < X::R; ++r) {
        const int xp = F::nat_pos(t, r);
        const T x0 = ok ? (bulk ? ra[xp] : RK_LDG(in + r0 + xp)) : (T)0;
        const T x1 = ok1 ? (bulk ? rb[xp] : RK_LDG(in + r1 + xp)) : (T)0;
        v[r] = ok ? cmk(x0 * mask_of<T>(a.in_mask, r0 + xp), ok1 ? x1 * mask_of<T>(a.in_mask, r1 + xp) : (T)0)
                  : cmk((T)0, (T)0);
      }
    }
    F::forward(v, t, buf, a.tw);
    for (int qq = a.g_begin[g]; qq < a.g_begin[g + 1]; ++qq) {
      const int m = a.term_m[qq];
#pragma unroll
      for (int r = 0; r < X::R; ++r) w[r] = spec_mul(v[r], a.coef, N, m, F::spec_idx(t, r), a.reflect);
      F::inverse(w, t, buf, a.tw);
      T* out = a.out[a.term_io[qq]];
      if (ok)
#pragma unroll
        for (int r = 0; r < X::R; ++r) {
          const int xp = F::nat_pos(t, r);
          out[r0 + xp] = w[r].x * mask_of<T>(a.out_mask, r0 + xp);
          if (ok1) out[r1 + xp] = w[r].y * mask_of<T>(a.out_mask, r1 + xp);
        }
    }
  }
}

// FEED: the CG variant (one group, an output mask, p . Ap epilogue) with the
// block's rows of p and of the mask arriving by bulk async copies while the block
// transforms.
template <typename T, int N, int LX, bool FEED>
__global__ void __launch_bounds__(XPass<T, N, LX>::THREADS, XPass<T, N, LX>::MIN_BLOCKS_MERGE)
    k_x_merge(const PassArgs<T> a) {
  using X = XPass<T, N, LX>;
  using F = typename X::F;
  RK_DYN_SMEM(unsigned char, smem);
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smem);
  const int t = threadIdx.x % X::P, l = threadIdx.x / X::P;
  const long long q = (long long)blockIdx.x * LX + l;
  const long long nrows_all = (long long)a.ny * a.nz;
  const long long npairs = (nrows_all + 1) / 2;  // an odd last row pairs with a row of zeros
  const bool ok = q < npairs;
  const bool ok1 = 2 * q + 1 < nrows_all;
  const long long r0 = 2 * q * a.nx, r1 = r0 + a.nx;
  typename X::B buf{sm + (size_t)l * X::B::SIZE};
  cpx<T> v[X::R], acc[X::R];
  if (FEED) {
    T* ptile = reinterpret_cast<T*>(smem + X::SMEM);
    uint8_t* mtile = smem + X::SMEM + X::TILE;
    __shared__ uint64_t bar;
    const long long row0 = 2LL * blockIdx.x * LX;
    const int rows = (int)((nrows_all - row0) < X::ROWS ? (nrows_all - row0) : X::ROWS);
    if (threadIdx.x == 0) {
      mbar_init(&bar, 1);
      mbar_init_fence();
    }
    RK_SYNC();
    if (threadIdx.x < 32) {
      if (threadIdx.x == 0) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bar, (uint32_t)(rows * N * sizeof(T) + rows * N));
      }
      __syncwarp();
      for (int j = threadIdx.x; j < rows; j += 32)
        bulk_g2s(ptile + j * X::PITCH, a.cg_p + (row0 + j) * N, (uint32_t)(N * sizeof(T)), &bar);
      if (threadIdx.x == 0) bulk_g2s(mtile, a.out_mask + row0 * N, (uint32_t)(rows * N), &bar);
    }
#pragma unroll
    for (int r = 0; r < X::R; ++r) acc[r] = cmk((T)0, (T)0);
    for (int qq = a.g_begin[0]; qq < a.g_begin[1]; ++qq) {
      const T* in = a.in[a.term_io[qq]];
      const int m = a.term_m[qq];
#pragma unroll
      for (int r = 0; r < X::R; ++r) {
        const int xp = F::nat_pos(t, r);
        v[r] = cmk(ok ? RK_LDG(in + r0 + xp) : (T)0, ok1 ? RK_LDG(in + r1 + xp) : (T)0);
      }
      F::forward(v, t, buf, a.tw);
#pragma unroll
      for (int r = 0; r < X::R; ++r) acc[r] = acc[r] + spec_mul(v[r], a.coef, N, m, F::spec_idx(t, r), a.reflect);
    }
    F::inverse(acc, t, buf, a.tw);
    // the tiles: bounded wait; a thread whose wait runs out records it and waits
    // (bounded) for the copies still in flight.  The block then completes as usual
    // (its output is invalid and the call reports the time-out), so that it still
    // takes part in the p . Ap reduction and the counter ends the launch reset.
    if (!mbar_wait(&bar, 0u, a.short_wait ? 0u : kWaitLimit)) {
      flag_wait_error(a.err);
      mbar_wait(&bar, 0u);
    }
    // (rows past the end of the box: their mask bytes are not loaded, and neither
    // their outputs nor their p . Ap terms are used)
    const uint8_t* mk = mtile + (2 * l) * N;
#pragma unroll
    for (int r = 0; r < X::R; ++r) {
      const int xp = F::nat_pos(t, r);
      acc[r] = pmul(acc[r], cmk((T)mk[xp], (T)mk[N + xp]));
    }
    T* out = a.out[a.g_io[0]];
    if (ok)
#pragma unroll
      for (int r = 0; r < X::R; ++r) {
        const int xp = F::nat_pos(t, r);
        out[r0 + xp] = acc[r].x;
        if (ok1) out[r1 + xp] = acc[r].y;
      }
    DotAccPair<T> dot;
    const T* pa = ptile + (2 * l) * X::PITCH;
    if (ok)
#pragma unroll
      for (int r = 0; r < X::R; ++r) {
        const int xp = F::nat_pos(t, r);
        dot.add(cmk(pa[xp], ok1 ? pa[X::PITCH + xp] : (T)0), acc[r]);
      }
    if constexpr (X::THREADS % 32 == 0)
      cg_pap_reduce_warps<X::THREADS>(dot.value(), a);
    else
      cg_pap_reduce<X::THREADS>(dot.value(), a);
    return;
  }
  for (int g = 0; g < a.n_groups; ++g) {
#pragma unroll
    for (int r = 0; r < X::R; ++r) acc[r] = cmk((T)0, (T)0);
    for (int qq = a.g_begin[g]; qq < a.g_begin[g + 1]; ++qq) {
      const T* in = a.in[a.term_io[qq]];
      const int m = a.term_m[qq];
#pragma unroll
      for (int r = 0; r < X::R; ++r) {
        const int xp = F::nat_pos(t, r);
        v[r] = cmk(ok ? RK_LDG(in + r0 + xp) : (T)0, ok1 ? RK_LDG(in + r1 + xp) : (T)0);
      }
      F::forward(v, t, buf, a.tw);
#pragma unroll
      for (int r = 0; r < X::R; ++r) acc[r] = acc[r] + spec_mul(v[r], a.coef, N, m, F::spec_idx(t, r), a.reflect);
    }
    F::inverse(acc, t, buf, a.tw);
    T* out = a.out[a.g_io[g]];
    __shared__ __align__(16) uint8_t msk[2 * LX * N];
    if (a.out_mask) {
      if (N % 8 == 0) {
        stage_mask_rows<N, LX>(msk, a.out_mask, 2LL * blockIdx.x * LX, (long long)a.ny * a.nz);
      } else {
        for (int j = threadIdx.x; j < 2 * LX * N; j += blockDim.x) {
          const long long i = 2LL * blockIdx.x * LX * N + j;
          msk[j] = i < (long long)a.ny * a.nz * N ? RK_LDG(a.out_mask + i) : (uint8_t)0;
        }
        RK_SYNC();
      }
    }
    if (a.out_mask)
#pragma unroll
      for (int r = 0; r < X::R; ++r) {
        const int xp = F::nat_pos(t, r);
        acc[r] = pmul(acc[r], cmk((T)msk[(2 * l) * N + xp], (T)msk[(2 * l + 1) * N + xp]));
      }
    if (ok)
#pragma unroll
      for (int r = 0; r < X::R; ++r) {
        const int xp = F::nat_pos(t, r);
        out[r0 + xp] = acc[r].x;
        if (ok1) out[r1 + xp] = acc[r].y;
      }
    if (a.cg_p) {
      DotAccPair<T> dot;
      if (ok)
#pragma unroll
        for (int r = 0; r < X::R; ++r) {
          const int xp = F::nat_pos(t, r);
          dot.add(cmk(a.cg_p[r0 + xp], ok1 ? a.cg_p[r1 + xp] : (T)0), acc[r]);
        }
      cg_pap_reduce<X::THREADS>(dot.value(), a);
    }
  }
}

// The CG x merge of two terms (the linear basis) with every row it reads arriving
// by bulk async copies: the first input into the transpose buffer (read before the
// first transform writes it), the second into a row tile, and p and the output
// mask into that tile once the second input has been read, while the block
// transforms.  Four blocks per SM (128 registers): at N = 256, 74.3 us against
// 75-83 us for the variant that loads the inputs with per-thread loads.
template <typename T, int N, int LX>
__global__ void __launch_bounds__(XPass<T, N, LX>::THREADS, 4) k_x_merge_fed2(const PassArgs<T> a) {
  using X = XPass<T, N, LX>;
  using F = typename X::F;
  static_assert(X::SMEM >= X::TILE, "the first input tile lives in the transpose buffer");
  RK_DYN_SMEM(unsigned char, smem);
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smem);
  T* tileA = reinterpret_cast<T*>(smem);
  T* tileB = reinterpret_cast<T*>(smem + X::SMEM);
  uint8_t* mtile = smem + X::SMEM + X::TILE;
  __shared__ uint64_t bar[3];
  const int t = threadIdx.x % X::P, l = threadIdx.x / X::P;
  const long long q = (long long)blockIdx.x * LX + l;
  const long long nrows_all = (long long)a.ny * a.nz;
  const long long npairs = (nrows_all + 1) / 2;  // an odd last row pairs with a row of zeros
  const bool ok = q < npairs;
  const bool ok1 = 2 * q + 1 < nrows_all;
  const long long r0 = 2 * q * a.nx, r1 = r0 + a.nx;
  const long long row0 = 2LL * blockIdx.x * LX;
  const int rows = (int)((nrows_all - row0) < X::ROWS ? (nrows_all - row0) : X::ROWS);
  typename X::B buf{sm + (size_t)l * X::B::SIZE};
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init(&bar[2], 1);
    mbar_init_fence();
  }
  RK_SYNC();
  const int q0 = a.g_begin[0];
  const T* in0 = a.in[a.term_io[q0]];
  const T* in1 = a.in[a.term_io[q0 + 1]];
  const uint32_t row_bytes = (uint32_t)(N * sizeof(T));
  if (threadIdx.x < 32) {
    if (threadIdx.x == 0) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&bar[0], (uint32_t)rows * row_bytes);
      mbar_arrive_expect_tx(&bar[1], (uint32_t)rows * row_bytes);
    }
    __syncwarp();
    for (int j = threadIdx.x; j < rows; j += 32) bulk_g2s(tileA + j * X::PITCH, in0 + (row0 + j) * N, row_bytes, &bar[0]);
    for (int j = threadIdx.x; j < rows; j += 32) bulk_g2s(tileB + j * X::PITCH, in1 + (row0 + j) * N, row_bytes, &bar[1]);
  }
  // bounded waits: a thread whose wait runs out records it and waits (bounded) for
  // the copy still in flight; the block then completes as usual (its output is
  // invalid and the call reports the time-out) and takes part in the reduction
  auto wait = [&](int k, bool first) {
    if (!mbar_wait(&bar[k], 0u, (first && a.short_wait) ? 0u : kWaitLimit)) {
      flag_wait_error(a.err);
      mbar_wait(&bar[k], 0u);
    }
  };
  cpx<T> v[X::R], acc[X::R];
  wait(0, true);
  {
    const T* ta = tileA + (2 * l) * X::PITCH;
#pragma unroll
    for (int r = 0; r < X::R; ++r) {
      const int xp = F::nat_pos(t, r);
      v[r] = cmk(ok ? ta[xp] : (T)0, ok1 ? ta[X::PITCH + xp] : (T)0);
    }
  }
  F::forward(v, t, buf, a.tw);
#pragma unroll
  for (int r = 0; r < X::R; ++r) acc[r] = spec_mul(v[r], a.coef, N, a.term_m[q0], F::spec_idx(t, r), a.reflect);
  wait(1, false);
  {
    const T* tb = tileB + (2 * l) * X::PITCH;
#pragma unroll
    for (int r = 0; r < X::R; ++r) {
      const int xp = F::nat_pos(t, r);
      v[r] = cmk(ok ? tb[xp] : (T)0, ok1 ? tb[X::PITCH + xp] : (T)0);
    }
  }
  RK_SYNC();  // the second input is in registers: p and the mask may land in its tile
  if (threadIdx.x < 32) {
    if (threadIdx.x == 0) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&bar[2], (uint32_t)rows * row_bytes + (uint32_t)(rows * N));
    }
    __syncwarp();
    for (int j = threadIdx.x; j < rows; j += 32) bulk_g2s(tileB + j * X::PITCH, a.cg_p + (row0 + j) * N, row_bytes, &bar[2]);
    if (threadIdx.x == 0) bulk_g2s(mtile, a.out_mask + row0 * N, (uint32_t)(rows * N), &bar[2]);
  }
  F::forward(v, t, buf, a.tw);
#pragma unroll
  for (int r = 0; r < X::R; ++r) acc[r] = acc[r] + spec_mul(v[r], a.coef, N, a.term_m[q0 + 1], F::spec_idx(t, r), a.reflect);
  F::inverse(acc, t, buf, a.tw);
  wait(2, false);
  // (rows past the end of the box: their mask bytes are not loaded, and neither
  // their outputs nor their p . Ap terms are used)
  const uint8_t* mk = mtile + (2 * l) * N;
#pragma unroll
  for (int r = 0; r < X::R; ++r) {
    const int xp = F::nat_pos(t, r);
    acc[r] = pmul(acc[r], cmk((T)mk[xp], (T)mk[N + xp]));
  }
  T* out = a.out[a.g_io[0]];
  if (ok)
#pragma unroll
    for (int r = 0; r < X::R; ++r) {
      const int xp = F::nat_pos(t, r);
      out[r0 + xp] = acc[r].x;
      if (ok1) out[r1 + xp] = acc[r].y;
    }
  DotAccPair<T> dot;
  const T* pa = tileB + (2 * l) * X::PITCH;
  if (ok)
#pragma unroll
    for (int r = 0; r < X::R; ++r) {
      const int xp = F::nat_pos(t, r);
      dot.add(cmk(pa[xp], ok1 ? pa[X::PITCH + xp] : (T)0), acc[r]);
    }
  if constexpr (X::THREADS % 32 == 0)
    cg_pap_reduce_warps<X::THREADS>(dot.value(), a);
  else
    cg_pap_reduce<X::THREADS>(dot.value(), a);
}

// ------------------------------------------------------- fused z pass (Alg. 2-4)
enum ZMode { Z_STIFF = 0, Z_EVAL_U = 1, Z_TRANSPOSE_U = 2 };

template <typename T>
struct ZArgs {
  // groups of basis indices p sharing (alpha_x, alpha_y); terms carry alpha_z and p
  int n_groups;
  int g_begin[kMaxOut + 1];
  int term_mz[kMaxOut];
  int term_p[kMaxOut];
  const T* in[kMaxIn];   // Z_STIFF, Z_EVAL_U: one field per group (after x, y passes)
  T* out[kMaxIn];        // Z_STIFF, Z_TRANSPOSE_U: one field per group
  const T* in1;          // Z_TRANSPOSE_U: the input field (y)
  T* out1;               // Z_EVAL_U: the output field (u)
  const T* b;            // coefficient fields [4][s][nbox]: b^0, b^x, b^y, b^z
  int s;
  const T* wfield;       // Z_STIFF: chi*V;  Z_TRANSPOSE_U: optional weight (chi*V for f^r)
  const uint8_t* mask;   // Z_EVAL_U: output mask (chi);  Z_TRANSPOSE_U: optional weight (chi)
  const T* coef;         // z-axis spectral multipliers
  const cpx<T>* tw;      // z-axis twiddles
  int nx, ny, nz;
  long long nbox;
};

template <typename T, int N, int L, int MODE>
struct ZPass {
  using S = Strided<T, N, L>;
  using F = typename S::F;
  static constexpr int P = F::P, R = F::R;
  static constexpr int THREADS = L * P;
  static constexpr size_t SMEM_BUF = sizeof(cpx<T>) * (size_t)N * L;
  static constexpr size_t SMEM = SMEM_BUF * (MODE == Z_STIFF ? 4 : 1);
};

template <typename T, int N, int L, int MODE>
__global__ void __launch_bounds__(ZPass<T, N, L, MODE>::THREADS) k_z_fused(const ZArgs<T> a) {
  using Z = ZPass<T, N, L, MODE>;
  using S = typename Z::S;
  using F = typename Z::F;
  RK_DYN_SMEM(cpx<T>, sm);
  const int l = threadIdx.x % L, t = threadIdx.x / L;
  const int x = blockIdx.x * 2 * L + 2 * l;
  const bool ok = x < a.nx;
  const long long zs = (long long)a.nx * a.ny;  // line stride along z
  const long long base = (long long)x + (long long)blockIdx.y * a.nx;
  InterleavedBuf<T, F::N1, F::N2> buf{sm + l, L};
  // per-thread accumulators A^x, A^y, A^z (Eq. 90) at the thread's own nodes
  cpx<T>* Acc = sm + (size_t)N * L;
  auto A = [&](int k, int r) -> cpx<T>& { return Acc[((size_t)k * N + F::nat_pos(t, r)) * L + l]; };
  auto coef_pair = [&](int which, int p, long long off) -> cpx<T> {
    return ok ? S::load(a.b + ((long long)which * a.s + p) * a.nbox, off) : cmk((T)0, (T)0);
  };
  cpx<T> v[Z::R], w[Z::R];

  if (MODE == Z_STIFF || MODE == Z_EVAL_U) {
    cpx<T> u[MODE == Z_EVAL_U ? Z::R : 1];
    if (MODE == Z_STIFF) {
#pragma unroll
      for (int r = 0; r < Z::R; ++r) A(0, r) = A(1, r) = A(2, r) = cmk((T)0, (T)0);
    } else {
#pragma unroll
      for (int r = 0; r < Z::R; ++r) u[r] = cmk((T)0, (T)0);
    }
    // forward chain: D_p = conv_z(E_{ax,ay}, T_{az})   (Alg. 2 loop 1, Alg. 3)
    for (int g = 0; g < a.n_groups; ++g) {
      const T* in = a.in[g];
#pragma unroll
      for (int r = 0; r < Z::R; ++r) v[r] = ok ? S::load(in, base + F::nat_pos(t, r) * zs) : cmk((T)0, (T)0);
      F::forward(v, t, buf, a.tw);
      for (int q = a.g_begin[g]; q < a.g_begin[g + 1]; ++q) {
        const int mz = a.term_mz[q], p = a.term_p[q];
#pragma unroll
        for (int r = 0; r < Z::R; ++r) w[r] = spec_mul(v[r], a.coef, N, mz, F::spec_idx(t, r), 0);
        F::inverse(w, t, buf, a.tw);
#pragma unroll
        for (int r = 0; r < Z::R; ++r) {
          const long long off = base + F::nat_pos(t, r) * zs;
          if (MODE == Z_STIFF) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              cpx<T> bk = coef_pair(1 + k, p, off);
              cpx<T>& Ak = A(k, r);
              Ak = pfma(bk, w[r], Ak);
            }
          } else {
            cpx<T> b0 = coef_pair(0, p, off);
            u[r] = pfma(b0, w[r], u[r]);
          }
        }
      }
    }
    if (MODE == Z_EVAL_U) {
      if (ok)
#pragma unroll
        for (int r = 0; r < Z::R; ++r) {
          const long long off = base + F::nat_pos(t, r) * zs;
          T m0 = a.mask ? (T)a.mask[off] : (T)1, m1 = a.mask ? (T)a.mask[off + 1] : (T)1;
          S::store(a.out1, off, cmk(u[r].x * m0, u[r].y * m1));
        }
      return;
    }
  }

  // reflected chain: G_{ax,ay} = sum_az conv_z(g_p, Tbar_az)   (Alg. 2 loop 2, Alg. 4)
  cpx<T> y[MODE == Z_TRANSPOSE_U ? Z::R : 1];
  if (MODE == Z_TRANSPOSE_U) {
#pragma unroll
    for (int r = 0; r < Z::R; ++r) {
      const long long off = base + F::nat_pos(t, r) * zs;
      cpx<T> yv = ok ? S::load(a.in1, off) : cmk((T)0, (T)0);
      if (ok && a.wfield) {
        cpx<T> wv = S::load(a.wfield, off);
        yv = pmul(yv, wv);
      }
      if (ok && a.mask) yv = cmk(yv.x * (T)a.mask[off], yv.y * (T)a.mask[off + 1]);
      y[r] = yv;
    }
  }
  for (int g = 0; g < a.n_groups; ++g) {
    cpx<T> acc[Z::R];
#pragma unroll
    for (int r = 0; r < Z::R; ++r) acc[r] = cmk((T)0, (T)0);
    for (int q = a.g_begin[g]; q < a.g_begin[g + 1]; ++q) {
      const int mz = a.term_mz[q], p = a.term_p[q];
#pragma unroll
      for (int r = 0; r < Z::R; ++r) {
        const long long off = base + F::nat_pos(t, r) * zs;
        if (MODE == Z_STIFF) {
          // g_p = chi V sum_k b^k_p A^k   (Eq. 91: C^k_p = chi V b^k_p)
          cpx<T> cv = ok ? S::load(a.wfield, off) : cmk((T)0, (T)0);
          cpx<T> s = cmk((T)0, (T)0);
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            cpx<T> bk = coef_pair(1 + k, p, off);
            cpx<T> Ak = A(k, r);
            s = pfma(bk, Ak, s);
          }
          v[r] = pmul(cv, s);
        } else {
          // g_p = w b^0_p y   (Eq. 92 with w = chi V; its transpose use with w = chi)
          cpx<T> b0 = coef_pair(0, p, off);
          v[r] = pmul(b0, y[r]);
        }
      }
      F::forward(v, t, buf, a.tw);
#pragma unroll
      for (int r = 0; r < Z::R; ++r) acc[r] = acc[r] + spec_mul(v[r], a.coef, N, mz, F::spec_idx(t, r), 1);
    }
    F::inverse(acc, t, buf, a.tw);
    if (ok)
#pragma unroll
      for (int r = 0; r < Z::R; ++r) S::store(a.out[g], base + F::nat_pos(t, r) * zs, acc[r]);
  }
}

}  // namespace rk
