// rk_vec.cu -- per-node moment solve of Alg. 1 and the vector kernels of the
// conjugate-gradient driver (Alg. 5).
#include "rk_internal.cuh"
#include "rk_moment.cuh"

#include <cstring>

namespace rk {

std::atomic<long long> g_launches{0};

bool supported_length(int n) {
  switch (n) {
    case 8: case 16: case 32: case 36: case 48: case 64: case 72: case 96: case 100: case 128: case 144: case 162:
    case 256: return true;
    default: return false;
  }
}

cudaError_t launch_moment_solve(const MomentArgs& a, cudaStream_t s) {
  const long long nb = (a.nbox + 127) / 128;
  const unsigned grid = (unsigned)(nb < 152 * 64 ? nb : 152 * 64);
  switch (a.s) {  // the basis sizes of degree 1 and 2 in 1D, 2D and 3D
    case 2: count_launch(); k_moment_solve<2><<<grid, 128, 0, s>>>(a); break;
    case 3: count_launch(); k_moment_solve<3><<<grid, 128, 0, s>>>(a); break;
    case 4: count_launch(); k_moment_solve<4><<<grid, 128, 0, s>>>(a); break;
    case 6: count_launch(); k_moment_solve<6><<<grid, 128, 0, s>>>(a); break;
    case 10: count_launch(); k_moment_solve<10><<<grid, 128, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------- set-up: masks and the Eq. 66 gap
// chi and chi_gamma to 0/1 in place (chi_gamma restricted to chi), chi_omega = chi
// and not chi_gamma, the count of chi nodes (scratch[0..7]) and the occupied
// indices of each axis (scratch[16 + i], [16 + n0 + j], [16 + n0 + n1 + k]); each
// block gathers its occupied indices in shared memory first.
__global__ void k_setup_masks(uint8_t* chi, uint8_t* gam, uint8_t* omg, int n0, int n1, int n2, long long n,
                              uint8_t* scratch) {
  extern __shared__ uint8_t occ[];
  const int np = n0 + n1 + n2;
  for (int t = threadIdx.x; t < np; t += blockDim.x) occ[t] = 0;
  __syncthreads();
  unsigned cnt = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const uint8_t x = chi[i] ? 1 : 0;
    const uint8_t g = (gam[i] && x) ? 1 : 0;
    chi[i] = x;
    gam[i] = g;
    omg[i] = x & (uint8_t)(1 - g);
    if (x) {
      ++cnt;
      const long long jk = i / n0;
      occ[i - jk * n0] = 1;
      occ[n0 + (int)(jk % n1)] = 1;
      occ[n0 + n1 + (int)(jk / n1)] = 1;
    }
  }
  cnt = __reduce_add_sync(0xffffffffu, cnt);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(reinterpret_cast<unsigned long long*>(scratch), (unsigned long long)cnt);
  __syncthreads();
  for (int t = threadIdx.x; t < np; t += blockDim.x)
    if (occ[t]) scratch[16 + t] = 1;
}

// Eq. 66 in discrete form: along each axis of the problem the occupied indices must
// leave a circular run of at least `reach` empty ones, so that no two nodes of
// Omega are within the support through the periodic boundary; scratch[8..11] = 1
// if not.
__global__ void k_setup_gap(uint8_t* scratch, int n0, int n1, int n2, int dim, int reach) {
  const int ax = threadIdx.x;
  if (ax >= dim) return;
  const int n = ax == 0 ? n0 : (ax == 1 ? n1 : n2);
  const uint8_t* o = scratch + 16 + (ax == 0 ? 0 : (ax == 1 ? n0 : n0 + n1));
  int best = 0, run = 0;
  bool any = false;
  for (int t = 0; t < 2 * n; ++t) {
    if (o[t % n]) {
      any = true;
      run = 0;
    } else {
      run = min(run + 1, n);
      best = max(best, run);
    }
  }
  if (any && best < reach) *reinterpret_cast<int*>(scratch + 8) = 1;
}

cudaError_t launch_setup_masks(uint8_t* chi, uint8_t* gam, uint8_t* omg, const int n[3], int dim, int reach,
                               uint8_t* scratch, cudaStream_t s) {
  const long long nbox = (long long)n[0] * n[1] * n[2];
  const int np = n[0] + n[1] + n[2];
  cudaError_t e = cudaMemsetAsync(scratch, 0, (size_t)16 + np, s);
  if (e != cudaSuccess) return e;
  const long long nb = (nbox + 255) / 256;
  count_launch();
  k_setup_masks<<<(unsigned)(nb < 152 * 8 ? nb : 152 * 8), 256, np, s>>>(chi, gam, omg, n[0], n[1], n[2], nbox, scratch);
  count_launch();
  k_setup_gap<<<1, 32, 0, s>>>(scratch, n[0], n[1], n[2], dim, reach);
  return cudaGetLastError();
}

// ------------------------------------------------- coefficient compression
__global__ void k_erode(uint8_t* out, const uint8_t* in, int axis, int r, int nx, int ny, int nz) {
  const long long n = (long long)nx * ny * nz;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((long long)nx * ny));
    const int len = axis == 0 ? nx : (axis == 1 ? ny : nz);
    const int c = axis == 0 ? x : (axis == 1 ? y : z);
    const long long stride = axis == 0 ? 1 : (axis == 1 ? nx : (long long)nx * ny);
    uint8_t ok = in[i];
    for (int o = 1; o <= r && ok; ++o) {
      const int cp = (c + o) % len, cm = ((c - o) % len + len) % len;
      ok = in[i + (long long)(cp - c) * stride] && in[i + (long long)(cm - c) * stride];
    }
    out[i] = ok ? 1 : 0;
  }
}
cudaError_t launch_erode(uint8_t* out, const uint8_t* in, int axis, int r, const int n[3], cudaStream_t s) {
  const long long nb = ((long long)n[0] * n[1] * n[2] + 255) / 256;
  count_launch();
  k_erode<<<(unsigned)(nb < 152 * 32 ? nb : 152 * 32), 256, 0, s>>>(out, in, axis, r, n[0], n[1], n[2]);
  return cudaGetLastError();
}

__global__ void k_classify(uint8_t* cls, const uint8_t* chi, const uint8_t* er, const double* V, double vreg,
                           long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    cls[i] = !chi[i] ? 0 : ((er[i] && V[i] == vreg) ? 1 : 2);
}
cudaError_t launch_classify(uint8_t* cls, const uint8_t* chi, const uint8_t* eroded, const double* V, double vreg,
                            long long n, cudaStream_t s) {
  const long long nb = (n + 255) / 256;
  count_launch();
  k_classify<<<(unsigned)(nb < 152 * 32 ? nb : 152 * 32), 256, 0, s>>>(cls, chi, eroded, V, vreg, n);
  return cudaGetLastError();
}

// Classes of the 4-node groups g (nodes 4g .. 4g + 3): 0 all regular (cidx == 0),
// 1 all outside chi (cidx == -1), 2 any other; bit g of regbits / outbits marks
// classes 0 / 1.  One thread per 32 groups.
__global__ void k_group_class(uint8_t* gcls, uint32_t* regbits, uint32_t* outbits, const int* cidx, long long ngroups) {
  const long long nwords = (ngroups + 31) / 32;
  for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += (long long)gridDim.x * blockDim.x) {
    uint32_t rv = 0u, ov = 0u;
    for (int j = 0; j < 32; ++j) {
      const long long g = w * 32 + j;
      if (g >= ngroups) break;
      const int4 c = *reinterpret_cast<const int4*>(cidx + 4 * g);
      const bool reg = c.x == 0 && c.y == 0 && c.z == 0 && c.w == 0;
      const bool out = c.x == -1 && c.y == -1 && c.z == -1 && c.w == -1;
      rv |= (reg ? 1u : 0u) << j;
      ov |= (out ? 1u : 0u) << j;
      gcls[g] = reg ? 0 : (out ? 1 : 2);
    }
    regbits[w] = rv;
    outbits[w] = ov;
  }
}
cudaError_t launch_group_class(uint8_t* gcls, uint32_t* regbits, uint32_t* outbits, const int* cidx, long long ngroups,
                               cudaStream_t s) {
  const long long nwords = (ngroups + 31) / 32;
  const long long nb = (nwords + 255) / 256;
  count_launch();
  k_group_class<<<(unsigned)(nb < 152 * 32 ? (nb > 0 ? nb : 1) : 152 * 32), 256, 0, s>>>(gcls, regbits, outbits, cidx,
                                                                                         ngroups);
  return cudaGetLastError();
}

// ordered list of the entries with cls == 2 (offsets: exclusive scan of the
// per-block counts of k_count_irregular); one block per kScanBlock entries
__global__ void __launch_bounds__(256) k_list_compact(const uint8_t* cls, const int* offsets, long long n, int* list) {
  __shared__ int sh[256];
  const long long b0 = (long long)blockIdx.x * kScanBlock;
  constexpr int PER = kScanBlock / 256;
  int c = 0;
  for (int j = 0; j < PER; ++j) {
    const long long i = b0 + threadIdx.x * PER + j;
    c += (i < n && cls[i] == 2) ? 1 : 0;
  }
  sh[threadIdx.x] = c;
  __syncthreads();
  for (int o = 1; o < 256; o <<= 1) {
    const int v = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += v;
    __syncthreads();
  }
  int pos = offsets[blockIdx.x] + sh[threadIdx.x] - c;
  for (int j = 0; j < PER; ++j) {
    const long long i = b0 + threadIdx.x * PER + j;
    if (i < n && cls[i] == 2) list[pos++] = (int)i;
  }
}
cudaError_t launch_list_compact(const uint8_t* cls, const int* offsets, long long n, int* list, cudaStream_t s) {
  const long long nblk = (n + kScanBlock - 1) / kScanBlock;
  count_launch();
  k_list_compact<<<(unsigned)nblk, 256, 0, s>>>(cls, offsets, n, list);
  return cudaGetLastError();
}

// block b counts the irregular nodes of [b*kScanBlock, (b+1)*kScanBlock)
__global__ void __launch_bounds__(256) k_count_irregular(const uint8_t* cls, long long n, int* counts) {
  __shared__ int sh[256];
  const long long b0 = (long long)blockIdx.x * kScanBlock;
  int c = 0;
  for (int j = threadIdx.x; j < kScanBlock; j += 256) {
    const long long i = b0 + j;
    c += (i < n && cls[i] == 2) ? 1 : 0;
  }
  sh[threadIdx.x] = c;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) counts[blockIdx.x] = sh[0];
}
cudaError_t launch_count_irregular(const uint8_t* cls, long long n, int* counts, cudaStream_t s) {
  const long long nblk = (n + kScanBlock - 1) / kScanBlock;
  count_launch();
  k_count_irregular<<<(unsigned)nblk, 256, 0, s>>>(cls, n, counts);
  return cudaGetLastError();
}

// exclusive scan of nblk counts by one block (sequential chunks, fixed order)
__global__ void __launch_bounds__(1024) k_scan_counts(int* counts, int nblk, int* total) {
  __shared__ int part[1024];
  const int per = (nblk + 1023) / 1024;
  const int b = threadIdx.x * per;
  int sum = 0;
  for (int j = 0; j < per && b + j < nblk; ++j) sum += counts[b + j];
  part[threadIdx.x] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int t = 0; t < 1024; ++t) {
      const int v = part[t];
      part[t] = run;
      run += v;
    }
    *total = run;
  }
  __syncthreads();
  int run = part[threadIdx.x];
  for (int j = 0; j < per && b + j < nblk; ++j) {
    const int v = counts[b + j];
    counts[b + j] = run;
    run += v;
  }
}
cudaError_t launch_scan_counts(int* counts, int nblk, int* total, cudaStream_t s) {
  count_launch();
  k_scan_counts<<<1, 1024, 0, s>>>(counts, nblk, total);
  return cudaGetLastError();
}

// one block per compaction block: ordered compaction of the irregular nodes
template <typename T>
__global__ void __launch_bounds__(256) k_compact(const uint8_t* cls, const int* offsets, long long n, int* cidx,
                                                const T* b, int s, const T* chiV, T* tab, long long n_irr) {
  __shared__ int sh[256];
  const long long b0 = (long long)blockIdx.x * kScanBlock;
  constexpr int PER = kScanBlock / 256;
  int flags[PER];
  int c = 0;
  for (int j = 0; j < PER; ++j) {
    const long long i = b0 + threadIdx.x * PER + j;
    flags[j] = (i < n && cls[i] == 2) ? 1 : 0;
    c += flags[j];
  }
  sh[threadIdx.x] = c;
  __syncthreads();
  // inclusive scan over the 256 thread counts (Hillis-Steele)
  for (int o = 1; o < 256; o <<= 1) {
    const int v = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += v;
    __syncthreads();
  }
  int pos = offsets[blockIdx.x] + sh[threadIdx.x] - c;
  const int ncoef = 3 * s + 1;
  const int pitch = ctab_pitch<T>(s);
  for (int j = 0; j < PER; ++j) {
    const long long i = b0 + threadIdx.x * PER + j;
    if (i >= n) break;
    const uint8_t k = cls[i];
    if (k == 0) {
      cidx[i] = -1;
    } else if (k == 1) {
      cidx[i] = 0;
    } else {
      cidx[i] = 1 + pos;
      T* row = tab + (long long)pos * pitch;
      for (int q = 0; q < 3 * s; ++q) row[q] = b[((long long)s + q) * n + i];
      row[ncoef - 1] = chiV[i];
      for (int q = ncoef; q < pitch; ++q) row[q] = (T)0;
      ++pos;
    }
  }
}
template <typename T>
cudaError_t launch_compact(const uint8_t* cls, const int* offsets, long long n, int* cidx, const T* b, int s,
                           const T* chiV, T* tab, long long n_irr, cudaStream_t st) {
  const long long nblk = (n + kScanBlock - 1) / kScanBlock;
  count_launch();
  k_compact<T><<<(unsigned)nblk, 256, 0, st>>>(cls, offsets, n, cidx, b, s, chiV, tab, n_irr);
  return cudaGetLastError();
}
template cudaError_t launch_compact<double>(const uint8_t*, const int*, long long, int*, const double*, int,
                                            const double*, double*, long long, cudaStream_t);
template cudaError_t launch_compact<float>(const uint8_t*, const int*, long long, int*, const float*, int,
                                           const float*, float*, long long, cudaStream_t);

__global__ void k_gather(double* out, const double* src, long long stride, long long idx, int count) {
  for (int j = threadIdx.x; j < count; j += blockDim.x) out[j] = src[(long long)j * stride + idx];
}
cudaError_t launch_gather(double* out, const double* src, long long stride, long long idx, int count, cudaStream_t s) {
  count_launch();
  k_gather<<<1, 64, 0, s>>>(out, src, stride, idx, count);
  return cudaGetLastError();
}

// up to 10 field pointers by value (kernel arguments)
// ------------------------------------- z axis: regular part + local corrections
template <typename T, int S, int R>
cudaError_t zcorr_sr(const ZCorrArgs<T>& a, cudaStream_t s) {
  constexpr int W = zcorr_warps<T, S>();  // records (warps) per block
  const long long nb = (a.nwin + W - 1) / W;
  const unsigned grid = (unsigned)(nb < 152 * 32 ? nb : 152 * 32);
  count_launch();
  k_zcorr<T, S, R, W><<<grid, 32 * W, 0, s>>>(a);
  return cudaGetLastError();
}
template <typename T, int S>
cudaError_t zcorr_s(const ZCorrArgs<T>& a, cudaStream_t s) {
  switch (a.r) {
    case 1: return zcorr_sr<T, S, 1>(a, s);
    case 2: return zcorr_sr<T, S, 2>(a, s);
    case 3: return zcorr_sr<T, S, 3>(a, s);
    case 4: return zcorr_sr<T, S, 4>(a, s);
    default: return cudaErrorInvalidValue;
  }
}
template <typename T>
cudaError_t launch_zcorr(const ZCorrArgs<T>& a, cudaStream_t s) {
  if (a.nwin <= 0) return cudaSuccess;
  return a.s == 4 ? zcorr_s<T, 4>(a, s) : zcorr_s<T, 10>(a, s);
}
template cudaError_t launch_zcorr<float>(const ZCorrArgs<float>&, cudaStream_t);
template cudaError_t launch_zcorr<double>(const ZCorrArgs<double>&, cudaStream_t);

// need[i] = 1 where delta may be nonzero: a node that is not regular (cidx != 0)
// within the support of some chi node (dil[i] = 1: box dilation of chi by r).
__global__ void k_zwin_need(uint8_t* need, const uint8_t* dil, const int* cidx, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    need[i] = (dil[i] && cidx[i] != 0) ? 1 : 0;
}

// out[i] = 1 - in[i]
__global__ void k_u8_not(uint8_t* out, const uint8_t* in, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = in[i] ? 0 : 1;
}

cudaError_t launch_zwin_need(uint8_t* need, const uint8_t* dil, const int* cidx, long long n, cudaStream_t s) {
  const long long nb = (n + 255) / 256;
  count_launch();
  k_zwin_need<<<(unsigned)(nb < 152 * 32 ? nb : 152 * 32), 256, 0, s>>>(need, dil, cidx, n);
  return cudaGetLastError();
}
cudaError_t launch_u8_not(uint8_t* out, const uint8_t* in, long long n, cudaStream_t s) {
  const long long nb = (n + 255) / 256;
  count_launch();
  k_u8_not<<<(unsigned)(nb < 152 * 32 ? nb : 152 * 32), 256, 0, s>>>(out, in, n);
  return cudaGetLastError();
}
// Per z-line: nk[8 * line ..] = its `need` nodes (bit z), mk[8 * line ..] = the
// positions within r (circularly) of one, flags[line] = 1 (has a chi node) | 2 (has
// a need node).
__global__ void k_zwin_mark(const uint8_t* need, const uint8_t* chi, int nx, int ny, int nz, int r, uint32_t* mk,
                            uint32_t* nk, uint8_t* flags) {
  const long long nlines = (long long)nx * ny;
  for (long long L = (long long)blockIdx.x * blockDim.x + threadIdx.x; L < nlines; L += (long long)gridDim.x * blockDim.x) {
    uint32_t nb[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // n_z <= 256
    bool any_need = false, any_chi = false;
    for (int z = 0; z < nz; ++z) {
      const long long i = L + (long long)z * nlines;
      if (need[i]) {
        nb[z >> 5] |= 1u << (z & 31);
        any_need = true;
      }
      any_chi |= chi[i] != 0;
    }
    uint32_t m[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (any_need)
      for (int z = 0; z < nz; ++z) {
        bool hit = false;
        for (int o = -r; o <= r && !hit; ++o) {
          int zz = z + o;
          zz = zz < 0 ? zz + nz : (zz >= nz ? zz - nz : zz);
          hit = (nb[zz >> 5] >> (zz & 31)) & 1u;
        }
        if (hit) m[z >> 5] |= 1u << (z & 31);
      }
    for (int k = 0; k < 8; ++k) {
      mk[8 * L + k] = m[k];
      nk[8 * L + k] = nb[k];
    }
    flags[L] = (any_chi ? 1 : 0) | (any_need ? 2 : 0);
  }
}

cudaError_t launch_zwin_mark(const uint8_t* need, const uint8_t* chi, const int n[3], int r, uint32_t* mk,
                             uint32_t* nk, uint8_t* flags, cudaStream_t s) {
  const long long nl = (long long)n[0] * n[1];
  count_launch();
  k_zwin_mark<<<(unsigned)((nl + 127) / 128), 128, 0, s>>>(need, chi, n[0], n[1], n[2], r, mk, nk, flags);
  return cudaGetLastError();
}
cudaError_t launch_zwin_groups(int fill, const uint32_t* mk, const uint8_t* flags, const int n[3], int chunk,
                               int* counts, ZWin* out, cudaStream_t s) {
  const long long ng = (long long)((n[0] + kZGW - 1) / kZGW) * n[1];
  const unsigned grid = (unsigned)((ng + 127) / 128);
  count_launch();
  if (fill)
    k_zwin_groups<true><<<grid, 128, 0, s>>>(mk, flags, n[0], n[1], n[2], chunk, counts, out);
  else
    k_zwin_groups<false><<<grid, 128, 0, s>>>(mk, flags, n[0], n[1], n[2], chunk, counts, out);
  return cudaGetLastError();
}

template <typename T>
struct DPtrs {
  T* p[10];
};

// --------------------------------------------- pointwise stage of Alg. 2
// Each thread owns VEC consecutive nodes (one 16-byte vector per field).
template <typename T, int S>
__global__ void __launch_bounds__(256) k_pointwise_stiff(const PointwiseArgs<T> a) {
  constexpr int VEC = 16 / sizeof(T);  // nodes per thread and values per 16-byte vector
  __shared__ __align__(16) T br[ctab_pitch<T>(S)];
  pointwise_stage_breg<T, S>(a, br, threadIdx.x, blockDim.x);
  __syncthreads();
  const long long nv = a.nbox / VEC;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (long long)gridDim.x * blockDim.x)
    pointwise_vec<T, S, false>(a, br, v * VEC);
}

// The listed 4-node groups (neither all regular nor all outside chi) of a z SPLIT
// that applied the regular / outside cases itself (a.diag: D_x, D_y, D_z scaled).
template <typename T, int S>
__global__ void __launch_bounds__(256) k_pointwise_groups(const PointwiseArgs<T> a, const int* list, long long count) {
  __shared__ __align__(16) T br[ctab_pitch<T>(S)];
  pointwise_stage_breg<T, S>(a, br, threadIdx.x, blockDim.x);
  __syncthreads();
  // one node per thread: 4 threads per listed group
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < 4 * count;
       j += (long long)gridDim.x * blockDim.x) {
    const long long i = 4LL * __ldg(list + (j >> 2)) + (j & 3);
    const int c = __ldg(a.cidx + i);
    T d[S], g[S];
#pragma unroll
    for (int q = 0; q < S; ++q) d[q] = a.D[q][i];
#pragma unroll
    for (int k = 0; k < 3; ++k) d[1 + k] *= a.inv_c[k];
    T co[ctab_pitch<T>(S)];
    pointwise_coefs<T, S>(a, br, c, co);
    pointwise_node<T, S>(co, c, d, g);
#pragma unroll
    for (int p = 0; p < S; ++p) a.D[p][i] = g[p];
  }
}

template <typename T>
cudaError_t launch_pointwise_groups(const PointwiseArgs<T>& a, const int* list, long long count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const long long nb = (4 * count + 255) / 256;
  const unsigned grid = (unsigned)(nb < 152 * 16 ? nb : 152 * 16);
  count_launch();
  if (a.s == 4)
    k_pointwise_groups<T, 4><<<grid, 256, 0, s>>>(a, list, count);
  else
    k_pointwise_groups<T, 10><<<grid, 256, 0, s>>>(a, list, count);
  return cudaGetLastError();
}
template cudaError_t launch_pointwise_groups<float>(const PointwiseArgs<float>&, const int*, long long, cudaStream_t);
template cudaError_t launch_pointwise_groups<double>(const PointwiseArgs<double>&, const int*, long long, cudaStream_t);

template <typename T>
cudaError_t launch_pointwise_stiff(const PointwiseArgs<T>& a, cudaStream_t s) {
  constexpr int VEC = 16 / sizeof(T);
  if (a.nbox % VEC) return cudaErrorInvalidValue;
  const long long nb = (a.nbox / VEC + 255) / 256;
  const unsigned grid = (unsigned)(nb < 152 * 16 ? (nb > 0 ? nb : 1) : 152 * 16);
  count_launch();
  switch (a.s) {  // 3D bases (4, 10 monomials), 2D bases (3, 6) and 1D bases (2, 3)
    case 2: k_pointwise_stiff<T, 2><<<grid, 256, 0, s>>>(a); break;
    case 4: k_pointwise_stiff<T, 4><<<grid, 256, 0, s>>>(a); break;
    case 10: k_pointwise_stiff<T, 10><<<grid, 256, 0, s>>>(a); break;
    case 3: k_pointwise_stiff<T, 3><<<grid, 256, 0, s>>>(a); break;
    case 6: k_pointwise_stiff<T, 6><<<grid, 256, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------- Alg. 3 / Alg. 4 without a z axis (2D)
template <typename T>
__global__ void k_eval_u_fields(T* u, DPtrs<T> D, const T* b0, int s, const uint8_t* mask, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    T acc = (T)0;
    for (int p = 0; p < s; ++p) acc += b0[(long long)p * n + i] * D.p[p][i];
    u[i] = (mask && !mask[i]) ? (T)0 : acc;
  }
}
template <typename T>
cudaError_t launch_eval_u_fields(T* u, T* const* D, const T* b0, int s, const uint8_t* mask, long long n,
                                 cudaStream_t st) {
  if (s < 1 || s > 10) return cudaErrorInvalidValue;
  DPtrs<T> d;
  for (int p = 0; p < s; ++p) d.p[p] = D[p];
  const long long nb = (n + 255) / 256;
  count_launch();
  k_eval_u_fields<T><<<(unsigned)(nb < 152 * 16 ? (nb > 0 ? nb : 1) : 152 * 16), 256, 0, st>>>(u, d, b0, s, mask, n);
  return cudaGetLastError();
}
template cudaError_t launch_eval_u_fields<float>(float*, float* const*, const float*, int, const uint8_t*, long long,
                                                 cudaStream_t);
template cudaError_t launch_eval_u_fields<double>(double*, double* const*, const double*, int, const uint8_t*,
                                                  long long, cudaStream_t);

template <typename T>
__global__ void k_transpose_u_fields(DPtrs<T> D, const T* y, const T* b0, int s, const T* wfield,
                                     const uint8_t* wmask, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    T w = y[i];
    if (wfield) w *= wfield[i];
    if (wmask && !wmask[i]) w = (T)0;
    for (int p = 0; p < s; ++p) D.p[p][i] = b0[(long long)p * n + i] * w;
  }
}
template <typename T>
cudaError_t launch_transpose_u_fields(T* const* D, const T* y, const T* b0, int s, const T* wfield,
                                      const uint8_t* wmask, long long n, cudaStream_t st) {
  if (s < 1 || s > 10) return cudaErrorInvalidValue;
  DPtrs<T> d;
  for (int p = 0; p < s; ++p) d.p[p] = D[p];
  const long long nb = (n + 255) / 256;
  count_launch();
  k_transpose_u_fields<T><<<(unsigned)(nb < 152 * 16 ? (nb > 0 ? nb : 1) : 152 * 16), 256, 0, st>>>(d, y, b0, s,
                                                                                                    wfield, wmask, n);
  return cudaGetLastError();
}
template cudaError_t launch_transpose_u_fields<float>(float* const*, const float*, const float*, int, const float*,
                                                      const uint8_t*, long long, cudaStream_t);
template cudaError_t launch_transpose_u_fields<double>(double* const*, const double*, const double*, int,
                                                       const double*, const uint8_t*, long long, cudaStream_t);
template cudaError_t launch_pointwise_stiff<float>(const PointwiseArgs<float>&, cudaStream_t);
template cudaError_t launch_pointwise_stiff<double>(const PointwiseArgs<double>&, cudaStream_t);

// ------------------------------------------------ preconditioner symbol
// tab[kz][ky][kx] = scale / lam~(kx, ky, kz) for kx < nxp (padding columns use kx = 0)
template <typename T>
__global__ void k_symbol_table(const SymbolArgs<double> y, T* tab, int nxp, int ny, int nz) {
  const long long n = (long long)nxp * ny * nz;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int kx = (int)(i % nxp), ky = (int)((i / nxp) % ny), kz = (int)(i / ((long long)nxp * ny));
    tab[i] = (T)(y.scale / symbol_value(y, kx < y.n[0] ? kx : 0, ky, kz));
  }
}
template <typename T>
cudaError_t launch_symbol_table(const SymbolArgs<double>& y, T* tab, int nxp, int ny, int nz, cudaStream_t s) {
  const long long n = (long long)nxp * ny * nz;
  const unsigned grid = (unsigned)std::min<long long>((n + 255) / 256, 152LL * 16);
  count_launch();
  k_symbol_table<T><<<grid, 256, 0, s>>>(y, tab, nxp, ny, nz);
  return cudaGetLastError();
}
template cudaError_t launch_symbol_table<float>(const SymbolArgs<double>&, float*, int, int, int, cudaStream_t);
template cudaError_t launch_symbol_table<double>(const SymbolArgs<double>&, double*, int, int, int, cudaStream_t);

// ----------------------------------------------------------- reductions
// Fixed grid and fixed combination order: results are bit-reproducible.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[kRedThreads / 32];
  v = warp_sum(v);
  const int w = threadIdx.x / 32, ln = threadIdx.x % 32;
  if (ln == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = (ln < kRedThreads / 32) ? sh[ln] : 0.0;
    r = warp_sum(r);
  }
  __syncthreads();
  return r;  // valid in thread 0
}

template <typename Ta, typename Tb>
__global__ void __launch_bounds__(kRedThreads) k_dot(const Ta* __restrict__ a, const Tb* __restrict__ b, long long n,
                                                    double* __restrict__ part) {
  static_assert(std::is_same<Ta, Tb>::value, "dot of equal types");
  DotAcc<Ta> acc;
  for (long long i = (long long)blockIdx.x * kRedThreads + threadIdx.x; i < n; i += (long long)kRedBlocks * kRedThreads)
    acc.add(a[i], b[i]);
  const double v = block_sum(acc.value());
  if (threadIdx.x == 0) part[blockIdx.x] = v;
}

__device__ __forceinline__ double reduce_partials(const double* part) {
  double v = 0.0;
  for (int i = threadIdx.x; i < kRedBlocks; i += kRedThreads) v += part[i];
  return block_sum(v);
}

__global__ void __launch_bounds__(kRedThreads) k_reduce_to(const double* part, double* out) {
  const double v = reduce_partials(part);
  if (threadIdx.x == 0) *out = v;
}

template <typename Ta, typename Tb>
cudaError_t launch_dot(const Ta* a, const Tb* b, long long n, double* partials, double* out, cudaStream_t s) {
  count_launch();
  k_dot<Ta, Tb><<<kRedBlocks, kRedThreads, 0, s>>>(a, b, n, partials);
  count_launch();
  k_reduce_to<<<1, kRedThreads, 0, s>>>(partials, out);
  return cudaGetLastError();
}
template cudaError_t launch_dot<double, double>(const double*, const double*, long long, double*, double*, cudaStream_t);
template cudaError_t launch_dot<float, float>(const float*, const float*, long long, double*, double*, cudaStream_t);

// rr = sum(partials); alpha = beta = 0; without preconditioner rz = rr
__global__ void k_cg_init(const double* part, CGState* st, int pcg) {
  const double v = reduce_partials(part);
  if (threadIdx.x == 0) {
    st->rr = v;
    st->alpha = 0.0;
    st->beta = 0.0;
    st->flag = 0;
    st->pcg = pcg;
    if (!pcg) st->rz = st->rz_prev = v;
  }
}
cudaError_t launch_cg_init(const double* partials, CGState* st, int pcg, cudaStream_t s) {
  count_launch();
  k_cg_init<<<1, kRedThreads, 0, s>>>(partials, st, pcg);
  return cudaGetLastError();
}

// rr = sum(partials) after a residual replacement (rz too without preconditioner)
__global__ void k_cg_set_rr(const double* part, CGState* st) {
  const double v = reduce_partials(part);
  if (threadIdx.x == 0) {
    st->rr = v;
    if (!st->pcg) st->rz = v;
  }
}
cudaError_t launch_cg_set_rr(const double* partials, CGState* st, cudaStream_t s) {
  count_launch();
  k_cg_set_rr<<<1, kRedThreads, 0, s>>>(partials, st);
  return cudaGetLastError();
}

// ------------------------------------------------- nonlinear reaction terms
// N(u) and N'(u) of the built-in reaction nonlinearities (Appendix B, Eq. B.1)
__device__ __forceinline__ double nl_value(int kind, double c, double u) {
  switch (kind) {
    case 0: return c * u * u * u;  // cubic
    case 1: return c * sinh(u);
    case 2: return c * exp(u);
    default: return 0.0;
  }
}
__device__ __forceinline__ double nl_slope(int kind, double c, double u) {
  switch (kind) {
    case 0: return 3.0 * c * u * u;
    case 1: return c * cosh(u);
    case 2: return c * exp(u);
    default: return 0.0;
  }
}

// Nu = chi ? N(u) : 0
__global__ void k_nl_apply(double* Nu, const double* u, const uint8_t* chi, int kind, double c, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    Nu[i] = chi[i] ? nl_value(kind, c, u[i]) : 0.0;
}
cudaError_t launch_nl_apply(double* Nu, const double* u, const uint8_t* chi, int kind, double c, long long n,
                            cudaStream_t s) {
  count_launch();
  k_nl_apply<<<kRedBlocks, kRedThreads, 0, s>>>(Nu, u, chi, kind, c, n);
  return cudaGetLastError();
}

// Fields of the gradient-type force (Eq. B.10): g_p = chi V (sum_k a_k b^k_p) N_u,
// b = [4][s][n] (b^0, b^x, b^y, b^z), chiV = chi o V, Nu = N(u^h) (zero outside chi)
__global__ void k_grad_g(DPtrs<double> g, const double* b, const double* chiV, const double* Nu, double a0, double a1,
                         double a2, int s, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double w = chiV[i] * Nu[i];
    for (int p = 0; p < s; ++p) {
      const double bk = a0 * b[(size_t)(s + p) * n + i] + a1 * b[(size_t)(2 * s + p) * n + i] +
                        a2 * b[(size_t)(3 * s + p) * n + i];
      g.p[p][i] = w * bk;
    }
  }
}
cudaError_t launch_grad_g(double* const* g, const double* b, const double* chiV, const double* Nu, const double a[3],
                          int s, long long n, cudaStream_t st) {
  DPtrs<double> gp;
  for (int p = 0; p < 10; ++p) gp.p[p] = p < s ? g[p] : nullptr;
  count_launch();
  k_grad_g<<<kRedBlocks, kRedThreads, 0, st>>>(gp, b, chiV, Nu, a[0], a[1], a[2], s, n);
  return cudaGetLastError();
}

// Line search sums over chi: out[0] = sum V w N(u + alpha w), out[1] = sum V w^2 N'(u + alpha w)
// (fixed grid and order: reproducible)
__global__ void __launch_bounds__(kRedThreads) k_nl_line(const double* u, const double* w, const double* V,
                                                        const uint8_t* chi, int kind, double c, double alpha,
                                                        long long n, double* part) {
  double s0 = 0.0, s1 = 0.0;
  for (long long i = (long long)blockIdx.x * kRedThreads + threadIdx.x; i < n; i += (long long)kRedBlocks * kRedThreads)
    if (chi[i]) {
      const double wi = w[i], ui = u[i] + alpha * wi, vw = V[i] * wi;
      s0 += vw * nl_value(kind, c, ui);
      s1 += vw * wi * nl_slope(kind, c, ui);
    }
  s0 = block_sum(s0);
  s1 = block_sum(s1);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s0;
    part[kRedBlocks + blockIdx.x] = s1;
  }
}
__global__ void __launch_bounds__(kRedThreads) k_reduce2_to(const double* part, double* out) {
  const double a = reduce_partials(part);
  const double b = reduce_partials(part + kRedBlocks);
  if (threadIdx.x == 0) {
    out[0] = a;
    out[1] = b;
  }
}
cudaError_t launch_nl_line(const double* u, const double* w, const double* V, const uint8_t* chi, int kind, double c,
                           double alpha, long long n, double* partials2, double* out2, cudaStream_t s) {
  count_launch();
  k_nl_line<<<kRedBlocks, kRedThreads, 0, s>>>(u, w, V, chi, kind, c, alpha, n, partials2);
  count_launch();
  k_reduce2_to<<<1, kRedThreads, 0, s>>>(partials2, out2);
  return cudaGetLastError();
}

// 16-byte vectors of T (4 floats / 2 doubles)
template <typename T>
struct VecN {
  static constexpr int N = 16 / sizeof(T);
  T v[N];
};

template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_cg_xr_fused(T* __restrict__ x, T* __restrict__ r,
                                                            const T* __restrict__ p, const T* __restrict__ Ap,
                                                            CGState* st, long long n, double* __restrict__ part,
                                                            unsigned* counter) {
  using V = VecN<T>;
  const T al = (T)st->alpha;
  DotAccPair<T> acc;
  const long long nv = n / V::N;
  for (long long i = (long long)blockIdx.x * kRedThreads + threadIdx.x; i < nv; i += (long long)kRedBlocks * kRedThreads) {
    V xv = reinterpret_cast<V*>(x)[i];
    V rv = reinterpret_cast<V*>(r)[i];
    const V pv = reinterpret_cast<const V*>(p)[i];
    const V av = reinterpret_cast<const V*>(Ap)[i];
#pragma unroll
    for (int e = 0; e < V::N; ++e) {
      xv.v[e] += al * pv.v[e];
      rv.v[e] -= al * av.v[e];
    }
#pragma unroll
    for (int e = 0; e < V::N; e += 2) {
      const cpx<T> rr = cmk(rv.v[e], rv.v[e + 1]);
      acc.add(rr, rr);
    }
    reinterpret_cast<V*>(x)[i] = xv;
    reinterpret_cast<V*>(r)[i] = rv;
  }
  // scalar tail (n not a multiple of the vector width)
  for (long long i = nv * V::N + (long long)blockIdx.x * kRedThreads + threadIdx.x; i < n;
       i += (long long)kRedBlocks * kRedThreads) {
    x[i] += al * p[i];
    const T ri = r[i] - al * Ap[i];
    r[i] = ri;
    acc.add(cmk(ri, (T)0), cmk(ri, (T)0));
  }
  const double bs = block_sum(acc.value());
  __shared__ bool last;
  if (threadIdx.x == 0) {
    part[blockIdx.x] = bs;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double v = 0.0;
  for (int i = threadIdx.x; i < kRedBlocks; i += kRedThreads) v += ((volatile double*)part)[i];
  v = block_sum(v);
  if (threadIdx.x == 0) {
    st->rr_new = v;
    if (!st->pcg) {
      st->beta = (st->rr > 0.0) ? v / st->rr : 0.0;
      st->rz_prev = st->rz;
      st->rz = v;
    }
    st->rr = v;
    *counter = 0u;
  }
}
template <typename T>
cudaError_t launch_cg_xr_fused(T* x, T* r, const T* p, const T* Ap, CGState* st, long long n, double* partials,
                               unsigned* counter, cudaStream_t s) {
  count_launch();
  k_cg_xr_fused<T><<<kRedBlocks, kRedThreads, 0, s>>>(x, r, p, Ap, st, n, partials, counter);
  return cudaGetLastError();
}
template cudaError_t launch_cg_xr_fused<double>(double*, double*, const double*, const double*, CGState*, long long,
                                                double*, unsigned*, cudaStream_t);
template cudaError_t launch_cg_xr_fused<float>(float*, float*, const float*, const float*, CGState*, long long,
                                               double*, unsigned*, cudaStream_t);

// ------------------------------------------------------------ elementwise
#define RK_GRID_LOOP(i, n)                                                             \
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (n); \
       i += (long long)gridDim.x * blockDim.x)

static inline unsigned ew_grid(long long n) {
  const long long b = (n + 255) / 256;
  return (unsigned)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

__global__ void k_dirichlet_d0(double* d0, const double* g, const uint8_t* cg, long long n) {
  RK_GRID_LOOP(i, n) d0[i] = cg[i] ? g[i] : 0.0;
}
cudaError_t launch_dirichlet_d0(double* d0, const double* g, const uint8_t* chi_gamma, long long n, cudaStream_t s) {
  count_launch();
  k_dirichlet_d0<<<ew_grid(n), 256, 0, s>>>(d0, g, chi_gamma, n);
  return cudaGetLastError();
}

__global__ void k_masked_diff(double* F, const double* a, const double* b, const uint8_t* m, long long n) {
  RK_GRID_LOOP(i, n) F[i] = m[i] ? a[i] - b[i] : 0.0;
}
cudaError_t launch_masked_diff(double* F, const double* a, const double* b, const uint8_t* mask, long long n,
                               cudaStream_t s) {
  count_launch();
  k_masked_diff<<<ew_grid(n), 256, 0, s>>>(F, a, b, mask, n);
  return cudaGetLastError();
}

__global__ void k_to_f32(float* y, const double* x, double sc, long long n) {
  RK_GRID_LOOP(i, n) y[i] = (float)(x[i] * sc);
}
cudaError_t launch_to_f32(float* y, const double* x, double scale, long long n, cudaStream_t s) {
  count_launch();
  k_to_f32<<<ew_grid(n), 256, 0, s>>>(y, x, scale, n);
  return cudaGetLastError();
}

__global__ void k_acc_f32(double* x, const float* c, double sc, long long n) {
  RK_GRID_LOOP(i, n) x[i] += sc * (double)c[i];
}
cudaError_t launch_acc_f32(double* x, const float* c, double scale, long long n, cudaStream_t s) {
  count_launch();
  k_acc_f32<<<ew_grid(n), 256, 0, s>>>(x, c, scale, n);
  return cudaGetLastError();
}

__global__ void k_add(double* d, const double* a, const double* b, long long n) {
  RK_GRID_LOOP(i, n) d[i] = a[i] + b[i];
}
cudaError_t launch_add(double* d, const double* a, const double* b, long long n, cudaStream_t s) {
  count_launch();
  k_add<<<ew_grid(n), 256, 0, s>>>(d, a, b, n);
  return cudaGetLastError();
}

// y = a x + b y
__global__ void k_axpby(double* y, double a, const double* x, double b, long long n) {
  RK_GRID_LOOP(i, n) y[i] = a * x[i] + b * y[i];
}
cudaError_t launch_axpby(double* y, double a, const double* x, double b, long long n, cudaStream_t s) {
  count_launch();
  k_axpby<<<ew_grid(n), 256, 0, s>>>(y, a, x, b, n);
  return cudaGetLastError();
}

// forward Euler with lumped mass on the free nodes (Alg. C.3):
// d += dt (f - K d) / M^l where mask, d untouched elsewhere
__global__ void k_explicit_step(double* d, const double* f, const double* Kd, const double* ml, const uint8_t* mask,
                                double dt, long long n) {
  RK_GRID_LOOP(i, n) if (mask[i]) d[i] += dt * (f[i] - Kd[i]) / ml[i];
}
cudaError_t launch_explicit_step(double* d, const double* f, const double* Kd, const double* ml, const uint8_t* mask,
                                 double dt, long long n, cudaStream_t s) {
  count_launch();
  k_explicit_step<<<ew_grid(n), 256, 0, s>>>(d, f, Kd, ml, mask, dt, n);
  return cudaGetLastError();
}

__global__ void k_sub(double* d, const double* a, const double* b, long long n) {
  RK_GRID_LOOP(i, n) d[i] = a[i] - b[i];
}
cudaError_t launch_sub(double* out, const double* a, const double* b, long long n, cudaStream_t s) {
  count_launch();
  k_sub<<<ew_grid(n), 256, 0, s>>>(out, a, b, n);
  return cudaGetLastError();
}

__global__ void k_mask(double* o, const double* a, const uint8_t* m, long long n) {
  RK_GRID_LOOP(i, n) o[i] = m[i] ? a[i] : 0.0;
}
cudaError_t launch_mask(double* out, const double* a, const uint8_t* mask, long long n, cudaStream_t s) {
  count_launch();
  k_mask<<<ew_grid(n), 256, 0, s>>>(out, a, mask, n);
  return cudaGetLastError();
}

__global__ void k_mul(double* a, const double* b, long long n) {
  RK_GRID_LOOP(i, n) a[i] *= b[i];
}
cudaError_t launch_mul(double* a, const double* b, long long n, cudaStream_t s) {
  count_launch();
  k_mul<<<ew_grid(n), 256, 0, s>>>(a, b, n);
  return cudaGetLastError();
}

__global__ void k_u8_to_f64(double* o, const uint8_t* m, long long n) {
  RK_GRID_LOOP(i, n) o[i] = m[i] ? 1.0 : 0.0;
}
cudaError_t launch_u8_to_f64(double* out, const uint8_t* m, long long n, cudaStream_t s) {
  count_launch();
  k_u8_to_f64<<<ew_grid(n), 256, 0, s>>>(out, m, n);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_fill(T* p, T v, long long n) {
  RK_GRID_LOOP(i, n) p[i] = v;
}
template <typename T>
cudaError_t launch_fill(T* p, T v, long long n, cudaStream_t s) {
  count_launch();
  k_fill<T><<<ew_grid(n), 256, 0, s>>>(p, v, n);
  return cudaGetLastError();
}
template cudaError_t launch_fill<double>(double*, double, long long, cudaStream_t);
template cudaError_t launch_fill<float>(float*, float, long long, cudaStream_t);

template <typename T>
__global__ void k_copy(T* d, const T* s, long long n) {
  RK_GRID_LOOP(i, n) d[i] = s[i];
}
template <typename T>
cudaError_t launch_copy(T* dst, const T* src, long long n, cudaStream_t s) {
  count_launch();
  k_copy<T><<<ew_grid(n), 256, 0, s>>>(dst, src, n);
  return cudaGetLastError();
}
template cudaError_t launch_copy<double>(double*, const double*, long long, cudaStream_t);
template cudaError_t launch_copy<float>(float*, const float*, long long, cudaStream_t);

}  // namespace rk
