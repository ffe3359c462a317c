// rk_linefft.cuh -- length-N complex FFT of one line held by P cooperating
// threads, N = N1 * N2 (four-step: DFT over N2, twiddle, transpose through
// shared memory, DFT over N1).
//
// Layouts (thread t in [0, P)):
//   natural   v[a*N2 + j2] = x[(t + P a) + N1 j2],  a in [0, N1/P), j2 in [0, N2)
//   spectral  v[b*N1 + k1] = X[(t + P b) + N2 k1],  b in [0, N2/P), k1 in [0, N1)
// forward() maps natural -> spectral with X_k = sum_j x_j exp(-2 pi i jk/N)
// (Eq. 30), inverse() maps spectral -> natural with the conjugate kernel and no
// 1/N (Eq. 31 without its normalisation).  A pointwise product in between is a
// circular convolution (Eq. 33-34) without any reordering of the spectrum.
//
// The shared-memory transpose buffer is supplied by the caller through an
// addressing object:  fw(j1, k2) and iv(j1, k2) return the element used by the
// forward and the inverse transpose for the pair (j1, k2).
#pragma once

#include "rk_common.cuh"

namespace rk {

template <int N>
struct LineShape;
// (N1, N2, P): P divides N1 and N2; registers per thread R = N / P.
template <> struct LineShape<8> { static constexpr int N1 = 4, N2 = 2, P = 2; };
template <> struct LineShape<16> { static constexpr int N1 = 4, N2 = 4, P = 4; };
template <> struct LineShape<32> { static constexpr int N1 = 4, N2 = 8, P = 4; };
template <> struct LineShape<64> { static constexpr int N1 = 8, N2 = 8, P = 8; };
template <> struct LineShape<96> { static constexpr int N1 = 8, N2 = 12, P = 4; };
template <> struct LineShape<128> { static constexpr int N1 = 8, N2 = 16, P = 8; };
template <> struct LineShape<256> { static constexpr int N1 = 16, N2 = 16, P = 16; };
template <> struct LineShape<512> { static constexpr int N1 = 16, N2 = 32, P = 16; };
// 7-smooth sides used to pad uneven boxes
template <> struct LineShape<36> { static constexpr int N1 = 6, N2 = 6, P = 6; };
template <> struct LineShape<48> { static constexpr int N1 = 4, N2 = 12, P = 4; };
template <> struct LineShape<72> { static constexpr int N1 = 6, N2 = 12, P = 6; };
template <> struct LineShape<100> { static constexpr int N1 = 10, N2 = 10, P = 10; };
template <> struct LineShape<144> { static constexpr int N1 = 12, N2 = 12, P = 12; };
template <> struct LineShape<162> { static constexpr int N1 = 9, N2 = 18, P = 9; };

template <typename T, int N>
struct LineFFT {
  static constexpr int N1 = LineShape<N>::N1;
  static constexpr int N2 = LineShape<N>::N2;
  static constexpr int P = LineShape<N>::P;
  static_assert(N1 * N2 == N, "bad line shape");
  static_assert(N1 % P == 0 && N2 % P == 0, "P must divide N1 and N2");
  static constexpr int A = N1 / P;  // j1 values per thread
  static constexpr int B = N2 / P;  // k2 values per thread
  static constexpr int R = N / P;   // complex registers per thread

  // position of natural register r of thread t within the line
  RK_HD static int nat_pos(int t, int r) { return (t + P * (r / N2)) + N1 * (r % N2); }
  // spectral index of spectral register r of thread t
  RK_HD static int spec_idx(int t, int r) { return (t + P * (r / N1)) + N2 * (r % N1); }

  // tw[m] = exp(-2 pi i m / N), m in [0, N)
  template <class Buf>
  RK_DEV static void forward(cpx<T>* v, int t, const Buf& buf, const cpx<T>* tw) {
#pragma unroll
    for (int a = 0; a < A; ++a) {
      DFT<N2, -1, T>::run(v + a * N2);
      const int j1 = t + P * a;
#pragma unroll
      for (int k2 = 1; k2 < N2; ++k2) {
        cpx<T> w = tw[(j1 * k2) % N];
        v[a * N2 + k2] = cmul(v[a * N2 + k2], w);
      }
    }
    RK_SYNC();  // previous readers of the buffer are done
#pragma unroll
    for (int a = 0; a < A; ++a)
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) buf.fw(t + P * a, k2) = v[a * N2 + k2];
    RK_SYNC();
#pragma unroll
    for (int b = 0; b < B; ++b)
#pragma unroll
      for (int j1 = 0; j1 < N1; ++j1) v[b * N1 + j1] = buf.fw(j1, t + P * b);
#pragma unroll
    for (int b = 0; b < B; ++b) DFT<N1, -1, T>::run(v + b * N1);
  }

  template <class Buf>
  RK_DEV static void inverse(cpx<T>* v, int t, const Buf& buf, const cpx<T>* tw) {
#pragma unroll
    for (int b = 0; b < B; ++b) {
      DFT<N1, +1, T>::run(v + b * N1);
      const int k2 = t + P * b;
#pragma unroll
      for (int j1 = 1; j1 < N1; ++j1) {
        cpx<T> w = tw[(j1 * k2) % N];
        v[b * N1 + j1] = cmulc(v[b * N1 + j1], w);
      }
    }
    RK_SYNC();
#pragma unroll
    for (int b = 0; b < B; ++b)
#pragma unroll
      for (int j1 = 0; j1 < N1; ++j1) buf.iv(j1, t + P * b) = v[b * N1 + j1];
    RK_SYNC();
#pragma unroll
    for (int a = 0; a < A; ++a)
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) v[a * N2 + k2] = buf.iv(t + P * a, k2);
#pragma unroll
    for (int a = 0; a < A; ++a) DFT<N2, +1, T>::run(v + a * N2);
  }
};

// Transpose buffer for lines interleaved in shared memory (line l fastest):
// element (row, col) of line l at ((row * pitch + col) * L + l).  Used when the
// L lines of a block are adjacent in memory (x-pairs of y- or z-lines).
template <typename T, int N1, int N2>
struct InterleavedBuf {
  cpx<T>* base;  // points at slot l
  int L;
  RK_HD cpx<T>& fw(int j1, int k2) const { return base[(k2 * N1 + j1) * L]; }
  RK_HD cpx<T>& iv(int j1, int k2) const { return base[(j1 * N2 + k2) * L]; }
};

// Transpose buffer with one padded block per line (row pitch + 1 against bank
// conflicts).  Used when the P threads of a line are adjacent lanes (x-lines).
template <typename T, int N1, int N2>
struct PaddedBuf {
  static constexpr int SIZE = (N2 * (N1 + 1) > N1 * (N2 + 1)) ? N2 * (N1 + 1) : N1 * (N2 + 1);
  cpx<T>* base;  // points at the block of line l
  RK_HD cpx<T>& fw(int j1, int k2) const { return base[k2 * (N1 + 1) + j1]; }
  RK_HD cpx<T>& iv(int j1, int k2) const { return base[j1 * (N2 + 1) + k2]; }
};

}  // namespace rk
