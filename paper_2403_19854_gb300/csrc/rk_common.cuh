// rk_common.cuh -- shared device helpers for the FC-RKPM kernels: complex
// arithmetic, compile-time twiddle factors and small DFT codelets.
//
// The discrete Fourier transform convention is the one of Eq. 30-31: forward
// transform unnormalised with kernel exp(-2 pi i jk/n); inverse with
// exp(+2 pi i jk/n) and a factor 1/n.  The 1/n of the inverse is never applied
// here: callers fold it into the spectral multipliers.
#pragma once

#include <stdint.h>

#include <type_traits>
#include <utility>

#ifndef RK_HD
#define RK_HD __host__ __device__ __forceinline__
#endif
#ifndef RK_DEV
#define RK_DEV __device__ __forceinline__
#endif
#ifndef RK_SYNC
#define RK_SYNC() __syncthreads()
#endif
#ifndef RK_LDG
#define RK_LDG(p) __ldg(p)
#endif
// dynamic shared memory of a kernel, viewed as an array of T
#ifndef RK_DYN_SMEM
#define RK_DYN_SMEM(T, name)                                   \
  extern __shared__ __align__(128) unsigned char rk_smem_raw[]; \
  T* name = reinterpret_cast<T*>(rk_smem_raw)
#endif

namespace rk {

// ---------------------------------------------------------------- complex
template <typename T>
struct cpx {
  T x, y;
};

template <typename T>
struct vec2;
template <>
struct vec2<float> {
  using type = float2;
};
template <>
struct vec2<double> {
  using type = double2;
};

template <typename T>
RK_HD cpx<T> cmk(T x, T y) {
  cpx<T> r;
  r.x = x;
  r.y = y;
  return r;
}
template <typename T>
RK_HD cpx<T> operator+(cpx<T> a, cpx<T> b) { return cmk(a.x + b.x, a.y + b.y); }
template <typename T>
RK_HD cpx<T> operator-(cpx<T> a, cpx<T> b) { return cmk(a.x - b.x, a.y - b.y); }
template <typename T>
RK_HD cpx<T> cmul(cpx<T> a, cpx<T> b) { return cmk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
// a * conj(b)
template <typename T>
RK_HD cpx<T> cmulc(cpx<T> a, cpx<T> b) { return cmk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); }
template <typename T>
RK_HD cpx<T> cscale(cpx<T> a, T s) { return cmk(a.x * s, a.y * s); }
// element-wise products of the two components (two real lines / node pairs)
template <typename T>
RK_HD cpx<T> pmul(cpx<T> a, cpx<T> b) { return cmk(a.x * b.x, a.y * b.y); }
template <typename T>
RK_HD cpx<T> pfma(cpx<T> a, cpx<T> b, cpx<T> c) { return cmk(a.x * b.x + c.x, a.y * b.y + c.y); }

// FP32 pairs use the packed two-lane FP32 instructions of sm_100+ (one
// instruction per component pair) where both lanes take the same operation:
// sums, differences and lane-wise products.  Complex products stay scalar (four
// FP32 instructions): their packed form needs lane shuffles and measured 4 %
// slower over a K.u.  Other targets keep the scalar forms above.
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000)
#define RK_PACKED_F32 1
__device__ __forceinline__ float2 rk_f2(cpx<float> a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ cpx<float> rk_c2(float2 a) { return cmk(a.x, a.y); }
__device__ __forceinline__ cpx<float> operator+(cpx<float> a, cpx<float> b) {
  return rk_c2(__fadd2_rn(rk_f2(a), rk_f2(b)));
}
__device__ __forceinline__ cpx<float> operator-(cpx<float> a, cpx<float> b) {
  return rk_c2(__fadd2_rn(rk_f2(a), make_float2(-b.x, -b.y)));
}
__device__ __forceinline__ cpx<float> cscale(cpx<float> a, float s) {
  return rk_c2(__fmul2_rn(rk_f2(a), make_float2(s, s)));
}
__device__ __forceinline__ cpx<float> pmul(cpx<float> a, cpx<float> b) { return rk_c2(__fmul2_rn(rk_f2(a), rk_f2(b))); }
__device__ __forceinline__ cpx<float> pfma(cpx<float> a, cpx<float> b, cpx<float> c) {
  return rk_c2(__ffma2_rn(rk_f2(a), rk_f2(b), rk_f2(c)));
}
#endif
// multiply by i*s (s real)
template <typename T>
RK_HD cpx<T> ciscale(cpx<T> a, T s) { return cmk(-a.y * s, a.x * s); }

// ------------------------------------------------------ dot-product partials
// Per-thread partial sums of a dot product.  For double data: plain FP64 FMAs.
// For float data the products and the running sum are kept as an unevaluated
// pair (s + c) by the error-free transformations of Ogita, Rump and Oishi
// ("Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005, Dot2): the
// product error from one FMA, the addition error from Knuth's TwoSum.  The
// partial is then as accurate as an FP64 accumulation of the same terms while
// using FP32 instructions only (FP64 issues at a small fraction of the FP32
// rate on this GPU).  Explicit _rn intrinsics keep the compiler from fusing
// the product into the sum, which would break the error terms.
template <typename T>
struct DotAcc {
  double s = 0.0;
  RK_DEV void add(double a, double b) { s = fma(a, b, s); }
  RK_DEV double value() const { return s; }
};
template <>
struct DotAcc<float> {
  float s = 0.0f, c = 0.0f;
  RK_DEV void add(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);   // a*b = p + e exactly
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);       // TwoSum: s + p = t + err exactly
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
    s = t;
    c = __fadd_rn(c, __fadd_rn(err, e));
  }
  RK_DEV double value() const { return (double)s + (double)c; }
};

// Two partials in one: the component pairs a thread holds (two lines, two
// nodes) accumulate lane by lane, which for FP32 on sm_100+ runs the same
// compensated steps as DotAcc<float> in packed two-lane instructions.
template <typename T>
struct DotAccPair {
  DotAcc<T> d;
  RK_DEV void add(cpx<T> a, cpx<T> b) {
    d.add(a.x, b.x);
    d.add(a.y, b.y);
  }
  RK_DEV double value() const { return d.value(); }
};
#if defined(RK_PACKED_F32)
template <>
struct DotAccPair<float> {
  float2 s = make_float2(0.0f, 0.0f), c = make_float2(0.0f, 0.0f);
  static RK_DEV float2 neg(float2 v) { return make_float2(-v.x, -v.y); }
  RK_DEV void add(cpx<float> a, cpx<float> b) {
    const float2 fa = rk_f2(a), fb = rk_f2(b);
    const float2 p = __fmul2_rn(fa, fb);
    const float2 e = __ffma2_rn(fa, fb, neg(p));
    const float2 t = __fadd2_rn(s, p);
    const float2 z = __fadd2_rn(t, neg(s));
    const float2 err = __fadd2_rn(__fadd2_rn(s, neg(__fadd2_rn(t, neg(z)))), __fadd2_rn(p, neg(z)));
    s = t;
    c = __fadd2_rn(c, __fadd2_rn(err, e));
  }
  RK_DEV double value() const { return ((double)s.x + (double)c.x) + ((double)s.y + (double)c.y); }
};
#endif

// ------------------------------------------------- compile-time trigonometry
// cos and sin of 2*pi*m/R.  The angle is reduced exactly in integer arithmetic
// to [0, pi/4] (octant symmetries), then evaluated with the Maclaurin series of
// sin and cos (18 terms, far below double rounding for |x| <= pi/4).
namespace trig {
constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double maclaurin_sin(double x) {
  double term = x, sum = x;
  for (int k = 1; k < 18; ++k) {
    term *= -x * x / (double)((2 * k) * (2 * k + 1));
    sum += term;
  }
  return sum;
}
constexpr double maclaurin_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 18; ++k) {
    term *= -x * x / (double)((2 * k - 1) * (2 * k));
    sum += term;
  }
  return sum;
}
// angle = pi * w / (4R) with 0 <= w <= R  (i.e. in [0, pi/4])
constexpr double small_cos(long long w, long long R) { return maclaurin_cos(kPi * (double)w / (double)(4 * R)); }
constexpr double small_sin(long long w, long long R) { return maclaurin_sin(kPi * (double)w / (double)(4 * R)); }
// returns cos (which = 0) or sin (which = 1) of 2 pi m / R
constexpr double cs2pi(long long m, long long R, int which) {
  m %= R;
  if (m < 0) m += R;
  double ssign = 1.0, csign = 1.0;
  if (2 * m > R) {  // angle in (pi, 2pi): reflect, sin changes sign
    m = R - m;
    ssign = -1.0;
  }
  // angle = 2 pi m / R = pi * u / R with u = 2m in [0, R]
  long long u = 2 * m;
  if (2 * u > R) {  // angle > pi/2: cos(pi - x) = -cos x, sin(pi - x) = sin x
    u = R - u;
    csign = -1.0;
  }
  // angle = pi * u / R in [0, pi/2]; as pi * w / (4R) with w = 4u in [0, 2R]
  long long w = 4 * u;
  double c = 0.0, s = 0.0;
  if (w > R) {  // angle > pi/4: swap with the complement pi/2 - x = pi (2R - w)/(4R)
    c = small_sin(2 * R - w, R);
    s = small_cos(2 * R - w, R);
  } else {
    c = small_cos(w, R);
    s = small_sin(w, R);
  }
  return which == 0 ? csign * c : ssign * s;
}
constexpr double cos2pi(long long m, long long R) { return cs2pi(m, R, 0); }
constexpr double sin2pi(long long m, long long R) { return cs2pi(m, R, 1); }
}  // namespace trig

// Compile-time twiddle w_R^M = exp(DIR * 2 pi i M / R), DIR = -1 forward, +1 inverse.
template <int M, int R, int DIR>
struct Tw {
  static constexpr double c = trig::cos2pi(M, R);
  static constexpr double s = DIR * trig::sin2pi(M, R);
  static constexpr int mr = ((M % R) + R) % R;
  static constexpr bool one = (mr == 0);
  static constexpr bool minus_one = (2 * mr == R);
  static constexpr bool plus_i = (DIR > 0) ? (4 * mr == R) : (4 * mr == 3 * R);   // w = +i
  static constexpr bool minus_i = (DIR > 0) ? (4 * mr == 3 * R) : (4 * mr == R);  // w = -i
};

template <int M, int R, int DIR, typename T>
RK_HD cpx<T> twmul(cpx<T> v) {
  using W = Tw<M, R, DIR>;
  if constexpr (W::one) {
    return v;
  } else if constexpr (W::minus_one) {
    return cmk(-v.x, -v.y);
  } else if constexpr (W::plus_i) {
    return cmk(-v.y, v.x);
  } else if constexpr (W::minus_i) {
    return cmk(v.y, -v.x);
  } else {
    return cmul(v, cmk((T)W::c, (T)W::s));
  }
}

// --------------------------------------------------------- compile-time for
template <typename F, int... Is>
RK_HD void sfor_impl(F&& f, std::integer_sequence<int, Is...>) {
  (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, typename F>
RK_HD void sfor(F&& f) {
  sfor_impl(f, std::make_integer_sequence<int, N>{});
}

// ------------------------------------------------------------ DFT codelets
// In-place DFT of length R on v[0..R-1] (natural order in and out):
//   X_k = sum_j x_j exp(DIR 2 pi i jk / R).
constexpr int first_factor(int R) {
  return (R % 4 == 0 && R != 4) ? 4 : (R % 2 == 0 ? 2 : (R % 3 == 0 ? 3 : (R % 5 == 0 ? 5 : (R % 7 == 0 ? 7 : R))));
}
constexpr bool is_base(int R) { return R == 1 || R == 2 || R == 3 || R == 4 || R == 5 || R == 7; }

template <int R, int DIR, typename T, bool BASE = is_base(R)>
struct DFT;

template <int DIR, typename T>
struct DFT<1, DIR, T, true> {
  RK_HD static void run(cpx<T>*) {}
};
template <int DIR, typename T>
struct DFT<2, DIR, T, true> {
  RK_HD static void run(cpx<T>* v) {
    cpx<T> a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
  }
};
template <int DIR, typename T>
struct DFT<4, DIR, T, true> {
  RK_HD static void run(cpx<T>* v) {
    cpx<T> s02 = v[0] + v[2], d02 = v[0] - v[2];
    cpx<T> s13 = v[1] + v[3], d13 = v[1] - v[3];
    // w_4 = DIR * i
    cpx<T> wd = (DIR > 0) ? cmk(-d13.y, d13.x) : cmk(d13.y, -d13.x);
    v[0] = s02 + s13;
    v[2] = s02 - s13;
    v[1] = d02 + wd;
    v[3] = d02 - wd;
  }
};
// odd prime lengths (3, 5, 7): pairwise symmetric form
//   X_k = x_0 + sum_{j=1}^{(R-1)/2} [cos(2 pi jk/R) (x_j + x_{R-j}) + i DIR sin(2 pi jk/R) (x_j - x_{R-j})]
template <int R, int DIR, typename T>
struct DFTOddPrime {
  RK_HD static void run(cpx<T>* v) {
    constexpr int H = (R - 1) / 2;
    cpx<T> t[H], u[H];
    cpx<T> x0 = v[0];
    cpx<T> sum = x0;
    sfor<H>([&](auto J) {
      constexpr int j = decltype(J)::value + 1;
      t[j - 1] = v[j] + v[R - j];
      u[j - 1] = v[j] - v[R - j];
      sum = sum + t[j - 1];
    });
    cpx<T> out[R];
    out[0] = sum;
    sfor<H>([&](auto K) {
      constexpr int k = decltype(K)::value + 1;
      cpx<T> re = x0, im = cmk((T)0, (T)0);
      sfor<H>([&](auto J) {
        constexpr int j = decltype(J)::value + 1;
        constexpr double c = trig::cos2pi(j * k, R);
        constexpr double s = DIR * trig::sin2pi(j * k, R);
        re = pfma(t[j - 1], cmk((T)c, (T)c), re);
        im = pfma(u[j - 1], cmk((T)s, (T)s), im);
      });
      // + i*im and - i*im
      out[k] = cmk(re.x - im.y, re.y + im.x);
      out[R - k] = cmk(re.x + im.y, re.y - im.x);
    });
    sfor<R>([&](auto K) { v[decltype(K)::value] = out[decltype(K)::value]; });
  }
};
template <int DIR, typename T>
struct DFT<3, DIR, T, true> : DFTOddPrime<3, DIR, T> {};
template <int DIR, typename T>
struct DFT<5, DIR, T, true> : DFTOddPrime<5, DIR, T> {};
template <int DIR, typename T>
struct DFT<7, DIR, T, true> : DFTOddPrime<7, DIR, T> {};

// composite length R = F * Q (four-step in registers):
//   x index j = j1 + F j2, spectrum index k = k2 + Q k1
//   step 1: DFT_Q over j2 for each j1; step 2: twiddle w_R^{j1 k2}; step 3: DFT_F over j1.
template <int R, int DIR, typename T>
struct DFT<R, DIR, T, false> {
  static constexpr int F = first_factor(R);
  static constexpr int Q = R / F;
  static_assert(F * Q == R && F > 1 && Q > 1, "unsupported DFT length");
  RK_HD static void run(cpx<T>* v) {
    cpx<T> tmp[R];
    sfor<F>([&](auto J1) {
      constexpr int j1 = decltype(J1)::value;
      cpx<T> s[Q];
      sfor<Q>([&](auto J2) { s[decltype(J2)::value] = v[j1 + F * decltype(J2)::value]; });
      DFT<Q, DIR, T>::run(s);
      sfor<Q>([&](auto K2) {
        constexpr int k2 = decltype(K2)::value;
        tmp[j1 * Q + k2] = twmul<j1 * k2, R, DIR>(s[k2]);
      });
    });
    sfor<Q>([&](auto K2) {
      constexpr int k2 = decltype(K2)::value;
      cpx<T> s[F];
      sfor<F>([&](auto J1) { s[decltype(J1)::value] = tmp[decltype(J1)::value * Q + k2]; });
      DFT<F, DIR, T>::run(s);
      sfor<F>([&](auto K1) { v[k2 + Q * decltype(K1)::value] = s[decltype(K1)::value]; });
    });
  }
};

// ----------------------------------------------------------------- misc
template <typename T>
RK_HD T rk_abs(T v) {
  return v < (T)0 ? -v : v;
}

}  // namespace rk
