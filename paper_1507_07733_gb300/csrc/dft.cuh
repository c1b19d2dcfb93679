// dft.cuh -- complex helpers and fully unrolled in-register DFTs (sm_103a).
//
// The transforms of the unfolding path (forward transform of the station voltages,
// inverse transform of the unfolded E-field spectrum; arXiv 1507.07733 Sec. 2 and 4) are
// built from small DFTs held in registers. All twiddles inside these DFTs are compile-time
// constants: their cosines and sines are evaluated at compile time from Taylor series in
// double precision after exact integer reduction of the angle 2*pi*k/R, then rounded once
// to float.
#pragma once
#include <cuda_runtime.h>
#include <type_traits>
#include <utility>

namespace aerafold {

// ---- compile-time trigonometry ---------------------------------------------------------

__host__ __device__ constexpr double cx_sin_poly(double x) {
  double t = x, s = x;
  const double x2 = x * x;
  for (int i = 1; i < 16; ++i) {
    t *= -x2 / double((2 * i) * (2 * i + 1));
    s += t;
  }
  return s;
}

__host__ __device__ constexpr double cx_cos_poly(double x) {
  double t = 1.0, s = 1.0;
  const double x2 = x * x;
  for (int i = 1; i < 16; ++i) {
    t *= -x2 / double((2 * i - 1) * (2 * i));
    s += t;
  }
  return s;
}

constexpr double kTwoPi = 6.283185307179586476925286766559;

// cos(2 pi k / R) and sin(2 pi k / R) for R a multiple of 4 (or R in {1, 2}); k any integer.
struct CS { double c, s; };
__host__ __device__ constexpr CS cx_cossin(long k, long R) {
  k %= R;
  if (k < 0) k += R;
  if (R == 1) return {1.0, 0.0};
  if (R == 2) return k == 0 ? CS{1.0, 0.0} : CS{-1.0, 0.0};
  const long q = (4 * k) / R;          // quadrant 0..3
  const long kr = k - q * (R / 4);     // 0 <= kr < R/4
  double c = 0.0, s = 0.0;
  if (2 * kr <= R / 4) {               // angle <= pi/4
    const double a = kTwoPi * double(kr) / double(R);
    c = cx_cos_poly(a);
    s = cx_sin_poly(a);
  } else {                             // use the complementary angle pi/2 - a
    const double a = kTwoPi * double(R / 4 - kr) / double(R);
    c = cx_sin_poly(a);
    s = cx_cos_poly(a);
  }
  switch (q) {                         // rotate by q quarter turns
    case 0: return {c, s};
    case 1: return {-s, c};
    case 2: return {-c, -s};
    default: return {s, -c};
  }
}

// W_R^k with sign: exp(SIGN * 2 pi i k / R), rounded to float.
template <long K, long R, int SIGN>
struct Tw {
  static constexpr CS cs = cx_cossin(K, R);
  static constexpr float re = float(cs.c);
  static constexpr float im = float(SIGN > 0 ? cs.s : -cs.s);
};

// ---- complex helpers ---------------------------------------------------------------------

// Complex add and subtract on the (re, im) register pair as one packed FP32x2 instruction
// (sm_100 and later); a - b is formed as fma(b, -1, a), which rounds like a subtraction.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

// multiply by exp(SIGN * 2 pi i K / R), with the trivial angles done by swaps and signs
template <long K, long R, int SIGN>
__device__ __forceinline__ float2 twmul(float2 a) {
  constexpr long k = ((K % R) + R) % R;
  if constexpr (k == 0) {
    return a;
  } else if constexpr (2 * k == R) {
    return make_float2(-a.x, -a.y);
  } else if constexpr (4 * k == R) {            // SIGN * i
    return SIGN > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
  } else if constexpr (4 * k == 3 * R) {        // -SIGN * i
    return SIGN > 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
  } else if constexpr ((8 * k) % R == 0) {      // odd multiples of pi/4: |re| == |im|
    constexpr float c = Tw<k, R, SIGN>::re;
    constexpr float s = Tw<k, R, SIGN>::im;
    constexpr float sc = (s > 0) == (c > 0) ? 1.0f : -1.0f;  // s == sc * c
    return make_float2(c * (a.x - sc * a.y), c * (sc * a.x + a.y));
  } else {
    constexpr float c = Tw<k, R, SIGN>::re;
    constexpr float s = Tw<k, R, SIGN>::im;
    return make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.x, s, a.y * c));
  }
}

// ---- compile-time loop -------------------------------------------------------------------

template <int I, int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, N>(f);
  }
}

// ---- in-register DFTs: v[k] <- sum_n v[n] exp(SIGN 2 pi i k n / R), natural order ------

template <int R, int SIGN>
__device__ __forceinline__ void dft(float2 (&v)[R]);

template <int SIGN>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  const float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <int SIGN>
__device__ __forceinline__ void dft4(float2 (&v)[4]) {
  const float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
  const float2 s13 = cadd(v[1], v[3]), d13 = csub(v[1], v[3]);
  v[0] = cadd(s02, s13);
  v[2] = csub(s02, s13);
  // d02 +- SIGN i d13: the rotation mixes components, so these stay scalar
  if constexpr (SIGN > 0) {
    v[1] = make_float2(d02.x - d13.y, d02.y + d13.x);
    v[3] = make_float2(d02.x + d13.y, d02.y - d13.x);
  } else {
    v[1] = make_float2(d02.x + d13.y, d02.y - d13.x);
    v[3] = make_float2(d02.x - d13.y, d02.y + d13.x);
  }
}

// R = R1 * R2: input n = n1 + R1 n2, output k = k2 + R2 k1 (decimation in time).
template <int R1, int R2, int SIGN>
__device__ __forceinline__ void dft_two_level(float2 (&v)[R1 * R2]) {
  constexpr int R = R1 * R2;
  float2 t[R1][R2];
  static_for<0, R1>([&](auto n1) {
    static_for<0, R2>([&](auto n2) { t[n1][n2] = v[n1 + R1 * n2]; });
    dft<R2, SIGN>(t[n1]);
    static_for<0, R2>([&](auto k2) {
      t[n1][k2] = twmul<long(decltype(n1)::value) * long(decltype(k2)::value), R, SIGN>(t[n1][k2]);
    });
  });
  static_for<0, R2>([&](auto k2) {
    float2 u[R1];
    static_for<0, R1>([&](auto n1) { u[n1] = t[n1][k2]; });
    dft<R1, SIGN>(u);
    static_for<0, R1>([&](auto k1) { v[k2 + R2 * k1] = u[k1]; });
  });
}

template <int R, int SIGN>
__device__ __forceinline__ void dft(float2 (&v)[R]) {
  if constexpr (R == 1) {
  } else if constexpr (R == 2) {
    dft2<SIGN>(v[0], v[1]);
  } else if constexpr (R == 4) {
    dft4<SIGN>(v);
  } else if constexpr (R == 8) {
    dft_two_level<2, 4, SIGN>(v);
  } else {
    static_assert(R % 4 == 0, "DFT size must be 1, 2 or a multiple of 4");
    dft_two_level<4, R / 4, SIGN>(v);
  }
}

}  // namespace aerafold
