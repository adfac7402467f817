// Register-resident small DFTs for the pencil FFT passes.
//
// Dft<R, DIR>::run(a) replaces a[0..R-1] by X[k] = sum_n a[n] exp(DIR * 2 pi i n k / R)
// (DIR = -1 forward, +1 inverse, unnormalised).  Composite sizes use one
// in-register Cooley-Tukey split R = A * B with compile-time twiddles.
#pragma once

#include "common.cuh"

namespace lsgpu {

// sin/cos of 2 pi j / R evaluated at compile time by a Taylor series in double.
__host__ __device__ constexpr double cx_pi() { return 3.14159265358979323846264338327950288; }

__host__ __device__ constexpr double cx_sin_series(double x) {
  double term = x, sum = x;
  for (int k = 1; k < 30; ++k) {
    term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double cx_cos_series(double x) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 30; ++k) {
    term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
    sum += term;
  }
  return sum;
}
// angle 2 pi j / R reduced to [-pi, pi]
__host__ __device__ constexpr double cx_angle(int j, int R) {
  int jj = ((j % R) + R) % R;
  if (2 * jj > R) jj -= R;
  return 2.0 * cx_pi() * (double)jj / (double)R;
}
__host__ __device__ constexpr double cx_cos(int j, int R) { return cx_cos_series(cx_angle(j, R)); }
__host__ __device__ constexpr double cx_sin(int j, int R) { return cx_sin_series(cx_angle(j, R)); }

// a *= exp(DIR * 2 pi i J / R), with the trivial angles (multiples of pi/2) done without multiplies.
template <int J, int R, int DIR>
__device__ __forceinline__ float2 twc(float2 a) {
  constexpr int jj = ((J % R) + R) % R;
  if constexpr (jj == 0) {
    return a;
  } else if constexpr (4 * jj == R) {  // exp(DIR i pi/2) = DIR i
    return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
  } else if constexpr (2 * jj == R) {
    return make_float2(-a.x, -a.y);
  } else if constexpr (4 * jj == 3 * R) {  // exp(DIR i 3pi/2) = -DIR i
    return DIR < 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
  } else {
    constexpr float c = (float)cx_cos(jj, R);
    constexpr float s = (float)(DIR * cx_sin(jj, R));
    return make_float2(a.x * c - a.y * s, a.x * s + a.y * c);
  }
}

template <int R, int DIR>
struct Dft;

template <int DIR>
struct Dft<1, DIR> {
  __device__ __forceinline__ static void run(float2*) {}
};

template <int DIR>
struct Dft<2, DIR> {
  __device__ __forceinline__ static void run(float2* a) {
    float2 t = a[1];
    a[1] = csub(a[0], t);
    a[0] = cadd(a[0], t);
  }
};

template <int DIR>
struct Dft<3, DIR> {
  __device__ __forceinline__ static void run(float2* a) {
    // X0 = a0 + a1 + a2 ; X1,2 = a0 - (a1+a2)/2 -/+ DIR i (sqrt3/2)(a1 - a2)
    constexpr float h = 0.86602540378443864676f;
    float2 s = cadd(a[1], a[2]);
    float2 d = csub(a[1], a[2]);
    float2 m = make_float2(a[0].x - 0.5f * s.x, a[0].y - 0.5f * s.y);
    // DIR * i * h * d
    float2 r = DIR < 0 ? make_float2(h * d.y, -h * d.x) : make_float2(-h * d.y, h * d.x);
    a[0] = cadd(a[0], s);
    a[1] = cadd(m, r);
    a[2] = csub(m, r);
  }
};

template <int DIR>
struct Dft<4, DIR> {
  __device__ __forceinline__ static void run(float2* a) {
    float2 s0 = cadd(a[0], a[2]), d0 = csub(a[0], a[2]);
    float2 s1 = cadd(a[1], a[3]), d1 = csub(a[1], a[3]);
    float2 d1r = twc<1, 4, DIR>(d1);
    a[0] = cadd(s0, s1);
    a[2] = csub(s0, s1);
    a[1] = cadd(d0, d1r);
    a[3] = csub(d0, d1r);
  }
};

// Split for composite sizes: R = A * B, A chosen below.
template <int R> struct Split;
template <> struct Split<6>  { static constexpr int A = 2; };
template <> struct Split<8>  { static constexpr int A = 2; };
template <> struct Split<12> { static constexpr int A = 4; };
template <> struct Split<16> { static constexpr int A = 4; };
template <> struct Split<24> { static constexpr int A = 8; };
template <> struct Split<32> { static constexpr int A = 8; };

// X[k1 + A k2] = sum_{n2<B} W_B^{n2 k2} W_R^{n2 k1} sum_{n1<A} x[B n1 + n2] W_A^{n1 k1}
template <int R, int DIR>
struct Dft {
  static constexpr int A = Split<R>::A;
  static constexpr int B = R / A;
  __device__ __forceinline__ static void run(float2* a) {
    float2 t[B][A];
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) {
#pragma unroll
      for (int n1 = 0; n1 < A; ++n1) t[n2][n1] = a[B * n1 + n2];
      Dft<A, DIR>::run(t[n2]);
    }
    apply_tw<1>(t);
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) {
      float2 u[B];
#pragma unroll
      for (int n2 = 0; n2 < B; ++n2) u[n2] = t[n2][k1];
      Dft<B, DIR>::run(u);
#pragma unroll
      for (int k2 = 0; k2 < B; ++k2) a[k1 + A * k2] = u[k2];
    }
  }
  // internal twiddles W_R^{n2 k1}, unrolled at compile time
  template <int N2>
  __device__ __forceinline__ static void apply_tw(float2 (&t)[B][A]) {
    if constexpr (N2 < B) {
      apply_tw_k<N2, 1>(t);
      apply_tw<N2 + 1>(t);
    }
  }
  template <int N2, int K1>
  __device__ __forceinline__ static void apply_tw_k(float2 (&t)[B][A]) {
    if constexpr (K1 < A) {
      t[N2][K1] = twc<N2 * K1, R, DIR>(t[N2][K1]);
      apply_tw_k<N2, K1 + 1>(t);
    }
  }
};

}  // namespace lsgpu
