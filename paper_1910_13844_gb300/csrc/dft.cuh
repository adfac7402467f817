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
__host__ __device__ __forceinline__ float2 twc(float2 a) {
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

// Dft<R, DIR, NIN, NOUT>: only a[0..NIN-1] may be nonzero (the rest is never
// read) and only X[0..NOUT-1] are produced (the other entries are left
// undefined).  Zero padding and cropping of the transforms use this to skip
// the corresponding arithmetic.
template <int R, int DIR, int NIN = R, int NOUT = R>
struct Dft;

template <int DIR, int NIN, int NOUT>
struct Dft<1, DIR, NIN, NOUT> {
  __host__ __device__ __forceinline__ static void run(float2*) {}
};

template <int DIR, int NIN, int NOUT>
struct Dft<2, DIR, NIN, NOUT> {
  __host__ __device__ __forceinline__ static void run(float2* a) {
    if constexpr (NIN >= 2) {
      float2 t = a[1];
      if constexpr (NOUT >= 2) a[1] = csub(a[0], t);
      a[0] = cadd(a[0], t);
    } else {
      if constexpr (NOUT >= 2) a[1] = a[0];
    }
  }
};

template <int DIR, int NIN, int NOUT>
struct Dft<3, DIR, NIN, NOUT> {
  __host__ __device__ __forceinline__ static void run(float2* a) {
    // X0 = a0 + a1 + a2 ; X1,2 = a0 - (a1+a2)/2 +/- DIR i (sqrt3/2)(a1 - a2)
    constexpr float h = 0.86602540378443864676f;
    const float2 a1 = NIN > 1 ? a[1] : make_float2(0.f, 0.f);
    const float2 a2 = NIN > 2 ? a[2] : make_float2(0.f, 0.f);
    float2 s = cadd(a1, a2);
    float2 d = csub(a1, a2);
    float2 m = make_float2(a[0].x - 0.5f * s.x, a[0].y - 0.5f * s.y);
    float2 r = DIR < 0 ? make_float2(h * d.y, -h * d.x) : make_float2(-h * d.y, h * d.x);
    a[0] = cadd(a[0], s);
    if constexpr (NOUT > 1) a[1] = cadd(m, r);
    if constexpr (NOUT > 2) a[2] = csub(m, r);
  }
};

template <int DIR, int NIN, int NOUT>
struct Dft<4, DIR, NIN, NOUT> {
  __host__ __device__ __forceinline__ static void run(float2* a) {
    if constexpr (NIN <= 2) {
      // a2 = a3 = 0: X0 = a0 + a1, X1 = a0 + w a1, X2 = a0 - a1, X3 = a0 - w a1 (w = DIR i)
      const float2 b = NIN > 1 ? a[1] : make_float2(0.f, 0.f);
      const float2 br = twc<1, 4, DIR>(b);
      const float2 a0 = a[0];
      a[0] = cadd(a0, b);
      if constexpr (NOUT > 1) a[1] = cadd(a0, br);
      if constexpr (NOUT > 2) a[2] = csub(a0, b);
      if constexpr (NOUT > 3) a[3] = csub(a0, br);
    } else {
      const float2 a3 = NIN > 3 ? a[3] : make_float2(0.f, 0.f);
      float2 s0 = cadd(a[0], a[2]), d0 = csub(a[0], a[2]);
      float2 s1 = cadd(a[1], a3), d1 = csub(a[1], a3);
      float2 d1r = twc<1, 4, DIR>(d1);
      a[0] = cadd(s0, s1);
      if constexpr (NOUT > 1) a[1] = cadd(d0, d1r);
      if constexpr (NOUT > 2) a[2] = csub(s0, s1);
      if constexpr (NOUT > 3) a[3] = csub(d0, d1r);
    }
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

__host__ __device__ constexpr int cdiv_pos(int a, int b) { return a <= 0 ? 0 : (a + b - 1) / b; }

// X[k1 + A k2] = sum_{n2<B} W_B^{n2 k2} W_R^{n2 k1} sum_{n1<A} x[B n1 + n2] W_A^{n1 k1}
// Input x[B n1 + n2] is nonzero only for B n1 + n2 < NIN; output X[k1 + A k2] is needed only for
// k1 + A k2 < NOUT.
template <int R, int DIR, int NIN, int NOUT>
struct Dft {
  static constexpr int A = Split<R>::A;
  static constexpr int B = R / A;
  __host__ __device__ __forceinline__ static void run(float2* a) {
    float2 t[B][A];
    inner<0>(a, t);
    outer<0>(a, t);
  }
  // step 1: the B sub-DFTs of length A, with their own input pruning, then the internal twiddles
  template <int N2>
  __host__ __device__ __forceinline__ static void inner(float2* a, float2 (&t)[B][A]) {
    if constexpr (N2 < B) {
      constexpr int nin = cdiv_pos(NIN - N2, B);
      if constexpr (nin > 0) {
#pragma unroll
        for (int n1 = 0; n1 < nin; ++n1) t[N2][n1] = a[B * n1 + N2];
        Dft<A, DIR, nin, A>::run(t[N2]);
      } else {
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1) t[N2][k1] = make_float2(0.f, 0.f);
      }
      apply_tw_k<N2, 1>(t);
      inner<N2 + 1>(a, t);
    }
  }
  // step 2: the A sub-DFTs of length B, each producing only the outputs that are needed
  template <int K1>
  __host__ __device__ __forceinline__ static void outer(float2* a, float2 (&t)[B][A]) {
    if constexpr (K1 < A) {
      constexpr int nout = cdiv_pos(NOUT - K1, A);
      if constexpr (nout > 0) {
        float2 u[B];
#pragma unroll
        for (int n2 = 0; n2 < B; ++n2) u[n2] = t[n2][K1];
        Dft<B, DIR, B, nout>::run(u);
#pragma unroll
        for (int k2 = 0; k2 < nout; ++k2) a[K1 + A * k2] = u[k2];
      }
      outer<K1 + 1>(a, t);
    }
  }
  template <int N2, int K1>
  __host__ __device__ __forceinline__ static void apply_tw_k(float2 (&t)[B][A]) {
    if constexpr (K1 < A && N2 > 0) {
      t[N2][K1] = twc<N2 * K1, R, DIR>(t[N2][K1]);
      apply_tw_k<N2, K1 + 1>(t);
    }
  }
};

}  // namespace lsgpu
