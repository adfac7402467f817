// Host-side check of the register DFTs used by the pencil passes (compiled by tests/test_dft_host.py).
#include <cstdio>
#include <cmath>
#include <complex>
#include <random>
#include "dft.cuh"
using namespace lsgpu;
template <int R, int DIR, int NIN, int NOUT>
double check() {
  std::mt19937 g(R * 131 + NIN * 7 + NOUT + (DIR > 0));
  std::normal_distribution<float> nd;
  float2 a[R]; std::complex<double> x[R];
  for (int i = 0; i < R; ++i) { a[i] = i < NIN ? make_float2(nd(g), nd(g)) : make_float2(NAN, NAN); x[i] = i < NIN ? std::complex<double>(a[i].x, a[i].y) : 0.0; }
  Dft<R, DIR, NIN, NOUT>::run(a);
  double err = 0, mag = 0;
  for (int k = 0; k < NOUT; ++k) {
    std::complex<double> X = 0;
    for (int n = 0; n < R; ++n) X += x[n] * std::polar(1.0, DIR * 2 * M_PI * n * k / R);
    err = std::max(err, std::abs(X - std::complex<double>(a[k].x, a[k].y)));
    mag = std::max(mag, std::abs(X));
  }
  return err / mag;
}
#define C(R, D, I, O) { double e = check<R, D, I, O>(); printf("R=%2d dir=%+d nin=%2d nout=%2d err=%.2e\n", R, D, I, O, e); worst = e > worst ? e : worst; }
int main() {
  double worst = 0;
  // every radix of the passes, both directions, full and half inputs (zero padding), full and
  // half outputs (cropping)
  C(2,-1,1,1) C(2,-1,1,2) C(2,-1,2,1) C(2,-1,2,2) C(2,1,1,1) C(2,1,1,2) C(2,1,2,1) C(2,1,2,2)
  C(3,-1,1,1) C(3,-1,1,3) C(3,-1,3,1) C(3,-1,3,3) C(3,1,1,1) C(3,1,1,3) C(3,1,3,1) C(3,1,3,3)
  C(4,-1,2,2) C(4,-1,2,4) C(4,-1,4,2) C(4,-1,4,4) C(4,1,2,2) C(4,1,2,4) C(4,1,4,2) C(4,1,4,4)
  C(6,-1,3,3) C(6,-1,3,6) C(6,-1,6,3) C(6,-1,6,6) C(6,1,3,3) C(6,1,3,6) C(6,1,6,3) C(6,1,6,6)
  C(8,-1,4,4) C(8,-1,4,8) C(8,-1,8,4) C(8,-1,8,8) C(8,1,4,4) C(8,1,4,8) C(8,1,8,4) C(8,1,8,8)
  C(12,-1,6,6) C(12,-1,6,12) C(12,-1,12,6) C(12,-1,12,12) C(12,1,6,6) C(12,1,6,12) C(12,1,12,6) C(12,1,12,12)
  C(16,-1,8,8) C(16,-1,8,16) C(16,-1,16,8) C(16,-1,16,16) C(16,1,8,8) C(16,1,8,16) C(16,1,16,8) C(16,1,16,16)
  C(24,-1,12,12) C(24,-1,12,24) C(24,-1,24,12) C(24,-1,24,24) C(24,1,12,12) C(24,1,12,24) C(24,1,24,12) C(24,1,24,24)
  C(32,-1,16,16) C(32,-1,16,32) C(32,-1,32,16) C(32,-1,32,32) C(32,1,16,16) C(32,1,16,32) C(32,1,32,16) C(32,1,32,32)
  printf("worst %.3e\n", worst);
  return worst < 3e-7 ? 0 : 1;
}
