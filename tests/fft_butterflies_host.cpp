// Host build of the register butterflies in csrc/fft.cuh (radix 8, 16, 32 and
// the pruned variants whose upper half of inputs is zero), checked against the
// DFT definition X_k = sum_r x_r exp(-+2 pi i r k / N) evaluated in double
// precision.  Prints one line per butterfly: name, direction, worst error
// |X - X_ref| / sqrt(N) over 20 seeded random inputs.
#include <cuda_runtime.h>
static inline void __syncthreads() {}  // fft.cuh's block FFT names it; the butterflies never call it
#include <cmath>
#include <complex>
#include <cstdio>
#include <random>

#include "fft.cuh"

using namespace cisor;

template <int N, bool INV, class F> static double check(F f, bool lower_half_only) {
  std::mt19937 gen(1);
  std::normal_distribution<double> nd;
  double worst = 0;
  for (int trial = 0; trial < 20; ++trial) {
    float2 v[N];
    std::complex<double> x[N];
    for (int i = 0; i < N; ++i) {
      x[i] = (lower_half_only && i >= N / 2) ? 0.0 : std::complex<double>(nd(gen), nd(gen));
      v[i] = make_float2((float)x[i].real(), (float)x[i].imag());
    }
    f(v);
    for (int k = 0; k < N; ++k) {
      std::complex<double> s = 0;
      for (int r = 0; r < N; ++r) s += x[r] * std::polar(1.0, (INV ? 2.0 : -2.0) * M_PI * r * k / N);
      worst = std::max(worst, std::abs(s - std::complex<double>(v[k].x, v[k].y)) / std::sqrt((double)N));
    }
  }
  return worst;
}

int main() {
  printf("dft8 fwd %.3e\n", check<8, false>([](float2* v) { dft8<false>(v); }, false));
  printf("dft8 inv %.3e\n", check<8, true>([](float2* v) { dft8<true>(v); }, false));
  printf("dft8_lo fwd %.3e\n", check<8, false>([](float2* v) { dft8_lo<false>(v); }, true));
  printf("dft16 fwd %.3e\n", check<16, false>([](float2* v) { dft16<false>(v); }, false));
  printf("dft16 inv %.3e\n", check<16, true>([](float2* v) { dft16<true>(v); }, false));
  printf("dft16_lo fwd %.3e\n", check<16, false>([](float2* v) { dft16_lo<false>(v); }, true));
  printf("dft32 fwd %.3e\n", check<32, false>([](float2* v) { dft32<false>(v); }, false));
  printf("dft32 inv %.3e\n", check<32, true>([](float2* v) { dft32<true>(v); }, false));
  printf("dft32_lo fwd %.3e\n", check<32, false>([](float2* v) { dft32_lo<false>(v); }, true));
  return 0;
}
