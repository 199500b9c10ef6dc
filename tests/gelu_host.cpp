// Host build of csrc/gelu.cuh checked against the definitions in double
// precision: gelu(x) = x (1 + erf(x / sqrt 2)) / 2 and its derivative
// (1 + erf(x / sqrt 2)) / 2 + x exp(-x^2 / 2) / sqrt(2 pi), on a dense grid of
// [-12, 12] (gelu_f, gelu_grad_f and the combined gelu_and_grad).  Prints:
// worst |gelu error| / max(1, |x|), worst |gelu' error|, worst erf error.
#include <cuda_runtime.h>
#include <cmath>
#include <cstdio>

#include "gelu.cuh"

int main() {
  double eg = 0, ed = 0, ee = 0;
  for (int i = 0; i <= 2400000; ++i) {
    const double x = -12.0 + i * 1e-5;
    const float xf = (float)x;
    const double xd = (double)xf;
    const double erf_ref = std::erf(xd / std::sqrt(2.0));
    const double g = 0.5 * xd * (1.0 + erf_ref);
    const double d = 0.5 * (1.0 + erf_ref) + xd * std::exp(-0.5 * xd * xd) / std::sqrt(2.0 * M_PI);
    float g2, d2;
    cisor::gelu_and_grad(xf, g2, d2);
    eg = std::fmax(eg, std::fabs((double)cisor::gelu_f(xf) - g) / std::fmax(1.0, std::fabs(xd)));
    eg = std::fmax(eg, std::fabs((double)g2 - g) / std::fmax(1.0, std::fabs(xd)));
    ed = std::fmax(ed, std::fabs((double)cisor::gelu_grad_f(xf) - d));
    ed = std::fmax(ed, std::fabs((double)d2 - d));
    if (xd >= 0) ee = std::fmax(ee, std::fabs((double)cisor::erf_pos(xf) - std::erf(xd)));
  }
  std::printf("%.3e %.3e %.3e\n", eg, ed, ee);
  return 0;
}
