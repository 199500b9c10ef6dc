// GELU and its derivative for the FNO kernels, without a branch and with one
// reciprocal (plus one exponential for the derivative):
//   gelu(x)  = x Phi(x) = (x + |x| erf(|x| / sqrt 2)) / 2
//   gelu'(x) = Phi(x) + x phi(x),  phi(x) = exp(-x^2 / 2) / sqrt(2 pi)
// erf on z >= 0 is the rational form of Abramowitz & Stegun, Handbook of
// Mathematical Functions, 7.1.28 (after Hastings):
//   erf(z) = 1 - (1 + a1 z + a2 z^2 + ... + a6 z^6)^-16,  |error| <= 3e-7,
// with z clamped at 4 (erf(4) = 1 - 1.5e-8), which keeps the 16th power finite.
// In FP32 the 16th power multiplies the polynomial's rounding by 16: the
// evaluated erf is within 2e-6 (the host build of this header is checked
// against std::erf), far below the BF16-split GEMMs' 1.5e-5.
#pragma once
#include <math.h>

namespace cisor {

__host__ __device__ __forceinline__ float gelu_rcp(float p) {
#ifdef __CUDA_ARCH__
  return __fdividef(1.f, p);
#else
  return 1.f / p;
#endif
}

__host__ __device__ __forceinline__ float gelu_exp(float x) {
#ifdef __CUDA_ARCH__
  return __expf(x);
#else
  return expf(x);
#endif
}

// erf(z) for z >= 0
__host__ __device__ __forceinline__ float erf_pos(float z) {
  z = fminf(z, 4.f);
  float p = fmaf(4.30638e-5f, z, 2.765672e-4f);
  p = fmaf(p, z, 1.520143e-4f);
  p = fmaf(p, z, 9.2705272e-3f);
  p = fmaf(p, z, 4.22820123e-2f);
  p = fmaf(p, z, 7.05230784e-2f);
  p = fmaf(p, z, 1.f);
  p *= p;
  p *= p;
  p *= p;
  p *= p;
  return 1.f - gelu_rcp(p);
}

__host__ __device__ __forceinline__ float gelu_f(float x) {
  const float a = fabsf(x);
  return 0.5f * fmaf(a, erf_pos(a * 0.70710678118654752f), x);
}

__host__ __device__ __forceinline__ float gelu_grad_f(float x) {
  const float e = erf_pos(fabsf(x) * 0.70710678118654752f);
  const float phi = 0.5f * (1.f + copysignf(e, x));
  return fmaf(x * 0.39894228040143268f, gelu_exp(-0.5f * x * x), phi);
}

// both at once (one erf): g = gelu(x), gp = gelu'(x)
__host__ __device__ __forceinline__ void gelu_and_grad(float x, float& g, float& gp) {
  const float a = fabsf(x);
  const float e = erf_pos(a * 0.70710678118654752f);
  g = 0.5f * fmaf(a, e, x);
  gp = fmaf(x * 0.39894228040143268f, gelu_exp(-0.5f * x * x), 0.5f * (1.f + copysignf(e, x)));
}

}  // namespace cisor
