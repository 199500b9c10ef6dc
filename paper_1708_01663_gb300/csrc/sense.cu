// Sensing operator and gradient assembly.
//
//  sense_forward : Z[t, m] = sum_n H[m, n] f[n] u_t[n]          (Eq. 5, Z = H diag(u) f)
//                  a complex GEMM [T x N] . [N x M] with split-K; the product
//                  f .* u is formed while staging the tile.
//  residual_and_D: w = Z - y, D = 1/2 sum |w|^2                  (Eq. 7, Prop. 1)
//                  (w = 0 at receivers a transmitter does not record)
//  sense_adjoint : z_t = H^H w_t and b_t = conj(f) .* z_t        (Eq. 13 right-hand side)
//  grad_assemble : g = sum_t conj(u_t) .* (z_t + G^H v_t)        (Eq. 12 before Re)
//                  and the gradient step s - gamma grad D        (Eq. 9 argument)
// The GEMMs run on the FP32 pipes: complex64 parity (1e-4) rules out TF32.
#include <math.h>

#include "common.cuh"

namespace cisor {

constexpr int GT = 32;  // transmitters per CTA tile
constexpr int GM = 64;  // receivers (forward) / pixels (adjoint) per CTA tile
constexpr int GK = 32;  // reduction tile

__global__ void __launch_bounds__(256) sense_fwd_kernel(const float2* __restrict__ H, const float2* __restrict__ f,
                                                        const float2* __restrict__ u, float2* __restrict__ part, int T,
                                                        int M, long long N, long long chunk) {
  __shared__ float2 Qs[GK][GT + 1];
  __shared__ float2 Hs[GK][GM + 1];
  const int m0 = blockIdx.x * GM, t0 = blockIdx.y * GT, ks = blockIdx.z;
  const long long kb = (long long)ks * chunk;
  const long long ke = min(N, kb + chunk);
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  float2 acc[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j] = make_float2(0.f, 0.f);
  for (long long k0 = kb; k0 < ke; k0 += GK) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = tid + 256 * q, kk = e & 31, mm = e >> 5;
      const long long k = k0 + kk;
      const int m = m0 + mm;
      Hs[kk][mm] = (k < ke && m < M) ? H[(long long)m * N + k] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + 256 * q, kk = e & 31, tt = e >> 5;
      const long long k = k0 + kk;
      const int t = t0 + tt;
      Qs[kk][tt] = (k < ke && t < T) ? c_mul(f[k], u[(long long)t * N + k]) : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < GK; ++kk) {
      float2 a[4], b[2];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = Qs[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 2; ++j) b[j] = Hs[kk][tx * 2 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) acc[i][j] = c_add(acc[i][j], c_mul(a[i], b[j]));
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int t = t0 + ty * 4 + i, m = m0 + tx * 2 + j;
      if (t < T && m < M) part[((long long)ks * T + t) * M + m] = acc[i][j];
    }
}

__global__ void __launch_bounds__(256) sense_reduce_kernel(const float2* __restrict__ part, int ks, int T, int M,
                                                           const float2* __restrict__ y, float2* __restrict__ Z,
                                                           float2* __restrict__ w, double* __restrict__ dsum,
                                                           const unsigned char* __restrict__ mask) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  double d = 0.0;
  if (idx < T * M) {
    double sx = 0.0, sy = 0.0;
    for (int k = 0; k < ks; ++k) {
      const float2 p = part[(long long)k * T * M + idx];
      sx += p.x;
      sy += p.y;
    }
    if (Z) Z[idx] = make_float2((float)sx, (float)sy);
    if (y) {
      const float2 yv = y[idx];
      const double on = (mask && !mask[idx]) ? 0.0 : 1.0;  // inactive receivers leave D and the adjoint
      const double wx = on * (sx - yv.x), wy = on * (sy - yv.y);
      if (w) w[idx] = make_float2((float)wx, (float)wy);
      d = 0.5 * (wx * wx + wy * wy);
    }
  }
  if (dsum) {
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
      atomicAdd(dsum, s);
    }
  }
}

__global__ void __launch_bounds__(256) sense_adj_kernel(const float2* __restrict__ H, const float2* __restrict__ w,
                                                        const float2* __restrict__ f, float2* __restrict__ z,
                                                        float2* __restrict__ b, int T, int M, long long N) {
  __shared__ float2 Hs[GK][GM];
  __shared__ float2 Ws[GK][GT + 1];
  const long long n0 = (long long)blockIdx.x * GM;
  const int t0 = blockIdx.y * GT;
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  float2 acc[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j] = make_float2(0.f, 0.f);
  for (int m0 = 0; m0 < M; m0 += GK) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = tid + 256 * q, nn = e & 63, mm = e >> 6;
      const int m = m0 + mm;
      const long long n = n0 + nn;
      Hs[mm][nn] = (m < M && n < N) ? H[(long long)m * N + n] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + 256 * q, mm = e & 31, tt = e >> 5;
      const int m = m0 + mm, t = t0 + tt;
      Ws[mm][tt] = (m < M && t < T) ? w[(long long)t * M + m] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll 8
    for (int mm = 0; mm < GK; ++mm) {
      float2 a[4], h[2];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = Ws[mm][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 2; ++j) h[j] = Hs[mm][tx * 2 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) acc[i][j] = c_add(acc[i][j], c_cjmul(h[j], a[i]));
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int t = t0 + ty * 4 + i;
      const long long n = n0 + tx * 2 + j;
      if (t < T && n < N) {
        const long long idx = (long long)t * N + n;
        if (z) z[idx] = acc[i][j];
        if (b) b[idx] = c_cjmul(f[n], acc[i][j]);
      }
    }
}

__global__ void __launch_bounds__(256) grad_kernel(const float2* __restrict__ u, const float2* __restrict__ gz, int T,
                                                   long long N, const float2* __restrict__ s, float gamma, int complex_f,
                                                   float2* __restrict__ grad, float2* __restrict__ zstep) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float2 g = make_float2(0.f, 0.f);
  for (int t = 0; t < T; ++t) g = c_add(g, c_cjmul(u[(long long)t * N + n], gz[(long long)t * N + n]));
  if (grad) grad[n] = g;
  if (zstep) {
    const float2 sv = s[n];
    zstep[n] = complex_f ? make_float2(sv.x - gamma * g.x, sv.y - gamma * g.y) : make_float2(sv.x - gamma * g.x, 0.f);
  }
}

// z = s - gamma g (real f: the real part of g only, Im z = 0): the gradient step of Eq. 9
__global__ void __launch_bounds__(256) grad_step_kernel(const float2* __restrict__ s, const float2* __restrict__ g,
                                                        long long N, float gamma, int complex_f,
                                                        float2* __restrict__ z) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const float2 sv = s[n], gv = g[n];
  z[n] = complex_f ? make_float2(sv.x - gamma * gv.x, sv.y - gamma * gv.y) : make_float2(sv.x - gamma * gv.x, 0.f);
}

cisor_status gradient_step(cisor_ctx* c, const float2* s, const float2* g, double gamma, float2* z) {
  grad_step_kernel<<<(unsigned)((c->N + 255) / 256), 256, 0, c->stream>>>(s, g, c->N, (float)gamma, c->complex_f, z);
  CISOR_CUDA(cudaGetLastError());
  c->launches += 1;
  return CISOR_OK;
}

cisor_status sense_forward(cisor_ctx* c, const float2* f, const float2* u, float2* Z, int ntx) {
  const long long chunk = ((c->N + c->ksplit - 1) / c->ksplit + GK - 1) / GK * GK;
  const int ks = (int)((c->N + chunk - 1) / chunk);
  dim3 g((c->M + GM - 1) / GM, (ntx + GT - 1) / GT, ks);
  sense_fwd_kernel<<<g, 256, 0, c->stream>>>(c->H, f, u, c->sense_part, ntx, c->M, c->N, chunk);
  CISOR_CUDA(cudaGetLastError());
  const int tm = ntx * c->M;
  sense_reduce_kernel<<<(tm + 255) / 256, 256, 0, c->stream>>>(c->sense_part, ks, ntx, c->M, nullptr, Z, nullptr,
                                                               nullptr, nullptr);
  CISOR_CUDA(cudaGetLastError());
  c->launches += 2;
  return CISOR_OK;
}

cisor_status residual_and_D(cisor_ctx* c, const float2* f, const float2* u, const float2* y, float2* Z, float2* w,
                            int ntx) {
  const long long chunk = ((c->N + c->ksplit - 1) / c->ksplit + GK - 1) / GK * GK;
  const int ks = (int)((c->N + chunk - 1) / chunk);
  dim3 g((c->M + GM - 1) / GM, (ntx + GT - 1) / GT, ks);
  sense_fwd_kernel<<<g, 256, 0, c->stream>>>(c->H, f, u, c->sense_part, ntx, c->M, c->N, chunk);
  CISOR_CUDA(cudaGetLastError());
  CISOR_CUDA(cudaMemsetAsync(c->dsum, 0, sizeof(double), c->stream));
  const int tm = ntx * c->M;
  sense_reduce_kernel<<<(tm + 255) / 256, 256, 0, c->stream>>>(c->sense_part, ks, ntx, c->M, y, Z, w, c->dsum,
                                                               c->rx_mask);
  CISOR_CUDA(cudaGetLastError());
  c->launches += 2;
  return CISOR_OK;
}

cisor_status sense_adjoint(cisor_ctx* c, const float2* f, const float2* w, float2* z, float2* b, int ntx) {
  dim3 g((unsigned)((c->N + GM - 1) / GM), (ntx + GT - 1) / GT);
  sense_adj_kernel<<<g, 256, 0, c->stream>>>(c->H, w, f, z, b, ntx, c->M, c->N);
  CISOR_CUDA(cudaGetLastError());
  c->launches += 1;
  return CISOR_OK;
}

cisor_status grad_assemble(cisor_ctx* c, const float2* u, const float2* gz, const float2* s, double gamma,
                           float2* grad, float2* zstep, int ntx) {
  grad_kernel<<<(unsigned)((c->N + 255) / 256), 256, 0, c->stream>>>(u, gz, ntx, c->N, s, (float)gamma, c->complex_f,
                                                                     grad, zstep);
  CISOR_CUDA(cudaGetLastError());
  c->launches += 1;
  return CISOR_OK;
}

}  // namespace cisor
