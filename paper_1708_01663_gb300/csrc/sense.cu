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
// The GEMMs run on the tensor cores (TF32 hi / lo products, sense_tc.cu) where
// the sizes allow it (T <= 128, even M and field length) and otherwise on the
// FP32 pipes with the tiles below; a single TF32 product would break the 1e-5
// sensing parity.
#include <math.h>

#include "common.cuh"

namespace cisor {

// Tiles of the two complex GEMMs: 32 transmitters x 128 receivers (forward) or
// pixels (adjoint) per CTA, 16 along the reduction.  Thread (tx, ty) = (lane,
// warp) owns transmitters ty + 8i and receivers / pixels tx + 32j (i, j < 4):
// the transmitter operand is a warp-wide broadcast and the other one is read
// at consecutive addresses, so the shared-memory reads are conflict-free; the
// transposed stores use a pitch of 129 / 33 elements.  Tiles are staged
// through registers one step ahead (double buffer, one barrier per step).
constexpr int GT = 32;   // transmitters per CTA tile
constexpr int GM = 128;  // receivers (forward) / pixels (adjoint) per CTA tile
constexpr int GK = 16;   // reduction tile

int sense_tiles(int M, int T) { return ((M + GM - 1) / GM) * ((T + GT - 1) / GT); }

// N is the reduction length (the field length: pixels x components); f repeats with period NP (pixels).
__device__ __forceinline__ long long fperiod(long long k, long long NP) {
  while (k >= NP) k -= NP;
  return k;
}

__global__ void __launch_bounds__(256, 2) sense_fwd_kernel(const float2* __restrict__ H, const float2* __restrict__ f,
                                                        const float2* __restrict__ u, float2* __restrict__ part, int T,
                                                        int M, long long N, long long chunk, long long NP) {
  __shared__ float2 Hs[2][GK][GM + 1];
  __shared__ float2 Qs[2][GK][GT + 1];
  const int m0 = blockIdx.x * GM, t0 = blockIdx.y * GT, ks = blockIdx.z;
  const long long kb = (long long)ks * chunk;
  const long long ke = min(N, kb + chunk);
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  float2 hr[8], qr[2];
  auto load = [&](long long k0) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = tid + 256 * q, kk = e & (GK - 1), mm = e >> 4;
      const long long k = k0 + kk;
      const int m = m0 + mm;
      hr[q] = (k < ke && m < M) ? H[(long long)m * N + k] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int e = tid + 256 * q, kk = e & (GK - 1), tt = e >> 4;
      const long long k = k0 + kk;
      const int t = t0 + tt;
      qr[q] = (k < ke && t < T) ? c_mul(f[fperiod(k, NP)], u[(long long)t * N + k]) : make_float2(0.f, 0.f);
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = tid + 256 * q;
      Hs[buf][e & (GK - 1)][e >> 4] = hr[q];
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int e = tid + 256 * q;
      Qs[buf][e & (GK - 1)][e >> 4] = qr[q];
    }
  };
  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  load(kb);
  stash(0);
  __syncthreads();
  int buf = 0;
  for (long long k0 = kb; k0 < ke; k0 += GK) {
    const bool more = k0 + GK < ke;
    if (more) load(k0 + GK);
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      float2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = Qs[buf][kk][ty + 8 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Hs[buf][kk][tx + 32 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = c_fma(a[i], b[j], acc[i][j]);
    }
    if (more) stash(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int t = t0 + ty + 8 * i, m = m0 + tx + 32 * j;
      if (t < T && m < M) part[((long long)ks * T + t) * M + m] = acc[i][j];
    }
}

// Z = sum of the ks split-K partials in FP64, w = Z - y (0 at receivers a transmitter does not record), and
// D += 1/2 sum |w|^2.  A CTA takes 32 consecutive entries (lanes, coalesced); its 8 warps sum the partials
// k = w, w + 8, ... and warp 0 adds the 8 sums in warp order (the same order every call).
constexpr int RED_WARPS = 8;
__global__ void __launch_bounds__(32 * RED_WARPS) sense_reduce_kernel(const float2* __restrict__ part, int ks, int T,
                                                                     int M, const float2* __restrict__ y,
                                                                     float2* __restrict__ Z, float2* __restrict__ w,
                                                                     double* __restrict__ dsum,
                                                                     const unsigned char* __restrict__ mask) {
  __shared__ double2 red[RED_WARPS][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int idx = blockIdx.x * 32 + lane;
  const long long TM = (long long)T * M;
  double sx = 0.0, sy = 0.0;
  if (idx < TM) {
#pragma unroll 4
    for (int k = warp; k < ks; k += RED_WARPS) {
      const float2 p = part[(long long)k * TM + idx];
      sx += p.x;
      sy += p.y;
    }
  }
  red[warp][lane] = make_double2(sx, sy);
  __syncthreads();
  if (warp != 0) return;
  double d = 0.0;
  if (idx < TM) {
    sx = 0.0;
    sy = 0.0;
#pragma unroll
    for (int i = 0; i < RED_WARPS; ++i) {
      sx += red[i][lane].x;
      sy += red[i][lane].y;
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
    if (lane == 0) atomicAdd(dsum, d);
  }
}

// One stage of the adjoint's operand tiles: H rows m0..m0+15 at pixels n0..n0+127
// (coalesced along n) and w of the 32 transmitters at those receivers.
__device__ __forceinline__ void adj_load(const float2* __restrict__ H, const float2* __restrict__ w, int tid, int m0,
                                         long long n0, int t0, int T, int M, long long N, float2 (&hr)[8],
                                         float2 (&wr)[2]) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int e = tid + 256 * q, nn = e & (GM - 1), mm = e >> 7;
    const int m = m0 + mm;
    const long long n = n0 + nn;
    hr[q] = (m < M && n < N) ? H[(long long)m * N + n] : make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int e = tid + 256 * q, mm = e & (GK - 1), tt = e >> 4;
    const int m = m0 + mm, t = t0 + tt;
    wr[q] = (m < M && t < T) ? w[(long long)t * M + m] : make_float2(0.f, 0.f);
  }
}

__global__ void __launch_bounds__(256, 2) sense_adj_kernel(const float2* __restrict__ H, const float2* __restrict__ w,
                                                        const float2* __restrict__ f, float2* __restrict__ z,
                                                        float2* __restrict__ b, int T, int M, long long N,
                                                        long long NP) {
  __shared__ float2 Hs[2][GK][GM];
  __shared__ float2 Ws[2][GK][GT + 1];
  const long long n0 = (long long)blockIdx.x * GM;
  const int t0 = blockIdx.y * GT;
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  float2 hr[8], wr[2];
  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  adj_load(H, w, tid, 0, n0, t0, T, M, N, hr, wr);
#pragma unroll
  for (int q = 0; q < 8; ++q) Hs[0][(tid + 256 * q) >> 7][(tid + 256 * q) & (GM - 1)] = hr[q];
#pragma unroll
  for (int q = 0; q < 2; ++q) Ws[0][(tid + 256 * q) & (GK - 1)][(tid + 256 * q) >> 4] = wr[q];
  __syncthreads();
  int buf = 0;
  for (int m0 = 0; m0 < M; m0 += GK) {
    const bool more = m0 + GK < M;
    if (more) adj_load(H, w, tid, m0 + GK, n0, t0, T, M, N, hr, wr);
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      float2 a[4], h[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = Ws[buf][kk][ty + 8 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) h[j] = Hs[buf][kk][tx + 32 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = c_cjfma(h[j], a[i], acc[i][j]);
    }
    if (more) {
#pragma unroll
      for (int q = 0; q < 8; ++q) Hs[buf ^ 1][(tid + 256 * q) >> 7][(tid + 256 * q) & (GM - 1)] = hr[q];
#pragma unroll
      for (int q = 0; q < 2; ++q) Ws[buf ^ 1][(tid + 256 * q) & (GK - 1)][(tid + 256 * q) >> 4] = wr[q];
    }
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int t = t0 + ty + 8 * i;
      const long long n = n0 + tx + 32 * j;
      if (t < T && n < N) {
        const long long idx = (long long)t * N + n;
        if (z) z[idx] = acc[i][j];
        if (b) b[idx] = c_cjmul(f[fperiod(n, NP)], acc[i][j]);
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

// split-K partials of Z = H (f .* u) into c->sense_part: tensor cores where available, else the FP32 pipes
static cisor_status sense_partials(cisor_ctx* c, const float2* f, const float2* u, int ntx, int* splits) {
  if (c->Ht) return sense_tc_forward(c, f, u, ntx, splits);
  const long long chunk = ((c->Nf + c->ksplit - 1) / c->ksplit + GK - 1) / GK * GK;
  const int ks = (int)((c->Nf + chunk - 1) / chunk);
  dim3 g((c->M + GM - 1) / GM, (ntx + GT - 1) / GT, ks);
  sense_fwd_kernel<<<g, 256, 0, c->stream>>>(c->H, f, u, c->sense_part, ntx, c->M, c->Nf, chunk, c->N);
  CISOR_CUDA(cudaGetLastError());
  *splits = ks;
  return CISOR_OK;
}

cisor_status sense_forward(cisor_ctx* c, const float2* f, const float2* u, float2* Z, int ntx) {
  int ks = 0;
  CISOR_TRY(sense_partials(c, f, u, ntx, &ks));
  const int tm = ntx * c->M;
  sense_reduce_kernel<<<(tm + 31) / 32, 32 * RED_WARPS, 0, c->stream>>>(c->sense_part, ks, ntx, c->M, nullptr, Z,
                                                                      nullptr, nullptr, nullptr);
  CISOR_CUDA(cudaGetLastError());
  c->launches += 2;
  return CISOR_OK;
}

cisor_status residual_and_D(cisor_ctx* c, const float2* f, const float2* u, const float2* y, float2* Z, float2* w,
                            int ntx) {
  int ks = 0;
  CISOR_TRY(sense_partials(c, f, u, ntx, &ks));
  CISOR_CUDA(cudaMemsetAsync(c->dsum, 0, sizeof(double), c->stream));
  const int tm = ntx * c->M;
  sense_reduce_kernel<<<(tm + 31) / 32, 32 * RED_WARPS, 0, c->stream>>>(c->sense_part, ks, ntx, c->M, y, Z, w,
                                                                      c->dsum, c->rx_mask);
  CISOR_CUDA(cudaGetLastError());
  c->launches += 2;
  return CISOR_OK;
}

cisor_status sense_adjoint(cisor_ctx* c, const float2* f, const float2* w, float2* z, float2* b, int ntx) {
  if (c->Ht) {
    CISOR_TRY(sense_tc_adjoint(c, f, w, z, b, ntx));
    c->launches += 1;
    return CISOR_OK;
  }
  dim3 g((unsigned)((c->Nf + GM - 1) / GM), (ntx + GT - 1) / GT);
  sense_adj_kernel<<<g, 256, 0, c->stream>>>(c->H, w, f, z, b, ntx, c->M, c->Nf, c->N);
  CISOR_CUDA(cudaGetLastError());
  c->launches += 1;
  return CISOR_OK;
}

cisor_status grad_assemble(cisor_ctx* c, const float2* u, const float2* gz, const float2* s, double gamma,
                           float2* grad, float2* zstep, int ntx) {
  // the components of the vectorial model are consecutive [N] blocks of a transmitter: sum them too
  grad_kernel<<<(unsigned)((c->N + 255) / 256), 256, 0, c->stream>>>(u, gz, ntx * c->ncomp, c->N, s, (float)gamma,
                                                                     c->complex_f, grad, zstep);
  CISOR_CUDA(cudaGetLastError());
  c->launches += 1;
  return CISOR_OK;
}

}  // namespace cisor
