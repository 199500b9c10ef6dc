// Learned warm start for the field solves: a Fourier neural operator (FNO)
// that predicts the scattered field u - u_in from (f, u_in), trained on
// fields the solver itself produces.  Not part of the paper; the plain solve
// stays the fallback and still decides convergence (the prediction is only an
// initial guess x0 for A u = u_in).
//
// Network (grid 128 x 128, width 32, 16 modes, 4 Fourier layers, hidden 128):
//   a  = (Re f, Im f, Re u_in, Im u_in, d_x, d_y, x, y)  8 channels; d is the
//        unit local propagation direction of u_in (phase gradient by central
//        differences, clamped at the edges)
//   v0 = W0 a + b0                                       1x1 lifting
//   v_l = GELU(Lsyn(R_l . S(v_{l-1})) + W_l v_{l-1} + b_l)  (no GELU on the last)
//   out = P2 GELU(P1 v_4 + c1) + c2,  e = out_0 + j out_1, predicted u - u_in = u_in e
// (the demodulated target keeps forward-scattered energy at low frequencies,
// inside the 16 retained modes; the incident carrier itself sits at 16 cycles
// per side at lambda/8)
// S keeps kx in {0..15, 112..127} (rows) x ky in {0..15} (columns) of the
// 2D DFT; Lsyn is (1/128^2) Re of the truncated inverse with weight 2 on
// ky > 0.  Loss: mean over samples of ||out - t|| / ||t||.
// Weights are held in FP32 (master, Adam state) and read by the kernels from
// a BF16 copy; activations and accumulation are FP32.  The 2D transforms use
// the register-boundary Stockham FFT (P = 128) with pruned inputs/outputs.
#include <math.h>
#include <cuda_bf16.h>

#include <new>

#include "common.cuh"
#include "regfft.cuh"

namespace cisor {

constexpr int FN = 128, FNN = FN * FN, FC = 32, FM = 16, FKX = 2 * FM, FMODES = FKX * FM, FH = 128, FL = 4;
constexpr long long F_LAYER = (long long)FMODES * FC * FC * 2 + FC * FC + FC;  // floats per Fourier layer
constexpr int FIN = 8;  // input channels
constexpr long long F_W0 = 0, F_B0 = FC * FIN, F_LAYERS = F_B0 + FC;
constexpr long long F_P1 = F_LAYERS + FL * F_LAYER, F_C1 = F_P1 + FH * FC, F_P2 = F_C1 + FH, F_C2 = F_P2 + 2 * FH;
constexpr long long F_TOTAL = F_C2 + 2;
__host__ __device__ constexpr long long f_R(int l) { return F_LAYERS + l * F_LAYER; }
__host__ __device__ constexpr long long f_W(int l) { return f_R(l) + (long long)FMODES * FC * FC * 2; }
__host__ __device__ constexpr long long f_B(int l) { return f_W(l) + FC * FC; }

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

// ------------------------------------------------------------------ kernels

__global__ void fno_features_lift(const float2* __restrict__ f, int f_per_sample, const float2* __restrict__ u_in,
                                  const __nv_bfloat16* __restrict__ wbf, const float* __restrict__ pm, int B,
                                  float* __restrict__ feat, float* __restrict__ v0) {
  __shared__ float W[FC * FIN], bb[FC];
  for (int i = threadIdx.x; i < FC * FIN; i += blockDim.x) W[i] = __bfloat162float(wbf[F_W0 + i]);
  for (int i = threadIdx.x; i < FC; i += blockDim.x) bb[i] = pm[F_B0 + i];
  __syncthreads();
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)B * FNN) return;
  const int b = (int)(idx / FNN), pix = (int)(idx % FNN);
  const int iy = pix / FN, ix = pix % FN;
  const float2 fv = f[(f_per_sample ? (long long)b * FNN : 0) + pix];
  const float2* ub = u_in + (long long)b * FNN;
  const float2 u = ub[pix];
  // central differences, clamped at the edges
  const float2 gx = c_scale(c_sub(ub[iy * FN + min(ix + 1, FN - 1)], ub[iy * FN + max(ix - 1, 0)]), 0.5f);
  const float2 gy = c_scale(c_sub(ub[min(iy + 1, FN - 1) * FN + ix], ub[max(iy - 1, 0) * FN + ix]), 0.5f);
  const float vx = c_cjmul(u, gx).y, vy = c_cjmul(u, gy).y;
  const float nv = sqrtf(vx * vx + vy * vy);
  const float dx = nv > 0.f ? vx / nv : 0.f, dy = nv > 0.f ? vy / nv : 0.f;
  const float a[FIN] = {fv.x, fv.y, u.x, u.y, dx, dy, (ix + 0.5f) / FN - 0.5f, (iy + 0.5f) / FN - 0.5f};
#pragma unroll
  for (int k = 0; k < FIN; ++k) feat[((long long)b * FIN + k) * FNN + pix] = a[k];
#pragma unroll 4
  for (int c = 0; c < FC; ++c) {
    float s = bb[c];
#pragma unroll
    for (int k = 0; k < FIN; ++k) s += W[c * FIN + k] * a[k];
    v0[((long long)b * FC + c) * FNN + pix] = s;
  }
}

// X[img][kx_idx*16 + ky] = wscale(ky) * sum v[iy][ix] exp(-2 pi j (kx iy + ky ix)/128), one CTA per image.
// wscale(ky) = scale * (weighted && ky > 0 ? 2 : 1).
__global__ void __launch_bounds__(256) fno_analysis(const float* __restrict__ v, float2* __restrict__ X,
                                                    const float2* __restrict__ twst, float scale, int weighted) {
  typedef TwTable<FN, false> TT;
  constexpr int PP = FN + FN / 16;
  __shared__ float2 tw[TT::SIZE];
  __shared__ float2 xbuf[16 * PP];    // exchange buffer (rows, then columns)
  __shared__ float2 colbuf[FN * FM];  // row-transform outputs ky < 16, column layout
  const long long img = blockIdx.x;
  const float* src = v + img * FNN;
  for (int i = threadIdx.x; i < TT::SIZE; i += 256) tw[i] = twst[i];
  const int lt = threadIdx.x & 15, row = threadIdx.x >> 4;
  const ColLay<FM> clay{lt};
  for (int r0 = 0; r0 < FN; r0 += 16) {
    const int iy = r0 + row;
    float2 x[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) x[r] = make_float2(src[iy * FN + lt + 16 * r], 0.f);
    reg_fft<FN, false, false>(x, xbuf, RowLayA<FN>{row * PP}, RowLayB<FN>{row * PP}, lt, tw);
    // output element lt (ky = lt) sits in x[0]
    colbuf[ColLay<FM>{lt}(iy)] = x[0];
  }
  __syncthreads();
  // column transforms: thread (w = ky, lt)
  const int ky = threadIdx.x % FM, ct = threadIdx.x / FM;
  const ColLay<FM> lay{ky};
  float2 x[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) x[r] = colbuf[lay(ct + 16 * r)];
  reg_fft<FN, false, false>(x, xbuf, lay, lay, ct, tw);
  const float ws = scale * ((weighted && ky > 0) ? 2.f : 1.f);
  // outputs: kx = ct in x[0], kx = 112 + ct in x[7]
  float2* dst = X + img * FMODES;
  dst[ct * FM + ky] = make_float2(x[0].x * ws, x[0].y * ws);
  dst[(FM + ct) * FM + ky] = make_float2(x[7].x * ws, x[7].y * ws);
  (void)clay;
}

// s[iy][ix] (+)= scale * Re sum_{kx,ky} w_ky Y[kx][ky] exp(+2 pi j (kx iy + ky ix)/128), one CTA per image.
__global__ void __launch_bounds__(256) fno_synthesis(const float2* __restrict__ Y, float* __restrict__ s,
                                                     const float2* __restrict__ twst, float scale, int weighted,
                                                     int accumulate) {
  typedef TwTable<FN, true> TT;
  constexpr int PP = FN + FN / 16;
  __shared__ float2 tw[TT::SIZE];
  __shared__ float2 xbuf[16 * PP];
  __shared__ float2 colbuf[FN * FM];
  const long long img = blockIdx.x;
  for (int i = threadIdx.x; i < TT::SIZE; i += 256) tw[i] = twst[TW_STRIDE + i];
  const float2* src = Y + img * FMODES;
  // column inverse transforms (along iy) of the 32 kept kx modes, thread (w = ky, ct)
  {
    const int ky = threadIdx.x % FM, ct = threadIdx.x / FM;
    const float ws = scale * ((weighted && ky > 0) ? 2.f : 1.f);
    const ColLay<FM> lay{ky};
    float2 x[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) x[r] = make_float2(0.f, 0.f);
    // reversed plan for 128 starts with radix 2: input element ct + 16 q + 64 r sits in x[2 q + r]
    const float2 a = src[ct * FM + ky], b = src[(FM + ct) * FM + ky];
    x[0] = make_float2(a.x * ws, a.y * ws);             // kx = ct        (q = 0, r = 0)
    x[7] = make_float2(b.x * ws, b.y * ws);             // kx = 112 + ct  (q = 3, r = 1)
    reg_fft<FN, true, true>(x, xbuf, lay, lay, ct, tw);
    // outputs iy = ct + 16 r in x[r]
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 8; ++r) colbuf[lay(ct + 16 * r)] = x[r];
  }
  __syncthreads();
  float* dst = s + img * FNN;
  const int lt = threadIdx.x & 15, row = threadIdx.x >> 4;
  for (int r0 = 0; r0 < FN; r0 += 16) {
    const int iy = r0 + row;
    float2 x[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) x[r] = make_float2(0.f, 0.f);
    x[0] = colbuf[ColLay<FM>{lt}(iy)];                   // ky = lt (element lt, q = 0, r = 0)
    reg_fft<FN, true, true>(x, xbuf, RowLayA<FN>{row * PP}, RowLayB<FN>{row * PP}, lt, tw);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      float* o = dst + iy * FN + lt + 16 * r;
      *o = accumulate ? (*o + x[r].x) : x[r].x;
    }
  }
}

// Y[b][o][m] = sum_i R[m][i][o] X[b][i][m], one CTA per mode.
__global__ void __launch_bounds__(256) fno_mix_fwd(const float2* __restrict__ X, const __nv_bfloat16* __restrict__ wbf,
                                                   long long roff, int B, float2* __restrict__ Y) {
  __shared__ float2 R[FC * FC];
  __shared__ float2 Xm[64 * FC];
  const int m = blockIdx.x;
  const __nv_bfloat16* rw = wbf + roff + (long long)m * FC * FC * 2;
  for (int e = threadIdx.x; e < FC * FC; e += 256)
    R[e] = make_float2(__bfloat162float(rw[2 * e]), __bfloat162float(rw[2 * e + 1]));
  for (int b0 = 0; b0 < B; b0 += 64) {
    const int nb = min(64, B - b0);
    __syncthreads();
    for (int e = threadIdx.x; e < nb * FC; e += 256) {
      const int b = e / FC, i = e % FC;
      Xm[e] = X[((long long)(b0 + b) * FC + i) * FMODES + m];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nb * FC; e += 256) {
      const int b = e / FC, o = e % FC;
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll 8
      for (int i = 0; i < FC; ++i) acc = c_add(acc, c_mul(R[i * FC + o], Xm[b * FC + i]));
      Y[((long long)(b0 + b) * FC + o) * FMODES + m] = acc;
    }
  }
}

// dX[b][i] = sum_o conj(R[i][o]) dY[b][o];  dR[m][i][o] += sum_b conj(X[b][i]) dY[b][o].
__global__ void __launch_bounds__(256) fno_mix_bwd(const float2* __restrict__ X, const float2* __restrict__ dY,
                                                   const __nv_bfloat16* __restrict__ wbf, long long roff, int B,
                                                   float2* __restrict__ dX, float* __restrict__ grad) {
  __shared__ float2 R[FC * FC];
  __shared__ float2 Xm[64 * FC];
  __shared__ float2 Gm[64 * FC];
  const int m = blockIdx.x;
  const __nv_bfloat16* rw = wbf + roff + (long long)m * FC * FC * 2;
  for (int e = threadIdx.x; e < FC * FC; e += 256)
    R[e] = make_float2(__bfloat162float(rw[2 * e]), __bfloat162float(rw[2 * e + 1]));
  float2 dr[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  for (int b0 = 0; b0 < B; b0 += 64) {
    const int nb = min(64, B - b0);
    __syncthreads();
    for (int e = threadIdx.x; e < nb * FC; e += 256) {
      const int b = e / FC, i = e % FC;
      Xm[e] = X[((long long)(b0 + b) * FC + i) * FMODES + m];
      Gm[e] = dY[((long long)(b0 + b) * FC + i) * FMODES + m];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nb * FC; e += 256) {
      const int b = e / FC, i = e % FC;
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll 8
      for (int o = 0; o < FC; ++o) acc = c_add(acc, c_cjmul(R[i * FC + o], Gm[b * FC + o]));
      dX[((long long)(b0 + b) * FC + i) * FMODES + m] = acc;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int e = threadIdx.x + 256 * k;
      const int i = e / FC, o = e % FC;
      for (int b = 0; b < nb; ++b) dr[k] = c_add(dr[k], c_cjmul(Xm[b * FC + i], Gm[b * FC + o]));
    }
  }
  float* g = grad + roff + (long long)m * FC * FC * 2;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int e = threadIdx.x + 256 * k;
    g[2 * e] += dr[k].x;
    g[2 * e + 1] += dr[k].y;
  }
}

// pre = s + W v_prev + b (pre holds s on entry), v_out = GELU(pre) or pre; one thread per pixel.
__global__ void __launch_bounds__(128) fno_pointwise_fwd(float* __restrict__ pre, const float* __restrict__ vprev,
                                                         const __nv_bfloat16* __restrict__ wbf, const float* __restrict__ pm,
                                                         long long woff, long long boff, int B, int act,
                                                         float* __restrict__ vout) {
  __shared__ float W[FC * FC], bb[FC];
  for (int i = threadIdx.x; i < FC * FC; i += blockDim.x) W[i] = __bfloat162float(wbf[woff + i]);
  for (int i = threadIdx.x; i < FC; i += blockDim.x) bb[i] = pm[boff + i];
  __syncthreads();
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)B * FNN) return;
  const long long b = idx / FNN, pix = idx % FNN;
  const float* vp = vprev + b * FC * FNN + pix;
  float vin[FC];
#pragma unroll
  for (int i = 0; i < FC; ++i) vin[i] = vp[(long long)i * FNN];
  float* pp = pre + b * FC * FNN + pix;
  float* vo = vout + b * FC * FNN + pix;
#pragma unroll 4
  for (int o = 0; o < FC; ++o) {
    float acc = pp[(long long)o * FNN] + bb[o];
#pragma unroll
    for (int i = 0; i < FC; ++i) acc += W[o * FC + i] * vin[i];
    pp[(long long)o * FNN] = acc;
    vo[(long long)o * FNN] = act ? gelu_f(acc) : acc;
  }
}

// dpre = dv * GELU'(pre) (or dv), dv_prev = W^T dpre; one thread per pixel.
__global__ void __launch_bounds__(128) fno_pointwise_bwd(const float* __restrict__ dv, const float* __restrict__ pre,
                                                         const __nv_bfloat16* __restrict__ wbf, long long woff, int B,
                                                         int act, float* __restrict__ dpre, float* __restrict__ dvprev) {
  __shared__ float W[FC * FC];
  for (int i = threadIdx.x; i < FC * FC; i += blockDim.x) W[i] = __bfloat162float(wbf[woff + i]);
  __syncthreads();
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)B * FNN) return;
  const long long b = idx / FNN, pix = idx % FNN;
  const long long base = b * FC * FNN + pix;
  float acc[FC];
#pragma unroll
  for (int i = 0; i < FC; ++i) acc[i] = 0.f;
#pragma unroll 2
  for (int o = 0; o < FC; ++o) {
    float d = dv[base + (long long)o * FNN];
    if (act) d *= gelu_grad_f(pre[base + (long long)o * FNN]);
    dpre[base + (long long)o * FNN] = d;
#pragma unroll
    for (int i = 0; i < FC; ++i) acc[i] += W[o * FC + i] * d;
  }
#pragma unroll
  for (int i = 0; i < FC; ++i) dvprev[base + (long long)i * FNN] = acc[i];
}

// z = P1 v + c1, h = GELU(z), out = P2 h + c2; one thread per pixel.
__global__ void __launch_bounds__(128) fno_proj_fwd(const float* __restrict__ vL, const __nv_bfloat16* __restrict__ wbf,
                                                    const float* __restrict__ pm, int B, float* __restrict__ z,
                                                    float* __restrict__ h, float2* __restrict__ out) {
  __shared__ float P1[FH * FC], P2[2 * FH], c1[FH];
  for (int i = threadIdx.x; i < FH * FC; i += blockDim.x) P1[i] = __bfloat162float(wbf[F_P1 + i]);
  for (int i = threadIdx.x; i < 2 * FH; i += blockDim.x) P2[i] = __bfloat162float(wbf[F_P2 + i]);
  for (int i = threadIdx.x; i < FH; i += blockDim.x) c1[i] = pm[F_C1 + i];
  __syncthreads();
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)B * FNN) return;
  const long long b = idx / FNN, pix = idx % FNN;
  float vin[FC];
#pragma unroll
  for (int i = 0; i < FC; ++i) vin[i] = vL[(b * FC + i) * FNN + pix];
  float o0 = pm[F_C2], o1 = pm[F_C2 + 1];
#pragma unroll 2
  for (int k = 0; k < FH; ++k) {
    float acc = c1[k];
#pragma unroll
    for (int i = 0; i < FC; ++i) acc += P1[k * FC + i] * vin[i];
    const float hv = gelu_f(acc);
    z[(b * FH + k) * FNN + pix] = acc;
    h[(b * FH + k) * FNN + pix] = hv;
    o0 += P2[k] * hv;
    o1 += P2[FH + k] * hv;
  }
  out[b * FNN + pix] = make_float2(o0, o1);
}

// Tensor-core projection: z = P1 v + c1 on mma.sync m16n8k16 (BF16 operands,
// FP32 accumulation), h = GELU(z), out = P2 h + c2.  A warp owns 16 pixels x
// 128 hidden units (16 n-tiles, K = 32 channels in two k-steps).  Activations
// are split into BF16 hi + lo parts (two MMAs), so the product keeps ~16
// mantissa bits of v; the BF16 weights are exact.  store != 0 keeps z and h
// for the backward pass.
__device__ __forceinline__ uint32_t pack_bf16(float lo_col, float hi_col) {
  const uint32_t a = __bfloat16_as_ushort(__float2bfloat16_rn(lo_col));
  const uint32_t b = __bfloat16_as_ushort(__float2bfloat16_rn(hi_col));
  return a | (b << 16);
}
__device__ __forceinline__ float bf16_residual(float x) { return x - __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int STORE>
__global__ void __launch_bounds__(128) fno_proj_fwd_tc(const float* __restrict__ vL,
                                                       const __nv_bfloat16* __restrict__ wbf,
                                                       const float* __restrict__ pm, int B, float* __restrict__ z,
                                                       float* __restrict__ h, float2* __restrict__ out) {
  __shared__ uint32_t P1w[FH * FC / 2];  // P1[n][k] as bf16 pairs along k
  __shared__ float P2s[2 * FH], c1s[FH];
  const uint32_t* p1g = reinterpret_cast<const uint32_t*>(wbf + F_P1);
  for (int i = threadIdx.x; i < FH * FC / 2; i += 128) P1w[i] = p1g[i];
  for (int i = threadIdx.x; i < 2 * FH; i += 128) P2s[i] = __bfloat162float(wbf[F_P2 + i]);
  for (int i = threadIdx.x; i < FH; i += 128) c1s[i] = pm[F_C1 + i];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const long long P0 = ((long long)blockIdx.x * 4 + warp) * 16;  // first pixel of this warp
  if (P0 >= (long long)B * FNN) return;
  const long long b = P0 / FNN;
  const int pix0 = (int)(P0 % FNN);  // 16 pixels never straddle samples (FNN % 16 == 0)
  const float* vb = vL + b * FC * FNN + pix0;
  // A fragments (hi and lo) for the two k-steps
  uint32_t ahi[2][4], alo[2][4];
#pragma unroll
  for (int ks = 0; ks < 2; ++ks) {
    const int k0 = ks * 16 + 2 * t;
    float x[8];
    x[0] = vb[(long long)(k0)*FNN + g];
    x[1] = vb[(long long)(k0 + 1) * FNN + g];
    x[2] = vb[(long long)(k0)*FNN + g + 8];
    x[3] = vb[(long long)(k0 + 1) * FNN + g + 8];
    x[4] = vb[(long long)(k0 + 8) * FNN + g];
    x[5] = vb[(long long)(k0 + 9) * FNN + g];
    x[6] = vb[(long long)(k0 + 8) * FNN + g + 8];
    x[7] = vb[(long long)(k0 + 9) * FNN + g + 8];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      ahi[ks][r] = pack_bf16(x[2 * r], x[2 * r + 1]);
      alo[ks][r] = pack_bf16(bf16_residual(x[2 * r]), bf16_residual(x[2 * r + 1]));
    }
  }
  float o0a = 0.f, o1a = 0.f, o0b = 0.f, o1b = 0.f;  // outputs of pixels g (a) and g + 8 (b)
#pragma unroll 4
  for (int j = 0; j < FH / 8; ++j) {
    float d[4] = {0.f, 0.f, 0.f, 0.f};
    const int n = 8 * j + g;
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      const uint32_t b0 = P1w[n * (FC / 2) + ks * 8 + t];      // k = ks*16 + 2t, 2t+1
      const uint32_t b1 = P1w[n * (FC / 2) + ks * 8 + 4 + t];  // k + 8
      mma_bf16_16816(d, ahi[ks], b0, b1);
      mma_bf16_16816(d, alo[ks], b0, b1);
    }
    // d[0], d[1]: pixel g, hidden 8j + 2t, +1 ; d[2], d[3]: pixel g + 8
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int hh = 8 * j + 2 * t + (e & 1);
      const int px = g + (e >> 1) * 8;
      const float zz = d[e] + c1s[hh];
      const float hv = gelu_f(zz);
      if (STORE) {
        z[(b * FH + hh) * FNN + pix0 + px] = zz;
        h[(b * FH + hh) * FNN + pix0 + px] = hv;
      }
      if (e < 2) {
        o0a += P2s[hh] * hv;
        o1a += P2s[FH + hh] * hv;
      } else {
        o0b += P2s[hh] * hv;
        o1b += P2s[FH + hh] * hv;
      }
    }
  }
  // sum over the four lanes (t) that share a pixel row g
#pragma unroll
  for (int m = 1; m < 4; m <<= 1) {
    o0a += __shfl_xor_sync(0xffffffffu, o0a, m);
    o1a += __shfl_xor_sync(0xffffffffu, o1a, m);
    o0b += __shfl_xor_sync(0xffffffffu, o0b, m);
    o1b += __shfl_xor_sync(0xffffffffu, o1b, m);
  }
  if (t == 0) {
    const float c20 = pm[F_C2], c21 = pm[F_C2 + 1];
    out[b * FNN + pix0 + g] = make_float2(o0a + c20, o1a + c21);
    out[b * FNN + pix0 + g + 8] = make_float2(o0b + c20, o1b + c21);
  }
}

// dz = (P2^T dout) * GELU'(z) (overwrites z), dv = P1^T dz; one thread per pixel.
__global__ void __launch_bounds__(128) fno_proj_bwd(const float* __restrict__ dout, float* __restrict__ z,
                                                    const __nv_bfloat16* __restrict__ wbf, int B,
                                                    float* __restrict__ dvL) {
  __shared__ float P1[FH * FC], P2[2 * FH];
  for (int i = threadIdx.x; i < FH * FC; i += blockDim.x) P1[i] = __bfloat162float(wbf[F_P1 + i]);
  for (int i = threadIdx.x; i < 2 * FH; i += blockDim.x) P2[i] = __bfloat162float(wbf[F_P2 + i]);
  __syncthreads();
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)B * FNN) return;
  const long long b = idx / FNN, pix = idx % FNN;
  const float d0 = dout[(b * 2) * FNN + pix], d1 = dout[(b * 2 + 1) * FNN + pix];
  float acc[FC];
#pragma unroll
  for (int i = 0; i < FC; ++i) acc[i] = 0.f;
#pragma unroll 2
  for (int k = 0; k < FH; ++k) {
    float* zp = z + (b * FH + k) * FNN + pix;
    const float dz = (P2[k] * d0 + P2[FH + k] * d1) * gelu_grad_f(*zp);
    *zp = dz;
#pragma unroll
    for (int i = 0; i < FC; ++i) acc[i] += P1[k * FC + i] * dz;
  }
#pragma unroll
  for (int i = 0; i < FC; ++i) dvL[(b * FC + i) * FNN + pix] = acc[i];
}

// Per-sample relative L2 loss and its gradient (planar [B][2][FNN]); one CTA per sample.
__global__ void __launch_bounds__(256) fno_loss(const float2* __restrict__ out, const float2* __restrict__ t, int B,
                                                float* __restrict__ dout, float* __restrict__ loss) {
  __shared__ float red[2][8];
  const long long b = blockIdx.x;
  float nd = 0.f, nt = 0.f;
  for (int p = threadIdx.x; p < FNN; p += 256) {
    const float2 o = out[b * FNN + p], tv = t[b * FNN + p];
    const float dx = o.x - tv.x, dy = o.y - tv.y;
    nd += dx * dx + dy * dy;
    nt += tv.x * tv.x + tv.y * tv.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    nd += __shfl_xor_sync(0xffffffffu, nd, o);
    nt += __shfl_xor_sync(0xffffffffu, nt, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = nd;
    red[1][threadIdx.x >> 5] = nt;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    float* r = red[threadIdx.x];
    for (int w = 4; w > 0; w >>= 1)
      for (int i = 0; i < w; ++i) r[i] += r[i + w];
  }
  __syncthreads();
  const float ndn = sqrtf(red[0][0]), ntn = sqrtf(red[1][0]);
  if (threadIdx.x == 0) loss[b] = ndn / ntn;
  const float sc = (ndn > 0.f && ntn > 0.f) ? 1.f / (ndn * ntn * B) : 0.f;
  if (!dout) return;
  for (int p = threadIdx.x; p < FNN; p += 256) {
    const float2 o = out[b * FNN + p], tv = t[b * FNN + p];
    dout[(b * 2) * FNN + p] = (o.x - tv.x) * sc;
    dout[(b * 2 + 1) * FNN + p] = (o.y - tv.y) * sc;
  }
}

// G[o][i] += sum_p X[b][o][p] Y[b][i][p] over all B * FNN pixels (and gb[o] += sum_p X[o][p]).
// Each CTA reduces a 1024-pixel chunk in shared tiles of 32 pixels, then adds atomically.
template <int O, int I>
__global__ void __launch_bounds__(256) fno_outer(const float* __restrict__ X, const float* __restrict__ Y, int B,
                                                 float* __restrict__ G, float* __restrict__ gb) {
  constexpr int TP = 32, CH = 1024;
  constexpr int PER = (O * I + 255) / 256;
  __shared__ float Xs[O][TP + 1];
  __shared__ float Ys[I][TP + 1];
  const long long p0 = (long long)blockIdx.x * CH;
  float acc[PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) acc[k] = 0.f;
  float bacc = 0.f;
  for (int t0 = 0; t0 < CH; t0 += TP) {
    __syncthreads();
    for (int e = threadIdx.x; e < (O + I) * TP; e += 256) {
      const int ch = e / TP, pp = e % TP;
      const long long p = p0 + t0 + pp;
      const long long b = p / FNN, pix = p % FNN;
      if (ch < O)
        Xs[ch][pp] = (b < B) ? X[(b * O + ch) * FNN + pix] : 0.f;
      else
        Ys[ch - O][pp] = (b < B) ? Y[(b * I + (ch - O)) * FNN + pix] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int e = threadIdx.x + 256 * k;
      if (e < O * I) {
        const int o = e / I, i = e % I;
        float s = 0.f;
#pragma unroll 8
        for (int pp = 0; pp < TP; ++pp) s += Xs[o][pp] * Ys[i][pp];
        acc[k] += s;
      }
    }
    if (gb && threadIdx.x < O) {
      float s = 0.f;
      for (int pp = 0; pp < TP; ++pp) s += Xs[threadIdx.x][pp];
      bacc += s;
    }
  }
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int e = threadIdx.x + 256 * k;
    if (e < O * I) atomicAdd(G + e, acc[k]);
  }
  if (gb && threadIdx.x < O) atomicAdd(gb + threadIdx.x, bacc);
}

__global__ void fno_to_bf16(const float* __restrict__ pm, __nv_bfloat16* __restrict__ wbf, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) wbf[i] = __float2bfloat16_rn(pm[i]);
}

__global__ void fno_round_bf16(const __nv_bfloat16* __restrict__ wbf, const float* __restrict__ pm,
                               float* __restrict__ out, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  // weights as the kernels read them (BF16), biases exact
  bool bias = (i >= F_B0 && i < F_LAYERS) || (i >= F_C1 && i < F_P2) || i >= F_C2;
  for (int l = 0; l < FL && !bias; ++l) bias = (i >= f_B(l) && i < f_B(l) + FC);
  out[i] = bias ? pm[i] : __bfloat162float(wbf[i]);
}

// Adam (Kingma and Ba 2015) on the FP32 master parameters, then the BF16 copy.
__global__ void fno_adam(float* __restrict__ pm, const float* __restrict__ g, float* __restrict__ m1,
                         float* __restrict__ m2, __nv_bfloat16* __restrict__ wbf, long long n, float lr, float b1,
                         float b2, float eps, float c1, float c2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float a = b1 * m1[i] + (1.f - b1) * gi;
  const float v = b2 * m2[i] + (1.f - b2) * gi * gi;
  m1[i] = a;
  m2[i] = v;
  const float p = pm[i] - lr * (a / c1) / (sqrtf(v / c2) + eps);
  pm[i] = p;
  wbf[i] = __float2bfloat16_rn(p);
}

// x0 = u_in + u_in e (e = demodulated scattered field)
__global__ void fno_add_incident(const float2* __restrict__ u_in, const float2* __restrict__ e,
                                 float2* __restrict__ x0, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x0[i] = c_add(u_in[i], c_mul(u_in[i], e[i]));
}

// Seeded initialisation (SplitMix64 per element): weights uniform in
// [-1, 1] x (1 / sqrt(fan_in)) (spectral weights x 1 / C), biases 0.
__device__ __forceinline__ float init_uniform(unsigned long long seed, long long i) {
  unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (float)((double)(z >> 11) * (1.0 / 9007199254740992.0)) * 2.f - 1.f;
}

__global__ void fno_init(float* __restrict__ pm, long long n, unsigned long long seed) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float scale = 0.f;
  if (i < F_B0) scale = 0.35355339f;  // 1/sqrt(8)
  else if (i >= F_P1 && i < F_C1) scale = 0.17677670f;  // 1/sqrt(32)
  else if (i >= F_P2 && i < F_C2) scale = 0.08838835f;  // 1/sqrt(128)
  else if (i >= F_LAYERS && i < F_P1) {
    const long long l = (i - F_LAYERS) / F_LAYER, off = (i - F_LAYERS) % F_LAYER;
    (void)l;
    if (off < (long long)FMODES * FC * FC * 2) scale = 1.f / FC;
    else if (off < (long long)FMODES * FC * FC * 2 + FC * FC) scale = 0.17677670f;
  }
  pm[i] = scale * init_uniform(seed, i);
}

}  // namespace cisor

using namespace cisor;

struct cisor_fno {
  int max_batch;
  cudaStream_t user_stream, stream;
  cudaEvent_t ev_a, ev_b;
  float *pm, *grad, *m1, *m2;
  __nv_bfloat16* wbf;
  float2* twst;
  long long adam_t;
  // activations [max_batch, ...]
  float *feat, *v[FL + 1], *pre[FL], *z, *h, *dout, *dvA, *dvB, *dpre, *loss;
  float2 *X[FL], *Y, *dY, *dX, *out, *fbuf, *ubuf, *tbuf, *usc;
  float* h_loss;
};

namespace {

cisor_status fno_enter(cisor_fno* F) {
  CISOR_CUDA(cudaEventRecord(F->ev_a, F->user_stream));
  CISOR_CUDA(cudaStreamWaitEvent(F->stream, F->ev_a, 0));
  return CISOR_OK;
}
cisor_status fno_leave(cisor_fno* F) {
  CISOR_CUDA(cudaEventRecord(F->ev_b, F->stream));
  CISOR_CUDA(cudaStreamWaitEvent(F->user_stream, F->ev_b, 0));
  return CISOR_OK;
}

unsigned grid_of(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// forward pass on F->fbuf / F->ubuf (f_per_sample as given), leaves F->out;
// store keeps the projection's z and h for a backward pass
cisor_status fno_forward_core(cisor_fno* F, int fps, int B, int store = 1) {
  cudaStream_t s = F->stream;
  const long long BP = (long long)B * FNN;
  fno_features_lift<<<grid_of(BP, 256), 256, 0, s>>>(F->fbuf, fps, F->ubuf, F->wbf, F->pm, B, F->feat, F->v[0]);
  CISOR_CUDA(cudaGetLastError());
  for (int l = 0; l < FL; ++l) {
    fno_analysis<<<B * FC, 256, 0, s>>>(F->v[l], F->X[l], F->twst, 1.f, 0);
    CISOR_CUDA(cudaGetLastError());
    fno_mix_fwd<<<FMODES, 256, 0, s>>>(F->X[l], F->wbf, f_R(l), B, F->Y);
    CISOR_CUDA(cudaGetLastError());
    fno_synthesis<<<B * FC, 256, 0, s>>>(F->Y, F->pre[l], F->twst, 1.f / FNN, 1, 0);
    CISOR_CUDA(cudaGetLastError());
    fno_pointwise_fwd<<<grid_of(BP, 128), 128, 0, s>>>(F->pre[l], F->v[l], F->wbf, F->pm, f_W(l), f_B(l), B,
                                                       l < FL - 1, F->v[l + 1]);
    CISOR_CUDA(cudaGetLastError());
  }
  if (store)
    fno_proj_fwd_tc<1><<<grid_of(BP, 64), 128, 0, s>>>(F->v[FL], F->wbf, F->pm, B, F->z, F->h, F->out);
  else
    fno_proj_fwd_tc<0><<<grid_of(BP, 64), 128, 0, s>>>(F->v[FL], F->wbf, F->pm, B, F->z, F->h, F->out);
  CISOR_CUDA(cudaGetLastError());
  return CISOR_OK;
}

// loss and gradients (into F->grad) for targets in F->tbuf
cisor_status fno_backward_core(cisor_fno* F, int B) {
  cudaStream_t s = F->stream;
  const long long BP = (long long)B * FNN;
  const unsigned gch = grid_of(BP, 1024);
  CISOR_CUDA(cudaMemsetAsync(F->grad, 0, sizeof(float) * F_TOTAL, s));
  fno_loss<<<B, 256, 0, s>>>(F->out, F->tbuf, B, F->dout, F->loss);
  CISOR_CUDA(cudaGetLastError());
  fno_outer<2, FH><<<gch, 256, 0, s>>>(F->dout, F->h, B, F->grad + F_P2, F->grad + F_C2);
  CISOR_CUDA(cudaGetLastError());
  fno_proj_bwd<<<grid_of(BP, 128), 128, 0, s>>>(F->dout, F->z, F->wbf, B, F->dvA);
  CISOR_CUDA(cudaGetLastError());
  fno_outer<FH, FC><<<gch, 256, 0, s>>>(F->z, F->v[FL], B, F->grad + F_P1, F->grad + F_C1);
  CISOR_CUDA(cudaGetLastError());
  float* dv = F->dvA;
  float* dvn = F->dvB;
  for (int l = FL - 1; l >= 0; --l) {
    fno_pointwise_bwd<<<grid_of(BP, 128), 128, 0, s>>>(dv, F->pre[l], F->wbf, f_W(l), B, l < FL - 1, F->dpre, dvn);
    CISOR_CUDA(cudaGetLastError());
    fno_outer<FC, FC><<<gch, 256, 0, s>>>(F->dpre, F->v[l], B, F->grad + f_W(l), F->grad + f_B(l));
    CISOR_CUDA(cudaGetLastError());
    fno_analysis<<<B * FC, 256, 0, s>>>(F->dpre, F->dY, F->twst, 1.f / FNN, 1);
    CISOR_CUDA(cudaGetLastError());
    fno_mix_bwd<<<FMODES, 256, 0, s>>>(F->X[l], F->dY, F->wbf, f_R(l), B, F->dX, F->grad);
    CISOR_CUDA(cudaGetLastError());
    fno_synthesis<<<B * FC, 256, 0, s>>>(F->dX, dvn, F->twst, 1.f, 0, 1);
    CISOR_CUDA(cudaGetLastError());
    float* t = dv;
    dv = dvn;
    dvn = t;
  }
  fno_outer<FC, FIN><<<gch, 256, 0, s>>>(dv, F->feat, B, F->grad + F_W0, F->grad + F_B0);
  CISOR_CUDA(cudaGetLastError());
  return CISOR_OK;
}

cisor_status stage_inputs(cisor_fno* F, const void* f, int fps, const void* u_in, const void* target, int B) {
  const size_t vb = sizeof(float2) * (size_t)B * FNN;
  CISOR_CUDA(cudaMemcpyAsync(F->fbuf, f, fps ? vb : sizeof(float2) * FNN, cudaMemcpyDefault, F->stream));
  CISOR_CUDA(cudaMemcpyAsync(F->ubuf, u_in, vb, cudaMemcpyDefault, F->stream));
  if (target) CISOR_CUDA(cudaMemcpyAsync(F->tbuf, target, vb, cudaMemcpyDefault, F->stream));
  return CISOR_OK;
}

bool bad_batch(cisor_fno* F, int B) {
  if (B < 1 || B > F->max_batch) {
    set_error("FNO batch %d outside [1, %d]", B, F->max_batch);
    return true;
  }
  return false;
}

cisor_status mean_loss(cisor_fno* F, int B, double* loss) {
  CISOR_CUDA(cudaMemcpyAsync(F->h_loss, F->loss, sizeof(float) * B, cudaMemcpyDeviceToHost, F->stream));
  CISOR_CUDA(cudaStreamSynchronize(F->stream));
  double s = 0.0;
  for (int b = 0; b < B; ++b) s += F->h_loss[b];
  if (loss) *loss = s / B;
  return CISOR_OK;
}

void fno_free(cisor_fno* F) {
  if (!F) return;
  if (F->stream) cudaStreamSynchronize(F->stream);
  void* d[] = {F->pm, F->grad, F->m1, F->m2, F->wbf, F->twst, F->feat, F->z, F->h, F->dout, F->dvA, F->dvB,
               F->dpre, F->loss, F->Y, F->dY, F->dX, F->out, F->fbuf, F->ubuf, F->tbuf, F->usc};
  for (void* p : d)
    if (p) cudaFree(p);
  for (int l = 0; l <= FL; ++l)
    if (F->v[l]) cudaFree(F->v[l]);
  for (int l = 0; l < FL; ++l) {
    if (F->pre[l]) cudaFree(F->pre[l]);
    if (F->X[l]) cudaFree(F->X[l]);
  }
  if (F->h_loss) cudaFreeHost(F->h_loss);
  if (F->ev_a) cudaEventDestroy(F->ev_a);
  if (F->ev_b) cudaEventDestroy(F->ev_b);
  if (F->stream) cudaStreamDestroy(F->stream);
  delete F;
}

}  // namespace

extern "C" {

cisor_status cisor_fno_create(cisor_fno** out, int max_batch, unsigned long long seed, void* stream) {
  if (!out || max_batch < 1 || max_batch > 256) {
    set_error("cisor_fno_create: NULL argument or max_batch outside [1, 256]");
    return CISOR_ERR_INVALID_ARG;
  }
  *out = nullptr;
  cisor_fno* F = new (std::nothrow) cisor_fno();
  if (!F) {
    set_error("out of host memory");
    return CISOR_ERR_OOM;
  }
  F->max_batch = max_batch;
  F->user_stream = (cudaStream_t)stream;
  auto fail = [&](cudaError_t e, const char* what) {
    cisor_status st = cuda_fail(e, what, __FILE__, __LINE__);
    fno_free(F);
    return st;
  };
  cudaError_t e = cudaStreamCreateWithFlags(&F->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&F->ev_a, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&F->ev_b, cudaEventDisableTiming);
  if (e != cudaSuccess) return fail(e, "FNO stream/events");
  const size_t act = sizeof(float) * (size_t)max_batch * FC * FNN;
  const size_t hid = sizeof(float) * (size_t)max_batch * FH * FNN;
  const size_t md = sizeof(float2) * (size_t)max_batch * FC * FMODES;
  const size_t fld = sizeof(float2) * (size_t)max_batch * FNN;
  struct A {
    void** p;
    size_t n;
  } allocs[] = {{(void**)&F->pm, sizeof(float) * F_TOTAL}, {(void**)&F->grad, sizeof(float) * F_TOTAL},
                {(void**)&F->m1, sizeof(float) * F_TOTAL},  {(void**)&F->m2, sizeof(float) * F_TOTAL},
                {(void**)&F->wbf, sizeof(__nv_bfloat16) * F_TOTAL}, {(void**)&F->twst, sizeof(float2) * 2 * TW_STRIDE},
                {(void**)&F->feat, sizeof(float) * (size_t)max_batch * FIN * FNN}, {(void**)&F->z, hid},
                {(void**)&F->h, hid}, {(void**)&F->dout, sizeof(float) * (size_t)max_batch * 2 * FNN},
                {(void**)&F->dvA, act}, {(void**)&F->dvB, act}, {(void**)&F->dpre, act},
                {(void**)&F->loss, sizeof(float) * max_batch}, {(void**)&F->Y, md}, {(void**)&F->dY, md},
                {(void**)&F->dX, md}, {(void**)&F->out, fld}, {(void**)&F->fbuf, fld}, {(void**)&F->ubuf, fld},
                {(void**)&F->tbuf, fld}, {(void**)&F->usc, fld}};
  for (auto& a : allocs) {
    e = cudaMalloc(a.p, a.n);
    if (e != cudaSuccess) return fail(e, "FNO cudaMalloc");
  }
  for (int l = 0; l <= FL && e == cudaSuccess; ++l) e = cudaMalloc((void**)&F->v[l], act);
  for (int l = 0; l < FL && e == cudaSuccess; ++l) {
    e = cudaMalloc((void**)&F->pre[l], act);
    if (e == cudaSuccess) e = cudaMalloc((void**)&F->X[l], md);
  }
  if (e == cudaSuccess) e = cudaMallocHost((void**)&F->h_loss, sizeof(float) * max_batch);
  if (e != cudaSuccess) return fail(e, "FNO cudaMalloc");
  fno_init<<<grid_of(F_TOTAL, 256), 256, 0, F->stream>>>(F->pm, F_TOTAL, seed);
  fno_to_bf16<<<grid_of(F_TOTAL, 256), 256, 0, F->stream>>>(F->pm, F->wbf, F_TOTAL);
  e = cudaMemsetAsync(F->m1, 0, sizeof(float) * F_TOTAL, F->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(F->m2, 0, sizeof(float) * F_TOTAL, F->stream);
  if (e != cudaSuccess) return fail(e, "FNO init");
  cisor_ctx tw{};
  tw.P = FN;
  tw.twst = F->twst;
  tw.stream = F->stream;
  cisor_status st = make_stage_twiddles(&tw);
  if (st != CISOR_OK) {
    fno_free(F);
    return st;
  }
  e = cudaStreamSynchronize(F->stream);
  if (e != cudaSuccess) return fail(e, "FNO init sync");
  *out = F;
  return CISOR_OK;
}

cisor_status cisor_fno_destroy(cisor_fno* F) {
  fno_free(F);
  return CISOR_OK;
}

cisor_status cisor_fno_num_params(const cisor_fno* F, long long* count) {
  if (!F || !count) {
    set_error("cisor_fno_num_params: NULL argument");
    return CISOR_ERR_INVALID_ARG;
  }
  *count = F_TOTAL;
  return CISOR_OK;
}

cisor_status cisor_fno_get_params(cisor_fno* F, float* out, int as_used) {
  if (!F || !out) {
    set_error("cisor_fno_get_params: NULL argument");
    return CISOR_ERR_INVALID_ARG;
  }
  CISOR_TRY(fno_enter(F));
  if (as_used) {
    fno_round_bf16<<<grid_of(F_TOTAL, 256), 256, 0, F->stream>>>(F->wbf, F->pm, F->grad, F_TOTAL);
    CISOR_CUDA(cudaGetLastError());
    CISOR_CUDA(cudaMemcpyAsync(out, F->grad, sizeof(float) * F_TOTAL, cudaMemcpyDefault, F->stream));
  } else {
    CISOR_CUDA(cudaMemcpyAsync(out, F->pm, sizeof(float) * F_TOTAL, cudaMemcpyDefault, F->stream));
  }
  CISOR_CUDA(cudaStreamSynchronize(F->stream));
  return fno_leave(F);
}

cisor_status cisor_fno_set_params(cisor_fno* F, const float* in) {
  if (!F || !in) {
    set_error("cisor_fno_set_params: NULL argument");
    return CISOR_ERR_INVALID_ARG;
  }
  CISOR_TRY(fno_enter(F));
  CISOR_CUDA(cudaMemcpyAsync(F->pm, in, sizeof(float) * F_TOTAL, cudaMemcpyDefault, F->stream));
  fno_to_bf16<<<grid_of(F_TOTAL, 256), 256, 0, F->stream>>>(F->pm, F->wbf, F_TOTAL);
  CISOR_CUDA(cudaGetLastError());
  CISOR_CUDA(cudaMemsetAsync(F->m1, 0, sizeof(float) * F_TOTAL, F->stream));
  CISOR_CUDA(cudaMemsetAsync(F->m2, 0, sizeof(float) * F_TOTAL, F->stream));
  F->adam_t = 0;
  CISOR_CUDA(cudaStreamSynchronize(F->stream));
  return fno_leave(F);
}

cisor_status cisor_fno_forward(cisor_fno* F, const void* f, int f_per_sample, const void* u_in, int B, void* u_sc_out) {
  if (!F || !f || !u_in || !u_sc_out) {
    set_error("cisor_fno_forward: NULL argument");
    return CISOR_ERR_INVALID_ARG;
  }
  if (bad_batch(F, B)) return CISOR_ERR_INVALID_ARG;
  CISOR_TRY(fno_enter(F));
  CISOR_TRY(stage_inputs(F, f, f_per_sample, u_in, nullptr, B));
  CISOR_TRY(fno_forward_core(F, f_per_sample, B, 0));
  CISOR_CUDA(cudaMemcpyAsync(u_sc_out, F->out, sizeof(float2) * (size_t)B * FNN, cudaMemcpyDefault, F->stream));
  CISOR_CUDA(cudaStreamSynchronize(F->stream));
  return fno_leave(F);
}

cisor_status cisor_fno_loss_grad(cisor_fno* F, const void* f, int f_per_sample, const void* u_in, const void* target,
                                 int B, double* loss, float* grad_out) {
  if (!F || !f || !u_in || !target) {
    set_error("cisor_fno_loss_grad: NULL argument");
    return CISOR_ERR_INVALID_ARG;
  }
  if (bad_batch(F, B)) return CISOR_ERR_INVALID_ARG;
  CISOR_TRY(fno_enter(F));
  CISOR_TRY(stage_inputs(F, f, f_per_sample, u_in, target, B));
  CISOR_TRY(fno_forward_core(F, f_per_sample, B));
  CISOR_TRY(fno_backward_core(F, B));
  if (grad_out)
    CISOR_CUDA(cudaMemcpyAsync(grad_out, F->grad, sizeof(float) * F_TOTAL, cudaMemcpyDefault, F->stream));
  CISOR_TRY(mean_loss(F, B, loss));
  return fno_leave(F);
}

cisor_status cisor_fno_train_step(cisor_fno* F, const void* f, int f_per_sample, const void* u_in, const void* target,
                                  int B, double lr, double* loss) {
  if (!F || !f || !u_in || !target || !(lr > 0.0)) {
    set_error("cisor_fno_train_step: NULL argument or lr <= 0");
    return CISOR_ERR_INVALID_ARG;
  }
  if (bad_batch(F, B)) return CISOR_ERR_INVALID_ARG;
  CISOR_TRY(fno_enter(F));
  CISOR_TRY(stage_inputs(F, f, f_per_sample, u_in, target, B));
  CISOR_TRY(fno_forward_core(F, f_per_sample, B));
  CISOR_TRY(fno_backward_core(F, B));
  F->adam_t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)F->adam_t), c2 = 1.f - powf(b2, (float)F->adam_t);
  fno_adam<<<grid_of(F_TOTAL, 256), 256, 0, F->stream>>>(F->pm, F->grad, F->m1, F->m2, F->wbf, F_TOTAL, (float)lr, b1,
                                                         b2, 1e-8f, c1, c2);
  CISOR_CUDA(cudaGetLastError());
  CISOR_TRY(mean_loss(F, B, loss));
  return fno_leave(F);
}

cisor_status cisor_fno_warm_start(cisor_fno* F, cisor_ctx* c, const void* f, void* x0_out) {
  if (!F || !c || !f || !x0_out) {
    set_error("cisor_fno_warm_start: NULL argument");
    return CISOR_ERR_INVALID_ARG;
  }
  if (c->dim != 2 || c->n != FN || c->T > F->max_batch) {
    set_error("cisor_fno_warm_start: the network is for 128 x 128 grids and at most %d transmitters", F->max_batch);
    return CISOR_ERR_INVALID_ARG;
  }
  const int B = c->T;
  CISOR_TRY(fno_enter(F));
  CISOR_CUDA(cudaMemcpyAsync(F->fbuf, f, sizeof(float2) * FNN, cudaMemcpyDefault, F->stream));
  CISOR_CUDA(cudaMemcpyAsync(F->ubuf, c->u_in, sizeof(float2) * (size_t)B * FNN, cudaMemcpyDeviceToDevice, F->stream));
  CISOR_TRY(fno_forward_core(F, 0, B, 0));
  fno_add_incident<<<grid_of((long long)B * FNN, 256), 256, 0, F->stream>>>(F->ubuf, F->out, F->usc, (long long)B * FNN);
  CISOR_CUDA(cudaGetLastError());
  CISOR_CUDA(cudaMemcpyAsync(x0_out, F->usc, sizeof(float2) * (size_t)B * FNN, cudaMemcpyDefault, F->stream));
  CISOR_CUDA(cudaStreamSynchronize(F->stream));
  return fno_leave(F);
}

}  // extern "C"
