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
//   v_{l+1} = GELU(Lsyn(R_l . S(v_l)) + W_l v_l + b_l)   (no GELU on the last)
//   out = P2 GELU(P1 v_4 + c1) + c2,  e = out_0 + j out_1, predicted u - u_in = u_in e
// S keeps kx in {0..15, 112..127} (rows) x ky in {0..15} (columns) of the 2D
// DFT; Lsyn is (1/128^2) Re of the truncated inverse with weight 2 on ky > 0.
// Loss: mean over samples of ||out - t|| / ||t||.
//
// Every contraction of the network runs on the tensor cores with BF16
// operands and FP32 accumulation: the truncated DFTs are small dense GEMMs
// against FP64-built cosine/sine tables (16 of 128 frequencies per axis, so a
// GEMM reads each value once where a full FFT would transform 8x more), the
// 1x1 channel mixings, the projection, and the weight gradients (reductions
// over pixels or samples).  Weights are BF16 (the model is defined by their
// BF16 values; FP32 master copies and Adam state), so a weight operand is
// exact; activations and tables are split into BF16 hi + lo parts and a
// product takes two or three MMAs (about 16 mantissa bits, the accuracy of
// FP32 arithmetic for these sums).  The forward row kernels and the column
// DFTs (forward and backward) issue fifth-generation tensor-core tiles
// (tcgen05, accumulators in tensor memory); the lifting and the backward row
// and projection kernels use warp-level mma.sync tiles.  Only the per-mode
// 32 x 32 complex mixing (a matrix per mode applied to every sample's vector)
// and grad R run on the FP32 pipes.
//
// A layer is four kernels:
//   row kernel     (one sample, 2 image rows, all 32 channels): inverse row
//                  DFT of the mode-mixed spectrum + W v + b, GELU, and the
//                  forward row DFT of the result for the next layer (or the
//                  projection after the last layer);
//   column DFT     (one sample, 4 ky): the 32 kept kx of every channel;
//   mode mixing    (one mode, all samples): Y = R_l X;
//   inverse column DFT (one sample, 4 ky): back to the 128 rows.
// Between the row and column kernels the spectra travel as [B][64 row pairs]
// [16 ky][32 ch][2 rows] complex64 blocks (a row kernel reads and writes one
// contiguous 8 KB block), between the column kernels as [mode][B][32 ch].
// The backward pass mirrors
// this (row-backward, column DFT of dT, the mixing's transpose with grad R,
// inverse column DFT), recomputing the projection's hidden layer and the
// input features instead of storing them.
#include <math.h>
#include <cuda_bf16.h>

#include <new>

#include "common.cuh"
#include "gelu.cuh"
#include "tc5.cuh"

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

constexpr int RB = 2;              // image rows per row-kernel item
constexpr int NP = RB * FN;        // pixels per item
constexpr int NIB = FN / RB;       // row blocks per image
constexpr int BLK = FM * FC * RB;  // complex values of one spectral row block [ky][c][r]
constexpr int NTH = 256;           // threads of every FNO kernel
constexpr int NPP = NP + 4;        // shared-memory pitch (floats) of one channel's NP pixels
constexpr int PART_W = FC * FC + FC;                 // dW_l, db_l
constexpr int PART_P = FH * FC + FH + 2 * FH + 2;    // dP1, dc1, dP2, dc2
constexpr int PART_0 = FC * FIN + FC;                // dW0, db0
constexpr int PART_MAX = PART_P;

// DFT tables, FP64-built, as BF16 hi / lo pairs.  E(ix, kyc) = cos(2 pi ky ix / 128) (kyc = 2 ky),
// -sin (kyc = 2 ky + 1); F(kx, iy) = exp(-2 pi j kx' iy / 128), kx' = kx for kx < 16, kx + 96 otherwise.
// mma.sync tables (lifting and backward row kernels), laid out so that every fragment register is ONE
// 32-bit load (the two BF16 values of a register are adjacent along the contraction index) and, from
// shared memory, conflict-free:
//   RowF  B operand [kyc][ix], pitch RFP
//   RowI  B operand [ix][kyc], pitch RIP (the same values, transposed)
constexpr int RFP = FN + 8, RIP = 2 * FM + 8;
constexpr int T_RF = 2 * FM * RFP, T_RI = FN * RIP;
constexpr int T_ROW = 2 * (T_RF + T_RI);  // bf16 of the row tables (hi and lo), copied to shared memory
// tcgen05 tables in the tensor cores' core-matrix layout (tc5.cuh), each as a hi and a lo plane:
//   RowI  A operand E^T [128 ix][32 kyc]                (LBO 128, SBO 512)
//   RowF  B operand E [32 kyc][128 ix]                  (LBO 128, SBO 2048)
//   ColF  B operand [64 j][256 k], k = 2 iy + p (p: Re / Im of the input), j < 32: Re X(kx = j),
//         j >= 32: Im X(kx = j - 32); entries Fr, -Fi / Fi, Fr      (LBO 128, SBO 4096)
//   ColI  B operand [256 j][64 k], j = 2 iy + p (Re / Im of the output), k = 2 kx + p' (Re / Im of the
//         input): conj(F) as [[Fr, Fi], [-Fi, Fr]] per (iy, kx)    (LBO 128, SBO 1024)
constexpr int T_TCP = FN * 2 * FM;     // BF16 per plane of the row tables
constexpr int T_TCF = 2 * FKX * 2 * FN;  // BF16 per plane of the column tables
constexpr int T_TROW = T_ROW;                  // RowI A hi, lo, RowF B hi, lo
constexpr int T_TCOLF = T_TROW + 4 * T_TCP;    // ColF B hi, lo
constexpr int T_TCOLI = T_TCOLF + 2 * T_TCF;   // ColI B hi, lo
constexpr int T_ALL = T_TCOLI + 2 * T_TCF;
constexpr int WP = FC + 8;                        // pitch (bf16) of a 32-wide weight row in shared memory
constexpr int P1TP = FH + 8;                      // pitch (bf16) of P1^T rows


// ------------------------------------------------------------------ tensor-core tiles
// m16n8k16 fragments (PTX ISA, mma.sync .bf16): lane = 4 g + t;
//   A (16 x 16): a0 a1 (row g, k 2t, 2t+1), a2 a3 (row g + 8), a4 a5 (row g, k 2t + 8, +9), a6 a7 (row g + 8)
//   B (16 x 8):  b0 b1 (k 2t, 2t+1; col g), b2 b3 (k 2t + 8, +9; col g)
//   D (16 x 8):  d0 d1 (row g, col 2t, 2t+1), d2 d3 (row g + 8)
__device__ __forceinline__ uint32_t bf_bits(__nv_bfloat16 h) { return (uint32_t)__bfloat16_as_ushort(h); }
__device__ __forceinline__ void split_pair(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);  // one packed conversion, x0 in the low half
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}
struct FragA {
  uint32_t h[4], l[4];
};
struct FragB {
  uint32_t h[2], l[2];
};
// A fragment of FP32 values A(m, k), split into BF16 hi + lo
template <class F>
__device__ __forceinline__ FragA load_a(F A, int m0, int k0, int g, int t) {
  FragA f;
  split_pair(A(m0 + g, k0 + 2 * t), A(m0 + g, k0 + 2 * t + 1), f.h[0], f.l[0]);
  split_pair(A(m0 + g + 8, k0 + 2 * t), A(m0 + g + 8, k0 + 2 * t + 1), f.h[1], f.l[1]);
  split_pair(A(m0 + g, k0 + 2 * t + 8), A(m0 + g, k0 + 2 * t + 9), f.h[2], f.l[2]);
  split_pair(A(m0 + g + 8, k0 + 2 * t + 8), A(m0 + g + 8, k0 + 2 * t + 9), f.h[3], f.l[3]);
  return f;
}
// B fragment of FP32 values B(k, n), split into BF16 hi + lo
template <class F>
__device__ __forceinline__ FragB load_b(F B, int k0, int n0, int g, int t) {
  FragB f;
  split_pair(B(k0 + 2 * t, n0 + g), B(k0 + 2 * t + 1, n0 + g), f.h[0], f.l[0]);
  split_pair(B(k0 + 2 * t + 8, n0 + g), B(k0 + 2 * t + 9, n0 + g), f.h[1], f.l[1]);
  return f;
}
// B fragment from a BF16 matrix stored [n][k] (k pairs adjacent), pitch pw 32-bit words
__device__ __forceinline__ void load_b_tab(const uint32_t* tab, int pw, int k0, int n0, int g, int t,
                                           uint32_t (&b)[2]) {
  const uint32_t* row = tab + (n0 + g) * pw + (k0 >> 1) + t;
  b[0] = row[0];
  b[1] = row[4];
}
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// d += A B with both operands split (three products; lo x lo is below FP32 rounding)
__device__ __forceinline__ void mma3(float (&d)[4], const FragA& a, const FragB& b) {
  mma16816(d, a.h, b.h);
  mma16816(d, a.l, b.h);
  mma16816(d, a.h, b.l);
}
__device__ __forceinline__ void mma3t(float (&d)[4], const FragA& a, const uint32_t (&bh)[2], const uint32_t (&bl)[2]) {
  mma16816(d, a.h, bh);
  mma16816(d, a.l, bh);
  mma16816(d, a.h, bl);
}
// d += A B with an exact BF16 B (weights)
__device__ __forceinline__ void mma2(float (&d)[4], const FragA& a, const uint32_t (&b)[2]) {
  mma16816(d, a.h, b);
  mma16816(d, a.l, b);
}

__device__ __forceinline__ void cp16(void* dst, const void* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}
// bytes (multiple of 16, both 16-byte aligned) from global to shared by the whole CTA
__device__ __forceinline__ void cta_copy(void* dst, const void* src, int bytes) {
  for (int i = threadIdx.x * 16; i < bytes; i += NTH * 16) cp16((char*)dst + i, (const char*)src + i);
}
// a [FC][NP] block of sample b's planar [B][FC][FNN] field (pixels pix0 ..) into shared memory, pitch NPP
__device__ __forceinline__ void load_planar(float* dst, const float* src, int b, long long pix0) {
  for (int i = threadIdx.x; i < FC * NP / 4; i += NTH) {
    const int c = i / (NP / 4), q = i % (NP / 4);
    cp16(dst + c * NPP + 4 * q, src + ((long long)b * FC + c) * FNN + pix0 + 4 * q);
  }
}
// a 32 x 32 BF16 weight matrix W[o][i] into shared memory, as Ws[o][i] (pitch WP) and / or Wt[i][o]
__device__ __forceinline__ void load_w(const __nv_bfloat16* __restrict__ w, __nv_bfloat16* ws, __nv_bfloat16* wt) {
  for (int e = threadIdx.x; e < FC * FC; e += NTH) {
    const int o = e / FC, i = e % FC;
    const __nv_bfloat16 v = w[e];
    if (ws) ws[o * WP + i] = v;
    if (wt) wt[i * WP + o] = v;
  }
}

// ------------------------------------------------------------------ shared phases of the row kernels
__device__ __forceinline__ const uint32_t* tab_rf(const __nv_bfloat16* tb, int lo) {
  return reinterpret_cast<const uint32_t*>(tb + lo * T_RF);
}
__device__ __forceinline__ const uint32_t* tab_ri(const __nv_bfloat16* tb, int lo) {
  return reinterpret_cast<const uint32_t*>(tb + 2 * T_RF + lo * T_RI);
}

// S(rr, ix) = Re sum_ky Z[ky][c][r] exp(+2 pi j ky ix / 128), rr = 32 r + c: GEMM
// M = 64 (rr), N = 128 (ix), K = 32 (Re / Im of the 16 ky).  Adds into
// dst[c * NPP + r * FN + ix] (accumulate) or stores there.
__device__ __forceinline__ void row_inverse(const float2* zs, const __nv_bfloat16* tb, float* dst, bool accumulate) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  const float* zf = reinterpret_cast<const float*>(zs);
  auto A = [&](int rr, int k) { return zf[(((k >> 1) * FC + (rr & 31)) * RB + (rr >> 5)) * 2 + (k & 1)]; };
  const uint32_t *th = tab_ri(tb, 0), *tl = tab_ri(tb, 1);
  const int mt = warp & 3, nt0 = (warp >> 2) * 8;
  float d[8][4];
#pragma unroll
  for (int j = 0; j < 8; ++j) d[j][0] = d[j][1] = d[j][2] = d[j][3] = 0.f;
#pragma unroll
  for (int ks = 0; ks < 2; ++ks) {
    const FragA a = load_a(A, 16 * mt, 16 * ks, g, t);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      uint32_t bh[2], bl[2];
      load_b_tab(th, RIP / 2, 16 * ks, 8 * (nt0 + j), g, t, bh);
      load_b_tab(tl, RIP / 2, 16 * ks, 8 * (nt0 + j), g, t, bl);
      mma3t(d[j], a, bh, bl);
    }
  }
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int rr = 16 * mt + g + (e >> 1) * 8, ix = 8 * (nt0 + j) + 2 * t + (e & 1);
      float* p = dst + (rr & 31) * NPP + (rr >> 5) * FN + ix;
      *p = accumulate ? *p + d[j][e] : d[j][e];
    }
}

// T[ky][c][r] = sum_ix src[c * NPP + r * FN + ix] exp(-2 pi j ky ix / 128): GEMM
// M = 64 (rr), N = 32 (Re / Im of 16 ky), K = 128 (ix); result in stage [BLK].
__device__ __forceinline__ void row_forward(const float* src, const __nv_bfloat16* tb, float2* stage) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  auto A = [&](int rr, int ix) { return src[(rr & 31) * NPP + (rr >> 5) * FN + ix]; };
  const uint32_t *th = tab_rf(tb, 0), *tl = tab_rf(tb, 1);
  const int mt = warp & 3, nt0 = (warp >> 2) * 2;
  float d[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll 2
  for (int ks = 0; ks < FN / 16; ++ks) {
    const FragA a = load_a(A, 16 * mt, 16 * ks, g, t);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      uint32_t bh[2], bl[2];
      load_b_tab(th, RFP / 2, 16 * ks, 8 * (nt0 + j), g, t, bh);
      load_b_tab(tl, RFP / 2, 16 * ks, 8 * (nt0 + j), g, t, bl);
      mma3t(d[j], a, bh, bl);
    }
  }
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int rr = 16 * mt + g + 8 * h, ky = 4 * (nt0 + j) + t;
      stage[(ky * FC + (rr & 31)) * RB + (rr >> 5)] = make_float2(d[j][2 * h], d[j][2 * h + 1]);
    }
}

// out[p][o] (+)= sum_i A(p, i) W[o][i] over the NP pixels (M = NP, N = FC, K = FC), W exact BF16 in
// ws ([o][i], pitch WP); epi(p, o, value) consumes each result once.
template <class FA, class Epi>
__device__ __forceinline__ void pixel_mix(FA A, const __nv_bfloat16* ws, Epi epi) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  const uint32_t* w32 = reinterpret_cast<const uint32_t*>(ws);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int mt = 2 * warp + h;
    const FragA a0 = load_a(A, 16 * mt, 0, g, t), a1 = load_a(A, 16 * mt, 16, g, t);
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      uint32_t b0[2], b1[2];
      load_b_tab(w32, WP / 2, 0, 8 * nt, g, t, b0);
      load_b_tab(w32, WP / 2, 16, 8 * nt, g, t, b1);
      float d[4] = {0.f, 0.f, 0.f, 0.f};
      mma2(d, a0, b0);
      mma2(d, a1, b1);
#pragma unroll
      for (int e = 0; e < 4; ++e) epi(16 * mt + g + (e >> 1) * 8, 8 * nt + 2 * t + (e & 1), d[e]);
    }
  }
}

// the 8 input features of the NP pixels of rows iy0, iy0 + 1 into as[k * NPP + p]
// (us: rows iy0 - 1 .. iy0 + RB clamped, fs: rows iy0 .. iy0 + RB - 1)
__device__ __forceinline__ void features(const float2* us, const float2* fs, int iy0, float* as) {
  for (int p = threadIdx.x; p < NP; p += NTH) {
    const int r = p / FN, ix = p % FN;
    const float2 u = us[(r + 1) * FN + ix];
    const float2 gx = c_scale(c_sub(us[(r + 1) * FN + min(ix + 1, FN - 1)], us[(r + 1) * FN + max(ix - 1, 0)]), 0.5f);
    const float2 gy = c_scale(c_sub(us[(r + 2) * FN + ix], us[r * FN + ix]), 0.5f);
    const float vx = c_cjmul(u, gx).y, vy = c_cjmul(u, gy).y;
    const float nv = sqrtf(vx * vx + vy * vy);
    const float2 fv = fs[p];
    as[0 * NPP + p] = fv.x;
    as[1 * NPP + p] = fv.y;
    as[2 * NPP + p] = u.x;
    as[3 * NPP + p] = u.y;
    as[4 * NPP + p] = nv > 0.f ? vx / nv : 0.f;
    as[5 * NPP + p] = nv > 0.f ? vy / nv : 0.f;
    as[6 * NPP + p] = (ix + 0.5f) / FN - 0.5f;
    as[7 * NPP + p] = (iy0 + r + 0.5f) / FN - 0.5f;
  }
}

// rows iy0 - 1 .. iy0 + RB of u_in (clamped) and rows iy0 .. of f into shared memory
__device__ __forceinline__ void load_inputs(const float2* u_in, const float2* f, int fps, int b, int iy0, float2* us,
                                            float2* fs) {
#pragma unroll
  for (int r = 0; r < RB + 2; ++r) {
    const int iy = min(max(iy0 - 1 + r, 0), FN - 1);
    cta_copy(us + r * FN, u_in + (long long)b * FNN + iy * FN, FN * 8);
  }
  cta_copy(fs, f + (fps ? (long long)b * FNN : 0) + iy0 * FN, NP * 8);
}

// float4-wide elementwise pass over a [FC][NPP] shared block and its global [FC][FNN] rows
template <class Op>
__device__ __forceinline__ void planar_pass(float* sm, long long gbase, Op op) {
  for (int i = threadIdx.x; i < FC * NP / 4; i += NTH) {
    const int c = i / (NP / 4), q = i % (NP / 4);
    op(reinterpret_cast<float4*>(sm + c * NPP)[q], gbase + (long long)c * FNN + 4 * q);
  }
}

// ------------------------------------------------------------------ forward kernels
// v0 = W0 a + b0 (lifting), v0 to global, and its row DFT (the first column kernel's input).
constexpr int SM_LIFT = (FC * NPP + FIN * NPP) * 4 + ((RB + 2) * FN + NP + BLK) * 8 + T_ROW * 2;
__global__ void __launch_bounds__(NTH, 2) fno_lift_fwd(const float2* __restrict__ f, int fps,
                                                       const float2* __restrict__ u_in,
                                                       const __nv_bfloat16* __restrict__ wbf,
                                                       const float* __restrict__ pm,
                                                       const __nv_bfloat16* __restrict__ tabs,
                                                       float* __restrict__ v0, float2* __restrict__ T1) {
  extern __shared__ __align__(16) float smem[];
  float* ps = smem;                                         // [FC][NPP] v0
  float* as = ps + FC * NPP;                                // [FIN][NPP] features
  float2* us = reinterpret_cast<float2*>(as + FIN * NPP);   // [(RB + 2) FN]
  float2* fs = us + (RB + 2) * FN;                          // [NP]
  float2* stage = fs + NP;                                  // [BLK]
  __nv_bfloat16* tb = reinterpret_cast<__nv_bfloat16*>(stage + BLK);  // [T_ROW]
  __shared__ __nv_bfloat16 w0[FC * FIN];
  __shared__ float b0[FC];
  const int b = blockIdx.y, iyb = blockIdx.x, iy0 = iyb * RB;
  load_inputs(u_in, f, fps, b, iy0, us, fs);
  cta_copy(tb, tabs, T_ROW * 2);
  for (int i = threadIdx.x; i < FC * FIN; i += NTH) w0[i] = wbf[F_W0 + i];
  if (threadIdx.x < FC) b0[threadIdx.x] = pm[F_B0 + threadIdx.x];
  cp_wait_all();
  __syncthreads();
  features(us, fs, iy0, as);
  __syncthreads();
  {  // GEMM M = NP, N = FC, K = 16 (8 features, zero padded)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    auto A = [&](int p, int k) { return k < FIN ? as[k * NPP + p] : 0.f; };
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int mt = 2 * warp + i;
      const FragA a = load_a(A, 16 * mt, 0, g, t);
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int c = 8 * nt + g;
        uint32_t bb[2];
        bb[0] = bf_bits(w0[c * FIN + 2 * t]) | (bf_bits(w0[c * FIN + 2 * t + 1]) << 16);
        bb[1] = 0u;  // k >= 8: zero padding
        float d[4] = {0.f, 0.f, 0.f, 0.f};
        mma2(d, a, bb);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int p = 16 * mt + g + (e >> 1) * 8, cc = 8 * nt + 2 * t + (e & 1);
          ps[cc * NPP + p] = d[e] + b0[cc];
        }
      }
    }
  }
  __syncthreads();
  planar_pass(ps, (long long)b * FC * FNN + (long long)iy0 * FN,
              [&](float4& x, long long gi) { *reinterpret_cast<float4*>(v0 + gi) = x; });
  row_forward(ps, tb, stage);
  __syncthreads();
  float4* dst = reinterpret_cast<float4*>(T1 + ((long long)b * NIB + iyb) * BLK);
  for (int i = threadIdx.x; i < BLK / 2; i += NTH) dst[i] = reinterpret_cast<float4*>(stage)[i];
}

// Layer l: pre = Lsyn(Y) + W v + b (Lsyn: row inverse of the column kernel's Z),
// v_{l+1} = GELU(pre) (or pre), then either the row DFT of v_{l+1} for the
// next layer (PROJ = 0) or the projection out = P2 GELU(P1 v + c1) + c2 and,
// when x0 is given, the warm start x0 = u_in (1 + out_0 + j out_1) (PROJ = 1).
// Persistent over (sample, row block) items, on the fifth-generation tensor
// cores (tcgen05): one thread issues each GEMM as whole tiles, the operands
// staged once per item in BF16 hi / lo core-matrix layout (tc5.cuh), the
// accumulators in tensor memory:
//   D[ix][32 r + c] = sum_kyc E(ix, kyc) Z(32 r + c, kyc)   M 128, N 64, K 32  (inverse row DFT, transposed)
//   D[ix][32 r + o] += sum_i v(r, ix, i) W[o][i]             M 128, N 32, K 32  (W v, one tile per row r)
//   D3[32 r + c][kyc] = sum_ix v'(r, ix, c) E(ix, kyc)        M 64,  N 32, K 128 (row DFT of v_{l+1})
//   D4_r[ix][hid] = sum_c v'(r, ix, c) P1[hid][c]            M 128, N 128, K 32 (projection, PROJ)
// The first two accumulate into the same columns, so TMEM holds pre - b.
// Thread (warp w, lane l) owns pixel ix = 32 (w % 4) + l of image row r = w / 4:
// TMEM lane ix holds its row of D and D4_r, so pre = D + b, the GELU, the
// global stores of pre and v_{l+1} (consecutive lanes, consecutive addresses)
// and, for the projection, the 128 hidden units and P2 of its pixel stay in
// that thread.  D3 (M = 64) sits in lanes 16 q + m of warp quarter q.  The
// next item's v_l and Z values are loaded into registers while the current
// item's GEMMs and epilogues run.  Every wait on the MMAs is bounded; on a
// timeout the kernel records it in *err, frees its tensor memory and returns.
constexpr int TC_LBO = 128, TC_SBO = 512;             // K = 32 operands: 4 K groups of 128 bytes per 8 rows
constexpr int TC_RF_LBO = 160, TC_RF_SBO = 16 * 160;  // row-DFT A operand (K = 128), padded: conflict-free staging
constexpr int TC_TAB = T_TCP * 2;                     // bytes of one table plane
constexpr int TC_PL_MIX = NP * FC * 2;                // bytes of one plane of a [256 p][32 c] operand
constexpr int TC_PL_RF = 8 * TC_RF_SBO;               // bytes of one plane of the [64 rr][128 ix] operand
constexpr int TC_PL_Z = 2 * FC * 2 * FM * 2;          // bytes of one plane of Z [64 rr][32 kyc]
constexpr int TC_AREG = 2 * (TC_PL_RF > TC_PL_MIX ? TC_PL_RF : TC_PL_MIX);
constexpr int TSM_A = 4 * TC_TAB, TSM_Z = TSM_A + TC_AREG, TSM_W = TSM_Z + 2 * TC_PL_Z, TSM_BIAS = TSM_W + FC * FC * 2,
              TSM_C1 = TSM_BIAS + FC * 4, TSM_P2 = TSM_C1 + FH * 4, SM_ROW_TC = TSM_P2 + 2 * FH * 4;
constexpr int TC_WAIT = 1 << 20;  // polls of an MMA completion barrier before giving up
template <int PROJ>
__global__ void __launch_bounds__(NTH, 2) fno_row_tc(const float* __restrict__ vin, const float2* __restrict__ Z,
                                                     const __nv_bfloat16* __restrict__ wbf,
                                                     const float* __restrict__ pm, long long woff, long long boff,
                                                     const __nv_bfloat16* __restrict__ tabs, int act, int B,
                                                     float* __restrict__ pre_out, float* __restrict__ vout,
                                                     float2* __restrict__ T1, float2* __restrict__ out,
                                                     const float2* __restrict__ u_in, float2* __restrict__ x0,
                                                     int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  constexpr uint32_t NCOL = PROJ ? 256 : 128;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int q4 = warp & 3, r = warp >> 2, ix = 32 * q4 + lane;  // this thread's pixel (r, ix) and TMEM lane
  const int zr = tid & 63, zq = tid >> 6;                         // this thread's Z row and K group
  const int items = B * NIB;
  if (blockIdx.x >= items) return;
  float* bias = reinterpret_cast<float*>(sm + TSM_BIAS);
  float* c1 = reinterpret_cast<float*>(sm + TSM_C1);
  float* p2 = reinterpret_cast<float*>(sm + TSM_P2);
  // tables (RowI A; RowF B, or P1 for the projection), W, bias
  cta_copy(sm, tabs + T_TROW, (PROJ ? 2 : 4) * TC_TAB);
  for (int e = tid; e < FC * FC; e += NTH)
    *reinterpret_cast<__nv_bfloat16*>(sm + TSM_W + core_off(e / FC, e % FC, TC_LBO, TC_SBO)) = wbf[woff + e];
  if (tid < FC) bias[tid] = pm[boff + tid];
  if (PROJ) {
    for (int e = tid; e < FH * FC; e += NTH)
      *reinterpret_cast<__nv_bfloat16*>(sm + 2 * TC_TAB + core_off(e / FC, e % FC, TC_LBO, TC_SBO)) = wbf[F_P1 + e];
    for (int i = tid; i < FH; i += NTH) c1[i] = pm[F_C1 + i];
    for (int i = tid; i < 2 * FH; i += NTH) p2[i] = __bfloat162float(wbf[F_P2 + i]);
  }
  if (tid == 0) mbar_init(&mbar);
  if (warp == 0) tmem_alloc(&tslot, NCOL);
  cp_wait_all();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot;
  const uint32_t s0 = smem_addr(sm);
  const uint32_t tl = tmem + ((uint32_t)(32 * q4) << 16);  // this warp's TMEM lane quarter
  const float c20 = PROJ ? pm[F_C2] : 0.f, c21 = PROJ ? pm[F_C2 + 1] : 0.f;
  float nv[FC];
  float2 nz[4];
  auto fetch = [&](int it) {
    const int b = it / NIB, iyb = it % NIB;
    const float* src = vin + (long long)b * FC * FNN + (long long)(iyb * RB + r) * FN + ix;
#pragma unroll
    for (int c = 0; c < FC; ++c) nv[c] = __ldg(src + (long long)c * FNN);
    const float2* zb = Z + ((long long)b * NIB + iyb) * BLK;
#pragma unroll
    for (int m = 0; m < 4; ++m) nz[m] = __ldg(zb + ((4 * zq + m) * FC + (zr & 31)) * RB + (zr >> 5));
  };
  // 32 values of one [256 p][32 c] row p into the hi / lo planes at byte offset a (uint4 stores)
  auto stage_row32 = [&](int a, int p, const float (&x)[FC]) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      uint4 h, l;
      split_pair(x[8 * j + 0], x[8 * j + 1], h.x, l.x);
      split_pair(x[8 * j + 2], x[8 * j + 3], h.y, l.y);
      split_pair(x[8 * j + 4], x[8 * j + 5], h.z, l.z);
      split_pair(x[8 * j + 6], x[8 * j + 7], h.w, l.w);
      const int o = core_off(p, 8 * j, TC_LBO, TC_SBO);
      *reinterpret_cast<uint4*>(sm + a + o) = h;
      *reinterpret_cast<uint4*>(sm + a + TC_PL_MIX + o) = l;
    }
  };
  auto sync_mma = [&]() {  // thread-written operands visible to the tensor cores, TMEM reads ordered
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  };
  uint32_t ph = 0;
  bool failed = false;
  auto wait_mma = [&]() {  // true if the committed MMAs completed in every thread's view
    const bool ok = mbar_wait(&mbar, ph, TC_WAIT);
    ph ^= 1u;
    tc_fence_after();
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicExch(err, 1);
      failed = true;
    }
    return !failed;
  };
  const uint32_t id_i = tc_idesc_bf16(128, 64), id_w = tc_idesc_bf16(128, 32), id_f = tc_idesc_bf16(64, 32),
                 id_p = tc_idesc_bf16(128, 128);
  fetch(blockIdx.x);
  for (int it = blockIdx.x; it < items; it += gridDim.x) {
    const int b = it / NIB, iyb = it % NIB, iy0 = iyb * RB;
    const long long pix0 = (long long)iy0 * FN;
    const long long gbase = (long long)b * FC * FNN + pix0;
    // stage v_l (A of W v) and Z (B of the inverse row DFT), then fetch the next item
    stage_row32(TSM_A, FN * r + ix, nv);
    {
      uint4 h, l;
      split_pair(nz[0].x, nz[0].y, h.x, l.x);
      split_pair(nz[1].x, nz[1].y, h.y, l.y);
      split_pair(nz[2].x, nz[2].y, h.z, l.z);
      split_pair(nz[3].x, nz[3].y, h.w, l.w);
      const int o = core_off(zr, 8 * zq, TC_LBO, TC_SBO);
      *reinterpret_cast<uint4*>(sm + TSM_Z + o) = h;
      *reinterpret_cast<uint4*>(sm + TSM_Z + TC_PL_Z + o) = l;
    }
    const int nxt = it + gridDim.x;
    if (nxt < items) fetch(nxt);
    sync_mma();
    if (tid == 0) {
      // inverse row DFT: E (hi, lo) x Z (hi, lo), three products per K step
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        const uint32_t ah = s0 + ks * 2 * TC_LBO, al = ah + TC_TAB;
        const uint32_t bh = s0 + TSM_Z + ks * 2 * TC_LBO, bl = bh + TC_PL_Z;
        tc_mma(tmem, tc_desc(ah, TC_LBO, TC_SBO), tc_desc(bh, TC_LBO, TC_SBO), id_i, ks > 0);
        tc_mma(tmem, tc_desc(al, TC_LBO, TC_SBO), tc_desc(bh, TC_LBO, TC_SBO), id_i, 1);
        tc_mma(tmem, tc_desc(ah, TC_LBO, TC_SBO), tc_desc(bl, TC_LBO, TC_SBO), id_i, 1);
      }
      // + W v, row by row into the same columns (W exact in BF16, v as hi + lo)
#pragma unroll
      for (int rr = 0; rr < RB; ++rr)
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
          const uint32_t ah = s0 + TSM_A + rr * (TC_PL_MIX / 2) + ks * 2 * TC_LBO, al = ah + TC_PL_MIX;
          const uint64_t bw = tc_desc(s0 + TSM_W + ks * 2 * TC_LBO, TC_LBO, TC_SBO);
          tc_mma(tmem + 32 * rr, tc_desc(ah, TC_LBO, TC_SBO), bw, id_w, 1);
          tc_mma(tmem + 32 * rr, tc_desc(al, TC_LBO, TC_SBO), bw, id_w, 1);
        }
      tc_commit(&mbar);
    }
    if (!wait_mma()) break;
    // epilogue: pre = D + b (to global when training), v_{l+1} = act(pre) to global, staged as the next A
    float v[FC];
    tmem_ld32(tl + 32 * r, v);
#pragma unroll
    for (int j = 0; j < FC / 4; ++j) {
      const float4 bj = reinterpret_cast<const float4*>(bias)[j];
      v[4 * j] += bj.x;
      v[4 * j + 1] += bj.y;
      v[4 * j + 2] += bj.z;
      v[4 * j + 3] += bj.w;
    }
    {
      const long long g0 = gbase + (long long)r * FN + ix;
#pragma unroll
      for (int c = 0; c < FC; ++c) {
        if (pre_out) pre_out[g0 + (long long)c * FNN] = v[c];
        if (act) v[c] = gelu_f(v[c]);
        if (vout) vout[g0 + (long long)c * FNN] = v[c];
      }
    }
    if (!PROJ) {
      // A of the row DFT, [32 r + c][ix]: lanes ix, ix + 1 exchange so that each stores a 32-bit pair
      const bool odd = lane & 1;
#pragma unroll
      for (int m = 0; m < FC / 2; ++m) {
        const float y = __shfl_xor_sync(0xffffffffu, odd ? v[2 * m] : v[2 * m + 1], 1);
        const int row = 32 * r + 2 * m + (odd ? 1 : 0), k = ix & ~1;
        uint32_t h, l;
        if (odd)
          split_pair(y, v[2 * m + 1], h, l);
        else
          split_pair(v[2 * m], y, h, l);
        const int o = core_off(row, k, TC_RF_LBO, TC_RF_SBO);
        *reinterpret_cast<uint32_t*>(sm + TSM_A + o) = h;
        *reinterpret_cast<uint32_t*>(sm + TSM_A + TC_PL_RF + o) = l;
      }
    } else {
      stage_row32(TSM_A, FN * r + ix, v);
    }
    sync_mma();
    if (tid == 0) {
      if (!PROJ) {  // row DFT: v' (hi, lo) x E (hi, lo) into columns 64 ..
#pragma unroll
        for (int ks = 0; ks < FN / 16; ++ks) {
          const uint32_t ah = s0 + TSM_A + ks * 2 * TC_RF_LBO, al = ah + TC_PL_RF;
          const uint32_t bh = s0 + 2 * TC_TAB + ks * 2 * TC_LBO, bl = bh + TC_TAB;
          tc_mma(tmem + 64, tc_desc(ah, TC_RF_LBO, TC_RF_SBO), tc_desc(bh, TC_LBO, 2048), id_f, ks > 0);
          tc_mma(tmem + 64, tc_desc(al, TC_RF_LBO, TC_RF_SBO), tc_desc(bh, TC_LBO, 2048), id_f, 1);
          tc_mma(tmem + 64, tc_desc(ah, TC_RF_LBO, TC_RF_SBO), tc_desc(bl, TC_LBO, 2048), id_f, 1);
        }
      } else {  // z = P1 v' per row r into columns 128 r ..
#pragma unroll
        for (int rr = 0; rr < RB; ++rr)
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            const uint32_t ah = s0 + TSM_A + rr * (TC_PL_MIX / 2) + ks * 2 * TC_LBO, al = ah + TC_PL_MIX;
            const uint64_t bp = tc_desc(s0 + 2 * TC_TAB + ks * 2 * TC_LBO, TC_LBO, TC_SBO);
            tc_mma(tmem + 128 * rr, tc_desc(ah, TC_LBO, TC_SBO), bp, id_p, ks > 0);
            tc_mma(tmem + 128 * rr, tc_desc(al, TC_LBO, TC_SBO), bp, id_p, 1);
          }
      }
      tc_commit(&mbar);
    }
    if (!wait_mma()) break;
    if (!PROJ) {  // T1 block [ky][c][r] from rows 32 r + c (lanes 16 q + m), columns split by warp half
      float2* dst = T1 + ((long long)b * NIB + iyb) * BLK;
      const int rr = 16 * q4 + lane;
      float d[16];
      tmem_ld16(tl + 64 + 16 * r, d);
      if (lane < 16)
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int ky = 8 * r + k;
          dst[(ky * FC + (rr & 31)) * RB + (rr >> 5)] = make_float2(d[2 * k], d[2 * k + 1]);
        }
    } else {  // out = P2 GELU(z + c1) + c2 for this thread's pixel; warm start x0 = u_in (1 + out)
      float o0 = c20, o1 = c21;
      const float4 *c14 = reinterpret_cast<const float4*>(c1), *p204 = reinterpret_cast<const float4*>(p2),
                   *p214 = reinterpret_cast<const float4*>(p2 + FH);
#pragma unroll 1
      for (int j = 0; j < FH / 32; ++j) {
        float d[32];
        tmem_ld32(tl + 128 * r + 32 * j, d);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float4 cc = c14[8 * j + k], q0 = p204[8 * j + k], q1 = p214[8 * j + k];
          const float h0 = gelu_f(d[4 * k] + cc.x), h1 = gelu_f(d[4 * k + 1] + cc.y);
          const float h2 = gelu_f(d[4 * k + 2] + cc.z), h3 = gelu_f(d[4 * k + 3] + cc.w);
          o0 += q0.x * h0 + q0.y * h1 + q0.z * h2 + q0.w * h3;
          o1 += q1.x * h0 + q1.y * h1 + q1.z * h2 + q1.w * h3;
        }
      }
      const long long pix = (long long)b * FNN + pix0 + (long long)r * FN + ix;
      const float2 e = make_float2(o0, o1);
      if (out) out[pix] = e;
      if (x0) {
        const float2 u = u_in[pix];
        x0[pix] = c_add(u, c_mul(u, e));
      }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, NCOL);
}

// ------------------------------------------------------------------ column stage
// Layer l's spectral convolution along iy, between the row kernels' spectra T
// ([B][64 row pairs][16 ky][32 c][2] blocks) and Z in the same layout:
//   X = ColF(T)               the 32 kept kx of the column DFT       (fno_colf_tc, tensor cores)
//   Y = mix_R(X) w_ky / 128^2 per mode (kx, ky): 32 x 32 complex   (fno_mix, FP32 pipes)
//   Z = ColI(Y)               inverse column DFT at all 128 iy       (fno_coli_tc, tensor cores)
// The backward runs the same chain on dT: dY = ColF(dT) w_ky / 128^2,
// dX = mix_R^H(dY) with grad R = sum_b conj(X) dY in the same kernel
// (fno_mix_bwd), dU = ColI(dX).  X and dY stay in HBM / L2 between the
// kernels, mode-major [mode = kx * 16 + ky][B][32 c]: the forward's X is the
// backward's operand for grad R.
//
// The column DFTs are GEMMs with 128 rows = (4 ky) x (32 channels) of one
// sample, issued as whole tiles by one thread (tc5.cuh), operands in BF16 hi /
// lo planes (three products, the FP32 accuracy of the other FNO contractions),
// accumulators in TMEM with row n in lane n: thread (warp w, lane l) owns
// channel l of ky = 4 g + w % 4, and warps w, w + 4 split its columns.
constexpr int KY_G = 4;                           // ky per column CTA
constexpr int CF_SBO = 4096, CI_SBO = 1024;       // 8-row strides of the K = 256 and K = 64 operands
constexpr int KCF_PA = 128 * 2 * FN * 2;          // bytes of one plane of T [128 n][256 k]
constexpr int KCI_PA = 128 * 2 * FKX * 2;         // bytes of one plane of Y [128 n][64 k]
constexpr int KC_PB = T_TCF * 2;                  // bytes of one plane of a column table
constexpr int SM_COLF = 2 * KCF_PA + 2 * KC_PB;   // 192 KB: one CTA per SM
constexpr int SM_COLI = 2 * KCI_PA + 2 * KC_PB;   // 96 KB: two CTAs per SM
__device__ __forceinline__ float ky_scale(int ky) { return (ky ? 2.f : 1.f) / FNN; }

// One thread issues the MMAs, every thread waits (bounded) for their completion: false (and *err set)
// if the wait gave up anywhere in the CTA.
__device__ __forceinline__ bool tc_wait_all(uint64_t* mbar, int* err) {
  const bool ok = mbar_wait(mbar, 0, TC_WAIT);
  tc_fence_after();
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) atomicExch(err, 1);
    return false;
  }
  return true;
}

// X[kx][ky][b][c] = sum_iy F(kx, iy) T[iy][ky][b][c] for ky in [4 g, 4 g + 4): D[n][j] = sum_k T[n][k] ColF[j][k]
// (M 128, N 64, K 256).  BWD: dT in, dY = X w_ky / 128^2 out.  Grid (16 / 4, B).
template <int BWD>
__global__ void __launch_bounds__(NTH, 1) fno_colf_tc(const float2* __restrict__ Tin,
                                                      const __nv_bfloat16* __restrict__ tabs, int B,
                                                      float2* __restrict__ Xout, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ky0 = blockIdx.x * KY_G, b = blockIdx.y;
  cta_copy(sm + 2 * KCF_PA, tabs + T_TCOLF, 2 * KC_PB);
  // T[n = 32 kyl + c][k = 2 iy + p]: one 16-byte load per (n, row pair) = k 4 iyb .. 4 iyb + 3.  A warp
  // covers 8 n x 4 row pairs: 128-byte global pieces, 8-byte stores on all 32 banks.
  const float2* tb = Tin + (long long)b * NIB * BLK + ky0 * FC * RB;
#pragma unroll 8
  for (int it = 0; it < NIB * 128 / NTH; ++it) {
    const int idx = tid + NTH * it;
    const int n = 8 * ((idx >> 5) & 15) + (idx & 7), iyb = 4 * (idx >> 9) + ((idx >> 3) & 3);
    const float4 v = __ldg(reinterpret_cast<const float4*>(tb + (long long)iyb * BLK + n * RB));
    uint2 h, l;
    split_pair(v.x, v.y, h.x, l.x);
    split_pair(v.z, v.w, h.y, l.y);
    const int o = core_off(n, 4 * iyb, TC_LBO, CF_SBO);
    *reinterpret_cast<uint2*>(sm + o) = h;
    *reinterpret_cast<uint2*>(sm + KCF_PA + o) = l;
  }
  if (tid == 0) mbar_init(&mbar);
  if (warp == 0) tmem_alloc(&tslot, 64);
  cp_wait_all();
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot, s0 = smem_addr(sm);
  if (tid == 0) {
    const uint32_t id = tc_idesc_bf16(128, 64);
#pragma unroll
    for (int ks = 0; ks < 2 * FN / 16; ++ks) {
      const uint32_t ah = s0 + ks * 2 * TC_LBO, al = ah + KCF_PA;
      const uint32_t bh = s0 + 2 * KCF_PA + ks * 2 * TC_LBO, bl = bh + KC_PB;
      tc_mma(tmem, tc_desc(ah, TC_LBO, CF_SBO), tc_desc(bh, TC_LBO, CF_SBO), id, ks > 0);
      tc_mma(tmem, tc_desc(al, TC_LBO, CF_SBO), tc_desc(bh, TC_LBO, CF_SBO), id, 1);
      tc_mma(tmem, tc_desc(ah, TC_LBO, CF_SBO), tc_desc(bl, TC_LBO, CF_SBO), id, 1);
    }
    tc_commit(&mbar);
  }
  if (tc_wait_all(&mbar, err)) {
    const int q = warp & 3, h = warp >> 2, ky = ky0 + q;
    const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);
    const float sc = BWD ? ky_scale(ky) : 1.f;
#pragma unroll
    for (int half = 0; half < 2; ++half) {  // kx 16 h + 8 half .. + 7: Re in column kx, Im in column 32 + kx
      float re[8], im[8];
      tmem_ld8(tl + 16 * h + 8 * half, re);
      tmem_ld8(tl + FKX + 16 * h + 8 * half, im);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int kx = 16 * h + 8 * half + t;
        Xout[((long long)(kx * FM + ky) * B + b) * FC + lane] = make_float2(re[t] * sc, im[t] * sc);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 64);
}

// Z[iy][ky][b][o] = sum_kx conj(F(kx, iy)) Y[kx][ky][b][o] for ky in [4 g, 4 g + 4): D[n][j] = sum_k Y[n][k]
// ColI[j][k] (M 128, N 256, K 64), j = 2 iy + p, written as the row kernels' [iyb][ky][o][2] blocks.
__global__ void __launch_bounds__(NTH, 2) fno_coli_tc(const float2* __restrict__ Yin,
                                                      const __nv_bfloat16* __restrict__ tabs, int B,
                                                      float2* __restrict__ Zout, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ky0 = blockIdx.x * KY_G, b = blockIdx.y;
  cta_copy(sm + 2 * KCI_PA, tabs + T_TCOLI, 2 * KC_PB);
  // Y[n = 32 kyl + o][k = 2 kx + p]: a warp covers 8 n x 4 kx (64-byte global pieces, 4-byte stores on
  // all 32 banks)
#pragma unroll 8
  for (int it = 0; it < FKX * 128 / NTH; ++it) {
    const int idx = tid + NTH * it;
    const int n = 8 * ((idx >> 5) & 15) + (idx & 7), kx = 4 * (idx >> 9) + ((idx >> 3) & 3);
    const float2 v = __ldg(Yin + ((long long)(kx * FM + ky0 + (n >> 5)) * B + b) * FC + (n & 31));
    uint32_t h, l;
    split_pair(v.x, v.y, h, l);
    const int o = core_off(n, 2 * kx, TC_LBO, CI_SBO);
    *reinterpret_cast<uint32_t*>(sm + o) = h;
    *reinterpret_cast<uint32_t*>(sm + KCI_PA + o) = l;
  }
  if (tid == 0) mbar_init(&mbar);
  if (warp == 0) tmem_alloc(&tslot, 256);
  cp_wait_all();
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot, s0 = smem_addr(sm);
  if (tid == 0) {
    const uint32_t id = tc_idesc_bf16(128, 256);
#pragma unroll
    for (int ks = 0; ks < 2 * FKX / 16; ++ks) {
      const uint32_t ah = s0 + ks * 2 * TC_LBO, al = ah + KCI_PA;
      const uint32_t bh = s0 + 2 * KCI_PA + ks * 2 * TC_LBO, bl = bh + KC_PB;
      tc_mma(tmem, tc_desc(ah, TC_LBO, CI_SBO), tc_desc(bh, TC_LBO, CI_SBO), id, ks > 0);
      tc_mma(tmem, tc_desc(al, TC_LBO, CI_SBO), tc_desc(bh, TC_LBO, CI_SBO), id, 1);
      tc_mma(tmem, tc_desc(ah, TC_LBO, CI_SBO), tc_desc(bl, TC_LBO, CI_SBO), id, 1);
    }
    tc_commit(&mbar);
  }
  if (tc_wait_all(&mbar, err)) {
    const int q = warp & 3, h = warp >> 2, ky = ky0 + q;
    const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);
    float4* zb = reinterpret_cast<float4*>(Zout + (long long)b * NIB * BLK + (ky * FC + lane) * RB);
#pragma unroll 4
    for (int m = 0; m < 16; ++m) {  // columns 128 h + 8 m ..: iy 64 h + 4 m .. + 3 = row pairs 32 h + 2 m, + 1
      float d[8];
      tmem_ld8(tl + 128 * h + 8 * m, d);
      const int iyb = 32 * h + 2 * m;
      zb[(long long)iyb * (BLK / 2)] = make_float4(d[0], d[1], d[2], d[3]);
      zb[(long long)(iyb + 1) * (BLK / 2)] = make_float4(d[4], d[5], d[6], d[7]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 256);
}

// Y[m][b][o] = w_ky / 128^2 sum_c X[m][b][c] R[m][c][o], one CTA per mode m = (kx, ky), samples in chunks
// of 32: thread (warp w, lane o) forms samples w, w + 8, w + 16, w + 24 of the chunk.
constexpr int MIXP = FC + 1;  // shared pitch (complex) of a 32-wide row
__global__ void __launch_bounds__(NTH) fno_mix(const float2* __restrict__ X, const __nv_bfloat16* __restrict__ wbf,
                                               long long roff, int B, float2* __restrict__ Y) {
  __shared__ float2 rs[FC * MIXP], xs[32 * MIXP];
  const int m = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const __nv_bfloat162* R = reinterpret_cast<const __nv_bfloat162*>(wbf + roff) + (long long)m * FC * FC;
  for (int e = threadIdx.x; e < FC * FC; e += NTH) rs[(e / FC) * MIXP + e % FC] = __bfloat1622float2(R[e]);
  const float sc = ky_scale(m % FM);
  for (int b0 = 0; b0 < B; b0 += 32) {
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * FC; e += NTH) {
      const int bb = b0 + e / FC;
      xs[(e / FC) * MIXP + e % FC] = bb < B ? X[((long long)m * B + bb) * FC + e % FC] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2 acc[4] = {};
#pragma unroll 8
    for (int c = 0; c < FC; ++c) {
      const float2 r = rs[c * MIXP + lane];
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[i] = c_fma(xs[(warp + 8 * i) * MIXP + c], r, acc[i]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int bb = b0 + warp + 8 * i;
      if (bb < B) Y[((long long)m * B + bb) * FC + lane] = c_scale(acc[i], sc);
    }
  }
}

// Backward of the mixing for mode m: dX[b][c] = sum_o conj(R[c][o]) dY[b][o] (thread: lane c, samples w + 8 i)
// and grad R[m][c][o] = sum_b conj(X[b][c]) dY[b][o] (thread: rows c = w + 8 i, lane o), the batch summed in
// one CTA in sample order (deterministic), written as (Re, Im) pairs.
__global__ void __launch_bounds__(NTH) fno_mix_bwd(const float2* __restrict__ X, const float2* __restrict__ dY,
                                                   const __nv_bfloat16* __restrict__ wbf, long long roff, int B,
                                                   float2* __restrict__ dX, float* __restrict__ gradR) {
  __shared__ float2 rs[FC * MIXP], xs[32 * MIXP], gs[32 * MIXP];
  const int m = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const __nv_bfloat162* R = reinterpret_cast<const __nv_bfloat162*>(wbf + roff) + (long long)m * FC * FC;
  for (int e = threadIdx.x; e < FC * FC; e += NTH) rs[(e / FC) * MIXP + e % FC] = __bfloat1622float2(R[e]);
  float2 gr[4] = {};
  for (int b0 = 0; b0 < B; b0 += 32) {
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * FC; e += NTH) {
      const int bb = b0 + e / FC;
      const long long src = ((long long)m * B + bb) * FC + e % FC;
      xs[(e / FC) * MIXP + e % FC] = bb < B ? X[src] : make_float2(0.f, 0.f);
      gs[(e / FC) * MIXP + e % FC] = bb < B ? dY[src] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2 acc[4] = {};
#pragma unroll 8
    for (int o = 0; o < FC; ++o) {
      const float2 r = rs[lane * MIXP + o];
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[i] = c_cjfma(r, gs[(warp + 8 * i) * MIXP + o], acc[i]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int bb = b0 + warp + 8 * i;
      if (bb < B) dX[((long long)m * B + bb) * FC + lane] = acc[i];
    }
    const int nb = B - b0 < 32 ? B - b0 : 32;
    for (int bb = 0; bb < nb; ++bb) {
      const float2 g = gs[bb * MIXP + lane];
#pragma unroll
      for (int i = 0; i < 4; ++i) gr[i] = c_cjfma(xs[bb * MIXP + warp + 8 * i], g, gr[i]);
    }
  }
  float2* out = reinterpret_cast<float2*>(gradR) + (long long)m * FC * FC;
#pragma unroll
  for (int i = 0; i < 4; ++i) out[(warp + 8 * i) * FC + lane] = gr[i];
}

// Layer l backward, persistent over (sample, row block) items:
//   dv  = dvp + RowI(dU)          (dvp = W_{l+1}^T dpre_{l+1} or the projection's; dU from the column kernel)
//   dpre = dv * GELU'(pre_l)      (or dv on the last layer)
//   dvp_out = W_l^T dpre, dT = RowF(dpre),
//   per-CTA partials of grad W_l = sum_p dpre v_l^T and grad b_l = sum_p dpre.
constexpr int SM_RBWD = (2 * FC * NPP) * 4 + BLK * 8 + T_ROW * 2 + FC * WP * 2;
__global__ void __launch_bounds__(NTH, 2) fno_row_bwd(const float* __restrict__ dvp, const float2* __restrict__ dU,
                                                      const float* __restrict__ pre, const float* __restrict__ v,
                                                      const __nv_bfloat16* __restrict__ wbf, long long woff,
                                                      const __nv_bfloat16* __restrict__ tabs, int B, int act,
                                                      float* __restrict__ dvp_out, float2* __restrict__ dT,
                                                      float* __restrict__ part) {
  extern __shared__ __align__(16) float smem[];
  float* gs = smem;                                        // [FC][NPP] dv, then dpre
  float* vs = gs + FC * NPP;                               // [FC][NPP] v_l
  float2* zs = reinterpret_cast<float2*>(vs + FC * NPP);   // [BLK] dU block, then the dT block
  __nv_bfloat16* tb = reinterpret_cast<__nv_bfloat16*>(zs + BLK);  // [T_ROW]
  __nv_bfloat16* wt = tb + T_ROW;                          // [FC][WP]: W^T (i, o)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  cta_copy(tb, tabs, T_ROW * 2);
  load_w(wbf + woff, nullptr, wt);
  float dw[4] = {0.f, 0.f, 0.f, 0.f};
  float db = 0.f;
  const int items = B * NIB;
  for (int it = blockIdx.x; it < items; it += gridDim.x) {
    const int b = it / NIB, iyb = it % NIB, iy0 = iyb * RB;
    const long long pix0 = (long long)iy0 * FN;
    const long long gbase = (long long)b * FC * FNN + pix0;
    load_planar(gs, dvp, b, pix0);
    load_planar(vs, v, b, pix0);
    if (dU) cta_copy(zs, dU + ((long long)b * NIB + iyb) * BLK, BLK * 8);
    cp_wait_all();
    __syncthreads();
    if (dU) {
      row_inverse(zs, tb, gs, true);
      __syncthreads();
    }
    if (act)
      planar_pass(gs, gbase, [&](float4& x, long long gi) {
        const float4 p = *reinterpret_cast<const float4*>(pre + gi);
        x.x *= gelu_grad_f(p.x);
        x.y *= gelu_grad_f(p.y);
        x.z *= gelu_grad_f(p.z);
        x.w *= gelu_grad_f(p.w);
      });
    __syncthreads();
    // dvp_out = W^T dpre: GEMM M = NP, N = FC (i), K = FC (o)
    pixel_mix([&](int p, int o) { return gs[o * NPP + p]; }, wt,
              [&](int p, int i, float val) { dvp_out[gbase + (long long)i * FNN + p] = val; });
    {  // grad W += dpre v^T: GEMM M = FC (o), N = FC (i), K = NP; warp = one 16 x 8 tile
      auto A = [&](int o, int p) { return gs[o * NPP + p]; };
      auto Bv = [&](int p, int i) { return vs[i * NPP + p]; };
      const int mt = warp & 1, nt = warp >> 1;
#pragma unroll 4
      for (int ks = 0; ks < NP / 16; ++ks) mma3(dw, load_a(A, 16 * mt, 16 * ks, g, t), load_b(Bv, 16 * ks, 8 * nt, g, t));
      const int o = threadIdx.x >> 3;
      for (int p = threadIdx.x & 7; p < NP; p += 8) db += gs[o * NPP + p];
    }
    row_forward(gs, tb, zs);
    __syncthreads();
    float4* dst = reinterpret_cast<float4*>(dT + ((long long)b * NIB + iyb) * BLK);
    for (int i = threadIdx.x; i < BLK / 2; i += NTH) dst[i] = reinterpret_cast<float4*>(zs)[i];
    __syncthreads();
  }
  float* pp = part + (long long)blockIdx.x * PART_W;
  {
    const int mt = warp & 1, nt = warp >> 1;
#pragma unroll
    for (int e = 0; e < 4; ++e) pp[(16 * mt + g + (e >> 1) * 8) * FC + 8 * nt + 2 * t + (e & 1)] = dw[e];
  }
  db += __shfl_xor_sync(0xffffffffu, db, 1);
  db += __shfl_xor_sync(0xffffffffu, db, 2);
  db += __shfl_xor_sync(0xffffffffu, db, 4);
  if ((threadIdx.x & 7) == 0) pp[FC * FC + (threadIdx.x >> 3)] = db;
}

// Projection backward, persistent over items: recomputes z = P1 v4 + c1 per chunk of 32 hidden
// units, dz = (P2^T dout) GELU'(z); dvp_out = P1^T dz; per-CTA partials of grad P1, c1, P2, c2.
constexpr int SM_PBWD = (3 * FC * NPP + 2 * NPP + FH + 2 * FH) * 4 + (FH * WP + FC * P1TP) * 2;
__global__ void __launch_bounds__(NTH, 1) fno_proj_bwd(const float* __restrict__ v4, const float* __restrict__ dout,
                                                       const __nv_bfloat16* __restrict__ wbf,
                                                       const float* __restrict__ pm, int B,
                                                       float* __restrict__ dvp_out, float* __restrict__ part) {
  extern __shared__ __align__(16) float smem[];
  float* vs = smem;              // [FC][NPP] v4
  float* zs = vs + FC * NPP;     // [32][NPP] dz of the chunk
  float* hs = zs + FC * NPP;     // [32][NPP] h of the chunk
  float* ds = hs + FC * NPP;     // [2][NPP] dout
  float* c1 = ds + 2 * NPP;      // [FH]
  float* p2 = c1 + FH;           // [2][FH]
  __nv_bfloat16* p1 = reinterpret_cast<__nv_bfloat16*>(p2 + 2 * FH);  // [FH][WP] P1[hid][c]
  __nv_bfloat16* p1t = p1 + FH * WP;                                   // [FC][P1TP] P1^T[c][hid]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  for (int e = threadIdx.x; e < FH * FC; e += NTH) {
    const __nv_bfloat16 w = wbf[F_P1 + e];
    p1[(e / FC) * WP + e % FC] = w;
    p1t[(e % FC) * P1TP + e / FC] = w;
  }
  for (int i = threadIdx.x; i < FH; i += NTH) c1[i] = pm[F_C1 + i];
  for (int i = threadIdx.x; i < 2 * FH; i += NTH) p2[i] = __bfloat162float(wbf[F_P2 + i]);
  const uint32_t* p132 = reinterpret_cast<const uint32_t*>(p1);
  const uint32_t* p1t32 = reinterpret_cast<const uint32_t*>(p1t);
  float ap1[4][4];
#pragma unroll
  for (int q = 0; q < 4; ++q) ap1[q][0] = ap1[q][1] = ap1[q][2] = ap1[q][3] = 0.f;
  float ac1[4] = {0.f, 0.f, 0.f, 0.f}, ap2[4][2] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}}, ac2 = 0.f;
  const int items = B * NIB;
  auto Av = [&](int p, int c) { return vs[c * NPP + p]; };
  for (int it = blockIdx.x; it < items; it += gridDim.x) {
    const int b = it / NIB, iyb = it % NIB, iy0 = iyb * RB;
    const long long pix0 = (long long)iy0 * FN;
    load_planar(vs, v4, b, pix0);
    for (int o = 0; o < 2; ++o) cta_copy(ds + o * NPP, dout + ((long long)b * 2 + o) * FNN + pix0, NP * 4);
    cp_wait_all();
    __syncthreads();
    {
      const int o = threadIdx.x >> 7;
      for (int p = threadIdx.x & 127; p < NP; p += 128) ac2 += ds[o * NPP + p];
    }
    FragA av[2][2];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) av[h][ks] = load_a(Av, 16 * (2 * warp + h), 16 * ks, g, t);
    float adv[2][4][4];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int j = 0; j < 4; ++j) adv[h][j][0] = adv[h][j][1] = adv[h][j][2] = adv[h][j][3] = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int mt = 2 * warp + h;
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          uint32_t b0[2], b1[2];
          load_b_tab(p132, WP / 2, 0, 32 * q + 8 * nt, g, t, b0);
          load_b_tab(p132, WP / 2, 16, 32 * q + 8 * nt, g, t, b1);
          float d[4] = {0.f, 0.f, 0.f, 0.f};
          mma2(d, av[h][0], b0);
          mma2(d, av[h][1], b1);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int p = 16 * mt + g + (e >> 1) * 8, hl = 8 * nt + 2 * t + (e & 1), hid = 32 * q + hl;
            const float z = d[e] + c1[hid];
            const float dh = p2[hid] * ds[p] + p2[FH + hid] * ds[NPP + p];
            float gv, gd;
            gelu_and_grad(z, gv, gd);
            hs[hl * NPP + p] = gv;
            zs[hl * NPP + p] = dh * gd;
          }
        }
      }
      __syncthreads();
      {  // dv += P1_chunk^T dz: GEMM M = NP, N = FC, K = 32 (B = P1^T rows, pairs along hidden)
        auto Ad = [&](int p, int hl) { return zs[hl * NPP + p]; };
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int mt = 2 * warp + h;
          const FragA a0 = load_a(Ad, 16 * mt, 0, g, t), a1 = load_a(Ad, 16 * mt, 16, g, t);
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) {
            uint32_t b0[2], b1[2];
            load_b_tab(p1t32, P1TP / 2, 32 * q, 8 * nt, g, t, b0);
            load_b_tab(p1t32, P1TP / 2, 32 * q + 16, 8 * nt, g, t, b1);
            mma2(adv[h][nt], a0, b0);
            mma2(adv[h][nt], a1, b1);
          }
        }
      }
      {  // grad P1_chunk += dz v4^T: GEMM M = 32 (hidden), N = FC, K = NP; one tile per warp
        auto Ad = [&](int hl, int p) { return zs[hl * NPP + p]; };
        auto Bv = [&](int p, int c) { return vs[c * NPP + p]; };
        const int mt = warp & 1, nt = warp >> 1;
#pragma unroll 4
        for (int ks = 0; ks < NP / 16; ++ks)
          mma3(ap1[q], load_a(Ad, 16 * mt, 16 * ks, g, t), load_b(Bv, 16 * ks, 8 * nt, g, t));
        const int hl = threadIdx.x >> 3;
        for (int p = threadIdx.x & 7; p < NP; p += 8) {
          ac1[q] += zs[hl * NPP + p];
          ap2[q][0] += ds[p] * hs[hl * NPP + p];
          ap2[q][1] += ds[NPP + p] * hs[hl * NPP + p];
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int p = 16 * (2 * warp + h) + g + (e >> 1) * 8, c = 8 * nt + 2 * t + (e & 1);
          dvp_out[((long long)b * FC + c) * FNN + pix0 + p] = adv[h][nt][e];
        }
  }
  __shared__ float red2[NTH];
  float* pp = part + (long long)blockIdx.x * PART_P;
  {
    const int mt = warp & 1, nt = warp >> 1;
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int e = 0; e < 4; ++e)
        pp[(32 * q + 16 * mt + g + (e >> 1) * 8) * FC + 8 * nt + 2 * t + (e & 1)] = ap1[q][e];
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float s = ac1[q], s0 = ap2[q][0], s1 = ap2[q][1];
#pragma unroll
    for (int k = 1; k < 8; k <<= 1) {
      s += __shfl_xor_sync(0xffffffffu, s, k);
      s0 += __shfl_xor_sync(0xffffffffu, s0, k);
      s1 += __shfl_xor_sync(0xffffffffu, s1, k);
    }
    if ((threadIdx.x & 7) == 0) {
      const int hid = 32 * q + (threadIdx.x >> 3);
      pp[FH * FC + hid] = s;
      pp[FH * FC + FH + hid] = s0;
      pp[FH * FC + 2 * FH + hid] = s1;
    }
  }
  red2[threadIdx.x] = ac2;
  __syncthreads();
  if (threadIdx.x < 2) {
    float s = 0.f;
    for (int i = 0; i < 128; ++i) s += red2[threadIdx.x * 128 + i];
    pp[FH * FC + 3 * FH + threadIdx.x] = s;
  }
}

// Lifting backward, persistent: dv0 = dvp + RowI(dU0); per-CTA partials of
// grad W0 = sum_p dv0 a^T (features recomputed) and grad b0 = sum_p dv0.
constexpr int SM_LBWD = (FC * NPP + FIN * NPP) * 4 + ((RB + 2) * FN + NP + BLK) * 8 + T_ROW * 2;
__global__ void __launch_bounds__(NTH, 2) fno_lift_bwd(const float* __restrict__ dvp, const float2* __restrict__ dU,
                                                       const float2* __restrict__ f, int fps,
                                                       const float2* __restrict__ u_in,
                                                       const __nv_bfloat16* __restrict__ tabs, int B,
                                                       float* __restrict__ part) {
  extern __shared__ __align__(16) float smem[];
  float* gs = smem;                                        // [FC][NPP]
  float* as = gs + FC * NPP;                               // [FIN][NPP]
  float2* us = reinterpret_cast<float2*>(as + FIN * NPP);  // [(RB + 2) FN]
  float2* fs = us + (RB + 2) * FN;                         // [NP]
  float2* zs = fs + NP;                                    // [BLK]
  __nv_bfloat16* tb = reinterpret_cast<__nv_bfloat16*>(zs + BLK);  // [T_ROW]
  __shared__ float red[NTH / 32][4][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  cta_copy(tb, tabs, T_ROW * 2);
  float dw[4] = {0.f, 0.f, 0.f, 0.f};
  float db = 0.f;
  const int items = B * NIB;
  for (int it = blockIdx.x; it < items; it += gridDim.x) {
    const int b = it / NIB, iyb = it % NIB, iy0 = iyb * RB;
    load_planar(gs, dvp, b, (long long)iy0 * FN);
    cta_copy(zs, dU + ((long long)b * NIB + iyb) * BLK, BLK * 8);
    load_inputs(u_in, f, fps, b, iy0, us, fs);
    cp_wait_all();
    __syncthreads();
    row_inverse(zs, tb, gs, true);
    features(us, fs, iy0, as);
    __syncthreads();
    {  // grad W0 += dv0 a^T: M = FC, N = 8, K = NP split over warp quarters
      auto A = [&](int c, int p) { return gs[c * NPP + p]; };
      auto Ba = [&](int p, int k) { return as[k * NPP + p]; };
      const int mt = warp & 1, kq = warp >> 1;
#pragma unroll
      for (int ks = 0; ks < NP / 64; ++ks)
        mma3(dw, load_a(A, 16 * mt, 64 * kq + 16 * ks, g, t), load_b(Ba, 64 * kq + 16 * ks, 0, g, t));
      const int c = threadIdx.x >> 3;
      for (int p = threadIdx.x & 7; p < NP; p += 8) db += gs[c * NPP + p];
    }
    __syncthreads();
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) red[warp][e][lane] = dw[e];
  db += __shfl_xor_sync(0xffffffffu, db, 1);
  db += __shfl_xor_sync(0xffffffffu, db, 2);
  db += __shfl_xor_sync(0xffffffffu, db, 4);
  __syncthreads();
  float* pp = part + (long long)blockIdx.x * PART_0;
  if (warp < 2) {  // sum the four K quarters of tile mt = warp in a fixed order
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float s = red[warp][e][lane] + red[warp + 2][e][lane] + red[warp + 4][e][lane] + red[warp + 6][e][lane];
      pp[(16 * warp + g + (e >> 1) * 8) * FIN + 2 * t + (e & 1)] = s;
    }
  }
  if ((threadIdx.x & 7) == 0) pp[FC * FIN + (threadIdx.x >> 3)] = db;
}

// out[i] = sum_p part[p][i] in a fixed order (deterministic): a CTA takes 32 consecutive i (lanes, coalesced),
// its RED_W warps sum the partials p = w, w + RED_W, ... and warp 0 adds the RED_W sums in warp order.
constexpr int RED_W = 16;
__global__ void __launch_bounds__(32 * RED_W) fno_reduce(const float* __restrict__ part, int nparts, int count,
                                                        float* __restrict__ out) {
  __shared__ float sw[RED_W][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  float s = 0.f;
  if (i < count) {
#pragma unroll 4
    for (int p = warp; p < nparts; p += RED_W) s += part[(long long)p * count + i];
  }
  sw[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && i < count) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < RED_W; ++w) t += sw[w][lane];
    out[i] = t;
  }
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

// FP64 DFT tables as BF16 hi / lo pairs in the fragment layouts described above.
__device__ double row_entry(int ix, int kyc) {  // E(ix, kyc)
  double s, c;
  sincospi(2.0 * (((kyc >> 1) * ix) % FN) / FN, &s, &c);
  return (kyc & 1) ? -s : c;
}
__device__ double2 col_entry(int kx, int iy) {  // F(kx, iy) = exp(-2 pi j kx' iy / 128)
  const int kv = kx < FM ? kx : kx + FN - FKX;
  double s, c;
  sincospi(2.0 * ((kv * iy) % FN) / FN, &s, &c);
  return make_double2(c, -s);
}
__global__ void fno_tables(__nv_bfloat16* __restrict__ tabs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  __nv_bfloat16 *hi, *lo;
  if (i < T_RF) {  // RowF [kyc][ix]
    const int kyc = i / RFP, ix = i % RFP;
    if (ix < FN) v = row_entry(ix, kyc);
    hi = tabs + i;
    lo = tabs + T_RF + i;
  } else if (i < T_RF + T_RI) {  // RowI [ix][kyc]
    const int j = i - T_RF, ix = j / RIP, kyc = j % RIP;
    if (kyc < 2 * FM) v = row_entry(ix, kyc);
    hi = tabs + 2 * T_RF + j;
    lo = hi + T_RI;
  } else if (i < T_RF + T_RI + T_TCP) {  // tcgen05 RowI A: row ix, K = kyc
    const int j = i - (T_RF + T_RI), ix = j / (2 * FM), kyc = j % (2 * FM);
    v = row_entry(ix, kyc);
    hi = tabs + T_TROW + core_off(ix, kyc, 128, 512) / 2;
    lo = hi + T_TCP;
  } else if (i < T_RF + T_RI + 2 * T_TCP) {  // tcgen05 RowF B: row kyc, K = ix
    const int j = i - (T_RF + T_RI + T_TCP), kyc = j / FN, ix = j % FN;
    v = row_entry(ix, kyc);
    hi = tabs + T_TROW + 2 * T_TCP + core_off(kyc, ix, 128, 2048) / 2;
    lo = hi + T_TCP;
  } else if (i < T_RF + T_RI + 2 * T_TCP + T_TCF) {  // tcgen05 ColF B: row j, K = 2 iy + p
    const int e = i - (T_RF + T_RI + 2 * T_TCP), j = e / (2 * FN), k = e % (2 * FN);
    const double2 F = col_entry(j & 31, k >> 1);
    v = (j < FKX) ? ((k & 1) ? -F.y : F.x) : ((k & 1) ? F.x : F.y);
    hi = tabs + T_TCOLF + core_off(j, k, 128, 4096) / 2;
    lo = hi + T_TCF;
  } else if (i < T_RF + T_RI + 2 * T_TCP + 2 * T_TCF) {  // tcgen05 ColI B: row j = 2 iy + p, K = 2 kx + p'
    const int e = i - (T_RF + T_RI + 2 * T_TCP + T_TCF), j = e / (2 * FKX), k = e % (2 * FKX);
    const double2 F = col_entry(k >> 1, j >> 1);
    v = (j & 1) ? ((k & 1) ? F.x : -F.y) : ((k & 1) ? F.y : F.x);
    hi = tabs + T_TCOLI + core_off(j, k, 128, 1024) / 2;
    lo = hi + T_TCF;
  } else {
    return;
  }
  const __nv_bfloat16 h = __float2bfloat16_rn((float)v);
  *hi = h;
  *lo = __float2bfloat16_rn((float)(v - (double)__bfloat162float(h)));
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
    const long long off = (i - F_LAYERS) % F_LAYER;
    if (off < (long long)FMODES * FC * FC * 2) scale = 1.f / FC;
    else if (off < (long long)FMODES * FC * FC * 2 + FC * FC) scale = 0.17677670f;
  }
  pm[i] = scale * init_uniform(seed, i);
}

}  // namespace cisor

using namespace cisor;

struct cisor_fno {
  int max_batch;
  int grid_bwd;  // CTAs of the persistent backward kernels
  cudaStream_t user_stream, stream;
  cudaEvent_t ev_a, ev_b;
  float *pm, *grad, *m1, *m2, *part;
  __nv_bfloat16* wbf;
  __nv_bfloat16* tabs;  // [T_ALL] DFT tables (BF16 hi / lo)
  long long adam_t;
  // activations [max_batch, ...]
  float *v[FL + 1], *pre[FL], *dout, *dvA, *dvB, *loss;
  float2 *Xst[FL], *dYst, *T1, *Zb, *out, *fbuf, *ubuf, *tbuf, *usc;
  float2 *Xsc, *Ysc;  // column-stage intermediates [mode][B][FC]: X of an inference pass / dX, and Y
  float* h_loss;
  int* dflag;   // set by a kernel whose bounded wait on the tensor cores gave up
  int* h_flag;  // pinned copy of dflag
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

cisor_status fno_kernel_attrs() {
  CISOR_CUDA(cudaFuncSetAttribute(fno_lift_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, SM_LIFT));
  CISOR_CUDA(cudaFuncSetAttribute(fno_row_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, SM_ROW_TC));
  CISOR_CUDA(cudaFuncSetAttribute(fno_row_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, SM_ROW_TC));
  CISOR_CUDA(cudaFuncSetAttribute(fno_colf_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, SM_COLF));
  CISOR_CUDA(cudaFuncSetAttribute(fno_colf_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, SM_COLF));
  CISOR_CUDA(cudaFuncSetAttribute(fno_coli_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SM_COLI));
  CISOR_CUDA(cudaFuncSetAttribute(fno_row_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, SM_RBWD));
  CISOR_CUDA(cudaFuncSetAttribute(fno_proj_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, SM_PBWD));
  CISOR_CUDA(cudaFuncSetAttribute(fno_lift_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, SM_LBWD));
  return CISOR_OK;
}

// Forward pass on F->fbuf / F->ubuf (f_per_sample as given); train keeps pre, v_4
// and the spectra X for the backward pass.  out (may be null) receives e; x0 (may be
// null) receives the warm start u_in (1 + e) for u_in = xin.
cisor_status fno_forward_core(cisor_fno* F, int fps, int B, int train, const float2* xin, float2* x0) {
  cudaStream_t s = F->stream;
  const dim3 grow(NIB, B), gcol(FM / KY_G, B);
  const int gper = (int)((long long)B * NIB < F->grid_bwd ? (long long)B * NIB : F->grid_bwd);
  fno_lift_fwd<<<grow, NTH, SM_LIFT, s>>>(F->fbuf, fps, xin, F->wbf, F->pm, F->tabs, F->v[0], F->T1);
  CISOR_CUDA(cudaGetLastError());
  for (int l = 0; l < FL; ++l) {
    float2* X = train ? F->Xst[l] : F->Xsc;
    fno_colf_tc<0><<<gcol, NTH, SM_COLF, s>>>(F->T1, F->tabs, B, X, F->dflag);
    CISOR_CUDA(cudaGetLastError());
    fno_mix<<<FMODES, NTH, 0, s>>>(X, F->wbf, f_R(l), B, F->Ysc);
    CISOR_CUDA(cudaGetLastError());
    fno_coli_tc<<<gcol, NTH, SM_COLI, s>>>(F->Ysc, F->tabs, B, F->Zb, F->dflag);
    CISOR_CUDA(cudaGetLastError());
    const int last = l == FL - 1;
    float* pre = train ? F->pre[l] : nullptr;
    if (!last) {
      fno_row_tc<0><<<gper, NTH, SM_ROW_TC, s>>>(F->v[l], F->Zb, F->wbf, F->pm, f_W(l), f_B(l), F->tabs, 1, B, pre,
                                                 F->v[l + 1], F->T1, nullptr, nullptr, nullptr, F->dflag);
    } else {
      fno_row_tc<1><<<gper, NTH, SM_ROW_TC, s>>>(F->v[l], F->Zb, F->wbf, F->pm, f_W(l), f_B(l), F->tabs, 0, B, pre,
                                                 train ? F->v[FL] : nullptr, nullptr, F->out, xin, x0, F->dflag);
    }
    CISOR_CUDA(cudaGetLastError());
  }
  return CISOR_OK;
}

// loss and gradients (into F->grad) for targets in F->tbuf, after a training forward pass
cisor_status fno_backward_core(cisor_fno* F, int fps, int B) {
  cudaStream_t s = F->stream;
  const int G = F->grid_bwd;
  const int Gi = (int)((long long)B * NIB < G ? (long long)B * NIB : G);
  const dim3 gcol(FM / KY_G, B);
  fno_loss<<<B, 256, 0, s>>>(F->out, F->tbuf, B, F->dout, F->loss);
  CISOR_CUDA(cudaGetLastError());
  fno_proj_bwd<<<Gi, NTH, SM_PBWD, s>>>(F->v[FL], F->dout, F->wbf, F->pm, B, F->dvA, F->part);
  CISOR_CUDA(cudaGetLastError());
  fno_reduce<<<grid_of(PART_P, 32), 32 * RED_W, 0, s>>>(F->part, Gi, PART_P, F->grad + F_P1);
  CISOR_CUDA(cudaGetLastError());
  float* dv = F->dvA;
  float* dvn = F->dvB;
  for (int l = FL - 1; l >= 0; --l) {
    fno_row_bwd<<<Gi, NTH, SM_RBWD, s>>>(dv, l == FL - 1 ? nullptr : F->Zb, F->pre[l], F->v[l], F->wbf, f_W(l),
                                         F->tabs, B, l < FL - 1, dvn, F->T1, F->part);
    CISOR_CUDA(cudaGetLastError());
    fno_reduce<<<grid_of(PART_W, 32), 32 * RED_W, 0, s>>>(F->part, Gi, PART_W, F->grad + f_W(l));
    CISOR_CUDA(cudaGetLastError());
    fno_colf_tc<1><<<gcol, NTH, SM_COLF, s>>>(F->T1, F->tabs, B, F->dYst, F->dflag);
    CISOR_CUDA(cudaGetLastError());
    fno_mix_bwd<<<FMODES, NTH, 0, s>>>(F->Xst[l], F->dYst, F->wbf, f_R(l), B, F->Xsc, F->grad + f_R(l));
    CISOR_CUDA(cudaGetLastError());
    fno_coli_tc<<<gcol, NTH, SM_COLI, s>>>(F->Xsc, F->tabs, B, F->Zb, F->dflag);
    CISOR_CUDA(cudaGetLastError());
    float* tmp = dv;
    dv = dvn;
    dvn = tmp;
  }
  fno_lift_bwd<<<Gi, NTH, SM_LBWD, s>>>(dv, F->Zb, F->fbuf, fps, F->ubuf, F->tabs, B, F->part);
  CISOR_CUDA(cudaGetLastError());
  fno_reduce<<<grid_of(PART_0, 32), 32 * RED_W, 0, s>>>(F->part, Gi, PART_0, F->grad + F_W0);
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

// waits for the FNO stream; an error if a tensor-core wait timed out in the work it ran (the flag is reset)
cisor_status fno_sync(cisor_fno* F) {
  CISOR_CUDA(cudaMemcpyAsync(F->h_flag, F->dflag, sizeof(int), cudaMemcpyDeviceToHost, F->stream));
  CISOR_CUDA(cudaStreamSynchronize(F->stream));
  if (*F->h_flag) {
    CISOR_CUDA(cudaMemsetAsync(F->dflag, 0, sizeof(int), F->stream));
    CISOR_CUDA(cudaStreamSynchronize(F->stream));
    set_error("FNO: a wait on the tensor cores timed out; the outputs of this call are invalid");
    return CISOR_ERR_CUDA;
  }
  return CISOR_OK;
}

cisor_status mean_loss(cisor_fno* F, int B, double* loss) {
  CISOR_CUDA(cudaMemcpyAsync(F->h_loss, F->loss, sizeof(float) * B, cudaMemcpyDeviceToHost, F->stream));
  CISOR_TRY(fno_sync(F));
  double s = 0.0;
  for (int b = 0; b < B; ++b) s += F->h_loss[b];
  if (loss) *loss = s / B;
  return CISOR_OK;
}

void fno_free(cisor_fno* F) {
  if (!F) return;
  if (F->stream) cudaStreamSynchronize(F->stream);
  void* d[] = {F->pm,  F->grad, F->m1,   F->m2,  F->part, F->wbf,  F->tabs, F->dout, F->dvA,
               F->dvB, F->loss, F->dYst, F->T1,  F->Zb,   F->out,  F->fbuf, F->ubuf, F->tbuf, F->usc,
               F->Xsc, F->Ysc};
  for (void* p : d)
    if (p) cudaFree(p);
  for (int l = 0; l <= FL; ++l)
    if (F->v[l]) cudaFree(F->v[l]);
  for (int l = 0; l < FL; ++l) {
    if (F->pre[l]) cudaFree(F->pre[l]);
    if (F->Xst[l]) cudaFree(F->Xst[l]);
  }
  if (F->h_loss) cudaFreeHost(F->h_loss);
  if (F->h_flag) cudaFreeHost(F->h_flag);
  if (F->dflag) cudaFree(F->dflag);
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
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail(e, "device query");
  F->grid_bwd = 2 * sms;
  e = cudaStreamCreateWithFlags(&F->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&F->ev_a, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&F->ev_b, cudaEventDisableTiming);
  if (e != cudaSuccess) return fail(e, "FNO stream/events");
  const size_t act = sizeof(float) * (size_t)max_batch * FC * FNN;
  const size_t spec = sizeof(float2) * (size_t)max_batch * NIB * BLK;
  const size_t md = sizeof(float2) * (size_t)max_batch * FC * FMODES;
  const size_t fld = sizeof(float2) * (size_t)max_batch * FNN;
  struct A {
    void** p;
    size_t n;
  } allocs[] = {{(void**)&F->pm, sizeof(float) * F_TOTAL},
                {(void**)&F->grad, sizeof(float) * F_TOTAL},
                {(void**)&F->m1, sizeof(float) * F_TOTAL},
                {(void**)&F->m2, sizeof(float) * F_TOTAL},
                {(void**)&F->part, sizeof(float) * (size_t)F->grid_bwd * PART_MAX},
                {(void**)&F->wbf, sizeof(__nv_bfloat16) * F_TOTAL},
                {(void**)&F->tabs, sizeof(__nv_bfloat16) * T_ALL},
                {(void**)&F->dout, sizeof(float) * (size_t)max_batch * 2 * FNN},
                {(void**)&F->dvA, act},
                {(void**)&F->dvB, act},
                {(void**)&F->loss, sizeof(float) * max_batch},
                {(void**)&F->dYst, md},
                {(void**)&F->Xsc, md},
                {(void**)&F->Ysc, md},
                {(void**)&F->T1, spec},
                {(void**)&F->Zb, spec},
                {(void**)&F->out, fld},
                {(void**)&F->fbuf, fld},
                {(void**)&F->ubuf, fld},
                {(void**)&F->tbuf, fld},
                {(void**)&F->usc, fld},
                {(void**)&F->dflag, sizeof(int)}};
  for (auto& a : allocs) {
    e = cudaMalloc(a.p, a.n);
    if (e != cudaSuccess) return fail(e, "FNO cudaMalloc");
  }
  for (int l = 0; l <= FL && e == cudaSuccess; ++l) e = cudaMalloc((void**)&F->v[l], act);
  for (int l = 0; l < FL && e == cudaSuccess; ++l) {
    e = cudaMalloc((void**)&F->pre[l], act);
    if (e == cudaSuccess) e = cudaMalloc((void**)&F->Xst[l], md);
  }
  if (e == cudaSuccess) e = cudaMallocHost((void**)&F->h_loss, sizeof(float) * max_batch);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&F->h_flag, sizeof(int));
  if (e != cudaSuccess) return fail(e, "FNO cudaMalloc");
  cisor_status st = fno_kernel_attrs();
  if (st != CISOR_OK) {
    fno_free(F);
    return st;
  }
  fno_init<<<grid_of(F_TOTAL, 256), 256, 0, F->stream>>>(F->pm, F_TOTAL, seed);
  fno_to_bf16<<<grid_of(F_TOTAL, 256), 256, 0, F->stream>>>(F->pm, F->wbf, F_TOTAL);
  fno_tables<<<grid_of(T_RF + T_RI + 2 * T_TCP + 2 * T_TCF, 256), 256, 0, F->stream>>>(F->tabs);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemsetAsync(F->m1, 0, sizeof(float) * F_TOTAL, F->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(F->m2, 0, sizeof(float) * F_TOTAL, F->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(F->dflag, 0, sizeof(int), F->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(F->stream);
  if (e != cudaSuccess) return fail(e, "FNO init");
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
  CISOR_TRY(fno_forward_core(F, f_per_sample, B, 0, F->ubuf, nullptr));
  CISOR_CUDA(cudaMemcpyAsync(u_sc_out, F->out, sizeof(float2) * (size_t)B * FNN, cudaMemcpyDefault, F->stream));
  CISOR_TRY(fno_sync(F));
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
  CISOR_TRY(fno_forward_core(F, f_per_sample, B, 1, F->ubuf, nullptr));
  CISOR_TRY(fno_backward_core(F, f_per_sample, B));
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
  CISOR_TRY(fno_forward_core(F, f_per_sample, B, 1, F->ubuf, nullptr));
  CISOR_TRY(fno_backward_core(F, f_per_sample, B));
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
  if (c->dim != 2 || c->n != FN || c->ncomp != 1 || c->T > F->max_batch) {
    set_error("cisor_fno_warm_start: the network is for scalar 128 x 128 grids and at most %d transmitters",
              F->max_batch);
    return CISOR_ERR_INVALID_ARG;
  }
  const int B = c->T;
  CISOR_TRY(fno_enter(F));
  CISOR_CUDA(cudaMemcpyAsync(F->fbuf, f, sizeof(float2) * FNN, cudaMemcpyDefault, F->stream));
  CISOR_CUDA(cudaStreamWaitEvent(F->stream, c->ev_b, 0));  // the context's incident fields are ready
  CISOR_TRY(fno_forward_core(F, 0, B, 0, c->u_in, F->usc));
  CISOR_CUDA(cudaMemcpyAsync(x0_out, F->usc, sizeof(float2) * (size_t)B * FNN, cudaMemcpyDefault, F->stream));
  CISOR_TRY(fno_sync(F));
  return fno_leave(F);
}

}  // extern "C"
