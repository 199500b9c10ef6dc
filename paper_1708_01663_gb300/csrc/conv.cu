// Batched FFT convolution with G and G^H (Sec. II, Eqs. 3-4; FFT evaluation
// of the convolution, Sec. III-A), fused with the vector work of the Krylov
// solver.  One pass over `ntx` transmitters is three kernels:
//
//  1. rows_fwd : prologue (copy / p = r + beta (p - omega v) / s = r - alpha v,
//                written back), times f for A; zero-pad each row to P; FFT
//                along x; store the n non-zero rows of the padded image
//                into R [T, n, P].  Rows n..P-1 of the padded image are zero
//                and never touched (pruned).
//  2. cols     : for a block of W columns: load the n rows, zero-pad to P,
//                FFT along y, multiply by ghat (or conj(ghat) for G^H, since
//                G is symmetric and G^H = conj(G)), inverse FFT along y, keep
//                the first n rows, store in place.
//  3. rows_inv : inverse FFT along x, keep the first n columns (crop), then
//                the epilogue: A x = x - G(f x), A^H x = x - conj(f) G^H x,
//                the residual b - A x, or G^H v + z; plus up to three
//                per-transmitter inner products, summed per thread in FP32
//                and across the block in FP64.
// ghat is pre-scaled by 1/P^2, so the inverse transforms are unnormalised.
#include "common.cuh"
#include "fft.cuh"

namespace cisor {

template <int P> struct ConvCfg {
  static constexpr int RB = (2048 / P) < 1 ? 1 : 2048 / P;  // rows per CTA, row passes
  static constexpr int W = 8;                               // columns per CTA, column pass
  static constexpr int NT = 256;
};

int conv_rows_per_block(int P) { return (2048 / P) < 1 ? 1 : 2048 / P; }

template <int P, int PRO>
__global__ void __launch_bounds__(256) conv_rows_fwd(const ConvOp op, const float2* __restrict__ tw_g,
                                                     float2* __restrict__ R, int n) {
  constexpr int RB = ConvCfg<P>::RB, NT = ConvCfg<P>::NT;
  __shared__ float2 tw[P];
  __shared__ float2 bufA[RB * P];
  __shared__ float2 bufB[RB * P];
  const int t = blockIdx.y;
  if (op.active && !op.active[t]) return;
  const int tid = threadIdx.x;
  const int row0 = blockIdx.x * RB;
  const long long N = (long long)n * n;
  for (int i = tid; i < P; i += NT) tw[i] = tw_g[i];
  float2 alpha = make_float2(0.f, 0.f), beta = alpha, omega = alpha;
  if (PRO != PRO_COPY) {
    const double2* sc = reinterpret_cast<const double2*>(op.scal) + (size_t)t * SC_STRIDE;
    alpha = z_to_c(sc[SC_ALPHA]);
    beta = z_to_c(sc[SC_BETA]);
    omega = z_to_c(sc[SC_OMEGA]);
  }
  const bool mulf = op.mul_f && !op.adjoint;
  for (int e = tid; e < RB * P; e += NT) {
    const int row = e / P, ix = e % P;
    const int iy = row0 + row;
    float2 q = make_float2(0.f, 0.f);
    if (ix < n && iy < n) {
      const long long idx = t * N + (long long)iy * n + ix;
      if (PRO == PRO_COPY) {
        q = op.src[idx];
      } else if (PRO == PRO_PUPDATE) {
        float2 r = op.src[idx], p = r;
        if (beta.x != 0.f || beta.y != 0.f) {  // beta = 0 starts (or restarts) with p = r
          const float2 pold = op.pvec[idx], v = op.vvec[idx];
          p = c_add(r, c_mul(beta, c_sub(pold, c_mul(omega, v))));
        }
        op.pvec[idx] = p;
        q = p;
      } else {  // PRO_AXPY
        float2 r = op.src[idx], v = op.vvec[idx];
        float2 s = c_sub(r, c_mul(alpha, v));
        op.svec[idx] = s;
        q = s;
      }
      if (mulf) q = c_mul(q, op.f[(long long)iy * n + ix]);
    }
    bufA[e] = q;
  }
  __syncthreads();
  const float2* res = block_fft<P, false, false>(bufA, bufB, RB, P, 1, tw, tid, NT);
  for (int e = tid; e < RB * P; e += NT) {
    const int row = e / P, ix = e % P;
    const int iy = row0 + row;
    if (iy < n) R[((long long)t * n + iy) * P + ix] = res[e];
  }
}

template <int P, bool ADJ>
__global__ void __launch_bounds__(256) conv_cols(const int* __restrict__ active, const float2* __restrict__ tw_g,
                                                 const float2* __restrict__ ghat, float2* __restrict__ R, int n) {
  constexpr int W = ConvCfg<P>::W, NT = ConvCfg<P>::NT;
  extern __shared__ float2 smc[];
  float2* tw = smc;
  float2* A = tw + P;
  float2* B = A + P * W;
  const int t = blockIdx.y;
  if (active && !active[t]) return;
  const int tid = threadIdx.x;
  const int c0 = blockIdx.x * W;
  for (int i = tid; i < P; i += NT) tw[i] = tw_g[i];
  float2* base = R + (long long)t * n * P + c0;
  for (int e = tid; e < P * W; e += NT) {
    const int i = e / W, w = e % W;
    A[e] = (i < n) ? base[(long long)i * P + w] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  float2* res = block_fft<P, false, true>(A, B, W, 1, W, tw, tid, NT);
  float2* other = (res == A) ? B : A;
  for (int e = tid; e < P * W; e += NT) {
    const int i = e / W, w = e % W;
    float2 g = ghat[(long long)i * P + c0 + w];
    if (ADJ) g.y = -g.y;
    res[e] = c_mul(res[e], g);
  }
  __syncthreads();
  const float2* res2 = block_fft<P, true, true>(res, other, W, 1, W, tw, tid, NT);
  for (int e = tid; e < n * W; e += NT) {
    const int i = e / W, w = e % W;
    base[(long long)i * P + w] = res2[e];
  }
}

__device__ __forceinline__ float2 pick(int code, float2 y, float2 s, float2 a) {
  return code == OP_Y ? y : (code == OP_SRC ? s : a);
}

// Block-wide sum of three complex FP32 partials into FP64, written to part.
template <int NT>
__device__ __forceinline__ void block_dots(const float2 acc[DOT_SLOTS], double2* out) {
  __shared__ double red[NT / 32][2 * DOT_SLOTS];
  double v[2 * DOT_SLOTS];
#pragma unroll
  for (int s = 0; s < DOT_SLOTS; ++s) {
    v[2 * s] = acc[s].x;
    v[2 * s + 1] = acc[s].y;
  }
#pragma unroll
  for (int k = 0; k < 2 * DOT_SLOTS; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 2 * DOT_SLOTS; ++k) red[wid][k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x < 2 * DOT_SLOTS) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) s += red[w][threadIdx.x];
    reinterpret_cast<double*>(out)[threadIdx.x] = s;
  }
}

template <int P, int EPI>
__global__ void __launch_bounds__(256) conv_rows_inv(const ConvOp op, const float2* __restrict__ tw_g,
                                                     const float2* __restrict__ R, int n, int nblk) {
  constexpr int RB = ConvCfg<P>::RB, NT = ConvCfg<P>::NT;
  __shared__ float2 tw[P];
  __shared__ float2 bufA[RB * P];
  __shared__ float2 bufB[RB * P];
  const int t = blockIdx.y;
  if (op.active && !op.active[t]) return;
  const int tid = threadIdx.x;
  const int row0 = blockIdx.x * RB;
  const long long N = (long long)n * n;
  for (int i = tid; i < P; i += NT) tw[i] = tw_g[i];
  for (int e = tid; e < RB * P; e += NT) {
    const int row = e / P, ix = e % P;
    const int iy = row0 + row;
    bufA[e] = (iy < n) ? R[((long long)t * n + iy) * P + ix] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const float2* res = block_fft<P, true, false>(bufA, bufB, RB, P, 1, tw, tid, NT);
  const bool postf = op.mul_f && op.adjoint;
  const bool any_dot = (op.dot_a[0] | op.dot_a[1] | op.dot_a[2]) != 0;
  float2 acc[DOT_SLOTS];
#pragma unroll
  for (int s = 0; s < DOT_SLOTS; ++s) acc[s] = make_float2(0.f, 0.f);
  for (int e = tid; e < RB * n; e += NT) {
    const int row = e / n, ix = e % n;
    const int iy = row0 + row;
    if (iy >= n) continue;
    const long long pix = (long long)iy * n + ix;
    const long long idx = t * N + pix;
    float2 c = res[row * P + ix];
    if (postf) c = c_cjmul(op.f[pix], c);
    float2 src = make_float2(0.f, 0.f), aux = src, y;
    if (EPI == EPI_MATVEC) {
      src = op.esrc[idx];
      y = c_sub(src, c);
    } else if (EPI == EPI_RESID) {
      src = op.esrc[idx];
      aux = op.aux[idx];
      y = c_sub(aux, c_sub(src, c));
    } else {
      if (op.aux) aux = op.aux[idx];
      y = c_add(c, aux);
    }
    op.out[idx] = y;
    if (op.out2) op.out2[idx] = y;
    if (any_dot) {
      if (EPI == EPI_MATVEC && (op.dot_a[0] == OP_AUX || op.dot_b[0] == OP_AUX)) aux = op.aux[idx];
#pragma unroll
      for (int s = 0; s < DOT_SLOTS; ++s) {
        if (op.dot_a[s]) {
          float2 a = pick(op.dot_a[s], y, src, aux), b = pick(op.dot_b[s], y, src, aux);
          acc[s] = c_add(acc[s], c_cjmul(a, b));
        }
      }
    }
  }
  if (any_dot) block_dots<NT>(acc, reinterpret_cast<double2*>(op.part) + ((size_t)t * nblk + blockIdx.x) * DOT_SLOTS);
}

template <int P>
static cisor_status conv_pass_t(cisor_ctx* c, const ConvOp& op) {
  constexpr int RB = ConvCfg<P>::RB, W = ConvCfg<P>::W, NT = ConvCfg<P>::NT;
  const int n = c->n;
  dim3 grow((n + RB - 1) / RB, op.ntx);
  dim3 gcol(P / W, op.ntx);
  switch (op.prologue) {
    case PRO_COPY: conv_rows_fwd<P, PRO_COPY><<<grow, NT, 0, c->stream>>>(op, c->tw, c->R, n); break;
    case PRO_PUPDATE: conv_rows_fwd<P, PRO_PUPDATE><<<grow, NT, 0, c->stream>>>(op, c->tw, c->R, n); break;
    default: conv_rows_fwd<P, PRO_AXPY><<<grow, NT, 0, c->stream>>>(op, c->tw, c->R, n); break;
  }
  CISOR_CUDA(cudaGetLastError());
  const size_t smc = (size_t)(P + 2 * P * W) * sizeof(float2);
  if (op.adjoint)
    conv_cols<P, true><<<gcol, NT, smc, c->stream>>>(op.active, c->tw, c->ghat, c->R, n);
  else
    conv_cols<P, false><<<gcol, NT, smc, c->stream>>>(op.active, c->tw, c->ghat, c->R, n);
  CISOR_CUDA(cudaGetLastError());
  switch (op.epilogue) {
    case EPI_MATVEC: conv_rows_inv<P, EPI_MATVEC><<<grow, NT, 0, c->stream>>>(op, c->tw, c->R, n, c->nblk); break;
    case EPI_RESID: conv_rows_inv<P, EPI_RESID><<<grow, NT, 0, c->stream>>>(op, c->tw, c->R, n, c->nblk); break;
    default: conv_rows_inv<P, EPI_CONV_ADD><<<grow, NT, 0, c->stream>>>(op, c->tw, c->R, n, c->nblk); break;
  }
  CISOR_CUDA(cudaGetLastError());
  c->launches += 3;
  return CISOR_OK;
}

template <int P>
static cisor_status conv_init_t() {
  constexpr int W = ConvCfg<P>::W;
  const int smc = (P + 2 * P * W) * (int)sizeof(float2);
  CISOR_CUDA(cudaFuncSetAttribute(conv_cols<P, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smc));
  CISOR_CUDA(cudaFuncSetAttribute(conv_cols<P, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smc));
  return CISOR_OK;
}

cisor_status conv_init(int P) {
  switch (P) {
    case 64: return conv_init_t<64>();
    case 128: return conv_init_t<128>();
    case 256: return conv_init_t<256>();
    case 512: return conv_init_t<512>();
  }
  set_error("unsupported FFT size %d", P);
  return CISOR_ERR_INVALID_ARG;
}

cisor_status conv_pass(cisor_ctx* c, const ConvOp& op) {
  switch (c->P) {
    case 64: return conv_pass_t<64>(c, op);
    case 128: return conv_pass_t<128>(c, op);
    case 256: return conv_pass_t<256>(c, op);
    case 512: return conv_pass_t<512>(c, op);
  }
  set_error("unsupported FFT size %d", c->P);
  return CISOR_ERR_INVALID_ARG;
}

}  // namespace cisor
