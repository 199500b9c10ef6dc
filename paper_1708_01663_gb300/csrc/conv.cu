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
#include "regfft.cuh"

namespace cisor {

template <int P> struct ConvCfg {
  static constexpr int NTF = P / 8;         // threads per P-point transform
  static constexpr int RB = 256 / NTF;      // rows per CTA, row passes (256 threads)
  static constexpr int PP = P + P / 16;     // padded row pitch in shared memory
  template <int NT> struct Col { static constexpr int W = NT / NTF; };  // columns per CTA, column pass
};

int conv_rows_per_block(int P) { return 2048 / P; }

template <int P, int PRO>
__global__ void __launch_bounds__(256) conv_rows_fwd(const ConvOp op, const float2* __restrict__ tw_g,
                                                     float2* __restrict__ R, int n) {
  typedef ConvCfg<P> C;
  typedef RPlan<P> PL;
  __shared__ float2 tw[TwTable<P, false>::SIZE];
  __shared__ float2 buf[C::RB * C::PP];
  const int tx = blockIdx.y;
  if (op.active && !op.active[tx]) return;
  const int lt = threadIdx.x % C::NTF, row = threadIdx.x / C::NTF;
  const int iy = blockIdx.x * C::RB + row;
  const bool rowok = iy < n;
  const long long N = (long long)n * n;
  for (int i = threadIdx.x; i < TwTable<P, false>::SIZE; i += 256) tw[i] = tw_g[i];
  float2 alpha = make_float2(0.f, 0.f), beta = alpha, omega = alpha;
  if (PRO != PRO_COPY) {
    const double2* sc = reinterpret_cast<const double2*>(op.scal) + (size_t)tx * SC_STRIDE;
    alpha = z_to_c(sc[SC_ALPHA]);
    beta = z_to_c(sc[SC_BETA]);
    omega = z_to_c(sc[SC_OMEGA]);
  }
  const bool mulf = op.mul_f && !op.adjoint;
  const bool fresh = (beta.x == 0.f && beta.y == 0.f);  // beta = 0 starts (or restarts) with p = r
  constexpr int R0 = PL::template first<false>();
  float2 v[8];
#pragma unroll
  for (int q = 0; q < 8 / R0; ++q)
#pragma unroll
    for (int r = 0; r < R0; ++r) {
      const int ix = PL::elem(lt, q, r, R0);
      float2 val = make_float2(0.f, 0.f);
      if (rowok && ix < n) {
        const long long pix = (long long)iy * n + ix;
        const long long idx = tx * N + pix;
        if (PRO == PRO_COPY) {
          val = op.src[idx];
        } else if (PRO == PRO_PUPDATE) {
          const float2 rv = op.src[idx];
          float2 p = rv;
          if (!fresh) p = c_add(rv, c_mul(beta, c_sub(op.pvec[idx], c_mul(omega, op.vvec[idx]))));
          op.pvec[idx] = p;
          val = p;
        } else {  // PRO_AXPY
          const float2 s = c_sub(op.src[idx], c_mul(alpha, op.vvec[idx]));
          op.svec[idx] = s;
          val = s;
        }
        if (mulf) val = c_mul(val, op.f[pix]);
      }
      v[q * R0 + r] = val;
    }
  reg_fft<P, false, false>(v, buf, RowLayA{row * C::PP}, RowLayB{row * C::PP}, lt, tw);
  if (!rowok) return;
  constexpr int RL = PL::template last<false>();
  float2* dst = R + ((long long)tx * n + iy) * P;
#pragma unroll
  for (int q = 0; q < 8 / RL; ++q)
#pragma unroll
    for (int r = 0; r < RL; ++r) dst[PL::elem(lt, q, r, RL)] = v[q * RL + r];
}

template <int P, bool ADJ, int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) conv_cols(const int* __restrict__ active, const float2* __restrict__ tw_g,
                                                    const float2* __restrict__ ghat, float2* __restrict__ R, int n) {
  typedef ConvCfg<P> C;
  typedef RPlan<P> PL;
  __shared__ float2 tw[TwTable<P, false>::SIZE];
  __shared__ float2 twr[TwTable<P, true>::SIZE];
  constexpr int W = C::template Col<NT>::W;
  __shared__ float2 buf[P * W];
  const int tx = blockIdx.y;
  if (active && !active[tx]) return;
  const int w = threadIdx.x % W, lt = threadIdx.x / W;
  const int c0 = blockIdx.x * W;
  for (int i = threadIdx.x; i < TwTable<P, false>::SIZE; i += NT) tw[i] = tw_g[i];
  for (int i = threadIdx.x; i < TwTable<P, true>::SIZE; i += NT) twr[i] = tw_g[TW_STRIDE + i];
  float2* base = R + (long long)tx * n * P + c0 + w;
  constexpr int R0 = PL::template first<false>();
  float2 v[8];
#pragma unroll
  for (int q = 0; q < 8 / R0; ++q)
#pragma unroll
    for (int r = 0; r < R0; ++r) {
      const int i = PL::elem(lt, q, r, R0);
      v[q * R0 + r] = (i < n) ? base[(long long)i * P] : make_float2(0.f, 0.f);
    }
  const ColLay<W> lay{w};
  reg_fft<P, false, false>(v, buf, lay, lay, lt, tw);
  // spectrum product in registers: forward outputs are the inverse (reversed plan) inputs
  constexpr int RL = PL::template last<false>();
#pragma unroll
  for (int q = 0; q < 8 / RL; ++q)
#pragma unroll
    for (int r = 0; r < RL; ++r) {
      const int ky = PL::elem(lt, q, r, RL);
      float2 g = __ldg(ghat + (long long)ky * P + c0 + w);
      if (ADJ) g.y = -g.y;
      v[q * RL + r] = c_mul(v[q * RL + r], g);
    }
  reg_fft<P, true, true>(v, buf, lay, lay, lt, twr);
  constexpr int RI = PL::template last<true>();
#pragma unroll
  for (int q = 0; q < 8 / RI; ++q)
#pragma unroll
    for (int r = 0; r < RI; ++r) {
      const int i = PL::elem(lt, q, r, RI);
      if (i < n) base[(long long)i * P] = v[q * RI + r];
    }
}

__device__ __forceinline__ float2 pick(int code, float2 y, float2 s, float2 a) {
  return code == OP_Y ? y : (code == OP_SRC ? s : a);
}

// Block-wide sum of three complex FP32 partials: warp shuffles, then the
// per-warp sums pairwise in shared memory (all FP32), written to part.
template <int NT>
__device__ __forceinline__ void block_dots(const float2 acc[DOT_SLOTS], float2* out) {
  __shared__ float red[2 * DOT_SLOTS][NT / 32];
  float v[2 * DOT_SLOTS];
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
    for (int k = 0; k < 2 * DOT_SLOTS; ++k) red[k][wid] = v[k];
  }
  __syncthreads();
  if (threadIdx.x < 2 * DOT_SLOTS) {
    float* r = red[threadIdx.x];
#pragma unroll
    for (int w = NT / 64; w > 0; w >>= 1)
#pragma unroll
      for (int i = 0; i < w; ++i) r[i] += r[i + w];
    reinterpret_cast<float*>(out)[threadIdx.x] = r[0];
  }
}

template <int P, int EPI>
__global__ void __launch_bounds__(256) conv_rows_inv(const ConvOp op, const float2* __restrict__ tw_g,
                                                     const float2* __restrict__ R, int n, int nblk) {
  typedef ConvCfg<P> C;
  typedef RPlan<P> PL;
  __shared__ float2 tw[TwTable<P, true>::SIZE];
  __shared__ float2 buf[C::RB * C::PP];
  const int tx = blockIdx.y;
  if (op.active && !op.active[tx]) return;
  const int lt = threadIdx.x % C::NTF, row = threadIdx.x / C::NTF;
  const int iy = blockIdx.x * C::RB + row;
  const bool rowok = iy < n;
  const long long N = (long long)n * n;
  for (int i = threadIdx.x; i < TwTable<P, true>::SIZE; i += 256) tw[i] = tw_g[TW_STRIDE + i];
  constexpr int R0 = PL::template first<true>();
  const float2* srow = R + ((long long)tx * n + (rowok ? iy : 0)) * P;
  float2 v[8];
#pragma unroll
  for (int q = 0; q < 8 / R0; ++q)
#pragma unroll
    for (int r = 0; r < R0; ++r) v[q * R0 + r] = rowok ? srow[PL::elem(lt, q, r, R0)] : make_float2(0.f, 0.f);
  const bool postf = op.mul_f && op.adjoint;
  const bool any_dot = (op.dot_a[0] | op.dot_a[1] | op.dot_a[2]) != 0;
  const bool aux0 = EPI == EPI_MATVEC && (op.dot_a[0] == OP_AUX || op.dot_b[0] == OP_AUX);
  const bool need_aux = EPI == EPI_RESID || aux0 || (EPI == EPI_CONV_ADD && op.aux);
  constexpr int RL = PL::template last<true>();
  // epilogue operands are loaded before the transform so their latency overlaps it
  float2 pre_src[8], pre_aux[8];
#pragma unroll
  for (int q = 0; q < 8 / RL; ++q)
#pragma unroll
    for (int r = 0; r < RL; ++r) {
      const int ix = PL::elem(lt, q, r, RL);
      const bool ok = rowok && ix < n;
      const long long idx = tx * N + (long long)(rowok ? iy : 0) * n + (ix < n ? ix : 0);
      pre_src[q * RL + r] = (ok && EPI != EPI_CONV_ADD) ? op.esrc[idx] : make_float2(0.f, 0.f);
      pre_aux[q * RL + r] = (ok && need_aux) ? op.aux[idx] : make_float2(0.f, 0.f);
    }
  reg_fft<P, true, true>(v, buf, RowLayA{row * C::PP}, RowLayB{row * C::PP}, lt, tw);
  float2 acc[DOT_SLOTS];
#pragma unroll
  for (int s = 0; s < DOT_SLOTS; ++s) acc[s] = make_float2(0.f, 0.f);
  if (rowok) {
#pragma unroll
    for (int q = 0; q < 8 / RL; ++q)
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        const int ix = PL::elem(lt, q, r, RL);
        if (ix >= n) continue;
        const long long pix = (long long)iy * n + ix;
        const long long idx = tx * N + pix;
        float2 c = v[q * RL + r];
        if (postf) c = c_cjmul(op.f[pix], c);
        const float2 src = pre_src[q * RL + r], aux = pre_aux[q * RL + r];
        float2 y;
        if (EPI == EPI_MATVEC) {
          y = c_sub(src, c);
        } else if (EPI == EPI_RESID) {
          y = c_sub(aux, c_sub(src, c));
        } else {
          y = c_add(c, aux);
        }
        op.out[idx] = y;
        if (op.out2) op.out2[idx] = y;
        if (any_dot) {
#pragma unroll
          for (int s = 0; s < DOT_SLOTS; ++s) {
            if (op.dot_a[s]) {
              const float2 a = pick(op.dot_a[s], y, src, aux), b = pick(op.dot_b[s], y, src, aux);
              acc[s] = c_add(acc[s], c_cjmul(a, b));
            }
          }
        }
      }
  }
  if (any_dot) block_dots<256>(acc, reinterpret_cast<float2*>(op.part) + ((size_t)tx * nblk + blockIdx.x) * DOT_SLOTS);
}

template <int P>
static cisor_status conv_pass_t(cisor_ctx* c, const ConvOp& op) {
  typedef ConvCfg<P> C;
  const int n = c->n;
  dim3 grow((n + C::RB - 1) / C::RB, op.ntx);
  switch (op.prologue) {
    case PRO_COPY: conv_rows_fwd<P, PRO_COPY><<<grow, 256, 0, c->stream>>>(op, c->twst, c->R, n); break;
    case PRO_PUPDATE: conv_rows_fwd<P, PRO_PUPDATE><<<grow, 256, 0, c->stream>>>(op, c->twst, c->R, n); break;
    default: conv_rows_fwd<P, PRO_AXPY><<<grow, 256, 0, c->stream>>>(op, c->twst, c->R, n); break;
  }
  CISOR_CUDA(cudaGetLastError());
  if (c->cols_nt == 256) {
    dim3 gcol(P / C::template Col<256>::W, op.ntx);
    if (op.adjoint)
      conv_cols<P, true, 256><<<gcol, 256, 0, c->stream>>>(op.active, c->twst, c->ghat, c->R, n);
    else
      conv_cols<P, false, 256><<<gcol, 256, 0, c->stream>>>(op.active, c->twst, c->ghat, c->R, n);
  } else {
    dim3 gcol(P / C::template Col<512>::W, op.ntx);
    if (op.adjoint)
      conv_cols<P, true, 512><<<gcol, 512, 0, c->stream>>>(op.active, c->twst, c->ghat, c->R, n);
    else
      conv_cols<P, false, 512><<<gcol, 512, 0, c->stream>>>(op.active, c->twst, c->ghat, c->R, n);
  }
  CISOR_CUDA(cudaGetLastError());
  switch (op.epilogue) {
    case EPI_MATVEC: conv_rows_inv<P, EPI_MATVEC><<<grow, 256, 0, c->stream>>>(op, c->twst, c->R, n, c->nblk); break;
    case EPI_RESID: conv_rows_inv<P, EPI_RESID><<<grow, 256, 0, c->stream>>>(op, c->twst, c->R, n, c->nblk); break;
    default: conv_rows_inv<P, EPI_CONV_ADD><<<grow, 256, 0, c->stream>>>(op, c->twst, c->R, n, c->nblk); break;
  }
  CISOR_CUDA(cudaGetLastError());
  c->launches += 3;
  return CISOR_OK;
}

template <int P>
static cisor_status conv_init_t() {
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
