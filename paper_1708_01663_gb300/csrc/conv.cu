// Batched FFT convolution with G and G^H (Sec. II, Eqs. 3-4; FFT evaluation
// of the convolution, Sec. III-A), fused with the vector work of the Krylov
// solver.  One 2D pass over `ntx` transmitters is three kernels:
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
//                per-transmitter inner products (FP32 trees).
// A 3D pass (R is [T, n, P, P]: the n non-zero z slabs of the padded volume)
// is five kernels: rows_fwd over the n^2 x rows; cols in forward-only mode
// along y (n inputs, P outputs per column, in each z slab); cols with the
// spectrum product along z (stride P^2; n of the P z planes kept); cols in
// inverse-only mode along y (P inputs, n kept); rows_inv.
// ghat is pre-scaled by 1/P^d, so the inverse transforms are unnormalised.
#include "common.cuh"
#include "dots.cuh"
#include "fft.cuh"
#include "regfft.cuh"

namespace cisor {

template <int P> struct ConvCfg {
  static constexpr int NTF = P / 8;         // threads per P-point transform
  static constexpr int RB = 256 / NTF;      // rows per CTA, row passes (256 threads)
  static constexpr int PP = row_pitch(P);   // padded row pitch in shared memory
  template <int NT> struct Col { static constexpr int W = NT / NTF; };  // columns per CTA, column pass
};

int conv_rows_per_block(int P) { return 2048 / P; }

void conv_geometry(cisor_ctx* c) {
  const int n = c->n, P = c->P;
  c->nrows = c->dim == 3 ? n * n : n;
  c->rslab = c->dim == 3 ? (long long)P * P : (long long)n * P;
  c->rtstride = conv_scratch_elems(c->dim, n, P);
  const int RB = conv_rows_per_block(P);
  c->nblk = (c->nrows + RB - 1) / RB;
}

long long conv_scratch_elems(int dim, int n, int P) {
  return dim == 3 ? (long long)n * P * P : (long long)n * P;
}

int conv_kernels_per_pass(int dim) { return dim == 3 ? 5 : 3; }

// x rows of a field: row q (q < nrows) holds pixels q*n .. q*n + n - 1 and
// its transform is row  tx * tstride + (q / n) * slab + (q % n) * P  of R.
struct RowGeo {
  int n, nrows;
  long long slab, tstride;
};
template <int P>
__device__ __forceinline__ long long r_row(const RowGeo& g, int tx, int q) {
  const int z = q < g.n ? 0 : q / g.n;  // 2D rows never divide
  return tx * g.tstride + (long long)z * g.slab + (long long)(q - z * g.n) * P;
}

template <int P, int PRO>
__global__ void __launch_bounds__(256) conv_rows_fwd(const ConvOp op, const float2* __restrict__ tw_g,
                                                     float2* __restrict__ R, const RowGeo geo) {
  typedef ConvCfg<P> C;
  typedef RPlan<P> PL;
  __shared__ float2 tw[TwTable<P, false>::SIZE];
  __shared__ float2 buf[C::RB * C::PP];
  pdl_trigger();
  pdl_wait();
  const int tx = op.tx0 + blockIdx.y;                    // transform (vectors, scalars, flags)
  const int txs = op.tx_div > 1 ? tx / op.tx_div : tx;  // transmitter of this transform
  if (op.active && !op.active[txs]) return;
  const int n = geo.n;
  const int lt = threadIdx.x % C::NTF, row = threadIdx.x / C::NTF;
  const int iy = blockIdx.x * C::RB + row;
  const bool rowok = iy < geo.nrows;
  const long long N = (long long)geo.nrows * n;
  for (int i = threadIdx.x; i < TwTable<P, false>::SIZE; i += 256) tw[i] = tw_g[i];
  if (P / 8 < 32) __syncthreads();  // the twiddle table is shared by rows that sync per warp
  float2 alpha = make_float2(0.f, 0.f), beta = alpha, omega = alpha;
  if (PRO != PRO_COPY) {
    const double2* sc = reinterpret_cast<const double2*>(op.scal) + (size_t)txs * SC_STRIDE;
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
      if (PL::lower(q, r, R0) && rowok && ix < n) {  // n <= P/2: the upper half is padding
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
  reg_fft<P, false, false, true>(v, buf, RowLayA<P>{row * C::PP}, RowLayB<P>{row * C::PP}, lt, tw,
                                 RowSync<P>{row});
  if (!rowok) return;
  constexpr int RL = PL::template last<false>();
  float2* dst = R + r_row<P>(geo, blockIdx.y, iy);  // R holds the chunk's transforms from its start
#pragma unroll
  for (int q = 0; q < 8 / RL; ++q)
#pragma unroll
    for (int r = 0; r < RL; ++r) dst[PL::elem(lt, q, r, RL)] = v[q * RL + r];
}

// Column transforms over R.  Column (j, c) of transmitter tx starts at
//   R + tx * tstride + j * slab + c        (c < P contiguous, W columns per CTA)
// and its element i sits es further per i.  Modes:
//   COL_G   : load i < n, forward FFT, times ghat[k * es + j * slab + c]
//             (conjugated for G^H), inverse FFT, store i < n;
//   COL_FWD : load i < n, forward FFT, store all P outputs;
//   COL_INV : load all P, inverse FFT, store i < n.
enum { COL_G = 0, COL_FWD = 1, COL_INV = 2 };

struct ColGeo {
  int n, cps;  // column blocks per slab (P / W)
  long long es, slab, tstride;
  int tx_div;
  int tx0;     // first transform of the launch (R starts at the chunk's first transform)
};

// Dynamic shared memory of the column kernel, in float2: the exchange
// buffers, the forward and reversed twiddle tables.  Three-stage plans
// ping-pong their two exchanges between two buffers (one barrier per
// exchange instead of two), which exceeds the 48 KB of static shared memory
// at W P = 4096.  TWALL: with W >= 16 columns per CTA a warp's threads span at
// most two twiddle indices, so reading all twiddle powers from the table
// (broadcast reads) is cheaper than forming them by products.
template <int P, int MODE, int NT> struct ColSmem {
  static constexpr int W = ConvCfg<P>::template Col<NT>::W;
  static constexpr bool PING = RPlan<P>::NSTAGE == 3;
  static constexpr bool TWALL = W >= 16;
  static constexpr int BUF = P * W;
  static constexpr int BUF2 = PING ? P * W : 0;
  static constexpr int TW = MODE == COL_INV ? 0 : TwTable<P, false>::SIZE;
  static constexpr int TWR = MODE == COL_FWD ? 0 : TwTable<P, true>::SIZE;
  static constexpr size_t BYTES = sizeof(float2) * (size_t)(BUF + BUF2 + TW + TWR);
};

// D3 = false (2D) fixes es = P and a single slab at compile time.
template <int P, int MODE, bool ADJ, int NT, bool D3>
__global__ void __launch_bounds__(NT, 1024 / NT) conv_cols(const int* __restrict__ active, const float2* __restrict__ tw_g,
                                                    const float2* __restrict__ ghat, float2* __restrict__ R,
                                                    const ColGeo geo) {
  typedef ConvCfg<P> C;
  typedef RPlan<P> PL;
  typedef ColSmem<P, MODE, NT> SM;
  constexpr int W = SM::W;
  extern __shared__ __align__(16) float2 smem[];
  float2* buf = smem;
  float2* buf2 = buf + SM::BUF;
  float2* tw = buf2 + SM::BUF2;
  float2* twr = tw + SM::TW;
  pdl_trigger();
  pdl_wait();
  const int tx = geo.tx0 + blockIdx.y;
  if (active && !active[geo.tx_div > 1 ? tx / geo.tx_div : tx]) return;
  const int n = geo.n;
  const int w = threadIdx.x % W, lt = threadIdx.x / W;
  const int j = D3 ? blockIdx.x / geo.cps : 0;
  const int c0 = (D3 ? blockIdx.x % geo.cps : blockIdx.x) * W;
  const long long es = D3 ? geo.es : P;
  if (MODE != COL_INV)
    for (int i = threadIdx.x; i < TwTable<P, false>::SIZE; i += NT) tw[i] = tw_g[i];
  if (MODE != COL_FWD)
    for (int i = threadIdx.x; i < TwTable<P, true>::SIZE; i += NT) twr[i] = tw_g[TW_STRIDE + i];
  float2* base = R + blockIdx.y * geo.tstride + j * geo.slab + c0 + w;
  const ColLay<W> lay{w};
  const ColLayRev<P, W> layr{w};
  float2 v[8];
  if (MODE == COL_INV) {
    constexpr int RI0 = PL::template first<true>();
#pragma unroll
    for (int q = 0; q < 8 / RI0; ++q)
#pragma unroll
      for (int r = 0; r < RI0; ++r) v[q * RI0 + r] = base[PL::elem(lt, q, r, RI0) * es];
  } else {
    constexpr int R0 = PL::template first<false>();
#pragma unroll
    for (int q = 0; q < 8 / R0; ++q)
#pragma unroll
      for (int r = 0; r < R0; ++r) {
        const int i = PL::elem(lt, q, r, R0);
        v[q * R0 + r] = (PL::lower(q, r, R0) && i < n) ? base[i * es] : make_float2(0.f, 0.f);
      }
    reg_fft<P, false, false, true, SM::TWALL, SM::PING>(v, buf, lay, lay, lt, tw, CtaSync(), buf2);
  }
  constexpr int RL = PL::template last<false>();
  if (MODE == COL_FWD) {
#pragma unroll
    for (int q = 0; q < 8 / RL; ++q)
#pragma unroll
      for (int r = 0; r < RL; ++r) base[PL::elem(lt, q, r, RL) * es] = v[q * RL + r];
    return;
  }
  if (MODE == COL_G) {
    // spectrum product in registers: forward outputs are the inverse (reversed plan) inputs
    const float2* gcol = ghat + j * geo.slab + c0 + w;
#pragma unroll
    for (int q = 0; q < 8 / RL; ++q)
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        float2 g = __ldg(gcol + PL::elem(lt, q, r, RL) * es);
        if (ADJ) g.y = -g.y;
        v[q * RL + r] = c_mul(v[q * RL + r], g);
      }
  }
  // PING: both transforms use buf, then buf2, and each exchange's barrier orders the reads of
  // the one before (reg_fft); otherwise the leading barrier of each exchange does
  reg_fft<P, true, true, false, SM::TWALL, SM::PING>(v, buf, layr, layr, lt, twr, CtaSync(), buf2);
  constexpr int RI = PL::template last<true>();
#pragma unroll
  for (int q = 0; q < 8 / RI; ++q)
#pragma unroll
    for (int r = 0; r < RI; ++r) {
      const int i = PL::elem(lt, q, r, RI);
      if (PL::lower(q, r, RI) && i < n) base[i * es] = v[q * RI + r];
    }
}

// Two-stage column kernels (column shape COLS_TWO_STAGE): P = E x NT with E
// elements a thread and NT threads a column (512 = 32 x 16, 256 = 16 x 16,
// 128 = 16 x 8), so each transform needs one shared-memory exchange instead of
// the two of the three-stage plans.  The second radix equals NT, and with j
// the item, lt the thread's place in its column and tw[m] = exp(-2 pi i m / P):
//  forward : radix E on elements lt + NT r (r >= E/2 is padding when the
//            input has n <= P/2 rows), outputs to row E lt + k; radix NT on
//            items j = lt + NT q (q < E / NT) reading rows j + E r with
//            twiddles tw[r j]; register NT q + r then holds frequency
//            lt + NT q + E r;
//  inverse : (the reversed plan, on those registers) radix NT in place,
//            outputs to row NT j + r; radix E on rows lt + NT r with
//            conj(tw[r lt]); output k is element lt + NT k, k < E/2 kept.
// Modes as for conv_cols: COL_G (forward, ghat product, inverse), COL_FWD
// (forward, all P outputs stored), COL_INV (inverse of all P inputs).
// W = 256 / NT columns per 256-thread CTA: a half-warp's lanes share one row,
// so every exchange access is a contiguous row segment (no bank conflicts) and
// the twiddle reads, from a copy of the table in shared memory, are
// broadcasts.  E = 32 takes 128 registers (2 CTAs per SM), E = 16 about 64.
template <int P> struct TwoStage {
  static constexpr int E = P == 512 ? 32 : 16;
  static constexpr int NT = P / E;
  static constexpr int Q = E / NT;
  static constexpr int W = 256 / NT;
  static constexpr int MINB = E == 32 ? 2 : 3;
  static constexpr size_t SMEM = sizeof(float2) * (size_t)(P * W + P);  // exchange buffer, then twiddles
  static_assert(P == 128 || P == 256 || P == 512, "two-stage plans: P = 128, 256, 512");
};

// Compiler-only ordering point: memory accesses are not moved across it, which
// keeps the loads of one butterfly group from being hoisted above the
// arithmetic of the previous one (bounding live registers).  The loads it
// orders are plain ones: read-only (non-coherent) loads may move across it.
__device__ __forceinline__ void reorder_fence() { asm volatile("" ::: "memory"); }

template <int P, int MODE, bool ADJ, bool D3>
__global__ void __launch_bounds__(256, TwoStage<P>::MINB)
    conv_cols_2s(const int* __restrict__ active, const float2* tw_g, const float2* ghat, float2* __restrict__ R,
                 const ColGeo geo) {
  typedef TwoStage<P> TS;
  constexpr int E = TS::E, NT = TS::NT, Q = TS::Q, W = TS::W;
  extern __shared__ __align__(16) float2 smem[];  // [P rows][W columns], then P twiddles
  pdl_trigger();
  pdl_wait();
  const int tx = geo.tx0 + blockIdx.y;
  if (active && !active[geo.tx_div > 1 ? tx / geo.tx_div : tx]) return;
  const int n = geo.n;
  const int w = threadIdx.x % W, lt = threadIdx.x / W;
  const int j3 = D3 ? blockIdx.x / geo.cps : 0;
  const int c0 = (D3 ? blockIdx.x % geo.cps : blockIdx.x) * W;
  const long long es = D3 ? geo.es : P;
  float2* base = R + blockIdx.y * geo.tstride + j3 * geo.slab + c0 + w;
  // the twiddle table in shared memory (first read after a barrier); read from
  // global memory it cost 6 % more time at P = 512
  float2* tws = smem + P * W;
  for (int i = threadIdx.x; i < P; i += 256) tws[i] = tw_g[i];
  const float2* tw = tws;
  float2 v[E];
  if constexpr (MODE != COL_INV) {
#pragma unroll
    for (int r = 0; r < E / 2; ++r) {
      const int i = lt + NT * r;
      v[r] = i < n ? base[i * es] : make_float2(0.f, 0.f);
    }
    dft_n_lo<E, false>(v);
#pragma unroll
    for (int k = 0; k < E; ++k) smem[(E * lt + k) * W + w] = v[k];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int j = lt + NT * q;
#pragma unroll
      for (int r = 0; r < NT; ++r) {
        const float2 x = smem[(j + E * r) * W + w];
        v[NT * q + r] = r == 0 ? x : c_mul(x, tw[r * j]);
      }
      dft_n<NT, false>(v + NT * q);
      reorder_fence();
    }
    if constexpr (MODE == COL_FWD) {
#pragma unroll
      for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int r = 0; r < NT; ++r) base[(lt + NT * q + E * r) * es] = v[NT * q + r];
      return;
    }
    const float2* gcol = ghat + j3 * geo.slab + c0 + w;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
#pragma unroll
      for (int r = 0; r < NT; ++r) {
        float2 g = gcol[(lt + NT * q + E * r) * es];
        if (ADJ) g.y = -g.y;
        v[NT * q + r] = c_mul(v[NT * q + r], g);
      }
      dft_n<NT, true>(v + NT * q);
      reorder_fence();
    }
    __syncthreads();  // every read of the first exchange is done
  } else {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
#pragma unroll
      for (int r = 0; r < NT; ++r) v[NT * q + r] = base[(lt + NT * q + E * r) * es];
      dft_n<NT, true>(v + NT * q);
      reorder_fence();
    }
  }
#pragma unroll
  for (int q = 0; q < Q; ++q)
#pragma unroll
    for (int r = 0; r < NT; ++r) smem[(NT * (lt + NT * q) + r) * W + w] = v[NT * q + r];
  __syncthreads();
#pragma unroll
  for (int r = 0; r < E; ++r) {
    const float2 x = smem[(lt + NT * r) * W + w];
    v[r] = r == 0 ? x : c_mulcj(x, tw[r * lt]);
    if (r % 8 == 7) reorder_fence();
  }
  dft_n<E, true>(v);
#pragma unroll
  for (int k = 0; k < E / 2; ++k) {
    const int i = lt + NT * k;
    if (i < n) base[i * es] = v[k];
  }
}


template <int P, int EPI, int DK>
__global__ void __launch_bounds__(256) conv_rows_inv(const ConvOp op, const float2* __restrict__ tw_g,
                                                     const float2* __restrict__ R, const RowGeo geo, int nblk) {
  typedef ConvCfg<P> C;
  typedef RPlan<P> PL;
  __shared__ float2 tw[TwTable<P, true>::SIZE];
  __shared__ float2 buf[C::RB * C::PP];
  pdl_trigger();
  pdl_wait();
  const int tx = op.tx0 + blockIdx.y;
  if (op.active && !op.active[op.tx_div > 1 ? tx / op.tx_div : tx]) return;
  const int n = geo.n;
  const int lt = threadIdx.x % C::NTF, row = threadIdx.x / C::NTF;
  const int iy = blockIdx.x * C::RB + row;
  const bool rowok = iy < geo.nrows;
  const long long N = (long long)geo.nrows * n;
  for (int i = threadIdx.x; i < TwTable<P, true>::SIZE; i += 256) tw[i] = tw_g[TW_STRIDE + i];
  if (P / 8 < 32) __syncthreads();  // the twiddle table is shared by rows that sync per warp
  constexpr int R0 = PL::template first<true>();
  const float2* srow = R + r_row<P>(geo, blockIdx.y, rowok ? iy : 0);
  float2 v[8];
#pragma unroll
  for (int q = 0; q < 8 / R0; ++q)
#pragma unroll
    for (int r = 0; r < R0; ++r) v[q * R0 + r] = rowok ? srow[PL::elem(lt, q, r, R0)] : make_float2(0.f, 0.f);
  const bool postf = op.mul_f && op.adjoint;
  bool need_aux = EPI == EPI_RESID || (EPI == EPI_CONV_ADD && op.aux) || DK == DOTS_RV || DK == DOTS_RES;
  if (DK == DOTS_ANY)
    for (int s = 0; s < DOT_SLOTS; ++s) need_aux |= op.dot_a[s] == OP_AUX || op.dot_b[s] == OP_AUX;
  constexpr int RL = PL::template last<true>();
  // epilogue operands are loaded before the transform so their latency overlaps
  // it; only outputs below P/2 can be kept (n <= P/2)
  float2 pre_src[8], pre_aux[8];
#pragma unroll
  for (int q = 0; q < 8 / RL; ++q)
#pragma unroll
    for (int r = 0; r < RL; ++r) {
      if (!PL::lower(q, r, RL)) continue;
      const int ix = PL::elem(lt, q, r, RL);
      const bool ok = rowok && ix < n;
      const long long idx = tx * N + (long long)(rowok ? iy : 0) * n + (ix < n ? ix : 0);
      pre_src[q * RL + r] = (ok && EPI != EPI_CONV_ADD) ? op.esrc[idx] : make_float2(0.f, 0.f);
      pre_aux[q * RL + r] = (ok && need_aux) ? op.aux[idx] : make_float2(0.f, 0.f);
    }
  reg_fft<P, true, true>(v, buf, RowLayA<P>{row * C::PP}, RowLayB<P>{row * C::PP}, lt, tw, RowSync<P>{row});
  float2 acc[DOT_SLOTS];
#pragma unroll
  for (int s = 0; s < DOT_SLOTS; ++s) acc[s] = make_float2(0.f, 0.f);
  if (rowok) {
#pragma unroll
    for (int q = 0; q < 8 / RL; ++q)
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        if (!PL::lower(q, r, RL)) continue;
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
        if constexpr (DK == DOTS_RV) {
          acc[0] = c_add(acc[0], c_cjmul(aux, y));
        } else if constexpr (DK == DOTS_TS) {
          acc[1] = c_add(acc[1], c_cjmul(y, src));
          acc[2].x = fmaf(y.x, y.x, fmaf(y.y, y.y, acc[2].x));
        } else if constexpr (DK == DOTS_RES) {
          acc[0].x = fmaf(aux.x, aux.x, fmaf(aux.y, aux.y, acc[0].x));
          acc[2].x = fmaf(y.x, y.x, fmaf(y.y, y.y, acc[2].x));
        } else if constexpr (DK == DOTS_ANY) {
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
  if constexpr (DK != DOTS_NONE)
    block_dots<256, DotSlots<DK>::MASK>(acc, reinterpret_cast<float2*>(op.part) + ((size_t)tx * nblk + blockIdx.x) * DOT_SLOTS);
}

template <int P, int MODE, bool ADJ, int NT>
static void launch_cols(cisor_ctx* c, const ConvOp& op, int nslab, long long es, long long slab) {
  constexpr int W = ConvCfg<P>::template Col<NT>::W;
  constexpr size_t SMB = ColSmem<P, MODE, NT>::BYTES;
  const ColGeo geo{c->n, P / W, es, slab, c->rtstride, op.tx_div, op.tx0};
  dim3 g((P / W) * nslab, op.ntx);
  if constexpr (P <= 256) {  // 3D grids use P <= 256
    if (c->dim == 3) {
      (void)launch_pdl(conv_cols<P, MODE, ADJ, NT, true>, g, dim3(NT), SMB, c->stream, op.active, c->twst, c->ghat, c->R,
                       geo);
      return;
    }
  }
  if constexpr (MODE == COL_G)
    (void)launch_pdl(conv_cols<P, MODE, ADJ, NT, false>, g, dim3(NT), SMB, c->stream, op.active, c->twst, c->ghat, c->R,
                     geo);
}

// The column kernels' dynamic shared memory may exceed the 48 KB default: raise
// each instantiation's limit once, when a context picks its FFT size.
template <int P, int MODE, bool ADJ, int NT, bool D3>
static cudaError_t cols_attr() {
  return cudaFuncSetAttribute(conv_cols<P, MODE, ADJ, NT, D3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)ColSmem<P, MODE, NT>::BYTES);
}
template <int P, bool ADJ, int NT>
static cudaError_t cols_attrs() {
  cudaError_t e = cols_attr<P, COL_G, ADJ, NT, false>();
  if constexpr (P <= 256) {
    if (e == cudaSuccess) e = cols_attr<P, COL_G, ADJ, NT, true>();
    if (e == cudaSuccess) e = cols_attr<P, COL_FWD, ADJ, NT, true>();
    if (e == cudaSuccess) e = cols_attr<P, COL_INV, ADJ, NT, true>();
  }
  return e;
}
template <int P>
static cisor_status conv_init_t() {
  if constexpr (P >= 128) {
    constexpr int smb = (int)TwoStage<P>::SMEM;
    for (int adj = 0; adj < 2; ++adj) {
      CISOR_CUDA(cudaFuncSetAttribute(adj ? conv_cols_2s<P, COL_G, true, false> : conv_cols_2s<P, COL_G, false, false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, smb));
      if constexpr (P <= 256) {
        CISOR_CUDA(cudaFuncSetAttribute(adj ? conv_cols_2s<P, COL_G, true, true> : conv_cols_2s<P, COL_G, false, true>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, smb));
        CISOR_CUDA(cudaFuncSetAttribute(adj ? conv_cols_2s<P, COL_FWD, true, true> : conv_cols_2s<P, COL_FWD, false, true>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, smb));
        CISOR_CUDA(cudaFuncSetAttribute(adj ? conv_cols_2s<P, COL_INV, true, true> : conv_cols_2s<P, COL_INV, false, true>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, smb));
      }
    }
  }
  CISOR_CUDA((cols_attrs<P, false, 256>()));
  CISOR_CUDA((cols_attrs<P, true, 256>()));
  CISOR_CUDA((cols_attrs<P, false, 512>()));
  CISOR_CUDA((cols_attrs<P, true, 512>()));
  return CISOR_OK;
}

// the two-stage kernels (P = 128, 256 in 2D and 3D; P = 512 in 2D; the API
// admits the shape only there)
template <int P, int MODE, bool ADJ>
static void launch_cols_2s(cisor_ctx* c, const ConvOp& op, int nslab, long long es, long long slab) {
  if constexpr (P >= 128) {
    typedef TwoStage<P> TS;
    const ColGeo geo{c->n, P / TS::W, es, slab, c->rtstride, op.tx_div, op.tx0};
    const dim3 g((P / TS::W) * nslab, op.ntx);
    if constexpr (P <= 256) {
      if (c->dim == 3) {
        (void)launch_pdl(conv_cols_2s<P, MODE, ADJ, true>, g, dim3(256), TS::SMEM, c->stream, op.active, c->tw, c->ghat,
                         c->R, geo);
        return;
      }
    }
    if constexpr (MODE == COL_G)
      (void)launch_pdl(conv_cols_2s<P, MODE, ADJ, false>, g, dim3(256), TS::SMEM, c->stream, op.active, c->tw, c->ghat,
                       c->R, geo);
  }
}

template <int P, int MODE>
static void cols_pass(cisor_ctx* c, const ConvOp& op, int nslab, long long es, long long slab) {
  if (c->cols_nt == COLS_TWO_STAGE || c->cols_nt == COLS_CLUSTER) {  // (combinations the cluster pass lacks)
    if (op.adjoint)
      launch_cols_2s<P, MODE, true>(c, op, nslab, es, slab);
    else
      launch_cols_2s<P, MODE, false>(c, op, nslab, es, slab);
    return;
  }
  if (c->cols_nt == 256) {
    if (op.adjoint)
      launch_cols<P, MODE, true, 256>(c, op, nslab, es, slab);
    else
      launch_cols<P, MODE, false, 256>(c, op, nslab, es, slab);
  } else {
    if (op.adjoint)
      launch_cols<P, MODE, true, 512>(c, op, nslab, es, slab);
    else
      launch_cols<P, MODE, false, 512>(c, op, nslab, es, slab);
  }
}

template <int P>
static cisor_status conv_chunk_t(cisor_ctx* c, const ConvOp& op) {
  typedef ConvCfg<P> C;
  if constexpr (P == 512) {  // the one-kernel cluster pass where the shape asks for it and the combination exists
    if (c->cols_nt == COLS_CLUSTER && conv_fused_ok(c)) {
      cudaError_t e = cudaSuccess;
      if (conv_fused_pass(c, op, dots_kind(op), &e)) {
        CISOR_CUDA(e);
        c->launches += 1;
        return CISOR_OK;
      }
    }
  }
  const int n = c->n;
  const RowGeo rg{n, c->nrows, c->rslab, c->rtstride};
  dim3 grow((c->nrows + C::RB - 1) / C::RB, op.ntx);
  switch (op.prologue) {
    case PRO_COPY: (void)launch_pdl(conv_rows_fwd<P, PRO_COPY>, grow, dim3(256), 0, c->stream, op, c->twst, c->R, rg); break;
    case PRO_PUPDATE:
      (void)launch_pdl(conv_rows_fwd<P, PRO_PUPDATE>, grow, dim3(256), 0, c->stream, op, c->twst, c->R, rg);
      break;
    default: (void)launch_pdl(conv_rows_fwd<P, PRO_AXPY>, grow, dim3(256), 0, c->stream, op, c->twst, c->R, rg); break;
  }
  CISOR_CUDA(cudaGetLastError());
  if (c->dim == 3) {
    const long long PP = (long long)P * P;
    cols_pass<P, COL_FWD>(c, op, n, P, PP);   // y, in each of the n z slabs
    CISOR_CUDA(cudaGetLastError());
    cols_pass<P, COL_G>(c, op, P, PP, P);     // z, for each of the P y frequencies
    CISOR_CUDA(cudaGetLastError());
    cols_pass<P, COL_INV>(c, op, n, P, PP);   // y back, n rows kept
  } else {
    cols_pass<P, COL_G>(c, op, 1, P, 0);
  }
  CISOR_CUDA(cudaGetLastError());
  const int dk = dots_kind(op);
#define CISOR_ROWS_INV(E, D) \
  (void)launch_pdl(conv_rows_inv<P, E, D>, grow, dim3(256), 0, c->stream, op, c->twst, c->R, rg, c->nblk)
  switch (op.epilogue) {
    case EPI_MATVEC:
      if (dk == DOTS_NONE) CISOR_ROWS_INV(EPI_MATVEC, DOTS_NONE);
      else if (dk == DOTS_RV) CISOR_ROWS_INV(EPI_MATVEC, DOTS_RV);
      else if (dk == DOTS_TS) CISOR_ROWS_INV(EPI_MATVEC, DOTS_TS);
      else CISOR_ROWS_INV(EPI_MATVEC, DOTS_ANY);
      break;
    case EPI_RESID:
      if (dk == DOTS_RES) CISOR_ROWS_INV(EPI_RESID, DOTS_RES);
      else CISOR_ROWS_INV(EPI_RESID, DOTS_ANY);
      break;
    default:
      if (dk == DOTS_NONE) CISOR_ROWS_INV(EPI_CONV_ADD, DOTS_NONE);
      else CISOR_ROWS_INV(EPI_CONV_ADD, DOTS_ANY);
      break;
  }
#undef CISOR_ROWS_INV
  CISOR_CUDA(cudaGetLastError());
  c->launches += conv_kernels_per_pass(c->dim);
  return CISOR_OK;
}

// One pass over op.ntx transforms, as consecutive chunks of c->tx_chunk
// transforms (all at once when 0): each chunk runs the whole row / column /
// row chain before the next starts and they all use the start of R, so with
// a chunk's intermediate sized below L2 it is written and read back there
// instead of round-tripping through HBM.
template <int P>
static cisor_status conv_pass_t(cisor_ctx* c, const ConvOp& op) {
  const int chunk = (c->tx_chunk > 0 && c->tx_chunk < op.ntx) ? c->tx_chunk : op.ntx;
  for (int t0 = 0; t0 < op.ntx; t0 += chunk) {
    ConvOp o = op;
    o.tx0 = op.tx0 + t0;
    o.ntx = op.ntx - t0 < chunk ? op.ntx - t0 : chunk;
    CISOR_TRY(conv_chunk_t<P>(c, o));
  }
  return CISOR_OK;
}

cisor_status conv_init(int P) {
  if (P == 512) CISOR_TRY(conv_fused_init());
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
