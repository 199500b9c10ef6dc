// One batched FFT-convolution pass for 2D grids with P = 512 (n <= 256) in
// ONE kernel: a cluster of 8 CTAs convolves one transmitter's field with the
// whole padded intermediate held in the cluster's distributed shared memory,
// so it never goes to HBM (the three-kernel pass of conv.cu writes it to
// global memory and reads it back twice).
//
//  stage 1  each CTA: row FFTs of its 32 rows (prologue, f, zero padding to
//           P, forward transform; the row's shared-memory slot is the
//           transform's exchange buffer and then holds its spectrum)
//  cluster barrier
//  stage 2  each CTA: 64 of the P columns, 8 at a time: the n non-zero rows
//           of a column are read from the 8 CTAs' slots (distributed shared
//           memory), forward FFT along y, times ghat (conj for G^H), inverse
//           FFT, and the first n outputs written back to their owners' slots
//  cluster barrier
//  stage 3  each CTA: inverse row FFTs of its 32 rows, crop to n, and the
//           epilogue of conv_rows_inv (A x, residual or G^H v + z, and the
//           per-4-row dot-product partials in the same layout)
//
// Shared memory per CTA: 32 row slots of row_pitch(512) complex64 (139 KB),
// the column transforms' two exchange buffers (64 KB) and both stage-twiddle
// tables; one CTA per SM.  Every CTA of a cluster takes the same path through
// both cluster barriers: the only early exit (a converged transmitter) reads
// the same flag in all eight.
#include <cooperative_groups.h>

#include "common.cuh"
#include "dots.cuh"
#include "fft.cuh"
#include "regfft.cuh"

namespace cg = cooperative_groups;

namespace cisor {

namespace {

constexpr int ZP = 512;                 // FFT side
constexpr int ZCL = 8;                  // CTAs per cluster (one transmitter)
constexpr int ZNT = 512;                // threads per CTA
constexpr int ZRPC = 32;                // row slots per CTA (ZCL * ZRPC = 256 >= n)
constexpr int ZPP = row_pitch(ZP);      // slot pitch (complex)
constexpr int ZNTF = ZP / 8;            // threads per transform
constexpr int ZRB = ZNT / ZNTF;         // rows per row batch (8)
constexpr int ZW = ZNT / ZNTF;          // columns per column batch (8)
constexpr int ZCPC = ZP / ZCL;          // columns per CTA (64)
constexpr int ZTWF = TwTable<ZP, false>::SIZE, ZTWR = TwTable<ZP, true>::SIZE;
constexpr size_t ZSMEM = sizeof(float2) * ((size_t)ZRPC * ZPP + 2 * (size_t)ZP * ZW + ZTWF + ZTWR);

// position of element i of a row in its slot (the layout of the row transforms' first exchange)
__device__ __forceinline__ int zpos(int i) { return i + (i >> 4); }

template <int PRO, int EPI, int DK, bool ADJ>
__global__ void __launch_bounds__(ZNT, 1) conv_fused512(const ConvOp op, const float2* __restrict__ tw_g,
                                                        const float2* __restrict__ ghat, int n, int nblk) {
  typedef RPlan<ZP> PL;
  extern __shared__ __align__(16) float2 smem[];
  float2* Rs = smem;                      // [ZRPC][ZPP]
  float2* cb = Rs + ZRPC * ZPP;           // [ZP * ZW] column exchange buffers (ping-pong)
  float2* cb2 = cb + ZP * ZW;
  float2* twf = cb2 + ZP * ZW;            // forward plan stage twiddles
  float2* twr = twf + ZTWF;               // reversed plan stage twiddles
  __shared__ float red[2 * DOT_SLOTS][ZNT / 32];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  pdl_trigger();
  pdl_wait();
  const int tx = op.tx0 + (int)(blockIdx.x / ZCL);
  const int txs = op.tx_div > 1 ? tx / op.tx_div : tx;
  if (op.active && !op.active[txs]) return;  // the same flag for every CTA of the cluster
  for (int i = threadIdx.x; i < ZTWF; i += ZNT) twf[i] = tw_g[i];
  for (int i = threadIdx.x; i < ZTWR; i += ZNT) twr[i] = tw_g[TW_STRIDE + i];
  const long long N = (long long)n * n;
  float2 alpha = make_float2(0.f, 0.f), beta = alpha, omega = alpha;
  if (PRO != PRO_COPY) {
    const double2* sc = reinterpret_cast<const double2*>(op.scal) + (size_t)txs * SC_STRIDE;
    alpha = z_to_c(sc[SC_ALPHA]);
    beta = z_to_c(sc[SC_BETA]);
    omega = z_to_c(sc[SC_OMEGA]);
  }
  const bool fresh = (beta.x == 0.f && beta.y == 0.f);
  const bool mulf = op.mul_f && !ADJ;
  __syncthreads();

  // ---------------------------------------------------------------- stage 1: row FFTs
  {
    const int lt = threadIdx.x % ZNTF, rb = threadIdx.x / ZNTF;
    constexpr int R0 = PL::template first<false>();
    constexpr int RL = PL::template last<false>();
#pragma unroll 1
    for (int bt = 0; bt < ZRPC / ZRB; ++bt) {
      const int slot = bt * ZRB + rb, iy = rank * ZRPC + slot;
      const bool rowok = iy < n;
      float2 v[8];
#pragma unroll
      for (int q = 0; q < 8 / R0; ++q)
#pragma unroll
        for (int r = 0; r < R0; ++r) {
          const int ix = PL::elem(lt, q, r, R0);
          float2 val = make_float2(0.f, 0.f);
          if (PL::lower(q, r, R0) && rowok && ix < n) {
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
            } else {
              const float2 s = c_sub(op.src[idx], c_mul(alpha, op.vvec[idx]));
              op.svec[idx] = s;
              val = s;
            }
            if (mulf) val = c_mul(val, op.f[pix]);
          }
          v[q * R0 + r] = val;
        }
      reg_fft<ZP, false, false, true>(v, Rs, RowLayA<ZP>{slot * ZPP}, RowLayB<ZP>{slot * ZPP}, lt, twf,
                                      RowSync<ZP>{slot});
      __syncthreads();  // the last exchange's reads of the slot are done
#pragma unroll
      for (int q = 0; q < 8 / RL; ++q)
#pragma unroll
        for (int r = 0; r < RL; ++r) Rs[slot * ZPP + zpos(PL::elem(lt, q, r, RL))] = v[q * RL + r];
      __syncthreads();
    }
  }
  cl.sync();

  // ---------------------------------------------------------------- stage 2: columns
  {
    const int w = threadIdx.x % ZW, lt = threadIdx.x / ZW;
    const ColLay<ZW> lay{w};
    const ColLayRev<ZP, ZW> layr{w};
    constexpr int R0 = PL::template first<false>();
    constexpr int RL = PL::template last<false>();
    constexpr int RI = PL::template last<true>();
#pragma unroll 1
    for (int bc = 0; bc < ZCPC / ZW; ++bc) {
      const int c = rank * ZCPC + bc * ZW + w;
      const int cpos = zpos(c);
      float2 v[8];
#pragma unroll
      for (int q = 0; q < 8 / R0; ++q)
#pragma unroll
        for (int r = 0; r < R0; ++r) {
          const int i = PL::elem(lt, q, r, R0);
          float2 val = make_float2(0.f, 0.f);
          if (PL::lower(q, r, R0) && i < n) val = *cl.map_shared_rank(Rs + (i % ZRPC) * ZPP + cpos, i / ZRPC);
          v[q * R0 + r] = val;
        }
      reg_fft<ZP, false, false, true, false, true>(v, cb, lay, lay, lt, twf, CtaSync(), cb2);
      const float2* gcol = ghat + c;
#pragma unroll
      for (int q = 0; q < 8 / RL; ++q)
#pragma unroll
        for (int r = 0; r < RL; ++r) {
          float2 g = __ldg(gcol + (long long)PL::elem(lt, q, r, RL) * ZP);
          if (ADJ) g.y = -g.y;
          v[q * RL + r] = c_mul(v[q * RL + r], g);
        }
      reg_fft<ZP, true, true, false, false, true>(v, cb, layr, layr, lt, twr, CtaSync(), cb2);
#pragma unroll
      for (int q = 0; q < 8 / RI; ++q)
#pragma unroll
        for (int r = 0; r < RI; ++r) {
          const int i = PL::elem(lt, q, r, RI);
          if (PL::lower(q, r, RI) && i < n) *cl.map_shared_rank(Rs + (i % ZRPC) * ZPP + cpos, i / ZRPC) = v[q * RI + r];
        }
    }
  }
  cl.sync();

  // ---------------------------------------------------------------- stage 3: inverse rows + epilogue
  {
    const int lt = threadIdx.x % ZNTF, rb = threadIdx.x / ZNTF;
    constexpr int R0 = PL::template first<true>();
    constexpr int RL = PL::template last<true>();
    const bool postf = op.mul_f && ADJ;
    constexpr bool need_aux = EPI == EPI_RESID || DK == DOTS_RV || DK == DOTS_RES;
#pragma unroll 1
    for (int bt = 0; bt < ZRPC / ZRB; ++bt) {
      const int slot = bt * ZRB + rb, iy = rank * ZRPC + slot;
      const bool rowok = iy < n;
      float2 v[8];
#pragma unroll
      for (int q = 0; q < 8 / R0; ++q)
#pragma unroll
        for (int r = 0; r < R0; ++r) v[q * R0 + r] = Rs[slot * ZPP + zpos(PL::elem(lt, q, r, R0))];
      const bool has_aux = need_aux || (EPI == EPI_CONV_ADD && op.aux);
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
          pre_aux[q * RL + r] = (ok && has_aux) ? op.aux[idx] : make_float2(0.f, 0.f);
        }
      reg_fft<ZP, true, true>(v, Rs, RowLayA<ZP>{slot * ZPP}, RowLayB<ZP>{slot * ZPP}, lt, twr, RowSync<ZP>{slot});
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
            float2 cv = v[q * RL + r];
            if (postf) cv = c_cjmul(op.f[pix], cv);
            const float2 src = pre_src[q * RL + r], aux = pre_aux[q * RL + r];
            float2 y;
            if (EPI == EPI_MATVEC) {
              y = c_sub(src, cv);
            } else if (EPI == EPI_RESID) {
              y = c_sub(aux, c_sub(src, cv));
            } else {
              y = c_add(cv, aux);
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
            }
          }
      }
      if constexpr (DK != DOTS_NONE) {
        // one partial per 4 rows (threads 0-255: rows 0-3 of the batch, 256-511: rows 4-7), the layout of
        // the three-kernel pass at P = 512
        constexpr int MASK = DotSlots<DK>::MASK;
        float vals[2 * DOT_SLOTS];
#pragma unroll
        for (int s = 0; s < DOT_SLOTS; ++s) {
          vals[2 * s] = acc[s].x;
          vals[2 * s + 1] = acc[s].y;
        }
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
        for (int k = 0; k < 2 * DOT_SLOTS; ++k) {
          if (!((MASK >> (k / 2)) & 1)) continue;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) vals[k] += __shfl_xor_sync(0xffffffffu, vals[k], o);
          if (lane == 0) red[k][wid] = vals[k];
        }
        __syncthreads();
        if (threadIdx.x < 4 * DOT_SLOTS) {
          const int grp = threadIdx.x / (2 * DOT_SLOTS), k = threadIdx.x % (2 * DOT_SLOTS);
          const int row0 = rank * ZRPC + bt * ZRB + 4 * grp;
          float sum = 0.f;
          if ((MASK >> (k / 2)) & 1) {
            float* rr = red[k] + 8 * grp;
#pragma unroll
            for (int wdt = 4; wdt > 0; wdt >>= 1)
#pragma unroll
              for (int i = 0; i < wdt; ++i) rr[i] += rr[i + wdt];
            sum = rr[0];
          }
          if (row0 < n) reinterpret_cast<float*>(op.part)[((size_t)tx * nblk + row0 / 4) * DOT_SLOTS * 2 + k] = sum;
        }
      }
      __syncthreads();  // the slot and red are reused by the next batch
    }
  }
}

template <int PRO, int EPI, int DK, bool ADJ>
cudaError_t fused_attr() {
  return cudaFuncSetAttribute(conv_fused512<PRO, EPI, DK, ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)ZSMEM);
}

template <int PRO, int EPI, int DK, bool ADJ>
cudaError_t fused_launch(cisor_ctx* c, const ConvOp& op) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ZCL * op.ntx);
  cfg.blockDim = dim3(ZNT);
  cfg.dynamicSmemBytes = ZSMEM;
  cfg.stream = c->stream;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = ZCL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = CISOR_PDL;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, conv_fused512<PRO, EPI, DK, ADJ>, op, (const float2*)c->twst,
                            (const float2*)c->ghat, c->n, c->nblk);
}

// the prologue / epilogue / dot-set combinations the solver and the operators use
template <bool ADJ>
int fused_dispatch(cisor_ctx* c, const ConvOp& op, int dk, cudaError_t* e) {
  if (op.prologue == PRO_COPY && op.epilogue == EPI_MATVEC && dk == DOTS_NONE)
    *e = fused_launch<PRO_COPY, EPI_MATVEC, DOTS_NONE, ADJ>(c, op);
  else if (op.prologue == PRO_PUPDATE && op.epilogue == EPI_MATVEC && dk == DOTS_RV)
    *e = fused_launch<PRO_PUPDATE, EPI_MATVEC, DOTS_RV, ADJ>(c, op);
  else if (op.prologue == PRO_AXPY && op.epilogue == EPI_MATVEC && dk == DOTS_TS)
    *e = fused_launch<PRO_AXPY, EPI_MATVEC, DOTS_TS, ADJ>(c, op);
  else if (op.prologue == PRO_COPY && op.epilogue == EPI_RESID && dk == DOTS_RES)
    *e = fused_launch<PRO_COPY, EPI_RESID, DOTS_RES, ADJ>(c, op);
  else if (op.prologue == PRO_COPY && op.epilogue == EPI_CONV_ADD && dk == DOTS_NONE)
    *e = fused_launch<PRO_COPY, EPI_CONV_ADD, DOTS_NONE, ADJ>(c, op);
  else
    return 0;
  return 1;
}

template <bool ADJ>
cudaError_t fused_attrs_adj() {
  cudaError_t e = fused_attr<PRO_COPY, EPI_MATVEC, DOTS_NONE, ADJ>();
  if (e == cudaSuccess) e = fused_attr<PRO_PUPDATE, EPI_MATVEC, DOTS_RV, ADJ>();
  if (e == cudaSuccess) e = fused_attr<PRO_AXPY, EPI_MATVEC, DOTS_TS, ADJ>();
  if (e == cudaSuccess) e = fused_attr<PRO_COPY, EPI_RESID, DOTS_RES, ADJ>();
  if (e == cudaSuccess) e = fused_attr<PRO_COPY, EPI_CONV_ADD, DOTS_NONE, ADJ>();
  return e;
}

}  // namespace

cisor_status conv_fused_init() {
  CISOR_CUDA(fused_attrs_adj<false>());
  CISOR_CUDA(fused_attrs_adj<true>());
  return CISOR_OK;
}

bool conv_fused_ok(const cisor_ctx* c) { return c->dim == 2 && c->P == ZP && c->n <= ZCL * ZRPC && c->ncomp == 1; }

// 1: launched (the status in *e); 0: this combination is not compiled in (the caller runs the three kernels)
int conv_fused_pass(cisor_ctx* c, const ConvOp& op, int dk, cudaError_t* e) {
  return op.adjoint ? fused_dispatch<true>(c, op, dk, e) : fused_dispatch<false>(c, op, dk, e);
}

}  // namespace cisor
