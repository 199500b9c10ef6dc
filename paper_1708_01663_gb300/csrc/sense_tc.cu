// The sensing GEMMs (Eq. 5 forward, Eq. 13's H^H w adjoint) on the fifth-
// generation tensor cores, TF32 with a hi / lo split: every FP32 operand x is
// held as hi = x with its 13 low mantissa bits cleared (exactly a TF32 value)
// and lo = x - hi (exact in FP32, read as TF32 by the MMA), and a product is
// hi.hi + lo.hi + hi.lo: about 21 mantissa bits; with the accumulation below
// the GEMMs are within 8e-7 of an FP64 product, inside the 1e-5 sensing
// tolerance that a single TF32 or a BF16 hi / lo product (1.5e-5) misses.
//
// The complex GEMM is one real GEMM: H is read as interleaved (Re, Im) floats,
// K = 2 x (complex columns), and each transmitter t contributes two rows of the
// small operand, so that D[row][2t] and D[row][2t + 1] are Re and Im of its
// result:
//   forward  Y[t][m] = sum_n H[m][n] X_t[n], X_t = f u_t (Eq. 5):
//            rows 2t = (Re X, -Im X), 2t + 1 = (Im X, Re X) per n
//   adjoint  z_t[n] = sum_m conj(H[m][n]) w_t[m] (H^H w, Eq. 13), read from the
//            transposed copy Ht[n][m] so that both GEMMs stream K-major rows:
//            rows 2t = (Re w, Im w), 2t + 1 = (Im w, -Re w) per m
// A CTA owns 128 rows of the big operand (receivers forward, field entries
// adjoint) and 2T (rounded to 16) accumulator columns in tensor memory; it
// streams 32 floats of K per chunk: each thread loads 4 x 16 bytes of the big
// operand for the next chunk into registers while the current chunk's MMAs
// run, splits them and stores them as core-matrix rows (8 rows x 16 bytes, K
// groups 144 bytes apart so that the 8 lanes of a 16-byte store phase hit
// distinct banks).  The forward pass splits K over CTAs (partials [split][T][M]
// summed by sense_reduce_kernel, in a fixed order); the adjoint CTA covers all
// of K (2M) and writes z and conj(f) z.  Every wait on the MMAs is bounded (a
// timeout sets the context's error flag, read by the host after the call).
#include "common.cuh"
#include "tc5.cuh"

namespace cisor {

constexpr int SK = 32;                       // K (floats) per chunk
constexpr int SLBO = 144, SSBO = 8 * SLBO;   // K-group and 8-row strides of the operand tiles (bytes)
constexpr int SPA = 16 * SSBO;               // bytes of one plane of the 128-row tile
constexpr int STH = 256;                     // threads per CTA
constexpr int S_WAIT = 1 << 20;              // polls of the MMA completion barrier before giving up
// K (floats) per CTA of the forward GEMM: splits of 64 chunks, 2048 and more CTAs at C3, measured faster than one
// wave of 432-chunk CTAs (1.04 against 1.59 ms): CTAs that start together read the same slab of the small
// operand, which then stays in L2 while H streams past it.
constexpr long long S_KMAX = 64 * SK;
constexpr long long S_MAX = 256;  // at most this many splits (partials T x M x 8 bytes each)


__host__ __device__ constexpr int soff(int row, int k) {
  return (row >> 3) * SSBO + (k >> 2) * SLBO + (row & 7) * 16 + (k & 3) * 4;
}
__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }
__device__ __forceinline__ long long wrap(long long j, long long NP) {
  while (j >= NP) j -= NP;
  return j;
}

// accumulator columns for ntx transmitters (2 ntx rounded up to an instantiated width)
int sense_tc_cols(int ntx) {
  const int need = 2 * ntx;
  return need <= 32 ? 32 : need <= 64 ? 64 : need <= 96 ? 96 : need <= 128 ? 128 : need <= 192 ? 192 : 256;
}
int sense_tc_smem(int ntx) { return 2 * SPA + 2 * (sense_tc_cols(ntx) / 8) * SSBO; }

// ADJ = 0: A = H [rows = M][lda = 2 Nf], K range [ks KS, ks KS + KS) of 2 Nf, small operand from f and u [T][Nf];
//          out0 = partials [(ks T + t) M + m].
// ADJ = 1: A = Ht [rows = Nf][lda = 2 M], all of K = 2 M, small operand from w [T][M];
//          out0 = z [t Nf + n], out1 (may be null) = conj(f) z.
// NB = 2T rounded up to one of 32, 64, 96, 128, 192, 256 accumulator columns.  Each chunk's 12 MMAs start a
// fresh accumulator, alternating between two TMEM buffers: while chunk c's MMAs run, the threads add chunk
// c - 1's result into FP32 registers (round to nearest).  The tensor cores' FP32 accumulation rounds its sums
// more coarsely: accumulating a whole split in TMEM (64 to 432 chunks, hundreds of MMAs) left the products
// 1.2e-5 to 1.5e-5 from FP64 on random inputs; with chains of 12 they are within 8e-7 (C2, C3 sizes).
template <int ADJ, int NB>
__global__ void __launch_bounds__(STH, NB > 128 ? 1 : 2) sense_tc_kernel(const float* __restrict__ A, long long lda, long long rows,
                                                       long long K, long long KS, const float2* __restrict__ src,
                                                       long long lds, const float2* __restrict__ f, long long NP,
                                                       int T, int M, long long Nf, float2* __restrict__ out0,
                                                       float2* __restrict__ out1, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  constexpr int SPB = (NB / 8) * SSBO;
  constexpr int NH = NB / 2;  // accumulator columns per thread
  constexpr uint32_t ncol = 2 * NB <= 64 ? 64u : 2 * NB <= 128 ? 128u : 2 * NB <= 256 ? 256u : 512u;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long row0 = (long long)blockIdx.x * 128;
  const long long kb = ADJ ? 0 : (long long)blockIdx.y * KS;
  const long long ke = ADJ ? K : (kb + KS < K ? kb + KS : K);
  const int nch = (int)((ke - kb + SK - 1) / SK);
  unsigned char* sb = sm + 2 * SPA;
  for (int i = tid * 16; i < 2 * SPB; i += STH * 16) *reinterpret_cast<uint4*>(sb + i) = make_uint4(0, 0, 0, 0);
  if (tid == 0) mbar_init(&mbar);
  if (warp == 0) tmem_alloc(&tslot, ncol);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot, s0 = smem_addr(sm);
  const int nitems = T * 16;  // (transmitter, complex column) pairs of a chunk
  float4 ra[4];
  float2 rb[8], rf[8];
  auto fetch = [&](long long k0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = tid + STH * q, r = idx >> 3, kg = idx & 7;
      const long long gr = row0 + r, kk = k0 + 4 * kg;
      ra[q] = (gr < rows && kk < ke) ? __ldg(reinterpret_cast<const float4*>(A + gr * lda + kk))
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int item = tid + STH * q;
      const long long j = k0 / 2 + (item & 15);
      const bool ok = item < nitems && 2 * j < ke;
      rb[q] = ok ? __ldg(src + (long long)(item >> 4) * lds + j) : make_float2(0.f, 0.f);
      if (!ADJ) rf[q] = ok ? __ldg(f + wrap(j, NP)) : make_float2(0.f, 0.f);
    }
  };
  auto stage = [&]() {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = tid + STH * q, o = soff(idx >> 3, 4 * (idx & 7));
      const float4 x = ra[q];
      const float4 h = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
      *reinterpret_cast<float4*>(sm + o) = h;
      *reinterpret_cast<float4*>(sm + SPA + o) = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int item = tid + STH * q;
      if (item < nitems) {
        const int c = item & 15, t = item >> 4;
        const float2 x = ADJ ? rb[q] : c_mul(rf[q], rb[q]);
        const float2 e0 = ADJ ? x : make_float2(x.x, -x.y);
        const float2 e1 = ADJ ? make_float2(x.y, -x.x) : make_float2(x.y, x.x);
        const int o0 = soff(2 * t, 2 * c), o1 = soff(2 * t + 1, 2 * c);
        const float2 h0 = make_float2(tf32_hi(e0.x), tf32_hi(e0.y)), h1 = make_float2(tf32_hi(e1.x), tf32_hi(e1.y));
        *reinterpret_cast<float2*>(sb + o0) = h0;
        *reinterpret_cast<float2*>(sb + SPB + o0) = make_float2(e0.x - h0.x, e0.y - h0.y);
        *reinterpret_cast<float2*>(sb + o1) = h1;
        *reinterpret_cast<float2*>(sb + SPB + o1) = make_float2(e1.x - h1.x, e1.y - h1.y);
      }
    }
  };
  uint32_t ph = 0;
  bool failed = false;
  auto wait_mma = [&]() {
    const bool ok = mbar_wait(&mbar, ph, S_WAIT);
    ph ^= 1u;
    tc_fence_after();
    if (__syncthreads_or(!ok)) {
      if (tid == 0) *reinterpret_cast<volatile int*>(err) = 1;  // mapped host memory: a plain store
      failed = true;
    }
    return !failed;
  };
  const uint32_t id = tc_idesc_tf32(128, NB);
  // row 32 (w % 4) + lane of the tile in this warp's TMEM lane quarter; warps w, w + 4 split the columns
  const int q = warp & 3, half = warp >> 2;
  const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16) + half * NH;
  float acc[NH];
#pragma unroll
  for (int j = 0; j < NH; ++j) acc[j] = 0.f;
  auto gather = [&](int buf) {  // acc += this thread's columns of accumulator buffer buf
#pragma unroll
    for (int c0 = 0; c0 < NH; c0 += 8) {
      float d[8];
      tmem_ld8(tl + buf * NB + c0, d);
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[c0 + j] += d[j];
    }
  };
  fetch(kb);
  for (int ch = 0; ch < nch; ++ch) {
    if (ch > 0 && !wait_mma()) break;  // the previous chunk's MMAs have read the tiles
    stage();
    if (ch + 1 < nch) fetch(kb + (long long)(ch + 1) * SK);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      const uint32_t d = tmem + (ch & 1) * NB;
#pragma unroll
      for (int ks = 0; ks < SK / 8; ++ks) {
        const uint32_t ah = s0 + ks * 2 * SLBO, al = ah + SPA;
        const uint32_t bh = s0 + 2 * SPA + ks * 2 * SLBO, bl = bh + SPB;
        const uint64_t dah = tc_desc(ah, SLBO, SSBO), dbh = tc_desc(bh, SLBO, SSBO);
        tc_mma_tf32(d, dah, dbh, id, ks > 0 ? 1u : 0u);
        tc_mma_tf32(d, tc_desc(al, SLBO, SSBO), dbh, id, 1u);
        tc_mma_tf32(d, dah, tc_desc(bl, SLBO, SSBO), id, 1u);
      }
      tc_commit(&mbar);
    }
    if (ch > 0) gather((ch - 1) & 1);  // the previous chunk's result, while this chunk's MMAs run
  }
  if (!failed && nch > 0 && wait_mma()) gather((nch - 1) & 1);
  if (!failed) {
    const long long row = row0 + 32 * q + lane;
#pragma unroll
    for (int c0 = 0; c0 < NH; c0 += 2) {
      {
        const int t = (half * NH + c0) / 2;
        if (t < T && row < rows) {
          const float2 v = make_float2(acc[c0], acc[c0 + 1]);
          if (!ADJ) {
            out0[((long long)blockIdx.y * T + t) * M + row] = v;
          } else {
            out0[(long long)t * Nf + row] = v;
            if (out1) out1[(long long)t * Nf + row] = c_cjmul(__ldg(f + wrap(row, NP)), v);
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, ncol);
}

// Ht[n][m] = H[m][n], 32 x 32 complex tiles through shared memory
__global__ void __launch_bounds__(256) sense_transpose_kernel(const float2* __restrict__ H, int M, long long Nf,
                                                              float2* __restrict__ Ht) {
  __shared__ float2 tile[32][33];
  const long long n0 = (long long)blockIdx.x * 32;
  const int m0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int i = ty; i < 32; i += 8) {
    const int m = m0 + i;
    const long long n = n0 + tx;
    if (m < M && n < Nf) tile[i][tx] = H[(long long)m * Nf + n];
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    const long long n = n0 + i;
    const int m = m0 + tx;
    if (m < M && n < Nf) Ht[n * M + m] = tile[tx][i];
  }
}

// ------------------------------------------------------------------ host side
bool sense_tc_ok(const cisor_ctx* c) {
  // 16-byte rows of H and Ht (2 Nf and 2 M floats), 2T accumulator columns <= 256
  return c->T <= 128 && c->Nf % 2 == 0 && c->M % 2 == 0;
}

// the kernel instance for nb accumulator columns (sense_tc_cols)
template <int ADJ>
using sense_fn = void (*)(const float*, long long, long long, long long, long long, const float2*, long long,
                          const float2*, long long, int, int, long long, float2*, float2*, int*);
template <int ADJ>
sense_fn<ADJ> sense_kernel_for(int nb) {
  switch (nb) {
    case 32: return sense_tc_kernel<ADJ, 32>;
    case 64: return sense_tc_kernel<ADJ, 64>;
    case 96: return sense_tc_kernel<ADJ, 96>;
    case 128: return sense_tc_kernel<ADJ, 128>;
    case 192: return sense_tc_kernel<ADJ, 192>;
    default: return sense_tc_kernel<ADJ, 256>;
  }
}

// kernel attributes (shared memory, carveout) and the forward kernel's resident CTAs per SM
cisor_status sense_tc_setup(cisor_ctx* c) {
  const int widths[] = {32, 64, 96, 128, 192, 256};
  for (int nb : widths) {
    const int smem = 2 * SPA + 2 * (nb / 8) * SSBO;
    for (const void* fn : {(const void*)sense_kernel_for<0>(nb), (const void*)sense_kernel_for<1>(nb)}) {
      CISOR_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
      CISOR_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    }
  }
  int occ = 0;
  CISOR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, sense_kernel_for<0>(sense_tc_cols(c->T)), STH,
                                                           sense_tc_smem(c->T)));
  c->sense_tc_occ = occ < 1 ? 1 : occ;
  return CISOR_OK;
}

// splits of the forward GEMM's K (2 Nf floats): at least one wave of resident CTAs, at most S_KMAX floats each;
// *KS = floats per split (a multiple of SK)
int sense_tc_splits(const cisor_ctx* c, long long* KS) {
  const long long K = 2 * c->Nf;
  const int mt = (c->M + 127) / 128;
  int S = c->sense_tc_occ * c->sms / mt;
  if (S < 1) S = 1;
  long long ks = ((K + S - 1) / S + SK - 1) / SK * SK;
  if (ks > S_KMAX) ks = S_KMAX;
  if ((K + ks - 1) / ks > S_MAX) ks = ((K + S_MAX - 1) / S_MAX + SK - 1) / SK * SK;  // bounds the partials
  if (KS) *KS = ks;
  return (int)((K + ks - 1) / ks);
}

cisor_status sense_tc_prepare(cisor_ctx* c) {
  if (!c->Ht) return CISOR_OK;
  const dim3 g((unsigned)((c->Nf + 31) / 32), (unsigned)((c->M + 31) / 32));
  sense_transpose_kernel<<<g, 256, 0, c->stream>>>(c->H, c->M, c->Nf, c->Ht);
  CISOR_CUDA(cudaGetLastError());
  return CISOR_OK;
}

// partials of Y = H (f .* u) for ntx transmitters into c->sense_part; *splits receives their count
cisor_status sense_tc_forward(cisor_ctx* c, const float2* f, const float2* u, int ntx, int* splits) {
  long long KS = 0;
  const int S = sense_tc_splits(c, &KS);
  const dim3 g((unsigned)((c->M + 127) / 128), (unsigned)S);
  sense_kernel_for<0>(sense_tc_cols(ntx))<<<g, STH, sense_tc_smem(ntx), c->stream>>>(
      reinterpret_cast<const float*>(c->H), 2 * c->Nf, c->M, 2 * c->Nf, KS, u, c->Nf, f, c->N, ntx, c->M, c->Nf,
      c->sense_part, nullptr, c->tc_err);
  CISOR_CUDA(cudaGetLastError());
  c->tc_used = true;
  *splits = S;
  return CISOR_OK;
}

// z = H^H w and b = conj(f) .* z (b may be null) for ntx transmitters
cisor_status sense_tc_adjoint(cisor_ctx* c, const float2* f, const float2* w, float2* z, float2* b, int ntx) {
  const dim3 g((unsigned)((c->Nf + 127) / 128));
  sense_kernel_for<1>(sense_tc_cols(ntx))<<<g, STH, sense_tc_smem(ntx), c->stream>>>(
      reinterpret_cast<const float*>(c->Ht), 2 * (long long)c->M, c->Nf, 2 * (long long)c->M, 2 * (long long)c->M, w,
      c->M, f, c->N, ntx, c->M, c->Nf, z, b, c->tc_err);
  CISOR_CUDA(cudaGetLastError());
  c->tc_used = true;
  return CISOR_OK;
}

// after a call that ran the kernels above: an error if one of their waits on the tensor cores gave up.  The
// flag lives in mapped host memory, so reading it needs no synchronisation: synced = true when the call has
// already waited for its stream (every kernel it launched has finished), else the flag stays armed and the next
// call that synchronises reports a timeout of this one.
cisor_status sense_tc_check(cisor_ctx* c, bool synced) {
  if (!c->tc_used) return CISOR_OK;
  volatile int* flag = c->h_tc_err;
  if (*flag) {
    *flag = 0;
    c->tc_used = false;
    set_error("sensing: a wait on the tensor cores timed out; the outputs of this or an earlier call are invalid");
    return CISOR_ERR_CUDA;
  }
  if (synced) c->tc_used = false;
  return CISOR_OK;
}

}  // namespace cisor

// ------------------------------------------------------------------ self-test of the bounded waits
namespace cisor {
// One CTA: warp 0 takes 32 TMEM columns, every thread waits at most `polls` polls on an mbarrier that thread 0
// arrives on (arrive = 1) or that nothing completes (arrive = 0), the CTA agrees on the outcome, frees its
// tensor memory and writes 1 (completed) or 0 (gave up) to *out.  The path every tensor-core kernel above
// takes when its MMAs do not complete, without an MMA: nothing faults or hangs.
__global__ void __launch_bounds__(128) tc_wait_selftest_kernel(int arrive, int polls, int* __restrict__ out) {
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) mbar_init(&mbar);
  if (warp == 0) tmem_alloc(&tslot, 32);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (arrive && threadIdx.x == 0)
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&mbar)) : "memory");
  const bool ok = mbar_wait(&mbar, 0, polls);
  const bool all = !__syncthreads_or(!ok);
  if (threadIdx.x == 0) *out = all ? 1 : 0;
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tslot, 32);
}
}  // namespace cisor

extern "C" cisor_status cisor_tc_wait_selftest(int arrive, int polls, int* completed) {
  using namespace cisor;
  if (!completed || polls < 1) {
    set_error("cisor_tc_wait_selftest: NULL output or polls < 1");
    return CISOR_ERR_INVALID_ARG;
  }
  int* d = nullptr;
  CISOR_CUDA(cudaMalloc(&d, sizeof(int)));
  cudaError_t e = cudaMemset(d, 0xff, sizeof(int));
  if (e == cudaSuccess) {
    tc_wait_selftest_kernel<<<1, 128>>>(arrive ? 1 : 0, polls, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(completed, d, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "cisor_tc_wait_selftest", __FILE__, __LINE__);
  return CISOR_OK;
}
