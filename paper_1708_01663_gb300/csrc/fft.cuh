// Block-level Stockham FFTs in shared memory.
//
// A CTA transforms `nfft` independent sequences of length P (a power of two,
// 64..512).  Element i of sequence b lives at buf[b * fs + i * es].  Each
// stage is the Stockham autosort step (Govindaraju et al., "High performance
// discrete Fourier transforms on graphics processors", SC 2008): work item j
// of a sequence reads R inputs at stride P/R, multiplies input r by the
// twiddle w^(r * (j mod Ns)) with w = exp(-2 pi i / (Ns R)), takes a radix-R
// DFT in registers and writes the outputs at stride Ns starting from
// (j - j mod Ns) R + j mod Ns.  Stages ping-pong between two buffers and the
// result comes out in natural order.  Plan: radix-8 stages, then one radix-4
// or radix-2 stage for the remaining factor.
//
// Twiddles come from a table tw[m] = exp(-2 pi i m / P) (built once in FP64);
// the inverse transform uses conj(tw) and +i in the butterflies (unnormalised).
#pragma once
#include <cuda_runtime.h>

namespace cisor {

template <typename C> struct cx;
template <> struct cx<float2> {
  typedef float R;
  static __device__ __forceinline__ float2 make(float a, float b) { return make_float2(a, b); }
};
template <> struct cx<double2> {
  typedef double R;
  static __device__ __forceinline__ double2 make(double a, double b) { return make_double2(a, b); }
};

template <typename C> __device__ __forceinline__ C f_add(C a, C b) { return cx<C>::make(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C f_sub(C a, C b) { return cx<C>::make(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C f_mul(C a, C b) {
  return cx<C>::make(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * (-i) for the forward transform, a * (+i) for the inverse
template <bool INV, typename C> __device__ __forceinline__ C f_rot(C a) {
  return INV ? cx<C>::make(-a.y, a.x) : cx<C>::make(a.y, -a.x);
}

template <bool INV, typename C> __device__ __forceinline__ void dft2(C& a0, C& a1) {
  C t = a0;
  a0 = f_add(t, a1);
  a1 = f_sub(t, a1);
}

template <bool INV, typename C> __device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
  C t0 = f_add(a0, a2), t1 = f_sub(a0, a2);
  C t2 = f_add(a1, a3), t3 = f_rot<INV>(f_sub(a1, a3));
  a0 = f_add(t0, t2);
  a1 = f_add(t1, t3);
  a2 = f_sub(t0, t2);
  a3 = f_sub(t1, t3);
}

// radix-8 = two radix-4 DFTs (even / odd inputs) joined by w8^k, k = 0..3
template <bool INV, typename C> __device__ __forceinline__ void dft8(C* v) {
  typedef typename cx<C>::R R;
  C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  const R h = (R)0.70710678118654752440;
  // w8 = (1 -+ i)/sqrt2 ; w8^2 = -+i ; w8^3 = (-1 -+ i)/sqrt2
  C w1o = INV ? cx<C>::make(h * (o1.x - o1.y), h * (o1.x + o1.y)) : cx<C>::make(h * (o1.x + o1.y), h * (o1.y - o1.x));
  C w2o = f_rot<INV>(o2);
  C w3o = INV ? cx<C>::make(-h * (o3.x + o3.y), h * (o3.x - o3.y)) : cx<C>::make(h * (o3.y - o3.x), -h * (o3.x + o3.y));
  v[0] = f_add(e0, o0);
  v[4] = f_sub(e0, o0);
  v[1] = f_add(e1, w1o);
  v[5] = f_sub(e1, w1o);
  v[2] = f_add(e2, w2o);
  v[6] = f_sub(e2, w2o);
  v[3] = f_add(e3, w3o);
  v[7] = f_sub(e3, w3o);
}

// radix-8 DFT of inputs whose upper half v[4..7] is zero (the first stage of a
// transform of a zero-padded sequence, padding >= half the length): each
// radix-4 half sees two non-zero inputs, so its first butterfly layer is a
// copy: DFT4(a, b, 0, 0) = (a + b, a + rot(b), a - b, a - rot(b)).
template <bool INV, typename C> __device__ __forceinline__ void dft8_lo(C* v) {
  typedef typename cx<C>::R R;
  const C re1 = f_rot<INV>(v[2]), ro1 = f_rot<INV>(v[3]);
  C e0 = f_add(v[0], v[2]), e1 = f_add(v[0], re1), e2 = f_sub(v[0], v[2]), e3 = f_sub(v[0], re1);
  C o0 = f_add(v[1], v[3]), o1 = f_add(v[1], ro1), o2 = f_sub(v[1], v[3]), o3 = f_sub(v[1], ro1);
  const R h = (R)0.70710678118654752440;
  C w1o = INV ? cx<C>::make(h * (o1.x - o1.y), h * (o1.x + o1.y)) : cx<C>::make(h * (o1.x + o1.y), h * (o1.y - o1.x));
  C w2o = f_rot<INV>(o2);
  C w3o = INV ? cx<C>::make(-h * (o3.x + o3.y), h * (o3.x - o3.y)) : cx<C>::make(h * (o3.y - o3.x), -h * (o3.x + o3.y));
  v[0] = f_add(e0, o0);
  v[4] = f_sub(e0, o0);
  v[1] = f_add(e1, w1o);
  v[5] = f_sub(e1, w1o);
  v[2] = f_add(e2, w2o);
  v[6] = f_sub(e2, w2o);
  v[3] = f_add(e3, w3o);
  v[7] = f_sub(e3, w3o);
}

// cos(pi m / 16) and sin(pi m / 16) for 0 <= m <= 16 (decimal expansions).
__host__ __device__ constexpr double cos16(int m) {
  return m > 8 ? -cos16(16 - m)
               : (m == 0 ? 1.0
                  : m == 1 ? 0.98078528040323044913
                  : m == 2 ? 0.92387953251128675613
                  : m == 3 ? 0.83146961230254523708
                  : m == 4 ? 0.70710678118654752440
                  : m == 5 ? 0.55557023301960222474
                  : m == 6 ? 0.38268343236508977173
                  : m == 7 ? 0.19509032201612826785
                           : 0.0);
}
__host__ __device__ constexpr double sin16(int m) { return m > 8 ? cos16(m - 8) : cos16(8 - m); }

// a * w32^m, w32 = exp(-+2 pi i / 32) (- forward, + inverse), 0 <= m < 16; m = 0 and
// m = 8 (-+i) cost no multiplications
template <bool INV, int M> __device__ __forceinline__ float2 mul_w32(float2 a) {
  if constexpr (M == 0) {
    return a;
  } else if constexpr (M == 8) {
    return f_rot<INV>(a);
  } else {
    constexpr float c = (float)cos16(M), s = INV ? (float)sin16(M) : -(float)sin16(M);
    return make_float2(a.x * c - a.y * s, a.x * s + a.y * c);
  }
}

// radix-16 = two radix-8 DFTs (even / odd inputs) joined by w16^k = w32^(2k), k = 0..7
template <bool INV> __device__ __forceinline__ void dft16(float2* v) {
  float2 e[8], o[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    e[i] = v[2 * i];
    o[i] = v[2 * i + 1];
  }
  dft8<INV>(e);
  dft8<INV>(o);
  const float2 t0 = o[0], t1 = mul_w32<INV, 2>(o[1]), t2 = mul_w32<INV, 4>(o[2]), t3 = mul_w32<INV, 6>(o[3]),
               t4 = mul_w32<INV, 8>(o[4]), t5 = mul_w32<INV, 10>(o[5]), t6 = mul_w32<INV, 12>(o[6]),
               t7 = mul_w32<INV, 14>(o[7]);
  const float2 t[8] = {t0, t1, t2, t3, t4, t5, t6, t7};
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    v[k] = f_add(e[k], t[k]);
    v[k + 8] = f_sub(e[k], t[k]);
  }
}

// w32^k o[k] for k = 0..15 (compile-time exponents)
template <bool INV> __device__ __forceinline__ void mul_w32_ramp(float2* o) {
  o[1] = mul_w32<INV, 1>(o[1]);
  o[2] = mul_w32<INV, 2>(o[2]);
  o[3] = mul_w32<INV, 3>(o[3]);
  o[4] = mul_w32<INV, 4>(o[4]);
  o[5] = mul_w32<INV, 5>(o[5]);
  o[6] = mul_w32<INV, 6>(o[6]);
  o[7] = mul_w32<INV, 7>(o[7]);
  o[8] = mul_w32<INV, 8>(o[8]);
  o[9] = mul_w32<INV, 9>(o[9]);
  o[10] = mul_w32<INV, 10>(o[10]);
  o[11] = mul_w32<INV, 11>(o[11]);
  o[12] = mul_w32<INV, 12>(o[12]);
  o[13] = mul_w32<INV, 13>(o[13]);
  o[14] = mul_w32<INV, 14>(o[14]);
  o[15] = mul_w32<INV, 15>(o[15]);
}

// radix-32 = two radix-16 DFTs (even / odd inputs) joined by w32^k, k = 0..15
template <bool INV> __device__ __forceinline__ void dft32(float2* v) {
  float2 e[16], o[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    e[i] = v[2 * i];
    o[i] = v[2 * i + 1];
  }
  dft16<INV>(e);
  dft16<INV>(o);
  mul_w32_ramp<INV>(o);
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    v[k] = f_add(e[k], o[k]);
    v[k + 16] = f_sub(e[k], o[k]);
  }
}

// radix-32 DFT of inputs whose upper half v[16..31] is zero, split by output
// parity (decimation in frequency): X_2m = DFT16(x)_m, X_2m+1 = DFT16(w32^r x_r)_m.
template <bool INV> __device__ __forceinline__ void dft32_lo(float2* v) {
  float2 a[16], b[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) a[r] = b[r] = v[r];
  mul_w32_ramp<INV>(b);
  dft16<INV>(a);
  dft16<INV>(b);
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    v[2 * m] = a[m];
    v[2 * m + 1] = b[m];
  }
}

// radix-16 DFT of inputs whose upper half v[8..15] is zero, split by output
// parity: X_2m = DFT8(x)_m, X_2m+1 = DFT8(w16^r x_r)_m (w16^r = w32^(2r)).
template <bool INV> __device__ __forceinline__ void dft16_lo(float2* v) {
  float2 a[8], b[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) a[r] = v[r];
  b[0] = v[0];
  b[1] = mul_w32<INV, 2>(v[1]);
  b[2] = mul_w32<INV, 4>(v[2]);
  b[3] = mul_w32<INV, 6>(v[3]);
  b[4] = mul_w32<INV, 8>(v[4]);
  b[5] = mul_w32<INV, 10>(v[5]);
  b[6] = mul_w32<INV, 12>(v[6]);
  b[7] = mul_w32<INV, 14>(v[7]);
  dft8<INV>(a);
  dft8<INV>(b);
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    v[2 * m] = a[m];
    v[2 * m + 1] = b[m];
  }
}

// DFT of N = 8, 16, 32 registers, and of N = 16, 32 registers whose upper half is zero
template <int N, bool INV> __device__ __forceinline__ void dft_n(float2* v) {
  if constexpr (N == 32) dft32<INV>(v);
  else if constexpr (N == 16) dft16<INV>(v);
  else dft8<INV>(v);
}
template <int N, bool INV> __device__ __forceinline__ void dft_n_lo(float2* v) {
  if constexpr (N == 32) dft32_lo<INV>(v);
  else dft16_lo<INV>(v);
}

template <int R, bool INV, typename C> __device__ __forceinline__ void dft_r(C* v) {
  if constexpr (R == 8) dft8<INV>(v);
  else if constexpr (R == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
  else dft2<INV>(v[0], v[1]);
}

// One Stockham stage over all sequences.  FFT_FAST: consecutive threads walk
// consecutive sequences (column layouts, es > 1); otherwise consecutive
// work items of one sequence (row layouts, es = 1).
template <int P, int R, bool INV, bool FFT_FAST, typename C>
__device__ __forceinline__ void fft_stage(const C* __restrict__ in, C* __restrict__ out, int Ns, int nfft, int fs,
                                          int es, const C* __restrict__ tw, int tid, int nthr) {
  constexpr int Q = P / R;
  const int total = nfft * Q;
  for (int w = tid; w < total; w += nthr) {
    int b, j;
    if (FFT_FAST) {
      b = w % nfft;
      j = w / nfft;
    } else {
      b = w / Q;
      j = w % Q;
    }
    const C* src = in + b * fs;
    C* dst = out + b * fs;
    const int k = j & (Ns - 1);
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[(j + r * Q) * es];
    if (Ns > 1) {
      const int step = P / (Ns * R);
#pragma unroll
      for (int r = 1; r < R; ++r) {
        C t = tw[r * k * step];
        if (INV) t.y = -t.y;
        v[r] = f_mul(v[r], t);
      }
    }
    dft_r<R, INV>(v);
    const int d = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[(d + r * Ns) * es] = v[r];
  }
}

template <int P> struct fft_plan {
  static constexpr int n8 = (P == 64) ? 2 : (P == 128) ? 2 : (P == 256) ? 2 : (P == 512) ? 3 : -1;
  static constexpr int rem = (P == 64) ? 1 : (P == 128) ? 2 : (P == 256) ? 4 : (P == 512) ? 1 : -1;
  static_assert(n8 > 0, "unsupported FFT length");
  static constexpr int stages = n8 + (rem > 1 ? 1 : 0);
};

// Full transform.  Input in `a`; returns the buffer that holds the result
// (a or b).  Caller must __syncthreads() after writing `a` and before reading
// the result.
template <int P, bool INV, bool FFT_FAST, typename C>
__device__ __forceinline__ C* block_fft(C* a, C* b, int nfft, int fs, int es, const C* tw, int tid, int nthr) {
  C* in = a;
  C* out = b;
  int Ns = 1;
#pragma unroll
  for (int s = 0; s < fft_plan<P>::n8; ++s) {
    fft_stage<P, 8, INV, FFT_FAST>(in, out, Ns, nfft, fs, es, tw, tid, nthr);
    __syncthreads();
    C* t = in;
    in = out;
    out = t;
    Ns *= 8;
  }
  if constexpr (fft_plan<P>::rem == 4) {
    fft_stage<P, 4, INV, FFT_FAST>(in, out, Ns, nfft, fs, es, tw, tid, nthr);
    __syncthreads();
    C* t = in;
    in = out;
    out = t;
  } else if constexpr (fft_plan<P>::rem == 2) {
    fft_stage<P, 2, INV, FFT_FAST>(in, out, Ns, nfft, fs, es, tw, tid, nthr);
    __syncthreads();
    C* t = in;
    in = out;
    out = t;
  }
  return in;
}

}  // namespace cisor
