// Register-boundary Stockham FFT of length P (64..512) for the complex64 hot path.
//
// P/8 threads cooperate on one transform and each owns 8 elements in
// registers.  Stage s (radix R_s, sub-transform size Ns) runs entirely in
// registers: work item j = t + q P/8 (q < 8/R_s) holds the R_s inputs
// j + r P/R_s, multiplies input r by exp(-+2 pi i r (j mod Ns) / (Ns R_s)),
// and takes a radix-R_s DFT (Stockham autosort, Govindaraju et al., SC 2008).
// Between stages the outputs go to shared memory at (j - j mod Ns) R_s +
// j mod Ns + r Ns and the next stage's inputs are gathered back: a P-point
// transform costs (stages - 1) shared-memory exchanges.  The FIRST stage reads
// its inputs from registers (the caller loads elements t + q P/8 + r P/R_0
// straight from global memory) and the LAST stage leaves its outputs in
// registers (element t + q P/8 + r P/R_L), so the caller writes them without
// another pass.  Plans: 512 = 8.8.8, 256 = 8.8.4, 128 = 8.8.2, 64 = 8.8; the
// reversed plan (REV) starts with the last radix, so a forward transform's
// output registers are exactly the input registers of a REV inverse
// transform: a pointwise product between the two needs no data movement.
#pragma once
#include "common.cuh"
#include "fft.cuh"

namespace cisor {

template <int P> struct RPlan {
  static constexpr int NTF = P / 8;  // threads per transform
  static constexpr int NSTAGE = (P == 64) ? 2 : 3;
  static constexpr int LAST = (P == 512) ? 8 : (P == 256) ? 4 : (P == 128) ? 2 : 8;
  static_assert(P == 64 || P == 128 || P == 256 || P == 512, "unsupported FFT length");
  template <bool REV> __host__ __device__ static constexpr int radix(int s) {
    return NSTAGE == 2 ? 8 : (((REV ? 2 - s : s) == 2) ? LAST : 8);
  }
  template <bool REV> __host__ __device__ static constexpr int first() { return radix<REV>(0); }
  template <bool REV> __host__ __device__ static constexpr int last() { return radix<REV>(NSTAGE - 1); }
  // element held in register q*R + r at the input (R = first radix) / output (R = last radix)
  __host__ __device__ static constexpr int elem(int t, int q, int r, int R) { return t + q * NTF + r * (P / R); }
  // register (q, r) holds an element below P/2 for every t (t < NTF): its offset
  // q NTF + r P/R is a multiple of NTF, so the test is exact
  __host__ __device__ static constexpr bool lower(int q, int r, int R) { return q + r * (8 / R) < 4; }
};

// Shared-memory layouts, chosen so that the 16 threads of a half-warp (which
// move 8-byte elements) hit 16 distinct bank pairs in every exchange pattern
// of the forward and the reversed plans above (checked by enumeration for
// P = 64..512, both column-CTA shapes):
//  rows, first exchange : transform b at base b * row_pitch(P); one pad slot
//                         every 16 elements (P = 64, where a half-warp spans
//                         two transforms: pitch 72 and i ^ ((i >> 3) & 7));
//  rows, second exchange: bits 1-3 of the index flipped by bits 4-6 (P = 512:
//                         bit 3 flipped by bit 6, equally conflict-free there);
//  columns              : element i of column w at W * g(i) + w with
//                         g(i) = i ^ ((i >> 3) & 3), except the reversed plan
//                         of P = 256 at 8 columns per CTA: g(i) = i ^ ((i >> 2) & 1).
__host__ __device__ constexpr int row_pitch(int P) { return P == 64 ? 72 : P + P / 16; }
template <int P> struct RowLayA {
  int base;
  __device__ __forceinline__ int operator()(int i) const {
    return P == 64 ? base + (i ^ ((i >> 3) & 7)) : base + i + (i >> 4);
  }
};
template <int P> struct RowLayB {
  int base;
  __device__ __forceinline__ int operator()(int i) const {
    return P == 512 ? base + (i ^ (((i >> 6) & 1) << 3)) : base + (i ^ (((i >> 4) & 7) << 1));
  }
};
template <int W> struct ColLay {
  int w;
  __device__ __forceinline__ int operator()(int i) const { return W * (i ^ ((i >> 3) & 3)) + w; }
};
template <int P, int W> struct ColLayRev {
  int w;
  __device__ __forceinline__ int operator()(int i) const {
    return (P == 256 && W == 8) ? W * (i ^ ((i >> 2) & 1)) + w : W * (i ^ ((i >> 3) & 3)) + w;
  }
};

// Twiddle table of one plan, stage by stage: stage s (s >= 1, sub-transform
// size NS_s) holds w_s(r, k) = exp(-2 pi i r k / (NS_s R_s)) at
// offset_s + (r - 1) NS_s + k, so the threads of a warp, which have
// consecutive k, read consecutive words (no bank conflicts).
template <int P, bool REV> struct TwTable {
  static constexpr int R0 = RPlan<P>::template radix<REV>(0);
  static constexpr int R1 = RPlan<P>::template radix<REV>(1);
  static constexpr int R2 = RPlan<P>::NSTAGE == 3 ? RPlan<P>::template radix<REV>(2) : 1;
  static constexpr int OFF1 = 0;                      // stage 1: NS = R0
  static constexpr int OFF2 = (R1 - 1) * R0;          // stage 2: NS = R0 R1
  static constexpr int SIZE = OFF2 + (R2 - 1) * R0 * R1;
};
constexpr int TW_STRIDE = 512;  // floats2 reserved per plan table

// a * conj(b)
__device__ __forceinline__ float2 c_mulcj(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// One stage on the thread's registers.  TWALL = false: only w = tws[k] (the
// r = 1 row of the stage table) is read from shared memory and w^2 .. w^7 are
// formed by complex products (depth 3), trading shared-memory loads for FMAs;
// TWALL = true: all R - 1 powers are read from the table (the better trade
// where a warp's threads share few k, so each read is a broadcast).  LO: the
// upper half of each radix-8 input group is zero (first stage only).
template <int P, int R, int NS, bool INV, bool LO = false, bool TWALL = false>
__device__ __forceinline__ void rstage(float2 (&v)[8], int t, const float2* __restrict__ tws) {
  static_assert(!LO || (R == 8 && NS == 1), "pruned inputs only in a radix-8 first stage");
  constexpr int NTF = P / 8;
#pragma unroll
  for (int q = 0; q < 8 / R; ++q) {
    if constexpr (NS > 1 && TWALL) {
      const int k = (t + q * NTF) & (NS - 1);
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const float2 w = tws[(r - 1) * NS + k];
        v[q * R + r] = INV ? c_mulcj(v[q * R + r], w) : c_mul(v[q * R + r], w);
      }
    } else if constexpr (NS > 1) {
      const int j = t + q * NTF;
      const int k = j & (NS - 1);
      float2 w1 = tws[k];
      if (INV) w1.y = -w1.y;
      float2 w[8];
      w[1] = w1;
      if constexpr (R >= 4) {
        w[2] = c_mul(w1, w1);
        w[3] = c_mul(w[2], w1);
      }
      if constexpr (R == 8) {
        w[4] = c_mul(w[2], w[2]);
        w[5] = c_mul(w[4], w1);
        w[6] = c_mul(w[4], w[2]);
        w[7] = c_mul(w[4], w[3]);
      }
#pragma unroll
      for (int r = 1; r < R; ++r) v[q * R + r] = c_mul(v[q * R + r], w[r]);
    }
    if constexpr (LO)
      dft8_lo<INV>(v + q * R);
    else
      dft_r<R, INV>(v + q * R);
  }
}

// Barriers around an exchange.  CtaSync: the whole CTA (transforms that span
// all warps, e.g. the column kernels).  RowSync: row transforms, whose
// exchange regions no other row touches; when a row fits in one warp (P <= 128)
// the warp's own barrier suffices and the rows of a CTA do not wait for one
// another.  Wider rows keep the CTA barrier: per-row named barriers measured
// slower there (the P = 512 row kernel fell from 88 % to 42 % achieved
// occupancy).
struct CtaSync {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
template <int P> struct RowSync {
  int row;
  __device__ __forceinline__ void operator()() const {
    if constexpr (P / 8 >= 32)
      __syncthreads();
    else
      __syncwarp();
  }
};

// outputs of a stage (radix RO, size NS) to shared memory, then the inputs of
// the next stage (radix RI).  PRE: barrier before the writes, needed when an
// earlier exchange read buf with no barrier since.
template <int P, int RO, int NS, int RI, class LAY, class SYNC = CtaSync, bool PRE = true>
__device__ __forceinline__ void rexchange(float2 (&v)[8], float2* buf, const LAY& lay, int t,
                                          const SYNC& sync = SYNC()) {
  constexpr int NTF = P / 8;
  if constexpr (PRE) sync();
#pragma unroll
  for (int q = 0; q < 8 / RO; ++q) {
    const int j = t + q * NTF;
    const int k = j & (NS - 1);
    const int base = (j - k) * RO + k;
#pragma unroll
    for (int r = 0; r < RO; ++r) buf[lay(base + r * NS)] = v[q * RO + r];
  }
  sync();
#pragma unroll
  for (int q = 0; q < 8 / RI; ++q) {
    const int j = t + q * NTF;
#pragma unroll
    for (int r = 0; r < RI; ++r) v[q * RI + r] = buf[lay(j + r * (P / RI))];
  }
}

// Transform the registers v in place (see the file comment for the element
// mapping); tws is this plan's stage twiddle table (TwTable<P, REV>); lay0 and
// lay1 are the shared-memory layouts of the first and second exchange.
// LO_IN: the input is a sequence zero-padded to P from at most P/2 samples.
// With a radix-8 first stage its registers v[4..7] hold elements >= P/2, so
// they are zero; the caller need not set them.  A caller that wants only the
// outputs below P/2 reads v[0..3] of a radix-8 last stage and the compiler
// drops the rest of that stage's butterfly.
// PING (three-stage plans): the second exchange goes through buf2, so neither
// exchange needs a barrier before its writes.  The caller guarantees that
// every read of buf by an earlier exchange is separated from this call by a
// barrier; a three-stage PING transform followed by another one satisfies
// this for both buffers (each exchange's barrier orders the reads of the
// previous exchange, which used the other buffer).
template <int P, bool INV, bool REV, bool LO_IN = false, bool TWALL = false, bool PING = false, class LAY0,
          class LAY1, class SYNC = CtaSync>
__device__ __forceinline__ void reg_fft(float2 (&v)[8], float2* buf, const LAY0& lay0, const LAY1& lay1, int t,
                                        const float2* __restrict__ tws, const SYNC& sync = SYNC(),
                                        float2* buf2 = nullptr) {
  typedef TwTable<P, REV> TT;
  constexpr bool PP = PING && RPlan<P>::NSTAGE == 3;
  rstage<P, TT::R0, 1, INV, LO_IN>(v, t, tws);
  rexchange<P, TT::R0, 1, TT::R1, LAY0, SYNC, !PP>(v, buf, lay0, t, sync);
  rstage<P, TT::R1, TT::R0, INV, false, TWALL>(v, t, tws + TT::OFF1);
  if constexpr (RPlan<P>::NSTAGE == 3) {
    rexchange<P, TT::R1, TT::R0, TT::R2, LAY1, SYNC, !PP>(v, PP ? buf2 : buf, lay1, t, sync);
    rstage<P, TT::R2, TT::R0 * TT::R1, INV, false, TWALL>(v, t, tws + TT::OFF2);
  }
}

}  // namespace cisor
