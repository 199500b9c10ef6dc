// Epilogue inner products shared by the FFT and stencil epilogues.
#pragma once
#include "common.cuh"

namespace cisor {

// Inner-product sets of the inverse-row epilogue.  The solver's three are
// compiled with fixed operands; DOTS_ANY reads the operand codes of ConvOp.
//   DOTS_RV : slot 0 <aux, y>               (<rhat, v>, v = A p)
//   DOTS_TS : slot 1 <y, src>, slot 2 <y, y> (<t, s>, <t, t>, t = A s)
//   DOTS_RES: slot 0 <aux, aux>, slot 2 <y, y> (<b, b>, <r, r>, r = b - A x)
enum { DOTS_NONE = 0, DOTS_RV = 1, DOTS_TS = 2, DOTS_RES = 3, DOTS_ANY = 4 };

inline int dots_kind(const ConvOp& op) {
  auto is = [&](int a0, int b0, int a1, int b1, int a2, int b2) {
    return op.dot_a[0] == a0 && op.dot_b[0] == b0 && op.dot_a[1] == a1 && op.dot_b[1] == b1 &&
           op.dot_a[2] == a2 && op.dot_b[2] == b2;
  };
  if (is(0, 0, 0, 0, 0, 0)) return DOTS_NONE;
  if (is(OP_AUX, OP_Y, 0, 0, 0, 0)) return DOTS_RV;
  if (is(0, 0, OP_Y, OP_SRC, OP_Y, OP_Y)) return DOTS_TS;
  if (is(OP_AUX, OP_AUX, 0, 0, OP_Y, OP_Y)) return DOTS_RES;
  return DOTS_ANY;
}

template <int DK> struct DotSlots {
  static constexpr int MASK = DK == DOTS_NONE ? 0 : DK == DOTS_RV ? 1 : DK == DOTS_TS ? 6 : DK == DOTS_RES ? 5 : 7;
};

__device__ __forceinline__ float2 pick(int code, float2 y, float2 s, float2 a) {
  return code == OP_Y ? y : (code == OP_SRC ? s : a);
}

// Block-wide sum of three complex FP32 partials: warp shuffles, then the
// per-warp sums pairwise in shared memory (all FP32), written to part.  Only
// the slots in MASK (bit s: slot s) are reduced; the others are written as 0.
template <int NT, int MASK = 7>
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
    if (!((MASK >> (k / 2)) & 1)) continue;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 2 * DOT_SLOTS; ++k)
      if ((MASK >> (k / 2)) & 1) red[k][wid] = v[k];
  }
  __syncthreads();
  if (threadIdx.x < 2 * DOT_SLOTS) {
    float* r = red[threadIdx.x];
    float sum = 0.f;
    if ((MASK >> (threadIdx.x / 2)) & 1) {
#pragma unroll
      for (int w = NT / 64; w > 0; w >>= 1)
#pragma unroll
        for (int i = 0; i < w; ++i) r[i] += r[i + w];
      sum = r[0];
    }
    reinterpret_cast<float*>(out)[threadIdx.x] = sum;
  }
}

}  // namespace cisor
