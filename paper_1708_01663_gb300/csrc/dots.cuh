// Epilogue inner products shared by the FFT and stencil epilogues.
#pragma once
#include "common.cuh"

namespace cisor {

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
