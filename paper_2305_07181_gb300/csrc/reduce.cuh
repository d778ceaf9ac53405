// Block reduction shared by the kernels' entropy-production partials.
#pragma once

#include <cuda_runtime.h>

namespace esplit {

// ---------------------------------------------------------------------------
// block reduction helpers (deterministic: fixed shuffle tree + fixed warp order)
// ---------------------------------------------------------------------------
template <int W>
__device__ __forceinline__ void block_sum(double (&v)[W], double* out_row) {
  __shared__ double red[32][W];
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // a block of EB * NP threads may end in a partial warp: shuffle among the
  // lanes that exist and add only values read from them
  const int nl = min(32, (int)blockDim.x - (warp << 5));
  const unsigned mask = nl == 32 ? 0xffffffffu : ((1u << nl) - 1u);
#pragma unroll
  for (int k = 0; k < W; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_down_sync(mask, v[k], o);
      if (lane + o < nl) v[k] += y;
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < W; ++k) red[warp][k] = v[k];
  }
  __syncthreads();
  if (warp == 0) {
    int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      double x = lane < nw ? red[lane][k] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (lane == 0) out_row[k] = x;
    }
  }
}

}  // namespace esplit
