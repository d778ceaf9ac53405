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

__host__ __device__ constexpr int round32(int n) { return (n + 31) / 32 * 32; }

// The same sums with fewer float64 additions, for blocks of at most NT
// threads (NT a multiple of 32; the kernel's launch bound): every thread
// stores its W values to shared memory, then each full warp sums whole values
// (warp k takes values k, k + n_full_warps, ...: a strided pass of NT/32 - 1
// additions per lane, then the shuffle tree).  The shuffle tree above costs
// every warp 5 W additions; this one costs the block 12 W warp-wide additions
// for NT = 256.  Deterministic (fixed order); the order differs from
// block_sum's.  Blocks of at least 32 threads.
template <int W, int NT>
__device__ __forceinline__ void block_sum_t(const double (&v)[W], double* out_row) {
  static_assert(NT % 32 == 0, "NT is a whole number of warps");
  __shared__ double red[W][NT];
  const int n = blockDim.x;
#pragma unroll
  for (int k = 0; k < W; ++k) red[k][threadIdx.x] = v[k];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n_full = n >> 5;
  if (warp >= n_full) return;
  for (int k = warp; k < W; k += n_full) {
    double x = red[k][lane];
#pragma unroll
    for (int j = 1; j < NT / 32; ++j)
      if (lane + 32 * j < n) x += red[k][lane + 32 * j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) out_row[k] = x;
  }
}

}  // namespace esplit
