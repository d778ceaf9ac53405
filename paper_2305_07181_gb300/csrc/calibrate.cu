// Measurement aid: float64 throughput of the current device, the denominator
// of the roofline fraction the benchmark reports for the float64 kernels (they
// are bound by the float64 pipe, not by HBM), and the evidence for keeping the
// float64 contractions off the tensor cores.
//
// mode 0: every thread runs CHAINS independent FMA chains (x <- x * a + b);
//         with 8 warps per SM scheduler and 8 chains a thread the pipe never
//         waits on a dependency.  Rate = 2 * FMAs / time.
// mode 1: every warp runs CHAINS independent chains of the float64 tensor-core
//         MMA m8n8k4 (mma.sync, 256 FMAs per warp instruction).
// mode 2: both at once in every warp: CHAINS/2 MMA chains and CHAINS FMA
//         chains per thread, counted together.
// modes 3-6: the costs the kernels' design weighs against a float64 FMA, as
//         operations per second of CHAINS independent chains a thread:
//         3 float32 FMA (x <- x * a + b); 4 float64 divide (x <- a / (x + 1));
//         5 the library's float64 log (x <- log x + 2.5); 6 its float64 exp
//         (x <- exp(-x)); 7 and 8 the CUDA library's float64 log and exp in
//         the same chains; 9 a float64 -> float32 -> float64 round trip and an
//         FMA (x <- (double)(float)(x * a) + b).  Every chain has a stable
//         fixed point (0.62, 3.85, 0.57, 0.1) that its start values lead to,
//         so no value leaves the range the functions are timed on.  The add
//         of modes 4, 5, 7 and the FMA of mode 9 count as part of the
//         operation.
// mode 10: the warp-level bf16 tensor-core MMA (see bf16_mma_rate_kernel),
//         FLOP/s.
#include <cuda_runtime.h>

#include "../../include/esplit.h"
#include "fmath.cuh"

namespace {

constexpr int CHAINS = 8;
constexpr int THREADS = 256;

__device__ double g_calib_sink;

__device__ __forceinline__ void dmma_step(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

__device__ float g_calib_sink32;

// mode 10: the warp-level bf16 tensor-core MMA (mma.sync m16n8k16, float32
// accumulation, 4,096 FLOP per warp instruction), CHAINS independent
// accumulator tiles per warp; the bf16 operands are small constants, so the
// accumulators grow by at most 16 * 2^-14 a step
__global__ void __launch_bounds__(THREADS) bf16_mma_rate_kernel(int iters) {
  float d[CHAINS][4];
#pragma unroll
  for (int j = 0; j < CHAINS; ++j) d[j][0] = d[j][1] = d[j][2] = d[j][3] = 0.0f;
  const unsigned a = 0x3C003C00u;  // two bf16 2^-7
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < CHAINS; ++j)
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
          "{%0, %1, %2, %3};"
          : "+f"(d[j][0]), "+f"(d[j][1]), "+f"(d[j][2]), "+f"(d[j][3])
          : "r"(a), "r"(a), "r"(a), "r"(a), "r"(a), "r"(a));
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < CHAINS; ++j) s += d[j][0] + d[j][1] + d[j][2] + d[j][3];
  if (s == -1.0f) g_calib_sink32 = s;
}

__global__ void __launch_bounds__(THREADS) fp32_rate_kernel(int iters, float a, float b) {
  float x[CHAINS];
#pragma unroll
  for (int j = 0; j < CHAINS; ++j) x[j] = 1.0f + 1e-3f * (threadIdx.x + j);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) x[j] = fmaf(x[j], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < CHAINS; ++j) s += x[j];
  if (s == -1.0f) g_calib_sink32 = s;
}

template <int MODE>
__global__ void __launch_bounds__(THREADS) fp64_rate_kernel(int iters, double a, double b) {
  double x[CHAINS], y0[CHAINS], y1[CHAINS];
#pragma unroll
  for (int j = 0; j < CHAINS; ++j) {
    x[j] = 1.0 + 1e-3 * (threadIdx.x + j);
    y0[j] = 1e-3 * j;
    y1[j] = 2e-3 * j;
  }
  for (int it = 0; it < iters; ++it) {
    if constexpr (MODE == 0 || MODE == 2) {
#pragma unroll
      for (int j = 0; j < CHAINS; ++j) x[j] = fma(x[j], a, b);
    }
    if constexpr (MODE == 1) {
#pragma unroll
      for (int j = 0; j < CHAINS; ++j) dmma_step(y0[j], y1[j], a * 1e-3, b);
    }
    if constexpr (MODE == 2) {
#pragma unroll
      for (int j = 0; j < CHAINS / 2; ++j) dmma_step(y0[j], y1[j], a * 1e-3, b);
    }
    if constexpr (MODE == 4) {
#pragma unroll
      for (int j = 0; j < CHAINS; ++j) x[j] = a / (x[j] + 1.0);
    }
    if constexpr (MODE == 5) {
#pragma unroll
      for (int j = 0; j < CHAINS; ++j) x[j] = esplit::fm::log(x[j]) + 2.5;
    }
    if constexpr (MODE == 6) {
#pragma unroll
      for (int j = 0; j < CHAINS; ++j) x[j] = esplit::fm::exp(-x[j]);
    }
    if constexpr (MODE == 7) {
#pragma unroll
      for (int j = 0; j < CHAINS; ++j) x[j] = ::log(x[j]) + 2.5;
    }
    if constexpr (MODE == 8) {
#pragma unroll
      for (int j = 0; j < CHAINS; ++j) x[j] = ::exp(-x[j]);
    }
    if constexpr (MODE == 9) {
#pragma unroll
      for (int j = 0; j < CHAINS; ++j) x[j] = (double)__double2float_rn(x[j] * a) + b;
    }
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < CHAINS; ++j) s += x[j] + y0[j] + y1[j];
  if (s == -1.0) g_calib_sink = s;  // keeps the chains live; never true for these inputs
}

// FLOPs (modes 0-3: 2 per FMA) or operations (modes 4-6) per launch
template <int MODE>
double ops_per_launch(int blocks, int iters) {
  const double threads = (double)blocks * THREADS;
  const double warps = threads / 32.0;
  double f = 0.0;
  if (MODE == 0 || MODE == 2 || MODE == 3) f += 2.0 * threads * CHAINS * iters;
  if (MODE == 1) f += 2.0 * warps * CHAINS * iters * 256.0;
  if (MODE == 2) f += 2.0 * warps * (CHAINS / 2) * iters * 256.0;
  if (MODE >= 4 && MODE <= 9) f += threads * CHAINS * iters;
  if (MODE == 10) f += warps * CHAINS * iters * 4096.0;
  return f;
}

// iterations a launch, for ~20 ms at the rates measured on GB300
template <int MODE>
constexpr int iters_for() {
  return MODE == 0 ? 4096 : MODE == 3 ? 65536 : MODE == 4 ? 512 : MODE == 5 ? 128 : MODE == 6 ? 256
       : MODE == 7 ? 128 : MODE == 8 ? 256 : MODE == 9 ? 1024 : MODE == 10 ? 16384 : 512;
}

template <int MODE>
int measure(int n_sm, double* rate, double* ms_out) {
  const int blocks = n_sm * 8;  // 2048 threads per SM
  const int iters = iters_for<MODE>();
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return ESPLIT_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return ESPLIT_ERR_CUDA;
  }
  // |a| < 1 keeps every FMA chain bounded (x -> b / (1 - a)); the MMA chains
  // add 4 a b 1e-3 per step from small starting values
  const double a = 0.999999, b = 1e-7;
  float best = 1e30f;
  for (int rep = 0; rep < 6; ++rep) {
    cudaEventRecord(e0, 0);
    if constexpr (MODE == 3)
      fp32_rate_kernel<<<blocks, THREADS>>>(iters, (float)a, (float)b);
    else if constexpr (MODE == 10)
      bf16_mma_rate_kernel<<<blocks, THREADS>>>(iters);
    else
      fp64_rate_kernel<MODE><<<blocks, THREADS>>>(iters, a, b);
    cudaEventRecord(e1, 0);
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;  // the first launch is a warm-up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cudaGetLastError() != cudaSuccess || best >= 1e30f) return ESPLIT_ERR_CUDA;
  *rate = ops_per_launch<MODE>(blocks, iters) / (best * 1e-3);
  if (ms_out) *ms_out = best;
  return ESPLIT_OK;
}

}  // namespace

extern "C" int esplit_measure_fp64(int device, int mode, double* rate, double* ms_out) {
  if (!rate || mode < 0 || mode > 10) return ESPLIT_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return ESPLIT_ERR_CUDA;
  int n_sm = 0;
  if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return ESPLIT_ERR_CUDA;
  switch (mode) {
    case 0: return measure<0>(n_sm, rate, ms_out);
    case 1: return measure<1>(n_sm, rate, ms_out);
    case 2: return measure<2>(n_sm, rate, ms_out);
    case 3: return measure<3>(n_sm, rate, ms_out);
    case 4: return measure<4>(n_sm, rate, ms_out);
    case 5: return measure<5>(n_sm, rate, ms_out);
    case 6: return measure<6>(n_sm, rate, ms_out);
    case 7: return measure<7>(n_sm, rate, ms_out);
    case 8: return measure<8>(n_sm, rate, ms_out);
    case 9: return measure<9>(n_sm, rate, ms_out);
    default: return measure<10>(n_sm, rate, ms_out);
  }
}
