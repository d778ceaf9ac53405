// Arithmetic throughput of the GPU it runs on (not part of the library): four
// independent dependency chains per thread, 152 x 8 blocks of 256 threads,
// CUDA-event timing of three launches after one warm-up launch.  Reports
// operations per clock per SM at the device's maximum clock for float64 FMA
// and add, float32 FMA, a float64 -> float32 -> float64 round trip plus an
// add, float64 divide, log and exp, the float64 tensor-core MMA (m8n8k4, 256
// FMAs per warp instruction) alone and interleaved with float64 FMA chains
// (whether the two share a pipe).  These figures set the FP64 roofline peak
// of the residual kernels (FP64-pipe bound) and the cost model of their
// pointwise work.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o probe_arith probe_arith.cu && ./probe_arith
#include <cstdio>
#include <cuda_runtime.h>
#define ITERS 4096
__global__ void k_dfma(double* out, double a, double b) {
  double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  for (int i = 0; i < ITERS; ++i) { x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b); }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3;
}
__global__ void k_ffma(float* out, float a, float b) {
  float x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  for (int i = 0; i < ITERS; ++i) { x0 = fmaf(x0, a, b); x1 = fmaf(x1, a, b); x2 = fmaf(x2, a, b); x3 = fmaf(x3, a, b); }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3;
}
// double -> float -> double round trip (2 conversions per step)
__global__ void k_cvt(double* out, double a) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  for (int i = 0; i < ITERS; ++i) {
    x0 = (double)__double2float_rn(x0) + a; x1 = (double)__double2float_rn(x1) + a;
    x2 = (double)__double2float_rn(x2) + a; x3 = (double)__double2float_rn(x3) + a;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3;
}
__global__ void k_dadd(double* out, double a) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  for (int i = 0; i < ITERS; ++i) { x0 = x0 + a; x1 = x1 + a; x2 = x2 + a; x3 = x3 + a; x0 = x0 + a; x1 = x1 + a; x2 = x2 + a; x3 = x3 + a; }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3;
}
__global__ void k_ddiv(double* out, double a) {
  double x0 = threadIdx.x + 1.5, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  for (int i = 0; i < ITERS / 16; ++i) { x0 = a / x0; x1 = a / x1; x2 = a / x2; x3 = a / x3; }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3;
}
__global__ void k_dlog(double* out, double a) {
  double x0 = threadIdx.x + 1.5, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  for (int i = 0; i < ITERS / 64; ++i) { x0 = log(x0) + a; x1 = log(x1) + a; x2 = log(x2) + a; x3 = log(x3) + a; }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3;
}
__global__ void k_dexp(double* out, double a) {
  double x0 = threadIdx.x * 1e-4, x1 = x0 + 0.1, x2 = x0 + 0.2, x3 = x0 + 0.3;
  for (int i = 0; i < ITERS / 64; ++i) { x0 = exp(-x0) * a; x1 = exp(-x1) * a; x2 = exp(-x2) * a; x3 = exp(-x3) * a; }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3;
}
// D = A B + C, A 8x4 (row), B 4x8 (col), float64; per thread one element of
// A and of B and two of C / D
__device__ __forceinline__ void dmma(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}
__global__ void k_dmma(double* out, double a, double b) {
  double c0 = threadIdx.x * 1e-3, c1 = c0 + 1, c2 = c0 + 2, c3 = c0 + 3, c4 = c0 + 4, c5 = c0 + 5, c6 = c0 + 6,
         c7 = c0 + 7;
  for (int i = 0; i < ITERS / 4; ++i) {
    dmma(c0, c1, a, b); dmma(c2, c3, a, b); dmma(c4, c5, a, b); dmma(c6, c7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = c0 + c1 + c2 + c3 + c4 + c5 + c6 + c7;
}
// the DMMA chains of k_dmma plus the DFMA chains of k_dfma in one loop
__global__ void k_mix(double* out, double a, double b) {
  double c0 = threadIdx.x * 1e-3, c1 = c0 + 1, c2 = c0 + 2, c3 = c0 + 3, c4 = c0 + 4, c5 = c0 + 5, c6 = c0 + 6,
         c7 = c0 + 7;
  double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  for (int i = 0; i < ITERS / 4; ++i) {
    dmma(c0, c1, a, b); dmma(c2, c3, a, b); dmma(c4, c5, a, b); dmma(c6, c7, a, b);
#pragma unroll
    for (int k = 0; k < 4; ++k) { x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b); }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = c0 + c1 + c2 + c3 + c4 + c5 + c6 + c7 + x0 + x1 + x2 + x3;
}
int main() {
  int nb = 152 * 8, nt = 256;
  size_t n = (size_t)nb * nt;
  double* d; float* f;
  cudaMalloc(&d, n * sizeof(double)); cudaMalloc(&f, n * sizeof(float));
  cudaEvent_t a, b; cudaEventCreate(&a); cudaEventCreate(&b);
  int dev; cudaGetDevice(&dev); int clk; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
  double ghz = clk * 1e-6;
  auto run = [&](const char* name, auto launch, double ops_per_thread) {
    launch(); cudaDeviceSynchronize();
    cudaEventRecord(a); for (int r = 0; r < 3; ++r) launch(); cudaEventRecord(b); cudaEventSynchronize(b);
    float ms; cudaEventElapsedTime(&ms, a, b); ms /= 3;
    double ops = ops_per_thread * n;
    double per_clk_sm = ops / (ms * 1e-3) / (ghz * 1e9) / 152;
    printf("%-6s %8.3f ms  %8.2f ops/clk/SM (at %.2f GHz max)  err=%s\n", name, ms, per_clk_sm, ghz,
           cudaGetErrorString(cudaGetLastError()));
  };
  run("dfma", [&] { k_dfma<<<nb, nt>>>(d, 0.999, 1e-3); }, 4.0 * ITERS);
  run("ffma", [&] { k_ffma<<<nb, nt>>>(f, 0.999f, 1e-3f); }, 4.0 * ITERS);
  run("dadd", [&] { k_dadd<<<nb, nt>>>(d, 1e-7); }, 8.0 * ITERS);
  run("cvt2", [&] { k_cvt<<<nb, nt>>>(d, 1e-7); }, 4.0 * ITERS);   // one step = d->f, f->d, dadd
  run("ddiv", [&] { k_ddiv<<<nb, nt>>>(d, 1.0001); }, 4.0 * ITERS / 16);
  run("dlog", [&] { k_dlog<<<nb, nt>>>(d, 1.5); }, 4.0 * ITERS / 64);
  run("dexp", [&] { k_dexp<<<nb, nt>>>(d, 1.0); }, 4.0 * ITERS / 64);
  // per thread: ITERS MMAs of 256 FMAs per warp = 8 FMAs per thread each
  run("dmma", [&] { k_dmma<<<nb, nt>>>(d, 0.999, 1e-3); }, 8.0 * ITERS);
  // DMMA FMAs plus ITERS * 4 DFMAs per thread; if the two share a pipe the
  // time is the sum of the dmma and dfma lines
  run("mix", [&] { k_mix<<<nb, nt>>>(d, 0.999, 1e-3); }, 8.0 * ITERS + 4.0 * ITERS);
  cudaFree(d); cudaFree(f);
  return 0;
}
