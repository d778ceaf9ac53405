// Detector for the hybrid scheme of Sec. 4.4 (Thm. 4 allows any per-element
// choice between the entropy-split and the Hadamard volume terms; the paper
// leaves the choice of elements open).  The sensor used here: an element is
// troubled when, over its own nodes and the neighbours' facet nodes that
// coincide with its facet nodes, the largest nodal pressure exceeds
// `threshold` times the smallest one, or a pressure there is not positive and
// finite; the flagged set is then widened by one layer of face neighbours.
// The pressure p = (gam-1)(e - (0.5 |m|^2)/rho) is evaluated in this order
// with round-to-nearest intrinsics (no contraction into fused multiply-adds),
// so a host implementation of the same formula reproduces the flags bit for
// bit.  The flags become compacted element lists in element order (one
// block-level scan per 1024 elements, block offsets from the preceding
// blocks' counts; no atomics).  Included by kernels.cu.
#pragma once

namespace esplit {

template <int D>
__device__ __forceinline__ double det_pressure(const double* __restrict__ u, size_t e, int m, int NP, double gm1) {
  constexpr int NC = D + 2;
  double rho = __ldg(&u[(e * NC) * NP + m]);
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double mi = __ldg(&u[(e * NC + 1 + i) * NP + m]);
    s = (i == 0) ? __dmul_rn(mi, mi) : __dadd_rn(s, __dmul_rn(mi, mi));
  }
  double E = __ldg(&u[(e * NC + D + 1) * NP + m]);
  double k = __ddiv_rn(__dmul_rn(0.5, s), rho);
  return __dmul_rn(gm1, __dadd_rn(E, -k));
}

template <int D>
__global__ void __launch_bounds__(256) detect_ratio_kernel(const double* __restrict__ u, const int* __restrict__ pair,
                                                           int n_e, double gm1, double threshold,
                                                           unsigned char* __restrict__ flag0) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_e) return;
  const int NP = c_ref.n_p, NS = c_ref.n_slot;
  double mn = 0.0, mx = 0.0;
  bool bad = false;
  for (int m = 0; m < NP; ++m) {
    double p = det_pressure<D>(u, (size_t)e, m, NP, gm1);
    bad = bad || !(p > 0.0 && p < CUDART_INF);
    mn = (m == 0) ? p : fmin(mn, p);
    mx = (m == 0) ? p : fmax(mx, p);
  }
  for (int s = 0; s < NS; ++s) {
    int v = __ldg(&pair[((size_t)e * NS + s) * 2]);
    int s2 = __ldg(&pair[((size_t)e * NS + s) * 2 + 1]);
    if (v < 0) continue;  // boundary facet: no neighbour node
    double p = det_pressure<D>(u, (size_t)v, c_ref.slot_node[s2], NP, gm1);
    bad = bad || !(p > 0.0 && p < CUDART_INF);
    mn = fmin(mn, p);
    mx = fmax(mx, p);
  }
  double ratio = __ddiv_rn(mx, mn);
  flag0[e] = (bad || !(ratio <= threshold)) ? 1 : 0;
}

// flags = flag0 widened by the face neighbours; per-block flagged counts
__global__ void __launch_bounds__(1024) detect_widen_kernel(const unsigned char* __restrict__ flag0,
                                                            const int* __restrict__ pair, int n_e,
                                                            unsigned char* __restrict__ flags,
                                                            int* __restrict__ bcount) {
  const int NS = c_ref.n_slot;
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  int f = 0;
  if (e < n_e) {
    f = flag0[e];
    for (int s = 0; s < NS; ++s) {
      const int v = __ldg(&pair[((size_t)e * NS + s) * 2]);
      if (v >= 0) f |= flag0[v];  // boundary facets (v = -1) widen nothing
    }
    flags[e] = (unsigned char)f;
  }
  int cnt = __syncthreads_count(f);
  if (threadIdx.x == 0) bcount[blockIdx.x] = cnt;
}

// element lists in element order; total flagged count to *total
__global__ void __launch_bounds__(1024) detect_compact_kernel(const unsigned char* __restrict__ flags,
                                                              const int* __restrict__ bcount, int n_e,
                                                              int* __restrict__ list_split,
                                                              int* __restrict__ list_had, int* __restrict__ total) {
  __shared__ int red[32];
  __shared__ int wcnt[32];
  __shared__ int wex[32];
  __shared__ int base;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // base = flagged elements in the preceding blocks
  int part = 0;
  for (int b = threadIdx.x; b < (int)blockIdx.x; b += blockDim.x) part += bcount[b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
  if (lane == 0) red[w] = part;
  __syncthreads();
  if (w == 0) {
    int v = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) base = v;
  }
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  int f = (e < n_e) ? flags[e] : 0;
  unsigned bal = __ballot_sync(0xffffffffu, f);
  int pre = __popc(bal & ((1u << lane) - 1u));
  if (lane == 0) wcnt[w] = __popc(bal);
  __syncthreads();
  if (w == 0) {
    int v = (lane < (int)(blockDim.x >> 5)) ? wcnt[lane] : 0;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    wex[lane] = incl - v;
  }
  __syncthreads();
  if (e < n_e) {
    int pos = base + wex[w] + pre;  // flagged elements before e
    if (f)
      list_had[pos] = e;
    else
      list_split[e - pos] = e;
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total = base + bcount[blockIdx.x];
}

int launch_detect_hybrid(esplit_ctx* c, const double* u, double threshold, cudaStream_t s) {
  const double gm1 = c->prm.gam - 1.0;
  int nb256 = (c->n_e + 255) / 256;
  int nb1k = (c->n_e + 1023) / 1024;
  if (c->dim == 1)
    detect_ratio_kernel<1><<<nb256, 256, 0, s>>>(u, c->b.pair, c->n_e, gm1, threshold, c->b.hflag0);
  else if (c->dim == 2)
    detect_ratio_kernel<2><<<nb256, 256, 0, s>>>(u, c->b.pair, c->n_e, gm1, threshold, c->b.hflag0);
  else
    detect_ratio_kernel<3><<<nb256, 256, 0, s>>>(u, c->b.pair, c->n_e, gm1, threshold, c->b.hflag0);
  detect_widen_kernel<<<nb1k, 1024, 0, s>>>(c->b.hflag0, c->b.pair, c->n_e, c->b.hflags, c->b.hcount);
  detect_compact_kernel<<<nb1k, 1024, 0, s>>>(c->b.hflags, c->b.hcount, c->n_e, c->b.list_split, c->b.list_had,
                                              c->b.hcount + nb1k);
  c->launches += 3;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace esplit
