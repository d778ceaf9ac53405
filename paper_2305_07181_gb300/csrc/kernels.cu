// CUDA kernels of the entropy-split residual, its Hadamard-form counterpart,
// the entropy functionals and the relaxation RK4 root solve (sm_103a).
//
// Data layout in HBM (float64 unless noted):
//   u, r          [n_e][n_c][n_p]      element-major, node fastest
//   J             [n_e][n_p]
//   nu            [n_e][n_slot][d]     scaled outward normals at facet slots
//   face_pairs    int2 [n_pairs]       (k*n_slot+s, v*n_slot+s'), one per
//                                      coincident facet-node pair
//   ops64/ops32   [n_e][2d][n_p][n_p]  per-element operators, transposed:
//                 k < d: M_i^T with M_i = H^-1 (Q_x_i/(beta+1) + Q_x_i^T)
//                 k >= d: D_i^T with D_i = H^-1 Q_x_i
//   sat           [n_e][n_c][n_slot]   facet (SAT + dissipation) contributions
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include <cstdio>
#include <mutex>
#include <type_traits>

#include "internal.h"
#include "phys.cuh"
#include "visc_flux.cuh"
#include "reduce.cuh"
#include "bits32.cuh"

namespace esplit {

__constant__ RefTables c_ref;

int set_ref_tables(const RefTables& t) {
  if (cudaMemcpyToSymbol(c_ref, &t, sizeof(RefTables)) != cudaSuccess) return -1;
  return set_ref_tables_vjp(t);  // the reverse-mode unit's copy
}

// ---------------------------------------------------------------------------
// per-element operators (run once per mesh upload / beta change)
// Q_x_i = 1/2 sum_j (Lam_ij Q_xi_j - Q_xi_j^T Lam_ij) + 1/2 E_x_i
// ---------------------------------------------------------------------------
template <int D>
__global__ void build_ops_kernel(const double* __restrict__ Qref, const double* __restrict__ Lam,
                                 const double* __restrict__ J, const double* __restrict__ nu, int n_e,
                                 double inv_bp1, double* __restrict__ ops64, float* __restrict__ ops32,
                                 float* __restrict__ ops32lo) {
  const int NP = c_ref.n_p, NS = c_ref.n_slot;
  size_t per = (size_t)2 * D * NP * NP;
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= per * (size_t)n_e) return;
  int e = (int)(idx / per);
  int rem = (int)(idx - (size_t)e * per);
  int k = rem / (NP * NP);
  int nm = rem - k * NP * NP;
  int n = nm / NP, m = nm - n * NP;  // stored entry (k, n, m) = matrix[m][n]
  int i = k % D;
  auto Qx = [&](int a, int b) -> double {
    double s = 0.0;
    for (int j = 0; j < D; ++j) {
      const double* L = Lam + (((size_t)e * D + i) * D + j) * NP;
      s += L[a] * Qref[((size_t)j * NP + a) * NP + b] - Qref[((size_t)j * NP + b) * NP + a] * L[b];
    }
    s *= 0.5;
    if (a == b) {
      int sl = c_ref.node_slot[a];
      if (sl >= 0) s += 0.5 * nu[((size_t)e * NS + sl) * D + i];
    }
    return s;
  };
  double Hm = c_ref.H[m] * J[(size_t)e * NP + m];
  double val;
  if (k < D)
    val = (Qx(m, n) * inv_bp1 + Qx(n, m)) / Hm;
  else
    val = Qx(m, n) / Hm;
  ops64[idx] = val;
  float hi = (float)val;
  ops32[idx] = hi;
  ops32lo[idx] = (float)(val - (double)hi);
}

// row sums M_i 1 and D_i 1 of the stored float64 operators, summed in node
// order: rows[e][k][m] = sum_n ops64[e][k][n][m]
__global__ void build_rows_kernel(const double* __restrict__ ops64, int n_e, int two_d, double* __restrict__ rows) {
  const int NP = c_ref.n_p;
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n_e * two_d * NP) return;
  size_t ek = idx / NP;
  int m = (int)(idx - ek * NP);
  const double* op = ops64 + ek * NP * NP;
  double s = 0.0;
  for (int n = 0; n < NP; ++n) s += op[(size_t)n * NP + m];
  rows[idx] = s;
}

// opsD32[e][i][m][n] = D_i[m][n] (ops32 holds it at [e][d + i][n][m]) for
// n < n_p, zero in the row padding up to npp and after the d n_p npp entries
__global__ void build_opsD_kernel(const float* __restrict__ ops32, int n_e, int d, int np, int npp, int stride,
                                  float* __restrict__ opsD) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n_e * stride) return;
  const size_t e = idx / stride;
  const int j = (int)(idx - e * stride);
  float v = 0.0f;
  if (j < d * np * npp) {
    const int i = j / (np * npp), rem = j - i * np * npp;
    const int m = rem / npp, n = rem - m * npp;
    if (n < np) v = ops32[(((e * 2 * d) + d + i) * np + n) * np + m];
  }
  opsD[idx] = v;
}

// per-node 1/(H_m J_km) and per-slot |nu| and nu/|nu|, formed once here with
// the expressions the facet kernels used to evaluate per node pair (two
// divisions, a square root and d more divisions a pair on the float64 pipe)
template <int D>
__global__ void facet_tables_kernel(const double* __restrict__ J, const double* __restrict__ nu, int n_e,
                                    double* __restrict__ ihd, double* __restrict__ nscale) {
  const int NP = c_ref.n_p, NS = c_ref.n_slot;
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < (size_t)n_e * NP) ihd[idx] = 1.0 / (c_ref.H[idx % NP] * J[idx]);
  if (idx < (size_t)n_e * NS) {
    double nuv[D], b2 = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      nuv[i] = nu[idx * D + i];
      b2 += nuv[i] * nuv[i];
    }
    const double b = sqrt(b2);
    nscale[idx * (D + 1)] = b;
#pragma unroll
    for (int i = 0; i < D; ++i) nscale[idx * (D + 1) + 1 + i] = nuv[i] / b;
  }
}

int launch_build_ops(esplit_ctx* c, cudaStream_t s) {
  size_t total = (size_t)c->n_e * 2 * c->dim * c->n_p * c->n_p;
  int bs = 256;
  unsigned nb = (unsigned)((total + bs - 1) / bs);
  double inv_bp1 = 1.0 / (c->prm.beta + 1.0);
  if (c->dim == 1)
    build_ops_kernel<1><<<nb, bs, 0, s>>>(c->b.Qref, c->b.Lam, c->b.J, c->b.nu, c->n_e, inv_bp1, c->b.ops64,
                                          c->b.ops32, c->b.ops32lo);
  else if (c->dim == 2)
    build_ops_kernel<2><<<nb, bs, 0, s>>>(c->b.Qref, c->b.Lam, c->b.J, c->b.nu, c->n_e, inv_bp1, c->b.ops64,
                                          c->b.ops32, c->b.ops32lo);
  else
    build_ops_kernel<3><<<nb, bs, 0, s>>>(c->b.Qref, c->b.Lam, c->b.J, c->b.nu, c->n_e, inv_bp1, c->b.ops64,
                                          c->b.ops32, c->b.ops32lo);
  size_t nr = (size_t)c->n_e * 2 * c->dim * c->n_p;
  build_rows_kernel<<<(unsigned)((nr + 255) / 256), 256, 0, s>>>(c->b.ops64, c->n_e, 2 * c->dim, c->b.rows);
  c->launches += 2;
  {
    const size_t nn = (size_t)c->n_e * c->n_p, ns = (size_t)c->n_e * c->n_slot, nt = nn > ns ? nn : ns;
    const unsigned nbt = (unsigned)((nt + 255) / 256);
    if (c->dim == 1)
      facet_tables_kernel<1><<<nbt, 256, 0, s>>>(c->b.J, c->b.nu, c->n_e, c->b.ihd, c->b.nscale);
    else if (c->dim == 2)
      facet_tables_kernel<2><<<nbt, 256, 0, s>>>(c->b.J, c->b.nu, c->n_e, c->b.ihd, c->b.nscale);
    else
      facet_tables_kernel<3><<<nbt, 256, 0, s>>>(c->b.J, c->b.nu, c->n_e, c->b.ihd, c->b.nscale);
    c->launches++;
  }
  if (c->b.opsD32) {
    const size_t no = (size_t)c->n_e * c->opsD_stride;
    build_opsD_kernel<<<(unsigned)((no + 255) / 256), 256, 0, s>>>(c->b.ops32, c->n_e, c->dim, c->n_p,
                                                                    npp_for(c->n_p), c->opsD_stride, c->b.opsD32);
    c->launches++;
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// nu . F(u) = sum_i nu_i F^{I(i)}(u), Eq. (5)
template <int D, typename TN>
__device__ __forceinline__ void normal_flux(const Node<double, D>& n, const TN* nuv, double* out) {
  double vn = 0.0;
#pragma unroll
  for (int i = 0; i < D; ++i) vn += (double)nuv[i] * n.V[i];
  double mn = n.rho * vn;
  out[0] = mn;
#pragma unroll
  for (int j = 0; j < D; ++j) out[1 + j] = mn * n.V[j] + n.p * (double)nuv[j];
  out[D + 1] = (n.e + n.p) * vn;
}

// ---------------------------------------------------------------------------
// facet kernel: one thread per coincident facet-node pair (k, m) ~ (v, n).
//   G = sum_i nu_i F*_i(u_km, u_vn) + |nu|/2 X|L|SX^T (w_km - w_vn)
//   sat_k,m = -G / H_k,m ;  sat_v,n = +G / H_v,n       (Eqs. (43), (69))
// For a side whose element takes the entropy-split volume term, the facet
// part of its volume term, H^-1 sum_i E_i f_i = nu . f(u) / H at the node
// (M_i = H^-1 E_i - beta/(beta+1) D_i, see the split volume kernel), is added
// here too, next to the two-point flux it cancels against:
//   ef_mode 0: no side (Hadamard scheme), 1: both sides (split scheme),
//   2: sides whose hybrid flag is 0.
// ---------------------------------------------------------------------------
template <typename T, int D, bool VISC, int FLUX = 0>
__global__ void __launch_bounds__(128) face_kernel(const double* __restrict__ u, const int2* __restrict__ fp,
                                                   int n_pairs, const double* __restrict__ nu,
                                                   const double* __restrict__ ihd,
                                                   const double* __restrict__ nscale, double* __restrict__ sat,
                                                   Phys<T> c, int dissipation, int* __restrict__ status,
                                                   int ef_mode, const unsigned char* __restrict__ hflags,
                                                   int visc_heat, double* __restrict__ ah) {
  constexpr int NC = D + 2;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_pairs) return;
  const int NP = c_ref.n_p, NS = c_ref.n_slot;
  int2 pr = __ldg(&fp[t]);
  int k = pr.x / NS, s = pr.x - k * NS;
  int v = pr.y / NS, s2 = pr.y - v * NS;
  int m = c_ref.slot_node[s], n = c_ref.slot_node[s2];
  T uk[NC], uv[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    uk[q] = (T)__ldg(&u[((size_t)k * NC + q) * NP + m]);
    uv[q] = (T)__ldg(&u[((size_t)v * NC + q) * NP + n]);
  }
  Node<T, D> nk, nv;
  bool ok = node_from_u<T, D>(uk, c, nk);
  ok = node_from_u<T, D>(uv, c, nv) && ok;
  if (!ok) atomicOr(status, 1);
  T nuv[D];
#pragma unroll
  for (int i = 0; i < D; ++i) nuv[i] = (T)__ldg(&nu[((size_t)k * NS + s) * D + i]);
  T G[NC];
  if constexpr (FLUX == 1) {  // Ismail-Roe comparator, with its own dissipation
    IRNode<T, D> ik, iv;
    ir_node<T, D>(nk, ik);
    ir_node<T, D>(nv, iv);
    IRAvg<T, D> a;
    ir_avg<T, D>(ik, iv, c, a);
    ir_flux_dir<T, D>(a, c, nuv, G);
    if (dissipation) {
      const double* ns = nscale + (size_t)pr.x * (D + 1);  // |nu|, nu/|nu| of slot (k, s)
      const T b = (T)__ldg(&ns[0]);
      T nh[D];
#pragma unroll
      for (int i = 0; i < D; ++i) nh[i] = (T)__ldg(&ns[1 + i]);
      T wk[NC], wv[NC], dw[NC], out[NC];
      std_entropy_vars<T, D>(nk, ik, c, wk);
      std_entropy_vars<T, D>(nv, iv, c, wv);
#pragma unroll
      for (int q = 0; q < NC; ++q) dw[q] = wk[q] - wv[q];
      ir_diss_apply<T, D>(a, c, nh, dw, out);
#pragma unroll
      for (int q = 0; q < NC; ++q) G[q] += T(0.5) * b * out[q];
    }
  } else {
    ZNode<T, D> zk, zv;
    znode<T, D>(nk, c, zk);
    znode<T, D>(nv, c, zv);
    znode_recips<T, D>(zk);
    PairAvg<T, D> a;
    pair_avg<T, D>(zk, zv, c, a);
    sy_flux_dir<T, D>(a, c, nuv, G);
    if (dissipation) {
      const double* ns = nscale + (size_t)pr.x * (D + 1);  // |nu|, nu/|nu| of slot (k, s)
      const T b = (T)__ldg(&ns[0]);
      T nh[D];
#pragma unroll
      for (int i = 0; i < D; ++i) nh[i] = (T)__ldg(&ns[1 + i]);
      T dw[NC], out[NC];
#pragma unroll
      for (int q = 0; q < NC; ++q) dw[q] = nk.W[q] - nv.W[q];
      diss_apply<T, D>(a, c, nh, dw, out);
#pragma unroll
      for (int q = 0; q < NC; ++q) G[q] += T(0.5) * b * out[q];
    }
  }
  const double ihk = __ldg(&ihd[(size_t)k * NP + m]), ihv = __ldg(&ihd[(size_t)v * NP + n]);
  double ek[NC], ev[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) ek[q] = ev[q] = 0.0;
  if (ef_mode != 0) {
    bool sk = ef_mode == 1 || hflags[k] == 0;
    bool sv = ef_mode == 1 || hflags[v] == 0;
    if (sk) normal_flux<D>(nk, nuv, ek);
    if (sv) normal_flux<D>(nv, nuv, ev);
  }
  if constexpr (VISC) {
    // BO lift vectors of both sides, a = K~(u)^T (nu (w_k - w_v)), divided by
    // H; the comparator (FLUX 1) in its standard entropy variables
    double b[D][NC], ak[D][NC], av[D][NC];
    if constexpr (FLUX == 1) {
      double wk[NC], wv[NC];
      std_entropy_vars_node(nk, c, wk);
      std_entropy_vars_node(nv, c, wv);
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int q = 0; q < NC; ++q) b[i][q] = nuv[i] * (wk[q] - wv[q]);
      visc_flux_transpose<double, D, double, 1>(nk, c, visc_heat, b, ak);
      visc_flux_transpose<double, D, double, 1>(nv, c, visc_heat, b, av);
    } else {
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int q = 0; q < NC; ++q) b[i][q] = nuv[i] * (nk.W[q] - nv.W[q]);
      visc_flux_transpose<double, D>(nk, c, visc_heat, b, ak);
      visc_flux_transpose<double, D>(nv, c, visc_heat, b, av);
    }
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        ah[(((size_t)k * D + i) * NC + q) * NS + s] = ak[i][q] * ihk;
        ah[(((size_t)v * D + i) * NC + q) * NS + s2] = av[i][q] * ihv;
      }
  }
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    sat[((size_t)k * NC + q) * NS + s] = (ek[q] - (double)G[q]) * ihk;
    sat[((size_t)v * NC + q) * NS + s2] = ((double)G[q] - ev[q]) * ihv;
  }
}

// ---------------------------------------------------------------------------
// facet kernel after the volume kernels (entropy-split or hybrid scheme,
// inviscid, float64): the same terms as face_kernel (two-point flux,
// dissipation, the facet part nu . f / H of the split volume term), with the
// nodal quantities of both sides read from the cache the volume kernels wrote
// (rho, 1/rho, p, e, q, log q, log p, 1/q, 1/p, V) instead of recomputed, and
// the result added into r.  The
// entropy production of the facet terms, w . H sat = w_k . (nu f_k - G) +
// w_v . (G - nu f_v), goes to block partials after the volume kernel's.
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ void node_from_cache(const double* __restrict__ fc, size_t S, size_t ix,
                                                const Phys<double>& c, Node<double, D>& n, double& iq, double& ip) {
  n.rho = __ldg(&fc[0 * S + ix]);
  n.ir = __ldg(&fc[1 * S + ix]);
  n.p = __ldg(&fc[2 * S + ix]);
  n.e = __ldg(&fc[3 * S + ix]);
  n.q = __ldg(&fc[4 * S + ix]);
  n.lnq = __ldg(&fc[5 * S + ix]);
  n.lnp = __ldg(&fc[6 * S + ix]);
  iq = __ldg(&fc[7 * S + ix]);
  ip = __ldg(&fc[8 * S + ix]);
  n.v2 = 0.0;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    n.V[i] = __ldg(&fc[(9 + i) * S + ix]);
    n.v2 += n.V[i] * n.V[i];
  }
  n.W[0] = n.q * (c.w1c * n.p * n.ir - 0.5 * n.v2);
#pragma unroll
  for (int i = 0; i < D; ++i) n.W[1 + i] = n.q * n.V[i];
  n.W[D + 1] = -n.q;
}

template <int D>
__global__ void __launch_bounds__(128) face_cached_kernel(double* __restrict__ r, const int2* __restrict__ fp,
                                                          int n_pairs, const double* __restrict__ nu,
                                                          const double* __restrict__ ihd,
                                                          const double* __restrict__ nscale,
                                                          const double* __restrict__ fc, int n_slot_total,
                                                          Phys<double> c, int dissipation,
                                                          double* __restrict__ prod, int ef_mode,
                                                          const unsigned char* __restrict__ hflags) {
  constexpr int NC = D + 2;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  double hw = 0.0;
  if (t < n_pairs) {
    const int NP = c_ref.n_p, NS = c_ref.n_slot;
    const size_t S = (size_t)n_slot_total;
    int2 pr = __ldg(&fp[t]);
    int k = pr.x / NS, s = pr.x - k * NS;
    int v = pr.y / NS, s2 = pr.y - v * NS;
    int m = c_ref.slot_node[s], n = c_ref.slot_node[s2];
    Node<double, D> nk, nv;
    double iqk, ipk, iqv, ipv;
    node_from_cache<D>(fc, S, (size_t)pr.x, c, nk, iqk, ipk);
    node_from_cache<D>(fc, S, (size_t)pr.y, c, nv, iqv, ipv);
    ZNode<double, D> zk, zv;
    znode<double, D>(nk, c, zk);
    znode<double, D>(nv, c, zv);
    zk.iq = iqk;
    zk.ip = ipk;
    PairAvg<double, D> a;
    pair_avg<double, D>(zk, zv, c, a);
    double nuv[D];
#pragma unroll
    for (int i = 0; i < D; ++i) nuv[i] = __ldg(&nu[((size_t)k * NS + s) * D + i]);
    double G[NC];
    sy_flux_dir<double, D>(a, c, nuv, G);
    if (dissipation) {
      const double* ns = nscale + (size_t)pr.x * (D + 1);  // |nu|, nu/|nu| of slot (k, s)
      const double b = __ldg(&ns[0]);
      double nh[D];
#pragma unroll
      for (int i = 0; i < D; ++i) nh[i] = __ldg(&ns[1 + i]);
      double dw[NC], out[NC];
#pragma unroll
      for (int q = 0; q < NC; ++q) dw[q] = nk.W[q] - nv.W[q];
      diss_apply<double, D>(a, c, nh, dw, out);
#pragma unroll
      for (int q = 0; q < NC; ++q) G[q] += 0.5 * b * out[q];
    }
    // the facet part nu . f / H of the split volume term, for split-form sides
    // (ef_mode 1: both, 2: sides whose hybrid flag is 0, 0: none)
    double ek[NC], ev[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) ek[q] = ev[q] = 0.0;
    if (ef_mode == 1 || (ef_mode == 2 && __ldg(&hflags[k]) == 0)) normal_flux<D>(nk, nuv, ek);
    if (ef_mode == 1 || (ef_mode == 2 && __ldg(&hflags[v]) == 0)) normal_flux<D>(nv, nuv, ev);
    const double ihk = __ldg(&ihd[(size_t)k * NP + m]), ihv = __ldg(&ihd[(size_t)v * NP + n]);
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      double gk = ek[q] - G[q], gv = G[q] - ev[q];
      r[((size_t)k * NC + q) * NP + m] += gk * ihk;
      r[((size_t)v * NC + q) * NP + n] += gv * ihv;
      hw += nk.W[q] * gk + nv.W[q] * gv;
    }
  }
  if (prod) {
    double vv[1] = {hw};
    block_sum_t<1, 128>(vv, prod + blockIdx.x);
  }
}

// ---------------------------------------------------------------------------
// boundary facet slots (pair (-1, -1), bounded domains): the terms of
// face_kernel for side k alone, with the neighbour's state replaced by the
// prescribed exterior state u_b:
//   G = nu . F*(u_km, u_b) + |nu|/2 X|L|SX^T (w_km - w_b),
//   H_k,m r_k,m gets nu . f(u_km) [split-form element] - G.
// ADD = false: written to the facet scratch before the volume kernels (which
// add it); ADD = true: added into r after them, with the entropy-production
// block partials w . (H r) when prod is given.  FLUX 1: the Ismail-Roe
// comparator with its dissipation (standard entropy variables).
// ---------------------------------------------------------------------------
template <int D, int FLUX, bool ADD>
__global__ void __launch_bounds__(128) face_bc_kernel(const double* __restrict__ u, const int* __restrict__ bslot,
                                                      const double* __restrict__ bstate, int n_b,
                                                      const double* __restrict__ nu, const double* __restrict__ J,
                                                      double* __restrict__ out, Phys<double> c, int dissipation,
                                                      int* __restrict__ status, int ef_mode,
                                                      const unsigned char* __restrict__ hflags,
                                                      double* __restrict__ prod) {
  constexpr int NC = D + 2;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double hw = 0.0;
  if (t < n_b) {
    const int NP = c_ref.n_p, NS = c_ref.n_slot;
    const int a = __ldg(&bslot[t]);
    const int k = a / NS, s = a - k * NS;
    const int m = c_ref.slot_node[s];
    double uk[NC], ub[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      uk[q] = __ldg(&u[((size_t)k * NC + q) * NP + m]);
      ub[q] = __ldg(&bstate[(size_t)t * NC + q]);
    }
    Node<double, D> nk, nb;
    bool ok = node_from_u<double, D>(uk, c, nk);
    ok = node_from_u<double, D>(ub, c, nb) && ok;
    if (!ok) atomicOr(status, 1);
    double nuv[D], nh[D], b2 = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      nuv[i] = __ldg(&nu[((size_t)k * NS + s) * D + i]);
      b2 += nuv[i] * nuv[i];
    }
    const double b = sqrt(b2);
#pragma unroll
    for (int i = 0; i < D; ++i) nh[i] = nuv[i] / b;
    double G[NC], dw[NC], o[NC];
    if constexpr (FLUX == 1) {
      IRNode<double, D> ik, ib;
      ir_node<double, D>(nk, ik);
      ir_node<double, D>(nb, ib);
      IRAvg<double, D> av;
      ir_avg<double, D>(ik, ib, c, av);
      ir_flux_dir<double, D>(av, c, nuv, G);
      if (dissipation) {
        double wk[NC], wb[NC];
        std_entropy_vars<double, D>(nk, ik, c, wk);
        std_entropy_vars<double, D>(nb, ib, c, wb);
#pragma unroll
        for (int q = 0; q < NC; ++q) dw[q] = wk[q] - wb[q];
        ir_diss_apply<double, D>(av, c, nh, dw, o);
#pragma unroll
        for (int q = 0; q < NC; ++q) G[q] += 0.5 * b * o[q];
      }
    } else {
      ZNode<double, D> zk, zb;
      znode<double, D>(nk, c, zk);
      znode<double, D>(nb, c, zb);
      znode_recips<double, D>(zk);
      PairAvg<double, D> av;
      pair_avg<double, D>(zk, zb, c, av);
      sy_flux_dir<double, D>(av, c, nuv, G);
      if (dissipation) {
#pragma unroll
        for (int q = 0; q < NC; ++q) dw[q] = nk.W[q] - nb.W[q];
        diss_apply<double, D>(av, c, nh, dw, o);
#pragma unroll
        for (int q = 0; q < NC; ++q) G[q] += 0.5 * b * o[q];
      }
    }
    double ek[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) ek[q] = 0.0;
    if (ef_mode == 1 || (ef_mode == 2 && __ldg(&hflags[k]) == 0)) normal_flux<D>(nk, nuv, ek);
    const double ihk = 1.0 / (c_ref.H[m] * __ldg(&J[(size_t)k * NP + m]));
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      const double g = ek[q] - G[q];
      if constexpr (ADD) {
        out[((size_t)k * NC + q) * NP + m] += g * ihk;
        hw += nk.W[q] * g;
      } else {
        out[((size_t)k * NC + q) * NS + s] = g * ihk;
      }
    }
  }
  if (ADD && prod) {
    double vv[1] = {hw};
    block_sum_t<1, 128>(vv, prod + blockIdx.x);
  }
}

template <int D>
static int face_bc_d(esplit_ctx* c, const double* u, double* out, int add, double* prod, cudaStream_t s) {
  const Phys<double> ph = make_phys<double>(c->prm.gam, c->prm.beta, c->prm.R, c->prm.mu, c->prm.Pr);
  const int sch = c->prm.scheme;
  const int ef_mode = sch == ESPLIT_SCHEME_SPLIT ? 1 : (sch == ESPLIT_SCHEME_HYBRID ? 2 : 0);
  const int bs = 128, nb = (c->n_bslot + bs - 1) / bs;
  ProfScope ps(c, PG_FACE, s);
  if (add)
    face_bc_kernel<D, 0, true><<<nb, bs, 0, s>>>(u, c->b.bslot, c->b.bstate, c->n_bslot, c->b.nu, c->b.J, out, ph,
                                                 c->prm.dissipation, c->b.status, ef_mode, c->b.hflags, prod);
  else if (sch == ESPLIT_SCHEME_HADAMARD_IR)
    face_bc_kernel<D, 1, false><<<nb, bs, 0, s>>>(u, c->b.bslot, c->b.bstate, c->n_bslot, c->b.nu, c->b.J, out,
                                                  ph, c->prm.dissipation, c->b.status, 0, c->b.hflags, nullptr);
  else
    face_bc_kernel<D, 0, false><<<nb, bs, 0, s>>>(u, c->b.bslot, c->b.bstate, c->n_bslot, c->b.nu, c->b.J, out,
                                                  ph, c->prm.dissipation, c->b.status, ef_mode, c->b.hflags, nullptr);
  c->launches++;
  return (add && prod) ? nb : 0;
}

int launch_face_bc(esplit_ctx* c, const double* u, double* out, int add, double* prod, cudaStream_t s) {
  if (c->n_bslot == 0) return 0;
  if (c->dim == 1) return face_bc_d<1>(c, u, out, add, prod, s);
  if (c->dim == 2) return face_bc_d<2>(c, u, out, add, prod, s);
  return face_bc_d<3>(c, u, out, add, prod, s);
}

// ---------------------------------------------------------------------------
// entropy-split volume kernel (Eq. (100)): EB elements per block, one thread
// per node.  With M_i = H^-1 (Q_i/(beta+1) + Q_i^T) and Q_i + Q_i^T = E_i
// (Def. 1, E_i diagonal), M_i = H^-1 E_i - beta/(beta+1) D_i, so
//   r = H^-1 sum_i E_i f_i - beta/(beta+1) sum_i D_i f_i
//       - 1/(beta+1) sum_i A~_i (D_i w) + sat:
// only the D_i are applied (one operator entry serves the flux and the
// entropy-variable contraction); the E_i term is pointwise at the facet
// nodes (E_i = diag(nu_i) there) and the facet kernel adds it to the facet
// contributions.
//
// Node states, fluxes, entropy variables and the A~_i products are float64 in
// both precision modes.  T = double: plain float64 contractions.  T = float
// (FP32-bulk): the contractions act in float32 on the variation inside the
// element, relative to its node 0, and the node-0 values come back through
// the float64 row sums of the stored operators,
//   D_i f_i = D_i (f_i - f_i,0) + f_i,0 (D_i 1),  D_i w = D_i (w - w_0) + w_0 (D_i 1).
// Operator entries and variations are each held as an unevaluated float32
// sum hi + lo, and the products are accumulated by the compensated dot
// product of Ogita, Rump and Oishi (Dot2, SIAM J. Sci. Comput. 26, 2005):
// the rounding error of every product (exact through fmaf) and of every
// addition (TwoSum) goes to a second float32 accumulator, together with the
// cross terms hi*lo.  At low Mach number the energy-flux variation inside an
// element is ~(E + p)|dV|, hundreds of times the residual, and a plain
// float32 product would lose that factor.
// Optional: block partial of sum H w^T r (entropy production, float64).
// ---------------------------------------------------------------------------
template <typename T, int D, int NP, int EB>
struct SplitSmem {
  double rf[EB][D][D + 2][NP];  // fluxes
  double rw[EB][D + 2][NP];     // entropy variables
  T sf[EB][D][D + 2][NP];       // float32 variations, hi and lo parts (FP32-bulk only)
  T sw[EB][D + 2][NP];
  T sfl[EB][D][D + 2][NP];
  T swl[EB][D + 2][NP];
};

// acc + cmp += (ah + al) (bh + bl), Dot2 step: exact product error by fmaf,
// TwoSum for the addition; intrinsics keep the compiler from fusing them.
__device__ __forceinline__ void dot2_step(float ah, float al, float bh, float bl, float& acc, float& cmp) {
  float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  float s = __fadd_rn(acc, p);
  float z = __fsub_rn(s, acc);
  float t = __fadd_rn(__fsub_rn(acc, __fsub_rn(s, z)), __fsub_rn(p, z));
  acc = s;
  cmp = __fadd_rn(cmp, __fadd_rn(t, e));
}
template <int D, int NP, int EB>
struct SplitSmem<double, D, NP, EB> {
  double rf[EB][D][D + 2][NP];
  double rw[EB][D + 2][NP];
};

template <typename T, int D, int NP, int EB, bool VISC, bool CACHE = false, bool ENT = false>
__global__ void __launch_bounds__(EB * NP, (sizeof(T) == 4 && !VISC && D == 2) ? 4 : ((VISC && D == 3) ? 2 : 1)) split_volume_kernel(
    const double* __restrict__ u, double* __restrict__ r, const T* __restrict__ ops,
    const float* __restrict__ opslo, const double* __restrict__ rows, const double* __restrict__ J,
    const double* __restrict__ sat, const int* __restrict__ list, int n_list, Phys<T> c, Phys<double> c64,
    int* __restrict__ status, double* __restrict__ prod, int visc_heat, const double* __restrict__ nu,
    const double* __restrict__ ah, double* __restrict__ fvs, const double* __restrict__ ops64,
    double* __restrict__ fcache, int n_slot_total, double* __restrict__ ent_part = nullptr,
    double* __restrict__ ncache = nullptr, double* __restrict__ wsl = nullptr) {
  constexpr int NC = D + 2;
  constexpr bool F64 = sizeof(T) == sizeof(double);
  __shared__ SplitSmem<T, D, NP, EB> sm;
  const int NS = c_ref.n_slot;
  int el = threadIdx.x / NP;
  int m = threadIdx.x - el * NP;
  int li = blockIdx.x * EB + el;
  bool active = (el < EB) && (li < n_list);
  int e = active ? (list ? list[li] : li) : 0;
  Node<double, D> nd;
  if (active) {
    double uu[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) uu[q] = __ldg(&u[((size_t)e * NC + q) * NP + m]);
    if (!node_from_u<double, D>(uu, c64, nd)) atomicOr(status, 1);
#pragma unroll
    for (int i = 0; i < D; ++i) {
      double F[NC];
      euler_flux<double, D>(nd, i, F);
#pragma unroll
      for (int q = 0; q < NC; ++q) sm.rf[el][i][q][m] = F[q];
    }
#pragma unroll
    for (int q = 0; q < NC; ++q) sm.rw[el][q][m] = nd.W[q];
  }
  __syncthreads();
  if constexpr (!F64) {
    if (active) {
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int q = 0; q < NC; ++q) {
          float hi, lo;
          split_f64(sm.rf[el][i][q][m] - sm.rf[el][i][q][0], hi, lo);
          sm.sf[el][i][q][m] = hi;
          sm.sfl[el][i][q][m] = lo;
        }
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        float hi, lo;
        split_f64(sm.rw[el][q][m] - sm.rw[el][q][0], hi, lo);
        sm.sw[el][q][m] = hi;
        sm.swl[el][q][m] = lo;
      }
    }
    __syncthreads();
  }
  double hw = 0.0, ent_s = 0.0, ent_a = 0.0;
  const int sl = c_ref.node_slot[m];
  const T* op = ops + (size_t)e * (2 * D * NP * NP);
  const double* op64 = VISC ? ops64 + (size_t)e * (2 * D * NP * NP) : nullptr;
  double res[NC], Fp[D][NC], Hm = 0.0;
  if (active) {
    T acc[NC], g[D][NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) acc[q] = T(0);
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int q = 0; q < NC; ++q) g[i][q] = T(0);
    const float* oplo = F64 ? nullptr : opslo + (size_t)e * (2 * D * NP * NP);
    // float32 sums: second accumulators of the compensated dot products
    T cacc[NC], cg[D][NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) cacc[q] = T(0);
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int q = 0; q < NC; ++q) cg[i][q] = T(0);
#pragma unroll
    for (int i = 0; i < D; ++i) {
#pragma unroll 4
      for (int n = 0; n < NP; ++n) {
        T dt = __ldg(&op[((D + i) * NP + n) * NP + m]);
        float dtl = 0.f;
        if constexpr (!F64) dtl = __ldg(&oplo[((D + i) * NP + n) * NP + m]);
#pragma unroll
        for (int q = 0; q < NC; ++q) {
          if constexpr (F64) {
            acc[q] += dt * sm.rf[el][i][q][n];
            g[i][q] += dt * sm.rw[el][q][n];
          } else {
            dot2_step(dt, dtl, sm.sf[el][i][q][n], sm.sfl[el][i][q][n], acc[q], cacc[q]);
            dot2_step(dt, dtl, sm.sw[el][q][n], sm.swl[el][q][n], g[i][q], cg[i][q]);
          }
        }
      }
    }
    double accd[NC], gd[D][NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      if constexpr (F64)
        accd[q] = acc[q];
      else
        accd[q] = widen_f32(acc[q]) + widen_f32(cacc[q]);
    }
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        if constexpr (F64)
          gd[i][q] = g[i][q];
        else
          gd[i][q] = widen_f32(g[i][q]) + widen_f32(cg[i][q]);
      }
    if constexpr (!F64) {
      // add back the node-0 values through the stored operators' row sums
      const double* rs = rows + (size_t)e * (2 * D * NP);
#pragma unroll
      for (int i = 0; i < D; ++i) {
        double rd = __ldg(&rs[(D + i) * NP + m]);
#pragma unroll
        for (int q = 0; q < NC; ++q) {
          accd[q] += sm.rf[el][i][q][0] * rd;  // node-0 values, re-read (fewer live registers)
          gd[i][q] += sm.rw[el][q][0] * rd;
        }
      }
    }
    const JvpPrep<double> jp = jvp_prep<double, D>(nd, c64);
    if constexpr (ENT) {
      // entropy of u_n for the relaxation step (the entropy kernel's outputs):
      // S_H = beta q p, and the per-node values its evaluation passes reuse
      const size_t nn = (size_t)n_list * NP, g = (size_t)e * NP + m;
      const double sH = c64.beta * nd.q * nd.p;
      ncache[g] = sH;
      ncache[nn + g] = nd.ir;
      ncache[2 * nn + g] = jp.itheta * nd.ir;  // 1/p
      const double Hm0 = c_ref.H[m] * __ldg(&J[(size_t)e * NP + m]);
      ent_s = Hm0 * sH;
      ent_a = Hm0 * fabs(sH);
    }
    if constexpr (CACHE) {
      // nodal quantities of the facet nodes for the facet kernel that runs after
      // this one (it then needs no logarithm, exponential or division for them)
      const int sl0 = c_ref.node_slot[m];
      if (sl0 >= 0) {
        const size_t S = (size_t)n_slot_total, ix = (size_t)e * NS + sl0;
        fcache[0 * S + ix] = nd.rho;
        fcache[1 * S + ix] = nd.ir;
        fcache[2 * S + ix] = nd.p;
        fcache[3 * S + ix] = nd.e;
        fcache[4 * S + ix] = nd.q;
        fcache[5 * S + ix] = nd.lnq;
        fcache[6 * S + ix] = nd.lnp;
        fcache[7 * S + ix] = jp.iq;
        fcache[8 * S + ix] = jp.itheta * nd.ir;  // 1/p
#pragma unroll
        for (int i = 0; i < D; ++i) fcache[(9 + i) * S + ix] = nd.V[i];
      }
    }
    double nonc[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) nonc[q] = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      double dF[NC];
      dflux_dw<double, D>(nd, jp, c64, i, gd[i], dF);
#pragma unroll
      for (int q = 0; q < NC; ++q) nonc[q] += dF[q];
    }
    Hm = c_ref.H[m] * __ldg(&J[(size_t)e * NP + m]);
    const double kf = c64.beta * c64.inv_bp1;
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      // the facet contributions include H^-1 sum_i E_i f_i (added by the facet kernel)
      res[q] = -kf * accd[q] - c64.inv_bp1 * nonc[q];
      if (!CACHE && sl >= 0) res[q] += __ldg(&sat[((size_t)e * NC + q) * NS + sl]);
    }
    if constexpr (VISC) {
      {
        // viscous flux from the gradients just formed (gd = D_i w), plus the
        // folded BO lift a/(2H) at the facet nodes; F^V kept for the flux jump
        visc_flux<double, D>(nd, c64, visc_heat, gd, Fp);
        if (sl >= 0 && wsl) {
          // entropy variables at the facet slot, for the flux-jump kernel's
          // share of the entropy production
#pragma unroll
          for (int q = 0; q < NC; ++q) wsl[((size_t)e * NC + q) * NS + sl] = nd.W[q];
        }
        if (sl >= 0) {
#pragma unroll
          for (int i = 0; i < D; ++i)
#pragma unroll
            for (int q = 0; q < NC; ++q) {
              size_t ix = (((size_t)e * D + i) * NC + q) * NS + sl;
              fvs[ix] = Fp[i][q];
              Fp[i][q] += 0.5 * __ldg(&ah[ix]);
            }
        }
      }
    }
  }
  if constexpr (VISC) {  // float64 in both precision modes
    {
      __syncthreads();      // every thread is done with the fluxes in sm.rf
      if (active) {
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
          for (int q = 0; q < NC; ++q) sm.rf[el][i][q][m] = Fp[i][q];
      }
      __syncthreads();
      if (active) {
        // sum_i D_i (F^V_i + a_i/(2H)) - sum_i nu_i a_i/(2H^2) at the facet nodes
#pragma unroll
        for (int i = 0; i < D; ++i) {
#pragma unroll 4
          for (int n = 0; n < NP; ++n) {
            double dt = __ldg(&op64[((D + i) * NP + n) * NP + m]);
#pragma unroll
            for (int q = 0; q < NC; ++q) res[q] += dt * sm.rf[el][i][q][n];
          }
        }
        if (sl >= 0) {
          const double ih = 1.0 / Hm;
          double nv[D];
#pragma unroll
          for (int i = 0; i < D; ++i) nv[i] = __ldg(&nu[((size_t)e * NS + sl) * D + i]);
#pragma unroll
          for (int q = 0; q < NC; ++q) {
            double corr = 0.0;
#pragma unroll
            for (int i = 0; i < D; ++i) corr += nv[i] * __ldg(&ah[(((size_t)e * D + i) * NC + q) * NS + sl]);
            res[q] -= 0.5 * corr * ih;
          }
        }
      }
    }
  }
  if (active) {
#pragma unroll
    for (int q = 0; q < NC; ++q) r[((size_t)e * NC + q) * NP + m] = res[q];
    if (prod) {
#pragma unroll
      for (int q = 0; q < NC; ++q) hw += nd.W[q] * res[q];
      hw *= Hm;
    }
  }
  if (prod) {
    double v[1] = {hw};
    block_sum_t<1, round32(EB * NP)>(v, prod + blockIdx.x);
  }
  if constexpr (ENT) {
    __syncthreads();  // the block sum's shared scratch is reused
    double v2[2] = {ent_s, ent_a};
    block_sum_t<2, round32(EB * NP)>(v2, ent_part + 2 * blockIdx.x);
  }
}

// ---------------------------------------------------------------------------
// Hadamard-form volume kernel (Eq. (99)), Sjogreen-Yee flux, each unordered
// node pair evaluated once: thread m takes pairs (m, m+k mod NP),
// k = 1..NP/2 (k = NP/2 only for m < NP/2 when NP is even), and hands the
// partner's share through shared memory (no atomics).
//   G = sum_i S_i[m][n] F*_i(u_m, u_n),  S_i[m][n] = H_m D_i[m][n]
//   r_m -= 2 G / H_m,  r_n += 2 G / H_n
// ---------------------------------------------------------------------------
template <typename T, int D, int NP, int EB, int FLUX = 0, int KC = NP / 2>
__global__ void __launch_bounds__(EB * NP) hadamard_volume_kernel(
    const double* __restrict__ u, double* __restrict__ r, const T* __restrict__ ops,
    const double* __restrict__ J, const double* __restrict__ sat, const int* __restrict__ list, int n_list,
    Phys<T> c, Phys<double> c64, int* __restrict__ status, double* __restrict__ prod,
    double* __restrict__ fcache = nullptr, int n_slot_total = 0) {
  constexpr int NC = D + 2;
  constexpr int K = NP / 2;
  constexpr int NZ = D + 7;  // q, V[D], p, P1, P2, v2, 1/q, 1/p
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sz = reinterpret_cast<T*>(smem_raw);           // [EB][NZ][NP]
  T* sg = sz + EB * NZ * NP;                         // [EB][NP][KC][NC]
  T* sH = sg + EB * NP * KC * NC;                    // [EB][NP]
  const int NS = c_ref.n_slot;
  int el = threadIdx.x / NP;
  int m = threadIdx.x - el * NP;
  int li = blockIdx.x * EB + el;
  bool active = (el < EB) && (li < n_list);
  int e = active ? (list ? list[li] : li) : 0;
  Node<T, D> nd;
  if (active) {
    T uu[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) uu[q] = (T)__ldg(&u[((size_t)e * NC + q) * NP + m]);
    if (!node_from_u<T, D>(uu, c, nd)) atomicOr(status, 1);
    T* zz = sz + el * NZ * NP;
    if constexpr (FLUX == 1) {  // Ismail-Roe: z_1, z_nc, their logs, V
      IRNode<T, D> z;
      ir_node<T, D>(nd, z);
      zz[0 * NP + m] = z.z1;
      zz[1 * NP + m] = z.zn;
      zz[2 * NP + m] = z.l1;
      zz[3 * NP + m] = z.ln;
#pragma unroll
      for (int i = 0; i < D; ++i) zz[(4 + i) * NP + m] = z.V[i];
    } else {
      ZNode<T, D> z;
      znode<T, D>(nd, c, z);
      znode_recips<T, D>(z);
      if constexpr (sizeof(T) == sizeof(double)) {
        // nodal quantities of the facet nodes for the cached facet kernel
        // (Hadamard and hybrid schemes; for the hybrid scheme the split
        // volume kernel writes the others)
        const int sl0 = c_ref.node_slot[m];
        if (fcache && sl0 >= 0) {
          const size_t S = (size_t)n_slot_total, ix = (size_t)e * NS + sl0;
          fcache[0 * S + ix] = nd.rho;
          fcache[1 * S + ix] = nd.ir;
          fcache[2 * S + ix] = nd.p;
          fcache[3 * S + ix] = nd.e;
          fcache[4 * S + ix] = nd.q;
          fcache[5 * S + ix] = nd.lnq;
          fcache[6 * S + ix] = nd.lnp;
          fcache[7 * S + ix] = z.iq;
          fcache[8 * S + ix] = z.ip;
#pragma unroll
          for (int i = 0; i < D; ++i) fcache[(9 + i) * S + ix] = nd.V[i];
        }
      }
      zz[0 * NP + m] = z.q;
#pragma unroll
      for (int i = 0; i < D; ++i) zz[(1 + i) * NP + m] = z.V[i];
      zz[(D + 1) * NP + m] = z.p;
      zz[(D + 2) * NP + m] = z.P1;
      zz[(D + 3) * NP + m] = z.P2;
      zz[(D + 4) * NP + m] = z.v2;
      zz[(D + 5) * NP + m] = z.iq;
      zz[(D + 6) * NP + m] = z.ip;
    }
    sH[el * NP + m] = (T)(1.0 / (c_ref.H[m] * __ldg(&J[(size_t)e * NP + m])));  // 1/H
  }
  __syncthreads();
  T acc[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) acc[q] = T(0);
  const T* zz = sz + el * NZ * NP;
  ZNode<T, D> zm;
  IRNode<T, D> im;
  T iHm = T(0), Hm = T(0);
  if (active) {
    if constexpr (FLUX == 1) {
      im.z1 = zz[m];
      im.zn = zz[NP + m];
      im.l1 = zz[2 * NP + m];
      im.ln = zz[3 * NP + m];
#pragma unroll
      for (int i = 0; i < D; ++i) im.V[i] = zz[(4 + i) * NP + m];
    } else {
      zm.q = zz[m];
#pragma unroll
      for (int i = 0; i < D; ++i) zm.V[i] = zz[(1 + i) * NP + m];
      zm.p = zz[(D + 1) * NP + m];
      zm.P1 = zz[(D + 2) * NP + m];
      zm.P2 = zz[(D + 3) * NP + m];
      zm.v2 = zz[(D + 4) * NP + m];
      zm.iq = zz[(D + 5) * NP + m];
      zm.ip = zz[(D + 6) * NP + m];
    }
    iHm = sH[el * NP + m];
    Hm = T(1) / iHm;
  }
  const T* op = ops + (size_t)e * (2 * D * NP * NP);
  T* gout = sg + ((size_t)el * NP + m) * KC * NC;
  // pair offsets k = 1..K in chunks of KC (one chunk when KC = K): node m
  // forms the pairs (m, m + k) of the chunk, then gathers the chunk's pairs
  // (m - k, m) from shared memory; the chunk loop is uniform over the block
  for (int k0 = 1; k0 <= K; k0 += KC) {
    const int k1 = min(K, k0 + KC - 1);
    if (active) {
      for (int k = k0; k <= k1; ++k) {
        if ((NP % 2 == 0) && k == K && m >= K) break;
        int n = m + k;
        if (n >= NP) n -= NP;
        T Smn[D];
#pragma unroll
        for (int i = 0; i < D; ++i) Smn[i] = Hm * __ldg(&op[((D + i) * NP + n) * NP + m]);
        T G[NC];
        if constexpr (FLUX == 1) {
          IRNode<T, D> in_;
          in_.z1 = zz[n];
          in_.zn = zz[NP + n];
          in_.l1 = zz[2 * NP + n];
          in_.ln = zz[3 * NP + n];
#pragma unroll
          for (int i = 0; i < D; ++i) in_.V[i] = zz[(4 + i) * NP + n];
          IRAvg<T, D> ia;
          ir_avg<T, D>(im, in_, c, ia);
          ir_flux_dir<T, D>(ia, c, Smn, G);
        } else {
          ZNode<T, D> zn;
          zn.q = zz[n];
#pragma unroll
          for (int i = 0; i < D; ++i) zn.V[i] = zz[(1 + i) * NP + n];
          zn.p = zz[(D + 1) * NP + n];
          zn.P1 = zz[(D + 2) * NP + n];
          zn.P2 = zz[(D + 3) * NP + n];
          zn.v2 = zz[(D + 4) * NP + n];
          PairAvg<T, D> a;
          pair_avg<T, D>(zm, zn, c, a);
          sy_flux_dir<T, D>(a, c, Smn, G);
        }
#pragma unroll
        for (int q = 0; q < NC; ++q) {
          acc[q] -= T(2) * G[q] * iHm;
          gout[(k - k0) * NC + q] = T(2) * G[q];
        }
      }
    }
    __syncthreads();
    if (active) {
      for (int k = k0; k <= k1; ++k) {
        int src = m - k;
        if (src < 0) src += NP;
        if ((NP % 2 == 0) && k == K && src >= K) continue;
        const T* gin = sg + ((size_t)el * NP + src) * KC * NC + (k - k0) * NC;
#pragma unroll
        for (int q = 0; q < NC; ++q) acc[q] += gin[q] * iHm;
      }
    }
    if (k0 + KC <= K) __syncthreads();
  }
  double hw = 0.0;
  if (active) {
    int sl = c_ref.node_slot[m];
    double res[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      res[q] = (double)acc[q];
      if (sat && sl >= 0) res[q] += __ldg(&sat[((size_t)e * NC + q) * NS + sl]);
      r[((size_t)e * NC + q) * NP + m] = res[q];
    }
    if (prod) {
      double u64[NC];
#pragma unroll
      for (int q = 0; q < NC; ++q) u64[q] = __ldg(&u[((size_t)e * NC + q) * NP + m]);
      Node<double, D> n64;
      node_from_u<double, D>(u64, c64, n64);
#pragma unroll
      for (int q = 0; q < NC; ++q) hw += n64.W[q] * res[q];
      hw *= c_ref.H[m] * __ldg(&J[(size_t)e * NP + m]);
    }
  }
  if (prod) {
    double v[1] = {hw};
    block_sum<1>(v, prod + blockIdx.x);
  }
}

}  // namespace esplit

#include "visc.cuh"

namespace esplit {

template <int NP>
struct VolCfg {
  static constexpr int EB_SPLIT = (256 / NP) > 0 ? (256 / NP) : 1;
  // float64 on triangles: the float64-pipe-bound split kernel holds 2 blocks
  // of ~250 threads per SM, and the last of n_e / EB_SPLIT blocks leave the
  // SMs unevenly loaded by up to one block in ~15 (config 2).  Smaller blocks
  // that fill whole warps make that granularity finer and raise the warps
  // per SM: n_p = 7 and 18, 126 threads (4-5 blocks per SM; measured at 18:
  // 0.506 -> 0.490 ms per launch); n_p = 12, 192 threads (6 full warps, 3
  // blocks per SM; 0.285 -> 0.270 ms); n_p = 27, 189 threads (6 warps, 3
  // blocks per SM; 0.973 -> 0.952 ms).
  static constexpr int EB_SPLIT64_2D = NP == 7 ? 18 : NP == 12 ? 16 : NP == 18 ? 7 : NP == 27 ? 7 : EB_SPLIT;
  // larger operators (tetrahedra of degree 3 and 4): the pair contributions
  // pass through shared memory in chunks of HAD_KC pair offsets, which leaves
  // room for more elements per block
  static constexpr int EB_HAD = NP > 32 ? ((256 / NP) > 0 ? (256 / NP) : 1) : ((128 / NP) > 0 ? (128 / NP) : 1);
  static constexpr int HAD_KC = NP > 32 ? 8 : NP / 2;
};

template <typename T, int D, int NP>
static int residual_np(esplit_ctx* c, const double* u, double* r, cudaStream_t s, double* prod, int* n_partial,
                       double* sat) {
  const Phys<T> ph = make_phys<T>(c->prm.gam, c->prm.beta, c->prm.R, c->prm.mu, c->prm.Pr);
  const Phys<double> ph64 = make_phys<double>(c->prm.gam, c->prm.beta, c->prm.R, c->prm.mu, c->prm.Pr);
  const T* ops = std::is_same<T, double>::value ? (const T*)c->b.ops64 : (const T*)c->b.ops32;
  const bool visc = c->prm.viscous != 0;
  int scheme = c->prm.scheme;
  // inviscid split scheme: volume kernel first (it caches the facet nodes'
  // quantities), then the facet kernel adds into r; otherwise the facet terms
  // come first and fill the sat buffer the volume kernels add
  // (the Sjogreen-Yee Hadamard and hybrid schemes too in float64: the Hadamard
  // kernel caches its elements' facet nodes, and the facet kernel adds
  // nu . f / H for split-form sides only)
  const bool cached = (scheme == ESPLIT_SCHEME_SPLIT ||
                       ((scheme == ESPLIT_SCHEME_HYBRID || scheme == ESPLIT_SCHEME_HADAMARD) &&
                        std::is_same<T, double>::value)) &&
                      !visc && sat == c->b.sat && c->b.fcache != nullptr;
  if (!cached) {
    int bs = 128;
    int nb = (c->n_pairs + bs - 1) / bs;
    ProfScope ps(c, PG_FACE, s);
    // facet terms are O(1/h) and cancel against the volume's boundary part:
    // they stay float64 in both precision modes
    const int ef_mode = c->prm.scheme == ESPLIT_SCHEME_SPLIT ? 1 : (c->prm.scheme == ESPLIT_SCHEME_HYBRID ? 2 : 0);
    const int visc_heat = c->prm.viscous ? c->prm.heat_flux : -1;
    if (c->prm.scheme == ESPLIT_SCHEME_HADAMARD_IR && visc_heat >= 0)
      face_kernel<double, D, true, 1><<<nb, bs, 0, s>>>(u, c->b.face_pairs, c->n_pairs, c->b.nu, c->b.ihd, c->b.nscale, sat,
                                                        ph64, c->prm.dissipation, c->b.status, 0, c->b.hflags,
                                                        visc_heat, c->b.va);
    else if (c->prm.scheme == ESPLIT_SCHEME_HADAMARD_IR)
      face_kernel<double, D, false, 1><<<nb, bs, 0, s>>>(u, c->b.face_pairs, c->n_pairs, c->b.nu, c->b.ihd, c->b.nscale, sat,
                                                         ph64, c->prm.dissipation, c->b.status, 0, c->b.hflags, 0,
                                                         nullptr);
    else if (visc_heat >= 0)
      face_kernel<double, D, true><<<nb, bs, 0, s>>>(u, c->b.face_pairs, c->n_pairs, c->b.nu, c->b.ihd, c->b.nscale, sat, ph64,
                                                     c->prm.dissipation, c->b.status, ef_mode, c->b.hflags,
                                                     visc_heat, c->b.va);
    else
      face_kernel<double, D, false><<<nb, bs, 0, s>>>(u, c->b.face_pairs, c->n_pairs, c->b.nu, c->b.ihd, c->b.nscale, sat, ph64,
                                                      c->prm.dissipation, c->b.status, ef_mode, c->b.hflags, 0,
                                                      nullptr);
    c->launches++;
    // boundary facet slots into the same scratch (the volume kernels add them)
    launch_face_bc(c, u, sat, 0, nullptr, s);
  }
  int np_used = 0;
  int n_split = scheme == ESPLIT_SCHEME_SPLIT ? c->n_e : (scheme == ESPLIT_SCHEME_HYBRID ? c->n_split : 0);
  int n_had = (scheme == ESPLIT_SCHEME_HADAMARD || scheme == ESPLIT_SCHEME_HADAMARD_IR)
                  ? c->n_e
                  : (scheme == ESPLIT_SCHEME_HYBRID ? c->n_had : 0);
  const int* lsplit = scheme == ESPLIT_SCHEME_HYBRID ? c->b.list_split : nullptr;
  const int* lhad = scheme == ESPLIT_SCHEME_HYBRID ? c->b.list_had : nullptr;
  if (n_split > 0) {
    constexpr int EB = (std::is_same<T, double>::value && D == 2) ? VolCfg<NP>::EB_SPLIT64_2D : VolCfg<NP>::EB_SPLIT;
    int nb = (n_split + EB - 1) / EB;
    ProfScope ps(c, PG_SPLIT, s);
    // the split kernel also forms the viscous volume terms (it has D_i w)
    const int S = c->n_e * c->n_slot;
    {
      // the float32 variant is sized for four blocks per SM and the 3D viscous
      // variants for two: ask for the shared memory they need
      static bool carve_set = false;
      if (!carve_set) {
        if (!std::is_same<T, double>::value) {
          cudaFuncSetAttribute(split_volume_kernel<T, D, NP, EB, false, true>,
                               cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
          cudaFuncSetAttribute(split_volume_kernel<T, D, NP, EB, false, true, true>,
                               cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        }
        cudaFuncSetAttribute(split_volume_kernel<T, D, NP, EB, true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        cudaFuncSetAttribute(split_volume_kernel<T, D, NP, EB, true, false, true>,
                             cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        carve_set = true;
      }
    }
    if (visc && c->ent_part && c->b.node_cache) {
      // first stage of a relaxation step: the kernel also forms the entropy of u_n
      split_volume_kernel<T, D, NP, EB, true, false, true><<<nb, EB * NP, 0, s>>>(
          u, r, ops, c->b.ops32lo, c->b.rows, c->b.J, sat, lsplit, n_split, ph, ph64, c->b.status,
          prod ? prod + np_used : nullptr, c->prm.heat_flux, c->b.nu, c->b.va, c->b.fv, c->b.ops64, nullptr, S,
          c->ent_part, c->b.node_cache, prod ? c->b.wslot : nullptr);
      c->ent_n = nb;
    } else if (visc)
      split_volume_kernel<T, D, NP, EB, true><<<nb, EB * NP, 0, s>>>(
          u, r, ops, c->b.ops32lo, c->b.rows, c->b.J, sat, lsplit, n_split, ph, ph64, c->b.status,
          prod ? prod + np_used : nullptr, c->prm.heat_flux, c->b.nu, c->b.va, c->b.fv, c->b.ops64, nullptr, S,
          nullptr, nullptr, prod ? c->b.wslot : nullptr);
    else if (cached && scheme == ESPLIT_SCHEME_SPLIT && c->ent_part && c->b.node_cache) {
      split_volume_kernel<T, D, NP, EB, false, true, true><<<nb, EB * NP, 0, s>>>(
          u, r, ops, c->b.ops32lo, c->b.rows, c->b.J, sat, lsplit, n_split, ph, ph64, c->b.status,
          prod ? prod + np_used : nullptr, -1, nullptr, nullptr, nullptr, nullptr, c->b.fcache, S, c->ent_part,
          c->b.node_cache);
      c->ent_n = nb;
    } else if (cached)
      split_volume_kernel<T, D, NP, EB, false, true><<<nb, EB * NP, 0, s>>>(
          u, r, ops, c->b.ops32lo, c->b.rows, c->b.J, sat, lsplit, n_split, ph, ph64, c->b.status,
          prod ? prod + np_used : nullptr, -1, nullptr, nullptr, nullptr, nullptr, c->b.fcache, S);
    else
      split_volume_kernel<T, D, NP, EB, false><<<nb, EB * NP, 0, s>>>(
          u, r, ops, c->b.ops32lo, c->b.rows, c->b.J, sat, lsplit, n_split, ph, ph64, c->b.status,
          prod ? prod + np_used : nullptr, -1, nullptr, nullptr, nullptr, nullptr, nullptr, S);
    c->launches++;
    np_used += nb;
  }
  if (n_had > 0) {
    constexpr int EB = VolCfg<NP>::EB_HAD;
    constexpr int KC = VolCfg<NP>::HAD_KC;
    size_t smem = sizeof(T) * ((size_t)EB * (D + 7) * NP + (size_t)EB * NP * KC * (D + 2) + (size_t)EB * NP);
    static bool attr_set = false;
    if (!attr_set) {
      cudaFuncSetAttribute(hadamard_volume_kernel<T, D, NP, EB, 0, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
      cudaFuncSetAttribute(hadamard_volume_kernel<T, D, NP, EB, 1, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
      attr_set = true;
    }
    int nb = (n_had + EB - 1) / EB;
    ProfScope ps(c, PG_HAD, s);
    if (scheme == ESPLIT_SCHEME_HADAMARD_IR)
      hadamard_volume_kernel<T, D, NP, EB, 1, KC><<<nb, EB * NP, smem, s>>>(
          u, r, ops, c->b.J, sat, lhad, n_had, ph, ph64, c->b.status, prod ? prod + np_used : nullptr);
    else if (cached)
      // Hadamard or hybrid scheme on the cached path: no facet terms to add
      // here (the facet kernel adds them after), the facet nodes' quantities
      // written instead
      hadamard_volume_kernel<T, D, NP, EB, 0, KC><<<nb, EB * NP, smem, s>>>(
          u, r, ops, c->b.J, nullptr, lhad, n_had, ph, ph64, c->b.status, prod ? prod + np_used : nullptr,
          c->b.fcache, c->n_e * c->n_slot);
    else
      hadamard_volume_kernel<T, D, NP, EB, 0, KC><<<nb, EB * NP, smem, s>>>(
          u, r, ops, c->b.J, sat, lhad, n_had, ph, ph64, c->b.status, prod ? prod + np_used : nullptr);
    c->launches++;
    np_used += nb;
  }
  if (cached) {
    // after both volume kernels (the Hadamard kernel assigns r)
    int bs = 128;
    int nb = (c->n_pairs + bs - 1) / bs;
    ProfScope ps(c, PG_FACE, s);
    face_cached_kernel<D><<<nb, bs, 0, s>>>(r, c->b.face_pairs, c->n_pairs, c->b.nu, c->b.ihd, c->b.nscale,
                                            c->b.fcache,
                                            c->n_e * c->n_slot, ph64, c->prm.dissipation,
                                            prod ? prod + np_used : nullptr,
                                            scheme == ESPLIT_SCHEME_SPLIT ? 1 : (scheme == ESPLIT_SCHEME_HYBRID ? 2 : 0),
                                            c->b.hflags);
    c->launches++;
    if (prod) np_used += nb;
    np_used += launch_face_bc(c, u, r, 1, prod ? prod + np_used : nullptr, s);
  }
  if (visc) {
    ProfScope ps(c, PG_VISC, s);
    // viscous volume terms of the elements the split kernel did not take
    if (n_had > 0) viscous_volume_np<D, NP>(c, u, r, lhad, n_had, s);
    // with the production requested (split scheme only, n_had = 0) the jump
    // kernel adds its share of the block partials
    np_used += viscous_jump<D>(c, r, s, (prod && n_had == 0) ? prod + np_used : nullptr);
  }
  if (n_partial) *n_partial = np_used;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <typename T>
static int residual_t(esplit_ctx* c, const double* u, double* r, cudaStream_t s, double* prod, int* n_partial,
                      double* sat) {
  if (c->dim == 1) {
    switch (c->n_p) {
      case 2: return residual_np<T, 1, 2>(c, u, r, s, prod, n_partial, sat);
      case 3: return residual_np<T, 1, 3>(c, u, r, s, prod, n_partial, sat);
      case 4: return residual_np<T, 1, 4>(c, u, r, s, prod, n_partial, sat);
      case 5: return residual_np<T, 1, 5>(c, u, r, s, prod, n_partial, sat);
    }
  } else if (c->dim == 2) {
    switch (c->n_p) {
      case 7: return residual_np<T, 2, 7>(c, u, r, s, prod, n_partial, sat);
      case 12: return residual_np<T, 2, 12>(c, u, r, s, prod, n_partial, sat);
      case 18: return residual_np<T, 2, 18>(c, u, r, s, prod, n_partial, sat);
      case 27: return residual_np<T, 2, 27>(c, u, r, s, prod, n_partial, sat);
    }
  } else if (c->dim == 3) {
    switch (c->n_p) {
      case 12: return residual_np<T, 3, 12>(c, u, r, s, prod, n_partial, sat);
      case 25: return residual_np<T, 3, 25>(c, u, r, s, prod, n_partial, sat);
      case 58: return residual_np<T, 3, 58>(c, u, r, s, prod, n_partial, sat);
      case 78: return residual_np<T, 3, 78>(c, u, r, s, prod, n_partial, sat);
    }
  }
  return -2;
}

// the float32 deviation path (fp32.cu) covers the inviscid split scheme on
// lines and triangles; the other schemes, the viscous terms and tetrahedra
// take the FP32-bulk kernels there.  (The tetrahedron operators have rows with
// sum |D_mn| of 40 to 170 at facet nodes of small volume weight, which
// amplify the float32 rounding of the flux variations: 1.4e-5 at 25 nodes and
// up to 3.2e-5 at 78 without dissipation, above the 1e-5 bound of the float32
// path; triangles stay below 6e-6.)
static bool use_f32_path(const esplit_ctx* c) {
  return c->prm.precision == ESPLIT_FP32 && c->prm.scheme == ESPLIT_SCHEME_SPLIT && !c->prm.viscous && c->dim <= 2;
}

bool uses_f32_path(const esplit_ctx* c) { return use_f32_path(c); }

int launch_residual(esplit_ctx* c, const double* u, double* r, cudaStream_t s, double* prod, int* n_partial) {
  if (use_f32_path(c)) return launch_split_f32(c, u, r, s, prod, n_partial, c->b.sat);
  if (c->prm.precision != ESPLIT_FP64) return residual_t<float>(c, u, r, s, prod, n_partial, c->b.sat);
  return residual_t<double>(c, u, r, s, prod, n_partial, c->b.sat);
}

// ---------------------------------------------------------------------------
// Residual variant with no device allocation at all: its facet scratch is
// this file-scope array instead of the context's buffer.  Host code may not
// use the array's name as a device address; the address is looked up once
// per device with cudaGetSymbolAddress while that device is current.
// ---------------------------------------------------------------------------
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH_DOUBLES];

static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

int noalloc_scratch_ptr(int device, double** out) {
  if (device < 0 || device >= NOALLOC_MAX_DEVICES) return -1;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != device) return -1;
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return -1;
    g_noalloc_ptr[device] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[device];
  return 0;
}

int launch_residual_noalloc(esplit_ctx* c, const double* u, double* r, cudaStream_t s, double* scratch) {
  // kernel timing would create CUDA events: off for this thread's launches
  // (the context's setting, which other threads may be using, is untouched)
  t_no_events = true;
  int rc = use_f32_path(c) ? launch_split_f32(c, u, r, s, nullptr, nullptr, scratch)
           : c->prm.precision != ESPLIT_FP64 ? residual_t<float>(c, u, r, s, nullptr, nullptr, scratch)
                                              : residual_t<double>(c, u, r, s, nullptr, nullptr, scratch);
  t_no_events = false;
  // viscous terms (inside the residual launch) use the context's viscous
  // scratch, allocated when they were switched on
  return rc;
}

// ---------------------------------------------------------------------------
// entropy functionals, one thread per node
// ---------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(256) entropy_kernel(const double* __restrict__ u, const double* __restrict__ J,
                                                      size_t n_nodes, Phys<double> c, double* __restrict__ part,
                                                      double* __restrict__ cache) {
  constexpr int NC = D + 2;
  const int NP = c_ref.n_p;
  size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v[2] = {0.0, 0.0};
  if (g < n_nodes) {
    size_t e = g / NP;
    int m = (int)(g - e * NP);
    double uu[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) uu[q] = __ldg(&u[(e * NC + q) * NP + m]);
    // one division for 1/rho and 1/p: P = rho p = (gam-1)(rho E - |m|^2/2),
    // y = 1/(rho P), 1/rho = P y, 1/p = rho^2 y, p = P/rho
    const double rho = uu[0];
    double mm = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i) mm += uu[1 + i] * uu[1 + i];
    const double P = c.gm1 * (rho * uu[NC - 1] - 0.5 * mm);
    const double y = 1.0 / (rho * P);
    const double ir = P * y, ip = (rho * rho) * y, p = P * ir;
    // S_H = beta rho (p rho^-gam)^(1/(alpha+gam)) = beta q p, log q = a_q log rho + b_q log p
    const double lnq = c.a_q * fm::log(rho) + c.b_q * fm::log(p);
    const double sH = c.beta * fm::exp(lnq) * p;
    double H = c_ref.H[m] * __ldg(&J[e * NP + m]);
    v[0] = H * sH;
    v[1] = H * fabs(sH);
    if (cache) {  // per-node values the relaxation passes reuse: s, 1/rho, 1/p
      cache[g] = sH;
      cache[n_nodes + g] = ir;
      cache[2 * n_nodes + g] = ip;
    }
  }
  block_sum_t<2, 256>(v, part + 2 * blockIdx.x);
}

template <int D, int W>
__global__ void __launch_bounds__(256) entropy_rate_kernel(const double* __restrict__ u,
                                                           const double* __restrict__ r,
                                                           const double* __restrict__ J, size_t n_nodes,
                                                           Phys<double> c, double* __restrict__ part) {
  constexpr int NC = D + 2;
  const int NP = c_ref.n_p;
  size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v[2] = {0.0, 0.0};
  if (g < n_nodes) {
    size_t e = g / NP;
    int m = (int)(g - e * NP);
    double uu[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) uu[q] = __ldg(&u[(e * NC + q) * NP + m]);
    Node<double, D> nd;
    node_from_u<double, D>(uu, c, nd);
    double H = c_ref.H[m] * __ldg(&J[e * NP + m]);
    double wr = 0.0, w2 = 0.0, r2 = 0.0;
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      double rq = __ldg(&r[(e * NC + q) * NP + m]);
      wr += nd.W[q] * rq;
      w2 += nd.W[q] * nd.W[q];
      r2 += rq * rq;
    }
    v[0] = H * wr;
    v[1] = H * sqrt(w2 * r2);
  }
  if constexpr (W == 1) {
    double v1[1] = {v[0]};
    block_sum_t<1, 256>(v1, part + blockIdx.x);
  } else {
    block_sum_t<2, 256>(v, part + 2 * blockIdx.x);
  }
}

int launch_entropy(esplit_ctx* c, const double* u, cudaStream_t s, int* n_partial, double* cache, double* part) {
  size_t n = (size_t)c->n_e * c->n_p;
  int nb = (int)((n + 255) / 256);
  Phys<double> ph = make_phys<double>(c->prm.gam, c->prm.beta, c->prm.R, c->prm.mu, c->prm.Pr);
  ProfScope ps(c, PG_ENTROPY, s);
  double* out = part ? part : c->b.partial;
  if (c->dim == 1)
    entropy_kernel<1><<<nb, 256, 0, s>>>(u, c->b.J, n, ph, out, cache);
  else if (c->dim == 2)
    entropy_kernel<2><<<nb, 256, 0, s>>>(u, c->b.J, n, ph, out, cache);
  else
    entropy_kernel<3><<<nb, 256, 0, s>>>(u, c->b.J, n, ph, out, cache);
  c->launches++;
  *n_partial = nb;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_entropy_rate(esplit_ctx* c, const double* u, const double* r, cudaStream_t s, int* n_partial,
                        double* part, int width) {
  size_t n = (size_t)c->n_e * c->n_p;
  int nb = (int)((n + 255) / 256);
  Phys<double> ph = make_phys<double>(c->prm.gam, c->prm.beta, c->prm.R, c->prm.mu, c->prm.Pr);
  ProfScope ps(c, PG_ENTROPY, s);
  if (!part) part = c->b.partial;
  if (c->dim == 1) {
    if (width == 1)
      entropy_rate_kernel<1, 1><<<nb, 256, 0, s>>>(u, r, c->b.J, n, ph, part);
    else
      entropy_rate_kernel<1, 2><<<nb, 256, 0, s>>>(u, r, c->b.J, n, ph, part);
  } else if (c->dim == 2) {
    if (width == 1)
      entropy_rate_kernel<2, 1><<<nb, 256, 0, s>>>(u, r, c->b.J, n, ph, part);
    else
      entropy_rate_kernel<2, 2><<<nb, 256, 0, s>>>(u, r, c->b.J, n, ph, part);
  } else {
    if (width == 1)
      entropy_rate_kernel<3, 1><<<nb, 256, 0, s>>>(u, r, c->b.J, n, ph, part);
    else
      entropy_rate_kernel<3, 2><<<nb, 256, 0, s>>>(u, r, c->b.J, n, ph, part);
  }
  c->launches++;
  *n_partial = nb;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// fixed-order reduction of `n` rows of `width` partials into out[width]
__global__ void __launch_bounds__(1024) reduce_partials_kernel(const double* __restrict__ part, int n, int width,
                                                               double* __restrict__ out) {
  for (int k = 0; k < width; ++k) {
    double v[1] = {0.0};
    for (int i = threadIdx.x; i < n; i += blockDim.x) v[0] += part[(size_t)i * width + k];
    block_sum<1>(v, out + k);
    __syncthreads();
  }
}

// several block-partial regions reduced in one launch, one block per region,
// each in a fixed order (deterministic)
__global__ void __launch_bounds__(1024) reduce_regions_kernel(const double* __restrict__ part, ReduceRegions R) {
  const int g = blockIdx.x;
  if (g >= R.n) return;
  const double* p = part + R.off[g];
  const int w = R.width[g], cnt = R.cnt[g];
  for (int k = 0; k < w; ++k) {
    double v[1] = {0.0};
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) v[0] += p[(size_t)i * w + k];
    block_sum<1>(v, R.out[g] + k);
    __syncthreads();
  }
}

int launch_reduce_regions(esplit_ctx* c, const double* partial, const ReduceRegions& R, cudaStream_t s) {
  ProfScope ps(c, PG_ENTROPY, s);
  reduce_regions_kernel<<<R.n, 1024, 0, s>>>(partial, R);
  c->launches++;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_reduce(esplit_ctx* c, const double* partial, int n_partial, int width, double* out, cudaStream_t s) {
  ProfScope ps(c, PG_ENTROPY, s);
  reduce_partials_kernel<<<1, 1024, 0, s>>>(partial, n_partial, width, out);
  c->launches++;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ---------------------------------------------------------------------------
// RK4 stage combination: u_next = u_n + a_dt r ; dacc (=|+=) b_dt r
// ---------------------------------------------------------------------------
__global__ void stage_kernel(const double* __restrict__ un, const double* __restrict__ r, double a_dt, double b_dt,
                             int first, double* __restrict__ u_next, double* __restrict__ dacc, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (; i < n; i += stride) {
    double ri = r[i];
    if (u_next) u_next[i] = un[i] + a_dt * ri;
    dacc[i] = first ? b_dt * ri : dacc[i] + b_dt * ri;
  }
}

static unsigned grid_for(size_t n) {
  size_t nb = (n + 255) / 256;
  size_t cap = 152 * 16;
  return (unsigned)(nb < cap ? nb : cap);
}

int launch_stage(esplit_ctx* c, const double* un, const double* r, double a_dt, double b_dt, int first,
                 double* u_next, double* dacc, size_t n, cudaStream_t s) {
  ProfScope ps(c, PG_STAGE, s);
  stage_kernel<<<grid_for(n), 256, 0, s>>>(un, r, a_dt, b_dt, first, u_next, dacc, n);
  c->launches++;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

__global__ void axpy_kernel(const double* __restrict__ x, double a, const double* __restrict__ y,
                            double* __restrict__ out, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (; i < n; i += stride) out[i] = x[i] + a * y[i];
}

int launch_axpy(esplit_ctx* c, const double* x, double a, const double* y, double* out, size_t n, cudaStream_t s) {
  ProfScope ps(c, PG_STAGE, s);
  axpy_kernel<<<grid_for(n), 256, 0, s>>>(x, a, y, out, n);
  c->launches++;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ---------------------------------------------------------------------------
// relaxation root solve of Eq. (97) on the device
//   f(g) = sum H [s(u_n + g d) - s(u_n)] - g est,   f'(g) = sum H w(u_n + g d).d - est
// with the per-node entropy change evaluated without cancellation:
//   s(U+dU) - s(U) = s(U) expm1(A log1p(drho/rho) + B log1p(dp/p)),
//   A = alpha/(alpha+gam), B = 1/(alpha+gam), dp from the closure exactly.
// Pass 0 evaluates f and f' at g = 1.  f is convex with f(0) = 0, so Newton
// from g = 1 approaches the other root monotonically (from above after at
// most one step): when |f(1)| and |f'(1)| are both at the round-off floor
// 64 eps sum H|s| the step is a free stream and g = 1; when f'(1) > 0 and the
// Newton point lies in (0.5, 1.5) the Newton phase starts there.  Otherwise
// the bracketing path: g = 0.5 and 1.5 together (bracket and floor rule),
// halving lo / doubling hi, then Newton from the quadratic model through
// (0, 0), (lo, f_lo), (hi, f_hi).  Stops at |step| <= 4 eps g, |f| at its own
// round-off level, or ROOT_EVALS_MAX evaluations; no bracket -> status -5.
// ---------------------------------------------------------------------------
__global__ void root_init_kernel(RootState* st, const double* scal, double dt) {
  // scal[0..1] = S0, sum H |s| ; scal[2..5] = stage productions e_1..e_4
  const double b[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
  st->S0 = scal[0];
  st->Sabs = scal[1];
  double est = 0.0;
  for (int i = 0; i < 4; ++i) est += b[i] * scal[2 + i];
  st->est = dt * est;
  st->g = 1.0;
  st->ga = 1.0;
  st->gb = -1.0;
  st->lo = 0.5;
  st->hi = 1.5;
  st->flo = 0.0;
  st->fhi = 0.0;
  st->phase = 0;
  st->done = 0;
  st->iters = 0;
  st->status = 0;
  st->dg_last = 0.0;
  st->arrivals = 0;
}

// Entropy change s(u + g d) - s(u), slope w(u + g d) . d and (SECOND)
// curvature d . (dw/dg) at one node, from the cached s(u), 1/rho and 1/p of
// u.  Along u' = u + g d: drho' = d_0, dV' = (d_m - V' d_0)/rho',
// dp' = (gam-1)(d_E - V'.d_m + |V'|^2 d_0/2), dq'/q' = a_q d_0/rho' + b_q dp'/p'.
template <int D, bool SECOND = false>
__device__ __forceinline__ void entropy_change_and_slope(const double* u, const double* dd, double g, double s0,
                                                         double ir, double ip, const Phys<double>& c,
                                                         double& ds, double& wd, double* d2 = nullptr) {
  constexpr int NC = D + 2;
  double rho = u[0];
  double drho = g * dd[0], dE = g * dd[NC - 1];
  double mm = 0.0, mdm = 0.0, dmdm = 0.0;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double m = u[1 + i], dm = g * dd[1 + i];
    mm += m * m;
    mdm += m * dm;
    dmdm += dm * dm;
  }
  double ir1 = 1.0 / (rho + drho);  // 1/rho'
  double dke = 0.5 * ((2.0 * mdm + dmdm) - mm * drho * ir) * ir1;
  double dp = c.gm1 * (dE - dke);
  double l1 = fm::log1p(drho * ir), l2 = fm::log1p(dp * ip);
  ds = s0 * fm::expm1(c.a_q * l1 + (c.b_q + 1.0) * l2);
  // entropy variables at u' = u + g d (Eq. (25)); q' = s'/(beta p') with
  // s' = s + ds (S_H = beta q p), one division that also gives 1/p'
  double p1 = c.gm1 * (u[NC - 1] - 0.5 * mm * ir) + dp;
  double ibp1 = 1.0 / (c.beta * p1);
  double q1 = (s0 + ds) * ibp1;
  double v2 = 0.0, vd = 0.0;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double V = (u[1 + i] + g * dd[1 + i]) * ir1;
    v2 += V * V;
    vd += V * dd[1 + i];
  }
  double W0 = q1 * (c.w1c * p1 * ir1 - 0.5 * v2);
  wd = W0 * dd[0] + q1 * vd - q1 * dd[NC - 1];
  if constexpr (SECOND) {
    double Vs[D], dV[D], vdm = 0.0, vdv = 0.0, dvd = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      Vs[i] = (u[1 + i] + g * dd[1 + i]) * ir1;
      vdm += Vs[i] * dd[1 + i];
    }
#pragma unroll
    for (int i = 0; i < D; ++i) {
      dV[i] = (dd[1 + i] - Vs[i] * dd[0]) * ir1;
      vdv += Vs[i] * dV[i];
      dvd += dV[i] * dd[1 + i];
    }
    double dp1 = c.gm1 * (dd[NC - 1] - vdm + 0.5 * v2 * dd[0]);
    double dq1 = q1 * (c.a_q * dd[0] * ir1 + c.b_q * dp1 * (c.beta * ibp1));
    double dW0 = dq1 * (c.w1c * p1 * ir1 - 0.5 * v2) + q1 * (c.w1c * (dp1 - p1 * dd[0] * ir1) * ir1 - vdv);
    *d2 = dW0 * dd[0] + dq1 * vd + q1 * dvd - dq1 * dd[NC - 1];
  }
}

__device__ void root_update_body(const double* tot, RootState* st);

// One evaluation pass of the root solve and the update that follows it: every
// block writes its six partial sums; the block that finishes last (counted on
// the root state after a fence, so that it sees every partial) reduces them in
// block order and updates the root state, which the next pass reads.
// COND: launched inside a graph's while loop over the evaluation passes; the
// loop continues while the root is not done.  Every path sets done within
// ROOT_EVALS_MAX + 12 passes (the Newton phase stops at ROOT_EVALS_MAX, the
// bracket search after 10 halvings or 2 doublings); the hard stop below ends
// the loop even if that reasoning failed, with status "no root".
template <int D, bool COND>
__global__ void __launch_bounds__(256) root_eval_kernel(const double* __restrict__ un, const double* __restrict__ d,
                                                        const double* __restrict__ J,
                                                        const double* __restrict__ cache, size_t n_nodes,
                                                        Phys<double> c, RootState* __restrict__ st,
                                                        double* __restrict__ part, cudaGraphConditionalHandle h) {
  if (st->done) {
    if constexpr (COND)
      if (blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, 0u);
    return;
  }
  constexpr int NC = D + 2;
  const int NP = c_ref.n_p;
  const double ga = st->ga, gb = st->gb;
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  if (t < n_nodes) {
    size_t e = t / NP;
    int m = (int)(t - e * NP);
    double uu[NC], dd[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      size_t ix = (e * NC + q) * NP + m;
      dd[q] = __ldg(&d[ix]);
      uu[q] = __ldg(&un[ix]);
    }
    double s0 = __ldg(&cache[t]), ir = __ldg(&cache[n_nodes + t]);
    double ip = __ldg(&cache[2 * n_nodes + t]);
    double H = c_ref.H[m] * __ldg(&J[e * NP + m]);
    double ds, wd;
    double d2 = 0.0;
    entropy_change_and_slope<D, true>(uu, dd, ga, s0, ir, ip, c, ds, wd, &d2);
    v[0] = H * ds;
    v[1] = H * wd;
    v[2] = H * fabs(ds);
    v[3] = H * d2;  // curvature; replaced below when a second point is evaluated
    if (gb > 0.0) {
      entropy_change_and_slope<D>(uu, dd, gb, s0, ir, ip, c, ds, wd);
      v[3] = H * ds;
      v[4] = H * wd;
      v[5] = H * fabs(ds);
    }
  }
  block_sum_t<6, 256>(v, part + 6 * blockIdx.x);
  __threadfence();  // this block's partials, before it is counted
  __syncthreads();
  __shared__ int last;
  if (threadIdx.x == 0) last = atomicAdd(&st->arrivals, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  __shared__ double tot[6];
  double w[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  // unrolled so that the loads of several rounds are in flight together (the
  // partials come from L2; the sums keep each thread's round order)
#pragma unroll 4
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
#pragma unroll
    for (int k = 0; k < 6; ++k) w[k] += __ldcg(&part[(size_t)i * 6 + k]);
  }
  block_sum<6>(w, tot);
  if (threadIdx.x != 0) return;
  st->arrivals = 0;
  root_update_body(tot, st);
  if constexpr (COND) {
    if (!st->done && st->iters >= ROOT_EVALS_MAX + 16) {
      st->status = ESPLIT_ERR_RRK_NO_ROOT;
      st->done = 1;
    }
    cudaGraphSetConditional(h, st->done ? 0u : 1u);
  }
}

__device__ void root_update_body(const double* tot, RootState* st) {
  const double eps = 2.220446049250313e-16;
  const double est = st->est;
  st->iters += 1;
  if (st->phase == 0) {  // f, f', f'' at g = 1
    double f1 = tot[0] - est, df1 = tot[1] - est, d2f = tot[3];
    double floor = 64.0 * eps * st->Sabs;
    if (fabs(f1) <= floor && fabs(df1) <= floor) {
      st->g = 1.0;
      st->done = 1;
      return;
    }
    if (df1 > 0.0 && d2f >= 0.0) {
      // Halley's step from g = 1 (f is convex): its error is third order in the
      // Newton step dn, ~ (f''/f')^2 |dn|^3 / 4.  Accept it without a further
      // pass when f' times four times that error stays within the tolerance the
      // Newton phase stops at, 4 eps (sum H |ds| + |g est|)
      const double dn = -f1 / df1;
      const double den = 2.0 * df1 * df1 - f1 * d2f;
      const double k = d2f / df1;
      if (den > 0.0 && fabs(dn) < 0.25 &&
          df1 * k * k * fabs(dn) * dn * dn <= 4.0 * eps * (tot[2] + fabs(est))) {
        const double dh = -2.0 * f1 * df1 / den;
        st->g = 1.0 + dh;
        st->phase = 3;
        st->dS_last = tot[0] + dh * tot[1] + 0.5 * dh * dh * d2f;
        st->done = 1;
        return;
      }
    }
    double gn = df1 > 0.0 ? 1.0 - f1 / df1 : -1.0;
    if (gn > 0.5 && gn < 1.5) {
      st->phase = 3;
      st->dS_last = tot[0];
      st->f_last = f1;
      st->df_last = df1;
      if (f1 < 0.0) {
        st->lo = 1.0;
        st->flo = f1;
      } else {
        st->hi = 1.0;
        st->fhi = f1;
      }
      st->ga = gn;
      st->g = gn;
      st->dg_last = gn - 1.0;
      return;
    }
    st->phase = 4;  // bracketing path
    st->ga = 0.5;
    st->gb = 1.5;
    return;
  }
  if (st->phase == 4) {
    double flo = tot[0] - 0.5 * est, fhi = tot[3] - 1.5 * est;
    double floor = 64.0 * eps * st->Sabs;
    st->flo = flo;
    st->fhi = fhi;
    if (fabs(flo) <= floor && fabs(fhi) <= floor) {
      st->g = 1.0;
      st->done = 1;
      return;
    }
    if (flo >= 0.0) {
      st->phase = 1;
      st->ga = 0.25;
      st->gb = -1.0;
      return;
    }
    if (fhi <= 0.0) {
      st->phase = 2;
      st->ga = 3.0;
      st->gb = -1.0;
      return;
    }
  } else if (st->phase == 1) {  // shrink lo by halves (bracket [2^-10, 1.5])
    double f = tot[0] - st->ga * est;
    if (f >= 0.0) {
      double ng = 0.5 * st->ga;
      if (ng < 0.0009765625) {
        st->status = ESPLIT_ERR_RRK_NO_ROOT;
        st->done = 1;
        return;
      }
      st->ga = ng;
      return;
    }
    st->lo = st->ga;
    st->flo = f;
  } else if (st->phase == 2) {  // grow hi by doubling (up to 4)
    double f = tot[0] - st->ga * est;
    if (f <= 0.0) {
      double ng = 2.0 * st->ga;
      if (ng > 4.0) {
        st->status = ESPLIT_ERR_RRK_NO_ROOT;
        st->done = 1;
        return;
      }
      st->lo = st->ga;
      st->flo = f;
      st->ga = ng;
      return;
    }
    st->hi = st->ga;
    st->fhi = f;
  }
  if (st->phase != 3) {  // a bracket from phase 4, 1 or 2
    // quadratic model f ~ c g (g - g*) through (0,0), (lo, flo), (hi, fhi)
    double lo = st->lo, hi = st->hi;
    double cq = (st->fhi / hi - st->flo / lo) / (hi - lo);
    double g0 = cq > 0.0 ? lo - (st->flo / lo) / cq : 0.5 * (lo + hi);
    if (!(g0 > lo && g0 < hi)) g0 = 0.5 * (lo + hi);
    st->phase = 3;
    st->ga = g0;
    st->gb = -1.0;
    st->g = g0;
    return;
  }
  // Newton phase
  double g = st->ga;
  double f = tot[0] - g * est;
  st->dS_last = tot[0];
  double df = tot[1] - est;
  st->f_last = f;
  st->df_last = df;
  if (f < 0.0) {
    st->lo = g;
    st->flo = f;
  } else {
    st->hi = g;
    st->fhi = f;
  }
  st->g = g;
  if (fabs(f) <= 4.0 * eps * (tot[2] + fabs(g * est))) {
    st->done = 1;
    return;
  }
  double gn = (df > 0.0) ? g - f / df : 0.5 * (st->lo + st->hi);
  bool newton = df > 0.0 && gn > st->lo && gn < st->hi;
  if (!newton) gn = 0.5 * (st->lo + st->hi);
  const double dg = gn - g;
  // quadratic convergence: with the contraction seen from the previous step,
  // the next correction would be ~ (|dg| / dg_last^2) dg^2; below round-off,
  // accept gn without another pass (entropy change carried to gn to first order)
  const bool converged = newton && st->dg_last != 0.0 && fabs(dg) <= 1e-3 * fabs(st->dg_last) &&
                         fabs(dg) * (dg / st->dg_last) * (dg / st->dg_last) <= 4.0 * eps * fabs(gn);
  if (converged || fabs(dg) <= 4.0 * eps * fabs(g) || st->hi - st->lo <= 4.0 * eps * st->hi ||
      st->iters >= ROOT_EVALS_MAX) {
    st->g = gn;
    st->dS_last = tot[0] + dg * tot[1];
    st->done = 1;
    return;
  }
  st->dg_last = newton ? dg : 0.0;
  st->ga = gn;
}

template <bool COND>
static int root_eval_launch(esplit_ctx* c, const double* un, const double* d, cudaStream_t s,
                            cudaGraphConditionalHandle h) {
  size_t n = (size_t)c->n_e * c->n_p;
  int nb = (int)((n + 255) / 256);
  Phys<double> ph = make_phys<double>(c->prm.gam, c->prm.beta, c->prm.R, c->prm.mu, c->prm.Pr);
  if (c->dim == 1)
    root_eval_kernel<1, COND><<<nb, 256, 0, s>>>(un, d, c->b.J, c->b.node_cache, n, ph, c->b.root, c->b.partial, h);
  else if (c->dim == 2)
    root_eval_kernel<2, COND><<<nb, 256, 0, s>>>(un, d, c->b.J, c->b.node_cache, n, ph, c->b.root, c->b.partial, h);
  else
    root_eval_kernel<3, COND><<<nb, 256, 0, s>>>(un, d, c->b.J, c->b.node_cache, n, ph, c->b.root, c->b.partial, h);
  c->launches++;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_root_eval(esplit_ctx* c, const double* un, const double* d, cudaStream_t s) {
  ProfScope ps(c, PG_ROOT, s);
  return root_eval_launch<false>(c, un, d, s, 0);
}

int launch_root_eval_cond(esplit_ctx* c, const double* un, const double* d, cudaStream_t s,
                          cudaGraphConditionalHandle h) {
  return root_eval_launch<true>(c, un, d, s, h);
}

// one record per completed step of a graph-launched batch, at the slot the
// device counter names (the counter is reset by the host before each batch)
__global__ void step_record_kernel(const RootState* __restrict__ st, const int* __restrict__ status,
                                   const double* __restrict__ scal, StepRecord* __restrict__ hist, int* counter,
                                   int cap) {
  const int k = *counter;
  if (k < cap) {
    StepRecord r;
    r.g = st->g;
    r.est = st->est;
    r.S0 = st->S0;
    r.S_after = st->S0 + (st->phase == 3 ? st->dS_last : 0.0);
    for (int i = 0; i < 4; ++i) r.stage_rate[i] = scal[2 + i];
    r.iters = st->iters;
    r.status = (*status & 1) ? ESPLIT_ERR_NONPHYSICAL : st->status;
    hist[k] = r;
  }
  *counter = k + 1;
}

int launch_step_record(esplit_ctx* c, StepRecord* hist, int* counter, int cap, cudaStream_t s) {
  step_record_kernel<<<1, 1, 0, s>>>(c->b.root, c->b.status, c->b.scal, hist, counter, cap);
  c->launches++;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

__global__ void root_apply_kernel(double* __restrict__ un, const double* __restrict__ d, size_t n,
                                  const RootState* __restrict__ st, const int* __restrict__ status) {
  if (!st->done || st->status != 0 || *status != 0) return;
  double g = st->g;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (; i < n; i += stride) un[i] += g * d[i];
}

int launch_root_apply(esplit_ctx* c, double* un, const double* d, size_t n, cudaStream_t s) {
  ProfScope ps(c, PG_STAGE, s);
  root_apply_kernel<<<grid_for(n), 256, 0, s>>>(un, d, n, c->b.root, c->b.status);
  c->launches++;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_root_start(esplit_ctx* c, double dt, cudaStream_t s) {
  ProfScope ps(c, PG_ROOT, s);
  root_init_kernel<<<1, 1, 0, s>>>(c->b.root, c->b.scal, dt);
  c->launches++;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace esplit

#include "hybrid.cuh"

namespace esplit {

// elementwise evaluation of the table-driven functions (fn 0..3: log, log1p,
// exp, expm1) or of the CUDA library ones (fn 4..7), for their accuracy tests
__global__ void math_eval_kernel(int fn, const double* __restrict__ x, double* __restrict__ y, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v = x[i], out;
  switch (fn) {
    case 0: out = fm::log(v); break;
    case 1: out = fm::log1p(v); break;
    case 2: out = fm::exp(v); break;
    case 3: out = fm::expm1(v); break;
    case 4: out = ::log(v); break;
    case 5: out = ::log1p(v); break;
    case 6: out = ::exp(v); break;
    default: out = ::expm1(v); break;
  }
  y[i] = out;
}

int launch_math_eval(int fn, const double* x, double* y, size_t n, cudaStream_t s) {
  if (n == 0) return 0;
  math_eval_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(fn, x, y, n);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace esplit
