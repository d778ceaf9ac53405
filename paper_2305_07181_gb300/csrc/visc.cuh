// Viscous terms of the compressible Navier-Stokes residual with Baumann-Oden
// SATs, Sec. 5, Eqs. (83)-(85) and (96) (T1 = 0, T2 = T3 = B/2):
//   r += sum_i D_i F^V_i
//        - (1/(2 H_m)) nu . (F^V_k(m) - F^V_v(n))                 at facet nodes
//        - 1/2 H^-1 sum_j D_j^T a_j,   a_j(m) = sum_i K~_ij^T nu_i (w_k,m - w_v,n)
// with F^V_i = sum_j K~_ij dW/dx_j the flux of Eq. (5) written with the
// entropy-variable gradients (Sec. 3), D_j w = dW/dx_j.
//
// The lift is folded into the divergence: D_j = H^-1 Q_j and Q_j^T = E_j - Q_j
// (Def. 1) give H^-1 D_j^T a = (E_j/H)(a/H) - D_j (a/H), so
//   r += sum_i D_i (F^V_i + a_i/(2H))  -  sum_i nu_i a_i / (2 H^2)   (facet nodes)
//        + jump / H:
// one contraction instead of two.  The pieces are computed where their inputs
// already are: a_i/H by the facet kernel (it has both nodal states), F^V and
// the divergence by the entropy-split volume kernel (it has D_i w; float64 in
// both precision modes) or, for Hadamard-form elements, by visc_volume_kernel
// below; the flux jump needs F^V of both sides and runs last
// (visc_jump_kernel).  The facet
// arrays: ah [n_e][d][n_c][n_slot] (a/H), fvs [n_e][d][n_c][n_slot] (F^V at
// the facet nodes).  Included by kernels.cu.
#pragma once

namespace esplit {

// F^V, the folded divergence and the facet correction for the elements of
// `list` (all when null); adds into r, writes F^V at the facet slots.  ENT:
// the entropy variables the gradients are taken of (0 Harten's, 1 the
// standard ones of the Ismail-Roe comparator); the flux is the same physical
// viscous flux either way.
template <int D, int NP, int EB, int ENT = 0>
__global__ void __launch_bounds__(EB * NP) visc_volume_kernel(const double* __restrict__ u, double* __restrict__ r,
                                                              const double* __restrict__ ops,
                                                              const double* __restrict__ J,
                                                              const double* __restrict__ nu,
                                                              const double* __restrict__ ah, const int* __restrict__ list,
                                                              int n_list, double* __restrict__ fvs, Phys<double> c,
                                                              int heat) {
  constexpr int NC = D + 2;
  __shared__ double sw[EB][NC][NP];
  __shared__ double sF[EB][D][NC][NP];
  const int NS = c_ref.n_slot;
  int el = threadIdx.x / NP;
  int m = threadIdx.x - el * NP;
  int li = blockIdx.x * EB + el;
  bool active = li < n_list;
  int e = active ? (list ? list[li] : li) : 0;
  int sl = c_ref.node_slot[m];
  Node<double, D> nd;
  if (active) {
    double uu[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) uu[q] = __ldg(&u[((size_t)e * NC + q) * NP + m]);
    node_from_u<double, D>(uu, c, nd);
    if constexpr (ENT == 1) {
      double w[NC];
      std_entropy_vars_node(nd, c, w);
#pragma unroll
      for (int q = 0; q < NC; ++q) sw[el][q][m] = w[q];
    } else {
#pragma unroll
      for (int q = 0; q < NC; ++q) sw[el][q][m] = nd.W[q];
    }
  }
  __syncthreads();
  const double* op = ops + (size_t)e * (2 * D * NP * NP);
  double Hm = 0.0;
  if (active) {
    double g[D][NC];
#pragma unroll
    for (int j = 0; j < D; ++j)
#pragma unroll
      for (int q = 0; q < NC; ++q) g[j][q] = 0.0;
#pragma unroll
    for (int j = 0; j < D; ++j)
      for (int n = 0; n < NP; ++n) {
        double dt = __ldg(&op[((D + j) * NP + n) * NP + m]);  // D_j[m][n]
#pragma unroll
        for (int q = 0; q < NC; ++q) g[j][q] += dt * sw[el][q][n];
      }
    double F[D][NC];
    visc_flux<double, D, double, ENT>(nd, c, heat, g, F);
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        double f = F[i][q];
        if (sl >= 0) {
          size_t ix = (((size_t)e * D + i) * NC + q) * NS + sl;
          fvs[ix] = f;
          f += 0.5 * __ldg(&ah[ix]);
        }
        sF[el][i][q][m] = f;
      }
    Hm = c_ref.H[m] * __ldg(&J[(size_t)e * NP + m]);
  }
  __syncthreads();
  if (!active) return;
  double acc[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) acc[q] = 0.0;
#pragma unroll
  for (int i = 0; i < D; ++i)
    for (int n = 0; n < NP; ++n) {
      double dt = __ldg(&op[((D + i) * NP + n) * NP + m]);
#pragma unroll
      for (int q = 0; q < NC; ++q) acc[q] += dt * sF[el][i][q][n];
    }
  if (sl >= 0) {
    double ih = 1.0 / Hm;
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      double corr = 0.0;
#pragma unroll
      for (int i = 0; i < D; ++i)
        corr += __ldg(&nu[((size_t)e * NS + sl) * D + i]) * __ldg(&ah[(((size_t)e * D + i) * NC + q) * NS + sl]);
      acc[q] -= 0.5 * corr * ih;
    }
  }
#pragma unroll
  for (int q = 0; q < NC; ++q) r[((size_t)e * NC + q) * NP + m] += acc[q];
}

// flux jump, one thread per coincident node pair: -(1/2) nu . (F_k - F_v)
// divided by the node's H on both sides (identical on both since nu_v = -nu).
// With prod: block partials of its entropy production, (w_k + w_v) . jump
// (H r . w at both nodes), from the entropy variables at the slots (wsl).
template <int D>
__global__ void __launch_bounds__(128) visc_jump_kernel(double* __restrict__ r, const double* __restrict__ fvs,
                                                        const int2* __restrict__ fp, int n_pairs,
                                                        const double* __restrict__ nu, const double* __restrict__ J,
                                                        const double* __restrict__ wsl, double* __restrict__ prod) {
  constexpr int NC = D + 2;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  double hw = 0.0;
  if (t < n_pairs) {
    const int NP = c_ref.n_p, NS = c_ref.n_slot;
    int2 pr = __ldg(&fp[t]);
    int k = pr.x / NS, s = pr.x - k * NS;
    int v = pr.y / NS, s2 = pr.y - v * NS;
    int m = c_ref.slot_node[s], n = c_ref.slot_node[s2];
    double ihk = 1.0 / (c_ref.H[m] * __ldg(&J[(size_t)k * NP + m]));
    double ihv = 1.0 / (c_ref.H[n] * __ldg(&J[(size_t)v * NP + n]));
    double nuv[D];
#pragma unroll
    for (int i = 0; i < D; ++i) nuv[i] = __ldg(&nu[((size_t)k * NS + s) * D + i]);
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      double d = 0.0;
#pragma unroll
      for (int i = 0; i < D; ++i)
        d += nuv[i] * (__ldg(&fvs[(((size_t)k * D + i) * NC + q) * NS + s]) -
                       __ldg(&fvs[(((size_t)v * D + i) * NC + q) * NS + s2]));
      double jump = -0.5 * d;
      r[((size_t)k * NC + q) * NP + m] += jump * ihk;
      r[((size_t)v * NC + q) * NP + n] += jump * ihv;
      if (prod)
        hw += (__ldg(&wsl[((size_t)k * NC + q) * NS + s]) + __ldg(&wsl[((size_t)v * NC + q) * NS + s2])) * jump;
    }
  }
  if (prod) {
    double vv[1] = {hw};
    block_sum_t<1, 128>(vv, prod + blockIdx.x);
  }
}

template <int D, int NP>
static void viscous_volume_np(esplit_ctx* c, const double* u, double* r, const int* list, int n_list,
                              cudaStream_t s) {
  const Phys<double> ph = make_phys<double>(c->prm.gam, c->prm.beta, c->prm.R, c->prm.mu, c->prm.Pr);
  constexpr int EB = (128 / NP) > 0 ? (128 / NP) : 1;
  int nb = (n_list + EB - 1) / EB;
  if (c->prm.scheme == ESPLIT_SCHEME_HADAMARD_IR)
    visc_volume_kernel<D, NP, EB, 1><<<nb, EB * NP, 0, s>>>(u, r, c->b.ops64, c->b.J, c->b.nu, c->b.va, list,
                                                            n_list, c->b.fv, ph, c->prm.heat_flux);
  else
    visc_volume_kernel<D, NP, EB><<<nb, EB * NP, 0, s>>>(u, r, c->b.ops64, c->b.J, c->b.nu, c->b.va, list, n_list,
                                                         c->b.fv, ph, c->prm.heat_flux);
  c->launches += 1;
}

// returns the number of block partials written to prod (0 without prod)
template <int D>
static int viscous_jump(esplit_ctx* c, double* r, cudaStream_t s, double* prod = nullptr) {
  int bs = 128;
  int nb = (c->n_pairs + bs - 1) / bs;
  visc_jump_kernel<D><<<nb, bs, 0, s>>>(r, c->b.fv, c->b.face_pairs, c->n_pairs, c->b.nu, c->b.J, c->b.wslot,
                                        prod);
  c->launches += 1;
  return prod ? nb : 0;
}

}  // namespace esplit
