// Viscous terms of the compressible Navier-Stokes residual with Baumann-Oden
// SATs, Sec. 5, Eqs. (83)-(85) and (96) (T1 = 0, T2 = T3 = B/2):
//   r += sum_i D_i F^V_i
//        - (1/(2 H_m)) nu . (F^V_k(m) - F^V_v(n))                 at facet nodes
//        - 1/2 H^-1 sum_j D_j^T a_j,   a_j(m) = sum_i K~_ij^T nu_i (w_k,m - w_v,n)
// with F^V_i = sum_j K~_ij dW/dx_j the flux of Eq. (5) written with the
// entropy-variable gradients (Sec. 3), D_j w = dW/dx_j.  Included by kernels.cu.
#pragma once

namespace esplit {

// dT/dW of Eq. (39) (the exact derivative; the printed Eq. (40) has a sign
// typo in the momentum entries and drops alpha in the last entry).  T is
// double or a dual number (the reverse mode differentiates these in u).
template <typename T, int D>
__device__ __forceinline__ void dT_dW(const Node<T, D>& n, const Phys<double>& c, T* TW) {
  constexpr int NC = D + 2;
  T Wn = -n.q;
  T k = c.gm1 / (c.alpha * c.R * Wn);
  T T_ = n.p * n.ir / c.R;
  TW[0] = k;
#pragma unroll
  for (int l = 0; l < D; ++l) TW[1 + l] = k * n.V[l];
  TW[NC - 1] = -T_ / Wn + 0.5 * k * n.v2;
}

// F^V_i (i < D) from the entropy-variable gradients g[j] = dW/dx_j:
//   dV_l/dx_j = -(g_j[1+l] + V_l g_j[nc]) / W_nc,  dT/dx_j = dT/dW . g_j,
//   tau_ik = mu (dV_i/dx_k + dV_k/dx_i - 2/3 delta_ik div V),
//   F_i = [0, tau_i., V . tau_i. + kappa dT/dx_i]
template <typename T, int D, typename G>
__device__ __forceinline__ void visc_flux(const Node<T, D>& n, const Phys<double>& c, int heat, const G (&g)[D][D + 2],
                                          T (&F)[D][D + 2]) {
  constexpr int NC = D + 2;
  T iWn = -1.0 / n.q;
  T Lg[D][D];  // Lg[j][l] = dV_l/dx_j
  T div = T(0.0);
#pragma unroll
  for (int j = 0; j < D; ++j)
#pragma unroll
    for (int l = 0; l < D; ++l) Lg[j][l] = -(g[j][1 + l] + n.V[l] * g[j][NC - 1]) * iWn;
#pragma unroll
  for (int l = 0; l < D; ++l) div = div + Lg[l][l];
  T TW[NC];
  dT_dW<T, D>(n, c, TW);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    T e = T(0.0);
    F[i][0] = T(0.0);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      T tau = c.mu * (Lg[k][i] + Lg[i][k] - (k == i ? (2.0 / 3.0) * div : T(0.0)));
      F[i][1 + k] = tau;
      e = e + n.V[k] * tau;
    }
    if (heat) {
      T dT = T(0.0);
#pragma unroll
      for (int q = 0; q < NC; ++q) dT = dT + TW[q] * g[i][q];
      e = e + c.kappa * dT;
    }
    F[i][NC - 1] = e;
  }
}

// a_j = sum_i K~_ij^T b_i: the gradient of sum_i b_i . F^V_i with respect to
// g_j (F^V is linear in the gradients).
template <typename T, int D, typename B>
__device__ __forceinline__ void visc_flux_transpose(const Node<T, D>& n, const Phys<double>& c, int heat,
                                                    const B (&b)[D][D + 2], T (&a)[D][D + 2]) {
  constexpr int NC = D + 2;
  T iWn = -1.0 / n.q;
  T cc[D][D];
  T trc = T(0.0);
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int k = 0; k < D; ++k) cc[i][k] = b[i][1 + k] + b[i][NC - 1] * n.V[k];
#pragma unroll
  for (int i = 0; i < D; ++i) trc = trc + cc[i][i];
  T TW[NC];
  dT_dW<T, D>(n, c, TW);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    T hj = heat ? c.kappa * b[j][NC - 1] : T(0.0);
    T sv = T(0.0);
    a[j][0] = hj * TW[0];
#pragma unroll
    for (int l = 0; l < D; ++l) {
      T G = c.mu * (cc[j][l] + cc[l][j] - (j == l ? (2.0 / 3.0) * trc : T(0.0)));
      a[j][1 + l] = -G * iWn + hj * TW[1 + l];
      sv = sv + G * n.V[l];
    }
    a[j][NC - 1] = -sv * iWn + hj * TW[NC - 1];
  }
}

// element pass: F^V at the nodes (kept in fv for the facet pass) and
// r += sum_i D_i F^V_i
template <int D, int NP, int EB>
__global__ void __launch_bounds__(EB * NP) visc_volume_kernel(const double* __restrict__ u, double* __restrict__ r,
                                                              const double* __restrict__ ops, int n_e,
                                                              double* __restrict__ fv, Phys<double> c, int heat) {
  constexpr int NC = D + 2;
  __shared__ double sw[EB][NC][NP];
  __shared__ double sF[EB][D][NC][NP];
  int el = threadIdx.x / NP;
  int m = threadIdx.x - el * NP;
  int e = blockIdx.x * EB + el;
  bool active = e < n_e;
  Node<double, D> nd;
  if (active) {
    double uu[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) uu[q] = __ldg(&u[((size_t)e * NC + q) * NP + m]);
    node_from_u<double, D>(uu, c, nd);
#pragma unroll
    for (int q = 0; q < NC; ++q) sw[el][q][m] = nd.W[q];
  }
  __syncthreads();
  const double* op = ops + (size_t)(active ? e : 0) * (2 * D * NP * NP);
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
    visc_flux<double, D>(nd, c, heat, g, F);
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        sF[el][i][q][m] = F[i][q];
        fv[(((size_t)e * D + i) * NC + q) * NP + m] = F[i][q];
      }
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
#pragma unroll
  for (int q = 0; q < NC; ++q) r[((size_t)e * NC + q) * NP + m] += acc[q];
}

// facet pass, one thread per coincident node pair: the flux-jump term for
// both sides (-(1/2) nu . (F_k - F_v), identical on both sides since nu_v = -nu)
// and a_j on both sides (side v: sum_i K~_ij(u_v)^T nu_i dw with the same
// nu and dw = w_k - w_v, the two sign flips cancelling).
template <int D>
__global__ void __launch_bounds__(128) visc_face_kernel(const double* __restrict__ u, const double* __restrict__ fv,
                                                        const int2* __restrict__ fp, int n_pairs,
                                                        const double* __restrict__ nu, double* __restrict__ vsat,
                                                        double* __restrict__ va, Phys<double> c, int heat) {
  constexpr int NC = D + 2;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_pairs) return;
  const int NP = c_ref.n_p, NS = c_ref.n_slot;
  int2 pr = __ldg(&fp[t]);
  int k = pr.x / NS, s = pr.x - k * NS;
  int v = pr.y / NS, s2 = pr.y - v * NS;
  int m = c_ref.slot_node[s], n = c_ref.slot_node[s2];
  double uk[NC], uv[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    uk[q] = __ldg(&u[((size_t)k * NC + q) * NP + m]);
    uv[q] = __ldg(&u[((size_t)v * NC + q) * NP + n]);
  }
  Node<double, D> nk, nv;
  node_from_u<double, D>(uk, c, nk);
  node_from_u<double, D>(uv, c, nv);
  double nuv[D];
#pragma unroll
  for (int i = 0; i < D; ++i) nuv[i] = __ldg(&nu[((size_t)k * NS + s) * D + i]);
  double jump[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    double d = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i)
      d += nuv[i] * (__ldg(&fv[(((size_t)k * D + i) * NC + q) * NP + m]) -
                     __ldg(&fv[(((size_t)v * D + i) * NC + q) * NP + n]));
    jump[q] = -0.5 * d;
  }
  double b[D][NC];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int q = 0; q < NC; ++q) b[i][q] = nuv[i] * (nk.W[q] - nv.W[q]);
  double ak[D][NC], av[D][NC];
  visc_flux_transpose<double, D>(nk, c, heat, b, ak);
  visc_flux_transpose<double, D>(nv, c, heat, b, av);
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    vsat[((size_t)k * NC + q) * NS + s] = jump[q];
    vsat[((size_t)v * NC + q) * NS + s2] = jump[q];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      va[(((size_t)k * D + j) * NC + q) * NS + s] = ak[j][q];
      va[(((size_t)v * D + j) * NC + q) * NS + s2] = av[j][q];
    }
  }
}

// lift pass: r_m += vsat_m / H_m - (1/(2 H_m)) sum_j sum_(facet n) D_j[n][m] a_j(n)
template <int D, int NP, int EB>
__global__ void __launch_bounds__(EB * NP) visc_lift_kernel(double* __restrict__ r, const double* __restrict__ ops,
                                                            const double* __restrict__ J,
                                                            const double* __restrict__ vsat,
                                                            const double* __restrict__ va, int n_e) {
  constexpr int NC = D + 2;
  int el = threadIdx.x / NP;
  int m = threadIdx.x - el * NP;
  int e = blockIdx.x * EB + el;
  if (e >= n_e) return;
  const int NS = c_ref.n_slot;
  const double* op = ops + (size_t)e * (2 * D * NP * NP);
  double acc[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) acc[q] = 0.0;
  for (int s = 0; s < NS; ++s) {
    int n = c_ref.slot_node[s];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      double dt = __ldg(&op[((D + j) * NP + m) * NP + n]);  // D_j[n][m]
#pragma unroll
      for (int q = 0; q < NC; ++q) acc[q] += dt * __ldg(&va[(((size_t)e * D + j) * NC + q) * NS + s]);
    }
  }
  double ih = 1.0 / (c_ref.H[m] * __ldg(&J[(size_t)e * NP + m]));
  int sl = c_ref.node_slot[m];
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    double add = -0.5 * acc[q];
    if (sl >= 0) add += __ldg(&vsat[((size_t)e * NC + q) * NS + sl]);
    r[((size_t)e * NC + q) * NP + m] += add * ih;
  }
}

template <int D, int NP>
static int viscous_np(esplit_ctx* c, const double* u, double* r, cudaStream_t s) {
  const Phys<double> ph = make_phys<double>(c->prm.gam, c->prm.beta, c->prm.R, c->prm.mu, c->prm.Pr);
  constexpr int EB = (128 / NP) > 0 ? (128 / NP) : 1;
  int nb = (c->n_e + EB - 1) / EB;
  visc_volume_kernel<D, NP, EB><<<nb, EB * NP, 0, s>>>(u, r, c->b.ops64, c->n_e, c->b.fv, ph, c->prm.heat_flux);
  int bs = 128;
  visc_face_kernel<D><<<(c->n_pairs + bs - 1) / bs, bs, 0, s>>>(u, c->b.fv, c->b.face_pairs, c->n_pairs, c->b.nu,
                                                                  c->b.vsat, c->b.va, ph, c->prm.heat_flux);
  visc_lift_kernel<D, NP, EB><<<nb, EB * NP, 0, s>>>(r, c->b.ops64, c->b.J, c->b.vsat, c->b.va, c->n_e);
  c->launches += 3;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_viscous(esplit_ctx* c, const double* u, double* r, cudaStream_t s) {
  ProfScope ps(c, PG_VISC, s);
  if (c->dim == 2) {
    switch (c->n_p) {
      case 7: return viscous_np<2, 7>(c, u, r, s);
      case 12: return viscous_np<2, 12>(c, u, r, s);
      case 18: return viscous_np<2, 18>(c, u, r, s);
      case 27: return viscous_np<2, 27>(c, u, r, s);
    }
  } else if (c->dim == 3) {
    switch (c->n_p) {
      case 25: return viscous_np<3, 25>(c, u, r, s);
    }
  }
  return -2;
}

}  // namespace esplit
