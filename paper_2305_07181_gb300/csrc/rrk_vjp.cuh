// Reverse mode of one relaxation RK4 step (Sec. 6.1, Eqs. (97)-(98)) and the
// entropy gradient.  Included by kernels.cu.
//
// Forward (recomputed from the checkpoint u_n):
//   U_1 = u_n, U_i = u_n + a_i dt r_(i-1), r_i = R(U_i), e_i = 1^T H (w(U_i) . r_i)
//   d = dt sum b_i r_i, est = dt sum b_i e_i, f(g) = 1^T H [s(u_n + g d) - s(u_n)] - g est = 0,
//   u' = u_n + g d.
// Reverse for the cotangent ubar' of u':
//   gbar = ubar' . d;  lambda = -gbar / f_g,  f_g = 1^T H (w(u') . d) - est   (implicit function)
//   ubar_n = ubar' + lambda H (w(u') - w(u_n)),  dbar = g ubar' + lambda g H w(u'),
//   estbar = -lambda g,  ebar_i = dt b_i estbar,
//   rbar_i = dt b_i dbar + ebar_i H w(U_i) + a_(i+1) dt Ubar_(i+1),
//   Ubar_i = R'(U_i)^T rbar_i + ebar_i (dw/dU(U_i))^T H r_i,  ubar_n += Ubar_i.
#pragma once

namespace esplit {

// out = scale * H w(u)   (the gradient of 1^T H s(u) is H w(u), Eq. (17))
template <int D>
__global__ void __launch_bounds__(256) wH_kernel(const double* __restrict__ u, const double* __restrict__ J,
                                                 size_t n_nodes, Phys<double> c, double scale,
                                                 double* __restrict__ out) {
  constexpr int NC = D + 2;
  const int NP = c_ref.n_p;
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_nodes) return;
  size_t e = t / NP;
  int m = (int)(t - e * NP);
  double uu[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) uu[q] = __ldg(&u[(e * NC + q) * NP + m]);
  Node<double, D> nd;
  node_from_u<double, D>(uu, c, nd);
  double H = scale * c_ref.H[m] * __ldg(&J[e * NP + m]);
#pragma unroll
  for (int q = 0; q < NC; ++q) out[(e * NC + q) * NP + m] = H * nd.W[q];
}

// block partials of [ubar' . d, 1^T H (w(u') . d)]
template <int D>
__global__ void __launch_bounds__(256) rrk_vjp_dots_kernel(const double* __restrict__ u1,
                                                           const double* __restrict__ d,
                                                           const double* __restrict__ ubar1,
                                                           const double* __restrict__ J, size_t n_nodes,
                                                           Phys<double> c, double* __restrict__ part) {
  constexpr int NC = D + 2;
  const int NP = c_ref.n_p;
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v[2] = {0.0, 0.0};
  if (t < n_nodes) {
    size_t e = t / NP;
    int m = (int)(t - e * NP);
    double uu[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) uu[q] = __ldg(&u1[(e * NC + q) * NP + m]);
    Node<double, D> nd;
    node_from_u<double, D>(uu, c, nd);
    double H = c_ref.H[m] * __ldg(&J[e * NP + m]);
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      size_t ix = (e * NC + q) * NP + m;
      double dq = __ldg(&d[ix]);
      v[0] += __ldg(&ubar1[ix]) * dq;
      v[1] += H * nd.W[q] * dq;
    }
  }
  block_sum<2>(v, part + 2 * blockIdx.x);
}

// ubar_n = ubar' + lam H (w(u') - w(u_n)),  dbar = g ubar' + lam g H w(u')
template <int D>
__global__ void __launch_bounds__(256) rrk_vjp_combine_kernel(const double* __restrict__ un,
                                                              const double* __restrict__ u1,
                                                              const double* __restrict__ ubar1,
                                                              const double* __restrict__ J, size_t n_nodes,
                                                              Phys<double> c, double lam, double g,
                                                              double* __restrict__ ubar0, double* __restrict__ dbar) {
  constexpr int NC = D + 2;
  const int NP = c_ref.n_p;
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_nodes) return;
  size_t e = t / NP;
  int m = (int)(t - e * NP);
  double a[NC], b[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    a[q] = __ldg(&un[(e * NC + q) * NP + m]);
    b[q] = __ldg(&u1[(e * NC + q) * NP + m]);
  }
  Node<double, D> n0, n1;
  node_from_u<double, D>(a, c, n0);
  node_from_u<double, D>(b, c, n1);
  double H = c_ref.H[m] * __ldg(&J[e * NP + m]);
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    size_t ix = (e * NC + q) * NP + m;
    double ub = __ldg(&ubar1[ix]);
    ubar0[ix] = ub + lam * H * (n1.W[q] - n0.W[q]);
    dbar[ix] = g * ub + lam * g * H * n1.W[q];
  }
}

// rbar = c_d dbar + c_e H w(U) + c_u Ubar_next ;  extra = c_e (dw/dU(U))^T (H r)
template <int D>
__global__ void __launch_bounds__(128) rrk_vjp_stage_kernel(const double* __restrict__ U,
                                                            const double* __restrict__ r,
                                                            const double* __restrict__ dbar,
                                                            const double* __restrict__ ubar_next,
                                                            const double* __restrict__ J, size_t n_nodes,
                                                            Phys<double> c, double c_d, double c_e, double c_u,
                                                            double* __restrict__ rbar, double* __restrict__ extra) {
  constexpr int NC = D + 2;
  using TD = Dual<NC>;
  const int NP = c_ref.n_p;
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_nodes) return;
  size_t e = t / NP;
  int m = (int)(t - e * NP);
  TD ud[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    ud[q] = TD(__ldg(&U[(e * NC + q) * NP + m]));
    ud[q].d[q] = 1.0;
  }
  Node<TD, D> nd;
  node_from_u<TD, D>(ud, c, nd);
  double H = c_ref.H[m] * __ldg(&J[e * NP + m]);
  double ex[NC];
#pragma unroll
  for (int cc = 0; cc < NC; ++cc) ex[cc] = 0.0;
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    size_t ix = (e * NC + q) * NP + m;
    double rb = c_d * __ldg(&dbar[ix]) + c_e * H * nd.W[q].v;
    if (ubar_next) rb += c_u * __ldg(&ubar_next[ix]);
    rbar[ix] = rb;
    double hr = c_e * H * __ldg(&r[ix]);
#pragma unroll
    for (int cc = 0; cc < NC; ++cc) ex[cc] += hr * nd.W[q].d[cc];
  }
#pragma unroll
  for (int cc = 0; cc < NC; ++cc) extra[(e * NC + cc) * NP + m] = ex[cc];
}

static inline unsigned nblocks(size_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

int launch_wH(esplit_ctx* c, const double* u, double scale, double* out, cudaStream_t s) {
  size_t n = (size_t)c->n_e * c->n_p;
  Phys<double> ph = make_phys<double>(c->prm.gam, c->prm.beta, c->prm.R, c->prm.mu, c->prm.Pr);
  if (c->dim == 1)
    wH_kernel<1><<<nblocks(n, 256), 256, 0, s>>>(u, c->b.J, n, ph, scale, out);
  else if (c->dim == 2)
    wH_kernel<2><<<nblocks(n, 256), 256, 0, s>>>(u, c->b.J, n, ph, scale, out);
  else
    wH_kernel<3><<<nblocks(n, 256), 256, 0, s>>>(u, c->b.J, n, ph, scale, out);
  c->launches++;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_rrk_vjp_dots(esplit_ctx* c, const double* u1, const double* d, const double* ubar1, cudaStream_t s,
                        int* n_partial) {
  size_t n = (size_t)c->n_e * c->n_p;
  Phys<double> ph = make_phys<double>(c->prm.gam, c->prm.beta, c->prm.R, c->prm.mu, c->prm.Pr);
  unsigned nb = nblocks(n, 256);
  if (c->dim == 1)
    rrk_vjp_dots_kernel<1><<<nb, 256, 0, s>>>(u1, d, ubar1, c->b.J, n, ph, c->b.partial);
  else if (c->dim == 2)
    rrk_vjp_dots_kernel<2><<<nb, 256, 0, s>>>(u1, d, ubar1, c->b.J, n, ph, c->b.partial);
  else
    rrk_vjp_dots_kernel<3><<<nb, 256, 0, s>>>(u1, d, ubar1, c->b.J, n, ph, c->b.partial);
  c->launches++;
  *n_partial = (int)nb;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_rrk_vjp_combine(esplit_ctx* c, const double* un, const double* u1, const double* ubar1, double lam,
                           double g, double* ubar0, double* dbar, cudaStream_t s) {
  size_t n = (size_t)c->n_e * c->n_p;
  Phys<double> ph = make_phys<double>(c->prm.gam, c->prm.beta, c->prm.R, c->prm.mu, c->prm.Pr);
  if (c->dim == 1)
    rrk_vjp_combine_kernel<1><<<nblocks(n, 256), 256, 0, s>>>(un, u1, ubar1, c->b.J, n, ph, lam, g, ubar0, dbar);
  else if (c->dim == 2)
    rrk_vjp_combine_kernel<2><<<nblocks(n, 256), 256, 0, s>>>(un, u1, ubar1, c->b.J, n, ph, lam, g, ubar0, dbar);
  else
    rrk_vjp_combine_kernel<3><<<nblocks(n, 256), 256, 0, s>>>(un, u1, ubar1, c->b.J, n, ph, lam, g, ubar0, dbar);
  c->launches++;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_rrk_vjp_stage(esplit_ctx* c, const double* U, const double* r, const double* dbar,
                         const double* ubar_next, double c_d, double c_e, double c_u, double* rbar, double* extra,
                         cudaStream_t s) {
  size_t n = (size_t)c->n_e * c->n_p;
  Phys<double> ph = make_phys<double>(c->prm.gam, c->prm.beta, c->prm.R, c->prm.mu, c->prm.Pr);
  if (c->dim == 1)
    rrk_vjp_stage_kernel<1><<<nblocks(n, 128), 128, 0, s>>>(U, r, dbar, ubar_next, c->b.J, n, ph, c_d, c_e, c_u,
                                                            rbar, extra);
  else if (c->dim == 2)
    rrk_vjp_stage_kernel<2><<<nblocks(n, 128), 128, 0, s>>>(U, r, dbar, ubar_next, c->b.J, n, ph, c_d, c_e, c_u,
                                                            rbar, extra);
  else
    rrk_vjp_stage_kernel<3><<<nblocks(n, 128), 128, 0, s>>>(U, r, dbar, ubar_next, c->b.J, n, ph, c_d, c_e, c_u,
                                                            rbar, extra);
  c->launches++;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace esplit
