// Reverse mode of the viscous Baumann-Oden terms (Sec. 5, Eqs. (83)-(85),
// (96)), added to the inviscid VJP.  With g_j = D_j w (entropy-variable
// gradients), F_i = F^V_i(u, g) = sum_j K~_ij(u) g_j, the viscous part of the
// residual at node m of element k is
//   sum_i (D_i F_i)_m                                   (volume)
//   + jump_m / H_m,  jump = -1/2 nu . (F_k(m) - F_v(n)) (facet pair, both sides)
//   - 1/(2 H_m) sum_j (D_j^T a_j)_m,  a_j(n) = sum_i K~_ij(u_n)^T nu_i (w_k - w_v)
// Given the cotangent cb, its transpose runs backwards through these:
//   Fb_i   = D_i^T cb  +  at facet pairs -/+ 1/2 nu_i (cb_k/H_k + cb_v/H_v)
//   ab_j   = -1/2 (D_j (cb/H)) at the facet nodes (both sides)
//   b_i    = nu_i (w_k - w_v);  bb = K~(u_k) ab_k + K~(u_v) ab_v (F^V applied
//            to ab as if it were a gradient), dwb = sum_i nu_i bb_i -> +w_k, -w_v
//   gb_j   = sum_i K~_ij^T Fb_i           (visc_flux_transpose)
//   wb     = sum_j D_j^T gb_j  + the facet dwb
//   grad  += (dw/du)^T wb + d/du[Fb . F^V(u, g)]|_g + d/du[ab . K~(u)^T b]|_b
// The u-derivatives at fixed g / b are exact, by dual numbers over u (the
// same templates as the forward kernels).  Three passes: element (gradients,
// D_i^T cb, ab), facet pairs (jump and lift transposes), element (the
// K~^T products, the D_j^T contraction, the pointwise Jacobians).  Float64.
// Included by kernels.cu.
#pragma once

namespace esplit {

// pass 1: g = D w -> gs, Fb_vol = D^T cb -> fbv, ab at the facet slots -> abs_
template <int D, int NP, int EB>
__global__ void __launch_bounds__(EB * NP) visc_vjp1_kernel(const double* __restrict__ u,
                                                            const double* __restrict__ cot,
                                                            const double* __restrict__ ops,
                                                            const double* __restrict__ J, int n_e,
                                                            double* __restrict__ gs, double* __restrict__ fbv,
                                                            double* __restrict__ abs_, Phys<double> c) {
  constexpr int NC = D + 2;
  __shared__ double sw[EB][NC][NP];
  __shared__ double sc[EB][NC][NP];   // cot
  __shared__ double sch[EB][NC][NP];  // cot / H
  const int NS = c_ref.n_slot;
  int el = threadIdx.x / NP;
  int m = threadIdx.x - el * NP;
  int e = blockIdx.x * EB + el;
  bool active = e < n_e;
  if (active) {
    double uu[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) uu[q] = __ldg(&u[((size_t)e * NC + q) * NP + m]);
    Node<double, D> nd;
    node_from_u<double, D>(uu, c, nd);
    double ih = 1.0 / (c_ref.H[m] * __ldg(&J[(size_t)e * NP + m]));
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      double cb = __ldg(&cot[((size_t)e * NC + q) * NP + m]);
      sw[el][q][m] = nd.W[q];
      sc[el][q][m] = cb;
      sch[el][q][m] = cb * ih;
    }
  }
  __syncthreads();
  if (!active) return;
  const double* op = ops + (size_t)e * (2 * D * NP * NP);
  double g[D][NC], fb[D][NC], ab[D][NC];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int q = 0; q < NC; ++q) g[i][q] = fb[i][q] = ab[i][q] = 0.0;
#pragma unroll
  for (int i = 0; i < D; ++i)
    for (int n = 0; n < NP; ++n) {
      double dmn = __ldg(&op[((D + i) * NP + n) * NP + m]);  // D_i[m][n]
      double dnm = __ldg(&op[((D + i) * NP + m) * NP + n]);  // D_i[n][m]
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        g[i][q] += dmn * sw[el][q][n];
        ab[i][q] += dmn * sch[el][q][n];
        fb[i][q] += dnm * sc[el][q][n];
      }
    }
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      gs[(((size_t)e * D + i) * NC + q) * NP + m] = g[i][q];
      fbv[(((size_t)e * D + i) * NC + q) * NP + m] = fb[i][q];
    }
  int sl = c_ref.node_slot[m];
  if (sl >= 0) {
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int q = 0; q < NC; ++q) abs_[(((size_t)e * D + i) * NC + q) * NS + sl] = -0.5 * ab[i][q];
  }
}

// pass 2, one thread per facet node pair: Fb facet parts -> fbs (both slots),
// dwb -> wbs (+ side k, - side v), d/du[ab . K~(u)^T b] -> ubs (both slots)
template <int D>
__global__ void __launch_bounds__(64) visc_vjp2_kernel(const double* __restrict__ u, const double* __restrict__ cot,
                                                       const int2* __restrict__ fp, int n_pairs,
                                                       const double* __restrict__ nu, const double* __restrict__ J,
                                                       const double* __restrict__ abs_, double* __restrict__ fbs,
                                                       double* __restrict__ wbs, double* __restrict__ ubs,
                                                       Phys<double> c, int heat) {
  constexpr int NC = D + 2;
  using TD = Dual<NC>;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_pairs) return;
  const int NP = c_ref.n_p, NS = c_ref.n_slot;
  int2 pr = __ldg(&fp[t]);
  int k = pr.x / NS, s = pr.x - k * NS;
  int v = pr.y / NS, s2 = pr.y - v * NS;
  int m = c_ref.slot_node[s], n = c_ref.slot_node[s2];
  double nuv[D];
#pragma unroll
  for (int i = 0; i < D; ++i) nuv[i] = __ldg(&nu[((size_t)k * NS + s) * D + i]);
  double ihk = 1.0 / (c_ref.H[m] * __ldg(&J[(size_t)k * NP + m]));
  double ihv = 1.0 / (c_ref.H[n] * __ldg(&J[(size_t)v * NP + n]));
  // flux-jump transpose
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    double jb = __ldg(&cot[((size_t)k * NC + q) * NP + m]) * ihk + __ldg(&cot[((size_t)v * NC + q) * NP + n]) * ihv;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      fbs[(((size_t)k * D + i) * NC + q) * NS + s] = -0.5 * nuv[i] * jb;
      fbs[(((size_t)v * D + i) * NC + q) * NS + s2] = 0.5 * nuv[i] * jb;
    }
  }
  // lift transpose; states with dual parts for the u-derivatives at fixed b
  TD uk[NC], uv[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    uk[q] = TD(__ldg(&u[((size_t)k * NC + q) * NP + m]));
    uv[q] = TD(__ldg(&u[((size_t)v * NC + q) * NP + n]));
    uk[q].d[q] = 1.0;
    uv[q].d[q] = 1.0;
  }
  Node<TD, D> nk, nv;
  node_from_u<TD, D>(uk, c, nk);
  node_from_u<TD, D>(uv, c, nv);
  double b[D][NC], abk[D][NC], abv[D][NC];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      b[i][q] = nuv[i] * (nk.W[q].v - nv.W[q].v);
      abk[i][q] = __ldg(&abs_[(((size_t)k * D + i) * NC + q) * NS + s]);
      abv[i][q] = __ldg(&abs_[(((size_t)v * D + i) * NC + q) * NS + s2]);
    }
  // a = K~(u)^T b on each side, differentiated in u at fixed b
  TD ak[D][NC], av[D][NC];
  visc_flux_transpose<TD, D>(nk, c, heat, b, ak);
  visc_flux_transpose<TD, D>(nv, c, heat, b, av);
  double gk[NC], gv[NC];
#pragma unroll
  for (int cc = 0; cc < NC; ++cc) {
    double sk = 0.0, sv = 0.0;
#pragma unroll
    for (int j = 0; j < D; ++j)
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        sk += abk[j][q] * ak[j][q].d[cc];
        sv += abv[j][q] * av[j][q].d[cc];
      }
    gk[cc] = sk;
    gv[cc] = sv;
  }
  // bb = K~(u_k) ab_k + K~(u_v) ab_v; dwb = sum_i nu_i bb_i
  Node<double, D> nk0, nv0;
  {
    double u0[NC], u1[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      u0[q] = uk[q].v;
      u1[q] = uv[q].v;
    }
    node_from_u<double, D>(u0, c, nk0);
    node_from_u<double, D>(u1, c, nv0);
  }
  double Fk[D][NC], Fv[D][NC];
  visc_flux<double, D>(nk0, c, heat, abk, Fk);
  visc_flux<double, D>(nv0, c, heat, abv, Fv);
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    double dwb = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i) dwb += nuv[i] * (Fk[i][q] + Fv[i][q]);
    wbs[((size_t)k * NC + q) * NS + s] = dwb;
    wbs[((size_t)v * NC + q) * NS + s2] = -dwb;
    ubs[((size_t)k * NC + q) * NS + s] = gk[q];
    ubs[((size_t)v * NC + q) * NS + s2] = gv[q];
  }
}

// pass 3: Fb = fbv (+ fbs), gb = K~^T Fb, wb = sum_j D_j^T gb_j (+ wbs),
// grad += (dw/du)^T wb + d/du[Fb . F^V(u, g)] (+ ubs)
template <int D, int NP, int EB>
__global__ void __launch_bounds__(EB * NP) visc_vjp3_kernel(const double* __restrict__ u,
                                                            const double* __restrict__ ops, int n_e,
                                                            const double* __restrict__ gs,
                                                            const double* __restrict__ fbv,
                                                            const double* __restrict__ fbs,
                                                            const double* __restrict__ wbs,
                                                            const double* __restrict__ ubs,
                                                            double* __restrict__ grad, Phys<double> c, int heat) {
  constexpr int NC = D + 2;
  using TD = Dual<NC>;
  __shared__ double sgb[EB][D][NC][NP];
  const int NS = c_ref.n_slot;
  int el = threadIdx.x / NP;
  int m = threadIdx.x - el * NP;
  int e = blockIdx.x * EB + el;
  bool active = e < n_e;
  int sl = c_ref.node_slot[m];
  double gr[NC];
  TD ud[NC];
  Node<TD, D> ndd;
  if (active) {
    double fb[D][NC], g[D][NC];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        size_t ix = (((size_t)e * D + i) * NC + q) * NP + m;
        fb[i][q] = __ldg(&fbv[ix]);
        g[i][q] = __ldg(&gs[ix]);
        if (sl >= 0) fb[i][q] += __ldg(&fbs[(((size_t)e * D + i) * NC + q) * NS + sl]);
      }
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      ud[q] = TD(__ldg(&u[((size_t)e * NC + q) * NP + m]));
      ud[q].d[q] = 1.0;
    }
    node_from_u<TD, D>(ud, c, ndd);
    // d/du [Fb . F^V(u, g)] at fixed g
    TD F[D][NC];
    visc_flux<TD, D>(ndd, c, heat, g, F);
#pragma unroll
    for (int cc = 0; cc < NC; ++cc) {
      double sacc = 0.0;
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int q = 0; q < NC; ++q) sacc += fb[i][q] * F[i][q].d[cc];
      gr[cc] = sacc;
    }
    // gb = K~^T Fb at u_m
    Node<double, D> nd;
    double u0[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) u0[q] = ud[q].v;
    node_from_u<double, D>(u0, c, nd);
    double gb[D][NC];
    visc_flux_transpose<double, D>(nd, c, heat, fb, gb);
#pragma unroll
    for (int j = 0; j < D; ++j)
#pragma unroll
      for (int q = 0; q < NC; ++q) sgb[el][j][q][m] = gb[j][q];
  }
  __syncthreads();
  if (!active) return;
  const double* op = ops + (size_t)e * (2 * D * NP * NP);
  double wb[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) wb[q] = (sl >= 0) ? __ldg(&wbs[((size_t)e * NC + q) * NS + sl]) : 0.0;
#pragma unroll
  for (int j = 0; j < D; ++j)
    for (int n = 0; n < NP; ++n) {
      double dnm = __ldg(&op[((D + j) * NP + m) * NP + n]);  // D_j[n][m]
#pragma unroll
      for (int q = 0; q < NC; ++q) wb[q] += dnm * sgb[el][j][q][n];
    }
#pragma unroll
  for (int q = 0; q < NC; ++q)
#pragma unroll
    for (int cc = 0; cc < NC; ++cc) gr[cc] += wb[q] * ndd.W[q].d[cc];
#pragma unroll
  for (int cc = 0; cc < NC; ++cc) {
    if (sl >= 0) gr[cc] += __ldg(&ubs[((size_t)e * NC + cc) * NS + sl]);
    grad[((size_t)e * NC + cc) * NP + m] += gr[cc];
  }
}

template <int D, int NP>
static int visc_vjp_np(esplit_ctx* c, const double* u, const double* cot, double* grad, cudaStream_t s) {
  const Phys<double> ph = make_phys<double>(c->prm.gam, c->prm.beta, c->prm.R, c->prm.mu, c->prm.Pr);
  const int heat = c->prm.heat_flux;
  constexpr int EB = (128 / NP) > 0 ? (128 / NP) : 1;
  int nb = (c->n_e + EB - 1) / EB;
  double* gs = c->b.fv;       // [n_e][d][n_c][n_p]
  double* fbv = c->b.vfb;     // [n_e][d][n_c][n_p]
  double* abs_ = c->b.va;     // [n_e][d][n_c][n_slot]
  double* fbs = c->b.vfs;     // [n_e][d][n_c][n_slot]
  double* wbs = c->b.vsat;    // [n_e][n_c][n_slot]
  double* ubs = c->b.vus;     // [n_e][n_c][n_slot]
  ProfScope ps(c, PG_VISC, s);
  visc_vjp1_kernel<D, NP, EB><<<nb, EB * NP, 0, s>>>(u, cot, c->b.ops64, c->b.J, c->n_e, gs, fbv, abs_, ph);
  int bs = 64;
  visc_vjp2_kernel<D><<<(c->n_pairs + bs - 1) / bs, bs, 0, s>>>(u, cot, c->b.face_pairs, c->n_pairs, c->b.nu, c->b.J,
                                                                  abs_, fbs, wbs, ubs, ph, heat);
  visc_vjp3_kernel<D, NP, EB><<<nb, EB * NP, 0, s>>>(u, c->b.ops64, c->n_e, gs, fbv, fbs, wbs, ubs, grad, ph, heat);
  c->launches += 3;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_viscous_vjp(esplit_ctx* c, const double* u, const double* cot, double* grad, cudaStream_t s) {
  if (c->dim == 2) {
    switch (c->n_p) {
      case 7: return visc_vjp_np<2, 7>(c, u, cot, grad, s);
      case 12: return visc_vjp_np<2, 12>(c, u, cot, grad, s);
      case 18: return visc_vjp_np<2, 18>(c, u, cot, grad, s);
      case 27: return visc_vjp_np<2, 27>(c, u, cot, grad, s);
    }
  } else if (c->dim == 3) {
    switch (c->n_p) {
      case 12: return visc_vjp_np<3, 12>(c, u, cot, grad, s);
      case 25: return visc_vjp_np<3, 25>(c, u, cot, grad, s);
      case 58: return visc_vjp_np<3, 58>(c, u, cot, grad, s);
      case 78: return visc_vjp_np<3, 78>(c, u, cot, grad, s);
    }
  }
  return -2;
}

}  // namespace esplit
