// Reverse mode (vector-Jacobian product) of the entropy-split residual with
// EC SATs and matrix interface dissipation: grad = (d dudt / d u)^T cot.
//
// The residual of element k at node m is
//   r_m = sum_i (M_i f_i)_m - 1/(beta+1) sum_i A~_i(u_m) (D_i w)_m + sat_m,
// with f_i, w pointwise in u and sat_m = -G(u_km, u_vn)/H_km for the facet
// node pair (k, m) ~ (v, n) (and +G/H_vn on the other side).  Its transpose:
//   gbar_i   = -1/(beta+1) A~_i(u_m) cot_m          (A~_i symmetric, Sec. 2.4)
//   fbar_i   = M_i^T cot,   wbar = sum_i D_i^T gbar_i           (per element)
//   grad_m   = sum_i (df_i/du)^T fbar_i + (dw/du)^T wbar
//              - 1/(beta+1) d/du [cot_m . sum_i A~_i(u) g_i]|_(g_i = (D_i w)_m)
//              + facet part (dG/du)^T (-cot_km/H_km + cot_vn/H_vn).
// The facet Jacobians are exact, from the same physics templates run on
// forward-mode dual numbers (dual.cuh); the volume's pointwise part needs one
// dual direction (see split_vjp_kernel); the contractions are transposed
// applications of the stored per-element operators.  Float64 throughout.
// Included by kernels.cu (one device translation unit: the constant-memory
// operator tables are shared).
#pragma once

namespace esplit {

// facet pairs: each thread writes the facet part of grad at its two slots
// x (derivatives with respect to one side's four state components) placed at
// derivative slots [off, off + N) of an M-direction dual
template <int M, int N>
__device__ __forceinline__ Dual<M> embed(const Dual<N>& x, int off) {
  Dual<M> r(x.v);
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[off + i] = x.d[i];
  return r;
}

template <int D, int N, int M>
__device__ __forceinline__ void embed_znode(const ZNode<Dual<N>, D>& a, int off, ZNode<Dual<M>, D>& b) {
  b.q = embed<M>(a.q, off);
  b.p = embed<M>(a.p, off);
  b.P1 = embed<M>(a.P1, off);
  b.P2 = embed<M>(a.P2, off);
  b.v2 = embed<M>(a.v2, off);
  b.iq = embed<M>(a.iq, off);
  b.ip = embed<M>(a.ip, off);
#pragma unroll
  for (int i = 0; i < D; ++i) b.V[i] = embed<M>(a.V[i], off);
}

// X^ |Lambda_n| S^ X^T dw of Eq. (69), as diss_apply, one column of X^ at a
// time (the eight-direction dual version would otherwise hold all n_c^2
// entries); n and dw may be plain doubles (no derivative parts).
template <typename T, typename TN, typename TW, int D, typename C>
__device__ __forceinline__ void diss_apply_cols(const PairAvg<T, D>& a, const C& c, const TN* n, const TW* dw,
                                                T* out) {
  constexpr int NC = D + 2;
  T rho_h = a.z1a / (a.A1 * a.E1);
  T iz = T(1.0) / a.z1a;
  T Vh[D];
  T vh2 = T(0.0), vn = T(0.0);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    Vh[i] = a.qV[i] * iz;
    vh2 = vh2 + Vh[i] * Vh[i];
    vn = vn + Vh[i] * n[i];
  }
  T p_h = a.pa;
  T theta = rho_h / (p_h * a.A1 * a.E1);
  T eta = T(1.0) / (a.z1a * a.E2 * a.E1);
  T ah = t_sqrt(c.gam * p_h / rho_h);
  T Hh = ah * ah * c.inv_gm1 + 0.5 * vh2;
#pragma unroll
  for (int r = 0; r < NC; ++r) out[r] = T(0.0);
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    T col[NC];
    T ls;
    if (k == 0 || k == NC - 1) {
      const double sg = (k == 0) ? -1.0 : 1.0;
      col[0] = T(1.0);
#pragma unroll
      for (int i = 0; i < D; ++i) col[1 + i] = Vh[i] + sg * (ah * n[i]);
      col[NC - 1] = Hh + sg * (ah * vn);
      ls = t_abs(vn + sg * ah) * (c.s_ac * theta);
    } else if (k == 1) {
      col[0] = T(1.0);
#pragma unroll
      for (int i = 0; i < D; ++i) col[1 + i] = Vh[i];
      col[NC - 1] = 0.5 * vh2;
      ls = t_abs(vn) * (c.s_en * theta);
    } else {
      // tangential columns as printed: (0, n2, -n1, 0, V1 n2 - V2 n1) and
      // (0, -n3, 0, n1, V3 n1 - V1 n3) (2D: the first without its 4th row)
#pragma unroll
      for (int r = 0; r < NC; ++r) col[r] = T(0.0);
      if (k == 2) {
        col[1] = T(n[1]);
        col[2] = T(-n[0]);
        col[NC - 1] = Vh[0] * n[1] - Vh[1] * n[0];
      } else {
        col[1] = T(-n[D - 1]);
        col[3] = T(n[0]);
        col[NC - 1] = Vh[D - 1] * n[0] - Vh[0] * n[D - 1];
      }
      ls = t_abs(vn) * eta;
    }
    T y = col[0] * dw[0];
#pragma unroll
    for (int r = 1; r < NC; ++r) y = y + col[r] * dw[r];
    y = y * ls;
#pragma unroll
    for (int r = 0; r < NC; ++r) out[r] = out[r] + col[r] * y;
  }
}

// Derivative parts (N directions) of s = gb . X^|L|S^X^T dw with gb, dw fixed,
// the hat state on the duals.  With r_k the columns of X^ and l_k = |lambda_k| S_k,
// s = sum_k l_k (r_k . gb)(r_k . dw), so
//   ds = sum_k [(r_k.gb)(r_k.dw) dl_k + l_k ((r_k.dw) gb + (r_k.gb) dw) . dr_k]:
// only the columns and weights are formed on the duals.
template <int N, int D, typename C>
__device__ __forceinline__ void diss_scalar_grad(const PairAvg<Dual<N>, D>& a, const C& c, const double* n,
                                                 const double* gb, const double* dw, double* ds) {
  using T = Dual<N>;
  constexpr int NC = D + 2;
  T rho_h = a.z1a / (a.A1 * a.E1);
  T iz = T(1.0) / a.z1a;
  T Vh[D];
  T vh2 = T(0.0), vn = T(0.0);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    Vh[i] = a.qV[i] * iz;
    vh2 = vh2 + Vh[i] * Vh[i];
    vn = vn + Vh[i] * n[i];
  }
  T p_h = a.pa;
  T theta = rho_h / (p_h * a.A1 * a.E1);
  T eta = T(1.0) / (a.z1a * a.E2 * a.E1);
  T ah = t_sqrt(c.gam * p_h / rho_h);
  T Hh = ah * ah * c.inv_gm1 + 0.5 * vh2;
#pragma unroll
  for (int i = 0; i < N; ++i) ds[i] = 0.0;
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    T col[NC];
    T ls;
    if (k == 0 || k == NC - 1) {
      const double sg = (k == 0) ? -1.0 : 1.0;
      col[0] = T(1.0);
#pragma unroll
      for (int i = 0; i < D; ++i) col[1 + i] = Vh[i] + sg * (ah * n[i]);
      col[NC - 1] = Hh + sg * (ah * vn);
      ls = t_abs(vn + sg * ah) * (c.s_ac * theta);
    } else if (k == 1) {
      col[0] = T(1.0);
#pragma unroll
      for (int i = 0; i < D; ++i) col[1 + i] = Vh[i];
      col[NC - 1] = 0.5 * vh2;
      ls = t_abs(vn) * (c.s_en * theta);
    } else {
#pragma unroll
      for (int r = 0; r < NC; ++r) col[r] = T(0.0);
      if (k == 2) {
        col[1] = T(n[1]);
        col[2] = T(-n[0]);
        col[NC - 1] = Vh[0] * n[1] - Vh[1] * n[0];
      } else {
        col[1] = T(-n[D - 1]);
        col[3] = T(n[0]);
        col[NC - 1] = Vh[D - 1] * n[0] - Vh[0] * n[D - 1];
      }
      ls = t_abs(vn) * eta;
    }
    double al = 0.0, be = 0.0;
#pragma unroll
    for (int r = 0; r < NC; ++r) {
      al += col[r].v * gb[r];
      be += col[r].v * dw[r];
    }
    const double ab = al * be;
#pragma unroll
    for (int i = 0; i < N; ++i) ds[i] += ab * ls.d[i];
#pragma unroll
    for (int r = 0; r < NC; ++r) {
      const double w = ls.v * (be * gb[r] + al * dw[r]);
#pragma unroll
      for (int i = 0; i < N; ++i) ds[i] += w * col[r].d[i];
    }
  }
}

// Derivative parts of s = gb . sum_i nu_i F*_i (Eq. (48), as sy_flux_dir):
// F = [mn, mn {V} + nu {p}, mn h], mn = nu.{z_1 V}/({z_1^a}{z_nc^b}_e),
// h = gam/(gam-1) {.}{.}_e + ke, so s = mn (gb_0 + gb_m.{V} + gb_e h) + {p} gb_m.nu.
template <int N, int D, typename C>
__device__ __forceinline__ void flux_scalar_grad(const PairAvg<Dual<N>, D>& a, const C& c, const double* nu,
                                                 const double* gb, double* ds) {
  using T = Dual<N>;
  constexpr int NC = D + 2;
  T inv_den = T(1.0) / (a.A1 * a.E1);
  T mq = T(0.0);
#pragma unroll
  for (int i = 0; i < D; ++i) mq = mq + nu[i] * a.qV[i];
  T mn = mq * inv_den;
  T h = c.gam_gm1 * (a.A2 * a.E2) + a.ke;
  double gmv = gb[0] + gb[NC - 1] * h.v, gmn = 0.0;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    gmv += gb[1 + j] * a.Va[j].v;
    gmn += gb[1 + j] * nu[j];
  }
  // ds = gmv dmn + mn (gb_m . d{V} + gb_e dh) + gmn d{p}
#pragma unroll
  for (int i = 0; i < N; ++i) {
    double t = gb[NC - 1] * h.d[i];
#pragma unroll
    for (int j = 0; j < D; ++j) t += gb[1 + j] * a.Va[j].d[i];
    ds[i] = gmv * mn.d[i] + mn.v * t + gmn * a.pa.d[i];
  }
}

template <int D, int N>
__device__ __forceinline__ PairAvg<double, D> strip_avg(const PairAvg<Dual<N>, D>& a) {
  PairAvg<double, D> b;
  b.A1 = a.A1.v;
  b.E1 = a.E1.v;
  b.A2 = a.A2.v;
  b.E2 = a.E2.v;
  b.z1a = a.z1a.v;
  b.pa = a.pa.v;
  b.ke = a.ke.v;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    b.qV[i] = a.qV[i].v;
    b.Va[i] = a.Va[i].v;
  }
  return b;
}

// facet pairs: each thread writes the facet part of grad at its two slots.
// Each side's nodal chain (logarithms, exponentials, divisions) depends on its
// own four state components only: it runs on four-direction duals, and the
// results enter the eight-direction pair computation (averages, two-point
// flux, dissipation) at that side's slots.
template <int D>
__global__ void __launch_bounds__(64) face_vjp_kernel(const double* __restrict__ u, const double* __restrict__ cot,
                                                      const int2* __restrict__ fp, int n_pairs,
                                                      const double* __restrict__ nu, const double* __restrict__ J,
                                                      double* __restrict__ gsat, Phys<double> c, int dissipation) {
  constexpr int NC = D + 2;
  constexpr int N2 = 2 * NC;
  using T = Dual<N2>;
  using TS = Dual<NC>;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_pairs) return;
  const int NP = c_ref.n_p, NS = c_ref.n_slot;
  int2 pr = __ldg(&fp[t]);
  int k = pr.x / NS, s = pr.x - k * NS;
  int v = pr.y / NS, s2 = pr.y - v * NS;
  int m = c_ref.slot_node[s], n = c_ref.slot_node[s2];
  ZNode<T, D> zk, zv;
  TS Wk[NC], Wv[NC];  // each side's entropy variables with their own Jacobian
  {
    TS uk[NC], uv[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      uk[q] = TS(__ldg(&u[((size_t)k * NC + q) * NP + m]));
      uv[q] = TS(__ldg(&u[((size_t)v * NC + q) * NP + n]));
      uk[q].d[q] = 1.0;
      uv[q].d[q] = 1.0;
    }
    Node<TS, D> nk, nv;
    node_from_u<TS, D>(uk, c, nk);
    node_from_u<TS, D>(uv, c, nv);
    ZNode<TS, D> sk, sv;
    znode<TS, D>(nk, c, sk);
    znode<TS, D>(nv, c, sv);
    znode_recips<TS, D>(sk);
    embed_znode<D>(sk, 0, zk);
    embed_znode<D>(sv, NC, zv);
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      Wk[q] = nk.W[q];
      Wv[q] = nv.W[q];
    }
  }
  PairAvg<T, D> a;
  pair_avg<T, D>(zk, zv, c, a);
  double nud[D];
  double b2 = 0.0;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    nud[i] = __ldg(&nu[((size_t)k * NS + s) * D + i]);
    b2 += nud[i] * nud[i];
  }
  double ihk = 1.0 / (c_ref.H[m] * __ldg(&J[(size_t)k * NP + m]));
  double ihv = 1.0 / (c_ref.H[n] * __ldg(&J[(size_t)v * NP + n]));
  double gb[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q)
    gb[q] = -__ldg(&cot[((size_t)k * NC + q) * NP + m]) * ihk + __ldg(&cot[((size_t)v * NC + q) * NP + n]) * ihv;
  // gb . G(u_k, u_v): the two-point flux, and with dissipation
  //   d[gb . M(a) (w_k - w_v)] = gb . (dM) dw + (M gb) . (dw_k - dw_v)   (M symmetric)
  double ds[N2];
  flux_scalar_grad<N2, D>(a, c, nud, gb, ds);
  double gk[NC], gv[NC];
#pragma unroll
  for (int cc = 0; cc < NC; ++cc) {
    gk[cc] = ds[cc];
    gv[cc] = ds[NC + cc];
  }
  if (dissipation) {
    const double b = sqrt(b2);
    double nh[D];
#pragma unroll
    for (int i = 0; i < D; ++i) nh[i] = nud[i] / b;
    double dw[NC], Mgb[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) dw[q] = Wk[q].v - Wv[q].v;
    diss_scalar_grad<N2, D>(a, c, nh, gb, dw, ds);
    const PairAvg<double, D> ar = strip_avg<D>(a);
    diss_apply_cols<double, double, double, D>(ar, c, nh, gb, Mgb);
#pragma unroll
    for (int cc = 0; cc < NC; ++cc) {
      gk[cc] += 0.5 * b * ds[cc];
      gv[cc] += 0.5 * b * ds[NC + cc];
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        gk[cc] += 0.5 * b * Mgb[q] * Wk[q].d[cc];
        gv[cc] -= 0.5 * b * Mgb[q] * Wv[q].d[cc];
      }
    }
  }
#pragma unroll
  for (int cc = 0; cc < NC; ++cc) {
    gsat[((size_t)k * NC + cc) * NS + s] = gk[cc];
    gsat[((size_t)v * NC + cc) * NS + s2] = gv[cc];
  }
}

template <int D, int NP, int EB>
__global__ void __launch_bounds__(EB * NP) split_vjp_kernel(const double* __restrict__ u,
                                                            const double* __restrict__ cot,
                                                            const double* __restrict__ ops,
                                                            const double* __restrict__ gsat, int n_e,
                                                            double* __restrict__ grad, Phys<double> c) {
  constexpr int NC = D + 2;
  __shared__ double sw[EB][NC][NP];
  __shared__ double sv[EB][NC][NP];
  __shared__ double sgb[EB][D][NC][NP];
  const int NS = c_ref.n_slot;
  int el = threadIdx.x / NP;
  int m = threadIdx.x - el * NP;
  int e = blockIdx.x * EB + el;
  bool active = e < n_e;
  Node<double, D> nd;
  double uu[NC], vv[NC];
  if (active) {
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      uu[q] = __ldg(&u[((size_t)e * NC + q) * NP + m]);
      vv[q] = __ldg(&cot[((size_t)e * NC + q) * NP + m]);
      sv[el][q][m] = vv[q];
    }
    node_from_u<double, D>(uu, c, nd);
#pragma unroll
    for (int q = 0; q < NC; ++q) sw[el][q][m] = nd.W[q];
  }
  __syncthreads();
  const double* op = ops + (size_t)(active ? e : 0) * (2 * D * NP * NP);
  double g[D][NC];
  if (active) {
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int q = 0; q < NC; ++q) g[i][q] = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i)
      for (int n = 0; n < NP; ++n) {
        double dt = __ldg(&op[((D + i) * NP + n) * NP + m]);  // D_i[m][n]
#pragma unroll
        for (int q = 0; q < NC; ++q) g[i][q] += dt * sw[el][q][n];
      }
    const JvpPrep<double> jp = jvp_prep<double, D>(nd, c);
#pragma unroll
    for (int i = 0; i < D; ++i) {
      double a[NC];
      dflux_dw<double, D>(nd, jp, c, i, vv, a);
#pragma unroll
      for (int q = 0; q < NC; ++q) sgb[el][i][q][m] = -c.inv_bp1 * a[q];
    }
  }
  __syncthreads();
  if (!active) return;
  double fb[D][NC], wb[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) wb[q] = 0.0;
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int q = 0; q < NC; ++q) fb[i][q] = 0.0;
#pragma unroll
  for (int i = 0; i < D; ++i)
    for (int n = 0; n < NP; ++n) {
      double mt = __ldg(&op[(i * NP + m) * NP + n]);        // M_i[n][m]
      double dt = __ldg(&op[((D + i) * NP + m) * NP + n]);  // D_i[n][m]
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        fb[i][q] += mt * sv[el][q][n];
        wb[q] += dt * sgb[el][i][q][n];
      }
    }
  // pointwise part.  With A~_i = dF_i/dW symmetric and dW/du the symmetric
  // Hessian of the entropy,
  //   (dF_i/du)^T fb_i = (dW/du) A~_i fb_i,   (dw/du)^T wb = (dW/du) wb,
  // and, F_i being the W-gradient of its flux potential (Sec. 2.4), the
  // derivative of A~_i(W) g along W is symmetric in its three arguments, so the
  // u-gradient of cot_m . A~_i(u) g_i is (dW/du) applied to the derivative of
  // A~_i g_i along W in the single direction cot_m (a one-direction dual
  // number, the state moved by (dU/dW) cot_m):
  //   grad_m = (dW/du) [sum_i A~_i fb_i + wb - 1/(beta+1) sum_i d_cot(A~_i g_i)].
  const JvpPrep<double> jp = jvp_prep<double, D>(nd, c);
  double z[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) z[q] = wb[q];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double a[NC];
    dflux_dw<double, D>(nd, jp, c, i, fb[i], a);
#pragma unroll
    for (int q = 0; q < NC; ++q) z[q] += a[q];
  }
  {
    using T1 = Dual<1>;
    double du[NC];
    dU_dW_apply<double, D>(nd, jp, c, vv, du);
    T1 ud[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      ud[q] = T1(uu[q]);
      ud[q].d[0] = du[q];
    }
    Node<T1, D> n1;
    node_from_u<T1, D>(ud, c, n1);
    const JvpPrep<T1> j1 = jvp_prep<T1, D>(n1, c);
#pragma unroll
    for (int i = 0; i < D; ++i) {
      T1 gi[NC], dF[NC];
#pragma unroll
      for (int q = 0; q < NC; ++q) gi[q] = T1(g[i][q]);
      dflux_dw<T1, D>(n1, j1, c, i, gi, dF);
#pragma unroll
      for (int q = 0; q < NC; ++q) z[q] -= c.inv_bp1 * dF[q].d[0];
    }
  }
  double gr[NC];
  dW_dU_apply<double, D>(nd, jp, c, z, gr);
  int sl = c_ref.node_slot[m];
#pragma unroll
  for (int cc = 0; cc < NC; ++cc) {
    if (sl >= 0) gr[cc] += __ldg(&gsat[((size_t)e * NC + cc) * NS + sl]);
    grad[((size_t)e * NC + cc) * NP + m] = gr[cc];
  }
}

template <int D, int NP>
static int vjp_np(esplit_ctx* c, const double* u, const double* cot, double* grad, cudaStream_t s) {
  const Phys<double> ph = make_phys<double>(c->prm.gam, c->prm.beta, c->prm.R, c->prm.mu, c->prm.Pr);
  {
    int bs = 64;
    int nb = (c->n_pairs + bs - 1) / bs;
    ProfScope ps(c, PG_FACE, s);
    face_vjp_kernel<D><<<nb, bs, 0, s>>>(u, cot, c->b.face_pairs, c->n_pairs, c->b.nu, c->b.J, c->b.sat, ph,
                                         c->prm.dissipation);
    c->launches++;
  }
  {
    constexpr int EB = (128 / NP) > 0 ? (128 / NP) : 1;
    int nb = (c->n_e + EB - 1) / EB;
    ProfScope ps(c, PG_SPLIT, s);
    split_vjp_kernel<D, NP, EB><<<nb, EB * NP, 0, s>>>(u, cot, c->b.ops64, c->b.sat, c->n_e, grad, ph);
    c->launches++;
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_residual_vjp(esplit_ctx* c, const double* u, const double* cot, double* grad, cudaStream_t s) {
  if (c->dim == 2) {
    switch (c->n_p) {
      case 7: return vjp_np<2, 7>(c, u, cot, grad, s);
      case 12: return vjp_np<2, 12>(c, u, cot, grad, s);
      case 18: return vjp_np<2, 18>(c, u, cot, grad, s);
      case 27: return vjp_np<2, 27>(c, u, cot, grad, s);
    }
  } else if (c->dim == 3) {
    switch (c->n_p) {
      case 25: return vjp_np<3, 25>(c, u, cot, grad, s);
    }
  }
  return -2;
}

}  // namespace esplit
