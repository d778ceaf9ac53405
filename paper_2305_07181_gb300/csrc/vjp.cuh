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
// The pointwise derivatives are exact: the facet terms by a hand-written
// reverse sweep at the values, the volume's pointwise part with closed-form
// products and one dual direction (dual.cuh; see split_vjp_kernel); the
// contractions are transposed applications of the stored per-element
// operators.  Float64 throughout.
// Included by kernels.cu (one device translation unit: the constant-memory
// operator tables are shared).
#pragma once

namespace esplit {

// X^ |Lambda_n| S^ X^T dw of Eq. (69), as diss_apply, one column of X^ at a
// time; n and dw may be plain doubles (no derivative parts).
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

__device__ __forceinline__ double sgn0(double x) { return x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0); }

// reverse of exp_avg (Eq. (47)) at the values: E = (ar - br)/(r (a - b)) or
// ar ia g(eps), eps = (b - a) ia; adds the adjoints of a, b, ar, br, ia for Eb
__device__ __forceinline__ void exp_avg_rev(double a, double b, double ar, double br, double r, double ia,
                                            const double* coef, double Eb, double& ab, double& bb, double& arb,
                                            double& brb, double& iab) {
  const double eps = (b - a) * ia;
  if (fabs(eps) >= ExpAvgCfg<double>::EPS_SWITCH) {
    const double q = 1.0 / (r * (a - b));
    const double E = (ar - br) * q;
    arb += Eb * q;
    brb -= Eb * q;
    ab -= Eb * E / (a - b);
    bb += Eb * E / (a - b);
    return;
  }
  double sv = coef[ExpAvgCfg<double>::NTERMS - 1], dv = 0.0;
#pragma unroll
  for (int k = ExpAvgCfg<double>::NTERMS - 2; k >= 0; --k) {
    dv = dv * eps + sv;
    sv = sv * eps + coef[k];
  }
  // E = ar ia sv(eps)
  arb += Eb * ia * sv;
  const double epsb = Eb * ar * ia * dv;
  iab += Eb * ar * sv + epsb * (b - a);
  bb += epsb * ia;
  ab -= epsb * ia;
}

// Adjoints of the nodal quantities of both sides (ZNode fields) for
//   s = gb . [sum_i nu_i F*_i(k, v) + (|nu|/2) X^|L|S^X^T dw]   (dw held fixed),
// the reverse sweep of pair_avg, sy_flux_dir and the dissipation's hat state
// and columns in plain float64.  With r_k the columns of X^ and l_k =
// |lambda_k| S_k, the dissipation part is (|nu|/2) sum_k l_k (r_k.gb)(r_k.dw):
// column adjoints (|nu|/2) l_k ((r_k.dw) gb + (r_k.gb) dw), weight adjoints
// (|nu|/2) (r_k.gb)(r_k.dw).
template <int D, typename C>
__device__ __forceinline__ void pair_reverse(const ZNode<double, D>& k, const ZNode<double, D>& v, const C& c,
                                             const double* nu, int dissipation, double b, const double* n,
                                             const double* gb, const double* dw, ZNode<double, D>& kb,
                                             ZNode<double, D>& vb) {
  constexpr int NC = D + 2;
  // ---- forward (values)
  PairAvg<double, D> a;
  pair_avg<double, D>(k, v, c, a);
  double A1b = 0.0, E1b = 0.0, A2b = 0.0, E2b = 0.0, z1ab = 0.0, pab = 0.0, keb = 0.0;
  double qVb[D], Vab[D];
#pragma unroll
  for (int i = 0; i < D; ++i) qVb[i] = Vab[i] = 0.0;
  // ---- two-point flux: s_f = mn C + pa (gb_m . nu)
  {
    const double den = a.A1 * a.E1, iden = 1.0 / den;
    double mq = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i) mq += nu[i] * a.qV[i];
    const double mn = mq * iden;
    const double h = c.gam_gm1 * a.A2 * a.E2 + a.ke;
    double Cc = gb[0] + gb[NC - 1] * h, gmn = 0.0;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      Cc += gb[1 + j] * a.Va[j];
      gmn += gb[1 + j] * nu[j];
    }
    const double mnb = Cc, hb = mn * gb[NC - 1];
#pragma unroll
    for (int j = 0; j < D; ++j) Vab[j] += mn * gb[1 + j];
    pab += gmn;
    const double mqb = mnb * iden, idenb = mnb * mq;
#pragma unroll
    for (int i = 0; i < D; ++i) qVb[i] += mqb * nu[i];
    A1b -= idenb * iden * iden * a.E1;
    E1b -= idenb * iden * iden * a.A1;
    A2b += hb * c.gam_gm1 * a.E2;
    E2b += hb * c.gam_gm1 * a.A2;
    keb += hb;
  }
  // ---- dissipation's averages part
  if (dissipation) {
    const double rho_h = a.z1a / (a.A1 * a.E1);
    const double iz = 1.0 / a.z1a;
    double Vh[D], vh2 = 0.0, vn = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      Vh[i] = a.qV[i] * iz;
      vh2 += Vh[i] * Vh[i];
      vn += Vh[i] * n[i];
    }
    const double p_h = a.pa;
    const double theta = rho_h / (p_h * a.A1 * a.E1);
    const double eta = 1.0 / (a.z1a * a.E2 * a.E1);
    const double ah = sqrt(c.gam * p_h / rho_h);
    const double Hh = ah * ah * c.inv_gm1 + 0.5 * vh2;
    double Vhb[D];
#pragma unroll
    for (int i = 0; i < D; ++i) Vhb[i] = 0.0;
    double vnb = 0.0, ahb = 0.0, Hhb = 0.0, vh2b = 0.0, thetab = 0.0, etab = 0.0;
    const double hb2 = 0.5 * b;
#pragma unroll
    for (int kk = 0; kk < NC; ++kk) {
      double col[NC];
      double l;
      const bool ac = (kk == 0 || kk == NC - 1);
      const double sg = (kk == 0) ? -1.0 : 1.0;
      if (ac) {
        col[0] = 1.0;
#pragma unroll
        for (int i = 0; i < D; ++i) col[1 + i] = Vh[i] + sg * ah * n[i];
        col[NC - 1] = Hh + sg * ah * vn;
        l = fabs(vn + sg * ah) * c.s_ac * theta;
      } else if (kk == 1) {
        col[0] = 1.0;
#pragma unroll
        for (int i = 0; i < D; ++i) col[1 + i] = Vh[i];
        col[NC - 1] = 0.5 * vh2;
        l = fabs(vn) * c.s_en * theta;
      } else {
#pragma unroll
        for (int r = 0; r < NC; ++r) col[r] = 0.0;
        if (kk == 2) {
          col[1] = n[1];
          col[2] = -n[0];
          col[NC - 1] = Vh[0] * n[1] - Vh[1] * n[0];
        } else {
          col[1] = -n[D - 1];
          col[3] = n[0];
          col[NC - 1] = Vh[D - 1] * n[0] - Vh[0] * n[D - 1];
        }
        l = fabs(vn) * eta;
      }
      double al = 0.0, be = 0.0;
#pragma unroll
      for (int r = 0; r < NC; ++r) {
        al += col[r] * gb[r];
        be += col[r] * dw[r];
      }
      const double lb = hb2 * al * be;
      double cb[NC];
#pragma unroll
      for (int r = 0; r < NC; ++r) cb[r] = hb2 * l * (be * gb[r] + al * dw[r]);
      if (ac) {
        double cn = 0.0;
#pragma unroll
        for (int i = 0; i < D; ++i) {
          Vhb[i] += cb[1 + i];
          cn += cb[1 + i] * n[i];
        }
        ahb += sg * cn + sg * cb[NC - 1] * vn;
        Hhb += cb[NC - 1];
        vnb += sg * cb[NC - 1] * ah;
        const double t = vn + sg * ah;
        const double w = lb * c.s_ac;
        vnb += w * sgn0(t) * theta;
        ahb += w * sgn0(t) * sg * theta;
        thetab += w * fabs(t);
      } else if (kk == 1) {
#pragma unroll
        for (int i = 0; i < D; ++i) Vhb[i] += cb[1 + i];
        vh2b += 0.5 * cb[NC - 1];
        vnb += lb * sgn0(vn) * c.s_en * theta;
        thetab += lb * fabs(vn) * c.s_en;
      } else {
        if (kk == 2) {
          Vhb[0] += cb[NC - 1] * n[1];
          Vhb[1] -= cb[NC - 1] * n[0];
        } else {
          Vhb[D - 1] += cb[NC - 1] * n[0];
          Vhb[0] -= cb[NC - 1] * n[D - 1];
        }
        vnb += lb * sgn0(vn) * eta;
        etab += lb * fabs(vn);
      }
    }
    // hat state back to the averages
    ahb += Hhb * 2.0 * ah * c.inv_gm1;
    vh2b += 0.5 * Hhb;
#pragma unroll
    for (int i = 0; i < D; ++i) Vhb[i] += 2.0 * vh2b * Vh[i] + vnb * n[i];
    double p_hb = ahb * ah / (2.0 * p_h);
    double rho_hb = -ahb * ah / (2.0 * rho_h);
    z1ab -= etab * eta / a.z1a;
    E2b -= etab * eta / a.E2;
    E1b -= etab * eta / a.E1;
    rho_hb += thetab * theta / rho_h;
    p_hb -= thetab * theta / p_h;
    A1b -= thetab * theta / a.A1;
    E1b -= thetab * theta / a.E1;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      qVb[i] += Vhb[i] * iz;
      z1ab -= Vhb[i] * Vh[i] * iz;
    }
    z1ab += rho_hb * rho_h / a.z1a;
    A1b -= rho_hb * rho_h / a.A1;
    E1b -= rho_hb * rho_h / a.E1;
    pab += p_hb;
  }
  // ---- pair averages back to the nodal quantities
  kb.q = kb.p = kb.P1 = kb.P2 = kb.v2 = kb.iq = kb.ip = 0.0;
  vb.q = vb.p = vb.P1 = vb.P2 = vb.v2 = vb.iq = vb.ip = 0.0;
#pragma unroll
  for (int i = 0; i < D; ++i) kb.V[i] = vb.V[i] = 0.0;
  kb.P1 += 0.5 * A1b;
  vb.P1 += 0.5 * A1b;
  kb.P2 += 0.5 * A2b;
  vb.P2 += 0.5 * A2b;
  kb.q += 0.5 * z1ab;
  vb.q += 0.5 * z1ab;
  kb.p += 0.5 * pab;
  vb.p += 0.5 * pab;
  kb.v2 -= 0.25 * keb;
  vb.v2 -= 0.25 * keb;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const double vab = Vab[i] + 2.0 * keb * a.Va[i];
    kb.V[i] += 0.5 * vab + 0.5 * qVb[i] * k.q;
    vb.V[i] += 0.5 * vab + 0.5 * qVb[i] * v.q;
    kb.q += 0.5 * qVb[i] * k.V[i];
    vb.q += 0.5 * qVb[i] * v.V[i];
  }
  exp_avg_rev(k.p, v.p, k.P2, v.P2, c.r2, k.ip, c.ser2, E1b, kb.p, vb.p, kb.P2, vb.P2, kb.ip);
  exp_avg_rev(k.q, v.q, k.P1, v.P1, c.r1, k.iq, c.ser1, E2b, kb.q, vb.q, kb.P1, vb.P1, kb.iq);
}

// Reverse of the nodal chain u -> (q, V, p, P1, P2, v2, 1/q, 1/p) at the
// values (ZNode adjoints zb -> state adjoint ub):
//   V = m/rho, v2 = |V|^2, p = (gam-1)(e - rho v2/2), q = rho^a_q p^b_q,
//   P1 = q^r1, P2 = p^r2.
template <int D, typename C>
__device__ __forceinline__ void node_chain_rev(const Node<double, D>& n, const ZNode<double, D>& z,
                                               const ZNode<double, D>& zb, const C& c, double* ub) {
  constexpr int NC = D + 2;
  const double iq = 1.0 / n.q, ip = 1.0 / n.p;
  const double qb = zb.q + zb.P1 * c.r1 * z.P1 * iq - zb.iq * iq * iq;
  const double pb = zb.p + zb.P2 * c.r2 * z.P2 * ip - zb.ip * ip * ip + qb * n.q * c.b_q * ip;
  double rhob = qb * n.q * c.a_q * n.ir - 0.5 * c.gm1 * n.v2 * pb;
  const double v2b = zb.v2 - 0.5 * c.gm1 * n.rho * pb;
  ub[NC - 1] = c.gm1 * pb;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const double Vb = zb.V[j] + 2.0 * v2b * n.V[j];
    ub[1 + j] = Vb * n.ir;
    rhob -= Vb * n.V[j] * n.ir;
  }
  ub[0] = rhob;
}

// facet pairs: each thread writes the facet part of grad at its two slots.
// A reverse sweep at the values: the pair computation (averages, two-point
// flux, dissipation; pair_reverse), then each side's nodal chain
// (node_chain_rev); no dual numbers.
template <int D>
__global__ void __launch_bounds__(64) face_vjp_kernel(const double* __restrict__ u, const double* __restrict__ cot,
                                                      const int2* __restrict__ fp, int n_pairs,
                                                      const double* __restrict__ nu, const double* __restrict__ J,
                                                      double* __restrict__ gsat, Phys<double> c, int dissipation) {
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
  ZNode<double, D> zk, zv;
  znode<double, D>(nk, c, zk);
  znode<double, D>(nv, c, zv);
  znode_recips<double, D>(zk);
  double nud[D];
  double b2 = 0.0;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    nud[i] = __ldg(&nu[((size_t)k * NS + s) * D + i]);
    b2 += nud[i] * nud[i];
  }
  const double b = sqrt(b2);
  double nh[D];
#pragma unroll
  for (int i = 0; i < D; ++i) nh[i] = nud[i] / b;
  double ihk = 1.0 / (c_ref.H[m] * __ldg(&J[(size_t)k * NP + m]));
  double ihv = 1.0 / (c_ref.H[n] * __ldg(&J[(size_t)v * NP + n]));
  double gb[NC], dw[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    gb[q] = -__ldg(&cot[((size_t)k * NC + q) * NP + m]) * ihk + __ldg(&cot[((size_t)v * NC + q) * NP + n]) * ihv;
    dw[q] = nk.W[q] - nv.W[q];
  }
  // d[gb . G(u_k, u_v)]: the pair computation reversed at the values, then
  // each side's nodal chain; with dissipation also (M gb) . (dw_k - dw_v),
  // M = X^|L|S^X^T symmetric, through the symmetric dW/du of each side
  ZNode<double, D> kb, vb;
  pair_reverse<D>(zk, zv, c, nud, dissipation, b, nh, gb, dw, kb, vb);
  double gk[NC], gv[NC];
  node_chain_rev<D>(nk, zk, kb, c, gk);
  node_chain_rev<D>(nv, zv, vb, c, gv);
  if (dissipation) {
    PairAvg<double, D> ar;
    pair_avg<double, D>(zk, zv, c, ar);
    double Mgb[NC], wk[NC], wv[NC];
    diss_apply_cols<double, double, double, D>(ar, c, nh, gb, Mgb);
    dW_dU_apply<double, D>(nk, jvp_prep<double, D>(nk, c), c, Mgb, wk);
    dW_dU_apply<double, D>(nv, jvp_prep<double, D>(nv, c), c, Mgb, wv);
#pragma unroll
    for (int cc = 0; cc < NC; ++cc) {
      gk[cc] += 0.5 * b * wk[cc];
      gv[cc] -= 0.5 * b * wv[cc];
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
    // the nodal quantities A~_i depends on, with their tangent along du in
    // closed form (no logarithm or exponential on the duals):
    //   drho = du_0, dV = (du_m - V drho)/rho, dv2 = 2 V.dV, de = du_E,
    //   dp = (gam-1)(de - (drho v2 + rho dv2)/2), dq = q (a_q drho/rho + b_q dp/p)
    Node<T1, D> n1;
    {
      const double drho = du[0];
      double dv2 = 0.0;
      n1.rho = T1(nd.rho);
      n1.rho.d[0] = drho;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const double dVj = (du[1 + j] - nd.V[j] * drho) * nd.ir;
        n1.V[j] = T1(nd.V[j]);
        n1.V[j].d[0] = dVj;
        dv2 += 2.0 * nd.V[j] * dVj;
      }
      const double de = du[NC - 1];
      const double dp = c.gm1 * (de - 0.5 * (drho * nd.v2 + nd.rho * dv2));
      n1.v2 = T1(nd.v2);
      n1.v2.d[0] = dv2;
      n1.e = T1(nd.e);
      n1.e.d[0] = de;
      n1.p = T1(nd.p);
      n1.p.d[0] = dp;
      n1.ir = T1(nd.ir);
      n1.ir.d[0] = -nd.ir * nd.ir * drho;
      n1.q = T1(nd.q);
      n1.q.d[0] = nd.q * (c.a_q * drho * nd.ir + c.b_q * dp * (jp.itheta * nd.ir));
    }
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
      case 12: return vjp_np<3, 12>(c, u, cot, grad, s);
      case 25: return vjp_np<3, 25>(c, u, cot, grad, s);
      case 58: return vjp_np<3, 58>(c, u, cot, grad, s);
      case 78: return vjp_np<3, 78>(c, u, cot, grad, s);
    }
  }
  return -2;
}

}  // namespace esplit
