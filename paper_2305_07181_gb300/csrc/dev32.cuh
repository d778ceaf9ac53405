// Float32 evaluation of the pointwise physics as DEVIATIONS from a reference
// state (precision ESPLIT_FP32).
//
// At the Mach numbers of interest the fluxes and entropy variables vary inside
// an element, and across a facet, by 1e-3 to 1e-1 of their size, and the
// residual is built from such variations (Q_x 1 = 0: a constant flux has no
// divergence; the SAT of Eq. (43) and the dissipation of Eq. (69) vanish for
// equal states).  Evaluated in float32 directly, each flux carries a rounding
// of ~6e-8 of its size, which the differences amplify by the size-to-
// variation ratio (1e3 to 1e5 in the low-Mach workloads).  Here every
// variation is computed from the float64 difference of the conservative
// states, du = u - u_ref, through exact algebraic rearrangements of Eqs. (5),
// (25), (45)-(48) and (73)-(78) in which no two large terms are subtracted:
// each variation then carries a float32 rounding relative to itself.
//
//   rho, V, p:  dV = (dm - V_0 drho) / rho_1,
//               dp = (gam-1) (de - [drho |V_1|^2 + rho_0 (V_1 + V_0).dV] / 2)
//   q = rho^a p^b (Eq. (41)):  dq = q_0 expm1(a log1p(drho/rho_0) + b log1p(dp/p_0))
//   W (Eq. (25)):  W_1 = q th, th = w1c p/rho - |V|^2/2,
//               dth = w1c (dp - (p_0/rho_0) drho)/rho_1 - (V_1 + V_0).dV / 2,
//               dW_1 = dq th_1 + q_0 dth,  dW_m = dq V_1 + q_0 dV,  dW_nc = -dq
//   F_i (Eq. (5)): d(m_i) = dm_i,  d(m_i V_j) = dm_i V_1j + m_0i dV_j,
//               d((e+p) V_i) = (de + dp) V_1i + (e_0 + p_0) dV_i
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "bits32.cuh"
#include "phys.cuh"

namespace esplit {

// float32 reference state (an element's node 0, or side k of a facet pair)
template <int D>
struct Ref32 {
  float rho, ir, V[D], m[D], p, ip, e, ep, q, v2, th;
  float W[D + 2];
};

// from the float32 values uf of the reference's conservative variables (the
// deviations du are taken from the float64 state; the reference's own float32
// rounding changes the variations by ~2^-23 of themselves)
template <int D>
__device__ __forceinline__ void ref32_from_u(const float* uf, const Phys<float>& c, Ref32<D>& r) {
  r.rho = uf[0];
  r.ir = 1.0f / r.rho;
  r.v2 = 0.0f;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    r.m[i] = uf[1 + i];
    r.V[i] = r.m[i] * r.ir;
    r.v2 += r.V[i] * r.V[i];
  }
  r.e = uf[D + 1];
  r.p = c.gm1 * (r.e - 0.5f * r.rho * r.v2);
  r.ip = 1.0f / r.p;
  r.ep = r.e + r.p;
  r.q = expf(c.a_q * logf(r.rho) + c.b_q * logf(r.p));
  r.th = c.w1c * r.p * r.ir - 0.5f * r.v2;
  r.W[0] = r.q * r.th;
#pragma unroll
  for (int i = 0; i < D; ++i) r.W[1 + i] = r.q * r.V[i];
  r.W[D + 1] = -r.q;
}

// variations of the primitives, q and W for du = u_1 - u_ref, and the state u_1
template <int D>
struct Dev32 {
  float dV[D], dp, dq, dW[D + 2], vdv;  // vdv = (V_1 + V_0) . dV
  float rho1, ir1, V1[D], v21, p1, e1, q1;
};

template <int D>
__device__ __forceinline__ void dev32(const Ref32<D>& r, const float* du, const Phys<float>& c, Dev32<D>& d) {
  d.rho1 = r.rho + du[0];
  d.ir1 = 1.0f / d.rho1;
  d.v21 = 0.0f;
  d.vdv = 0.0f;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    d.dV[i] = (du[1 + i] - r.V[i] * du[0]) * d.ir1;
    d.V1[i] = r.V[i] + d.dV[i];
    d.v21 += d.V1[i] * d.V1[i];
    d.vdv += (d.V1[i] + r.V[i]) * d.dV[i];
  }
  d.e1 = r.e + du[D + 1];
  d.dp = c.gm1 * (du[D + 1] - 0.5f * (du[0] * d.v21 + r.rho * d.vdv));
  d.p1 = r.p + d.dp;
  d.dq = r.q * expm1f(c.a_q * log1pf(du[0] * r.ir) + c.b_q * log1pf(d.dp * r.ip));
  d.q1 = r.q + d.dq;
  const float dth = c.w1c * (d.dp - r.p * r.ir * du[0]) * d.ir1 - 0.5f * d.vdv;
  d.dW[0] = d.dq * (r.th + dth) + r.q * dth;
#pragma unroll
  for (int i = 0; i < D; ++i) d.dW[1 + i] = d.dq * d.V1[i] + r.q * d.dV[i];
  d.dW[D + 1] = -d.dq;
}

// F(u_1) - F(u_ref) in the direction nu (sum_i nu_i F_i), Eq. (5)
template <int D>
__device__ __forceinline__ void dflux32_dir(const Ref32<D>& r, const float* du, const Dev32<D>& d, const float* nu,
                                            float* F) {
  float dmn = 0.0f, m0n = 0.0f, v1n = 0.0f, dvn = 0.0f;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    dmn += nu[i] * du[1 + i];
    m0n += nu[i] * r.m[i];
    v1n += nu[i] * d.V1[i];
    dvn += nu[i] * d.dV[i];
  }
  F[0] = dmn;
#pragma unroll
  for (int j = 0; j < D; ++j) F[1 + j] = dmn * d.V1[j] + m0n * d.dV[j] + nu[j] * d.dp;
  F[D + 1] = (du[D + 1] + d.dp) * v1n + r.ep * dvn;
}

// the same for the coordinate direction i
template <int D>
__device__ __forceinline__ void dflux32(const Ref32<D>& r, const float* du, const Dev32<D>& d, int i, float* F) {
  F[0] = du[1 + i];
#pragma unroll
  for (int j = 0; j < D; ++j) F[1 + j] = du[1 + i] * d.V1[j] + r.m[i] * d.dV[j] + (j == i ? d.dp : 0.0f);
  F[D + 1] = (du[D + 1] + d.dp) * d.V1[i] + r.ep * d.dV[i];
}

// the state u_1 as the Node the chain rule of A~_i (dflux_dw) reads
template <int D>
__device__ __forceinline__ void node32(const Ref32<D>& r, const Dev32<D>& d, Node<float, D>& n) {
  n.rho = d.rho1;
  n.ir = d.ir1;
#pragma unroll
  for (int i = 0; i < D; ++i) n.V[i] = d.V1[i];
  n.v2 = d.v21;
  n.p = d.p1;
  n.e = d.e1;
  n.q = d.q1;
  n.lnq = 0.0f;
  n.lnp = 0.0f;
#pragma unroll
  for (int q = 0; q < D + 2; ++q) n.W[q] = r.W[q] + d.dW[q];
}

// g_r(eps) - 1 with g_r(eps) = ((1 + eps)^r - 1)/(r eps), the ratio of the
// exponential average of Eq. (47) to its equal-state value u_k^(r-1); L =
// log1p(eps).  Series c_1 eps + c_2 eps^2 + ... (c_k of Phys::ser*) below
// |eps| = 0.25, the closed form above.
__device__ __forceinline__ float expavg_ratio_m1(float eps, float L, float r, const float* coef) {
  if (fabsf(eps) >= 0.25f) return (expm1f(r * L) - r * eps) / (r * eps);
  float s = coef[13];
#pragma unroll
  for (int k = 12; k >= 1; --k) s = s * eps + coef[k];
  return s * eps;
}

// Sjogreen-Yee flux of Eq. (48) minus the flux of side k, nu . (F*(u_k, u_v)
// - F(u_k)), and the pair averages the dissipation of Eq. (69) reads, from the
// reference k and the deviation d of side v (du = u_v - u_k).  With
// eps_q = dq/q_k, eps_p = dp/p_k and the ratios of the averages to their
// equal-state values,
//   c1 = {q^r1}/q_k^r1 - 1 = expm1(r1 log1p eps_q)/2,   c2 = {p^r2}_e / p_k^(r2-1) - 1,
//   c3 = {p^r2}/p_k^r2 - 1 = expm1(r2 log1p eps_p)/2,   c4 = {q^r1}_e / q_k^(r1-1) - 1,
// and the equal-state identities q^r1 p^(r2-1) = q/rho, p^r2 q^(r1-1) = p/rho,
// p^(r2-1) q^(r1-1) = 1/rho (consistency of Eq. (48)):
//   F*_1 = rho_k (V_k.nu + {d(qV).nu}/(2 q_k)) / (1 + c12),   c12 = c1 + c2 + c1 c2,
//   F*_1 - rho_k V_k.nu = rho_k ({d(qV).nu}/(2 q_k) - V_k.nu c12) / (1 + c12),
//   F*_m - F_m(u_k) = dF1 V_k + F*_1 dV/2 + nu dp/2,
//   F*_E = F*_1 B, B = gam/(gam-1) (p_k/rho_k)(1 + c34) + |V_k|^2/2 + V_k.dV/2,
//   F*_E - F_E(u_k) = dF1 B + rho_k V_k.nu dB,  dB = gam/(gam-1)(p_k/rho_k) c34 + V_k.dV/2.
template <int D>
__device__ __forceinline__ void sy_flux_dev32(const Ref32<D>& r, const Dev32<D>& d, const Phys<float>& c,
                                              const float* nu, float* G, PairAvg<float, D>& a) {
  const float eq = d.dq * (1.0f / r.q), ep = d.dp * r.ip;
  const float Lq = log1pf(eq), Lp = log1pf(ep);
  const float c1 = 0.5f * expm1f(c.r1 * Lq);
  const float c3 = 0.5f * expm1f(c.r2 * Lp);
  const float c2 = expavg_ratio_m1(ep, Lp, c.r2, c.ser2);
  const float c4 = expavg_ratio_m1(eq, Lq, c.r1, c.ser1);
  const float c12 = c1 + c2 + c1 * c2, c34 = c3 + c4 + c3 * c4;
  float vkn = 0.0f, dqvn = 0.0f, vkdv = 0.0f;
  float dqV[D];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    dqV[i] = d.dq * d.V1[i] + r.q * d.dV[i];
    vkn += nu[i] * r.V[i];
    dqvn += nu[i] * dqV[i];
    vkdv += r.V[i] * d.dV[i];
  }
  const float dF1 = r.rho * (0.5f * dqvn / r.q - vkn * c12) / (1.0f + c12);
  const float F1 = r.rho * vkn + dF1;
  G[0] = dF1;
#pragma unroll
  for (int j = 0; j < D; ++j) G[1 + j] = dF1 * r.V[j] + F1 * 0.5f * d.dV[j] + nu[j] * 0.5f * d.dp;
  const float pr = c.gam_gm1 * r.p * r.ir;
  const float dB = pr * c34 + 0.5f * vkdv;
  const float B = pr + 0.5f * r.v2 + dB;
  G[D + 1] = dF1 * B + r.rho * vkn * dB;
  // averages for diss_apply: it reads A1 E1 (= rho^ scale), E2 E1, z1a, qV, pa
  a.A1 = r.q * r.ir * (1.0f + c12);
  a.E1 = 1.0f;
  a.E2 = r.ir * (1.0f + c2) * (1.0f + c4);
  a.z1a = r.q * (1.0f + 0.5f * eq);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    a.qV[i] = r.q * r.V[i] + 0.5f * dqV[i];
    a.Va[i] = r.V[i] + 0.5f * d.dV[i];
  }
  a.pa = r.p + 0.5f * d.dp;
  a.A2 = 0.0f;
  a.ke = 0.0f;
}

}  // namespace esplit
