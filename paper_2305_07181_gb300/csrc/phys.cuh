// Pointwise physics of the entropy-split scheme, device side, templated on the
// arithmetic type T (double for the FP64 path, float for the FP32-bulk path)
// and the dimension D (n_c = D + 2 components).
//
// Paper: Worku & Zingg, entropy-split multidimensional SBP (Secs. 2-4).
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "dual.cuh"
#include "fmath.cuh"

namespace esplit {

// Constants derived from (gam, beta) on the host, Sec. 2.4 / Eq. (16):
// alpha = -gam - beta (gam - 1).
template <typename T>
struct Phys {
  T gam, alpha, beta;
  T gm1, inv_gm1;      // gam - 1, 1/(gam - 1)
  T a_q, b_q;          // q = rho^a_q p^b_q = (rho/p)(p rho^-gam)^(1/(alpha+gam)), Eq. (41)
  T w1c;               // -alpha/(gam-1): W_1 = q (w1c p/rho - |V|^2/2), Eq. (25)
  T inv_w1c;           // -(gam-1)/alpha
  T inv_apb;           // 1/(a_q + b_q) = (alpha+gam)/(1-gam)
  T r1, r2;            // -gam/alpha and (1-gam)/alpha: the powers of z_1 and z_nc
                       // appearing in Eq. (48) (arithmetic and exponential means)
  T inv_bp1;           // 1/(beta+1)
  T gam_gm1;           // gam/(gam-1)
  T gm1_gam;           // (gam-1)/gam
  T s_ac, s_en;        // S^ entries: 1/(2 gam), (gam-1)(gam+alpha)/(gam alpha), Eq. (76)
  T mu, kappa, R;      // viscosity, conductivity mu gam R/((gam-1) Pr), gas constant
  // Taylor coefficients of g(eps) = ((1+eps)^r - 1)/(r eps) for r = r1, r2
  // (c_0 = 1, c_k = c_(k-1) (r - k)/(k + 1)), used by exp_avg
  T ser1[16], ser2[16];
};

template <typename T>
__host__ inline Phys<T> make_phys(double gam, double beta, double R, double mu, double Pr) {
  Phys<T> c;
  double alpha = -gam - beta * (gam - 1.0);
  c.gam = (T)gam;
  c.alpha = (T)alpha;
  c.beta = (T)beta;
  c.gm1 = (T)(gam - 1.0);
  c.inv_gm1 = (T)(1.0 / (gam - 1.0));
  c.a_q = (T)(alpha / (alpha + gam));
  c.b_q = (T)((1.0 - alpha - gam) / (alpha + gam));
  c.w1c = (T)(-alpha / (gam - 1.0));
  c.inv_w1c = (T)(-(gam - 1.0) / alpha);
  c.inv_apb = (T)((alpha + gam) / (1.0 - gam));
  c.r1 = (T)(-gam / alpha);
  c.r2 = (T)((1.0 - gam) / alpha);
  c.inv_bp1 = (T)(1.0 / (beta + 1.0));
  c.gam_gm1 = (T)(gam / (gam - 1.0));
  c.gm1_gam = (T)((gam - 1.0) / gam);
  c.s_ac = (T)(1.0 / (2.0 * gam));
  c.s_en = (T)((gam - 1.0) * (gam + alpha) / (gam * alpha));
  c.mu = (T)mu;
  c.kappa = (T)(mu * gam * R / ((gam - 1.0) * Pr));
  c.R = (T)R;
  double r1 = -gam / alpha, r2 = (1.0 - gam) / alpha;
  double a1 = 1.0, a2 = 1.0;
  for (int k = 0; k < 16; ++k) {
    if (k > 0) {
      a1 *= (r1 - k) / (k + 1);
      a2 *= (r2 - k) / (k + 1);
    }
    c.ser1[k] = (T)a1;
    c.ser2[k] = (T)a2;
  }
  return c;
}

__device__ __forceinline__ double t_log(double x) { return fm::log(x); }
__device__ __forceinline__ float t_log(float x) { return logf(x); }
__device__ __forceinline__ double t_exp(double x) { return fm::exp(x); }
__device__ __forceinline__ float t_exp(float x) { return expf(x); }
__device__ __forceinline__ double t_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float t_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double t_abs(double x) { return fabs(x); }
__device__ __forceinline__ float t_abs(float x) { return fabsf(x); }
__device__ __forceinline__ double t_expm1(double x) { return fm::expm1(x); }
__device__ __forceinline__ float t_expm1(float x) { return expm1f(x); }
__device__ __forceinline__ double t_log1p(double x) { return fm::log1p(x); }
__device__ __forceinline__ float t_log1p(float x) { return log1pf(x); }
__device__ __forceinline__ bool t_isfinite(double x) { return ::isfinite(x); }
__device__ __forceinline__ bool t_isfinite(float x) { return ::isfinite(x); }
// x > 0 (NaN: false) and x finite, from the bit pattern: integer operations
// instead of float64 compares (which take the float64 pipe)
__device__ __forceinline__ bool t_positive(double x) {
  return (unsigned long long)__double_as_longlong(x) - 1ULL < 0x7FF0000000000000ULL;
}
__device__ __forceinline__ bool t_positive(float x) { return (unsigned)__float_as_uint(x) - 1u < 0x7F800000u; }
__device__ __forceinline__ bool t_finite_bits(double x) {
  return ((unsigned long long)__double_as_longlong(x) & 0x7FF0000000000000ULL) != 0x7FF0000000000000ULL;
}
__device__ __forceinline__ bool t_finite_bits(float x) { return (__float_as_uint(x) & 0x7F800000u) != 0x7F800000u; }
template <int N>
__device__ __forceinline__ bool t_positive(const Dual<N>& x) {
  return t_positive(x.v);
}
template <int N>
__device__ __forceinline__ bool t_finite_bits(const Dual<N>& x) {
  return t_finite_bits(x.v);
}

// Nodal state: primitives, q = z_1 of Eq. (45) (= -W_nc), Harten entropy
// variables W of Eq. (25).
template <typename T, int D>
struct Node {
  T rho, V[D], p, e, q, v2;
  T lnq, lnp;  // log q, log p (reused by the parameter-vector powers)
  T ir;        // 1/rho
  T W[D + 2];
};

// Returns false for a non-physical state (rho <= 0, p <= 0 or NaN).
template <typename T, int D, typename C>
__device__ __forceinline__ bool node_from_u(const T* u, const C& c, Node<T, D>& n) {
  n.rho = u[0];
  T ir = T(1) / n.rho;
  n.ir = ir;
  n.v2 = T(0);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    n.V[i] = u[1 + i] * ir;
    n.v2 += n.V[i] * n.V[i];
  }
  n.e = u[D + 1];
  n.p = c.gm1 * (n.e - T(0.5) * n.rho * n.v2);
  bool ok = t_positive(n.rho) && t_positive(n.p) && t_finite_bits(n.e);
  n.lnp = t_log(n.p);
  n.lnq = c.a_q * t_log(n.rho) + c.b_q * n.lnp;
  n.q = t_exp(n.lnq);
  n.W[0] = n.q * (c.w1c * n.p * ir - T(0.5) * n.v2);
#pragma unroll
  for (int i = 0; i < D; ++i) n.W[1 + i] = n.q * n.V[i];
  n.W[D + 1] = -n.q;
  return ok;
}

// Euler flux F^{I(i)} of Eq. (5).
template <typename T, int D>
__device__ __forceinline__ void euler_flux(const Node<T, D>& n, int i, T* F) {
  T m = n.rho * n.V[i];
  F[0] = m;
#pragma unroll
  for (int j = 0; j < D; ++j) F[1 + j] = m * n.V[j] + (j == i ? n.p : T(0));
  F[D + 1] = (n.e + n.p) * n.V[i];
}

// dF^{I(i)} = A~_i v (Eq. (19)): the change of F_i(U(W)) for a change v of
// the entropy variables, by the chain rule through (q, V, theta = p/rho, rho):
//   q = -W_nc, V = W_(1..d)/q, W_1/q = w1c theta - |V|^2/2,
//   q = rho^(a_q + b_q) theta^b_q.
// reciprocals shared by the d directions of dflux_dw
template <typename T>
struct JvpPrep {
  T iq, ir, theta, itheta;
  T w0q, rq, ep;  // w1c theta - |V|^2/2, rho/(a_q + b_q), e + p (shared by the directions)
};

template <typename T, int D, typename C>
__device__ __forceinline__ JvpPrep<T> jvp_prep(const Node<T, D>& n, const C& c) {
  JvpPrep<T> j;
  // one division for 1/q and rho/p: y = 1/(q p), 1/q = p y, 1/p = q y
  const T y = T(1) / (n.q * n.p);
  j.iq = n.p * y;
  j.ir = n.ir;
  j.theta = n.p * j.ir;
  j.itheta = n.rho * (n.q * y);
  j.w0q = c.w1c * j.theta - T(0.5) * n.v2;
  j.rq = n.rho * c.inv_apb;
  j.ep = n.e + n.p;
  return j;
}

template <typename T, int D, typename C>
__device__ __forceinline__ void dflux_dw(const Node<T, D>& n, const JvpPrep<T>& jp, const C& c, int i,
                                         const T* v, T* dF) {
  T iq = jp.iq;
  T dq = -v[D + 1];
  T dV[D];
  T vdv = T(0);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    dV[j] = (v[1 + j] - dq * n.V[j]) * iq;
    vdv += n.V[j] * dV[j];
  }
  T theta = jp.theta;
  T dtheta = c.inv_w1c * ((v[0] - dq * jp.w0q) * iq + vdv);
  T drho = jp.rq * (dq * iq - c.b_q * dtheta * jp.itheta);
  T dp = drho * theta + n.rho * dtheta;
  T dm = drho * n.V[i] + n.rho * dV[i];
  dF[0] = dm;
  T rvi = n.rho * n.V[i];
#pragma unroll
  for (int j = 0; j < D; ++j) dF[1 + j] = dm * n.V[j] + rvi * dV[j] + (j == i ? dp : T(0));
  T de = dp * c.inv_gm1 + T(0.5) * drho * n.v2 + n.rho * vdv;
  dF[D + 1] = (de + dp) * n.V[i] + jp.ep * dV[i];
}

// (dW/dU) z: the change of the entropy variables (Eq. (25)) for a change z of
// the conservative variables, by the chain rule through (rho, V, p, q):
//   dV = (dm - V drho)/rho, dp = (gam-1)(dE - V.dm + |V|^2 drho/2),
//   dq/q = a_q drho/rho + b_q dp/p, d(p/rho) = (dp - (p/rho) drho)/rho,
//   dW = [dq (w1c p/rho - |V|^2/2) + q (w1c d(p/rho) - V.dV), dq V + q dV, -dq].
// dW/dU is the Hessian of the entropy, symmetric.
template <typename T, int D, typename C>
__device__ __forceinline__ void dW_dU_apply(const Node<T, D>& n, const JvpPrep<T>& jp, const C& c, const T* z,
                                            T* out) {
  const T drho = z[0];
  T dV[D], vdm = T(0);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    vdm += n.V[j] * z[1 + j];
    dV[j] = (z[1 + j] - n.V[j] * drho) * jp.ir;
  }
  const T dp = c.gm1 * (z[D + 1] - vdm + T(0.5) * n.v2 * drho);
  const T ip = jp.itheta * jp.ir;  // 1/p
  const T dq = n.q * (c.a_q * drho * jp.ir + c.b_q * dp * ip);
  const T dth = (dp - jp.theta * drho) * jp.ir;
  T vdv = T(0);
#pragma unroll
  for (int j = 0; j < D; ++j) vdv += n.V[j] * dV[j];
  out[0] = dq * jp.w0q + n.q * (c.w1c * dth - vdv);
#pragma unroll
  for (int j = 0; j < D; ++j) out[1 + j] = dq * n.V[j] + n.q * dV[j];
  out[D + 1] = -dq;
}

// (dU/dW) v: the change of the conservative variables for a change v of the
// entropy variables (the inverse map of Eq. (25), the chain rule dflux_dw
// starts with): dq = -v_nc, dV = (v_m - dq V)/q,
// d(p/rho) = ((v_1 - dq W_1/q)/q + V.dV)/w1c, drho from q = rho^(a_q+b_q) (p/rho)^b_q,
// dU = [drho, drho V + rho dV, dp/(gam-1) + drho |V|^2/2 + rho V.dV].
template <typename T, int D, typename C>
__device__ __forceinline__ void dU_dW_apply(const Node<T, D>& n, const JvpPrep<T>& jp, const C& c, const T* v,
                                            T* out) {
  const T dq = -v[D + 1];
  T dV[D], vdv = T(0);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    dV[j] = (v[1 + j] - dq * n.V[j]) * jp.iq;
    vdv += n.V[j] * dV[j];
  }
  const T dth = c.inv_w1c * ((v[0] - dq * jp.w0q) * jp.iq + vdv);
  const T drho = jp.rq * (dq * jp.iq - c.b_q * dth * jp.itheta);
  const T dp = drho * jp.theta + n.rho * dth;
  out[0] = drho;
#pragma unroll
  for (int j = 0; j < D; ++j) out[1 + j] = drho * n.V[j] + n.rho * dV[j];
  out[D + 1] = dp * c.inv_gm1 + T(0.5) * drho * n.v2 + n.rho * vdv;
}

// Powers of the parameter vector used by the two-point flux and the
// dissipation: P1 = z_1^r1 = q^r1, P2 = z_nc^r2 = p^r2.
template <typename T, int D, typename C>
__device__ __forceinline__ void z_powers(const Node<T, D>& n, const C& c, T& P1, T& P2) {
  P1 = t_exp(c.r1 * n.lnq);
  P2 = t_exp(c.r2 * n.lnp);
}

// Exponential average of Eq. (47), {u^(r-1)}_e = (a^r - b^r)/(r (a - b)),
// given ar = a^r and br = b^r.  For |b/a - 1| >= EPS_SWITCH the quotient is
// used directly; below it the equivalent form a^(r-1) g(eps),
// g(eps) = ((1+eps)^r - 1)/(r eps) = sum_k c_k eps^k with c_0 = 1,
// c_k = c_(k-1) (r - k)/(k + 1), summed to NTERMS terms.  For gam > 1 and
// beta > 0 both exponents lie in (0, 1), so |c_k| <= 1 and the terms that
// float64's 13 drop weigh at most 0.05^13/0.95 = 0.12 ulp of g at
// |eps| = 0.05 (0.005 ulp for gam = 1.4, beta = 2.5: r = 7/12 and 1/6).
template <typename T>
struct ExpAvgCfg;
template <>
struct ExpAvgCfg<double> {
  static constexpr double EPS_SWITCH = 0.05;
  static constexpr int NTERMS = 13;
};
template <>
struct ExpAvgCfg<float> {
  static constexpr float EPS_SWITCH = 0.25f;
  static constexpr int NTERMS = 14;
};

template <int N>
struct ExpAvgCfg<Dual<N>> : ExpAvgCfg<double> {};

template <typename T, typename S>
__device__ __forceinline__ T exp_avg(T a, T b, T ar, T br, S r, T ia, const S* coef) {
  T eps = (b - a) * ia;
  if (t_abs(eps) >= ExpAvgCfg<T>::EPS_SWITCH) {
    return (ar - br) / (r * (a - b));
  }
  T sum = coef[ExpAvgCfg<T>::NTERMS - 1];
#pragma unroll
  for (int k = ExpAvgCfg<T>::NTERMS - 2; k >= 0; --k) sum = sum * eps + coef[k];  // Horner
  return ar * ia * sum;
}

// The same average on dual numbers: the series and its derivative by Horner's
// rule on the values, then one chain-rule step (d sum = g'(eps) d eps),
// instead of the series on the duals.
template <int N, typename S>
__device__ __forceinline__ Dual<N> exp_avg(const Dual<N>& a, const Dual<N>& b, const Dual<N>& ar,
                                           const Dual<N>& br, S r, const Dual<N>& ia, const S* coef) {
  const Dual<N> eps = (b - a) * ia;
  if (fabs(eps.v) >= ExpAvgCfg<double>::EPS_SWITCH) return (ar - br) / (r * (a - b));
  double sv = coef[ExpAvgCfg<double>::NTERMS - 1], dv = 0.0;
#pragma unroll
  for (int k = ExpAvgCfg<double>::NTERMS - 2; k >= 0; --k) {
    dv = dv * eps.v + sv;
    sv = sv * eps.v + coef[k];
  }
  Dual<N> sum(sv);
#pragma unroll
  for (int i = 0; i < N; ++i) sum.d[i] = dv * eps.d[i];
  return ar * ia * sum;
}

// Everything the two-point flux needs at one node.
template <typename T, int D>
struct ZNode {
  T q, V[D], p, P1, P2, v2;
  T iq, ip;  // 1/q, 1/p (used by the exponential averages)
};

template <typename T, int D, typename C>
__device__ __forceinline__ void znode(const Node<T, D>& n, const C& c, ZNode<T, D>& z) {
  z.q = n.q;
  z.p = n.p;
  z.v2 = n.v2;
#pragma unroll
  for (int i = 0; i < D; ++i) z.V[i] = n.V[i];
  z_powers<T, D>(n, c, z.P1, z.P2);
  z.iq = T(0);
  z.ip = T(0);
}

// the reciprocals the exponential averages of a pair need (side k only)
template <typename T, int D>
__device__ __forceinline__ void znode_recips(ZNode<T, D>& z) {
  z.iq = T(1) / z.q;
  z.ip = T(1) / z.p;
}

// Pair averages shared by the Sjogreen-Yee flux (Eq. (48)) and the
// intermediate state of the dissipation (Eqs. (73)-(78)).
template <typename T, int D>
struct PairAvg {
  T A1;       // {z_1^(-gam/alpha)}            arithmetic
  T E1;       // {z_nc^((1-gam-alpha)/alpha)}_e exponential
  T A2;       // {z_nc^(-(gam-1)/alpha)}       arithmetic
  T E2;       // {z_1^(-(gam+alpha)/alpha)}_e  exponential
  T z1a;      // {z_1}
  T qV[D];    // {z_1 z_(i+1)}
  T Va[D];    // {V}
  T pa;       // {p}
  T ke;       // sum {V_j}^2 - 1/2 {sum V_j^2}
};

template <typename T, int D, typename C>
__device__ __forceinline__ void pair_avg(const ZNode<T, D>& k, const ZNode<T, D>& v, const C& c,
                                         PairAvg<T, D>& a) {
  a.A1 = T(0.5) * (k.P1 + v.P1);
  a.E1 = exp_avg(k.p, v.p, k.P2, v.P2, c.r2, k.ip, c.ser2);
  a.A2 = T(0.5) * (k.P2 + v.P2);
  a.E2 = exp_avg(k.q, v.q, k.P1, v.P1, c.r1, k.iq, c.ser1);
  a.z1a = T(0.5) * (k.q + v.q);
  a.ke = T(0);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    a.qV[i] = T(0.5) * (k.q * k.V[i] + v.q * v.V[i]);
    a.Va[i] = T(0.5) * (k.V[i] + v.V[i]);
    a.ke += a.Va[i] * a.Va[i];
  }
  a.ke -= T(0.25) * (k.v2 + v.v2);
  a.pa = T(0.5) * (k.p + v.p);
}

// sum_i nu_i F*_i(U_k, U_v) (Eq. (48)) for a direction vector nu.
template <typename T, int D, typename C>
__device__ __forceinline__ void sy_flux_dir(const PairAvg<T, D>& a, const C& c, const T* nu, T* F) {
  T inv_den = T(1) / (a.A1 * a.E1);
  T mn = T(0);
#pragma unroll
  for (int i = 0; i < D; ++i) mn += nu[i] * a.qV[i];
  mn *= inv_den;
  F[0] = mn;
#pragma unroll
  for (int j = 0; j < D; ++j) F[1 + j] = mn * a.Va[j] + nu[j] * a.pa;
  F[D + 1] = mn * (c.gam_gm1 * a.A2 * a.E2 + a.ke);
}

// X^ |Lambda_n| S^ X^T dw of Eq. (69) at the intermediate state (Eqs.
// (73)-(80)); n is a unit normal.  3D eigenvectors as printed, 2D by
// deleting the fourth row and column.
template <typename T, int D, typename C>
__device__ __forceinline__ void diss_apply(const PairAvg<T, D>& a, const C& c, const T* n, const T* dw,
                                           T* out) {
  // the reciprocals of z1a, A1 E1 and p_h, and eta, from one division:
  // D0 = 1/(z1a A1 E1 E2 p_h)
  const T ae = a.A1 * a.E1;
  T p_h = a.pa;
  const T D0 = T(1) / (a.z1a * ae * a.E2 * p_h);
  const T iz = ae * a.E2 * p_h * D0;        // 1/z1a
  const T iae = a.z1a * a.E2 * p_h * D0;    // 1/(A1 E1)
  const T ip_h = a.z1a * ae * a.E2 * D0;    // 1/p_h
  T rho_h = a.z1a * iae;
  T Vh[D];
  T vh2 = T(0), vn = T(0);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    Vh[i] = a.qV[i] * iz;
    vh2 += Vh[i] * Vh[i];
    vn += Vh[i] * n[i];
  }
  T theta = rho_h * iae * ip_h;             // rho_h / (p_h A1 E1)
  T eta = a.A1 * p_h * D0;                  // 1/(z1a E2 E1)
  T ah = t_sqrt(c.gam * p_h * ae * iz);     // sqrt(gam p_h / rho_h)
  T Hh = ah * ah * c.inv_gm1 + T(0.5) * vh2;
  constexpr int NC = D + 2;
  // columns of X^
  T X[NC][NC];  // X[row][col]
  X[0][0] = T(1);
  X[0][1] = T(1);
  X[0][NC - 1] = T(1);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    X[1 + i][0] = Vh[i] - ah * n[i];
    X[1 + i][1] = Vh[i];
    X[1 + i][NC - 1] = Vh[i] + ah * n[i];
  }
  X[NC - 1][0] = Hh - ah * vn;
  X[NC - 1][1] = T(0.5) * vh2;
  X[NC - 1][NC - 1] = Hh + ah * vn;
  if constexpr (D == 1) {
    // no shear modes: the acoustic and entropy columns only
  } else if constexpr (D == 2) {
    X[0][2] = T(0);
    X[1][2] = n[1];
    X[2][2] = -n[0];
    X[3][2] = Vh[0] * n[1] - Vh[1] * n[0];
  } else {
    X[0][2] = T(0);
    X[1][2] = n[1];
    X[2][2] = -n[0];
    X[3][2] = T(0);
    X[4][2] = Vh[0] * n[1] - Vh[1] * n[0];
    X[0][3] = T(0);
    X[1][3] = -n[2];
    X[2][3] = T(0);
    X[3][3] = n[0];
    X[4][3] = Vh[2] * n[0] - Vh[0] * n[2];
  }
  T s_ac = c.s_ac * theta;
  T lam_s[NC];
  lam_s[0] = t_abs(vn - ah) * s_ac;
  lam_s[1] = t_abs(vn) * c.s_en * theta;
#pragma unroll
  for (int k = 2; k < NC - 1; ++k) lam_s[k] = t_abs(vn) * eta;
  lam_s[NC - 1] = t_abs(vn + ah) * s_ac;
  T y[NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    T s = T(0);
#pragma unroll
    for (int r = 0; r < NC; ++r) s += X[r][k] * dw[r];
    y[k] = s * lam_s[k];
  }
#pragma unroll
  for (int r = 0; r < NC; ++r) {
    T s = T(0);
#pragma unroll
    for (int k = 0; k < NC; ++k) s += X[r][k] * y[k];
    out[r] = s;
  }
}

// ---------------------------------------------------------------------------
// Comparator of Sec. 6: the Ismail-Roe entropy-conservative flux (Ismail &
// Roe, J. Comput. Phys. 228, 2009; not printed in the paper), for the
// standard entropy.  With z = sqrt(rho/p) [1, V, p]:
//   rho^ = {z_1} {z_nc}_log,  V^ = {z_1 V}/{z_1},  p1^ = {z_nc}/{z_1},
//   p2^ = (gam+1)/(2 gam) {z_nc}_log/{z_1}_log + (gam-1)/(2 gam) {z_nc}/{z_1},
//   H^ = gam p2^/((gam-1) rho^) + |V^|^2/2,
//   n . F = [m, m V^ + p1^ n, m H^],  m = rho^ V^ . n.
// Logarithmic mean from the nodal logs: (a - b)/(log a - log b), or, for
// u = ((a-b)/(a+b))^2 < 1e-2, (a+b)/2 / (1 + u/3 + u^2/5 + ... + u^8/17)
// (the next term is below 1e-18).
// ---------------------------------------------------------------------------
template <typename T, int D>
struct IRNode {
  T z1, zn, l1, ln;  // sqrt(rho/p), sqrt(rho p) and their logs
  T V[D];
};

template <typename T, int D>
__device__ __forceinline__ void ir_node(const Node<T, D>& n, IRNode<T, D>& z) {
  z.z1 = t_sqrt(n.rho / n.p);
  z.zn = n.p * z.z1;
  T lr = t_log(n.rho);
  z.l1 = T(0.5) * (lr - n.lnp);
  z.ln = T(0.5) * (lr + n.lnp);
#pragma unroll
  for (int i = 0; i < D; ++i) z.V[i] = n.V[i];
}

template <typename T>
__device__ __forceinline__ T log_mean(T a, T b, T la, T lb) {
  T s = a + b;
  T f = (a - b) / s;
  T u = f * f;
  if (u < T(1e-2)) {
    T q = T(1.0 / 17.0);
    q = q * u + T(1.0 / 15.0);
    q = q * u + T(1.0 / 13.0);
    q = q * u + T(1.0 / 11.0);
    q = q * u + T(1.0 / 9.0);
    q = q * u + T(1.0 / 7.0);
    q = q * u + T(1.0 / 5.0);
    q = q * u + T(1.0 / 3.0);
    q = q * u + T(1.0);
    return T(0.5) * s / q;
  }
  return (a - b) / (la - lb);
}

// Pair averages of the Ismail-Roe flux (shared with its dissipation)
template <typename T, int D>
struct IRAvg {
  T rh, p1, p2, vv;  // rho^, p1^, p2^, |V^|^2
  T Vh[D];
};

template <typename T, int D, typename C>
__device__ __forceinline__ void ir_avg(const IRNode<T, D>& k, const IRNode<T, D>& v, const C& c, IRAvg<T, D>& a) {
  T a1 = T(0.5) * (k.z1 + v.z1), an = T(0.5) * (k.zn + v.zn);
  T L1 = log_mean<T>(k.z1, v.z1, k.l1, v.l1), Ln = log_mean<T>(k.zn, v.zn, k.ln, v.ln);
  T ia1 = T(1) / a1;
  a.vv = T(0);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    a.Vh[i] = T(0.5) * (k.z1 * k.V[i] + v.z1 * v.V[i]) * ia1;
    a.vv += a.Vh[i] * a.Vh[i];
  }
  a.rh = a1 * Ln;
  a.p1 = an * ia1;
  a.p2 = (c.gam + T(1)) / (T(2) * c.gam) * (Ln / L1) + (c.gam - T(1)) / (T(2) * c.gam) * a.p1;
}

template <typename T, int D, typename C>
__device__ __forceinline__ void ir_flux_dir(const IRAvg<T, D>& a, const C& c, const T* nu, T* F) {
  T vn = T(0);
#pragma unroll
  for (int i = 0; i < D; ++i) vn += a.Vh[i] * nu[i];
  T Hh = c.gam * c.inv_gm1 * a.p2 / a.rh + T(0.5) * a.vv;
  T m = a.rh * vn;
  F[0] = m;
#pragma unroll
  for (int j = 0; j < D; ++j) F[1 + j] = m * a.Vh[j] + a.p1 * nu[j];
  F[D + 1] = m * Hh;
}

// Standard entropy variables w = [(gam - s)/(gam-1) - rho|V|^2/(2p), rho V/p,
// -rho/p], s = log p - gam log rho, from the nodal state and its IR node.
template <typename T, int D, typename C>
__device__ __forceinline__ void std_entropy_vars(const Node<T, D>& n, const IRNode<T, D>& z, const C& c, T* w) {
  const T b = n.rho / n.p;
  const T lr = z.l1 + z.ln, lp = z.ln - z.l1;  // log rho, log p
  w[0] = (c.gam - (lp - c.gam * lr)) * c.inv_gm1 - T(0.5) * b * n.v2;
#pragma unroll
  for (int i = 0; i < D; ++i) w[1 + i] = b * n.V[i];
  w[D + 1] = -b;
}

// Standard entropy variables of a node (log rho formed here; the comparator's
// viscous terms, whose nodes carry no parameter-vector logs).
template <typename C, int D>
__device__ __forceinline__ void std_entropy_vars_node(const Node<double, D>& n, const C& c, double* w) {
  const double b = n.rho / n.p;
  const double s = n.lnp - c.gam * t_log(n.rho);
  w[0] = (c.gam - s) * c.inv_gm1 - 0.5 * b * n.v2;
#pragma unroll
  for (int i = 0; i < D; ++i) w[1 + i] = b * n.V[i];
  w[D + 1] = -b;
}

// Matrix dissipation of the comparator (not printed in the paper; the form of
// Eq. (69) carried over to the standard entropy), applied to dw = jump of the
// standard entropy variables, n a unit normal:
//   out = sum_k |lambda_k| T_k r_k (r_k . dw) + |V^.n| p^ B^T (I - n n^T) B dw
// at rho^, V^, p^ = p1^; r_k the acoustic and entropy columns of Eq. (80),
// T = rho^/(2 gam), (gam-1) rho^/gam, rho^/(2 gam); B dw = dw_m + V^ dw_E.
template <typename T, int D, typename C>
__device__ __forceinline__ void ir_diss_apply(const IRAvg<T, D>& a, const C& c, const T* n, const T* dw, T* out) {
  constexpr int NC = D + 2;
  T ah = t_sqrt(c.gam * a.p1 / a.rh);
  T Hh = ah * ah * c.inv_gm1 + T(0.5) * a.vv;
  T vn = T(0);
#pragma unroll
  for (int i = 0; i < D; ++i) vn += a.Vh[i] * n[i];
  // r . dw for the three columns
  T vdm = T(0), ndm = T(0);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    vdm += a.Vh[i] * dw[1 + i];
    ndm += n[i] * dw[1 + i];
  }
  const T e = dw[NC - 1];
  const T base = dw[0] + vdm;
  T ym = (base - ah * ndm + (Hh - ah * vn) * e) * (t_abs(vn - ah) * a.rh * c.s_ac);
  T y0 = (base + T(0.5) * a.vv * e) * (t_abs(vn) * a.rh * c.gm1_gam);
  T yp = (base + ah * ndm + (Hh + ah * vn) * e) * (t_abs(vn + ah) * a.rh * c.s_ac);
  out[0] = ym + y0 + yp;
  // shear part
  T y[D], yn = T(0);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    y[i] = dw[1 + i] + a.Vh[i] * e;
    yn += n[i] * y[i];
  }
  const T sh = t_abs(vn) * a.p1;
  T vpy = T(0);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const T py = sh * (y[i] - n[i] * yn);
    out[1 + i] = ym * (a.Vh[i] - ah * n[i]) + y0 * a.Vh[i] + yp * (a.Vh[i] + ah * n[i]) + py;
    vpy += a.Vh[i] * py;
  }
  out[NC - 1] = ym * (Hh - ah * vn) + y0 * (T(0.5) * a.vv) + yp * (Hh + ah * vn) + vpy;
}

}  // namespace esplit
