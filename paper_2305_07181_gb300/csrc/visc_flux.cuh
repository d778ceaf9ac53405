// Viscous flux of the compressible Navier-Stokes equations written with the
// entropy-variable gradients (Sec. 3 and Sec. 5: F^V_i = sum_j K~_ij dW/dx_j),
// and its transpose in the gradients.  Shared by the facet, volume and
// reverse-mode kernels.  ENT selects the entropy variables the gradients are
// of: 0 Harten's W (Eq. (25), the entropy-split scheme), 1 the standard
// entropy variables v = [(gam - s)/(gam-1) - rho|V|^2/(2p), rho V/p, -rho/p]
// (the Ismail-Roe comparator).  In both sets V = -w_m / w_nc, so the velocity
// gradients have one form; T = -1/(R v_nc) in the standard set, whose dT/dv
// has the last entry 1/(R v_nc^2) only.
#pragma once

#include <type_traits>

namespace esplit {

// constants in the arithmetic of T: float for the float32 path, double for
// double and the dual numbers of the reverse mode
template <typename T>
using vscal_t = typename std::conditional<std::is_same<T, float>::value, float, double>::type;

// dT/dW of Eq. (39) (the exact derivative; the printed Eq. (40) has a sign
// typo in the momentum entries and drops alpha in the last entry).  T is
// double or a dual number (the reverse mode differentiates these in u).
template <typename T, int D, int ENT = 0, typename C = Phys<double>>
__device__ __forceinline__ void dT_dW(const Node<T, D>& n, const C& c, T* TW) {
  constexpr int NC = D + 2;
  using S = vscal_t<T>;
  if constexpr (ENT == 1) {
    const T pr = n.p * n.ir;  // p / rho = -1 / v_nc
#pragma unroll
    for (int q = 0; q < NC - 1; ++q) TW[q] = T(0.0);
    TW[NC - 1] = pr * pr / c.R;
    return;
  }
  T Wn = -n.q;
  T k = c.gm1 / (c.alpha * c.R * Wn);
  T T_ = n.p * n.ir / c.R;
  TW[0] = k;
#pragma unroll
  for (int l = 0; l < D; ++l) TW[1 + l] = k * n.V[l];
  TW[NC - 1] = -T_ / Wn + S(0.5) * k * n.v2;
}

// F^V_i (i < D) from the entropy-variable gradients g[j] = dW/dx_j:
//   dV_l/dx_j = -(g_j[1+l] + V_l g_j[nc]) / W_nc,  dT/dx_j = dT/dW . g_j,
//   tau_ik = mu (dV_i/dx_k + dV_k/dx_i - 2/3 delta_ik div V),
//   F_i = [0, tau_i., V . tau_i. + kappa dT/dx_i]
template <typename T, int D, typename G, int ENT = 0, typename C = Phys<double>>
__device__ __forceinline__ void visc_flux(const Node<T, D>& n, const C& c, int heat, const G (&g)[D][D + 2],
                                          T (&F)[D][D + 2]) {
  constexpr int NC = D + 2;
  using S = vscal_t<T>;
  T iWn;  // 1 / w_nc
  if constexpr (ENT == 1)
    iWn = -(n.p * n.ir);
  else
    iWn = S(-1.0) / n.q;
  T Lg[D][D];  // Lg[j][l] = dV_l/dx_j
  T div = T(0.0);
#pragma unroll
  for (int j = 0; j < D; ++j)
#pragma unroll
    for (int l = 0; l < D; ++l) Lg[j][l] = -(g[j][1 + l] + n.V[l] * g[j][NC - 1]) * iWn;
#pragma unroll
  for (int l = 0; l < D; ++l) div = div + Lg[l][l];
  T TW[NC];
  dT_dW<T, D, ENT>(n, c, TW);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    T e = T(0.0);
    F[i][0] = T(0.0);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      T tau = c.mu * (Lg[k][i] + Lg[i][k] - (k == i ? S(2.0 / 3.0) * div : T(0.0)));
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
template <typename T, int D, typename B, int ENT = 0, typename C = Phys<double>>
__device__ __forceinline__ void visc_flux_transpose(const Node<T, D>& n, const C& c, int heat,
                                                    const B (&b)[D][D + 2], T (&a)[D][D + 2]) {
  constexpr int NC = D + 2;
  using S = vscal_t<T>;
  T iWn;  // 1 / w_nc
  if constexpr (ENT == 1)
    iWn = -(n.p * n.ir);
  else
    iWn = S(-1.0) / n.q;
  T cc[D][D];
  T trc = T(0.0);
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int k = 0; k < D; ++k) cc[i][k] = b[i][1 + k] + b[i][NC - 1] * n.V[k];
#pragma unroll
  for (int i = 0; i < D; ++i) trc = trc + cc[i][i];
  T TW[NC];
  dT_dW<T, D, ENT>(n, c, TW);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    T hj = heat ? c.kappa * b[j][NC - 1] : T(0.0);
    T sv = T(0.0);
    a[j][0] = hj * TW[0];
#pragma unroll
    for (int l = 0; l < D; ++l) {
      T G = c.mu * (cc[j][l] + cc[l][j] - (j == l ? S(2.0 / 3.0) * trc : T(0.0)));
      a[j][1 + l] = -G * iWn + hj * TW[1 + l];
      sv = sv + G * n.V[l];
    }
    a[j][NC - 1] = -sv * iWn + hj * TW[NC - 1];
  }
}

}  // namespace esplit
