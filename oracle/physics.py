"""Pointwise physics of the oracle (plain PyTorch, float64).

State arrays carry the component index LAST: U (..., n_c) with
n_c = d + 2, U = [rho, rho V_1..V_d, e] (Sec. 2.2, Eq. (5)).

Pins (tests/test_oracle_physics.py):
  * W = dS_H/dU by autograd vs the closed form of Eq. (25),
  * A~_i symmetric (Sec. 2.4) and A~_i W = beta F_i (Eq. (26)),
  * beta/(beta+1) W^T F_i = V_i S (Eq. (30)), S = beta phi (Eq. (33)),
  * Sjogreen-Yee flux: consistency, symmetry, Tadmor's condition Eq. (49) on
    random state pairs (this fixes the reading of the printed Eq. (48)),
  * exponential average vs brute force in extended precision,
  * dissipation: X^ S^ X^T = dU/dW at equal states (2D) and A_n X^ = X^ Lambda,
  * T(W) (Eq. (39)) and W_nc (Eq. (41)) vs the primitive definitions; dT/dW
    vs the exact derivative of Eq. (39) (the printed Eq. (40) has a sign typo
    in the momentum entries and a missing alpha in the last entry),
  * heat-flux-free K~ positive semidefinite (Sec. 5, LDL^T statement).
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

DT = torch.float64


@dataclass(frozen=True)
class Params:
    """Physical and scheme parameters.

    gam   ratio of specific heats (7/5, Sec. 2.2)
    beta  split parameter; Harten's alpha = -gam - beta (gam - 1) follows from
          beta = -(gam + alpha)/(gam - 1) (Eq. (16)); beta = 2.5 (Sec. 6.4)
    R     gas constant (1, Secs. 7.4-7.5); mu dynamic viscosity; Pr Prandtl
    heat_flux  include the heat flux in the viscous flux
    """

    gam: float = 1.4
    beta: float = 2.5
    R: float = 1.0
    mu: float = 0.0
    Pr: float = 0.71
    heat_flux: bool = True

    @property
    def alpha(self) -> float:
        return -self.gam - self.beta * (self.gam - 1.0)

    @property
    def kappa(self) -> float:
        # heat conductivity mu c_p / Pr with c_p = gam R / (gam - 1)
        return self.mu * self.gam * self.R / ((self.gam - 1.0) * self.Pr)


def primitives(U, prm: Params):
    """rho, V (..., d), p from conservative variables (closure of Sec. 2.2)."""
    rho = U[..., 0]
    V = U[..., 1:-1] / rho[..., None]
    p = (prm.gam - 1.0) * (U[..., -1] - 0.5 * rho * (V * V).sum(-1))
    return rho, V, p


def conservative(rho, V, p, prm: Params):
    e = p / (prm.gam - 1.0) + 0.5 * rho * (V * V).sum(-1)
    return torch.cat([rho[..., None], rho[..., None] * V, e[..., None]], dim=-1)


def harten_entropy(U, prm: Params):
    """S_H = beta rho (p rho^-gam)^(1/(alpha+gam)), Eq. (16)."""
    rho, V, p = primitives(U, prm)
    return prm.beta * rho * (p * rho ** (-prm.gam)) ** (1.0 / (prm.alpha + prm.gam))


def harten_entropy_change(U, dU, prm: Params):
    """s(U + dU) - s(U) for Harten's entropy, Eq. (16), evaluated without
    cancellation (both states positive).

    With s = beta rho^A p^B, A = alpha/(alpha+gam), B = 1/(alpha+gam):
        s(U + dU) - s(U) = s(U) expm1(A log1p(drho/rho) + B log1p(dp/p)),
    where the pressure change follows exactly from the closure of Sec. 2.2:
        dp = (gam-1) (de - [(2 m.dm + |dm|^2) rho - |m|^2 drho] / (2 rho (rho + drho))),
    m = rho V.  Every quantity is a small difference computed directly, so the
    result carries relative (not absolute) round-off.  Used for the relaxation
    function of Eq. (97), whose root is defined by such differences."""
    g, a = prm.gam, prm.alpha
    A = a / (a + g)
    B = 1.0 / (a + g)
    rho, m, E = U[..., 0], U[..., 1:-1], U[..., -1]
    drho, dm, dE = dU[..., 0], dU[..., 1:-1], dU[..., -1]
    p = (g - 1.0) * (E - 0.5 * (m * m).sum(-1) / rho)
    dke = ((2.0 * (m * dm).sum(-1) + (dm * dm).sum(-1)) * rho - (m * m).sum(-1) * drho) / (2.0 * rho * (rho + drho))
    dp = (g - 1.0) * (dE - dke)
    s = prm.beta * rho ** A * p ** B
    return s * torch.expm1(A * torch.log1p(drho / rho) + B * torch.log1p(dp / p))


def entropy_variables(U, prm: Params):
    """Harten entropy variables, Eq. (25):
    W = (rho/p)(p rho^-gam)^(1/(alpha+gam)) [-alpha/(gam-1) p/rho - |V|^2/2, V, -1]."""
    rho, V, p = primitives(U, prm)
    q = (rho / p) * (p * rho ** (-prm.gam)) ** (1.0 / (prm.alpha + prm.gam))
    first = -prm.alpha / (prm.gam - 1.0) * p / rho - 0.5 * (V * V).sum(-1)
    return q[..., None] * torch.cat([first[..., None], V, -torch.ones_like(first)[..., None]], dim=-1)


def euler_flux(U, prm: Params):
    """Inviscid fluxes F^{I(i)} of Eq. (5) for all directions: (..., d, n_c)."""
    rho, V, p = primitives(U, prm)
    d = V.shape[-1]
    e = U[..., -1]
    out = []
    for i in range(d):
        mom = rho[..., None] * V[..., i:i + 1] * V
        mom = mom + p[..., None] * torch.nn.functional.one_hot(torch.tensor(i), d).to(U)
        out.append(torch.cat([(rho * V[..., i])[..., None], mom, ((e + p) * V[..., i])[..., None]], -1))
    return torch.stack(out, dim=-2)


def param_vector(U, prm: Params):
    """Parameter vector z = [(rho/p)(p rho^-gam)^(1/(alpha+gam)), V, p], Eq. (45)."""
    rho, V, p = primitives(U, prm)
    z1 = (rho / p) * (p * rho ** (-prm.gam)) ** (1.0 / (prm.alpha + prm.gam))
    return torch.cat([z1[..., None], V, p[..., None]], dim=-1)


def arith_avg(a, b):
    """{u} = (u_k + u_v)/2, Eq. (46)."""
    return 0.5 * (a + b)


def exp_avg(a, b, r):
    """Exponential average {u^(r-1)}_e = (u_k^r - u_v^r) / (r (u_k - u_v)), Eq. (47).

    Evaluated as u_k^(r-1) g(eps), eps = u_v/u_k - 1,
    g(eps) = ((1+eps)^r - 1)/(r eps) = expm1(r log1p(eps)) / (r eps), which is
    the same quotient without cancellation; g(0) = 1 (limit u_v -> u_k).  The
    eps == 0 branch keeps the first Taylor term so that autograd returns the
    correct derivative g'(0) = (r-1)/2 at coincident states."""
    eps = b / a - 1.0
    zero = eps == 0
    safe = torch.where(zero, torch.ones_like(eps), eps)
    g = torch.expm1(r * torch.log1p(safe)) / (r * safe)
    g = torch.where(zero, 1.0 + 0.5 * (r - 1.0) * eps, g)
    return a ** (r - 1.0) * g


def sy_flux(Uk, Uv, prm: Params):
    """Sjogreen-Yee two-point flux F*_i(U_k, U_v), Eq. (48), all directions:
    returns (..., d, n_c).

    Reading of the printed formula (the one that satisfies Tadmor's condition,
    Eq. (49), to round-off): {z_1 z_(i+1)} is the arithmetic mean of the
    product; the averages {z_1^(-gam/alpha)} and {z_nc^(-(gam-1)/alpha)} that
    carry no subscript e are arithmetic means of the powers; {.}_e terms are
    the exponential averages of Eq. (47) with r - 1 equal to the printed
    exponent."""
    g, a = prm.gam, prm.alpha
    zk, zv = param_vector(Uk, prm), param_vector(Uv, prm)
    d = Uk.shape[-1] - 2
    z1k, z1v, znk, znv = zk[..., 0], zv[..., 0], zk[..., -1], zv[..., -1]
    Vk, Vv = zk[..., 1:-1], zv[..., 1:-1]
    den = arith_avg(z1k ** (-g / a), z1v ** (-g / a)) * exp_avg(znk, znv, (1.0 - g - a) / a + 1.0)
    Vavg = arith_avg(Vk, Vv)
    ke = (Vavg * Vavg).sum(-1) - 0.5 * arith_avg((Vk * Vk).sum(-1), (Vv * Vv).sum(-1))
    enth = (g / (g - 1.0)) * arith_avg(znk ** (-(g - 1.0) / a), znv ** (-(g - 1.0) / a)) \
        * exp_avg(z1k, z1v, -(g + a) / a + 1.0)
    pavg = arith_avg(znk, znv)
    out = []
    for i in range(d):
        F1 = arith_avg(z1k * Vk[..., i], z1v * Vv[..., i]) / den
        mom = F1[..., None] * Vavg
        mom = mom + pavg[..., None] * torch.nn.functional.one_hot(torch.tensor(i), d).to(Uk)
        Fe = F1 * (enth + ke)
        out.append(torch.cat([F1[..., None], mom, Fe[..., None]], -1))
    return torch.stack(out, dim=-2)


def _jacobian(fn, U):
    """Pointwise Jacobian d fn(U) / dU for a batch of states (..., n_c)."""
    shp = U.shape
    flat = U.reshape(-1, shp[-1])
    J = torch.func.vmap(torch.func.jacrev(fn))(flat)
    return J.reshape(*shp[:-1], *J.shape[1:])


def dW_dU(U, prm: Params):
    return _jacobian(lambda x: entropy_variables(x, prm), U)


def conservative_from_entropy(W, prm: Params):
    """The inverse of the map of Eq. (25), U(W), in closed form.  With
    a = -alpha/(gam-1) and q = (rho/p)(p rho^-gam)^(1/(alpha+gam)):
        q = -W_last,  V = W_mom / q,  T' = p/rho = (W_0/q + |V|^2/2) / a,
        q T' = (T' rho^(1-gam))^(1/(alpha+gam))
          =>  rho = ((q T')^(alpha+gam) / T')^(1/(1-gam)),  p = rho T'."""
    g, al = prm.gam, prm.alpha
    a = -al / (g - 1.0)
    q = -W[..., -1]
    V = W[..., 1:-1] / q[..., None]
    v2 = (V * V).sum(-1)
    Tp = (W[..., 0] / q + 0.5 * v2) / a
    rho = ((q * Tp) ** (al + g) / Tp) ** (1.0 / (1.0 - g))
    p = rho * Tp
    return torch.cat([rho[..., None], rho[..., None] * V, (p / (g - 1.0) + 0.5 * rho * v2)[..., None]], dim=-1)


def dU_dW(U, prm: Params):
    """A~_0 = dU/dW, Eq. (19): the Jacobian of the inverse map U(W) at
    W = W(U).  (Inverting dW/dU instead would carry its condition number,
    ~4e5 at Mach 0.1, into the round-off.)"""
    return _jacobian(lambda w: conservative_from_entropy(w, prm), entropy_variables(U, prm))


def symmetrized_flux_jacobians(U, prm: Params):
    """A~_i = A_i A~_0 with A_i = dF^{I(i)}/dU (Eq. (19)); returns (..., d, n_c, n_c)."""
    A = _jacobian(lambda x: euler_flux(x, prm), U)        # (..., d, nc, nc)
    return A @ dU_dW(U, prm)[..., None, :, :]


# ----------------------------------------------------------------------------
# Comparator of Sec. 6: the Hadamard form with the Ismail-Roe flux, entropy
# conservative for the standard entropy S = -rho s/(gam-1), s = log(p rho^-gam)
# (the generalized-entropy family at the physical entropy).  The flux formula
# is not printed in the paper (it cites Ismail & Roe, J. Comput. Phys. 228,
# 2009); it is restated here from that published method.
# ----------------------------------------------------------------------------

def standard_entropy(U, prm: Params):
    """S = -rho s/(gam-1), s = log(p rho^-gam)."""
    rho, V, p = primitives(U, prm)
    return -rho * (torch.log(p) - prm.gam * torch.log(rho)) / (prm.gam - 1.0)


def standard_entropy_variables(U, prm: Params):
    """dS/dU = [(gam - s)/(gam-1) - rho|V|^2/(2p), rho V/p, -rho/p]."""
    rho, V, p = primitives(U, prm)
    s = torch.log(p) - prm.gam * torch.log(rho)
    b = rho / p
    first = (prm.gam - s) / (prm.gam - 1.0) - 0.5 * b * (V * V).sum(-1)
    return torch.cat([first[..., None], b[..., None] * V, -b[..., None]], dim=-1)


def log_mean(a, b):
    """Logarithmic mean (a - b)/(log a - log b) of positive a, b, written as
    b eps / log1p(eps) with eps = a/b - 1 (no cancellation; limit b at a = b)."""
    eps = a / b - 1.0
    safe = torch.where(eps == 0, torch.ones_like(eps), eps)
    q = torch.where(eps == 0, torch.ones_like(eps), safe / torch.log1p(safe))
    return b * q


def ir_averages(Uk, Uv, prm: Params):
    """The Ismail-Roe averages of a state pair.  With z = sqrt(rho/p) [1, V, p]:
      rho^ = {z_1} {z_nc}_log,  V^ = {z V}/{z_1},  p1^ = {z_nc}/{z_1},
      p2^ = (gam+1)/(2 gam) {z_nc}_log/{z_1}_log + (gam-1)/(2 gam) {z_nc}/{z_1}
    ({.} arithmetic mean, {.}_log logarithmic mean); returns rho^, V^, p1^, p2^."""
    g = prm.gam
    rk, Vk, pk = primitives(Uk, prm)
    rv, Vv, pv = primitives(Uv, prm)
    z1k, z1v = torch.sqrt(rk / pk), torch.sqrt(rv / pv)
    znk, znv = torch.sqrt(rk * pk), torch.sqrt(rv * pv)
    a1, an = arith_avg(z1k, z1v), arith_avg(znk, znv)
    l1, ln = log_mean(z1k, z1v), log_mean(znk, znv)
    Vh = arith_avg(z1k[..., None] * Vk, z1v[..., None] * Vv) / a1[..., None]
    rh = a1 * ln
    p1 = an / a1
    p2 = (g + 1.0) / (2.0 * g) * ln / l1 + (g - 1.0) / (2.0 * g) * an / a1
    return rh, Vh, p1, p2


def ir_flux(Uk, Uv, prm: Params):
    """Ismail-Roe entropy-conservative flux, all directions: (..., d, n_c).
    With the averages of ``ir_averages``,
      H^ = gam p2^/((gam-1) rho^) + |V^|^2/2,
      F_i = [rho^ V^_i, rho^ V^_i V^ + p1^ e_i, rho^ V^_i H^]."""
    g = prm.gam
    rh, Vh, p1, p2 = ir_averages(Uk, Uv, prm)
    Hh = g * p2 / ((g - 1.0) * rh) + 0.5 * (Vh * Vh).sum(-1)
    d = Uk.shape[-1] - 2
    out = []
    for i in range(d):
        m = rh * Vh[..., i]
        mom = m[..., None] * Vh + p1[..., None] * torch.nn.functional.one_hot(torch.tensor(i), d).to(Uk)
        out.append(torch.cat([m[..., None], mom, (m * Hh)[..., None]], -1))
    return torch.stack(out, dim=-2)


def ir_dissipation_matrix(Uk, Uv, n, prm: Params):
    """Matrix dissipation for the Ismail-Roe comparator (not printed in the
    paper; the construction of Eq. (69) carried over to the standard entropy):
    R^ |Lambda_n| T^ R^T at the state rho^, V^, p^ = p1^ of ``ir_averages``,
    to be applied to the jump of the standard entropy variables.  R^ T^ R^T is
    the eigenvector factorisation of dU/dw for the standard entropy (Barth's
    scaling): the acoustic and entropy columns of Eq. (80) with
    T^ = rho^/(2 gam), (gam-1) rho^/gam, rho^/(2 gam), and the shear modes
    with weight p^ written through the projector I - n n^T (so that no
    tangent basis is needed and the 3D form is exact):
      R^ |Lambda| T^ R^T = sum_k |lambda_k| T_k r_k r_k^T + |V^.n| p^ B^T (I - n n^T) B,
      B = [0 | I_d | V^] (d x n_c).
    Symmetric positive semi-definite for any pair, so the entropy production
    of the term is -|nu|/2 dw^T (...) dw <= 0; for equal states R^ T^ R^T
    equals dU/dw (pinned in the tests).  Returns (..., n_c, n_c)."""
    g = prm.gam
    rh, Vh, p1, _ = ir_averages(Uk, Uv, prm)
    d = Vh.shape[-1]
    a = torch.sqrt(g * p1 / rh)
    vv = (Vh * Vh).sum(-1)
    Hh = a * a / (g - 1.0) + 0.5 * vv
    vn = (Vh * n).sum(-1)
    one = torch.ones_like(vn)
    c_m = torch.cat([one[..., None], Vh - a[..., None] * n, (Hh - a * vn)[..., None]], -1)
    c_0 = torch.cat([one[..., None], Vh, (0.5 * vv)[..., None]], -1)
    c_p = torch.cat([one[..., None], Vh + a[..., None] * n, (Hh + a * vn)[..., None]], -1)
    w_m = (vn - a).abs() * rh / (2.0 * g)
    w_0 = vn.abs() * (g - 1.0) * rh / g
    w_p = (vn + a).abs() * rh / (2.0 * g)
    D = (w_m[..., None, None] * c_m[..., :, None] * c_m[..., None, :]
         + w_0[..., None, None] * c_0[..., :, None] * c_0[..., None, :]
         + w_p[..., None, None] * c_p[..., :, None] * c_p[..., None, :])
    eye = torch.eye(d, dtype=Vh.dtype).expand(*Vh.shape[:-1], d, d)
    B = torch.cat([torch.zeros(*Vh.shape[:-1], d, 1, dtype=Vh.dtype), eye, Vh[..., :, None]], -1)   # (..., d, nc)
    P = eye - n[..., :, None] * n[..., None, :]
    D = D + (vn.abs() * p1)[..., None, None] * (B.transpose(-1, -2) @ P @ B)
    return D


# ----------------------------------------------------------------------------
# Matrix interface dissipation ingredients, Sec. 4.5, Eqs. (69), (73)-(80)
# ----------------------------------------------------------------------------

def dissipation_factors(Uk, Uv, n, prm: Params):
    """X^ (..., n_c, n_c; columns are the eigenvectors of Eq. (80)), the
    eigenvalues Lambda_n (..., n_c) of Eq. (79) (signed) and the diagonal of
    S^ (..., n_c) of Eqs. (76)-(78), at the intermediate state of Eqs.
    (73)-(75) between U_k and U_v, for unit normal n (..., d).  3D as printed;
    2D by deleting the fourth row and column; 1D by deleting both shear
    modes."""
    g, a = prm.gam, prm.alpha
    zk, zv = param_vector(Uk, prm), param_vector(Uv, prm)
    d = Uk.shape[-1] - 2
    z1k, z1v, znk, znv = zk[..., 0], zv[..., 0], zk[..., -1], zv[..., -1]
    A1 = arith_avg(z1k ** (-g / a), z1v ** (-g / a))
    E1 = exp_avg(znk, znv, (1.0 - g - a) / a + 1.0)
    E2 = exp_avg(z1k, z1v, -(g + a) / a + 1.0)
    z1a = arith_avg(z1k, z1v)
    rho_h = z1a / (A1 * E1)
    V_h = arith_avg(z1k[..., None] * zk[..., 1:-1], z1v[..., None] * zv[..., 1:-1]) / z1a[..., None]
    p_h = arith_avg(znk, znv)
    theta = rho_h / (p_h * A1 * E1)
    eta = 1.0 / (z1a * E2 * E1)
    a_h = torch.sqrt(g * p_h / rho_h)
    H_h = a_h ** 2 / (g - 1.0) + 0.5 * (V_h * V_h).sum(-1)
    vn = (V_h * n).sum(-1)
    one = torch.ones_like(vn)
    zero = torch.zeros_like(vn)
    if d == 1:
        # 1D (the problems of Secs. 7.1-7.2): no shear modes
        n1, V1 = n[..., 0], V_h[..., 0]
        cols = [
            torch.stack([one, V1 - a_h * n1, H_h - a_h * vn], -1),
            torch.stack([one, V1, 0.5 * V1 * V1], -1),
            torch.stack([one, V1 + a_h * n1, H_h + a_h * vn], -1),
        ]
        lam = [vn - a_h, vn, vn + a_h]
        sc = [theta / (2 * g), (g - 1) * (g + a) * theta / (g * a), theta / (2 * g)]
    elif d == 2:
        n1, n2 = n[..., 0], n[..., 1]
        V1, V2 = V_h[..., 0], V_h[..., 1]
        cols = [
            torch.stack([one, V1 - a_h * n1, V2 - a_h * n2, H_h - a_h * vn], -1),
            torch.stack([one, V1, V2, 0.5 * (V_h * V_h).sum(-1)], -1),
            torch.stack([zero, n2, -n1, V1 * n2 - V2 * n1], -1),
            torch.stack([one, V1 + a_h * n1, V2 + a_h * n2, H_h + a_h * vn], -1),
        ]
        lam = [vn - a_h, vn, vn, vn + a_h]
        sc = [theta / (2 * g), (g - 1) * (g + a) * theta / (g * a), eta, theta / (2 * g)]
    else:
        n1, n2, n3 = n[..., 0], n[..., 1], n[..., 2]
        V1, V2, V3 = V_h[..., 0], V_h[..., 1], V_h[..., 2]
        cols = [
            torch.stack([one, V1 - a_h * n1, V2 - a_h * n2, V3 - a_h * n3, H_h - a_h * vn], -1),
            torch.stack([one, V1, V2, V3, 0.5 * (V_h * V_h).sum(-1)], -1),
            torch.stack([zero, n2, -n1, zero, V1 * n2 - V2 * n1], -1),
            torch.stack([zero, -n3, zero, n1, V3 * n1 - V1 * n3], -1),
            torch.stack([one, V1 + a_h * n1, V2 + a_h * n2, V3 + a_h * n3, H_h + a_h * vn], -1),
        ]
        lam = [vn - a_h, vn, vn, vn, vn + a_h]
        sc = [theta / (2 * g), (g - 1) * (g + a) * theta / (g * a), eta, eta, theta / (2 * g)]
    return torch.stack(cols, -1), torch.stack(lam, -1), torch.stack(sc, -1)


def dissipation_matrix(Uk, Uv, n, prm: Params):
    """X^ |Lambda_n| S^ X^T of Eq. (69) (..., n_c, n_c)."""
    X, lam, sc = dissipation_factors(Uk, Uv, n, prm)
    return (X * (lam.abs() * sc)[..., None, :]) @ X.transpose(-1, -2)


# ----------------------------------------------------------------------------
# Viscous fluxes, Eq. (5), written in terms of the entropy-variable gradient
# ----------------------------------------------------------------------------

def temperature(U, prm: Params):
    rho, V, p = primitives(U, prm)
    return p / (rho * prm.R)


def viscous_flux_from_prim_grads(U, dV, dT, prm: Params):
    """F^{V(i)} of Eq. (5) from velocity gradients dV (..., d, d) with
    dV[..., j, k] = dV_k/dx_j and temperature gradient dT (..., d); returns
    (..., d, n_c)."""
    rho, V, p = primitives(U, prm)
    d = V.shape[-1]
    div = torch.diagonal(dV, dim1=-2, dim2=-1).sum(-1)
    out = []
    for i in range(d):
        # tau_{x_i x_k} = mu (dV_i/dx_k + dV_k/dx_i - 2/3 delta_ik div V)
        tau = prm.mu * (dV[..., :, i] + dV[..., i, :])
        tau = tau - prm.mu * (2.0 / 3.0) * div[..., None] * torch.nn.functional.one_hot(torch.tensor(i), d).to(U)
        energy = (V * tau).sum(-1)
        if prm.heat_flux:
            energy = energy + prm.kappa * dT[..., i]
        out.append(torch.cat([torch.zeros_like(energy)[..., None], tau, energy[..., None]], -1))
    return torch.stack(out, dim=-2)


def conservative_from_standard_entropy(v, prm: Params):
    """The inverse of ``standard_entropy_variables`` in closed form: with
    v_nc = -rho/p, V = -v_m / v_nc, the specific entropy
    s = gam - (gam - 1)(v_1 - v_nc |V|^2 / 2), and s = log p - gam log rho,
    p = -rho / v_nc give log rho = (s + log(-v_nc)) / (1 - gam)."""
    vE = v[..., -1]
    V = -v[..., 1:-1] / vE[..., None]
    s = prm.gam - (prm.gam - 1.0) * (v[..., 0] - 0.5 * vE * (V * V).sum(-1))
    rho = torch.exp((s + torch.log(-vE)) / (1.0 - prm.gam))
    p = -rho / vE
    e = p / (prm.gam - 1.0) + 0.5 * rho * (V * V).sum(-1)
    return torch.cat([rho[..., None], rho[..., None] * V, e[..., None]], dim=-1)


def dU_dV_standard(U, prm: Params):
    """dU/dv for the standard entropy variables (the Hessian of the entropy
    potential: symmetric positive definite), by autograd of the closed-form
    inverse map."""
    return _jacobian(lambda v: conservative_from_standard_entropy(v, prm), standard_entropy_variables(U, prm))


def viscous_flux_from_w_grads(U, gW, prm: Params, entropy: str = "harten"):
    """Sum_j K~_ij dW/dx_j: the viscous flux of Eq. (5) with the primitive
    gradients obtained from the entropy-variable gradients gW (..., d, n_c)
    through dV/dW and dT/dW (both dq/dU (dW/dU)^-1 by autograd).  ``entropy``
    picks the variables the gradients are of: Harten's W (Eq. (25), the
    entropy-split scheme) or the standard entropy variables (the Ismail-Roe
    comparator)."""
    d = U.shape[-1] - 2
    Ainv = dU_dW(U, prm) if entropy == "harten" else dU_dV_standard(U, prm)
    JV = _jacobian(lambda x: primitives(x, prm)[1], U) @ Ainv    # (..., d, nc)
    JT = _jacobian(lambda x: temperature(x, prm)[..., None], U) @ Ainv  # (..., 1, nc)
    dV = torch.einsum("...kc,...jc->...jk", JV, gW)              # dV_k/dx_j
    dT = torch.einsum("...c,...jc->...j", JT[..., 0, :], gW)
    return viscous_flux_from_prim_grads(U, dV, dT, prm)


def viscous_K(U, prm: Params, entropy: str = "harten"):
    """K~_ij (..., d, d, n_c, n_c) by probing the linear map dW/dx_j -> F^V_i
    on unit vectors (exact; the map is linear in the gradient); ``entropy`` as
    in ``viscous_flux_from_w_grads``."""
    d = U.shape[-1] - 2
    nc = d + 2
    K = torch.zeros(*U.shape[:-1], d, d, nc, nc, dtype=U.dtype)
    for j in range(d):
        for c in range(nc):
            gW = torch.zeros(*U.shape[:-1], d, nc, dtype=U.dtype)
            gW[..., j, c] = 1.0
            Fv = viscous_flux_from_w_grads(U, gW, prm, entropy)  # (..., d, nc)
            K[..., :, j, :, c] = Fv
    return K
