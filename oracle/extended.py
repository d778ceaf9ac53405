"""Residual of single elements in extended precision (mpmath): test infrastructure.

Only ``tests/`` (and the script that writes ``tests/golden/*_extended.txt``)
use this module.  It evaluates the same discretization as ``residual.py`` --
the weak entropy-split form of Eq. (100) or the weak Hadamard form of Eq.
(99), the entropy-conservative SATs of Eq. (43) with the Sjogreen-Yee flux of
Eq. (48), and the matrix interface dissipation of Eq. (69) -- for a handful of
elements of a 2D mesh, with every operation carried to ``DPS`` significant
digits.  The float64 inputs (state, reference operator, metric terms, scaled
normals) are taken as exact numbers; the result is then the exact residual of
those inputs to about 10^-(DPS-10) relative to the terms it is summed from,
and the distance of a float64 implementation from it is that
implementation's own rounding.  Readings are those of ``residual.py`` and
``physics.py`` (the mean of the product in Eq. (48), arithmetic means where
no subscript e is printed, the physical operators of Sec. 2.1 formed from
Lambda_ij = J dxi_j/dx_i and the reference Q_xi_j, curved facets with
B_g -> |nu| and n = nu/|nu| in Eq. (69)).

Independent of ``residual.py``: plain Python loops over nodes on mpmath
numbers, no torch.  A~_i v (Eq. (19)) is the directional derivative
d/dh F_i(U(W + h v)) at h = 0 through the closed-form inverse of Eq. (25),
taken by a central difference at DPS digits with h = 10^-(DPS/2 - 5): its
truncation error, O(h^2) ~ 1e-40, and its cancellation, O(10^-DPS / h) ~
1e-30, are both far below float64 rounding.

Pins (tests/test_oracle_extended.py): equal-state flux = Euler flux, the
closed-form inverse of Eq. (25), and A~_i W = beta F_i (Eq. (26)); on a
periodic curved mesh with exactly opposite paired normals, the entropy rate
of the EC split residual is zero to 1e-38 of its scale (Thm. 2) and that of
the Hadamard form equals -2 sum psi^T Q_x 1 (the float64 metric terms'
defect in the discrete metric identity) to the same accuracy (Thm. 4), the
dissipation makes it negative; and the float64 oracle agrees with it to a
few eps of the summand scale on the config-2 mesh.
"""
from __future__ import annotations

import mpmath as mp

DPS = 50


def _mpf(x):
    return mp.mpf(float(x))


class _Phys:
    """gam and beta as the float64 numbers the other implementations use;
    Harten's alpha = -gam - beta (gam - 1) (Eq. (16)) formed at DPS digits."""

    def __init__(self, gam=1.4, beta=2.5):
        self.gam = _mpf(gam)
        self.beta = _mpf(beta)
        self.alpha = -self.gam - self.beta * (self.gam - 1)


def _prim(U, P):
    """rho, V, p, e from the conservative variables (Sec. 2.2)."""
    rho = U[0]
    d = len(U) - 2
    V = [U[1 + i] / rho for i in range(d)]
    e = U[-1]
    p = (P.gam - 1) * (e - rho * sum(v * v for v in V) / 2)
    return rho, V, p, e


def _q(rho, p, P):
    """z_1 of Eq. (45): (rho/p)(p rho^-gam)^(1/(alpha+gam))."""
    return (rho / p) * mp.power(p * mp.power(rho, -P.gam), 1 / (P.alpha + P.gam))


def entropy_vars(U, P):
    """Harten entropy variables of Eq. (25)."""
    rho, V, p, _ = _prim(U, P)
    q = _q(rho, p, P)
    first = -P.alpha / (P.gam - 1) * p / rho - sum(v * v for v in V) / 2
    return [q * first] + [q * v for v in V] + [-q]


def cons_from_entropy(W, P):
    """Closed-form inverse of Eq. (25): q = -W_nc, V = W_mom/q,
    p/rho = (W_1/q + |V|^2/2)/a with a = -alpha/(gam-1), and rho from
    q (p/rho) = ((p/rho) rho^(1-gam))^(1/(alpha+gam))."""
    g, al = P.gam, P.alpha
    a = -al / (g - 1)
    q = -W[-1]
    V = [w / q for w in W[1:-1]]
    v2 = sum(v * v for v in V)
    Tp = (W[0] / q + v2 / 2) / a
    rho = mp.power(mp.power(q * Tp, al + g) / Tp, 1 / (1 - g))
    p = rho * Tp
    return [rho] + [rho * v for v in V] + [p / (g - 1) + rho * v2 / 2]


def euler_flux(U, i, P):
    """F^{I(i)} of Eq. (5)."""
    rho, V, p, e = _prim(U, P)
    d = len(V)
    m = rho * V[i]
    return [m] + [m * V[j] + (p if j == i else 0) for j in range(d)] + [(e + p) * V[i]]


def at_times(U, i, v, P):
    """A~_i v = d/dh F_i(U(W(U) + h v)) at h = 0 (Eq. (19)), central difference."""
    W = entropy_vars(U, P)
    h = mp.mpf(10) ** (-(DPS // 2 - 5))
    Fp = euler_flux(cons_from_entropy([w + h * x for w, x in zip(W, v)], P), i, P)
    Fm = euler_flux(cons_from_entropy([w - h * x for w, x in zip(W, v)], P), i, P)
    return [(a - b) / (2 * h) for a, b in zip(Fp, Fm)]


def _param(U, P):
    rho, V, p, _ = _prim(U, P)
    return _q(rho, p, P), V, p


def _ari(a, b):
    return (a + b) / 2


def _expo(a, b, r):
    """{u^(r-1)}_e = (a^r - b^r)/(r (a - b)), Eq. (47); a^(r-1) when a = b."""
    if a == b:
        return mp.power(a, r - 1)
    return (mp.power(a, r) - mp.power(b, r)) / (r * (a - b))


def sy_flux(Uk, Uv, i, P):
    """Sjogreen-Yee two-point flux F*_i, Eq. (48), in the reading of physics.sy_flux."""
    g, a = P.gam, P.alpha
    z1k, Vk, znk = _param(Uk, P)
    z1v, Vv, znv = _param(Uv, P)
    d = len(Vk)
    den = _ari(mp.power(z1k, -g / a), mp.power(z1v, -g / a)) * _expo(znk, znv, (1 - g - a) / a + 1)
    Va = [_ari(x, y) for x, y in zip(Vk, Vv)]
    ke = sum(v * v for v in Va) - _ari(sum(v * v for v in Vk), sum(v * v for v in Vv)) / 2
    enth = g / (g - 1) * _ari(mp.power(znk, -(g - 1) / a), mp.power(znv, -(g - 1) / a)) \
        * _expo(z1k, z1v, -(g + a) / a + 1)
    F1 = _ari(z1k * Vk[i], z1v * Vv[i]) / den
    return [F1] + [F1 * Va[j] + (_ari(znk, znv) if j == i else 0) for j in range(d)] + [F1 * (enth + ke)]


def dissipation_times(Uk, Uv, n, dw, P):
    """X^ |Lambda_n| S^ X^T dw of Eq. (69) at the intermediate state of Eqs.
    (73)-(75), 2D (the fourth row and column of Eq. (80) deleted); n a unit
    normal."""
    g, a = P.gam, P.alpha
    z1k, Vk, znk = _param(Uk, P)
    z1v, Vv, znv = _param(Uv, P)
    A1 = _ari(mp.power(z1k, -g / a), mp.power(z1v, -g / a))
    E1 = _expo(znk, znv, (1 - g - a) / a + 1)
    E2 = _expo(z1k, z1v, -(g + a) / a + 1)
    z1a = _ari(z1k, z1v)
    rho_h = z1a / (A1 * E1)
    Vh = [_ari(z1k * x, z1v * y) / z1a for x, y in zip(Vk, Vv)]
    p_h = _ari(znk, znv)
    theta = rho_h / (p_h * A1 * E1)
    eta = 1 / (z1a * E2 * E1)
    ah = mp.sqrt(g * p_h / rho_h)
    vh2 = sum(v * v for v in Vh)
    Hh = ah * ah / (g - 1) + vh2 / 2
    vn = Vh[0] * n[0] + Vh[1] * n[1]
    cols = [
        [1, Vh[0] - ah * n[0], Vh[1] - ah * n[1], Hh - ah * vn],
        [1, Vh[0], Vh[1], vh2 / 2],
        [0, n[1], -n[0], Vh[0] * n[1] - Vh[1] * n[0]],
        [1, Vh[0] + ah * n[0], Vh[1] + ah * n[1], Hh + ah * vn],
    ]
    lam = [abs(vn - ah), abs(vn), abs(vn), abs(vn + ah)]
    sc = [theta / (2 * g), (g - 1) * (g + a) * theta / (g * a), eta, theta / (2 * g)]
    y = [lam[k] * sc[k] * sum(cols[k][r] * dw[r] for r in range(4)) for k in range(4)]
    return [sum(cols[k][r] * y[k] for k in range(4)) for r in range(4)]


def _element(u, ref, mesh, k):
    """Nodal states, reference data and physical operators of element k."""
    n_p, d = ref.n_p, ref.d
    U = [[_mpf(u[k, c, m]) for c in range(d + 2)] for m in range(n_p)]
    Hr = [_mpf(x) for x in ref.H]
    Qr = [[[_mpf(ref.Q[j, a, b]) for b in range(n_p)] for a in range(n_p)] for j in range(d)]
    J = [_mpf(x) for x in mesh.J[k]]
    Lam = [[[_mpf(mesh.Lam[k, i, j, m]) for m in range(n_p)] for j in range(d)] for i in range(d)]
    nu = mesh.nu[k].reshape(-1, d)
    fn = ref.facet_nodes.reshape(-1)
    E = [[mp.mpf(0)] * n_p for _ in range(d)]
    for s, m in enumerate(fn):
        for i in range(d):
            E[i][m] = _mpf(nu[s, i])
    # Q_x_i = 1/2 sum_j (Lam_ij Q_xi_j - Q_xi_j^T Lam_ij) + 1/2 E_x_i  (Sec. 2.1)
    Q = [[[sum(Lam[i][j][a] * Qr[j][a][b] - Qr[j][b][a] * Lam[i][j][b] for j in range(d)) / 2
           + (E[i][a] / 2 if a == b else 0) for b in range(n_p)] for a in range(n_p)] for i in range(d)]
    H = [Hr[m] * J[m] for m in range(n_p)]
    return U, Q, E, H


def residual_elements(u, ref, mesh, elems, scheme="split", dissipation=True, gam=1.4, beta=2.5, dps=DPS):
    """du/dt of the elements ``elems`` of a 2D mesh, as mpmath numbers:
    a list (one per element) of [n_c][n_p] lists.  u: float64 (n_e, n_c, n_p)."""
    assert ref.d == 2, "2D only"
    with mp.workdps(dps):
        P = _Phys(gam, beta)
        n_p, d = ref.n_p, ref.d
        nc = d + 2
        fn = ref.facet_nodes.reshape(-1)
        n_slot = len(fn)
        out = []
        for k in elems:
            U, Q, E, H = _element(u, ref, mesh, k)
            r = [[mp.mpf(0)] * n_p for _ in range(nc)]
            if scheme == "split":
                f = [[euler_flux(U[m], i, P) for i in range(d)] for m in range(n_p)]
                w = [entropy_vars(U[m], P) for m in range(n_p)]
                for m in range(n_p):
                    cons = [mp.mpf(0)] * nc
                    nonc = [mp.mpf(0)] * nc
                    for i in range(d):
                        # (Q_x_i/(beta+1) + Q_x_i^T) f_i, row m
                        for n in range(n_p):
                            cm = Q[i][m][n] / (P.beta + 1) + Q[i][n][m]
                            for c in range(nc):
                                cons[c] += cm * f[n][i][c]
                        # A~_i (H^-1 Q_x_i w), node m
                        Dw = [sum(Q[i][m][n] * w[n][c] for n in range(n_p)) / H[m] for c in range(nc)]
                        for c, x in enumerate(at_times(U[m], i, Dw, P)):
                            nonc[c] += x
                    for c in range(nc):
                        r[c][m] = cons[c] / H[m] - nonc[c] / (P.beta + 1)
            elif scheme == "hadamard":
                # -(1/H_m) sum_i sum_n 2 S_x_i,mn F*_i(u_m, u_n), S = Q - E/2
                for m in range(n_p):
                    acc = [mp.mpf(0)] * nc
                    for n in range(n_p):
                        for i in range(d):
                            s = Q[i][m][n] - (E[i][m] / 2 if m == n else 0)
                            if s == 0:
                                continue
                            F = sy_flux(U[m], U[n], i, P)
                            for c in range(nc):
                                acc[c] -= 2 * s * F[c]
                    for c in range(nc):
                        r[c][m] = acc[c] / H[m]
            else:
                raise ValueError(scheme)
            # facet terms: EC SAT and dissipation at every facet node of k
            nu = mesh.nu[k].reshape(-1, d)
            pair = mesh.pair[k].reshape(-1, 2)
            for s in range(n_slot):
                m = fn[s]
                v, s2 = int(pair[s, 0]), int(pair[s, 1])
                Uv = [_mpf(u[v, c, fn[s2]]) for c in range(nc)]
                nus = [_mpf(nu[s, i]) for i in range(d)]
                sat = [mp.mpf(0)] * nc
                for i in range(d):
                    F = sy_flux(U[m], Uv, i, P)
                    for c in range(nc):
                        sat[c] -= nus[i] * F[c] / H[m]
                if dissipation:
                    b = mp.sqrt(sum(x * x for x in nus))
                    nh = [x / b for x in nus]
                    wk, wv = entropy_vars(U[m], P), entropy_vars(Uv, P)
                    Dm = dissipation_times(U[m], Uv, nh, [x - y for x, y in zip(wk, wv)], P)
                    for c in range(nc):
                        sat[c] -= b / (2 * H[m]) * Dm[c]
                for c in range(nc):
                    r[c][m] += sat[c]
            out.append(r)
        return out
