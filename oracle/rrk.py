"""Relaxation RK4 step, Sec. 6.1, Eqs. (97)-(98) (plain PyTorch, float64).

Classical RK4 stages (b = 1/6, 1/3, 1/3, 1/6), then the relaxation parameter
g_n solving

    f(g) = 1^T H s(u_n + g d) - 1^T H s(u_n) - g dt sum_i b_i w_i^T H r_i = 0,
    d = dt sum_i b_i r_i,

by bisection to machine precision, and u_{n+1} = u_n + g_n d.

Readings (the paper is silent on these details):
  * the equality form of Eq. (97) is used for every scheme (relaxation RK);
  * f is evaluated as sum_k 1^T H_k [s(u_n + g d) - s(u_n)] - g est with the
    per-node entropy change computed without cancellation
    (physics.harten_entropy_change): the difference of the two global sums
    in Eq. (97) loses all but a few digits (|f| ~ 1e-13 |S| near the root),
    which would leave g undefined beyond ~1e-9; bisection "to machine
    precision" needs f itself to relative precision;
  * g = 0 is always a root; f is convex in g (S_H is convex), so the root
    wanted is the other one, near 1.  Bracket [0.5, 1.5]; while f(lo) >= 0
    halve lo (down to 2^-10); while f(hi) <= 0 double hi (up to 4); no
    bracket -> error;
  * bisection stops when hi - lo <= 4 eps hi or after 200 halvings and
    returns the midpoint;
  * when |f| at both ends of [0.5, 1.5] is below the round-off floor
    64 eps 1^T H |s(u_n)|, the step changes entropy only at round-off level
    and g = 1 is returned (e.g. a free stream);
  * time advances by g dt (relaxation convention).

Pins (tests/test_oracle_rrk.py): entropy after an EC step equals entropy
before to round-off; g close to 1; bisection root satisfies f(g) ~ 0 and
brackets sign change; RK4 order on a linear ODE; the step reverse
(rrk4_step_vjp) gives the closed form H w(u_n) for the gradient of the
conserved total entropy of an EC step, and agrees with central differences
of the step with dissipation.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from .physics import Params, harten_entropy, harten_entropy_change, entropy_variables

DT = torch.float64
RK4_A = (0.0, 0.5, 0.5, 1.0)
RK4_B = (1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0)


class NoRootError(RuntimeError):
    pass


@dataclass
class StepInfo:
    g: float
    estimate: float          # dt sum_i b_i w_i^T H r_i
    S_before: float
    S_after: float
    iterations: int
    stage_production: tuple  # w_i^T H r_i per stage


def _H(ref, mesh):
    return torch.as_tensor(ref.H, dtype=DT)[None, :] * torch.as_tensor(mesh.J, dtype=DT)


def _S_total(u, Hn, prm):
    return float((Hn * harten_entropy(u.transpose(1, 2), prm)).sum())


def relaxation_gamma(u_n, d, estimate, ref, mesh, prm: Params = Params(), max_iter=200):
    """Bisection root of f(g) of Eq. (97) (equality form). Returns (g, iterations)."""
    Hn = _H(ref, mesh)
    floor = 64.0 * np.finfo(float).eps * float((Hn * harten_entropy(u_n.transpose(1, 2), prm).abs()).sum())
    Ut, dt_ = u_n.transpose(1, 2), d.transpose(1, 2)

    def f(g):
        return float((Hn * harten_entropy_change(Ut, g * dt_, prm)).sum()) - g * estimate

    lo, hi = 0.5, 1.5
    flo, fhi = f(lo), f(hi)
    if abs(flo) <= floor and abs(fhi) <= floor:
        return 1.0, 0
    while flo >= 0.0:
        lo *= 0.5
        if lo < 2.0 ** -10:
            raise NoRootError("relaxation: no g with f(g) < 0")
        flo = f(lo)
    while fhi <= 0.0:
        hi *= 2.0
        if hi > 4.0:
            raise NoRootError("relaxation: no g with f(g) > 0")
        fhi = f(hi)
    it = 0
    eps = np.finfo(float).eps
    while hi - lo > 4.0 * eps * hi and it < max_iter:
        mid = 0.5 * (lo + hi)
        fm = f(mid)
        if fm < 0.0:
            lo = mid
        else:
            hi = mid
        it += 1
    return 0.5 * (lo + hi), it


def rrk4_step(u, dt, rhs, ref, mesh, prm: Params = Params()):
    """One relaxation RK4 step; ``rhs(u)`` returns du/dt (n_e, n_c, n_p)."""
    u_n = u if torch.is_tensor(u) else torch.as_tensor(np.asarray(u), dtype=DT)
    Hn = _H(ref, mesh)
    rs, prods = [], []
    for i in range(4):
        Ui = u_n if i == 0 else u_n + RK4_A[i] * dt * rs[-1]
        ri = torch.as_tensor(rhs(Ui), dtype=DT)
        w = entropy_variables(Ui.transpose(1, 2), prm)
        prods.append(float((Hn[..., None] * w * ri.transpose(1, 2)).sum()))
        rs.append(ri)
    d = dt * sum(b * r for b, r in zip(RK4_B, rs))
    est = dt * sum(b * e for b, e in zip(RK4_B, prods))
    g, it = relaxation_gamma(u_n, d, est, ref, mesh, prm)
    u_next = u_n + g * d
    return u_next, StepInfo(g=g, estimate=est, S_before=_S_total(u_n, Hn, prm),
                            S_after=_S_total(u_next, Hn, prm), iterations=it,
                            stage_production=tuple(prods))


def rrk4_step_vjp(u, dt, rhs, ubar1, ref, mesh, prm: Params = Params()):
    """Reverse of one relaxation RK4 step: (d u_{n+1} / d u_n)^T ubar1.

    u_{n+1} = u_n + g d(u_n) with the stages and d = dt sum_i b_i r_i
    differentiated by torch.autograd through ``rhs`` (which must be
    differentiable: the oracle residual is), and g(u_n) the root of f(g; u_n)
    of Eq. (97), differentiated by the implicit function theorem,
    dg/du_n = -(df/du_n) / (df/dg) at the root (a root found by bisection is
    piecewise constant in u_n, so autograd cannot see it):

        ubar_n = (d u_{n+1}/d u_n |_g)^T ubar1 + (ubar1 . d) dg/du_n.

    Returns (ubar_n, g)."""
    u_n = (u if torch.is_tensor(u) else torch.as_tensor(np.asarray(u), dtype=DT)).detach()
    ub = ubar1 if torch.is_tensor(ubar1) else torch.as_tensor(np.asarray(ubar1), dtype=DT)
    Hn = _H(ref, mesh)
    x = u_n.clone().requires_grad_(True)
    rs, prods = [], []
    for i in range(4):
        Ui = x if i == 0 else x + RK4_A[i] * dt * rs[-1]
        ri = rhs(Ui)
        w = entropy_variables(Ui.transpose(1, 2), prm)
        prods.append((Hn[..., None] * w * ri.transpose(1, 2)).sum())
        rs.append(ri)
    d = dt * sum(b * r for b, r in zip(RK4_B, rs))
    est = dt * sum(b * e for b, e in zip(RK4_B, prods))
    g, _ = relaxation_gamma(u_n, d.detach(), float(est.detach()), ref, mesh, prm)
    g_t = torch.tensor(g, dtype=DT, requires_grad=True)
    f = (Hn * harten_entropy_change(x.transpose(1, 2), g_t * d.transpose(1, 2), prm)).sum() - g_t * est
    f_x, f_g = torch.autograd.grad(f, (x, g_t), retain_graph=True)
    (part_a,) = torch.autograd.grad(x + g * d, x, grad_outputs=ub)
    return part_a - float((ub * d.detach()).sum()) / float(f_g) * f_x, g
