"""Pins of oracle/rrk.py (Sec. 6.1, Eqs. (97)-(98))."""
import numpy as np
import pytest
import torch

from esplit_inputs import tri_operator, periodic_tri_mesh, states
from oracle import residual as R, rrk, diagnostics as Dg
from oracle.physics import Params

P = Params()


def _vortex(p=2, N=4):
    op = tri_operator(p)
    m = periodic_tri_mesh(op, N, 10.0, 0.05)
    u = torch.as_tensor(states.add_uniform_noise(states.isentropic_vortex(m), 1e-3, 1))
    return op, m, u


def test_ec_step_conserves_entropy():
    op, m, u = _vortex()
    dt = states.cfl_timestep(m, u.numpy(), 0.1)
    rhs = lambda x: R.residual(x, op, m, P)
    for _ in range(3):
        u, info = rrk.rrk4_step(u, dt, rhs, op, m, P)
        assert abs(info.S_after - info.S_before) < 5e-15 * abs(info.S_before)
        assert abs(info.g - 1.0) < 1e-3
        assert abs(info.estimate) < 1e-12 * abs(info.S_before)


def test_dissipative_step_relaxes_to_estimate():
    """With dissipation the step removes exactly g * dt sum b_i w_i^T H r_i."""
    op, m, u = _vortex()
    dt = states.cfl_timestep(m, u.numpy(), 0.1)
    rhs = lambda x: R.residual(x, op, m, P, dissipation=True)
    u1, info = rrk.rrk4_step(u, dt, rhs, op, m, P)
    assert info.estimate < 0
    assert abs(info.S_after - info.S_before - info.g * info.estimate) < 1e-14 * abs(info.S_before)
    assert abs(info.g - 1.0) < 1e-2


def test_bisection_brackets_root():
    """The returned g sits at a sign change of f (Eq. (97), equality form)."""
    op, m, u = _vortex()
    dt = states.cfl_timestep(m, u.numpy(), 0.1)
    rhs = lambda x: R.residual(x, op, m, P, dissipation=True)
    rs, prods = [], []
    for i in range(4):
        Ui = u if i == 0 else u + rrk.RK4_A[i] * dt * rs[-1]
        rs.append(rhs(Ui))
        prods.append(float(Dg.entropy_rate(Ui, rs[-1], op, m, P)))
    d = dt * sum(b * r for b, r in zip(rrk.RK4_B, rs))
    est = dt * sum(b * e for b, e in zip(rrk.RK4_B, prods))
    g, it = rrk.relaxation_gamma(u, d, est, op, m, P)
    S0 = float(Dg.entropy_total(u, op, m, P))
    f = lambda gg: float(Dg.entropy_total(u + gg * d, op, m, P)) - S0 - gg * est
    assert f(g * (1 - 1e-6)) < 0 < f(g * (1 + 1e-6))
    assert it > 40
    u1, info = rrk.rrk4_step(u, dt, rhs, op, m, P)
    assert info.g == g


def test_freestream_returns_unit_gamma():
    op = tri_operator(1)
    m = periodic_tri_mesh(op, 2, 10.0, 0.05)
    u = torch.as_tensor(states.uniform_state(m.n_e, 2, op.n_p))
    rhs = lambda x: R.residual(x, op, m, P)
    u1, info = rrk.rrk4_step(u, 0.01, rhs, op, m, P)
    assert info.g == 1.0


def test_rk4_order():
    """Without relaxation effects (g ~ 1) the RK4 stages converge at 4th order:
    halving dt reduces the one-step defect against a fine reference by ~32."""
    op, m, u = _vortex(p=1, N=2)
    rhs = lambda x: R.residual(x, op, m, P)
    T = 0.02

    def run(n):
        x = u.clone()
        for _ in range(n):
            x, _ = rrk.rrk4_step(x, T / n, rhs, op, m, P)
        return x

    ref = run(16)
    e1 = float((run(1) - ref).abs().max())
    e2 = float((run(2) - ref).abs().max())
    assert np.log2(e1 / e2) > 3.5


def test_step_vjp_closed_form_for_ec():
    """EC scheme: the relaxation step conserves the total entropy for every
    u_n, so the gradient of S(u_{n+1}) with respect to u_n is H w(u_n); the
    step reverse applied to H w(u_{n+1}) must give it (the implicit-function
    term for g is needed: without it this fails)."""
    from oracle.physics import entropy_variables
    op, m, u = _vortex(p=2, N=3)
    dt = states.cfl_timestep(m, u.numpy(), 0.1)
    rhs = lambda x: R.residual(x, op, m, P)
    u1, info = rrk.rrk4_step(u, dt, rhs, op, m, P)
    Hn = rrk._H(op, m)
    gS1 = Hn[:, None, :] * entropy_variables(u1.transpose(1, 2), P).transpose(1, 2)
    gS0 = Hn[:, None, :] * entropy_variables(u.transpose(1, 2), P).transpose(1, 2)
    ub0, g = rrk.rrk4_step_vjp(u, dt, rhs, gS1, op, m, P)
    assert abs(g - info.g) == 0.0
    err = float((ub0 - gS0).abs().max() / gS0.abs().max())
    assert err <= 1e-11, err


def test_step_vjp_central_differences():
    """With dissipation: <ubar1, (step(u + h v) - step(u - h v)) / 2h> against
    <ubar0, v> on random unit directions (h = 1e-6)."""
    op, m, u = _vortex(p=2, N=3)
    dt = states.cfl_timestep(m, u.numpy(), 0.1)
    rhs = lambda x: R.residual(x, op, m, P, dissipation=True)
    rng = np.random.default_rng(12)
    ub1 = torch.as_tensor(rng.normal(size=tuple(u.shape)))
    ub0, g = rrk.rrk4_step_vjp(u, dt, rhs, ub1, op, m, P)
    h = 1e-6
    for _ in range(4):
        v = torch.as_tensor(rng.normal(size=tuple(u.shape)))
        v /= v.norm()
        up, _ = rrk.rrk4_step(u + h * v, dt, rhs, op, m, P)
        um, _ = rrk.rrk4_step(u - h * v, dt, rhs, op, m, P)
        fd = float(((up - um) / (2 * h) * ub1).sum())
        ad = float((ub0 * v).sum())
        assert abs(fd - ad) <= 1e-6 * max(1.0, abs(ad)), (fd, ad)
