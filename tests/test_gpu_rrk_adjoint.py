"""Reverse of the relaxation RK4 step (esplit_rrk_step_vjp) and gradients
through many steps with per-step checkpoints (config 4's second part)."""
import numpy as np
import pytest
import torch

from esplit_inputs import tri_operator, periodic_tri_mesh, states

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2305_07181_gb300 as es
    return es


def test_step_vjp_central_differences(lib):
    """<ubar', (Phi(u + h v) - Phi(u - h v)) / 2h> = <ubar, v> for the
    relaxation RK4 step Phi with dissipation (g depends on u)."""
    op = tri_operator(2)
    m = periodic_tri_mesh(op, 4, 10.0, 0.05)
    u0 = states.add_uniform_noise(states.isentropic_vortex(m), 1e-3, 7)
    dt = states.cfl_timestep(m, u0, 0.1)
    s = lib.Solver(op, m, lib.Params(dissipation=True))
    u = s.to_device(u0)
    rng = np.random.default_rng(8)
    ubar1 = s.to_device(rng.normal(size=u0.shape))
    ubar0, g = s.rrk_step_vjp(u, dt, ubar1)

    def phi(x):
        y = x.clone()
        s.rrk_step(y, dt)
        return y

    h = 1e-6
    for _ in range(8):
        v = rng.normal(size=u0.shape)
        v /= np.linalg.norm(v)
        vd = s.to_device(v)
        fd = float(((phi(u + h * vd) - phi(u - h * vd)) / (2 * h) * ubar1).sum())
        ad = float((ubar0 * vd).sum())
        assert abs(fd - ad) <= 2e-6 * max(1.0, abs(ad)), (fd, ad)
    s.close()


def test_entropy_gradient_through_50_steps_closed_form(lib):
    """Config 4: 128 x 128 quads -> 32,768 curved triangles, p = 3, vortex.
    With the entropy-conservative scheme relaxation RK keeps 1^T H s(u_n)
    equal to 1^T H s(u_0) for every u_0, so d S(u_50) / d u_0 = H w(u_0):
    the gradient through 50 steps, including the implicit dependence of every
    g_n on the state, must reproduce it (it would not with g frozen)."""
    from paper_2305_07181_gb300.adjoint import entropy_gradient_through_steps
    op = tri_operator(3)
    m = periodic_tri_mesh(op, 128, 10.0, 0.05)
    u0 = states.add_uniform_noise(states.isentropic_vortex(m), 1e-3, 4)
    dt = states.cfl_timestep(m, u0, 0.1)
    s = lib.Solver(op, m, lib.Params())
    ud = s.to_device(u0)
    grad, uN, gs = entropy_gradient_through_steps(s, ud, dt, 50)
    exact = s.entropy_grad(ud)
    err = float((grad - exact).abs().max() / exact.abs().max())
    print(f"50-step entropy gradient vs H w(u_0): rel err {err:.2e}; g range {min(gs):.9f}..{max(gs):.9f}")
    assert err <= 1e-12
    assert abs(s.entropy(uN) - s.entropy(ud)) <= 1e-13 * abs(s.entropy(ud)) * 50
    s.close()


def test_step_vjp_viscous_central_differences(lib):
    """The step reverse with the BO viscous terms (Navier-Stokes, 2D p = 2 and
    the Taylor-Green state on 48 tetrahedra)."""
    from esplit_inputs import tet_operator
    from esplit_inputs.mesh import periodic_tet_mesh
    cases = []
    op = tri_operator(2)
    m = periodic_tri_mesh(op, 4, 10.0, 0.05)
    cases.append((op, m, states.add_uniform_noise(states.isentropic_vortex(m), 1e-3, 17), 0.01))
    op3 = tet_operator(2)
    m3 = periodic_tet_mesh(op3, 2, 2 * np.pi, 0.02)
    cases.append((op3, m3, states.taylor_green(m3), 1.0 / 1600.0))
    rng = np.random.default_rng(18)
    for op, m, u0, mu in cases:
        dt = states.cfl_timestep(m, u0, 0.1)
        s = lib.Solver(op, m, lib.Params(dissipation=True, viscous=True, mu=mu))
        u = s.to_device(u0)
        ubar1 = s.to_device(rng.normal(size=u0.shape))
        ubar0, g = s.rrk_step_vjp(u, dt, ubar1)

        def phi(x):
            y = x.clone()
            s.rrk_step(y, dt)
            return y

        h = 1e-6
        for _ in range(4):
            v = rng.normal(size=u0.shape)
            v /= np.linalg.norm(v)
            vd = s.to_device(v)
            fd = float(((phi(u + h * vd) - phi(u - h * vd)) / (2 * h) * ubar1).sum())
            ad = float((ubar0 * vd).sum())
            assert abs(fd - ad) <= 2e-6 * max(1.0, abs(ad)), (fd, ad)
        s.close()


@pytest.mark.parametrize("case", ["dissipation", "viscous_2d", "viscous_tets"])
def test_step_vjp_against_oracle_adjoint(lib, case):
    """The GPU step reverse against the oracle's (oracle/rrk.py rrk4_step_vjp:
    torch.autograd through the oracle's stages and the implicit-function term
    for g, pinned by the closed-form entropy gradient and by central
    differences), on the same state, step and cotangent: dissipative 2D, the
    Navier-Stokes terms in 2D and on the Taylor-Green tetrahedra.  Both sides
    carry the rounding of four residual reverses summed against the
    cotangent: max-norm relative 1e-9."""
    from oracle import residual as R, rrk
    from oracle.physics import Params as OP
    from esplit_inputs import tet_operator
    from esplit_inputs.mesh import periodic_tet_mesh
    if case == "viscous_tets":
        op = tet_operator(2)
        m = periodic_tet_mesh(op, 2, 2 * np.pi, 0.02)
        u0 = states.taylor_green(m)
        mu = 1.0 / 1600.0
    else:
        op = tri_operator(2)
        m = periodic_tri_mesh(op, 4, 10.0, 0.05)
        u0 = states.add_uniform_noise(states.isentropic_vortex(m), 1e-3, 21)
        mu = 0.01 if case == "viscous_2d" else 0.0
    visc = case != "dissipation"
    dt = states.cfl_timestep(m, u0, 0.1)
    s = lib.Solver(op, m, lib.Params(dissipation=True, viscous=visc, mu=mu))
    ub1 = np.random.default_rng(22).normal(size=u0.shape)
    ub0, g = s.rrk_step_vjp(s.to_device(u0), dt, s.to_device(ub1))
    s.close()
    prm = OP(mu=mu)
    rhs = lambda x: R.residual(x, op, m, prm, dissipation=True, viscous=visc)
    ub0o, go = rrk.rrk4_step_vjp(torch.as_tensor(u0), dt, rhs, torch.as_tensor(ub1), op, m, prm)
    err = float((ub0.cpu() - ub0o).abs().max() / ub0o.abs().max())
    print(f"step reverse vs oracle adjoint ({case}): rel err {err:.2e}, g {g:.15f} vs {go:.15f}")
    assert abs(g - go) <= 1e-10
    assert err <= 1e-9
