"""The float32 path (precision "fp32", ESPLIT_FP32): the inviscid entropy-split
residual with every flux, entropy variable, A~_i product, two-point flux,
dissipation and contraction in float32, evaluated as deviations from float64
reference states, against the float64 oracle.

Stated bound: max-norm relative error per component <= FP32_BOUND = 1e-5 on
every workload below (triangles p 1..4 on the config-2 state kind, at small
and full size; random states with O(1) variations; 1D); the observed errors
are printed.  Tetrahedra take the FP32-bulk kernels under this setting.  A
uniform state gives a residual of exactly zero (free stream)."""
import numpy as np
import pytest
import torch

from esplit_inputs import tri_operator, tet_operator, line_operator, periodic_tri_mesh, states
from esplit_inputs.mesh import periodic_tet_mesh, periodic_line_mesh

pytestmark = pytest.mark.gpu

FP32_BOUND = 1e-5


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2305_07181_gb300 as es
    return es


def _oracle():
    from oracle import residual as R, diagnostics as Dg, rrk
    from oracle.physics import Params as OP
    return R, Dg, rrk, OP


def rel_err(a, b):
    num = np.abs(np.asarray(a) - np.asarray(b)).max(axis=(0, 2))
    den = np.abs(np.asarray(b)).max(axis=(0, 2))
    return float((num / den).max())


def _check(lib, op, m, u, diss, label, elems=None):
    R, Dg, rrk, OP = _oracle()
    s = lib.Solver(op, m, lib.Params(dissipation=diss, precision="fp32"))
    r = s.residual(s.to_device(u)).cpu().numpy()
    assert s.status() == 0
    s.close()
    if elems is not None:
        r = r[elems]
    ro = R.residual(u, op, m, OP(), dissipation=diss, elems=elems).numpy()
    err = rel_err(r, ro)
    print(f"fp32 {label} diss={diss}: rel err {err:.2e}")
    assert err <= FP32_BOUND
    return err


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("diss", [False, True])
def test_fp32_vortex_small(lib, p, diss):
    op = tri_operator(p)
    m = periodic_tri_mesh(op, 8, 10.0, 0.05)
    u = states.add_uniform_noise(states.isentropic_vortex(m), 1e-3, 2)
    _check(lib, op, m, u, diss, f"vortex p={p}")


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_fp32_random_states(lib, p):
    """O(1) variations between nodes and across facets: the deviation
    formulas away from their small-variation regime (the exponential averages
    take their closed form, |eps| >= 0.25)."""
    op = tri_operator(p)
    m = periodic_tri_mesh(op, 5, 10.0, 0.05)
    u = states.random_positive_state(m.n_e, 2, op.n_p, seed=60 + p)
    _check(lib, op, m, u, True, f"random p={p}")


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_fp32_full_size_sampled(lib, p):
    """Config 2 at full size (32,768 curved triangles, vortex + 1e-3 noise) in
    the bench's launch configuration, 48 sampled elements plus the first and
    last."""
    op = tri_operator(p)
    m = periodic_tri_mesh(op, 128, 10.0, 0.05)
    u = states.add_uniform_noise(states.isentropic_vortex(m), 1e-3, 2)
    el = np.concatenate([np.random.default_rng(70 + p).choice(m.n_e, 48, replace=False), [0, m.n_e - 1]])
    _check(lib, op, m, u, True, f"full size p={p}", elems=el)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_fp32_tetrahedra_take_fp32_bulk(lib, p):
    """Tetrahedra: their operator rows (sum |D_mn| of 40 to 170 at facet nodes
    of small volume weight) amplify the float32 rounding of the flux
    variations to 1.4e-5 (25 nodes) and 3.2e-5 (78 nodes, no dissipation) of
    the residual, above the bound; under precision "fp32" they take the
    FP32-bulk kernels, whose accuracy (<= 1e-11) this checks, on the
    Taylor-Green state with noise and on the plain low-Mach one."""
    R, Dg, rrk, OP = _oracle()
    op = tet_operator(p)
    m = periodic_tet_mesh(op, 3, 2 * np.pi, 0.0 if p == 1 else 0.02)
    for u in (states.add_uniform_noise(states.taylor_green(m), 1e-2, 5), states.taylor_green(m)):
        s = lib.Solver(op, m, lib.Params(dissipation=True, precision="fp32"))
        r = s.residual(s.to_device(u)).cpu().numpy()
        s.close()
        err = rel_err(r, R.residual(u, op, m, OP(), dissipation=True).numpy())
        print(f"fp32 setting, tets p={p} (FP32-bulk kernels): rel err {err:.2e}")
        assert err <= 1e-11


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_fp32_lines(lib, p):
    op = line_operator(p)
    m = periodic_line_mesh(op, 64, 1.0, amp=0.2)
    u = states.add_uniform_noise(states.uniform_state(m.n_e, 1, op.n_p), 1e-2, 4)
    _check(lib, op, m, u, True, f"1D p={p}")


@pytest.mark.parametrize("dim", [1, 2])
def test_fp32_free_stream_exact(lib, dim):
    """A uniform state has no variation: every float32 term is zero and so is
    the residual, exactly."""
    if dim == 1:
        op = line_operator(2)
        m = periodic_line_mesh(op, 16, 1.0, amp=0.2)
    else:
        op = tri_operator(3)
        m = periodic_tri_mesh(op, 6, 10.0, 0.05)
    u = states.uniform_state(m.n_e, dim, op.n_p)
    s = lib.Solver(op, m, lib.Params(dissipation=True, precision="fp32"))
    r = s.residual(s.to_device(u))
    assert float(r.abs().max()) == 0.0
    s.close()


def test_fp32_rrk_step(lib):
    """A relaxation RK4 step with float32 residuals (entropy, relaxation root
    and update in float64): g and the new state against the oracle's float64
    step, and the fused entropy production of the first stage against the
    oracle's w^T H r of the GPU's own float32 residual.  By Eq. (97) g
    balances the entropy change against the estimate dt sum b_i e_i; here the
    stage productions e_i are ~1e-5 of their scale sum H |w||r|, so the
    float32 residual's error (~3e-6 of r) moves them by ~5e-5 of themselves
    and g - 1 (~5e-6) by a comparable amount: g and the state (relative to the
    step's change, which carries g's error) are compared at G_BOUND = 5e-5
    (observed 2.6e-6 to 7.2e-6 over builds); the production itself against
    the oracle's w^T H r of the same residual to 1e-6 of its scale."""
    R, Dg, rrk, OP = _oracle()
    op = tri_operator(3)
    m = periodic_tri_mesh(op, 8, 10.0, 0.05)
    u0 = states.add_uniform_noise(states.isentropic_vortex(m), 1e-3, 2)
    dt = states.cfl_timestep(m, u0, 0.1)
    s = lib.Solver(op, m, lib.Params(dissipation=True, precision="fp32"))
    r0 = s.residual(s.to_device(u0)).cpu().numpy()
    ud = s.to_device(u0)
    g, info = s.rrk_step(ud, dt)
    uo, io = rrk.rrk4_step(torch.as_tensor(u0), dt, lambda x: R.residual(x, op, m, OP(), dissipation=True),
                           op, m, OP())
    rate0 = float(Dg.entropy_rate(u0, r0, op, m, OP()))
    scale0 = float(Dg.entropy_rate_scale(u0, r0, op, m, OP()))
    du = np.abs(ud.cpu().numpy() - u0).max()
    err_u = np.abs(ud.cpu().numpy() - uo.numpy()).max()
    print(f"fp32 RRK: g {g:.12f} (oracle {io.g:.12f}), state err {err_u:.2e} of a step change {du:.2e}, "
          f"stage-1 production {info.stage_rate[0]:.6e} vs {rate0:.6e} (scale {scale0:.2e})")
    G_BOUND = 5e-5
    assert abs(g - io.g) <= G_BOUND
    assert err_u <= G_BOUND * du
    assert abs(info.stage_rate[0] - rate0) <= 1e-6 * scale0
    s.close()
