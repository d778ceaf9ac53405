"""Batches of relaxation RK4 steps launched as a recorded CUDA graph per step
(esplit_rrk_steps): the same launches as esplit_rrk_step in the same order, so
states and relaxation parameters must equal those of single steps exactly,
for every scheme and precision, across re-recordings (new dt, new
parameters, new state pointer) and on a failing step."""
import numpy as np
import pytest
import torch

from esplit_inputs import tri_operator, tet_operator, periodic_tri_mesh, states
from esplit_inputs.mesh import periodic_tet_mesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2305_07181_gb300 as es
    return es


def _tri(p=2, N=8):
    op = tri_operator(p)
    m = periodic_tri_mesh(op, N, 10.0, 0.05)
    u0 = states.add_uniform_noise(states.isentropic_vortex(m), 1e-3, 11)
    return op, m, u0, states.cfl_timestep(m, u0, 0.1)


def _single(s, u, dt, n):
    gs = []
    for _ in range(n):
        g, _ = s.rrk_step(u, dt)
        gs.append(g)
    return gs


def _compare(lib, op, m, u0, dt, params, n=12, flags=None):
    a = lib.Solver(op, m, params)
    b = lib.Solver(op, m, params)
    if flags is not None:
        a.set_hybrid_flags(flags)
        b.set_hybrid_flags(flags)
    ua, ub = a.to_device(u0), b.to_device(u0)
    g_single = _single(a, ua, dt, n)
    # two batches: the first records the graph after one ordinary step, the
    # second reuses the recording
    g1, info1 = b.rrk_steps(ub, dt, 5)
    g2, info2 = b.rrk_steps(ub, dt, n - 5)
    assert torch.equal(ua, ub)
    assert g1 + g2 == g_single
    assert info2.g == g_single[-1] and info2.status == 0 and info2.iterations >= 1
    a.close()
    b.close()


def test_steps_match_single_steps_split(lib):
    op, m, u0, dt = _tri()
    _compare(lib, op, m, u0, dt, lib.Params(dissipation=True))
    _compare(lib, op, m, u0, dt, lib.Params(dissipation=False))


def test_steps_match_single_steps_schemes_and_precision(lib):
    op, m, u0, dt = _tri(p=3, N=6)
    _compare(lib, op, m, u0, dt, lib.Params(dissipation=True, scheme="hadamard"), n=8)
    _compare(lib, op, m, u0, dt, lib.Params(dissipation=True, precision="fp32_bulk"), n=8)
    flags = np.zeros(m.n_e, dtype=np.uint8)
    flags[::5] = 1
    _compare(lib, op, m, u0, dt, lib.Params(dissipation=True, scheme="hybrid"), n=8, flags=flags)


def test_steps_match_single_steps_viscous_3d(lib):
    op = tet_operator(2)
    m = periodic_tet_mesh(op, 2, 2 * np.pi, 0.02)
    u0 = states.add_uniform_noise(states.taylor_green(m), 1e-3, 3)
    dt = states.cfl_timestep(m, u0, 0.1)
    _compare(lib, op, m, u0, dt, lib.Params(mu=0.05, viscous=True, dissipation=True), n=6)


def test_rerecording_on_new_dt_params_and_pointer(lib):
    op, m, u0, dt = _tri()
    a = lib.Solver(op, m, lib.Params(dissipation=True))
    b = lib.Solver(op, m, lib.Params(dissipation=True))
    ua, ub = a.to_device(u0), b.to_device(u0)
    ref = _single(a, ua, dt, 3) + _single(a, ua, 0.5 * dt, 3)
    a.set_params(lib.Params(dissipation=False))
    ref += _single(a, ua, 0.5 * dt, 3)
    got = b.rrk_steps(ub, dt, 3)[0] + b.rrk_steps(ub, 0.5 * dt, 3)[0]
    b.set_params(lib.Params(dissipation=False))
    got += b.rrk_steps(ub, 0.5 * dt, 3)[0]
    # a different state buffer (the recording holds the pointer)
    uc = ub.clone()
    ref += _single(a, ua, 0.5 * dt, 2)
    got += b.rrk_steps(uc, 0.5 * dt, 2)[0]
    assert got == ref
    assert torch.equal(ua, uc)
    # n_steps = 0 does nothing
    assert b.rrk_steps(uc, dt, 0)[0] == []
    assert torch.equal(ua, uc)
    a.close()
    b.close()


def test_steps_on_a_side_stream(lib):
    op, m, u0, dt = _tri()
    a = lib.Solver(op, m, lib.Params(dissipation=True))
    b = lib.Solver(op, m, lib.Params(dissipation=True))
    ua, ub = a.to_device(u0), b.to_device(u0)
    ref = _single(a, ua, dt, 6)
    st = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(st):
        got = b.rrk_steps(ub, dt, 6, stream=st)[0]
    st.synchronize()
    assert got == ref and torch.equal(ua, ub)
    a.close()
    b.close()


def test_failing_step_leaves_last_good_state(lib):
    """A step size far above the stable one drives the state out of the
    admissible set after a few steps.  Single steps find the first failing
    step k >= 2 (the first step of a batch runs the ordinary way, the later
    ones as graph launches); a batch from the same state must stop there with
    k - 1 completed steps and u equal to the state after them."""
    op, m, u0, dt0 = _tri(p=2, N=4)
    seen = []
    for mult in (15.0, 20.0, 25.0, 30.0, 40.0):
        dt = mult * dt0
        a = lib.Solver(op, m, lib.Params(dissipation=True))
        ua = a.to_device(u0)
        snaps, k_fail = [ua.clone()], None
        for k in range(1, 9):
            try:
                a.rrk_step(ua, dt)
            except lib.EsplitError:
                k_fail = k
                break
            snaps.append(ua.clone())
        a.close()
        seen.append((mult, k_fail))
        if k_fail is not None and k_fail >= 2:
            break
    else:
        pytest.skip(f"no step size in the list fails at step 2..8: {seen}")
    b = lib.Solver(op, m, lib.Params(dissipation=True))
    ub = b.to_device(u0)
    with pytest.raises(lib.EsplitError) as ei:
        b.rrk_steps(ub, dt, k_fail + 3)
    assert ei.value.n_done == k_fail - 1
    assert len(ei.value.g) == k_fail - 1
    assert torch.equal(ub, snaps[k_fail - 1])
    # the context stays usable: a fresh state steps normally
    ub2 = b.to_device(u0)
    g, info = b.rrk_steps(ub2, dt0, 2)
    assert len(g) == 2 and info.status == 0
    b.close()


def test_launch_count_and_timing_small_mesh(lib):
    """128 triangles (8 x 8 quads), p = 2: the batch launches the same kernels
    per step, with one graph launch instead of ~19 kernel launches and no
    host round trip per step."""
    op, m, u0, dt = _tri(p=2, N=8)
    s = lib.Solver(op, m, lib.Params(dissipation=True))
    u = s.to_device(u0)
    s.rrk_steps(u, dt, 2)
    n0 = s.launch_count()
    s.rrk_steps(u, dt, 10)
    per_step = (s.launch_count() - n0) / 10
    assert 10 <= per_step <= 40
    s.close()


def _assembled_step(s, u, dt, g):
    """u_n + g d with d = dt sum_i b_i r_i from four separate residual calls
    and torch arithmetic (the relaxation parameter g taken from the library's
    own step)."""
    A, B = (0.0, 0.5, 0.5, 1.0), (1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0)
    d = torch.zeros_like(u)
    r = None
    for i in range(4):
        Ui = u if i == 0 else u + (A[i] * dt) * r
        r = s.residual(Ui)
        d += (B[i] * dt) * r
    return u + g * d


@pytest.mark.parametrize("case", ["split_fp64", "split_fp32_bulk", "split_fp32", "hybrid_fp64", "split_tet_fp32"])
def test_step_stage_updates_match_separate_residuals(lib, case):
    """The relaxation step (its stage states, the combination d of the four
    stage residuals and the update u_n + g d, all on the device) equals
    u_n + g d assembled from four esplit_residual calls and torch arithmetic, to the
    rounding of the stage sums: 1e-13 of the state's scale, component-wise.
    The float32 path takes 1e-9: torch forms the stage states U_i with a
    rounding of its own, and a last-bit change of U_i can flip the float32
    rounding of a deviation (one float32 ulp, 6e-8, of dU/dt there), which a
    step (dt |dU/dt| ~ 6e-3 of |u| here) carries to ~4e-10 of the state."""
    if case == "split_tet_fp32":
        op = tet_operator(1)
        m = periodic_tet_mesh(op, 3)
        u0 = states.add_uniform_noise(states.taylor_green(m), 1e-3, 5)
        dt = states.cfl_timestep(m, u0, 0.1)
    else:
        op, m, u0, dt = _tri(p=3, N=6)
    prec = {"split_fp64": "fp64", "split_fp32_bulk": "fp32_bulk", "split_fp32": "fp32", "hybrid_fp64": "fp64",
            "split_tet_fp32": "fp32"}[case]
    scheme = "hybrid" if case.startswith("hybrid") else "split"
    s = lib.Solver(op, m, lib.Params(scheme=scheme, dissipation=True, precision=prec))
    if scheme == "hybrid":
        s.set_hybrid_flags(np.random.default_rng(3).integers(0, 2, m.n_e).astype(np.uint8))
    u = s.to_device(u0)
    ref_in = u.clone()
    g, info = s.rrk_step(u, dt)
    assert info.status == 0
    ref = _assembled_step(s, ref_in, dt, g)
    scale = ref.abs().amax(dim=(0, 2))
    err = ((u - ref).abs().amax(dim=(0, 2)) / scale).max().item()
    print(f"{case}: step vs assembled stages, rel err {err:.2e}")
    assert err <= (1e-9 if prec == "fp32" and op.d == 2 else 1e-13)
    s.close()
