"""GPU hybrid scheme driven by the on-device troubled-element detector
(Sec. 4.4, Thm. 4), on the 2D Riemann-type quadrant problem: flags bit-exact
against the oracle's detector, element lists that reproduce the residual of
host-set flags, relaxation RK4 with re-detection before every step against
the oracle, and the full-size workload (256 x 256 quads -> 131,072
triangles, p = 2)."""
import numpy as np
import pytest
import torch

from esplit_inputs import tri_operator, periodic_tri_mesh, states

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2305_07181_gb300 as es
    return es


def _oracle():
    from oracle import residual as R, diagnostics as Dg, rrk, hybrid
    from oracle.physics import Params as OP
    return R, Dg, rrk, hybrid, OP


def rel_err(a, b):
    num = np.abs(np.asarray(a) - np.asarray(b)).max(axis=(0, 2))
    den = np.abs(np.asarray(b)).max(axis=(0, 2))
    return float((num / den).max())


def _quadrants(N, seed=5, noise=0.0):
    op = tri_operator(2)
    m = periodic_tri_mesh(op, N, 1.0, 0.0)
    u = states.quadrant_states(m, seed)
    if noise:
        u = states.add_uniform_noise(u, noise, seed + 1)
    return op, m, u


@pytest.mark.parametrize("N,thr,noise", [(16, 1.1, 0.0), (16, 1.001, 1e-3), (33, 1.1, 1e-3)])
def test_detector_flags_bit_exact(lib, N, thr, noise):
    R, Dg, rrk, hy, OP = _oracle()
    op, m, u = _quadrants(N, noise=noise)
    s = lib.Solver(op, m, lib.Params(scheme="hybrid", dissipation=True))
    n = s.detect_hybrid(s.to_device(u), thr)
    f = s.hybrid_flags()
    fo = hy.detect(u, op, m, thr)
    assert np.array_equal(f, fo)
    assert n == int(fo.sum()) and 0 < n < m.n_e
    s.close()


def test_detected_lists_reproduce_host_flags(lib):
    op, m, u = _quadrants(20, noise=1e-3)
    s = lib.Solver(op, m, lib.Params(scheme="hybrid", dissipation=True))
    ud = s.to_device(u)
    s.detect_hybrid(ud, 1.1)
    r_det = s.residual(ud).clone()
    s.set_hybrid_flags(s.hybrid_flags())
    r_host = s.residual(ud)
    assert torch.equal(r_det, r_host)
    s.close()


def test_detector_rejects_bad_threshold(lib):
    op, m, u = _quadrants(8)
    s = lib.Solver(op, m, lib.Params(scheme="hybrid"))
    with pytest.raises(lib.EsplitError) as ei:
        s.detect_hybrid(s.to_device(u), 0.5)
    assert ei.value.code == lib.capi.ESPLIT_ERR_ARG
    s.close()


def test_rrk_hybrid_redetect_parity(lib):
    """Ten relaxation RK4 steps on the quadrant problem (16 x 16 quads, p = 2,
    hybrid + matrix dissipation, CFL 0.1), re-detecting before each step on
    both sides: flags equal, g to 1e-10, stage entropy rates non-positive and
    equal to the oracle's, states to 1e-12."""
    R, Dg, rrk, hy, OP = _oracle()
    op, m, u0 = _quadrants(16)
    dt = states.cfl_timestep(m, u0, 0.1)
    s = lib.Solver(op, m, lib.Params(scheme="hybrid", dissipation=True))
    ud = s.to_device(u0)
    uo = torch.as_tensor(u0)
    for step in range(10):
        s.detect_hybrid(ud, 1.1)
        fo = hy.detect(uo.numpy(), op, m, 1.1)
        assert np.array_equal(s.hybrid_flags(), fo), step
        rhs = lambda x: R.residual(x, op, m, OP(), scheme="hybrid", dissipation=True, hybrid_flags=fo)
        g, info = s.rrk_step(ud, dt)
        uo, io = rrk.rrk4_step(uo, dt, rhs, op, m, OP())
        assert abs(g - io.g) <= 1e-10, (step, g, io.g)
        for e_gpu, e_or in zip(info.stage_rate, io.stage_production):
            assert e_gpu < 0 and e_or < 0
            assert abs(e_gpu - e_or) <= 1e-9 * abs(e_or)
    assert rel_err(ud.cpu().numpy(), uo.numpy()) <= 1e-12
    assert s.status() == 0
    s.close()


def test_full_size_quadrants(lib):
    """The full-size workload (256 x 256 quads -> 131,072 triangles, p = 2):
    flags bit-exact against the oracle detector, and the hybrid residual with
    those flags on 48 sampled elements (plus the first and last) against the
    oracle."""
    R, Dg, rrk, hy, OP = _oracle()
    op, m, u = _quadrants(256)
    s = lib.Solver(op, m, lib.Params(scheme="hybrid", dissipation=True))
    ud = s.to_device(u)
    n = s.detect_hybrid(ud, 1.1)
    f = s.hybrid_flags()
    fo = hy.detect(u, op, m, 1.1)
    assert np.array_equal(f, fo) and n == int(fo.sum())
    r = s.residual(ud).cpu().numpy()
    s.close()
    rng = np.random.default_rng(9)
    sample = np.concatenate([rng.choice(np.flatnonzero(fo), 24, replace=False),
                             rng.choice(np.flatnonzero(fo == 0), 24, replace=False), [0, m.n_e - 1]])
    ro = R.residual(u, op, m, OP(), scheme="hybrid", dissipation=True, hybrid_flags=fo, elems=sample).numpy()
    rs = r[sample]
    # piecewise-constant data: the residual is exactly zero away from the jumps;
    # compare on the max-norm of the sampled oracle residual
    assert np.abs(rs - ro).max() <= FP64_TOL * np.abs(ro).max()
