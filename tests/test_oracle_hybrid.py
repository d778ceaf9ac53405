"""Pins of the oracle's troubled-element detector (oracle/hybrid.py)."""
import numpy as np
import pytest

from esplit_inputs import tri_operator, tet_operator, periodic_tri_mesh, states
from esplit_inputs.mesh import periodic_tet_mesh
from oracle.hybrid import detect, detector_pressure


def _loop_detect(u, op, m, threshold, gam=1.4):
    """Element-by-element restatement with plain Python loops."""
    n_e, nc, n_p = u.shape
    d = nc - 2

    def pres(e, k):
        rho = u[e, 0, k]
        s = 0.0
        for i in range(d):
            s = u[e, 1 + i, k] * u[e, 1 + i, k] if i == 0 else s + u[e, 1 + i, k] * u[e, 1 + i, k]
        return (gam - 1.0) * (u[e, d + 1, k] - (0.5 * s) / rho)

    fn = op.facet_nodes.reshape(-1)
    pair = m.pair.reshape(n_e, -1, 2)
    flag0 = np.zeros(n_e, dtype=bool)
    for e in range(n_e):
        ps = [pres(e, k) for k in range(n_p)]
        ps += [pres(int(pair[e, s, 0]), int(fn[pair[e, s, 1]])) for s in range(pair.shape[1])]
        if not all(0 < x < np.inf for x in ps):
            flag0[e] = True
        else:
            flag0[e] = not (max(ps) / min(ps) <= threshold)
    flags = flag0.copy()
    for e in range(n_e):
        for s in range(pair.shape[1]):
            flags[e] |= flag0[pair[e, s, 0]]
    return flags.astype(np.uint8)


def test_pressure_formula():
    u = states.random_positive_state(5, 2, 7, seed=1)
    rho, m1, m2, E = u[:, 0], u[:, 1], u[:, 2], u[:, 3]
    p_ref = 0.4 * (E - 0.5 * (m1 ** 2 + m2 ** 2) / rho)
    assert np.allclose(detector_pressure(u), p_ref, rtol=1e-14, atol=0)


@pytest.mark.parametrize("thr", [1.001, 1.1])
def test_detect_matches_loop_tri(thr):
    op = tri_operator(2)
    m = periodic_tri_mesh(op, 12, 1.0, 0.0)
    u = states.add_uniform_noise(states.quadrant_states(m, 5), 1e-3, 3)
    f = detect(u, op, m, thr)
    assert np.array_equal(f, _loop_detect(u, op, m, thr))
    assert 0 < f.sum() < m.n_e


def test_detect_matches_loop_tet():
    op = tet_operator(2)
    m = periodic_tet_mesh(op, 2, 2 * np.pi, 0.02)
    u = states.add_uniform_noise(states.taylor_green(m), 1e-2, 4)
    f = detect(u, op, m, 1.0005)
    assert np.array_equal(f, _loop_detect(u, op, m, 1.0005))


def test_smooth_and_uniform_states_flag_nothing():
    op = tri_operator(3)
    m = periodic_tri_mesh(op, 6, 10.0, 0.05)
    assert detect(states.uniform_state(m.n_e, 2, op.n_p), op, m).sum() == 0
    u = states.add_uniform_noise(states.uniform_state(m.n_e, 2, op.n_p), 1e-3, 6)
    assert detect(u, op, m, 1.1).sum() == 0
    assert detect(u, op, m, 1.0 + 1e-9).sum() == m.n_e


def test_single_jump_flags_its_neighbourhood():
    op = tri_operator(2)
    m = periodic_tri_mesh(op, 6, 1.0, 0.0)
    u = states.uniform_state(m.n_e, 2, op.n_p)
    k, node = 17, int(op.facet_nodes[0, 0])
    u[k, 3, node] *= 1.5                                 # raise the pressure at one facet node of element k
    f = detect(u, op, m, 1.1)
    pair = m.pair.reshape(m.n_e, -1, 2)
    nb = set(int(v) for v in pair[k, :, 0])
    # element k and the neighbour sharing that node see the jump; then one layer more
    seen = {k, int(pair[k, 0, 0])}
    expect = set(seen)
    for e in seen:
        expect |= set(int(v) for v in pair[e, :, 0])
    assert set(np.flatnonzero(f)) == expect
    assert nb <= expect


def test_nonpositive_pressure_flags():
    op = tri_operator(1)
    m = periodic_tri_mesh(op, 3, 1.0, 0.0)
    u = states.uniform_state(m.n_e, 2, op.n_p)
    u[4, 3, 2] = 0.5 * (u[4, 1, 2] ** 2 + u[4, 2, 2] ** 2) / u[4, 0, 2]   # p = 0 exactly
    f = detect(u, op, m, 1e9)
    assert f[4] == 1
