"""End-to-end accuracy against the paper's printed grid-convergence study
(Sec. 7.3, Table 1; fixture tests/golden/vortex2d_table1.txt): the 2D
isentropic vortex on the Sec. 7.3 curvilinear triangle grids, run with the GPU
residual and relaxation RK4 (CFL 0.1) to t_f = 2, L^2 error as Sec. 7.3
measures it (tests/accuracy.py).

The paper does not print its operators' node sets, so errors are compared
with a factor band rather than digits: for p = 3, 4 (whose node counts match
the diagonal-E family the paper cites) the errors lie within a factor 2 of
the printed ones and the 60 -> 80 rates within 0.5 of the printed rates; for
every p the rates lie in the band [p - 0.2, p + 1.2] the paper reports
(rates between p and p + 1) and dissipation lowers the error.  Meshes 60^2 x 2
and 80^2 x 2 (the smallest two of the table) keep the run to about two
minutes; over the full table (N = 60..120) the p = 3, 4 errors were
observed at 0.65-0.9 of the printed ones at every mesh."""
import os

import numpy as np
import pytest
import torch

from esplit_inputs import tri_operator, states
from esplit_inputs.mesh import periodic_tri_mesh_rect
from accuracy import l2_error_vortex

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "vortex2d_table1.txt")


def _table():
    rows = np.loadtxt(GOLDEN, comments="#")
    return {(int(r[0]), int(r[1])): {"split_ec": r[2], "split_diss": r[3]} for r in rows}


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2305_07181_gb300 as es
    return es


def _run(lib, op, m, diss, tf=2.0):
    u0 = states.isentropic_vortex(m, center=(5.0, 0.0))
    dt = states.cfl_timestep(m, u0, 0.1)
    s = lib.Solver(op, m, lib.Params(dissipation=diss))
    u = s.to_device(u0)
    t = 0.0
    while t < tf - 1e-12:
        h = min(dt, tf - t)
        g, _ = s.rrk_step(u, h)
        t += g * h
    err = l2_error_vortex(u.cpu().numpy(), op, m, t)
    assert s.status() == 0
    s.close()
    return err


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_vortex_convergence_against_table1(lib, p):
    tab = _table()
    op = tri_operator(p)
    errs = {}
    for N in (60, 80):
        m = periodic_tri_mesh_rect(op, N, N)
        for kind, diss in (("split_ec", False), ("split_diss", True)):
            errs[(N, kind)] = _run(lib, op, m, diss)
    for kind in ("split_ec", "split_diss"):
        ours = [errs[(60, kind)], errs[(80, kind)]]
        paper = [tab[(p, 60)][kind], tab[(p, 80)][kind]]
        rate = np.log(ours[0] / ours[1]) / np.log(80 / 60)
        prate = np.log(paper[0] / paper[1]) / np.log(80 / 60)
        print(f"p={p} {kind}: ours {ours[0]:.3e} {ours[1]:.3e} rate {rate:.2f} | Table 1 {paper[0]:.3e} "
              f"{paper[1]:.3e} rate {prate:.2f}")
        assert p - 0.2 <= rate <= p + 1.2
        if p >= 3:
            for a, b in zip(ours, paper):
                assert 0.5 <= a / b <= 2.0
            assert abs(rate - prate) <= 0.5
    for N in (60, 80):
        assert errs[(N, "split_diss")] < errs[(N, "split_ec")]


GOLDEN3D = os.path.join(os.path.dirname(__file__), "golden", "vortex3d_table2.txt")


def test_vortex3d_p2_against_table2(lib):
    """The 3D vortex of Sec. 7.3 with the p = 2 tetrahedron operator (25
    nodes), GPU residual + relaxation RK4 at CFL 0.25 to t_f = 1, on the
    15^3 x 6 and 20^3 x 6 grids (Table 2's two smallest): errors within a
    factor 2 of the printed ones, rate in [p - 0.2, p + 1.2], dissipation
    lowers the error.  (Observed over 15..30: errors 1.3-1.6 times the
    printed ones, rates 2.3-2.6 against 2.5-2.8; the node sets differ.)"""
    from esplit_inputs import tet_operator
    from esplit_inputs.mesh import periodic_tet_mesh, vortex3d_warp
    from accuracy import l2_error_vortex_3d
    rows = np.loadtxt(GOLDEN3D, comments="#")
    tab = {(int(r[0]), int(r[1])): {"split_ec": r[2], "split_diss": r[3]} for r in rows}
    op = tet_operator(2)
    errs = {}
    for N in (15, 20):
        m = periodic_tet_mesh(op, N, 20.0, origin=-10.0, warp=vortex3d_warp)
        u0 = states.isentropic_vortex_3d(m)
        dt = states.cfl_timestep(m, u0, 0.25)
        for kind, diss in (("split_ec", False), ("split_diss", True)):
            s = lib.Solver(op, m, lib.Params(dissipation=diss))
            u = s.to_device(u0)
            t = 0.0
            while t < 1.0 - 1e-12:
                h = min(dt, 1.0 - t)
                g, _ = s.rrk_step(u, h)
                t += g * h
            errs[(N, kind)] = l2_error_vortex_3d(u.cpu().numpy(), op, m, t)
            assert s.status() == 0
            s.close()
    for kind in ("split_ec", "split_diss"):
        ours = [errs[(15, kind)], errs[(20, kind)]]
        paper = [tab[(2, 15)][kind], tab[(2, 20)][kind]]
        rate = np.log(ours[0] / ours[1]) / np.log(20 / 15)
        print(f"3D p=2 {kind}: ours {ours[0]:.3e} {ours[1]:.3e} rate {rate:.2f} | Table 2 {paper[0]:.3e} "
              f"{paper[1]:.3e}")
        assert 1.8 <= rate <= 3.2
        for a, b in zip(ours, paper):
            assert 0.5 <= a / b <= 2.0
    for N in (15, 20):
        assert errs[(N, "split_diss")] < errs[(N, "split_ec")]


def _run_rk4(lib, op, m, params, tf=2.0):
    """Classical RK4 at CFL 0.1 with the GPU residual (the stage combinations
    are torch arithmetic of this test: the library's relaxation step uses
    Harten's entropy, which the Ismail-Roe scheme does not conserve)."""
    u0 = states.isentropic_vortex(m, center=(5.0, 0.0))
    dt = states.cfl_timestep(m, u0, 0.1)
    s = lib.Solver(op, m, params)
    u = s.to_device(u0)
    t = 0.0
    while t < tf - 1e-12:
        h = min(dt, tf - t)
        k1 = s.residual(u)
        k2 = s.residual(u + 0.5 * h * k1)
        k3 = s.residual(u + 0.5 * h * k2)
        k4 = s.residual(u + h * k3)
        u = u + (h / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
        t += h
    err = l2_error_vortex(u.cpu().numpy(), op, m, t)
    assert s.status() == 0
    s.close()
    return err


@pytest.mark.parametrize("p", [3, 4])
def test_vortex_ismail_roe_against_table1(lib, p):
    """The Sec. 6 comparator (Ismail-Roe Hadamard form, conservative and with
    its matrix dissipation) on the same grids against Table 1's Ismail-Roe
    columns: errors within a factor 2 of the printed ones, rates in
    [p - 0.2, p + 1.2], dissipation lowers the error; and the entropy-split
    errors of the same runs (test above) are of the same size, which is the
    'equal accuracy' the throughput comparison assumes."""
    rows = np.loadtxt(GOLDEN, comments="#")
    tab = {(int(r[0]), int(r[1])): {"ir_ec": r[4], "ir_diss": r[5]} for r in rows}
    op = tri_operator(p)
    errs = {}
    for N in (60, 80):
        m = periodic_tri_mesh_rect(op, N, N)
        for kind, diss in (("ir_ec", False), ("ir_diss", True)):
            errs[(N, kind)] = _run_rk4(lib, op, m, lib.Params(scheme="hadamard_ir", dissipation=diss))
        errs[(N, "split_diss")] = _run_rk4(lib, op, m, lib.Params(dissipation=True))
    for kind in ("ir_ec", "ir_diss"):
        ours = [errs[(60, kind)], errs[(80, kind)]]
        paper = [tab[(p, 60)][kind], tab[(p, 80)][kind]]
        rate = np.log(ours[0] / ours[1]) / np.log(80 / 60)
        print(f"p={p} {kind}: ours {ours[0]:.3e} {ours[1]:.3e} rate {rate:.2f} | Table 1 {paper[0]:.3e} "
              f"{paper[1]:.3e}")
        assert p - 0.2 <= rate <= p + 1.2
        for a, b in zip(ours, paper):
            assert 0.5 <= a / b <= 2.0
    for N in (60, 80):
        print(f"p={p} N={N}: split+diss (RK4) {errs[(N, 'split_diss')]:.3e} vs IR+diss {errs[(N, 'ir_diss')]:.3e}")
        assert errs[(N, "ir_diss")] < errs[(N, "ir_ec")]
        assert 0.5 <= errs[(N, "split_diss")] / errs[(N, "ir_diss")] <= 2.0


def _run_3d(lib, op, m, params, rrk=True, tf=1.0):
    """The 3D vortex at CFL 0.25 to t_f: relaxation RK4 through the library
    for the entropy-split scheme, classical RK4 (torch stage combinations)
    for the Ismail-Roe comparator, whose entropy is not Harten's.  Returns
    the final state and time."""
    u0 = states.isentropic_vortex_3d(m)
    dt = states.cfl_timestep(m, u0, 0.25)
    s = lib.Solver(op, m, params)
    u = s.to_device(u0)
    t = 0.0
    while t < tf - 1e-12:
        h = min(dt, tf - t)
        if rrk:
            g, _ = s.rrk_step(u, h)
            t += g * h
        else:
            k1 = s.residual(u)
            k2 = s.residual(u + 0.5 * h * k1)
            k3 = s.residual(u + 0.5 * h * k2)
            k4 = s.residual(u + h * k3)
            u = u + (h / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
            t += h
    assert s.status() == 0
    s.close()
    return u.cpu().numpy(), t


def _errors_3d(op, m, runs):
    """L^2 errors of several (u, t) runs, one geometry pass per final time."""
    from accuracy import l2_error_vortex_3d
    out = [None] * len(runs)
    for t in sorted(set(t for _, t in runs)):
        idx = [i for i, (_, ti) in enumerate(runs) if ti == t]
        errs = l2_error_vortex_3d([runs[i][0] for i in idx], op, m, t)
        for i, e in zip(idx, errs):
            out[i] = e
    return out


# p = 4 takes about ten minutes (1,251 relaxation steps on 48,000 elements
# with 78 nodes, four schemes, two grids); it runs with ESPLIT_LONG_TESTS=1
_DEGREES = [1, 3] + ([4] if os.environ.get("ESPLIT_LONG_TESTS") == "1" else [])


@pytest.mark.parametrize("p", _DEGREES)
def test_vortex3d_degrees_against_table2(lib, p):
    """The 3D vortex of Sec. 7.3 with the degree 1, 3 and 4 tetrahedron
    operators on the 15^3 x 6 and 20^3 x 6 grids, all four columns of Table 2
    (entropy split and Ismail-Roe Hadamard form, each conservative and with
    its matrix dissipation): errors within a factor 2 of the printed ones,
    rates in [p - 0.2, p + 1.2], and the split and Ismail-Roe errors within a
    factor 2 of each other (the equal accuracy the throughput comparison on
    these grids assumes).  Observed: p = 3 within 0.97-1.08 of every printed
    error (rates 3.24-3.34 against 3.22-3.45), p = 4 within 1.07-1.20 (rates
    4.02-4.34 against 3.94-4.27), p = 1 (affine elements) 1.2-1.5 times the
    printed errors."""
    from esplit_inputs import tet_operator
    from esplit_inputs.mesh import periodic_tet_mesh, vortex3d_warp
    rows = np.loadtxt(GOLDEN3D, comments="#")
    cols = ("split_ec", "split_diss", "ir_ec", "ir_diss")
    tab = {(int(r[0]), int(r[1])): dict(zip(cols, r[2:])) for r in rows}
    op = tet_operator(p)
    errs = {}
    for N in (15, 20):
        m = periodic_tet_mesh(op, N, 20.0, origin=-10.0, warp=vortex3d_warp)
        runs = [_run_3d(lib, op, m, lib.Params(dissipation=False)),
                _run_3d(lib, op, m, lib.Params(dissipation=True)),
                _run_3d(lib, op, m, lib.Params(scheme="hadamard_ir", dissipation=False), rrk=False),
                _run_3d(lib, op, m, lib.Params(scheme="hadamard_ir", dissipation=True), rrk=False)]
        for kind, e in zip(cols, _errors_3d(op, m, runs)):
            errs[(N, kind)] = e
    for kind in cols:
        ours = [errs[(15, kind)], errs[(20, kind)]]
        paper = [tab[(p, 15)][kind], tab[(p, 20)][kind]]
        rate = np.log(ours[0] / ours[1]) / np.log(20 / 15)
        prate = np.log(paper[0] / paper[1]) / np.log(20 / 15)
        print(f"3D p={p} {kind}: ours {ours[0]:.3e} {ours[1]:.3e} rate {rate:.2f} | Table 2 {paper[0]:.3e} "
              f"{paper[1]:.3e} rate {prate:.2f}")
    for kind in cols:
        ours = [errs[(15, kind)], errs[(20, kind)]]
        paper = [tab[(p, 15)][kind], tab[(p, 20)][kind]]
        rate = np.log(ours[0] / ours[1]) / np.log(20 / 15)
        assert p - 0.2 <= rate <= p + 1.2
        for a, b in zip(ours, paper):
            assert 0.5 <= a / b <= 2.0
    for N in (15, 20):
        assert 0.5 <= errs[(N, "split_diss")] / errs[(N, "ir_diss")] <= 2.0
