"""Navier-Stokes accuracy against the paper's printed grid-convergence study
of the manufactured solution (Sec. 7.4, Table 4; fixture
tests/golden/nse_mms_table4.txt): the GPU residual (entropy split, EC SATs,
BO viscous SATs with the heat flux, no interface dissipation, mu = 0.01,
Pr = 0.71, R = 1) plus the manufactured source term (tests/mms.py, pinned by
differences in test_mms_source.py), classical RK4 to t_f = 0.001, L^2 error
as Sec. 7.3 measures it.

The paper takes 1000 steps; 100 are taken here (dt = 1e-5: the RK4 error,
~dt^4, is far below the spatial one).  The RK4 stage combinations are plain
torch arithmetic of this test (the relaxation step of the library has no
source term; the source is not part of the method).

3D (p = 2 tetrahedra, 6^3 x 6 .. 12^3 x 6): the errors are within 15 % of
the printed ones (observed 1.07 times them on every grid) and the rates near
3 (printed 2.81, 2.90).  2D: the rates are near p + 1 as printed; the printed
errors themselves are not matched, and cannot be by any degree-p scheme: the
best L^2 approximation of the initial state by degree-p polynomials on these
grids is already 2 to 10 times the printed error at t_f (the factor growing
with p), and the discrete H-norm
at the nodes does not match them either (they behave like ours on grids twice
as fine, divided by about two); Section 7.4 does not restate its 2D setup
beyond the formulas used here, so the 2D magnitudes are printed, not
asserted.  At p = 4 the 30 -> 40 rate drops (4.45 observed, 4.83 printed):
the scheme's own error over the run (the nodal H-norm, zero at t = 0, falls
at rate ~2.7) overtakes the projection error on the finest grid."""
import os

import numpy as np
import pytest
import torch

from esplit_inputs import tri_operator, tet_operator, states
from esplit_inputs.mesh import periodic_tri_mesh_rect, periodic_tet_mesh, mms_warp_2d, mms_warp_3d
from accuracy import l2_error_2d, l2_error_3d
from mms import mms_source_nodes

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "nse_mms_table4.txt")
TF, STEPS = 1e-3, 100


def _table():
    rows = np.loadtxt(GOLDEN, comments="#")
    return {(int(r[0]), int(r[1]), int(r[2])): r[3] for r in rows}


def _table_ir():
    rows = np.loadtxt(GOLDEN, comments="#")
    return {(int(r[0]), int(r[1]), int(r[2])): r[4] for r in rows}


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2305_07181_gb300 as es
    return es


def _run(lib, op, m, scheme="split"):
    s = lib.Solver(op, m, lib.Params(viscous=True, mu=0.01, Pr=0.71, R=1.0, heat_flux=True, dissipation=False,
                                     scheme=scheme))
    u = s.to_device(states.manufactured_state(m, 0.0))
    dt = TF / STEPS

    def rhs(x, t):
        return s.residual(x) + s.to_device(mms_source_nodes(m, t))

    for n in range(STEPS):
        t = n * dt
        k1 = rhs(u, t)
        k2 = rhs(u + 0.5 * dt * k1, t + 0.5 * dt)
        k3 = rhs(u + 0.5 * dt * k2, t + 0.5 * dt)
        k4 = rhs(u + dt * k3, t + dt)
        u = u + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    assert s.status() == 0
    s.close()
    return u.cpu().numpy()


def _nodal_error(u, op, m):
    """sqrt(sum_k sum_m H_k,m |u - u_exact|^2) at the nodes: zero at t = 0,
    so it measures what the scheme adds over the run."""
    ue = states.manufactured_state(m, TF)
    Hn = op.H[None] * m.J
    return float(np.sqrt((Hn[:, None, :] * (u - ue) ** 2).sum()))


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_mms_2d_against_table4(lib, p):
    tab = _table()
    op = tri_operator(p)
    Ns = (20, 30, 40)
    errs = []
    nod = []
    for N in Ns:
        m = periodic_tri_mesh_rect(op, N, N, origin=(-1.0, -1.0), size=(2.0, 2.0), warp=mms_warp_2d)
        u = _run(lib, op, m)
        errs.append(l2_error_2d(u, op, m, lambda X: states.manufactured_prims(X, TF)))
        nod.append(_nodal_error(u, op, m))
    print(f"2D p={p} nodal H-norm: " + " ".join(f"{e:.4e}" for e in nod) + " rates "
          + " ".join(f"{np.log(nod[i] / nod[i + 1]) / np.log(Ns[i + 1] / Ns[i]):.2f}" for i in range(2)))
    paper = [tab[(2, p, N)] for N in Ns]
    rates = [np.log(errs[i] / errs[i + 1]) / np.log(Ns[i + 1] / Ns[i]) for i in range(2)]
    prates = [np.log(paper[i] / paper[i + 1]) / np.log(Ns[i + 1] / Ns[i]) for i in range(2)]
    print(f"2D p={p}: ours " + " ".join(f"{e:.4e}" for e in errs) + " rates " + " ".join(f"{r:.2f}" for r in rates)
          + " | Table 4 " + " ".join(f"{e:.4e}" for e in paper) + " rates " + " ".join(f"{r:.2f}" for r in prates)
          + " | ratio " + " ".join(f"{a / b:.2f}" for a, b in zip(errs, paper)))
    for r in rates:
        assert p + 0.3 <= r <= p + 1.6


def test_mms_3d_p2_against_table4(lib):
    tab = _table()
    op = tet_operator(2)
    Ns = (6, 9, 12)
    errs = []
    nod = []
    for N in Ns:
        m = periodic_tet_mesh(op, N, 2.0, origin=-1.0, warp=mms_warp_3d)
        u = _run(lib, op, m)
        errs.append(l2_error_3d(u, op, m, lambda X: states.manufactured_prims(X, TF)))
        nod.append(_nodal_error(u, op, m))
    print(f"3D p=2 nodal H-norm: " + " ".join(f"{e:.4e}" for e in nod) + " rates "
          + " ".join(f"{np.log(nod[i] / nod[i + 1]) / np.log(Ns[i + 1] / Ns[i]):.2f}" for i in range(2)))
    paper = [tab[(3, 2, N)] for N in Ns]
    rates = [np.log(errs[i] / errs[i + 1]) / np.log(Ns[i + 1] / Ns[i]) for i in range(2)]
    print(f"3D p=2: ours " + " ".join(f"{e:.4e}" for e in errs) + " rates " + " ".join(f"{r:.2f}" for r in rates)
          + " | Table 4 " + " ".join(f"{e:.4e}" for e in paper)
          + " | ratio " + " ".join(f"{a / b:.2f}" for a, b in zip(errs, paper)))
    for r in rates:
        assert 2.5 <= r <= 3.5
    for a, b in zip(errs, paper):
        assert 0.85 <= a / b <= 1.15


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_mms_3d_degrees_both_schemes(lib, p):
    """3D, every tetrahedron degree (p = 1 on affine elements), both columns
    of Table 4: the entropy-split scheme and the Ismail-Roe comparator (BO
    terms in the standard entropy variables), 6^3 x 6 .. 12^3 x 6 grids.
    Rates near p + 1 (band [p + 0.3, p + 1.6]); the two schemes' errors
    within 5 % of each other, as in the table; errors within 20 % of the
    printed ones (observed 0.88-1.07 for the split scheme and 0.94-1.07 for
    the comparator over p = 1..4; the node sets differ from the paper's)."""
    tab, tab_ir = _table(), _table_ir()
    op = tet_operator(p)
    Ns = (6, 9, 12)
    errs = {"split": [], "hadamard_ir": []}
    for N in Ns:
        m = periodic_tet_mesh(op, N, 2.0, origin=-1.0, warp=mms_warp_3d)
        for scheme in errs:
            u = _run(lib, op, m, scheme)
            errs[scheme].append(l2_error_3d(u, op, m, lambda X: states.manufactured_prims(X, TF)))
    for scheme, t in (("split", tab), ("hadamard_ir", tab_ir)):
        e = errs[scheme]
        paper = [t[(3, p, N)] for N in Ns]
        rates = [np.log(e[i] / e[i + 1]) / np.log(Ns[i + 1] / Ns[i]) for i in range(2)]
        prates = [np.log(paper[i] / paper[i + 1]) / np.log(Ns[i + 1] / Ns[i]) for i in range(2)]
        print(f"3D p={p} {scheme}: ours " + " ".join(f"{x:.4e}" for x in e) + " rates "
              + " ".join(f"{r:.2f}" for r in rates) + " | Table 4 " + " ".join(f"{x:.4e}" for x in paper)
              + " rates " + " ".join(f"{r:.2f}" for r in prates)
              + " | ratio " + " ".join(f"{a / b:.2f}" for a, b in zip(e, paper)))
    for scheme, t in (("split", tab), ("hadamard_ir", tab_ir)):
        e = errs[scheme]
        for i in range(2):
            assert p + 0.3 <= np.log(e[i] / e[i + 1]) / np.log(Ns[i + 1] / Ns[i]) <= p + 1.6
        for a, N in zip(e, Ns):
            assert 0.8 <= a / t[(3, p, N)] <= 1.2
    for a, b in zip(errs["split"], errs["hadamard_ir"]):
        assert 0.95 <= a / b <= 1.05
