"""Pins of oracle/residual.py against the paper's exact results (Secs. 4-6)."""
import numpy as np
import pytest
import torch

from esplit_inputs import tri_operator, periodic_tri_mesh, states
from oracle import residual as R, diagnostics as Dg
from oracle.physics import (Params, euler_flux, entropy_variables, sy_flux,
                            symmetrized_flux_jacobians)
from oracle.operators import physical_operators

P = Params()
PS = [1, 2, 3, 4]


def setup(p, N=3, amp=0.05, seed=None):
    op = tri_operator(p)
    m = periodic_tri_mesh(op, N, 10.0, amp)
    u = states.random_positive_state(m.n_e, 2, op.n_p, seed=100 + p if seed is None else seed)
    return op, m, u


@pytest.mark.parametrize("p", PS)
@pytest.mark.parametrize("scheme", ["split", "hadamard"])
def test_weak_equals_strong(p, scheme):
    """Eq. (100) vs Eqs. (42)-(43); Eq. (99) vs Eq. (67) (algebraic equivalence, Sec. 6.2)."""
    op, m, u = setup(p)
    rw = R.residual(u, op, m, P, scheme=scheme, form="weak")
    rs = R.residual(u, op, m, P, scheme=scheme, form="strong")
    assert (rw - rs).abs().max() < 1e-13 * rw.abs().max()


@pytest.mark.parametrize("p", PS)
def test_freestream(p):
    op, m, _ = setup(p)
    u = states.uniform_state(m.n_e, 2, op.n_p)
    for scheme in ["split", "hadamard"]:
        r = R.residual(u, op, m, Params(mu=0.01), scheme=scheme, dissipation=True, viscous=True)
        # flux magnitudes are O(1), operator entries O(1/h)
        assert r.abs().max() < 1e-12


@pytest.mark.parametrize("p", PS)
@pytest.mark.parametrize("scheme", ["split", "hadamard", "hybrid"])
def test_entropy_conservation(p, scheme):
    """Thms. 2 and 4: sum_k w_k^T H_k du_k/dt = 0 for any state on a curved periodic mesh."""
    op, m, u = setup(p)
    flags = np.random.default_rng(p).integers(0, 2, m.n_e)
    r = R.residual(u, op, m, P, scheme=scheme, hybrid_flags=flags)
    rate = Dg.entropy_rate(u, r, op, m, P)
    scale = Dg.entropy_rate_scale(u, r, op, m, P)
    assert abs(float(rate)) < 1e-14 * float(scale)


@pytest.mark.parametrize("p", [1, 2, 4])
def test_dissipation_rate(p):
    """Eq. (69): the entropy rate of the dissipative scheme equals
    -1/2 sum over facet nodes of |nu| dw^T X|L|SX^T dw / 2 (each pair seen from
    both sides) and is negative."""
    op, m, u = setup(p)
    r0 = R.residual(u, op, m, P, scheme="split")
    r1 = R.residual(u, op, m, P, scheme="split", dissipation=True)
    rate = float(Dg.entropy_rate(u, r1 - r0, op, m, P))
    U = torch.as_tensor(u).transpose(1, 2)
    fn = op.facet_nodes.reshape(-1)
    pr = m.pair.reshape(m.n_e, -1, 2)
    Uk = U[:, fn]
    Uv = U[pr[..., 0], fn[pr[..., 1]]]
    nu = torch.as_tensor(m.nu.reshape(m.n_e, -1, 2))
    b = torch.linalg.norm(nu, dim=-1)
    from oracle.physics import dissipation_matrix
    Dm = dissipation_matrix(Uk, Uv, nu / b[..., None], P)
    dw = entropy_variables(Uk, P) - entropy_variables(Uv, P)
    closed = float(-0.5 * (0.5 * b * torch.einsum("esc,escd,esd->es", dw, Dm, dw)).sum())
    assert closed < 0
    assert abs(rate - closed) < 1e-12 * abs(closed)


@pytest.mark.parametrize("p", PS)
def test_hadamard_conservation(p):
    """Local (hence global) conservation of the Hadamard form (Thm. 4 proof)."""
    op, m, u = setup(p)
    r = R.residual(u, op, m, P, scheme="hadamard", dissipation=True)
    c = Dg.conservation(r, op, m)
    scale = float((torch.as_tensor(op.H)[None, :, None] * torch.as_tensor(m.J)[..., None]
                   * r.transpose(1, 2).abs()).sum())
    assert c.abs().max() < 1e-14 * scale


def test_split_conservation_error_converges():
    """Thm. 3: sum_k I^T H_k du_k/dt = O(h^(p+1)) for smooth solutions."""
    errs = []
    for N in [6, 12, 24]:
        op = tri_operator(2)
        m = periodic_tri_mesh(op, N, 10.0, 0.05)
        u = states.isentropic_vortex(m)
        r = R.residual(u, op, m, P, scheme="split")
        errs.append(float(Dg.conservation(r, op, m).abs().max()))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 2.5), rates


def test_split_accuracy():
    """Thm. 1 / Lemma 7: du/dt of the exact vortex approaches -div F, order ~p."""
    errs = []
    for N in [16, 32]:
        op = tri_operator(2)
        m = periodic_tri_mesh(op, N, 10.0, 0.05)
        u = states.isentropic_vortex(m)
        h = 1e-5
        dudt = (states.isentropic_vortex(m, t=h) - states.isentropic_vortex(m, t=-h)) / (2 * h)
        r = R.residual(u, op, m, P, scheme="split").numpy()
        errs.append(np.abs(r - dudt).max())
    assert np.log2(errs[0] / errs[1]) > 1.7


def test_subset_matches_full():
    op, m, u = setup(2)
    prm = Params(mu=0.02)
    full = R.residual(u, op, m, prm, scheme="split", dissipation=True, viscous=True)
    sub = [0, 3, 7, 11]
    part = R.residual(u, op, m, prm, scheme="split", dissipation=True, viscous=True, elems=sub)
    assert (part - full[sub]).abs().max() < 1e-13 * full.abs().max()


def test_dense_brute_force_two_elements():
    """Dense global assembly of Eqs. (42)-(44) with Kronecker products and
    Hadamard products, on the 2-element periodic mesh (N = 1), against the
    gathered oracle (strong form) and the weak form."""
    p = 1
    op = tri_operator(p)
    m = periodic_tri_mesh(op, 1, 10.0, 0.05)
    u = states.random_positive_state(m.n_e, 2, op.n_p, seed=5)
    n_p, nc, d = op.n_p, 4, 2
    U = torch.as_tensor(u).transpose(1, 2)
    ops = physical_operators(op, m)
    b = P.beta
    I = torch.eye(nc, dtype=torch.float64)
    out = []
    for k in range(2):
        v = 1 - k
        Dk = [torch.kron(ops["D"][k, i], I) for i in range(d)]
        Hinv = torch.kron(torch.diag(1 / ops["H"][k]), I)
        f = euler_flux(U[k], P)                         # (n_p, d, nc)
        w = entropy_variables(U[k], P).reshape(-1)
        At = symmetrized_flux_jacobians(U[k], P)        # (n_p, d, nc, nc)
        rhs = torch.zeros(n_p * nc, dtype=torch.float64)
        for i in range(d):
            Ablk = torch.block_diag(*[At[mm, i] for mm in range(n_p)])
            rhs -= b / (b + 1) * Dk[i] @ f[:, i].reshape(-1)
            rhs -= 1 / (b + 1) * Ablk @ (Dk[i] @ w)
            rhs += Hinv @ (torch.kron(torch.diag(ops["E"][k, i]), I) @ f[:, i].reshape(-1))
        # facet coupling: E^{kv}_xi = R_gk^T B N_xi R_gv (Eq. (3)), dense n_p x n_p
        Fblk = sy_flux(U[k][:, None, :].expand(n_p, n_p, nc), U[v][None, :, :].expand(n_p, n_p, nc), P)
        for g in range(op.n_fac):
            for i in range(d):
                Ekv = torch.zeros(n_p, n_p, dtype=torch.float64)
                for kk in range(op.n_f):
                    mm = op.facet_nodes[g, kk]
                    vv, ss = m.pair[k, g, kk]
                    assert vv == v
                    nn = op.facet_nodes.reshape(-1)[ss]
                    Ekv[mm, nn] = m.nu[k, g, kk, i]
                # F_i(u_k, u_v) of Eq. (44): blocks 2 diag(F*_i(u_k,m, u_v,n))
                Fi = torch.zeros(n_p * nc, n_p * nc, dtype=torch.float64)
                for mm in range(n_p):
                    for nn in range(n_p):
                        Fi[mm * nc:(mm + 1) * nc, nn * nc:(nn + 1) * nc] = 2 * torch.diag(Fblk[mm, nn, i])
                rhs -= 0.5 * Hinv @ ((torch.kron(Ekv, torch.ones(nc, nc, dtype=torch.float64)) * Fi)
                                     @ torch.ones(n_p * nc, dtype=torch.float64))
        out.append(rhs.reshape(n_p, nc).T)
    dense = torch.stack(out)
    for form in ["strong", "weak"]:
        r = R.residual(u, op, m, P, scheme="split", form=form)
        assert (r - dense).abs().max() < 1e-13 * dense.abs().max()


@pytest.mark.parametrize("heat", [False, True])
def test_viscous_bo_entropy_and_conservation(heat):
    """BO viscous SATs (Eq. (96)): the facet terms cancel in the entropy rate,
    leaving -sum_k sum_ij (D_i w)^T H K~_ij (D_j w) (<= 0 without heat flux),
    and the viscous terms are conservative (Eq. (93))."""
    op, m, u = setup(2)
    prm = Params(mu=0.05, heat_flux=heat)
    rv = R.residual(u, op, m, prm, viscous=True) - R.residual(u, op, m, prm)
    rate = float(Dg.entropy_rate(u, rv, op, m, prm))
    U = torch.as_tensor(u).transpose(1, 2)
    ops = physical_operators(op, m)
    w = entropy_variables(U, prm)
    g = torch.einsum("nimk,nkc->nimc", ops["D"], w)
    from oracle.physics import viscous_K
    K = viscous_K(U, prm)
    qf = float(-torch.einsum("nm,nimc,nmijcb,njmb->", ops["H"], g, K, g))
    assert abs(rate - qf) < 1e-12 * abs(qf)
    if not heat:
        assert qf < 0
    c = Dg.conservation(rv, op, m)
    assert c.abs().max() < 1e-11 * float(rv.abs().max())


TET_PS = [1, 2, 3, 4]


def _tets(N=2, seed=1, p=2):
    from esplit_inputs import tet_operator
    from esplit_inputs.mesh import periodic_tet_mesh
    op = tet_operator(p)
    m = periodic_tet_mesh(op, N, 2 * np.pi, 0.02)
    return op, m, states.random_positive_state(m.n_e, 3, op.n_p, seed=seed)


@pytest.mark.parametrize("p", TET_PS)
@pytest.mark.parametrize("scheme", ["split", "hadamard", "hybrid"])
def test_tet_entropy_conservation_and_forms(scheme, p):
    """Thms. 2 and 4 on curved periodic tetrahedra (affine for p = 1); weak =
    strong form."""
    op, m, u = _tets(p=p)
    flags = np.random.default_rng(2).integers(0, 2, m.n_e)
    r = R.residual(u, op, m, P, scheme=scheme, hybrid_flags=flags)
    assert abs(float(Dg.entropy_rate(u, r, op, m, P))) < 1e-14 * float(Dg.entropy_rate_scale(u, r, op, m, P))
    if scheme != "hybrid":
        rs = R.residual(u, op, m, P, scheme=scheme, form="strong")
        assert (r - rs).abs().max() < 1e-13 * r.abs().max()


@pytest.mark.parametrize("p", TET_PS)
def test_tet_freestream_and_dissipation_sign(p):
    op, m, u = _tets(p=p)
    uf = states.uniform_state(m.n_e, 3, op.n_p)
    assert R.residual(uf, op, m, Params(mu=0.01), dissipation=True, viscous=True).abs().max() < 1e-11
    r0 = R.residual(u, op, m, P)
    r1 = R.residual(u, op, m, P, dissipation=True)
    assert float(Dg.entropy_rate(u, r1 - r0, op, m, P)) < 0


@pytest.mark.parametrize("heat", [False, True])
def test_tet_viscous_bo_identity(heat):
    op, m, u = _tets()
    prm = Params(mu=0.05, heat_flux=heat)
    rv = R.residual(u, op, m, prm, viscous=True) - R.residual(u, op, m, prm)
    rate = float(Dg.entropy_rate(u, rv, op, m, prm))
    U = torch.as_tensor(u).transpose(1, 2)
    ops = physical_operators(op, m)
    w = entropy_variables(U, prm)
    g = torch.einsum("nimk,nkc->nimc", ops["D"], w)
    from oracle.physics import viscous_K
    K = viscous_K(U, prm)
    qf = float(-torch.einsum("nm,nimc,nmijcb,njmb->", ops["H"], g, K, g))
    assert abs(rate - qf) < 1e-11 * abs(qf)
    assert Dg.conservation(rv, op, m).abs().max() < 1e-10 * float(rv.abs().max())


@pytest.mark.parametrize("p", [1, 3])
def test_ir_hadamard_conserves_standard_entropy(p):
    """The Ismail-Roe Hadamard form (the Sec. 6 comparator) conserves the
    standard entropy on any state (Thm. 4 with the standard entropy's Tadmor
    condition), is conservative, preserves free stream, and weak = strong."""
    from oracle.physics import standard_entropy_variables
    op = tri_operator(p)
    m = periodic_tri_mesh(op, 4, 10.0, 0.05)
    u = states.random_positive_state(m.n_e, 2, op.n_p, seed=40 + p)
    r = R.residual(u, op, m, P, scheme="hadamard_ir")
    U = torch.as_tensor(u).transpose(1, 2)
    w = standard_entropy_variables(U, P)
    H = torch.as_tensor(op.H)[None] * torch.as_tensor(m.J)
    rt = r.transpose(1, 2)
    rate = float((H[..., None] * w * rt).sum())
    scale = float((H[..., None] * w.abs() * rt.abs()).sum())
    assert abs(rate) < 1e-13 * scale
    assert Dg.conservation(r, op, m).abs().max() < 1e-12 * float(r.abs().max())
    uf = states.uniform_state(m.n_e, 2, op.n_p)
    assert R.residual(uf, op, m, P, scheme="hadamard_ir").abs().max() < 1e-12
    rs = R.residual(u, op, m, P, scheme="hadamard_ir", form="strong")
    assert (r - rs).abs().max() < 1e-13 * r.abs().max()


@pytest.mark.parametrize("p", [1, 3])
def test_ir_dissipation_rate(p):
    """The comparator's dissipation: the standard-entropy rate of the added
    term equals -1/2 sum over facet nodes of |nu| dw^T D dw / 2 (each pair seen
    from both sides) and is negative; the scheme stays conservative and
    preserves free stream."""
    from oracle.physics import ir_dissipation_matrix, standard_entropy_variables
    op = tri_operator(p)
    m = periodic_tri_mesh(op, 4, 10.0, 0.05)
    u = states.random_positive_state(m.n_e, 2, op.n_p, seed=60 + p)
    r0 = R.residual(u, op, m, P, scheme="hadamard_ir")
    r1 = R.residual(u, op, m, P, scheme="hadamard_ir", dissipation=True)
    U = torch.as_tensor(u).transpose(1, 2)
    w = standard_entropy_variables(U, P)
    H = torch.as_tensor(op.H)[None] * torch.as_tensor(m.J)
    rate = float((H[..., None] * w * (r1 - r0).transpose(1, 2)).sum())
    fn = op.facet_nodes.reshape(-1)
    pr = m.pair.reshape(m.n_e, -1, 2)
    Uk = U[:, fn]
    Uv = U[pr[..., 0], fn[pr[..., 1]]]
    nu = torch.as_tensor(m.nu.reshape(m.n_e, -1, 2))
    b = torch.linalg.norm(nu, dim=-1)
    Dm = ir_dissipation_matrix(Uk, Uv, nu / b[..., None], P)
    dw = standard_entropy_variables(Uk, P) - standard_entropy_variables(Uv, P)
    closed = float(-0.5 * (0.5 * b * torch.einsum("esc,escd,esd->es", dw, Dm, dw)).sum())
    assert closed < 0
    assert abs(rate - closed) < 1e-12 * abs(closed)
    assert Dg.conservation(r1, op, m).abs().max() < 1e-12 * float(r1.abs().max())
    uf = states.uniform_state(m.n_e, 2, op.n_p)
    assert R.residual(uf, op, m, P, scheme="hadamard_ir", dissipation=True).abs().max() < 1e-12


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("heat", [False, True])
def test_ir_viscous_bo_identity(dim, heat):
    """The comparator's Navier-Stokes terms (the same BO SATs written with the
    standard entropy variables): their standard-entropy rate equals the volume
    quadratic form -sum H (D v)^T K~ (D v) (Thm. 3 for the standard entropy,
    with T1 = 0, T2 = T3 = B/2) and is negative with and without heat flux
    (K~ is symmetric PSD in these variables); conservation and free stream."""
    from oracle.physics import standard_entropy_variables, viscous_K
    if dim == 2:
        op = tri_operator(3)
        m = periodic_tri_mesh(op, 4, 10.0, 0.05)
        u = states.random_positive_state(m.n_e, 2, op.n_p, seed=71)
    else:
        op, m, u = _tets(seed=72)
    prm = Params(mu=0.05, heat_flux=heat)
    rv = (R.residual(u, op, m, prm, scheme="hadamard_ir", viscous=True)
          - R.residual(u, op, m, prm, scheme="hadamard_ir"))
    U = torch.as_tensor(u).transpose(1, 2)
    w = standard_entropy_variables(U, prm)
    H = torch.as_tensor(op.H)[None] * torch.as_tensor(m.J)
    rate = float((H[..., None] * w * rv.transpose(1, 2)).sum())
    ops = physical_operators(op, m)
    g = torch.einsum("nimk,nkc->nimc", ops["D"], w)
    qf = float(-torch.einsum("nm,nimc,nmijcb,njmb->", ops["H"], g, viscous_K(U, prm, "standard"), g))
    assert qf < 0
    assert abs(rate - qf) < 1e-11 * abs(qf)
    assert Dg.conservation(rv, op, m).abs().max() < 1e-10 * float(rv.abs().max())
    uf = states.uniform_state(m.n_e, dim, op.n_p)
    assert R.residual(uf, op, m, prm, scheme="hadamard_ir", viscous=True, dissipation=True).abs().max() < 1e-11
