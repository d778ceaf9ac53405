"""Pins of the oracle's boundary facets (the interface SAT of Eq. (43) and the
dissipation of Eq. (69) with a prescribed exterior state), on bounded line
meshes (Sec. 7.2's Shu-Osher problem runs on [-5, 5] with an inflow state).

  * free stream: a uniform state with the same exterior state has r = 0;
  * conservation (Hadamard forms): sum_k 1^T H_k r_k equals minus the
    boundary fluxes, -sum_b [nu F*(u_k, u_b) + |nu|/2 D (w_k - w_b)];
  * entropy (Thms. 2 and 4 on a bounded domain): the EC residual's rate is
    the closed boundary sum sum_b nu [psi(u_k) - w_k^T F*(u_k, u_b)], psi the
    entropy potential V S_H / beta of Harten's entropy; the dissipation
    lowers it by at least sum_b |nu|/2 (w_k - w_b)^T D (w_k - w_b) (interior
    facets dissipate too).
"""
import numpy as np
import pytest
import torch

from esplit_inputs import line_operator, states
from esplit_inputs.mesh import line_mesh
from oracle import residual as R
from oracle.physics import (Params, sy_flux, ir_flux, entropy_variables, harten_entropy, primitives,
                            dissipation_matrix, ir_dissipation_matrix, standard_entropy_variables)
from oracle.operators import physical_operators

P = Params()


def _setup(p=2, N=12, seed=3):
    op = line_operator(p)
    m = line_mesh(op, N, 1.0, 0.0, amp=0.2)
    u = states.random_positive_state(m.n_e, 1, op.n_p, seed=seed)
    ub = states.random_positive_state(2, 1, 1, seed=seed + 100)[:, :, 0]
    return op, m, u, (m.meta["boundary_slots"], ub)


def _boundary_nodes(op, m, u, bnd):
    """(U_k at the boundary nodes, U_b, nu) as (n_b, n_c), (n_b, n_c), (n_b, 1)."""
    fn = op.facet_nodes.reshape(-1)
    slots, ub = bnd
    k, s = slots // len(fn), slots % len(fn)
    Uk = torch.as_tensor(u[k, :, fn[s]])
    nu = torch.as_tensor(m.nu.reshape(m.n_e, -1, 1)[k, s])
    return Uk, torch.as_tensor(ub), nu


@pytest.mark.parametrize("scheme", ["split", "hadamard", "hybrid", "hadamard_ir"])
@pytest.mark.parametrize("diss", [False, True])
def test_boundary_free_stream(scheme, diss):
    op = line_operator(3)
    m = line_mesh(op, 10, 1.0, 0.0, amp=0.2)
    u = states.uniform_state(m.n_e, 1, op.n_p)
    ub = np.repeat(u[:1, :, 0], 2, axis=0)
    flags = np.random.default_rng(1).integers(0, 2, m.n_e)
    r = R.residual(u, op, m, P, scheme=scheme, dissipation=diss, hybrid_flags=flags,
                   boundary=(m.meta["boundary_slots"], ub))
    assert float(r.abs().max()) <= 1e-12   # terms ~1e2 (element size 0.1): a few eps of them


@pytest.mark.parametrize("scheme", ["hadamard", "hadamard_ir"])
@pytest.mark.parametrize("diss", [False, True])
def test_boundary_conservation(scheme, diss):
    op, m, u, bnd = _setup()
    r = R.residual(u, op, m, P, scheme=scheme, dissipation=diss, boundary=bnd)
    H = physical_operators(op, m)["H"]
    total = torch.einsum("nm,ncm->c", H, r)
    Uk, Ub, nu = _boundary_nodes(op, m, u, bnd)
    flux = ir_flux if scheme == "hadamard_ir" else sy_flux
    expect = -(nu[:, :, None] * flux(Uk, Ub, P)).sum(1)
    if diss:
        b = nu.abs()
        if scheme == "hadamard_ir":
            D = ir_dissipation_matrix(Uk, Ub, nu / b, P)
            dw = standard_entropy_variables(Uk, P) - standard_entropy_variables(Ub, P)
        else:
            D = dissipation_matrix(Uk, Ub, nu / b, P)
            dw = entropy_variables(Uk, P) - entropy_variables(Ub, P)
        expect = expect - 0.5 * b * torch.einsum("bcd,bd->bc", D, dw)
    expect = expect.sum(0)
    assert torch.allclose(total, expect, rtol=0, atol=1e-13 * float(expect.abs().max() + 1))


@pytest.mark.parametrize("scheme", ["split", "hadamard", "hybrid"])
def test_boundary_entropy_rate(scheme):
    op, m, u, bnd = _setup(p=3, seed=5)
    flags = np.random.default_rng(2).integers(0, 2, m.n_e)
    H = physical_operators(op, m)["H"]
    U = torch.as_tensor(u).transpose(1, 2)
    w = entropy_variables(U, P)
    Uk, Ub, nu = _boundary_nodes(op, m, u, bnd)
    wk, wb = entropy_variables(Uk, P), entropy_variables(Ub, P)
    rho, V, p = primitives(Uk, P)
    psi = V[:, 0] * harten_entropy(Uk, P) / P.beta
    Fs = sy_flux(Uk, Ub, P)[:, 0]
    closed = (nu[:, 0] * (psi - (wk * Fs).sum(-1))).sum()
    r = R.residual(u, op, m, P, scheme=scheme, hybrid_flags=flags, boundary=bnd).transpose(1, 2)
    rate = (H[..., None] * w * r).sum()
    scale = (H[..., None] * (w * r).abs()).sum()
    assert abs(float(rate - closed)) <= 1e-13 * float(scale)
    rd = R.residual(u, op, m, P, scheme=scheme, hybrid_flags=flags, dissipation=True,
                    boundary=bnd).transpose(1, 2)
    rate_d = (H[..., None] * w * rd).sum()
    D = dissipation_matrix(Uk, Ub, nu / nu.abs(), P)
    extra = 0.5 * (nu.abs()[:, 0] * torch.einsum("bc,bcd,bd->b", wk - wb, D, wk - wb)).sum()
    # interior facets dissipate too: the boundary part is the only closed-form piece,
    # so compare the dissipative rate with the EC rate minus everything dissipated
    assert float(rate_d) < float(rate - extra) + 1e-13 * float(scale)
    assert float(extra) > 0


def test_boundary_requires_states():
    op, m, u, bnd = _setup()
    with pytest.raises(ValueError):
        R.residual(u, op, m, P)
