"""The oracle adjoint is torch.autograd through the oracle residual; pin it
against central finite differences of the same residual (h = 1e-6)."""
import numpy as np
import pytest
import torch

from esplit_inputs import tri_operator, periodic_tri_mesh, states
from oracle import residual as R
from oracle.physics import Params


def vjp(u, cot, fn):
    x = torch.as_tensor(u).clone().requires_grad_(True)
    r = fn(x)
    (g,) = torch.autograd.grad(r, x, grad_outputs=cot)
    return g


@pytest.mark.parametrize("kw", [dict(scheme="split", dissipation=True),
                                dict(scheme="hadamard", dissipation=True),
                                dict(scheme="split", viscous=True)])
def test_vjp_matches_central_differences(kw):
    op = tri_operator(2)
    m = periodic_tri_mesh(op, 2, 10.0, 0.05)
    u = torch.as_tensor(states.add_uniform_noise(states.isentropic_vortex(m), 1e-2, 3))
    prm = Params(mu=0.02)
    fn = lambda x: R.residual(x, op, m, prm, **kw)
    rng = np.random.default_rng(4)
    cot = torch.as_tensor(rng.normal(size=u.shape))
    g = vjp(u, cot, fn)
    for t in range(6):
        dirn = torch.as_tensor(rng.normal(size=u.shape))
        dirn /= dirn.norm()
        h = 1e-6
        fd = ((fn(u + h * dirn) - fn(u - h * dirn)) / (2 * h) * cot).sum()
        ad = (g * dirn).sum()
        assert abs(float(fd - ad)) < 1e-6 * max(1.0, abs(float(ad)))


@pytest.mark.parametrize("heat", [False, True])
def test_oracle_viscous_vjp_central_differences(heat):
    """The oracle's adjoint (autograd) through the BO viscous terms agrees
    with central differences of the oracle residual."""
    from esplit_inputs import tri_operator, periodic_tri_mesh, states
    from oracle import residual as R
    from oracle.physics import Params as OP
    op = tri_operator(2)
    m = periodic_tri_mesh(op, 4, 10.0, 0.05)
    u = states.add_uniform_noise(states.isentropic_vortex(m), 1e-2, 3)
    prm = OP(mu=0.05, heat_flux=heat)
    rng = np.random.default_rng(1)
    cot = torch.as_tensor(rng.normal(size=u.shape))
    x = torch.as_tensor(u).clone().requires_grad_(True)
    (g,) = torch.autograd.grad(R.residual(x, op, m, prm, dissipation=True, viscous=True), x, grad_outputs=cot)
    h = 1e-6
    for _ in range(3):
        d = rng.normal(size=u.shape)
        fd = float(((R.residual(u + h * d, op, m, prm, dissipation=True, viscous=True)
                     - R.residual(u - h * d, op, m, prm, dissipation=True, viscous=True)) / (2 * h) * cot).sum())
        ad = float((g * torch.as_tensor(d)).sum())
        assert abs(fd - ad) <= 1e-6 * abs(ad)
