"""Pin of the Sec. 7.4 manufactured-solution source term (tests/mms.py):
dU/dt + sum_i dF^I_i/dx_i - sum_i dF^V_i/dx_i of the exact solution, by
fourth-order central differences through the oracle's inviscid flux and its
viscous flux from primitive gradients (Eq. (5)), at random points, 2D and 3D;
the velocity and temperature gradients the viscous flux takes are
differences too."""
import numpy as np
import pytest
import torch

from esplit_inputs.states import manufactured_prims, prim_to_cons
from mms import mms_source
from oracle.physics import Params, euler_flux, viscous_flux_from_prim_grads

PRM = Params(mu=0.01, Pr=0.71, R=1.0)
H = 1e-3


def _U(x, t):
    rho, V, p = manufactured_prims(x, t)
    return prim_to_cons(rho, V, p)                     # (nc, N)


def _d(f, x, i, h=H):
    e = np.zeros_like(x)
    e[i] = h
    return (-f(x + 2 * e) + 8 * f(x + e) - 8 * f(x - e) + f(x - 2 * e)) / (12 * h)


def _dt(f, x, t, h=H):
    return (-f(x, t + 2 * h) + 8 * f(x, t + h) - 8 * f(x, t - h) + f(x, t - 2 * h)) / (12 * h)


@pytest.mark.parametrize("d", [2, 3])
def test_mms_source_matches_differences(d):
    rng = np.random.default_rng(70 + d)
    x = rng.uniform(-1, 1, size=(d, 25))
    t = 0.3

    def FI(y):
        U = torch.as_tensor(np.moveaxis(_U(y, t), 0, -1))
        return np.moveaxis(euler_flux(U, PRM).numpy(), -1, 0)          # (nc, N, d)

    def vel(y):
        rho, V, p = manufactured_prims(y, t)
        return V                                                         # (d, N)

    def temp(y):
        rho, V, p = manufactured_prims(y, t)
        return p / (rho * PRM.R)

    def FV(y):
        U = torch.as_tensor(np.moveaxis(_U(y, t), 0, -1))
        dV = np.stack([_d(vel, y, j) for j in range(d)], axis=0)          # (j, k, N): dV_k/dx_j
        dT = np.stack([_d(temp, y, j) for j in range(d)], axis=0)         # (d, N)
        Fv = viscous_flux_from_prim_grads(U, torch.as_tensor(np.moveaxis(dV, -1, 0)),
                                          torch.as_tensor(dT.T), PRM)
        return np.moveaxis(Fv.numpy(), -1, 0)                             # (nc, N, d)

    dUdt = _dt(_U, x, t)
    divI = sum(_d(lambda y: FI(y)[..., i], x, i) for i in range(d))
    divV = sum(_d(lambda y: FV(y)[..., i], x, i) for i in range(d))
    S_fd = dUdt + divI - divV
    S = mms_source(x, t, gam=PRM.gam, mu=PRM.mu, Pr=PRM.Pr)
    assert np.abs(S - S_fd).max() < 1e-7 * np.abs(S).max()
    # the heat-flux part alone is what the viscous terms contribute
    assert np.abs(divV[:-1]).max() < 1e-8
    assert np.abs(divV[-1]).max() > 1e-3
