"""Pins of oracle/physics.py against identities the paper states (Secs. 2-5)."""
from decimal import Decimal, getcontext

import numpy as np
import pytest
import torch

from oracle.physics import (Params, primitives, conservative, harten_entropy, entropy_variables,
                            euler_flux, sy_flux, exp_avg, symmetrized_flux_jacobians, dU_dW,
                            dissipation_matrix, dissipation_factors, viscous_K, temperature, _jacobian)

P = Params()
DT = torch.float64


def rand_states(n, d, seed, lo=0.3):
    g = torch.Generator().manual_seed(seed)
    rho = lo + 2 * torch.rand(n, generator=g, dtype=DT)
    V = 2 * torch.rand(n, d, generator=g, dtype=DT) - 1
    p = lo + 2 * torch.rand(n, generator=g, dtype=DT)
    return conservative(rho, V, p, P)


@pytest.mark.parametrize("d", [2, 3])
def test_entropy_variables_are_gradient(d):
    """W^T = dS_H/dU (Eq. (17)) with S_H of Eq. (16) vs the closed form Eq. (25)."""
    U = rand_states(64, d, 1).requires_grad_(True)
    S = harten_entropy(U, P).sum()
    (g,) = torch.autograd.grad(S, U)
    W = entropy_variables(U.detach(), P)
    assert torch.allclose(g, W, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("d", [2, 3])
def test_symmetrized_jacobians(d):
    """A~_i symmetric (Sec. 2.4) and A~_i W = beta F_i (Eq. (26))."""
    U = rand_states(32, d, 2)
    At = symmetrized_flux_jacobians(U, P)
    assert (At - At.transpose(-1, -2)).abs().max() < 1e-12 * At.abs().max()
    W = entropy_variables(U, P)
    F = euler_flux(U, P)
    AW = torch.einsum("nicd,nd->nic", At, W)
    assert (AW - P.beta * F).abs().max() < 1e-12 * F.abs().max()


@pytest.mark.parametrize("d", [2, 3])
def test_potential_identities(d):
    """beta/(beta+1) W^T F_i = V_i S (Eq. (30)); S = beta phi, phi = W^T U - S (Eqs. (22), (33))."""
    U = rand_states(64, d, 3)
    W = entropy_variables(U, P)
    S = harten_entropy(U, P)
    F = euler_flux(U, P)
    rho, V, p = primitives(U, P)
    lhs = P.beta / (P.beta + 1) * torch.einsum("nc,nic->ni", W, F)
    assert torch.allclose(lhs, V * S[:, None], rtol=1e-12, atol=1e-13)
    phi = (W * U).sum(-1) - S
    assert torch.allclose(S, P.beta * phi, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("d", [2, 3])
def test_sy_flux_consistency_symmetry(d):
    Uk, Uv = rand_states(200, d, 4), rand_states(200, d, 5)
    assert torch.allclose(sy_flux(Uk, Uk, P), euler_flux(Uk, P), rtol=1e-13, atol=1e-13)
    assert torch.allclose(sy_flux(Uk, Uv, P), sy_flux(Uv, Uk, P), rtol=1e-14, atol=1e-14)
    # near-coincident states: continuity into the consistent flux
    Un = Uk * (1 + 1e-9)
    assert torch.allclose(sy_flux(Uk, Un, P), euler_flux(Uk, P), rtol=1e-7, atol=1e-8)


@pytest.mark.parametrize("d", [2, 3])
def test_sy_flux_tadmor(d):
    """Tadmor's condition, Eq. (49): (W'' - W')^T F*_i = psi_i'' - psi_i',
    psi_i = W^T F_i - V_i S (Eq. (23)), on 10^4 random state pairs."""
    Ua, Ub = rand_states(10000, d, 6), rand_states(10000, d, 7)
    Fs = sy_flux(Ua, Ub, P)
    Wa, Wb = entropy_variables(Ua, P), entropy_variables(Ub, P)

    def psi(U):
        W = entropy_variables(U, P)
        rho, V, p = primitives(U, P)
        return torch.einsum("nc,nic->ni", W, euler_flux(U, P)) - V * harten_entropy(U, P)[:, None]

    lhs = torch.einsum("nc,nic->ni", Wb - Wa, Fs)
    rhs = psi(Ub) - psi(Ua)
    scale = (torch.einsum("nc,nic->ni", Wb.abs() + Wa.abs(), Fs.abs()))
    assert ((lhs - rhs).abs() / scale).max() < 1e-13


def test_exp_avg_extended_precision():
    getcontext().prec = 60
    rng = np.random.default_rng(8)
    for r in [1.0 / 6.0, 7.0 / 12.0, -0.5, 2.5]:
        a = rng.uniform(0.2, 3.0, 300)
        eps = 10.0 ** rng.uniform(-15, 0, 300) * rng.choice([-0.9, 0.9], 300)
        b = a * (1 + eps)
        got = exp_avg(torch.tensor(a), torch.tensor(b), r).numpy()
        for ai, bi, gi in zip(a, b, got):
            A, B, R = Decimal(float(ai)), Decimal(float(bi)), Decimal(r)
            ex = (A ** R - B ** R) / (R * (A - B))
            assert abs(Decimal(float(gi)) - ex) / abs(ex) < Decimal(8e-16)
    # coincident states: the limit a^(r-1)
    a = torch.tensor([0.7, 1.3])
    assert torch.allclose(exp_avg(a, a, 0.3), a ** (-0.7), rtol=1e-15)


def _nhat(n, d, seed):
    g = torch.Generator().manual_seed(seed)
    v = torch.randn(n, d, generator=g, dtype=DT)
    return v / torch.linalg.norm(v, dim=-1, keepdim=True)


@pytest.mark.parametrize("d", [1, 2])
def test_dissipation_scaling_2d(d):
    """Barth scaling: X^ S^ X^T = dU/dW at coincident states (Sec. 4.5, 2D;
    1D with the shear modes deleted)."""
    U = rand_states(200, d, 9)
    n = _nhat(200, d, 10)
    X, lam, sc = dissipation_factors(U, U, n, P)
    A0 = dU_dW(U, P)
    got = X @ torch.diag_embed(sc) @ X.transpose(-1, -2)
    assert ((got - A0).abs().amax((-1, -2)) / A0.abs().amax((-1, -2))).max() < 1e-12


@pytest.mark.parametrize("d", [1, 2, 3])
def test_dissipation_eigenvectors(d):
    """A_n X^ = X^ Lambda_n (Eqs. (79)-(80)) at coincident states, n_1 != 0."""
    U = rand_states(100, d, 16)
    n = _nhat(100, d, 17)
    X, lam, sc = dissipation_factors(U, U, n, P)
    for k in range(100):
        nk = n[k]
        Ak = torch.func.jacrev(lambda x: torch.einsum("ic,i->c", euler_flux(x, P), nk))(U[k])
        assert (Ak @ X[k] - X[k] * lam[k]).abs().max() < 1e-12 * (1 + Ak.abs().max())


@pytest.mark.parametrize("d", [1, 2, 3])
def test_dissipation_symmetric_psd_and_flip(d):
    Uk, Uv = rand_states(100, d, 11), rand_states(100, d, 12)
    n = _nhat(100, d, 13)
    D = dissipation_matrix(Uk, Uv, n, P)
    assert (D - D.transpose(-1, -2)).abs().max() < 1e-13 * D.abs().max()
    assert torch.linalg.eigvalsh(D).min() > -1e-12 * D.abs().max()
    assert torch.allclose(D, dissipation_matrix(Uk, Uv, -n, P), rtol=1e-12, atol=1e-12)
    assert torch.allclose(D, dissipation_matrix(Uv, Uk, n, P), rtol=1e-12, atol=1e-12)


def test_temperature_closed_forms():
    """T(W) of Eq. (39) and W_nc of Eq. (41) (R = 1), and dT/dW.

    Eq. (40) as printed has two typos: differentiating Eq. (39) gives
    dT/dW_i = +(gam-1) V_i / (alpha R W_nc) (printed with a minus sign) and
    dT/dW_nc = -T/W_nc + (gam-1)|V|^2 / (2 alpha R W_nc) (printed without
    alpha).  The exact derivative of Eq. (39) is the reading used."""
    U = rand_states(40, 3, 14)
    W = entropy_variables(U, P)
    rho, V, p = primitives(U, P)
    g, a, R = P.gam, P.alpha, P.R
    Wn = W[:, -1]
    T = (g - 1) * (2 * W[:, 0] * Wn - (W[:, 1:-1] ** 2).sum(-1)) / (2 * a * R * Wn ** 2)
    assert torch.allclose(T, temperature(U, P), rtol=1e-12)
    assert torch.allclose(Wn, -p ** ((1 - a - g) / (a + g)) * rho ** (a / (a + g)), rtol=1e-13)
    dTdW = (_jacobian(lambda x: temperature(x, P)[..., None], U) @ dU_dW(U, P))[:, 0]
    ex = torch.cat([((g - 1) / (a * R * Wn))[:, None], (g - 1) * V / (a * R * Wn[:, None]),
                    (-T / Wn + (g - 1) * (V * V).sum(-1) / (2 * a * R * Wn))[:, None]], -1)
    assert torch.allclose(dTdW, ex, rtol=1e-10, atol=1e-12)
    printed = torch.cat([((g - 1) / (a * R * Wn))[:, None], -(g - 1) * V / (a * R * Wn[:, None]),
                         (-T / Wn + (g - 1) * (V * V).sum(-1) / (2 * R * Wn))[:, None]], -1)
    assert not torch.allclose(dTdW, printed, rtol=1e-6)


@pytest.mark.parametrize("d", [2, 3])
def test_viscous_tensor_psd_without_heat_flux(d):
    """K~ symmetric positive semidefinite without heat flux (Sec. 5); the heat
    flux breaks the symmetry (Sec. 3, Eq. (38))."""
    U = rand_states(10, d, 15)
    nc = d + 2
    for heat in [False, True]:
        prm = Params(mu=0.1, heat_flux=heat)
        K = viscous_K(U, prm)  # (n, d, d, nc, nc)
        Kb = K.permute(0, 1, 3, 2, 4).reshape(10, d * nc, d * nc)
        asym = (Kb - Kb.transpose(1, 2)).abs().max() / Kb.abs().max()
        if heat:
            assert asym > 1e-3
        else:
            assert asym < 1e-12
            assert torch.linalg.eigvalsh(Kb).min() > -1e-12 * Kb.abs().max()
            # rank of K~ equals the number of nonzero pivots of the LDL^T
            # statement of Sec. 5 (3D: pivots 4/3 delta and four delta -> 5; 2D: 3)
            ev = torch.linalg.eigvalsh(Kb)
            rank = (ev > 1e-10 * ev.amax(-1, keepdim=True)).sum(-1)
            assert torch.all(rank == {2: 3, 3: 5}[d])


def test_viscous_flux_special_cases():
    """Plane shear V = (s y, 0): tau_xy = mu s, tau_xx = 0; pure temperature
    gradient dT/dx: energy flux kappa dT/dx (Eq. (5)); and the flux from the
    entropy-variable gradient equals the flux from primitive gradients of a
    smooth field (chain rule through dU/dW)."""
    from oracle.physics import viscous_flux_from_prim_grads, viscous_flux_from_w_grads
    prm = Params(mu=0.3)
    U = rand_states(5, 2, 18)
    s = 0.7
    dV = torch.zeros(5, 2, 2, dtype=DT)
    dV[:, 1, 0] = s                      # dV_1/dx_2
    F = viscous_flux_from_prim_grads(U, dV, torch.zeros(5, 2, dtype=DT), prm)
    assert torch.allclose(F[:, 0, 2], torch.full((5,), prm.mu * s, dtype=DT))   # tau_xy in x-flux
    assert torch.allclose(F[:, 0, 1], torch.zeros(5, dtype=DT))                   # tau_xx
    dT = torch.zeros(5, 2, dtype=DT)
    dT[:, 0] = 2.0
    F = viscous_flux_from_prim_grads(U, torch.zeros(5, 2, 2, dtype=DT), dT, prm)
    assert torch.allclose(F[:, 0, 3], torch.full((5,), 2.0 * prm.kappa, dtype=DT))
    # smooth field x -> U(x): gradients by autograd in x
    x0 = torch.tensor([0.3, -0.2], dtype=DT)

    def Ufield(x):
        rho = 1.0 + 0.2 * torch.sin(x[0]) * torch.cos(x[1])
        V = torch.stack([0.3 + 0.1 * x[1] ** 2, -0.2 + 0.1 * torch.sin(x[0] + x[1])])
        p = 1.0 + 0.1 * torch.cos(2 * x[0] - x[1])
        return conservative(rho, V, p, prm)

    Ux = Ufield(x0)
    gW = torch.func.jacrev(lambda x: entropy_variables(Ufield(x), prm))(x0).T       # (d, nc)
    dVx = torch.func.jacrev(lambda x: primitives(Ufield(x), prm)[1])(x0).T          # [j, k] = dV_k/dx_j
    dTx = torch.func.jacrev(lambda x: temperature(Ufield(x), prm))(x0)
    Fa = viscous_flux_from_w_grads(Ux[None], gW[None], prm)[0]
    Fb = viscous_flux_from_prim_grads(Ux[None], dVx[None], dTx[None], prm)[0]
    assert torch.allclose(Fa, Fb, rtol=1e-12, atol=1e-13)


def test_entropy_change_extended_precision():
    """s(U+dU) - s(U) without cancellation (used by Eq. (97)) against the
    plain difference of Eq. (16) evaluated in 60-digit decimal arithmetic."""
    from oracle.physics import harten_entropy_change
    getcontext().prec = 60
    U = rand_states(200, 2, 21)
    g = torch.Generator().manual_seed(22)
    scale = 10.0 ** (-torch.randint(1, 12, (200, 1), generator=g).double())
    dU = (2 * torch.rand(200, 4, generator=g, dtype=DT) - 1) * scale * U.abs()
    got = harten_entropy_change(U, dU, P).numpy()
    gam, a, beta = Decimal(P.gam), Decimal(P.alpha), Decimal(P.beta)
    A, B = a / (a + gam), Decimal(1) / (a + gam)

    def sdec(u):
        rho, m1, m2, E = [Decimal(float(x)) for x in u]
        p = (gam - 1) * (E - (m1 * m1 + m2 * m2) / (2 * rho))
        return beta * rho ** A * p ** B

    eps = np.finfo(float).eps
    A_, B_ = float(A), float(B)
    for k in range(200):
        u0 = U[k].numpy()
        du = dU[k].numpy()
        u1 = [Decimal(float(x)) + Decimal(float(y)) for x, y in zip(u0, du)]
        ex = sdec([float(x) for x in u0])
        rho, m1, m2, E = u1
        p1 = (gam - 1) * (E - (m1 * m1 + m2 * m2) / (2 * rho))
        diff = beta * rho ** A * p1 ** B - ex
        # forward-error scale of the formula: |s| times the sizes of the small
        # relative changes it combines (not |s| itself, as a plain difference)
        r0, m, E0 = u0[0], u0[1:3], u0[3]
        p0 = (P.gam - 1) * (E0 - 0.5 * (m @ m) / r0)
        dke = (abs(2 * m @ du[1:3]) + du[1:3] @ du[1:3]) / (2 * r0) + (m @ m) * abs(du[0]) / (2 * r0 * r0)
        scale = abs(float(ex)) * (abs(A_) * abs(du[0]) / r0 + abs(B_) * (P.gam - 1) * (abs(du[3]) + dke) / p0)
        assert abs(Decimal(float(got[k])) - diff) <= Decimal(64 * eps * scale) + Decimal(1e-300)
        assert abs(Decimal(float(got[k])) - diff) <= Decimal(1e-9) * abs(diff) + Decimal(64 * eps * scale)


@pytest.mark.parametrize("d", [2, 3])
def test_inverse_entropy_map(d):
    """U(W(U)) = U, and dU/dW (Jacobian of the closed-form inverse) times
    dW/dU (Jacobian of Eq. (25)) is the identity: the two Jacobians come from
    independent formulas."""
    from oracle.physics import conservative_from_entropy, dW_dU
    U = rand_states(300, d, 21)
    back = conservative_from_entropy(entropy_variables(U, P), P)
    assert ((back - U).abs() / U.abs().amax(-1, keepdim=True)).max() < 1e-13
    prod = dU_dW(U, P) @ dW_dU(U, P)
    I = torch.eye(d + 2, dtype=DT)
    cond = torch.linalg.cond(dW_dU(U, P))
    assert ((prod - I).abs().amax((-1, -2)) / cond).max() < 1e-14
    # a low-Mach state (Mach 0.1, p ~ 71): the inverse map stays accurate
    # although cond(dW/dU) ~ 4e5
    Ulm = torch.tensor([[1.0, 0.3, -0.2, 71.43 / 0.4 + 0.065]], dtype=DT)
    back = conservative_from_entropy(entropy_variables(Ulm, P), P)
    assert ((back - Ulm).abs() / Ulm.abs()).max() < 1e-13


@pytest.mark.parametrize("d", [2, 3])
def test_ir_flux_consistency_symmetry_tadmor(d):
    """Ismail-Roe flux: F*(U, U) = F(U), symmetric in its arguments, and
    Tadmor's condition for the standard entropy,
    (w_v - w_k) . F*_i = psi_v - psi_k with psi_i = rho V_i."""
    from oracle.physics import ir_flux, standard_entropy_variables
    Uk = rand_states(400, d, 31)
    Uv = rand_states(400, d, 32)
    Fs = ir_flux(Uk, Uk, P)
    assert (Fs - euler_flux(Uk, P)).abs().max() < 1e-13 * euler_flux(Uk, P).abs().max()
    assert (ir_flux(Uk, Uv, P) - ir_flux(Uv, Uk, P)).abs().max() < 1e-13
    F = ir_flux(Uk, Uv, P)
    dw = standard_entropy_variables(Uv, P) - standard_entropy_variables(Uk, P)
    for i in range(d):
        lhs = (dw * F[..., i, :]).sum(-1)
        rhs = Uv[..., 1 + i] - Uk[..., 1 + i]
        scale = (dw.abs() * F[..., i, :].abs()).sum(-1) + rhs.abs()
        assert ((lhs - rhs).abs() / scale).max() < 1e-13
    # nearly equal states exercise the logarithmic-mean limit
    Ue = Uk * (1.0 + 1e-9 * torch.randn(Uk.shape, generator=torch.Generator().manual_seed(5), dtype=DT))
    assert (ir_flux(Uk, Ue, P) - euler_flux(Uk, P)).abs().max() < 1e-7 * euler_flux(Uk, P).abs().max()


def test_standard_entropy_variables_are_gradient():
    from oracle.physics import standard_entropy, standard_entropy_variables
    U = rand_states(50, 2, 33).requires_grad_(True)
    (g,) = torch.autograd.grad(standard_entropy(U, P).sum(), U)
    assert (g - standard_entropy_variables(U.detach(), P)).abs().max() < 1e-12


def test_log_mean():
    from oracle.physics import log_mean
    a = torch.tensor([1.0, 2.0, 3.0, 1e-3, 5.0], dtype=DT)
    b = torch.tensor([1.0, 2.0 + 1e-12, 1.5, 2e-3, 5.0 * (1 + 1e-6)], dtype=DT)
    ref = torch.tensor([float(Decimal(x) if x == y else (Decimal(x) - Decimal(y)) / (Decimal(x).ln() - Decimal(y).ln()))
                        for x, y in zip(a.tolist(), b.tolist())], dtype=DT)
    assert ((log_mean(a, b) - ref).abs() / ref).max() < 1e-15


@pytest.mark.parametrize("d", [2, 3])
def test_ir_dissipation_matrix_pins(d):
    """Matrix dissipation of the Ismail-Roe comparator: for equal states the
    eigenvector factorisation equals dU/dw of the standard entropy (inverse of
    the autograd Jacobian of w(U)) when all |lambda| are replaced by one, and
    R|L|TR^T = |A_n| dU/dw (A_n the normal flux Jacobian); for any pair it is
    symmetric, positive semi-definite, invariant under n -> -n and symmetric
    in the two states."""
    from oracle.physics import ir_dissipation_matrix, standard_entropy_variables
    U = rand_states(60, d, 51)
    g = torch.Generator().manual_seed(52)
    n = torch.randn(60, d, generator=g, dtype=DT)
    n = n / torch.linalg.norm(n, dim=-1, keepdim=True)
    Dm = ir_dissipation_matrix(U, U, n, P)
    dUdw = torch.linalg.inv(_jacobian(lambda x: standard_entropy_variables(x, P), U))
    An = torch.einsum("ni,nicd->ncd", n, _jacobian(lambda x: euler_flux(x, P), U))
    # |A_n| dU/dw through the eigen-decomposition of A_n (real spectrum)
    ev, evec = torch.linalg.eig(An)
    absA = (evec @ torch.diag_embed(ev.abs().to(evec.dtype)) @ torch.linalg.inv(evec)).real
    ref = absA @ dUdw
    assert ((Dm - ref).abs().amax((-1, -2)) / ref.abs().amax((-1, -2))).max() < 1e-11
    Uv = rand_states(60, d, 53)
    D2 = ir_dissipation_matrix(U, Uv, n, P)
    assert (D2 - D2.transpose(-1, -2)).abs().max() < 1e-13 * D2.abs().max()
    assert torch.linalg.eigvalsh(D2).min() > -1e-12 * D2.abs().max()
    assert (ir_dissipation_matrix(U, Uv, -n, P) - D2).abs().max() < 1e-13 * D2.abs().max()
    assert (ir_dissipation_matrix(Uv, U, n, P) - D2).abs().max() < 1e-13 * D2.abs().max()


@pytest.mark.parametrize("d", [2, 3])
def test_standard_entropy_inverse_map(d):
    """The closed-form inverse of the standard entropy variables: the round
    trip returns U; its Jacobian dU/dv is the inverse of dv/dU (autograd of
    the forward map) and, as the Hessian of the entropy potential, symmetric
    positive definite."""
    from oracle.physics import (standard_entropy_variables, conservative_from_standard_entropy,
                                dU_dV_standard, _jacobian)
    U = rand_states(20, d, 31)
    P0 = Params()
    back = conservative_from_standard_entropy(standard_entropy_variables(U, P0), P0)
    assert (back - U).abs().max() < 1e-13 * U.abs().max()
    A = dU_dV_standard(U, P0)
    B = _jacobian(lambda x: standard_entropy_variables(x, P0), U)
    I = torch.eye(d + 2, dtype=torch.float64)
    assert (A @ B - I).abs().max() < 1e-11
    assert (A - A.transpose(-1, -2)).abs().max() < 1e-13 * A.abs().max()
    assert torch.linalg.eigvalsh(A).min() > 0


@pytest.mark.parametrize("d", [2, 3])
def test_viscous_tensor_standard_entropy_symmetric_psd(d):
    """In the standard entropy variables K~ is symmetric positive semidefinite
    with and without the heat flux (the property the Harten variables lose
    with heat flux, Sec. 3); the heat flux raises its rank by d (one
    temperature-gradient direction per coordinate: 2D 3 -> 5, 3D 5 -> 8); and for any
    conservative-variable gradient the two variable sets give the same
    viscous flux (the flux is a property of the state and its gradient)."""
    from oracle.physics import viscous_flux_from_w_grads, standard_entropy_variables, _jacobian
    U = rand_states(10, d, 33)
    nc = d + 2
    for heat in [False, True]:
        prm = Params(mu=0.1, heat_flux=heat)
        K = viscous_K(U, prm, "standard")
        Kb = K.permute(0, 1, 3, 2, 4).reshape(10, d * nc, d * nc)
        assert (Kb - Kb.transpose(1, 2)).abs().max() < 1e-12 * Kb.abs().max()
        ev = torch.linalg.eigvalsh(Kb)
        assert ev.min() > -1e-12 * Kb.abs().max()
        rank = (ev > 1e-10 * ev.amax(-1, keepdim=True)).sum(-1)
        assert torch.all(rank == {2: 3, 3: 5}[d] + (d if heat else 0))
        gU = torch.as_tensor(np.random.default_rng(4).normal(size=(10, d, nc)))
        gv = torch.einsum("ncb,nib->nic", _jacobian(lambda x: standard_entropy_variables(x, prm), U), gU)
        gW = torch.einsum("ncb,nib->nic", _jacobian(lambda x: entropy_variables(x, prm), U), gU)
        Fs = viscous_flux_from_w_grads(U, gv, prm, "standard")
        Fh = viscous_flux_from_w_grads(U, gW, prm)
        assert (Fs - Fh).abs().max() < 1e-11 * Fh.abs().max()
