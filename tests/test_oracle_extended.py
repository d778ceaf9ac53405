"""Pins of the 50-digit residual (oracle/extended.py) and the float64
oracle's distance from it.

The extended-precision restatement is checked against what the paper fixes,
at 50 digits: the two-point flux of Eq. (48) is consistent (F*(U, U) = F(U)),
A~_i W = beta F_i (Eq. (26)), and the EC split and Hadamard residuals conserve
entropy exactly on a periodic mesh (Thms. 2 and 4), while the dissipation of
Eq. (69) only removes it.  Then the float64 oracle is compared with it on
sampled elements of the 32,768-triangle vortex mesh: within a small multiple
of eps times the summand scale, which is the premise of the rounding-scale
parity bound (tests/parity_bounds.py) -- while the plain max-norm relative
error of the float64 oracle itself is above 1e-12 there.
"""
import mpmath as mp
import numpy as np
import pytest

from esplit_inputs import tri_operator, periodic_tri_mesh, states
from oracle import extended as X
from parity_bounds import summand_scale, EPS
from extended_golden import golden_elements


def _rate(res, u, op, m, elems):
    """sum_k sum_m H w^T r at DPS digits, and its scale sum H |w||r|."""
    with mp.workdps(X.DPS):
        P = X._Phys()
        tot, scale = mp.mpf(0), mp.mpf(0)
        for k, r in zip(elems, res):
            for n in range(op.n_p):
                U = [X._mpf(u[k, c, n]) for c in range(op.d + 2)]
                w = X.entropy_vars(U, P)
                H = X._mpf(op.H[n]) * X._mpf(m.J[k, n])
                tot += H * sum(w[c] * r[c][n] for c in range(op.d + 2))
                scale += H * sum(abs(w[c] * r[c][n]) for c in range(op.d + 2))
        return tot, scale


def test_extended_flux_consistency_and_symmetrizer():
    rng = np.random.default_rng(3)
    with mp.workdps(X.DPS):
        P = X._Phys()
        for _ in range(5):
            rho, p = rng.uniform(0.5, 2.0), rng.uniform(0.5, 2.0)
            V = rng.uniform(-0.5, 0.5, 2)
            U = [X._mpf(rho)] + [X._mpf(rho * v) for v in V] + [X._mpf(p / 0.4 + 0.5 * rho * (V @ V))]
            W = X.entropy_vars(U, P)
            for i in range(2):
                F = X.euler_flux(U, i, P)
                Fs = X.sy_flux(U, U, i, P)
                AW = X.at_times(U, i, W, P)
                for c in range(4):
                    assert abs(Fs[c] - F[c]) <= mp.mpf(10) ** -45 * (1 + abs(F[c]))
                    # Eq. (26): A~_i W = beta F_i (the central difference is exact to ~1e-30)
                    assert abs(AW[c] - P.beta * F[c]) <= mp.mpf(10) ** -28 * (1 + abs(F[c]))
            # the closed-form inverse of Eq. (25)
            U2 = X.cons_from_entropy(W, P)
            assert max(abs(a - b) for a, b in zip(U, U2)) <= mp.mpf(10) ** -45


def _antisymmetric_normals(m):
    """The mesh with nu of every paired facet node set to exactly minus its
    partner's (the generated normals agree only to rounding)."""
    import copy
    m2 = copy.deepcopy(m)
    nu = m2.nu.reshape(m.n_e, -1, m.d)
    pr = m2.pair.reshape(m.n_e, -1, 2)
    for k in range(m.n_e):
        for s in range(nu.shape[1]):
            v, s2 = pr[k, s]
            if (v, s2) > (k, s):
                nu[v, s2] = -nu[k, s]
    m2.nu = nu.reshape(m.nu.shape)
    return m2


@pytest.mark.parametrize("scheme", ["split", "hadamard"])
def test_extended_entropy_conservation(scheme):
    """Thms. 2 and 4 at 50 digits on a periodic curved mesh whose paired
    normals are exactly opposite.  Split form: sum H w^T r = 0 exactly (the
    volume term's rate is w^T E f/(beta+1) by SBP and Eqs. (26), (30), which
    the EC SATs cancel through Tadmor's condition).  Hadamard form: the rate
    is -2 sum_k sum_i psi_i^T Q_x_i 1 with psi_i = V_i q p, which is zero only
    as far as the float64 metric terms satisfy the discrete metric identity
    (Q_x_i 1 = 0, Sec. 2.1) -- the identity itself is checked to 1e-38 of the
    rate's scale.  With the dissipation of Eq. (69) the rate is negative."""
    op = tri_operator(2)
    m = _antisymmetric_normals(periodic_tri_mesh(op, 2, 10.0, 0.05))
    u = states.random_positive_state(m.n_e, 2, op.n_p, seed=7)
    el = list(range(m.n_e))
    rate, scale = _rate(X.residual_elements(u, op, m, el, scheme=scheme, dissipation=False), u, op, m, el)
    expect = mp.mpf(0)
    if scheme == "hadamard":
        with mp.workdps(X.DPS):
            P = X._Phys()
            for k in el:
                U, Q, E, H = X._element(u, op, m, k)
                for n in range(op.n_p):
                    rho, V, p, _ = X._prim(U[n], P)
                    qp = X._q(rho, p, P) * p
                    for i in range(2):
                        expect -= 2 * V[i] * qp * sum(Q[i][n][j] for j in range(op.n_p))
        assert abs(expect) > mp.mpf(10) ** -25 * scale  # a float64-rounding-sized defect, not zero
    # the split form's A~_i products come from a central difference exact to
    # ~1e-30 (oracle/extended.py); the Hadamard form has no such step
    tol = mp.mpf(10) ** (-28 if scheme == "split" else -38)
    assert abs(rate - expect) <= tol * scale
    rate_d, _ = _rate(X.residual_elements(u, op, m, el, scheme=scheme, dissipation=True), u, op, m, el)
    assert rate_d < -mp.mpf(10) ** -6 * scale


def test_oracle_float64_against_extended():
    """The float64 oracle against the 50-digit residual (stored by
    tests/golden/make_extended_residual.py, which calls only oracle/) on 5
    sampled elements of config 2 at p = 3, split and Hadamard forms with
    dissipation, on the stored inputs: within 3 eps of the summand scale
    (observed 0.4 split, 1.5 Hadamard).  Its plain max-norm relative error is
    printed (about 1e-12 on this mesh)."""
    from oracle import residual as R
    from oracle.physics import Params
    op, m, u, el, gold = golden_elements()
    for scheme in ["split", "hadamard"]:
        ro = R.residual(u, op, m, Params(), scheme=scheme, dissipation=True, elems=el).numpy()
        sc = summand_scale(u, op, m, el, scheme, Params())
        err = np.abs(ro - gold[scheme])
        plain = float((err.max(axis=(0, 2)) / np.abs(gold[scheme]).max(axis=(0, 2))).max())
        print(f"oracle vs 50 digits, {scheme}: max err/(eps scale) {float((err / (EPS * sc)).max()):.2f}, "
              f"plain max-norm rel {plain:.2e}")
        assert np.all(err <= 3.0 * EPS * sc)


def test_golden_matches_a_fresh_extended_evaluation():
    """Two of the stored elements re-evaluated now (the stored file is what
    oracle/extended.py gives)."""
    op, m, u, el, gold = golden_elements()
    for scheme in ["split", "hadamard"]:
        r = X.residual_elements(u, op, m, el[:2], scheme=scheme, dissipation=True)
        got = np.array([[[float(v) for v in row] for row in e] for e in r])
        assert np.array_equal(got, gold[scheme][:2])
