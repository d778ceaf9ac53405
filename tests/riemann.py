"""Exact solution of the 1D Riemann problem of the Euler equations (test
scaffolding for the Sod shock tube of Sec. 7.1, not part of the method).

The classical construction: the star pressure p* solves
    f_L(p) + f_R(p) + u_R - u_L = 0,
with f_K the velocity change across the K-wave, a shock for p > p_K,
    f_K = (p - p_K) sqrt(A_K / (p + B_K)),  A_K = 2 / ((gam+1) rho_K),
                                            B_K = (gam-1)/(gam+1) p_K,
a rarefaction otherwise,
    f_K = 2 a_K / (gam-1) ((p / p_K)^((gam-1)/(2 gam)) - 1);
then u* = (u_L + u_R)/2 + (f_R(p*) - f_L(p*))/2, the star densities from the
shock (Rankine-Hugoniot) or isentropic relations, and the solution at
x / t = s is read off the wave fan.  Pinned by tests/test_oracle_1d.py against
the jump conditions, the Riemann invariants and the mirror symmetry.
"""
import numpy as np


def _f(p, rho, pk, a, gam):
    if p > pk:
        A = 2.0 / ((gam + 1.0) * rho)
        B = (gam - 1.0) / (gam + 1.0) * pk
        f = (p - pk) * np.sqrt(A / (p + B))
        df = np.sqrt(A / (p + B)) * (1.0 - 0.5 * (p - pk) / (p + B))
    else:
        e = (gam - 1.0) / (2.0 * gam)
        f = 2.0 * a / (gam - 1.0) * ((p / pk) ** e - 1.0)
        df = (p / pk) ** (-(gam + 1.0) / (2.0 * gam)) / (rho * a)
    return f, df


def star_state(left, right, gam=1.4):
    """(p*, u*) for primitive states left = (rho, u, p), right = (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    al, ar = np.sqrt(gam * pl / rl), np.sqrt(gam * pr / rr)
    p = max(1e-8, 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (al + ar))
    for _ in range(100):
        fl, dfl = _f(p, rl, pl, al, gam)
        fr, dfr = _f(p, rr, pr, ar, gam)
        dp = (fl + fr + ur - ul) / (dfl + dfr)
        p_new = max(1e-12, p - dp)
        if abs(p_new - p) <= 1e-15 * (p_new + p):
            p = p_new
            break
        p = p_new
    fl, _ = _f(p, rl, pl, al, gam)
    fr, _ = _f(p, rr, pr, ar, gam)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def sample(s, left, right, gam=1.4):
    """Primitive state (rho, u, p) at similarity coordinate s = (x - x0)/t."""
    ps, us = star_state(left, right, gam)
    g1 = (gam - 1.0) / (gam + 1.0)
    if s <= us:  # left of the contact
        rk, uk, pk = left
        ak = np.sqrt(gam * pk / rk)
        if ps > pk:  # left shock
            S = uk - ak * np.sqrt((gam + 1.0) / (2.0 * gam) * ps / pk + (gam - 1.0) / (2.0 * gam))
            if s <= S:
                return rk, uk, pk
            return rk * (ps / pk + g1) / (g1 * ps / pk + 1.0), us, ps
        rs = rk * (ps / pk) ** (1.0 / gam)
        as_ = ak * (ps / pk) ** ((gam - 1.0) / (2.0 * gam))
        if s <= uk - ak:
            return rk, uk, pk
        if s >= us - as_:
            return rs, us, ps
        u = 2.0 / (gam + 1.0) * (ak + 0.5 * (gam - 1.0) * uk + s)
        c = 2.0 / (gam + 1.0) * (ak + 0.5 * (gam - 1.0) * (uk - s))
        rho = rk * (c / ak) ** (2.0 / (gam - 1.0))
        return rho, u, pk * (c / ak) ** (2.0 * gam / (gam - 1.0))
    rk, uk, pk = right
    ak = np.sqrt(gam * pk / rk)
    if ps > pk:  # right shock
        S = uk + ak * np.sqrt((gam + 1.0) / (2.0 * gam) * ps / pk + (gam - 1.0) / (2.0 * gam))
        if s >= S:
            return rk, uk, pk
        return rk * (ps / pk + g1) / (g1 * ps / pk + 1.0), us, ps
    rs = rk * (ps / pk) ** (1.0 / gam)
    as_ = ak * (ps / pk) ** ((gam - 1.0) / (2.0 * gam))
    if s >= uk + ak:
        return rk, uk, pk
    if s <= us + as_:
        return rs, us, ps
    u = 2.0 / (gam + 1.0) * (-ak + 0.5 * (gam - 1.0) * uk + s)
    c = 2.0 / (gam + 1.0) * (ak - 0.5 * (gam - 1.0) * (uk - s))
    rho = rk * (c / ak) ** (2.0 / (gam - 1.0))
    return rho, u, pk * (c / ak) ** (2.0 * gam / (gam - 1.0))


def shock_speed(left, right, gam=1.4):
    """Speed of the right-moving shock (right wave a shock)."""
    ps, _ = star_state(left, right, gam)
    rk, uk, pk = right
    ak = np.sqrt(gam * pk / rk)
    return uk + ak * np.sqrt((gam + 1.0) / (2.0 * gam) * ps / pk + (gam - 1.0) / (2.0 * gam))
