"""Seeded initial states, laid out as the residual expects: (n_e, n_c, n_p)
float64 conservative variables [rho, rho V_1..V_d, e], e = p/(gam-1) + rho|V|^2/2
(Sec. 2.2).

The 2D isentropic vortex follows Sec. 7.3 with two readings of the printed
formula: the density coefficient is alpha^2 (gam-1) / (16 gam pi^2) (the
printed "16 gam pi" is a typo; the pi^2 is forced by the radial momentum
balance of the printed velocity field), and the vortex core sits at
(x_c + t, y_c) (the printed r^2 uses "+t").  Domain [0, L]^2, centre (L/2, L/2).
"""
from __future__ import annotations

import numpy as np

GAMMA = 1.4


def prim_to_cons(rho, V, p, gam=GAMMA):
    """rho (...), V (d, ...), p (...) -> U (d + 2, ...)."""
    ke = 0.5 * rho * np.sum(V * V, axis=0)
    return np.concatenate([rho[None], rho[None] * V, (p / (gam - 1) + ke)[None]], axis=0)


def isentropic_vortex_prims(x, y, t=0.0, xc=5.0, yc=5.0, alpha=3.0, gam=GAMMA):
    dx = x - xc - t
    dy = y - yc
    r2 = dx * dx + dy * dy
    ex = np.exp(1.0 - r2)
    rho = (1.0 - alpha ** 2 * (gam - 1.0) / (16.0 * gam * np.pi ** 2) * ex * ex) ** (1.0 / (gam - 1.0))
    p = rho ** gam
    u = 1.0 - alpha / (2.0 * np.pi) * dy * ex
    v = alpha / (2.0 * np.pi) * dx * ex
    return rho, np.stack([u, v]), p


def isentropic_vortex(mesh, t=0.0, alpha=3.0, gam=GAMMA, center=None):
    """Vortex of strength alpha centred at ``center`` (default: the centre of
    the [0, L]^2 square). Periodic images are left out: on [0, 10]^2 their
    perturbation is O(e^-24)."""
    L = mesh.L[0]
    xc, yc = (L / 2, L / 2) if center is None else center
    x, y = mesh.x[:, 0], mesh.x[:, 1]
    rho, V, p = isentropic_vortex_prims(x, y, t=t, xc=xc, yc=yc, alpha=alpha, gam=gam)
    return np.ascontiguousarray(np.moveaxis(prim_to_cons(rho, V, p, gam), 0, 1))


def isentropic_vortex_3d(mesh, t=0.0, gam=GAMMA):
    """3D isentropic vortex of Sec. 7.3 on [-10, 10]^3, moving with unit speed
    in x_2: with r^2 = x_1^2 + (x_2 - t)^2,
      rho = (1 - 2/25 (gam-1) exp(1 - r^2))^(1/(gam-1)),  p = rho^gam / gam,
      V_1 = -2/5 (x_2 - t) exp((1 - r^2)/2),  V_2 = 1 + 2/5 x_1 exp((1 - r^2)/2),  V_3 = 0.
    Reading: the printed exponent of V_1 carries (x_1 - t)^2; (x_2 - t)^2, as in
    V_2 and rho, is the one the radial momentum balance dp/dr = rho v_theta^2 / r
    of this density requires."""
    return np.ascontiguousarray(np.moveaxis(prim_to_cons(*vortex3d_prims(mesh.x[:, 0], mesh.x[:, 1], t, gam),
                                                         gam), 0, 1))


def vortex3d_prims(x1, x2, t=0.0, gam=GAMMA):
    a = x2 - t
    r2 = x1 * x1 + a * a
    ex = np.exp(0.5 * (1.0 - r2))
    rho = (1.0 - 2.0 / 25.0 * (gam - 1.0) * ex * ex) ** (1.0 / (gam - 1.0))
    p = rho ** gam / gam
    V = np.stack([-0.4 * a * ex, 1.0 + 0.4 * x1 * ex, 0.0 * x1])
    return rho, V, p


def manufactured_prims(x, t=0.0, gam=GAMMA):
    """Manufactured solution of Sec. 7.4 on [-1, 1]^d, x (d, ...):
    rho = 2 + 0.1 sin(pi (sum_i x_i - 0.6 t)), V_i = 1,
    p = (gam - 1)(rho^2 - rho |V|^2 / 2)  (so that the total energy is rho^2)."""
    d = x.shape[0]
    rho = 2.0 + 0.1 * np.sin(np.pi * (np.sum(x, axis=0) - 0.6 * t))
    V = np.ones((d,) + rho.shape)
    p = (gam - 1.0) * (rho * rho - 0.5 * rho * d)
    return rho, V, p


def manufactured_state(mesh, t=0.0, gam=GAMMA):
    """The Sec. 7.4 manufactured solution at the mesh nodes, (n_e, d+2, n_p)."""
    x = np.moveaxis(mesh.x, 1, 0)                       # (d, n_e, n_p)
    rho, V, p = manufactured_prims(x, t, gam)
    return np.ascontiguousarray(np.moveaxis(prim_to_cons(rho, V, p, gam), 0, 1))


def add_uniform_noise(u, amplitude, seed):
    """u + amplitude * U(-1, 1), drawn by numpy's PCG64 in C order of u."""
    rng = np.random.default_rng(seed)
    return u + amplitude * rng.uniform(-1.0, 1.0, size=u.shape)


def random_positive_state(n_e, d, n_p, seed, rho=(0.5, 2.0), vel=(-1.0, 1.0), p=(0.5, 2.0), gam=GAMMA):
    """Independent random primitive states at every node (well inside the
    admissible set), returned as conservative variables (n_e, d+2, n_p)."""
    rng = np.random.default_rng(seed)
    r = rng.uniform(*rho, size=(n_e, n_p))
    V = rng.uniform(*vel, size=(d, n_e, n_p))
    pr = rng.uniform(*p, size=(n_e, n_p))
    return np.ascontiguousarray(np.moveaxis(prim_to_cons(r, V, pr, gam), 0, 1))


def uniform_state(n_e, d, n_p, rho=1.0, V=(0.3, -0.2, 0.1), p=1.0, gam=GAMMA):
    r = np.full((n_e, n_p), rho)
    Vv = np.stack([np.full((n_e, n_p), V[i]) for i in range(d)])
    pr = np.full((n_e, n_p), p)
    return np.ascontiguousarray(np.moveaxis(prim_to_cons(r, Vv, pr, gam), 0, 1))


def quadrant_states(mesh, seed, pressure_ratio_max=10.0, gam=GAMMA):
    """Four piecewise-constant quadrant states on [0, L]^2 (a 2D Riemann-type
    problem): rho ~ U[0.5, 2], u, v ~ U[-0.5, 0.5], p ~ U[0.2, 2], redrawn
    until max p / min p <= pressure_ratio_max. A node belongs to the quadrant
    of its element centroid, so every element is constant."""
    rng = np.random.default_rng(seed)
    while True:
        rho = rng.uniform(0.5, 2.0, 4)
        vel = rng.uniform(-0.5, 0.5, (2, 4))
        pr = rng.uniform(0.2, 2.0, 4)
        if pr.max() / pr.min() <= pressure_ratio_max:
            break
    L = mesh.L[0]
    c = mesh.x.mean(axis=2)
    q = (c[:, 0] >= L / 2).astype(int) + 2 * (c[:, 1] >= L / 2).astype(int)
    r = np.repeat(rho[q][:, None], mesh.n_p, 1)
    V = np.stack([np.repeat(vel[i][q][:, None], mesh.n_p, 1) for i in range(2)])
    pp = np.repeat(pr[q][:, None], mesh.n_p, 1)
    return np.ascontiguousarray(np.moveaxis(prim_to_cons(r, V, pp, gam), 0, 1))


def cfl_timestep(mesh, u, cfl, gam=GAMMA):
    """Time step of Sec. 7.1: min over elements of CFL * h_min / |lambda|_max,
    |lambda|_max = max over the element's nodes of |V| + sqrt(gam p / rho)."""
    rho = u[:, 0]
    V = u[:, 1:-1] / rho[:, None]
    p = (gam - 1.0) * (u[:, -1] - 0.5 * rho * np.sum(V * V, axis=1))
    lam = np.sqrt(np.sum(V * V, axis=1)) + np.sqrt(gam * p / rho)
    return float(np.min(cfl * mesh.hmin / lam.max(axis=1)))


def taylor_green(mesh, Mach=0.1, gam=GAMMA, R=1.0):
    """Taylor-Green vortex initial state of Sec. 7.5 with u_0 = rho_0 = R = L = 1
    on the periodic [0, 2 pi]^3 box: p_0 = rho_0 u_0^2 / (gam M^2), T_0 = p_0,
    V = (sin x cos y cos z, -cos x sin y cos z, 0),
    p = p_0 + (cos 2x + cos 2y)(cos 2z + 2)/16, rho = p / (R T_0)."""
    x, y, z = mesh.x[:, 0], mesh.x[:, 1], mesh.x[:, 2]
    p0 = 1.0 / (gam * Mach ** 2)
    T0 = p0 / R
    V = np.stack([np.sin(x) * np.cos(y) * np.cos(z), -np.cos(x) * np.sin(y) * np.cos(z), 0.0 * x])
    p = p0 + (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0) / 16.0
    rho = p / (R * T0)
    return np.ascontiguousarray(np.moveaxis(prim_to_cons(rho, V, p, gam), 0, 1))


def sod_periodic(mesh, gam=GAMMA):
    """The Sod shock tube of Sec. 7.1 (rho, u, p = 1, 0, 1 left of x = 0.5 and
    0.125, 0, 0.1 right of it on [0, 1]) on the periodic [0, 2) with its mirror
    image on [1, 2): elements whose centre lies in [0.5, 1.5) take the right
    state.  Up to t = 0.2 no wave reaches x = 0 or x = 1 (rarefaction head
    0.26, shock 0.85 and their mirrors), so on [0, 1] the solution is the one
    of the shock tube with its walls.  Element-wise constant data."""
    xc = mesh.x[:, 0, :].mean(axis=1)
    right = (xc >= 0.5) & (xc < 1.5)
    r = np.where(right, 0.125, 1.0)[:, None] * np.ones((1, mesh.n_p))
    pr = np.where(right, 0.1, 1.0)[:, None] * np.ones((1, mesh.n_p))
    V = np.zeros((1, mesh.n_e, mesh.n_p))
    return np.ascontiguousarray(np.moveaxis(prim_to_cons(r, V, pr, gam), 0, 1))


SHU_OSHER_LEFT = (3.857143, 2.629369, 10.33333)   # rho, u, p for x <= -4 (Sec. 7.2)


def shu_osher_right(x):
    """rho, u, p of the Sec. 7.2 initial state for x > -4: 1 + 0.2 sin(5x), 0, 1."""
    x = np.asarray(x, dtype=float)
    return 1.0 + 0.2 * np.sin(5.0 * x), np.zeros_like(x), np.ones_like(x)


def shu_osher(mesh, gam=GAMMA):
    """The Shu-Osher problem of Sec. 7.2 on [-5, 5]: the left state (3.857143,
    2.629369, 10.33333) on elements whose centre is left of x = -4, the
    sinusoidal right state at the nodes elsewhere (a mesh with a vertex at
    x = -4 puts the jump on an element boundary)."""
    x = mesh.x[:, 0, :]
    left = (x.mean(axis=1) <= -4.0)[:, None] * np.ones((1, mesh.n_p), dtype=bool)
    rr, ur, pr = shu_osher_right(x)
    rl, ul, pl = SHU_OSHER_LEFT
    rho = np.where(left, rl, rr)
    V = np.where(left, ul, ur)[None]
    p = np.where(left, pl, pr)
    return np.ascontiguousarray(np.moveaxis(prim_to_cons(rho, V, p, gam), 0, 1))


def shu_osher_boundary(gam=GAMMA):
    """Exterior states of the two boundary facets of [-5, 5] (slots in the
    order of line_mesh's meta["boundary_slots"]): the supersonic inflow state
    at x = -5 and the undisturbed right state at x = 5, which no wave reaches
    before t = 1.8 (the shock is near x = 2.4 then).  (2, n_c) conservative."""
    rl, ul, pl = SHU_OSHER_LEFT
    rr, ur, pr = shu_osher_right(np.array([5.0]))
    left = prim_to_cons(np.array([rl]), np.array([[ul]]), np.array([pl]), gam)[:, 0]
    right = prim_to_cons(rr, ur[None], pr, gam)[:, 0]
    return np.stack([left, right])
