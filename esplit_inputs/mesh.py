"""Structured periodic meshes of curved triangles with nodal metric data.

Sec. 7.3 builds its 2D grids by cutting rectangles into two triangles and
perturbing node positions; Assumption 1 requires a polynomial map of degree
p_geom <= p + 1 (2D), so a quadratic (6-node) geometry is used for every p.
The perturbation is periodic, x_i = xhat_i + A prod_j sin(2 pi xhat_j / L),
applied to the geometry nodes, which keeps shared edges identical on both
sides (the edge curve depends only on its three geometry nodes).

Per element and SBP node the mesh stores (all float64):

* ``x``    (n_e, d, n_p)      physical node coordinates,
* ``J``    (n_e, n_p)         mapping Jacobian determinant,
* ``Lam``  (n_e, d, d, n_p)   Lam[i, j] = J dxi_j/dx_i (cofactors; degree 1
                               for a quadratic map, so the discrete metric
                               identity sum_j D_xi_j Lam_ij = 0 holds exactly),
* ``nu``   (n_e, n_fac, n_f, d) scaled outward normal at facet slots,
                               nu_i = Bhat sum_j Lam_ij nhat_j (= b * n_i),
* ``pair`` (n_e, n_fac, n_f, 2) int32: (neighbour element, neighbour flat
                               slot) of the coincident facet node,
* ``hmin`` (n_e,)             smallest node-to-node distance in the element.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .sbp import RefOperator


@dataclass
class Mesh:
    d: int
    n_e: int
    n_p: int
    n_fac: int
    n_f: int
    L: tuple
    x: np.ndarray
    J: np.ndarray
    Lam: np.ndarray
    nu: np.ndarray
    pair: np.ndarray
    hmin: np.ndarray
    meta: dict = field(default_factory=dict)

    def subset_info(self):
        return dict(d=self.d, n_e=self.n_e, n_p=self.n_p, n_fac=self.n_fac, n_f=self.n_f)


def _quad_shape(xi: np.ndarray):
    """Quadratic Lagrange shape functions on the reference triangle and their
    derivatives. Geometry node order: v0, v1, v2, m01, m12, m20."""
    x, y = xi[:, 0], xi[:, 1]
    l0, l1, l2 = 1.0 - x - y, x, y
    N = np.stack([l0 * (2 * l0 - 1), l1 * (2 * l1 - 1), l2 * (2 * l2 - 1),
                  4 * l0 * l1, 4 * l1 * l2, 4 * l2 * l0], axis=1)
    # d/dx: dl0=-1, dl1=1, dl2=0 ; d/dy: dl0=-1, dl1=0, dl2=1
    dNx = np.stack([-(4 * l0 - 1), 4 * l1 - 1, 0 * x,
                    4 * (l0 - l1), 4 * l2, -4 * l2], axis=1)
    dNy = np.stack([-(4 * l0 - 1), 0 * x, 4 * l2 - 1,
                    -4 * l1, 4 * l1, 4 * (l0 - l2)], axis=1)
    return N, np.stack([dNx, dNy])  # (n_p, 6), (2, n_p, 6)


def periodic_tri_mesh(op: RefOperator, N: int, L: float = 10.0, amp: float = 0.05) -> Mesh:
    """Periodic [0, L]^2 mesh of N x N quads, each cut along its lower-left to
    upper-right diagonal into two curved triangles (2 N^2 elements).

    Element numbering: e = 2 (j N + i) + t for quad (i, j), t = 0 for
    (A, B, C) and t = 1 for (A, C, D), A = (i, j), B = (i+1, j), C = (i+1, j+1),
    D = (i, j+1), all counter-clockwise.
    """
    assert op.d == 2
    h = L / N
    n_e = 2 * N * N
    # half-lattice indices (units of h/2) of the 6 geometry nodes per element
    I = np.zeros((n_e, 6), dtype=np.int64)
    Jx = np.zeros((n_e, 6), dtype=np.int64)
    for j in range(N):
        for i in range(N):
            A, B, C, D = (2 * i, 2 * j), (2 * i + 2, 2 * j), (2 * i + 2, 2 * j + 2), (2 * i, 2 * j + 2)
            for t, (a, b, c) in enumerate([(A, B, C), (A, C, D)]):
                e = 2 * (j * N + i) + t
                nodes = [a, b, c,
                         ((a[0] + b[0]) // 2, (a[1] + b[1]) // 2),
                         ((b[0] + c[0]) // 2, (b[1] + c[1]) // 2),
                         ((c[0] + a[0]) // 2, (c[1] + a[1]) // 2)]
                I[e] = [q[0] for q in nodes]
                Jx[e] = [q[1] for q in nodes]
    # periodic displacement evaluated on the wrapped lattice index so that
    # periodic images get bitwise identical displacements
    s = np.sin(2.0 * np.pi * (I % (2 * N)) / (2 * N)) * np.sin(2.0 * np.pi * (Jx % (2 * N)) / (2 * N))
    disp = amp * s
    G = np.stack([I * (h / 2) + disp, Jx * (h / 2) + disp], axis=1)  # (n_e, 2, 6)

    Nsh, dN = _quad_shape(op.xi)
    x = np.einsum("pa,eia->eip", Nsh, G)                     # (n_e, 2, n_p)
    Jm = np.einsum("jpa,eia->eijp", dN, G)                   # dx_i/dxi_j  (n_e, 2, 2, n_p)
    det = Jm[:, 0, 0] * Jm[:, 1, 1] - Jm[:, 0, 1] * Jm[:, 1, 0]
    Lam = np.empty_like(Jm)
    Lam[:, 0, 0] = Jm[:, 1, 1]
    Lam[:, 0, 1] = -Jm[:, 1, 0]
    Lam[:, 1, 0] = -Jm[:, 0, 1]
    Lam[:, 1, 1] = Jm[:, 0, 0]

    fn = op.facet_nodes
    nu = np.zeros((n_e, op.n_fac, op.n_f, 2))
    for g in range(op.n_fac):
        for k in range(op.n_f):
            m = fn[g, k]
            nu[:, g, k, :] = op.facet_w[g, k] * np.einsum("eij,j->ei", Lam[:, :, :, m], op.ref_normals[g])

    # facet pairing: an edge is identified by its midpoint's half-lattice index
    # modulo the period; both sides traverse it counter-clockwise, i.e. in
    # opposite directions, so slot k meets slot n_f - 1 - k.
    mid_of_facet = [3, 4, 5]
    owners: dict = {}
    for e in range(n_e):
        for g in range(op.n_fac):
            key = (int(I[e, mid_of_facet[g]] % (2 * N)), int(Jx[e, mid_of_facet[g]] % (2 * N)))
            owners.setdefault(key, []).append((e, g))
    pair = np.full((n_e, op.n_fac, op.n_f, 2), -1, dtype=np.int32)
    for key, lst in owners.items():
        assert len(lst) == 2, (key, lst)
        (e0, g0), (e1, g1) = lst
        for k in range(op.n_f):
            kk = op.n_f - 1 - k
            pair[e0, g0, k] = (e1, g1 * op.n_f + kk)
            pair[e1, g1, kk] = (e0, g0 * op.n_f + k)

    diff = x[:, :, :, None] - x[:, :, None, :]
    dist = np.sqrt((diff ** 2).sum(1))
    dist[:, np.arange(op.n_p), np.arange(op.n_p)] = np.inf
    hmin = dist.reshape(n_e, -1).min(1)
    return Mesh(d=2, n_e=n_e, n_p=op.n_p, n_fac=op.n_fac, n_f=op.n_f, L=(L, L),
                x=x, J=det, Lam=Lam, nu=nu, pair=pair, hmin=hmin,
                meta=dict(kind="periodic_tri", N=N, L=L, amp=amp, p=op.p))
