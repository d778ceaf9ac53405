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
    # the map's derivatives from element-local offsets (the shape-function
    # derivatives sum to zero): lattice differences are exact and displacement
    # differences carry rounding of the displacement's size, where G itself is
    # rounded at the size of the domain
    dG = np.stack([(I - I[:, :1]) * (h / 2) + (disp - disp[:, :1]),
                   (Jx - Jx[:, :1]) * (h / 2) + (disp - disp[:, :1])], axis=1)

    Nsh, dN = _quad_shape(op.xi)
    x = np.einsum("pa,eia->eip", Nsh, G)                     # (n_e, 2, n_p)
    Jm = np.einsum("jpa,eia->eijp", dN, dG)                  # dx_i/dxi_j  (n_e, 2, 2, n_p)
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


def chan_warp(xh, yh):
    """Perturbation of the 2D vortex grids of Sec. 7.3 (the paper takes it from
    Chan et al.) on [0, 20] x [-5, 5]:
        x1 = xh1 + 1/8 cos(pi/20 (xh1 - 10)) cos(3 pi/10 xh2),
        x2 = xh2 + 1/8 sin(pi/5 (x1 - 10)) cos(pi/10 xh2),
    x2 using the perturbed x1.  Returns the displacements."""
    dx = 0.125 * np.cos(np.pi / 20.0 * (xh - 10.0)) * np.cos(0.3 * np.pi * yh)
    x1 = xh + dx
    dy = 0.125 * np.sin(np.pi / 5.0 * (x1 - 10.0)) * np.cos(np.pi / 10.0 * yh)
    return dx, dy


def periodic_tri_mesh_rect(op: RefOperator, Nx: int, Ny: int, origin=(0.0, -5.0), size=(20.0, 10.0),
                           warp=chan_warp) -> Mesh:
    """Periodic rectangle [x0, x0 + Lx] x [y0, y0 + Ly] of Nx x Ny rectangles,
    each cut along its lower-left to upper-right diagonal into two curved
    triangles (2 Nx Ny elements), quadratic geometry displaced by
    warp(xh, yh) -> (dx, dy) evaluated at the unperturbed geometry nodes (on
    the wrapped lattice, so periodic images move identically; the warp must
    be periodic).  Element numbering as periodic_tri_mesh; the geometry nodes
    are kept in meta["geom"] (n_e, 2, 6) for error integration."""
    assert op.d == 2
    Lx, Ly = size
    hx, hy = Lx / Nx, Ly / Ny
    n_e = 2 * Nx * Ny
    I = np.zeros((n_e, 6), dtype=np.int64)
    Jx = np.zeros((n_e, 6), dtype=np.int64)
    for j in range(Ny):
        for i in range(Nx):
            A, B, C, D = (2 * i, 2 * j), (2 * i + 2, 2 * j), (2 * i + 2, 2 * j + 2), (2 * i, 2 * j + 2)
            for t, (a, b, c) in enumerate([(A, B, C), (A, C, D)]):
                e = 2 * (j * Nx + i) + t
                nodes = [a, b, c,
                         ((a[0] + b[0]) // 2, (a[1] + b[1]) // 2),
                         ((b[0] + c[0]) // 2, (b[1] + c[1]) // 2),
                         ((c[0] + a[0]) // 2, (c[1] + a[1]) // 2)]
                I[e] = [q[0] for q in nodes]
                Jx[e] = [q[1] for q in nodes]
    xw = origin[0] + (I % (2 * Nx)) * (hx / 2)
    yw = origin[1] + (Jx % (2 * Ny)) * (hy / 2)
    ddx, ddy = warp(xw, yw)
    G = np.stack([origin[0] + I * (hx / 2) + ddx, origin[1] + Jx * (hy / 2) + ddy], axis=1)  # (n_e, 2, 6)
    # derivatives from element-local offsets (see periodic_tri_mesh)
    dG = np.stack([(I - I[:, :1]) * (hx / 2) + (ddx - ddx[:, :1]),
                   (Jx - Jx[:, :1]) * (hy / 2) + (ddy - ddy[:, :1])], axis=1)

    Nsh, dN = _quad_shape(op.xi)
    x = np.einsum("pa,eia->eip", Nsh, G)
    Jm = np.einsum("jpa,eia->eijp", dN, dG)
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
    mid_of_facet = [3, 4, 5]
    owners: dict = {}
    for e in range(n_e):
        for g in range(op.n_fac):
            key = (int(I[e, mid_of_facet[g]] % (2 * Nx)), int(Jx[e, mid_of_facet[g]] % (2 * Ny)))
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
    return Mesh(d=2, n_e=n_e, n_p=op.n_p, n_fac=op.n_fac, n_f=op.n_f, L=(Lx, Ly),
                x=x, J=det, Lam=Lam, nu=nu, pair=pair, hmin=hmin,
                meta=dict(kind="periodic_tri_rect", Nx=Nx, Ny=Ny, origin=tuple(origin), size=(Lx, Ly),
                          p=op.p, geom=G))


def _quad_tet_shape(xi: np.ndarray):
    """Quadratic (10-node) Lagrange shape functions on the reference tetrahedron
    and their derivatives. Geometry node order: v0..v3, then the edge midpoints
    m01, m02, m03, m12, m13, m23."""
    l = [1.0 - xi[:, 0] - xi[:, 1] - xi[:, 2], xi[:, 0], xi[:, 1], xi[:, 2]]
    dl = np.array([[-1.0, -1.0, -1.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])  # d lambda_a / d xi_j
    edges = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    N = [l[a] * (2 * l[a] - 1) for a in range(4)] + [4 * l[a] * l[b] for a, b in edges]
    dN = np.zeros((3, len(xi), 10))
    for j in range(3):
        for a in range(4):
            dN[j, :, a] = (4 * l[a] - 1) * dl[a, j]
        for e, (a, b) in enumerate(edges):
            dN[j, :, 4 + e] = 4 * (dl[a, j] * l[b] + l[a] * dl[b, j])
    return np.stack(N, axis=1), dN


def mms_warp_2d(xh, yh):
    """Perturbation of the manufactured-solution grids of Sec. 7.4 on
    [-1, 1]^2 (the paper takes it from Chan et al.):
        x_i = xh_i + 1/8 cos(pi xh_i / 2) prod_{j != i} sin(pi xh_j).
    It vanishes on the boundary, so periodic images stay paired.  Returns
    the displacements (dx, dy)."""
    dx = 0.125 * np.cos(0.5 * np.pi * xh) * np.sin(np.pi * yh)
    dy = 0.125 * np.cos(0.5 * np.pi * yh) * np.sin(np.pi * xh)
    return dx, dy


def mms_warp_3d(xh):
    """The Sec. 7.4 perturbation on [-1, 1]^3, xh (..., 3) -> displacements:
    dx_i = 1/8 cos(pi xh_i / 2) prod_{j != i} sin(pi xh_j)."""
    c = np.cos(0.5 * np.pi * xh)
    sn = np.sin(np.pi * xh)
    out = np.empty_like(xh)
    for i in range(3):
        j, k = [a for a in range(3) if a != i]
        out[..., i] = 0.125 * c[..., i] * sn[..., j] * sn[..., k]
    return out


def vortex3d_warp(xh):
    """Perturbation of the 3D vortex grids of Sec. 7.3 on [-10, 10]^3:
    x_i = xh_i + 0.05 sin(pi xh_i / 2).  xh (..., 3) -> displacements."""
    return 0.05 * np.sin(0.5 * np.pi * xh)


def periodic_tet_mesh(op: RefOperator, N: int, L: float = 2 * np.pi, amp: float = 0.02, origin=0.0,
                      warp=None) -> Mesh:
    """Periodic [x0, x0 + L]^3 mesh of N^3 cubes, each cut into the six Kuhn
    tetrahedra around its main diagonal (6 N^3 elements), quadratic geometry
    (affine for p = 1) warped by x_i = xhat_i + A prod_j sin(2 pi (xhat_j - x0) / L) or, when
    given, by warp(xhat) -> displacements evaluated on the wrapped lattice
    (Sec. 7.3 builds its 3D grids the same way: hexahedra cut into six
    tetrahedra, then perturbed).  Facet nodes are paired by their (unwarped)
    positions modulo L; the geometry nodes are kept in meta["geom"]."""
    import itertools
    assert op.d == 3
    h = L / N
    perms = list(itertools.permutations(range(3)))
    n_e = 6 * N ** 3
    ii, jj, kk = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    base = 2 * np.stack([ii.ravel(order="F"), jj.ravel(order="F"), kk.ravel(order="F")], axis=1)  # i fastest
    V = np.zeros((N ** 3, 6, 4, 3), dtype=np.int64)  # vertex half-lattice indices
    for t, sgm in enumerate(perms):
        cur = base.copy()
        V[:, t, 0] = cur
        for a, ax in enumerate(sgm):
            cur = cur.copy()
            cur[:, ax] += 2
            V[:, t, a + 1] = cur
    V = V.reshape(n_e, 4, 3)
    # positive orientation: swap the last two vertices where needed
    d1, d2, d3 = V[:, 1] - V[:, 0], V[:, 2] - V[:, 0], V[:, 3] - V[:, 0]
    vol = np.einsum("ei,ei->e", d1, np.cross(d2, d3))
    neg = vol < 0
    V[neg, 2], V[neg, 3] = V[neg, 3].copy(), V[neg, 2].copy()
    edges = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    G_idx = np.concatenate([V, np.stack([(V[:, a] + V[:, b]) // 2 for a, b in edges], axis=1)], axis=1)  # (e,10,3)
    wrap = G_idx % (2 * N)
    if warp is None:
        s = np.prod(np.sin(2.0 * np.pi * wrap / (2 * N)), axis=2)  # (e, 10)
        disp = amp * s[..., None]
    else:
        disp = warp(origin + wrap * (h / 2))
    if op.p == 1:
        # degree-1 operators: affine elements (edge nodes at the midpoints of
        # the displaced vertices).  The metric terms J dxi/dx of a quadratic
        # map are cofactors of its Jacobian, quadratic in 3D, and the discrete
        # metric identities of Sec. 2 need D exact on them.
        disp = np.concatenate([disp[:, :4], np.stack([0.5 * (disp[:, a] + disp[:, b]) for a, b in edges], 1)], 1)
    G = origin + G_idx * (h / 2) + disp                        # (e, 10, 3)
    G = np.transpose(G, (0, 2, 1))                             # (e, 3, 10)
    # derivatives from element-local offsets (see periodic_tri_mesh)
    dG = np.transpose((G_idx - G_idx[:, :1]) * (h / 2) + (disp - disp[:, :1]), (0, 2, 1))
    Nsh, dN = _quad_tet_shape(op.xi)
    x = np.einsum("pa,eia->eip", Nsh, G)
    Jm = np.einsum("jpa,eia->eijp", dN, dG)                    # dx_i/dxi_j (e, 3, 3, n_p)
    Jt = np.transpose(Jm, (0, 3, 1, 2))                        # (e, n_p, 3, 3)
    det = np.linalg.det(Jt)
    adj = np.linalg.inv(Jt) * det[..., None, None]             # adj[j][i] = J dxi_j/dx_i
    # Lam[e, i, j, p] = adj[e, p, j, i]
    Lam = np.ascontiguousarray(np.transpose(np.transpose(adj, (0, 1, 3, 2)), (0, 2, 3, 1)))
    fn = op.facet_nodes
    nu = np.zeros((n_e, op.n_fac, op.n_f, 3))
    for g in range(op.n_fac):
        for kk in range(op.n_f):
            mnode = fn[g, kk]
            nu[:, g, kk, :] = op.facet_w[g, kk] * np.einsum("eij,j->ei", Lam[:, :, :, mnode], op.ref_normals[g])
    # pairing by straight positions modulo L
    Gs = np.transpose(G_idx * (h / 2), (0, 2, 1)).astype(float)  # unwarped geometry nodes
    xs = np.einsum("pa,eia->eip", Nsh, Gs)                         # straight node positions
    slots = fn.reshape(-1)
    key = np.round(xs[:, :, slots] / L * 2 ** 30).astype(np.int64) % (2 ** 30)  # (e, 3, n_slot)
    n_slot = op.n_fac * op.n_f
    kf = key.transpose(0, 2, 1).reshape(-1, 3)               # (n_e n_slot, 3)
    order = np.lexsort((kf[:, 2], kf[:, 1], kf[:, 0]))
    ks = kf[order]
    a, b = order[0::2], order[1::2]
    assert np.all(ks[0::2] == ks[1::2]), "facet nodes must coincide in pairs"
    if len(ks) > 2:
        assert not np.any(np.all(ks[2::2] == ks[1:-1:2], axis=1)), "a facet node is shared by more than two slots"
    pair = np.full((n_e * n_slot, 2), -1, dtype=np.int32)
    pair[a, 0], pair[a, 1] = b // n_slot, b % n_slot
    pair[b, 0], pair[b, 1] = a // n_slot, a % n_slot
    pair = pair.reshape(n_e, op.n_fac, op.n_f, 2)
    hmin = np.empty(n_e)
    ch = max(1, (1 << 24) // (op.n_p * op.n_p))    # elements per chunk of the pairwise distances
    for e0 in range(0, n_e, ch):
        xe = x[e0:e0 + ch]
        diff = xe[:, :, :, None] - xe[:, :, None, :]
        dist = np.sqrt((diff ** 2).sum(1))
        dist[:, np.arange(op.n_p), np.arange(op.n_p)] = np.inf
        hmin[e0:e0 + ch] = dist.reshape(len(xe), -1).min(1)
    return Mesh(d=3, n_e=n_e, n_p=op.n_p, n_fac=op.n_fac, n_f=op.n_f, L=(L, L, L), x=x, J=det, Lam=Lam, nu=nu,
                pair=pair, hmin=hmin, meta=dict(kind="periodic_tet", N=N, L=L, amp=amp, p=op.p, origin=origin,
                                                 geom=G))


def periodic_line_mesh(op: RefOperator, N: int, L: float = 1.0, origin: float = 0.0, amp: float = 0.0) -> Mesh:
    """Periodic [x0, x0 + L) cut into N elements, vertices moved by
    amp * h * sin(2 pi (x_k - x0) / L) (amp = 0: uniform).  Element k maps the
    reference interval affinely onto [x_k, x_k+1]: J = h_k, Lam = J dxi/dx = 1,
    nu = -1 at facet 0 (left end) and +1 at facet 1; facet 1 of element k
    pairs with facet 0 of element k + 1 (periodically)."""
    assert op.d == 1
    h0 = L / N
    xv = origin + h0 * np.arange(N + 1)
    xv = xv + amp * h0 * np.sin(2.0 * np.pi * (xv - origin) / L)
    xv[-1] = xv[0] + L
    h = np.diff(xv)
    x = (xv[:-1, None] + h[:, None] * op.xi[None, :, 0])[:, None, :]     # (n_e, 1, n_p)
    J = np.repeat(h[:, None], op.n_p, axis=1)
    Lam = np.ones((N, 1, 1, op.n_p))
    nu = np.zeros((N, 2, 1, 1))
    nu[:, 0, 0, 0] = -1.0
    nu[:, 1, 0, 0] = 1.0
    pair = np.zeros((N, 2, 1, 2), dtype=np.int32)
    k = np.arange(N)
    pair[:, 0, 0, 0] = (k - 1) % N      # left end: the previous element's facet 1 (slot 1)
    pair[:, 0, 0, 1] = 1
    pair[:, 1, 0, 0] = (k + 1) % N      # right end: the next element's facet 0 (slot 0)
    pair[:, 1, 0, 1] = 0
    xs = np.sort(op.xi[:, 0])
    hmin = h * np.diff(xs).min()
    return Mesh(d=1, n_e=N, n_p=op.n_p, n_fac=2, n_f=1, L=(L,), x=x, J=J, Lam=Lam, nu=nu, pair=pair, hmin=hmin,
                meta=dict(kind="periodic_line", N=N, L=L, amp=amp, p=op.p, origin=origin, vertices=xv))


def line_mesh(op: RefOperator, N: int, L: float = 1.0, origin: float = 0.0, amp: float = 0.0) -> Mesh:
    """The interval [x0, x0 + L] cut into N elements as periodic_line_mesh
    does, with two boundary facets instead of the periodic wrap: facet 0 of
    element 0 (x = x0, nu = -1) and facet 1 of element N - 1 (x = x0 + L,
    nu = +1) pair with no element, marked (-1, -1) in ``pair``; their flat
    slot indices (element * 2 + facet) are meta["boundary_slots"] = [0, 2N - 1]."""
    m = periodic_line_mesh(op, N, L, origin, amp)
    m.pair[0, 0, 0] = (-1, -1)
    m.pair[N - 1, 1, 0] = (-1, -1)
    m.meta["kind"] = "line"
    m.meta["boundary_slots"] = np.array([0, 2 * N - 1], dtype=np.int32)
    return m
