"""L^2 error of a nodal solution on curved triangles and tetrahedra, as
Secs. 7.3 and 7.4 measure it: the solution is carried from the SBP nodes to a quadrature rule of
degree 3p + 1 on each element (here the H-weighted least-squares fit of
degree p, exact for degree-p data), the square of the error summed over the
conservative variables is integrated with the element's Jacobian, summed
over the elements, and the square root taken.

Quadrature: the collapsed (Duffy) product of n-point Gauss-Legendre rules,
x = u, y = v (1 - u), weight w_u w_v (1 - u), exact for polynomials of total
degree 2n - 2 on the reference triangle.
"""
import numpy as np

from esplit_inputs.sbp import vandermonde
from esplit_inputs.states import isentropic_vortex_prims, prim_to_cons


def triangle_rule(degree):
    n = degree // 2 + 2
    g, w = np.polynomial.legendre.leggauss(n)
    g, w = 0.5 * (g + 1.0), 0.5 * w
    U, Vv = np.meshgrid(g, g, indexing="ij")
    WU, WV = np.meshgrid(w, w, indexing="ij")
    xi = np.stack([U.ravel(), (Vv * (1.0 - U)).ravel()], axis=1)
    wt = (WU * WV * (1.0 - U)).ravel()
    return xi, wt


def _quad_shape(xi):
    x, y = xi[:, 0], xi[:, 1]
    l0, l1, l2 = 1.0 - x - y, x, y
    N = np.stack([l0 * (2 * l0 - 1), l1 * (2 * l1 - 1), l2 * (2 * l2 - 1), 4 * l0 * l1, 4 * l1 * l2, 4 * l2 * l0], 1)
    dNx = np.stack([-(4 * l0 - 1), 4 * l1 - 1, 0 * x, 4 * (l0 - l1), 4 * l2, -4 * l2], 1)
    dNy = np.stack([-(4 * l0 - 1), 0 * x, 4 * l2 - 1, -4 * l1, 4 * l1, 4 * (l0 - l2)], 1)
    return N, dNx, dNy


def l2_error_2d(u, op, mesh, prims):
    """sqrt(sum_e int_e sum_c (u_h,c - u_c)^2) on curved triangles, the exact
    solution given by prims(X (2, ...)) -> (rho, V (2, ...), p)."""
    p = op.p
    xq, wq = triangle_rule(3 * p + 1)
    ctr = np.full(2, 1.0 / 3.0)
    Vn, _ = vandermonde(op.xi, p, ctr)
    Vq, _ = vandermonde(xq, p, ctr)
    H = op.H
    fit = Vq @ np.linalg.solve(Vn.T @ (H[:, None] * Vn), Vn.T * H[None, :])     # (n_q, n_p)
    uq = np.einsum("qm,ecm->ecq", fit, u)
    G = mesh.meta["geom"]                                                        # (n_e, 2, 6)
    N, dNx, dNy = _quad_shape(xq)
    X = np.einsum("qa,eia->eiq", N, G)
    dxs = np.einsum("qa,eia->eiq", dNx, G)
    dys = np.einsum("qa,eia->eiq", dNy, G)
    J = dxs[:, 0] * dys[:, 1] - dys[:, 0] * dxs[:, 1]
    rho, V, pr = prims(np.moveaxis(X, 1, 0))
    ue = np.moveaxis(prim_to_cons(rho, V, pr), 0, 1)                             # (n_e, n_c, n_q)
    err2 = np.einsum("q,eq,ecq->", wq, J, (uq - ue) ** 2)
    return float(np.sqrt(err2))


def l2_error_vortex(u, op, mesh, t, center=(5.0, 0.0)):
    """sqrt(sum_e int_e sum_c (u_h,c - u_c(t))^2) for the Sec. 7.3 vortex."""
    return l2_error_2d(u, op, mesh, lambda X: isentropic_vortex_prims(X[0], X[1], t=t, xc=center[0],
                                                                      yc=center[1]))


def tet_rule(degree):
    """Collapsed Gauss rule on the reference tetrahedron (vertices 0, e1, e2,
    e3): x = u, y = v (1 - u), z = w (1 - u)(1 - v), weight (1-u)^2 (1-v)."""
    n = degree // 2 + 2
    g, w = np.polynomial.legendre.leggauss(n)
    g, w = 0.5 * (g + 1.0), 0.5 * w
    U, Vv, Wd = np.meshgrid(g, g, g, indexing="ij")
    WU, WV, WW = np.meshgrid(w, w, w, indexing="ij")
    xi = np.stack([U.ravel(), (Vv * (1 - U)).ravel(), (Wd * (1 - U) * (1 - Vv)).ravel()], axis=1)
    wt = (WU * WV * WW * (1 - U) ** 2 * (1 - Vv)).ravel()
    return xi, wt


def l2_error_3d(u, op, mesh, prims, chunk=4096):
    """The L^2 error on curved tetrahedra, exact solution prims(X (3, ...));
    ``u`` may be a list of states on the same mesh (one error each, one pass
    over the geometry)."""
    if isinstance(u, (list, tuple)):
        return _l2_errors_3d(list(u), op, mesh, prims, chunk)
    return _l2_errors_3d([u], op, mesh, prims, chunk)[0]


def _l2_errors_3d(us, op, mesh, prims, chunk):
    from esplit_inputs.mesh import _quad_tet_shape
    p = op.p
    xq, wq = tet_rule(3 * p + 1)
    ctr = np.full(3, 0.25)
    Vn, _ = vandermonde(op.xi, p, ctr)
    Vq, _ = vandermonde(xq, p, ctr)
    H = op.H
    fit = Vq @ np.linalg.solve(Vn.T @ (H[:, None] * Vn), Vn.T * H[None, :])
    N, dN = _quad_tet_shape(xq)                                         # (q, 10), (3, q, 10)
    G = mesh.meta["geom"]                                               # (n_e, 3, 10)
    total = np.zeros(len(us))
    for a in range(0, mesh.n_e, chunk):
        Gc = G[a:a + chunk]
        X = np.einsum("qa,eia->eiq", N, Gc)
        Jm = np.einsum("jqa,eia->eqij", dN, Gc)
        J = np.linalg.det(Jm)
        rho, V, pr = prims(np.moveaxis(X, 1, 0))
        ue = np.moveaxis(prim_to_cons(rho, V, pr), 0, 1)
        for k, u in enumerate(us):
            uq = np.einsum("qm,ecm->ecq", fit, u[a:a + chunk])
            total[k] += float(np.einsum("q,eq,ecq->", wq, J, (uq - ue) ** 2))
    return [float(np.sqrt(t)) for t in total]


def l2_error_vortex_3d(u, op, mesh, t, chunk=4096):
    """The Sec. 7.3 L^2 error for the 3D vortex on curved tetrahedra."""
    from esplit_inputs.states import vortex3d_prims
    return l2_error_3d(u, op, mesh, lambda X: vortex3d_prims(X[0], X[1], t), chunk)
