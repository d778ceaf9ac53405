"""Troubled-element detector for the hybrid scheme (plain numpy, float64).

Test infrastructure: imported only by tests/, the smoke check and bench.py's
CPU legs.

Sec. 4.4 builds the hybrid scheme (Thm. 4: any per-element choice between
the entropy-split and the Hadamard volume terms keeps entropy conservation)
and leaves the choice of the Hadamard elements open.  Reading used here: an
element k is troubled when, over its own nodes and the neighbours' facet
nodes coincident with its facet nodes,

    max p / min p > threshold   (threshold 1.1),

or a pressure there is not positive and finite; the flagged set is then
widened by one layer of face neighbours.  The pressure is
p = (gam - 1)(e - (0.5 |m|^2) / rho), each operation rounded to nearest in
float64 in exactly this order (|m|^2 summed left to right), so that the
integer decision is taken in the same precision on both sides.

Pins (tests/test_oracle_hybrid.py): a pure-Python loop over elements on a
small mesh gives the same flags; uniform and smooth states flag nothing; a
single perturbed node flags its element, the elements whose facet nodes
touch it, and their face neighbours; non-positive pressure flags.
"""
from __future__ import annotations

import numpy as np


def detector_pressure(u, gam=1.4):
    """p = (gam-1) (e - (0.5 |m|^2)/rho) for u (..., n_c, n_p) -> (..., n_p)."""
    u = np.asarray(u, dtype=np.float64)
    d = u.shape[-2] - 2
    rho = u[..., 0, :]
    s = u[..., 1, :] * u[..., 1, :]
    for i in range(1, d):
        s = s + u[..., 1 + i, :] * u[..., 1 + i, :]
    k = (0.5 * s) / rho
    return (gam - 1.0) * (u[..., d + 1, :] - k)


def detect(u, ref, mesh, threshold=1.1, gam=1.4):
    """Flags (uint8, n_e): the pressure-ratio sensor above, widened by one
    layer of face neighbours."""
    p = detector_pressure(u, gam)                               # (n_e, n_p)
    fn = np.asarray(ref.facet_nodes).reshape(-1)
    pair = np.asarray(mesh.pair).reshape(mesh.n_e, -1, 2)       # (n_e, n_slot, 2)
    # boundary facets (pair (-1, -1)) have no neighbour: their own facet node
    # stands in for it (it changes neither the max nor the min) and they widen nothing
    own = np.broadcast_to(np.arange(mesh.n_e)[:, None], pair.shape[:2])
    bnd = pair[..., 0] < 0
    nb_e = np.where(bnd, own, pair[..., 0])
    nb_n = np.where(bnd, fn[None, :], fn[np.maximum(pair[..., 1], 0)])
    p_nb = p[nb_e, nb_n]                                        # neighbours' coincident facet nodes
    allp = np.concatenate([p, p_nb], axis=1)
    good = np.all((allp > 0) & (allp < np.inf), axis=1)
    with np.errstate(invalid="ignore", divide="ignore"):
        ratio = allp.max(axis=1) / allp.min(axis=1)
    flag0 = ~good | ~(ratio <= threshold)
    flags = flag0 | np.any(flag0[nb_e], axis=1)
    return flags.astype(np.uint8)
