"""Reference diagonal-E SBP operators on the reference triangle, the
reference tetrahedron and the reference interval (the last two in their own
sections below).

Definition 1 (Sec. 2.1) asks for D_xi = H^-1 Q_xi exact on P^p, H symmetric
positive definite, Q_xi = S_xi + E_xi/2 with S_xi skew and E_xi symmetric and
exact for boundary integrals of degree >= 2p products.  Sec. 2.1 restricts the
paper to diagonal H (a positive volume quadrature of degree >= 2p-1) and
diagonal E built facet by facet, E_xi = sum_g R_g^T B_g N_xi,g R_g, with the
facet quadrature (degree >= 2p) collocated with volume nodes.

The paper takes its node sets from the literature and prints none, so the sets
here are constructed from scratch:

* facet nodes: p+1 Gauss-Legendre points on every edge (degree 2p+1 >= 2p),
  symmetric about the edge midpoint so that two elements sharing an edge see
  the same physical points in reversed order; no vertex is a facet node, so
  every facet node belongs to exactly one facet;
* volume quadrature: an S3-symmetric positive rule that contains the edge
  nodes plus interior orbits, solved from the moment equations.  The solved
  orbit parameters are tabulated below (degree 2, 4, 5, 7 for p = 1..4;
  7, 12, 18, 27 nodes); ``solve_tri_quadrature`` re-derives them;
* S_xi: the minimum-norm skew matrix satisfying S V = H V_xi - E V / 2 on a
  P^p basis V (the accuracy conditions of Def. 1 rearranged).

Node ordering: the 3*(p+1) facet nodes first, facet by facet, each facet
traversed counter-clockwise (facet 0: (0,0)->(1,0), facet 1: (1,0)->(0,1),
facet 2: (0,1)->(0,0)), then the interior nodes.  Facet slot s therefore is
volume node s.
"""
from __future__ import annotations

from dataclasses import dataclass
from math import factorial

import numpy as np

# Tabulated orbit parameters, from ``solve_tri_quadrature`` (maximal smallest
# weight over seeded restarts).  Layout: edge orbit weights (one per pair of
# Gauss points t, 1-t, plus the midpoint orbit for even p+1 counts... ordered
# from the edge ends inwards), then per interior orbit its parameters.
_TRI_RULES = {
    1: dict(degree=2, interior=["S3"],
            x=[0.04166666666666667, 0.24999999999999997]),
    2: dict(degree=4, interior=["S21"],
            x=[0.012602515726039517, 0.02920240803236734, 0.20468064157076205,
               0.11225922718222028]),
    3: dict(degree=5, interior=["S21", "S21"],
            x=[0.007492641905837701, 0.0201774931715975, 0.2042412290450176,
               0.10294430361869249, 0.41941492873303443, 0.008382092893103772]),
    4: dict(degree=7, interior=["S111", "S21", "S21"],
            x=[0.0033172873454619376, 0.00771492016905887, 0.012269478590616632,
               0.09553488276835435, 0.7266791896728819, 0.028664781336347603,
               0.30073644818112955, 0.003531850203707962, 0.4246122619422098,
               0.07147136017060525]),
}

_TRI_VERTS = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
# outward unit normals and lengths of the three reference edges
_TRI_NORMALS = np.array([[0.0, -1.0], [1.0, 1.0], [-1.0, 0.0]])
_TRI_NORMALS[1] /= np.sqrt(2.0)
_TRI_LENGTHS = np.array([1.0, np.sqrt(2.0), 1.0])


def gauss_legendre01(n: int):
    """n-point Gauss-Legendre rule on [0, 1] (points ascending, weights sum 1)."""
    x, w = np.polynomial.legendre.leggauss(n)
    return (x + 1.0) / 2.0, w / 2.0


def _edge_orbits(nf: int):
    """Group Gauss points k of an edge into symmetric orbits {k, nf-1-k}."""
    orbs = []
    for a in range(nf):
        b = nf - 1 - a
        if a < b:
            orbs.append((a, b))
        elif a == b:
            orbs.append((a,))
    return orbs


def _tri_nodes(p: int, x):
    """Nodes (n_p, 2) and weights (n_p,) of the triangle rule for degree p."""
    rule = _TRI_RULES[p]
    nf = p + 1
    t, _ = gauss_legendre01(nf)
    orbs = _edge_orbits(nf)
    n_eo = len(orbs)
    ew = x[:n_eo]
    pts, wts = [], []
    for gam in range(3):
        a, b = _TRI_VERTS[gam], _TRI_VERTS[(gam + 1) % 3]
        for k in range(nf):
            pts.append(a + t[k] * (b - a))
            oi = [i for i, o in enumerate(orbs) if k in o][0]
            wts.append(ew[oi])
    i = n_eo
    for typ in rule["interior"]:
        if typ == "S3":
            pts.append(np.array([1 / 3, 1 / 3]))
            wts.append(x[i])
            i += 1
        elif typ == "S21":
            a, w = x[i], x[i + 1]
            i += 2
            for lam in [(a, a, 1 - 2 * a), (a, 1 - 2 * a, a), (1 - 2 * a, a, a)]:
                pts.append(np.array([lam[1], lam[2]]))
                wts.append(w)
        elif typ == "S111":
            a, b, w = x[i], x[i + 1], x[i + 2]
            i += 3
            c = 1 - a - b
            for lam in [(a, b, c), (a, c, b), (b, a, c), (b, c, a), (c, a, b), (c, b, a)]:
                pts.append(np.array([lam[1], lam[2]]))
                wts.append(w)
        else:  # pragma: no cover
            raise ValueError(typ)
    return np.array(pts), np.array(wts)


def tri_monomial_integral(i: int, j: int) -> float:
    """Exact integral of x^i y^j over the reference triangle (0,0),(1,0),(0,1)."""
    return factorial(i) * factorial(j) / factorial(i + j + 2)


def solve_tri_quadrature(p: int, degree: int, interior, seed: int = 0, tries: int = 40):
    """Re-derive a tabulated rule: seeded nonlinear least squares on the moment
    equations of all monomials up to ``degree``, keeping the positive rule with
    interior nodes strictly inside and the largest smallest weight."""
    from scipy.optimize import least_squares

    nf = p + 1
    n_eo = len(_edge_orbits(nf))
    mons = [(i, j) for i in range(degree + 1) for j in range(degree + 1 - i)]
    ex = np.array([tri_monomial_integral(i, j) for i, j in mons])
    saved = _TRI_RULES.get(p)
    _TRI_RULES[p] = dict(degree=degree, interior=list(interior), x=None)

    def res(x):
        pts, w = _tri_nodes(p, x)
        return np.array([np.sum(w * pts[:, 0] ** i * pts[:, 1] ** j) for i, j in mons]) - ex

    rng = np.random.default_rng(seed)
    best = None
    try:
        for _ in range(tries):
            x0 = list(rng.uniform(0.001, 0.05, n_eo))
            for typ in interior:
                if typ == "S3":
                    x0 += [rng.uniform(0.01, 0.2)]
                elif typ == "S21":
                    x0 += [rng.uniform(0.05, 0.45), rng.uniform(0.005, 0.1)]
                else:
                    a = rng.uniform(0.05, 0.4)
                    x0 += [a, rng.uniform(0.05, 0.9 - a), rng.uniform(0.005, 0.1)]
            r = least_squares(res, x0, xtol=1e-15, ftol=1e-15, gtol=1e-15, max_nfev=2000)
            pts, w = _tri_nodes(p, r.x)
            ip = pts[3 * nf:]
            inside = len(ip) == 0 or (np.all(ip > 1e-3) and np.all(ip.sum(1) < 1 - 1e-3))
            if np.all(w > 0) and inside and np.abs(res(r.x)).max() < 1e-14:
                if best is None or w.min() > best[0]:
                    best = (w.min(), r.x)
    finally:
        if saved is not None:
            _TRI_RULES[p] = saved
    return None if best is None else best[1]


def monomial_basis(p: int, d: int):
    """Exponent tuples of the monomial basis of P^p in d variables."""
    if d == 1:
        return [(i,) for i in range(p + 1)]
    if d == 2:
        return [(i, j) for tot in range(p + 1) for i in range(tot, -1, -1) for j in [tot - i]]
    if d == 3:
        return [(i, j, k) for tot in range(p + 1) for i in range(tot, -1, -1)
                for j in range(tot - i, -1, -1) for k in [tot - i - j]]
    raise ValueError(d)


def vandermonde(xi: np.ndarray, p: int, center: np.ndarray):
    """Monomial Vandermonde V (n_p x N_p) and its reference derivatives
    V_xi[j] (d x n_p x N_p), in coordinates shifted to ``center``."""
    n, d = xi.shape
    y = xi - center
    basis = monomial_basis(p, d)
    V = np.zeros((n, len(basis)))
    dV = np.zeros((d, n, len(basis)))
    for c, ex in enumerate(basis):
        V[:, c] = np.prod([y[:, a] ** ex[a] for a in range(d)], axis=0)
        for j in range(d):
            if ex[j] == 0:
                continue
            terms = []
            for a in range(d):
                e = ex[a] - (1 if a == j else 0)
                terms.append(y[:, a] ** e)
            dV[j, :, c] = ex[j] * np.prod(terms, axis=0)
    return V, dV


def min_norm_skew(H: np.ndarray, E: np.ndarray, V: np.ndarray, dV: np.ndarray) -> np.ndarray:
    """Minimum-norm skew S solving S V = diag(H) dV - diag(E) V / 2."""
    n, nb = V.shape
    rhs = H[:, None] * dV - 0.5 * E[:, None] * V
    iu = np.triu_indices(n, 1)
    m = len(iu[0])
    A = np.zeros((n * nb, m))
    for col, (a, b) in enumerate(zip(*iu)):
        # S[a,b] = s, S[b,a] = -s ; equation row (r, c): sum_k S[r,k] V[k,c]
        A[a * nb:(a + 1) * nb, col] += V[b, :]
        A[b * nb:(b + 1) * nb, col] -= V[a, :]
    s, *_ = np.linalg.lstsq(A, rhs.reshape(-1), rcond=None)
    S = np.zeros((n, n))
    S[iu] = s
    S -= S.T
    return S


@dataclass
class RefOperator:
    """A reference diagonal-E SBP operator (arrays are float64 / int32).

    d            spatial dimension
    p            degree
    n_p          number of volume nodes
    n_fac, n_f   facets per element, nodes per facet
    xi           (n_p, d) node coordinates on the reference element
    H            (n_p,) diagonal norm (quadrature weights)
    Q            (d, n_p, n_p) Q_xi_j
    E            (d, n_p) diagonal of E_xi_j
    facet_nodes  (n_fac, n_f) volume node index of each facet slot
    facet_w      (n_fac, n_f) facet quadrature weights on the reference facet
    ref_normals  (n_fac, d) outward unit normals of the reference facets
    """

    d: int
    p: int
    n_p: int
    n_fac: int
    n_f: int
    xi: np.ndarray
    H: np.ndarray
    Q: np.ndarray
    E: np.ndarray
    facet_nodes: np.ndarray
    facet_w: np.ndarray
    ref_normals: np.ndarray
    volume_degree: int

    @property
    def D(self) -> np.ndarray:
        return self.Q / self.H[None, :, None]

    @property
    def S(self) -> np.ndarray:
        return self.Q - 0.5 * np.stack([np.diag(e) for e in self.E])


# ---------------------------------------------------------------------------
# Tetrahedron, p = 1..4.  Facet nodes: an S3-symmetric rule of degree 2p on
# every face (all points inside the face, so every facet node belongs to one
# facet and paired faces see the same physical points whatever their relative
# orientation), orbits solved from the triangle moment equations:
#   p = 1: one S21 orbit (3 points), p = 2: two S21 orbits (6),
#   p = 3: two S21 + one S111 (12), p = 4: S3 + three S21 + one S111 (16).
# Volume: the 4 n_f facet nodes (each face orbit is one S4 orbit of the
# tetrahedron, one weight) plus S4-symmetric interior orbits, the weights and
# positions solved from the moment equations of degree 2p - 1 with all
# weights positive (``solve_tet_quadrature`` re-derives them):
#   p = 1: 12 nodes, p = 2: 25, p = 3: 58, p = 4: 78.
# Parameter layout of a face rule: per orbit its position parameters (none
# for S3, a for S21, a, b for S111), then its weight (weights sum to 1/2).
# Layout of a volume rule: one weight per face orbit, then per interior
# orbit its position parameters (none for S4, a for S31 and S22, a, b for
# S211) and its weight.
# ---------------------------------------------------------------------------
_TRI_FACE_RULES = {
    1: dict(degree=2, orbits=["S21"], x=[1.0 / 6.0, 1.0 / 6.0]),
    2: dict(degree=4, orbits=["S21", "S21"],
            x=[0.44594849091596483, 0.11169079483900565, 0.09157621350977083, 0.054975871827661026]),
    3: dict(degree=6, orbits=["S21", "S21", "S111"],
            x=[0.06308901449150953, 0.02542245318510883, 0.24928674517087093, 0.058393137863221665,
               0.31035245103381354, 0.0531450498447909, 0.04142553780916809]),
    4: dict(degree=8, orbits=["S3", "S21", "S21", "S21", "S111"],
            x=[0.07215780383889538, 0.05054722831703085, 0.016229248811598943, 0.4592925882927259,
               0.04754581713364107, 0.1705693077517623, 0.05160868526736049, 0.26311282963463273,
               0.008394777409958283, 0.013615157087217195]),
}
_TET_RULES = {
    1: dict(degree=1, interior=[], x=[1.0 / 72.0]),
    2: dict(degree=3, interior=["S4"], x=[0.006710441872127204, 0.002335214368444981, 0.058118791779800436]),
    3: dict(degree=5, interior=["S31", "S22"],
            x=[0.00068236186453178, 0.002856422538590274, 0.001334501736597179, 0.15457334884980922,
               0.015499652663895004, 0.13846669986348373, 0.00502910024921495]),
    4: dict(degree=7, interior=["S31", "S31", "S22"],
            x=[0.002485691614389907, 0.00030806911398383713, 0.0009130575817185983, 0.0018949943080682364,
               0.00030639411289908324, 0.11797912654527264, 0.007851322735386043, 0.29542463948861264,
               0.007073176720332001, 0.09879275592124274, 0.008713165271901467]),
}
_TET_VERTS = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
_TET_NORMALS = np.array([[1.0, 1.0, 1.0], [-1.0, 0.0, 0.0], [0.0, -1.0, 0.0], [0.0, 0.0, -1.0]])
_TET_NORMALS[0] /= np.sqrt(3.0)
_TET_FACE_SCALE = np.array([np.sqrt(3.0), 1.0, 1.0, 1.0])  # face area / (1/2)
_NPRM = {"S3": 0, "S21": 1, "S111": 2, "S4": 0, "S31": 1, "S22": 1, "S211": 2}


def _tri_orbit(typ, prm):
    """Barycentric points of one S3 orbit of the triangle (fixed order)."""
    if typ == "S3":
        return [(1 / 3, 1 / 3, 1 / 3)]
    if typ == "S21":
        a = prm[0]
        return [(a, a, 1 - 2 * a), (a, 1 - 2 * a, a), (1 - 2 * a, a, a)]
    a, b = prm
    c = 1 - a - b
    return [(a, b, c), (a, c, b), (b, a, c), (b, c, a), (c, a, b), (c, b, a)]


def _tet_orbit(typ, prm):
    """Barycentric points of one S4 orbit of the tetrahedron (fixed order)."""
    import itertools
    if typ == "S4":
        return [(0.25, 0.25, 0.25, 0.25)]
    if typ == "S31":
        a = prm[0]
        return [tuple(1 - 3 * a if k == v else a for k in range(4)) for v in range(4)]
    if typ == "S22":
        a = prm[0]
        return [tuple(a if k in ij else 0.5 - a for k in range(4)) for ij in itertools.combinations(range(4), 2)]
    a, b = prm
    return sorted(set(itertools.permutations((a, a, b, 1 - 2 * a - b))))


def tri_face_rule(p: int, x=None):
    """Barycentric points (n_f, 3), weights (n_f,) (sum 1/2) and the orbit index
    of every point, of the degree-2p face rule."""
    rule = _TRI_FACE_RULES[p]
    x = rule["x"] if x is None else x
    pts, w, orb, i = [], [], [], 0
    for o, typ in enumerate(rule["orbits"]):
        k = _NPRM[typ]
        for lam in _tri_orbit(typ, x[i:i + k]):
            pts.append(lam)
            w.append(x[i + k])
            orb.append(o)
        i += k + 1
    return np.array(pts), np.array(w), np.array(orb)


def tet_monomial_integral(a: int, b: int, c: int) -> float:
    """Exact integral of x^a y^b z^c over the reference tetrahedron."""
    return factorial(a) * factorial(b) * factorial(c) / factorial(a + b + c + 3)


def _tet_nodes(p: int, x, interior=None):
    """Nodes (n_p, 3) and weights (n_p,) of the tetrahedron rule for degree p:
    the facet nodes face by face (face g opposite vertex g), then the interior
    orbits."""
    fp, _, forb = tri_face_rule(p)
    interior = _TET_RULES[p]["interior"] if interior is None else interior
    pts, wts = [], []
    for face in range(4):
        others = [v for v in range(4) if v != face]
        for k in range(len(fp)):
            lam = np.zeros(4)
            for j, v in enumerate(others):
                lam[v] = fp[k][j]
            pts.append(lam[1:])
            wts.append(x[forb[k]])
    i = int(forb.max()) + 1
    for typ in interior:
        k = _NPRM[typ]
        for lam in _tet_orbit(typ, x[i:i + k]):
            pts.append(np.array(lam[1:]))
            wts.append(x[i + k])
        i += k + 1
    return np.array(pts), np.array(wts)


def solve_tet_quadrature(p: int, interior, seed: int = 0, tries: int = 20):
    """Re-derive a tabulated volume rule: seeded nonlinear least squares on the
    moment equations of all monomials up to degree 2p - 1 with the face nodes
    of ``tri_face_rule(p)`` fixed, keeping the positive rule with interior
    nodes strictly inside and the largest smallest weight."""
    from scipy.optimize import least_squares

    deg = 2 * p - 1
    n_fo = len(_TRI_FACE_RULES[p]["orbits"])
    mons = np.array([(a, b, c) for a in range(deg + 1) for b in range(deg + 1 - a) for c in range(deg + 1 - a - b)])
    ex = np.array([tet_monomial_integral(*m) for m in mons])

    def res(x):
        pts, w = _tet_nodes(p, x, interior)
        return w @ np.prod(pts[:, None, :] ** mons[None], axis=2) - ex

    rng = np.random.default_rng(seed)
    best = None
    for _ in range(tries):
        x0 = list(rng.uniform(1e-4, 1e-2, n_fo))
        for typ in interior:
            if typ == "S31":
                x0 += [rng.uniform(0.02, 0.32)]
            elif typ == "S22":
                x0 += [rng.uniform(0.02, 0.24)]
            elif typ == "S211":
                a = rng.uniform(0.02, 0.3)
                x0 += [a, rng.uniform(0.02, 0.9 - 2 * a)]
            x0 += [rng.uniform(1e-3, 2e-2)]
        r = least_squares(res, x0, xtol=1e-15, ftol=1e-15, gtol=1e-15, max_nfev=4000)
        pts, w = _tet_nodes(p, r.x, interior)
        ip = np.concatenate([pts, 1 - pts.sum(1, keepdims=True)], 1)[4 * len(tri_face_rule(p)[0]):]
        inside = len(ip) == 0 or np.all(ip > 1e-3)
        if np.all(w > 0) and inside and np.abs(res(r.x)).max() < 1e-14:
            if best is None or w.min() > best[0]:
                best = (w.min(), r.x)
    return None if best is None else best[1]


def tet_operator(p: int) -> RefOperator:
    """Diagonal-E SBP operator of degree p (1..4) on the reference tetrahedron."""
    key = ("tet", p)
    if key in _CACHE:
        return _CACHE[key]
    if p not in _TET_RULES:
        raise ValueError(f"no tetrahedron rule for p={p}")
    rule = _TET_RULES[p]
    xi, H = _tet_nodes(p, np.asarray(rule["x"], dtype=np.float64))
    _, fw, _ = tri_face_rule(p)
    n_fac, nf = 4, len(fw)
    n_p = len(H)
    facet_nodes = np.arange(n_fac * nf, dtype=np.int32).reshape(n_fac, nf)
    facet_w = np.stack([fw * _TET_FACE_SCALE[g] for g in range(n_fac)])
    E = np.zeros((3, n_p))
    for g in range(n_fac):
        for k in range(nf):
            E[:, facet_nodes[g, k]] += facet_w[g, k] * _TET_NORMALS[g]
    V, dV = vandermonde(xi, p, np.array([0.25, 0.25, 0.25]))
    Q = np.zeros((3, n_p, n_p))
    for j in range(3):
        S = min_norm_skew(H, E[j], V, dV[j])
        Q[j] = S + 0.5 * np.diag(E[j])
    op = RefOperator(d=3, p=p, n_p=n_p, n_fac=n_fac, n_f=nf, xi=xi, H=H, Q=Q, E=E,
                     facet_nodes=facet_nodes, facet_w=facet_w, ref_normals=_TET_NORMALS.copy(),
                     volume_degree=rule["degree"])
    _CACHE[key] = op
    return op


_CACHE: dict = {}


def tri_operator(p: int) -> RefOperator:
    """Diagonal-E SBP operator of degree p (1..4) on the reference triangle."""
    if p in _CACHE:
        return _CACHE[p]
    if p not in _TRI_RULES:
        raise ValueError(f"no triangle rule for p={p}")
    rule = _TRI_RULES[p]
    xi, H = _tri_nodes(p, np.asarray(rule["x"], dtype=np.float64))
    nf = p + 1
    n_fac = 3
    n_p = len(H)
    t, tw = gauss_legendre01(nf)
    facet_nodes = np.arange(n_fac * nf, dtype=np.int32).reshape(n_fac, nf)
    facet_w = np.stack([tw * _TRI_LENGTHS[g] for g in range(n_fac)])
    E = np.zeros((2, n_p))
    for g in range(n_fac):
        for k in range(nf):
            E[:, facet_nodes[g, k]] += facet_w[g, k] * _TRI_NORMALS[g]
    V, dV = vandermonde(xi, p, np.array([1 / 3, 1 / 3]))
    Q = np.zeros((2, n_p, n_p))
    for j in range(2):
        S = min_norm_skew(H, E[j], V, dV[j])
        Q[j] = S + 0.5 * np.diag(E[j])
    op = RefOperator(d=2, p=p, n_p=n_p, n_fac=n_fac, n_f=nf, xi=xi, H=H, Q=Q, E=E,
                     facet_nodes=facet_nodes, facet_w=facet_w,
                     ref_normals=_TRI_NORMALS.copy(), volume_degree=rule["degree"])
    _CACHE[p] = op
    return op


# ---------------------------------------------------------------------------
# Interval, p = 1..4 (the 1D problems of Secs. 7.1-7.2): the p + 1
# Gauss-Lobatto-Legendre points on the reference interval [0, 1], H their
# quadrature weights (exact to degree 2p - 1), E = diag(-1, 0, ..., 0, 1); with
# p + 1 nodes the accuracy conditions fix S uniquely.  Node order: the two end
# points (facet 0 at 0, facet 1 at 1), then the interior points ascending.
# ---------------------------------------------------------------------------
def lgl_points01(p: int):
    """Gauss-Lobatto-Legendre points (ascending) and weights on [0, 1]: the
    end points and the roots of P_p', weights 2 / (p (p + 1) P_p(x)^2) on
    [-1, 1], halved."""
    Pp = np.polynomial.legendre.Legendre.basis(p)
    inner = np.sort(Pp.deriv().roots().real) if p > 1 else np.array([])
    x = np.concatenate([[-1.0], inner, [1.0]])
    w = 2.0 / (p * (p + 1) * Pp(x) ** 2)
    return (x + 1.0) / 2.0, w / 2.0


def line_operator(p: int) -> RefOperator:
    """Diagonal-E SBP operator of degree p on the reference interval [0, 1]."""
    key = ("line", p)
    if key in _CACHE:
        return _CACHE[key]
    t, w = lgl_points01(p)
    order = [0, p] + list(range(1, p))
    xi = t[order][:, None]
    H = w[order]
    n_p = p + 1
    E = np.zeros((1, n_p))
    E[0, 0], E[0, 1] = -1.0, 1.0
    V, dV = vandermonde(xi, p, np.array([0.5]))
    S = min_norm_skew(H, E[0], V, dV[0])
    Q = (S + 0.5 * np.diag(E[0]))[None]
    op = RefOperator(d=1, p=p, n_p=n_p, n_fac=2, n_f=1, xi=xi, H=H, Q=Q, E=E,
                     facet_nodes=np.array([[0], [1]], dtype=np.int32), facet_w=np.ones((2, 1)),
                     ref_normals=np.array([[-1.0], [1.0]]), volume_degree=2 * p - 1)
    _CACHE[key] = op
    return op

