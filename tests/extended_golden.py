"""The stored 50-digit residual of sampled config-2 elements
(tests/golden/vortex128_p3_extended.txt, written by
tests/golden/make_extended_residual.py from oracle/extended.py), loaded
without mpmath so that the GPU tests can read it too."""
import os

import numpy as np

from esplit_inputs import tri_operator, periodic_tri_mesh, states

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "vortex128_p3_extended.txt")


def _load_golden():
    rows = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            scheme, k, c, n, val = line.split()
            rows[(scheme, int(k), int(c), int(n))] = float(val)
    return rows


def golden_elements():
    """(mesh inputs, the sampled elements, {scheme: (n, n_c, n_p) 50-digit residual as float64})."""
    op = tri_operator(3)
    m = periodic_tri_mesh(op, 128, 10.0, 0.05)
    u = states.add_uniform_noise(states.isentropic_vortex(m), 1e-3, 2)
    g = _load_golden()
    el = sorted({k for (_, k, _, _) in g})
    out = {}
    for scheme in ["split", "hadamard"]:
        out[scheme] = np.array([[[g[(scheme, k, c, n)] for n in range(op.n_p)] for c in range(4)] for k in el])
    return op, m, u, el, out
