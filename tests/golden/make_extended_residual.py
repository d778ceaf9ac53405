"""Writes vortex128_p3_extended.txt: the residual of 5 sampled elements of
the 32,768-triangle vortex mesh (128 x 128 quads, warp 0.05, p = 3, vortex +
1e-3 uniform noise, seed 2), split and Hadamard forms with the dissipation of
Eq. (69), evaluated at 50 digits by oracle/extended.py and rounded to
float64, together with every float64 input those residuals depend on (the
reference operator, the elements' J, Lambda, nu and states, the states of the
neighbours' paired facet nodes), as hexadecimal floats.  The inputs are
stored because the mesh and state generators call libm (sin, exp), whose
last-bit rounding differs between platforms: a reader of this file puts the
stored inputs into its own arrays (tests/extended_golden.py) and then has the
very numbers the residuals were computed from.

    python tests/golden/make_extended_residual.py

Calls only oracle/ (and the seeded input generators of esplit_inputs/).
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from esplit_inputs import tri_operator, periodic_tri_mesh, states  # noqa: E402
from oracle import extended as X  # noqa: E402


def main():
    op = tri_operator(3)
    m = periodic_tri_mesh(op, 128, 10.0, 0.05)
    u = states.add_uniform_noise(states.isentropic_vortex(m), 1e-3, 2)
    el = sorted(set(np.random.default_rng(2024).choice(m.n_e, 3, replace=False).tolist()) | {0, m.n_e - 1})
    lines = ["# float64 values as hexadecimal floats, one row per line: name indices : values along the last index",
             "# inputs H, Q, J, u, Lam, nu; outputs res scheme element component : residual at the nodes",
             "# 128 x 128 x 2 curved triangles, p = 3, vortex + 1e-3 noise (seed 2), dissipation on"]

    def row(name, idx, vals):
        lines.append(" ".join([name, *map(str, idx), ":", *(float.hex(float(x)) for x in vals)]))

    row("H", (), op.H)
    for j in range(op.d):
        for a in range(op.n_p):
            row("Q", (j, a), op.Q[j, a])
    fn = op.facet_nodes.reshape(-1)
    for k in el:
        row("J", (k,), m.J[k])
        for c in range(4):
            row("u", (k, c), u[k, c])
        for i in range(op.d):
            for j in range(op.d):
                row("Lam", (k, i, j), m.Lam[k, i, j])
        nu = m.nu[k].reshape(-1, op.d)
        pr = m.pair[k].reshape(-1, 2)
        row("nu", (k,), nu.reshape(-1))
        for s in range(len(fn)):
            v, n = int(pr[s, 0]), int(fn[pr[s, 1]])
            row("un", (v, n), u[v, :, n])
    for scheme in ["split", "hadamard"]:
        res = X.residual_elements(u, op, m, el, scheme=scheme, dissipation=True)
        for k, r in zip(el, res):
            for c in range(4):
                row(f"res_{scheme}", (k, c), r[c])
    with open(os.path.join(HERE, "vortex128_p3_extended.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
