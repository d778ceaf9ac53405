"""Writes vortex128_p3_extended.txt: the residual of 8 sampled elements of
the 32,768-triangle vortex mesh (128 x 128 quads, warp 0.05, p = 3, vortex +
1e-3 uniform noise, seed 2), split and Hadamard forms with the dissipation of
Eq. (69), evaluated at 50 digits by oracle/extended.py and rounded to
float64 (repr, round trip exact).

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
    el = sorted(set(np.random.default_rng(2024).choice(m.n_e, 6, replace=False).tolist()) | {0, m.n_e - 1})
    lines = ["# 50-digit residual (oracle/extended.py) rounded to float64: scheme element component node value",
             "# 128 x 128 x 2 curved triangles, p = 3, vortex + 1e-3 noise (seed 2), dissipation on"]
    for scheme in ["split", "hadamard"]:
        res = X.residual_elements(u, op, m, el, scheme=scheme, dissipation=True)
        for k, r in zip(el, res):
            for c in range(4):
                for n in range(op.n_p):
                    lines.append(f"{scheme} {k} {c} {n} {float(r[c][n])!r}")
    with open(os.path.join(HERE, "vortex128_p3_extended.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
