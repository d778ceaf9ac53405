"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package builds the *data* the semi-discrete residual consumes and nothing
of the residual itself:

* ``sbp``    -- reference diagonal-E SBP operators (Def. 1 and the diagonal-H /
                diagonal-E decomposition of Sec. 2.1) on the reference triangle,
* ``mesh``   -- structured periodic meshes of curved triangles (quadratic
                geometry, Assumption 1), nodal metric terms, scaled facet normals
                and the facet-node pairing table,
* ``states`` -- seeded initial states (isentropic vortex of Sec. 7.3, uniform
                noise, piecewise-constant quadrant states).

No flux, entropy, SAT, dissipation or time-integration arithmetic lives here;
both the oracle and the library receive these arrays as plain inputs.
"""
from .sbp import RefOperator, tri_operator, tet_operator, line_operator
from .mesh import Mesh, periodic_tri_mesh
from . import states

__all__ = ["RefOperator", "tri_operator", "tet_operator", "line_operator", "Mesh", "periodic_tri_mesh", "states"]
