"""Plain, slow, FP64 CPU oracle of the entropy-split SBP-SAT residual.

TEST INFRASTRUCTURE ONLY.  Nothing in the library path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` use it.  It shares no code with
the CUDA path (``paper_2305_07181_gb300``); the two meet only through the
seeded inputs of ``esplit_inputs`` (operators, meshes, states), which hold none
of the method's arithmetic.

Every function follows the paper (Worku & Zingg, "Entropy-split
multidimensional summation-by-parts discretization of the Euler and
compressible Navier-Stokes equations") in its own notation, written with plain
PyTorch CPU float64 tensor operations (einsum, elementwise math, small dense
solves, torch.func Jacobians) and no blocking, fusion or reordering beyond the
definitions.  Because every step is a differentiable PyTorch operation,
``torch.autograd`` of the oracle residual is the oracle adjoint.

Modules
  physics    pointwise physics: Harten entropy and variables, Euler fluxes,
             Sjogreen-Yee two-point flux, dissipation ingredients, viscous flux
  operators  physical SBP operators of curved elements
  residual   strong- and weak-form entropy-split, Hadamard-form and hybrid
             residuals with EC SATs, matrix interface dissipation and
             Baumann-Oden viscous SATs
  rrk        classical RK4 and the relaxation parameter by bisection
  diagnostics entropy totals, entropy rate, conservation sums

Parity status of each function (which pin in ``tests/test_oracle_*.py`` fixes
it) is listed in the module docstrings.
"""
from . import physics, operators, residual, rrk, diagnostics  # noqa: F401
from .physics import Params  # noqa: F401
