"""Gradients through many relaxation RK4 steps with per-step checkpoints.

The forward pass keeps u_n of every step (one state-sized device tensor per
step); the reverse pass walks the steps backwards with esplit_rrk_step_vjp,
which recomputes the four stages of a step from its checkpoint.  All
arithmetic runs in the CUDA library; this module only orders the calls.
"""
from __future__ import annotations

import torch


def entropy_gradient_through_steps(solver, u0: torch.Tensor, dt: float, n_steps: int):
    """d(1^T H s(u_N)) / d u_0 for N relaxation RK4 steps of size dt.

    Returns (gradient, final state, list of g_n)."""
    checkpoints = []
    u = u0.clone()
    gs = []
    for _ in range(n_steps):
        checkpoints.append(u.clone())
        g, _ = solver.rrk_step(u, dt)
        gs.append(g)
    ubar = solver.entropy_grad(u)
    nxt = solver.empty()
    for un in reversed(checkpoints):
        solver.rrk_step_vjp(un, dt, ubar, out=nxt)
        ubar, nxt = nxt, ubar
    return ubar, u, gs
