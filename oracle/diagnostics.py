"""Global functionals of Secs. 4.2, 4.3 and 6.1 (plain PyTorch, float64).

* entropy_total      1^T H_g s(u), the quantity Eq. (97) relaxes,
* entropy_rate       sum_k w_k^T H_k du_k/dt (Thm. 2: zero for the EC scheme),
* entropy_rate_scale sum_k sum_m H_m |w_m| |r_m|, the size a round-off
                     entropy rate is compared with,
* conservation       sum_k I^T H_k u_k per component (Sec. 4.3).
"""
from __future__ import annotations

import numpy as np
import torch

from .physics import Params, entropy_variables, harten_entropy

DT = torch.float64


def _nodes(ref, mesh):
    return torch.as_tensor(ref.H, dtype=DT)[None, :] * torch.as_tensor(mesh.J, dtype=DT)


def _U(u):
    t = u if torch.is_tensor(u) else torch.as_tensor(np.asarray(u), dtype=DT)
    return t.transpose(1, 2)


def entropy_total(u, ref, mesh, prm: Params = Params()):
    return (_nodes(ref, mesh) * harten_entropy(_U(u), prm)).sum()


def entropy_rate(u, r, ref, mesh, prm: Params = Params()):
    w = entropy_variables(_U(u), prm)
    return (_nodes(ref, mesh)[..., None] * w * _U(r)).sum()


def entropy_rate_scale(u, r, ref, mesh, prm: Params = Params()):
    w = entropy_variables(_U(u), prm)
    return (_nodes(ref, mesh) * torch.linalg.norm(w, dim=-1) * torch.linalg.norm(_U(r), dim=-1)).sum()


def conservation(u, ref, mesh):
    return (_nodes(ref, mesh)[..., None] * _U(u)).sum(dim=(0, 1))
