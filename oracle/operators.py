"""Physical SBP operators of curved elements (plain PyTorch, float64).

Def. 1 defines D_x_i,k = H_k^-1 Q_x_i,k on the physical element; Sec. 2.1 and
Assumption 1 defer the curved-element construction to the cited literature.
The construction used (the reading recorded for the oracle):

  H_k       = diag(H_ref * J_k)
  E_x_i,k   = sum_g R_g^T B_g N_x_i,g R_g  (Eq. (2)), i.e. diagonal with the
              scaled outward normal nu_i = b n_i at every facet node
  Q_x_i,k   = 1/2 sum_j (Lam_ij Q_xi_j - Q_xi_j^T Lam_ij) + 1/2 E_x_i,k
  S_x_i,k   = Q_x_i,k - 1/2 E_x_i,k

with Lam_ij = diag(J dxi_j/dx_i at the nodes).  Q + Q^T = E holds by
construction; Q 1 = 0 (free-stream preservation) follows from the discrete
metric identity that Assumption 1 guarantees.

Pins (tests/test_oracle_operators.py): SBP property, Q 1 = 0, D exact on P^p
for affine elements, sum of H = domain area, nu_k = -nu_v at paired nodes.
"""
from __future__ import annotations

import torch

DT = torch.float64


def physical_operators(ref, mesh, elems=None):
    """Dense per-element operators for the elements ``elems`` (all if None).

    Returns dict with H (n, n_p), Q (n, d, n_p, n_p), E (n, d, n_p) (diagonal),
    S (n, d, n_p, n_p), D (n, d, n_p, n_p)."""
    idx = slice(None) if elems is None else torch.as_tensor(elems, dtype=torch.long)
    Qr = torch.as_tensor(ref.Q, dtype=DT)                        # (d, n_p, n_p)
    Hr = torch.as_tensor(ref.H, dtype=DT)
    J = torch.as_tensor(mesh.J, dtype=DT)[idx]                   # (n, n_p)
    Lam = torch.as_tensor(mesh.Lam, dtype=DT)[idx]               # (n, d, d, n_p)
    nu = torch.as_tensor(mesh.nu, dtype=DT)[idx]                 # (n, n_fac, n_f, d)
    n, d = J.shape[0], ref.d
    n_p = ref.n_p
    fn = torch.as_tensor(ref.facet_nodes.reshape(-1), dtype=torch.long)
    E = torch.zeros(n, d, n_p, dtype=DT)
    E[:, :, fn] = nu.reshape(n, -1, d).transpose(1, 2)
    # Lam_ij Q_xi_j: row-scaling of Q by Lam_ij at node m;  Q^T Lam: column scaling
    LQ = torch.einsum("nijm,jmk->nijmk", Lam, Qr)
    QTL = torch.einsum("jkm,nijk->nijmk", Qr, Lam)   # (Q_j^T)_{mk} Lam_ij,k
    Q = 0.5 * (LQ - QTL).sum(2) + 0.5 * torch.diag_embed(E)
    H = Hr[None, :] * J
    S = Q - 0.5 * torch.diag_embed(E)
    D = Q / H[:, None, :, None]
    return dict(H=H, Q=Q, E=E, S=S, D=D)
