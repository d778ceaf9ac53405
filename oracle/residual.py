"""Semi-discrete residuals du/dt (plain PyTorch, float64).

Inputs: u (n_e, n_c, n_p) conservative variables (the library layout), the
reference operator and mesh of ``esplit_inputs``, Params.  Output: du/dt of
the requested elements, (n, n_c, n_p).

Schemes (per element; ``hybrid_flags`` selects per element, Thm. 4):
  * entropy split, strong form: Eq. (42) with the inviscid SATs of Eq. (43)
  * entropy split, weak form:   Eq. (100)  (the form the paper implements)
  * Hadamard form, strong:      Eq. (67);  weak: Eq. (99)
Facet terms, once per facet node of the element (diagonal E, Sec. 4 Remark):
  * EC SAT  -1/2 H^-1 sum_i [E^kv_x_i o F_i(u_k, u_v)] 1, which at facet node m
    paired with node n of the neighbour is -(1/H_m) sum_i nu_i F*_i(u_km, u_vn)
  * matrix interface dissipation, Eq. (69), with B_g -> |nu| and n = nu/|nu|
    on curved facets
Viscous terms (Sec. 5, Eqs. (83)-(85)) with Baumann-Oden coefficients
(Eq. (96)): T1 = 0, T2 = T3 = B/2.
Boundary facets (bounded 1D domains of Secs. 7.1-7.2; the paper's theory is
periodic and it does not print its boundary treatment): a facet slot whose
pair is (-1, -1) takes the same SAT and dissipation as an interior one, with
the neighbour's state replaced by a prescribed exterior state u_b (reading:
the interface coupling of Eq. (43) with a ghost state, weak imposition of
the boundary data; inviscid only).

Readings (the paper is ambiguous or has typos there):
  * Eq. (100): the facet sum runs over Gamma^I_k (printed Gamma^I);
  * Eq. (99): the stray w_k^T in the facet term is dropped;
  * curved facets: B_g N_x_i,g -> nu_i (scaled outward normal at the node).

Pins (tests/test_oracle_residual.py): strong = weak form; Hadamard strong =
weak; free-stream preservation; entropy rate zero (EC, any state, curved
periodic mesh; split, Hadamard and random hybrids); dissipation rate equals
the closed facet sum and is <= 0; Hadamard local conservation; split
conservation error falls with refinement; dense brute-force assembly of
Eqs. (42)-(44) on a 2-element mesh; viscous BO rate equals the volume
quadratic form.
"""
from __future__ import annotations

import numpy as np
import torch

from .physics import (Params, entropy_variables, euler_flux, sy_flux, ir_flux, ir_dissipation_matrix,
                      standard_entropy_variables,
                      symmetrized_flux_jacobians, dissipation_matrix,
                      viscous_flux_from_w_grads, viscous_K)
from .operators import physical_operators

DT = torch.float64

SPLIT, HADAMARD = 0, 1


def _as_U(u):
    t = torch.as_tensor(np.asarray(u) if not torch.is_tensor(u) else u, dtype=DT)
    return t.transpose(1, 2)  # (n_e, n_p, n_c)


def split_volume(U, ops, prm: Params, form="weak"):
    """Entropy-split volume terms of element(s), (n, n_p, n_c)."""
    b = prm.beta
    f = euler_flux(U, prm)                          # (n, n_p, d, nc)
    w = entropy_variables(U, prm)                   # (n, n_p, nc)
    At = symmetrized_flux_jacobians(U, prm)         # (n, n_p, d, nc, nc)
    Dw = torch.einsum("nimk,nkc->nimc", ops["D"], w)                 # (n, d, n_p, nc)
    nonc = torch.einsum("nmicd,nimd->nmc", At, Dw)                   # sum_i A~_i D_x_i w
    Q, H = ops["Q"], ops["H"]
    if form == "weak":
        M = Q / (b + 1.0) + Q.transpose(-1, -2)
        cons = torch.einsum("nimk,nkic->nmc", M, f) / H[..., None]
        return cons - nonc / (b + 1.0)
    # strong form, Eq. (42) moved to the right-hand side with the first SAT of Eq. (43)
    Df = torch.einsum("nimk,nkic->nmc", ops["D"], f)
    Ef = torch.einsum("nim,nmic->nmc", ops["E"], f) / H[..., None]
    return -b / (b + 1.0) * Df - nonc / (b + 1.0) + Ef


def hadamard_volume(U, ops, prm: Params, form="weak", flux=None):
    """Hadamard-form volume terms with the Sjogreen-Yee flux (or ``flux``),
    (n, n_p, n_c)."""
    flux = sy_flux if flux is None else flux
    n, n_p, nc = U.shape
    Um = U[:, :, None, :].expand(n, n_p, n_p, nc)
    Un = U[:, None, :, :].expand(n, n_p, n_p, nc)
    F2 = 2.0 * flux(Um, Un, prm)                    # (n, m, k, d, nc): block of Eq. (44)
    if form == "weak":
        return -torch.einsum("nimk,nmkic->nmc", ops["S"], F2) / ops["H"][..., None]
    vol = -torch.einsum("nimk,nmkic->nmc", ops["D"], F2)
    diagF = torch.diagonal(F2, dim1=1, dim2=2).permute(0, 3, 1, 2)  # (n, m, d, nc)
    return vol + 0.5 * torch.einsum("nim,nmic->nmc", ops["E"], diagF) / ops["H"][..., None]


def residual(u, ref, mesh, prm: Params = Params(), *, scheme="split", form="weak",
             dissipation=False, viscous=False, hybrid_flags=None, elems=None, boundary=None):
    """du/dt for the elements ``elems`` (all if None), layout (n, n_c, n_p).

    scheme: "split", "hadamard" or "hybrid" (per-element ``hybrid_flags``,
    1 = Hadamard), or "hadamard_ir": the Hadamard form with the Ismail-Roe
    flux in the volume and the SATs (entropy conservative for the standard
    entropy), with its own matrix dissipation (``ir_dissipation_matrix`` on the
    jump of the standard entropy variables) when ``dissipation``, and the
    same Baumann-Oden viscous terms written with the standard entropy
    variables when ``viscous``.  ``u`` may be a torch tensor requiring grad
    (the oracle adjoint differentiates through this function).
    ``boundary`` = (slots, states): flat facet slots (element * n_slot + slot)
    whose pair is (-1, -1), and their exterior states (n_b, n_c)."""
    U_all = _as_U(u)
    n_e, n_p, nc = U_all.shape
    d = nc - 2
    pair = torch.as_tensor(mesh.pair, dtype=torch.long)          # (n_e, n_fac, n_f, 2)
    n_slot = ref.n_fac * ref.n_f
    pair = pair.reshape(n_e, n_slot, 2)
    fn = torch.as_tensor(ref.facet_nodes.reshape(-1), dtype=torch.long)
    bmask = pair[..., 0] < 0                                      # boundary facet slots
    if bool(bmask.any()):
        if viscous:
            raise NotImplementedError("viscous terms on boundary facets")
        if boundary is None:
            raise ValueError("the mesh has boundary facets: pass boundary=(slots, states)")
        bslots = torch.as_tensor(np.asarray(boundary[0]), dtype=torch.long)
        Ub_all = torch.zeros(n_e * n_slot, nc, dtype=DT)
        Ub_all[bslots] = torch.as_tensor(np.asarray(boundary[1]), dtype=DT)
        Ub_all = Ub_all.reshape(n_e, n_slot, nc)
        pair = torch.where(bmask[..., None], torch.zeros_like(pair), pair)
    tgt = torch.arange(n_e) if elems is None else torch.as_tensor(elems, dtype=torch.long)
    nb = pair[tgt, :, 0]                                          # (n, slots)
    need = torch.unique(torch.cat([tgt, nb.reshape(-1)])) if viscous else tgt
    loc = torch.full((n_e,), -1, dtype=torch.long)
    loc[need] = torch.arange(len(need))

    ops = physical_operators(ref, mesh, need)
    U = U_all[need]
    t_loc = loc[tgt]
    H_t = ops["H"][t_loc]

    # ---- volume terms -------------------------------------------------------
    ops_t = {k: v[t_loc] for k, v in ops.items()}
    Ut = U[t_loc]
    if scheme == "split":
        vol = split_volume(Ut, ops_t, prm, form)
    elif scheme == "hadamard":
        vol = hadamard_volume(Ut, ops_t, prm, form)
    elif scheme == "hadamard_ir":
        vol = hadamard_volume(Ut, ops_t, prm, form, flux=ir_flux)
    elif scheme == "hybrid":
        flags = torch.as_tensor(np.asarray(hybrid_flags), dtype=torch.long)[tgt]
        vs = split_volume(Ut, ops_t, prm, form)
        vh = hadamard_volume(Ut, ops_t, prm, form)
        vol = torch.where((flags == HADAMARD)[:, None, None], vh, vs)
    else:
        raise ValueError(scheme)
    r = vol

    # ---- inviscid facet terms (EC SAT + dissipation) ------------------------
    nu = torch.as_tensor(mesh.nu, dtype=DT).reshape(n_e, n_slot, d)[tgt]   # (n, s, d)
    Uk = Ut[:, fn, :]                                                       # (n, s, nc)
    Uv = U_all[pair[tgt, :, 0], fn[pair[tgt, :, 1]], :]                     # (n, s, nc)
    if bool(bmask.any()):
        Uv = torch.where(bmask[tgt][..., None], Ub_all[tgt], Uv)           # exterior states
    Hm = H_t[:, fn]                                                         # (n, s)
    Fs = (ir_flux if scheme == "hadamard_ir" else sy_flux)(Uk, Uv, prm)    # (n, s, d, nc)
    sat = -torch.einsum("nsi,nsic->nsc", nu, Fs) / Hm[..., None]
    if dissipation:
        bmag = torch.linalg.norm(nu, dim=-1)
        nhat = nu / bmag[..., None]
        if scheme == "hadamard_ir":
            Dm = ir_dissipation_matrix(Uk, Uv, nhat, prm)
            dw = standard_entropy_variables(Uk, prm) - standard_entropy_variables(Uv, prm)
        else:
            Dm = dissipation_matrix(Uk, Uv, nhat, prm)
            dw = entropy_variables(Uk, prm) - entropy_variables(Uv, prm)
        sat = sat - (bmag / (2.0 * Hm))[..., None] * torch.einsum("nscd,nsd->nsc", Dm, dw)
    r = r.index_add(1, fn, sat)

    # ---- viscous terms, Eqs. (83)-(85) with BO SATs (Eq. (96)) --------------
    if viscous:
        # the BO terms in the entropy variables of the scheme's entropy: Harten's
        # for the split, Hadamard and hybrid schemes, the standard ones for the
        # Ismail-Roe comparator (Thm. 3 holds for either)
        ent = "standard" if scheme == "hadamard_ir" else "harten"
        wvars = standard_entropy_variables if scheme == "hadamard_ir" else entropy_variables
        w = wvars(U, prm)                                                    # (N, n_p, nc)
        gW = torch.einsum("nimk,nkc->nmic", ops["D"], w)                     # (N, n_p, d, nc)
        Fv = viscous_flux_from_w_grads(U, gW, prm, ent)                      # (N, n_p, d, nc)
        r = r + torch.einsum("nimk,nkic->nmc", ops_t["D"], Fv[t_loc])
        v_loc = loc[pair[tgt, :, 0]]
        Fv_k = Fv[t_loc][:, fn]                                              # (n, s, d, nc)
        Fv_v = Fv[v_loc, fn[pair[tgt, :, 1]]]                                # (n, s, d, nc)
        t1 = -0.5 * torch.einsum("nsi,nsic->nsc", nu, Fv_k - Fv_v) / Hm[..., None]
        r = r.index_add(1, fn, t1)
        Kt = viscous_K(Uk, prm, ent)                                         # (n, s, d, d, nc, nc)
        dw = wvars(Uk, prm) - wvars(Uv, prm)
        # a_j(m) = sum_i K~_ij^T nu_i dw  at facet nodes
        a = torch.einsum("nsijcb,nsi,nsc->nsjb", Kt, nu, dw)                 # (n, s, d, nc)
        a_full = torch.zeros(len(tgt), n_p, d, nc, dtype=DT).index_add(1, fn, a)
        lift = torch.einsum("njkm,nkjc->nmc", ops_t["Q"], a_full / H_t[:, :, None, None])
        r = r - 0.5 * lift / H_t[..., None]
    return r.transpose(1, 2)
