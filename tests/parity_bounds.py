"""Rounding scale of the residual for the FP64 parity bounds.

summand_scale returns, per node and component, the magnitude of the terms
whose sum is the residual.  FP64 rounding on either side (the GPU path or
the oracle) is a few eps times this, whatever the size of the result itself;
where the residual is much smaller than its terms (a state near a constant,
a low-Mach flow) a plain relative bound on the result is not met by either
side, and the parity tests bound |r_gpu - r_oracle| by
1e-12 max|r| + ROUNDING_C eps (summand scale).

ROUNDING_C = 8: against the residual evaluated at 50 digits
(oracle/extended.py, tests/test_oracle_extended.py) the float64 oracle is
within 1.5 eps (summand scale) of the exact value on the 32,768-triangle
vortex mesh; the GPU path is within 2.5 of the oracle there; the largest GPU-vs-oracle
difference seen on any workload is 4.2 eps (summand scale) (Taylor-Green,
Hadamard form with viscous terms).  The plain max-norm relative error is
printed beside every such check: at these sizes it is 1e-12 to 2e-10 for
either float64 implementation.
"""
import numpy as np
import torch

ROUNDING_C = 8.0
EPS = float(np.finfo(float).eps)


def rounding_bound(ro, sc, rel=1e-12):
    """|r_gpu - r_oracle| allowed per entry: rel max|r| + ROUNDING_C eps sc."""
    return rel * np.abs(ro).max() + ROUNDING_C * EPS * sc


def summand_scale(u, op, m, elems, scheme, prm, dissipation=True, viscous=False):
    """Terms, for the elements ``elems``:
      split:     sum_i |M_i||f_i| + |A~_i||D_i||w|/(beta+1)
      Hadamard:  2 sum_n sum_i |S_i,mn||F*_i(u_m,u_n)|/H_m
      facets:    |nu||F*|/H + |nu|/(2H) |X|L|SX^T| (|dw| + |w_k| + |w_v|)
      (the Ismail-Roe comparator: its flux, dissipation and standard entropy
    variables in the Hadamard and facet terms)
    viscous:   sum_i |D_i| G_i + |nu| (G(k) + G(v))/H
                 + 1/(2H) sum_j |D_j|^T sum_i |K~_ij||nu_i| (|w_k| + |w_v|)
                 with G_i = |F^V_i| + sum_j |K~_ij||D_j||w|
    Both sides form A~_i and the viscous flux from dU/dW written out in closed
    form (no matrix inverse), so no condition number of dW/dU enters."""
    from oracle.physics import (euler_flux, entropy_variables, symmetrized_flux_jacobians, sy_flux,
                                dissipation_matrix, viscous_K, viscous_flux_from_w_grads, ir_flux,
                                ir_dissipation_matrix, standard_entropy_variables)
    # the Ismail-Roe comparator: its flux, its dissipation and the standard
    # entropy variables in place of the Sjogreen-Yee ones
    ir = scheme == "hadamard_ir"
    flux = ir_flux if ir else sy_flux
    evars = standard_entropy_variables if ir else entropy_variables
    dmat = ir_dissipation_matrix if ir else dissipation_matrix
    from oracle.operators import physical_operators
    d = op.d
    el = torch.as_tensor(elems)
    ops = physical_operators(op, m, el)
    U_all = torch.as_tensor(u).transpose(1, 2)
    U = U_all[el]
    H = ops["H"]
    w = entropy_variables(U, prm).abs()
    if scheme == "split":
        f = euler_flux(U, prm).abs()
        M = ops["Q"] / (prm.beta + 1) + ops["Q"].transpose(-1, -2)
        sc = torch.einsum("nimk,nkic->nmc", M.abs(), f) / H[..., None]
        Dw = torch.einsum("nimk,nkc->nimc", ops["D"].abs(), w)
        At = symmetrized_flux_jacobians(U, prm).abs()
        sc = sc + torch.einsum("nmicd,nimd->nmc", At, Dw) / (prm.beta + 1)
    else:
        n_, npp, nc = U.shape
        F2 = 2 * flux(U[:, :, None, :].expand(n_, npp, npp, nc), U[:, None, :, :].expand(n_, npp, npp, nc),
                      prm).abs()
        sc = torch.einsum("nimk,nmkic->nmc", ops["S"].abs(), F2) / H[..., None]
    fn = torch.as_tensor(op.facet_nodes.reshape(-1))
    pr = torch.as_tensor(m.pair.reshape(m.n_e, -1, 2))[el]
    Uk, Uv = U[:, fn], U_all[pr[..., 0], fn[pr[..., 1]]]
    nu = torch.as_tensor(m.nu.reshape(m.n_e, -1, d))[el]
    b = torch.linalg.norm(nu, dim=-1)
    wk, wv = evars(Uk, prm), evars(Uv, prm)
    fac = torch.einsum("nsi,nsic->nsc", nu.abs(), flux(Uk, Uv, prm).abs())
    if dissipation:
        Dm = dmat(Uk, Uv, nu / b[..., None], prm).abs()
        dws = (wk - wv).abs() + wk.abs() + wv.abs()
        fac = fac + 0.5 * b[..., None] * torch.einsum("nscd,nsd->nsc", Dm, dws)
    sc = sc.index_add(1, fn, fac / H[:, fn][..., None])
    if viscous:
        # the viscous flux is needed on the elements and their face neighbours
        need = torch.unique(torch.cat([el, pr[..., 0].reshape(-1)]))
        loc = torch.full((m.n_e,), -1, dtype=torch.long)
        loc[need] = torch.arange(len(need))
        ops_n = physical_operators(op, m, need)
        Un = U_all[need]
        ent = "standard" if ir else "harten"
        wn = evars(Un, prm)
        gW = torch.einsum("nimk,nkc->nmic", ops_n["D"], wn)
        Fv = viscous_flux_from_w_grads(Un, gW, prm, ent).abs()              # (n, n_p, d, nc)
        Kn = viscous_K(Un, prm, ent).abs()                                  # (n, n_p, d, d, nc, nc)
        Dwn = torch.einsum("nimk,nkc->nmic", ops_n["D"].abs(), wn.abs())    # (n, n_p, d, nc)
        G = Fv + torch.einsum("nmijcb,nmjb->nmic", Kn, Dwn)
        Ge = G[loc[el]]
        sc = sc + torch.einsum("nimk,nkic->nmc", ops["D"].abs(), Ge)
        Gk, Gv = Ge[:, fn], G[loc[pr[..., 0]], fn[pr[..., 1]]]
        sc = sc.index_add(1, fn, torch.einsum("nsi,nsic->nsc", nu.abs(), Gk + Gv) / H[:, fn][..., None])
        Kk = Kn[loc[el]][:, fn]
        a = torch.einsum("nsijcb,nsi,nsc->nsjb", Kk, nu.abs(), wk.abs() + wv.abs())
        a_full = torch.zeros(len(el), op.n_p, d, U.shape[-1], dtype=U.dtype).index_add(1, fn, a)
        lift = torch.einsum("nimk,nmic->nkc", ops["D"].abs(), a_full)
        sc = sc + 0.5 * lift / H[..., None]
    return sc.transpose(1, 2).numpy()
