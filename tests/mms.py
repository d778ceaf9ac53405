"""Source term of the Sec. 7.4 manufactured solution (Table 4).

With rho = 2 + 0.1 sin(phi), phi = pi (sum_i x_i - 0.6 t), V_i = 1 and total
energy e = rho^2 (p = (gam - 1)(rho^2 - rho d / 2)), the velocity is constant,
so the viscous stress vanishes and the viscous flux is the heat flux alone,
kappa dT/dx_i with T = p/(rho R) = (gam - 1)(rho - d/2)/R and
kappa = mu gam R/((gam - 1) Pr).  Substituting into
dU/dt + sum_i dF^I_i/dx_i = sum_i dF^V_i/dx_i + S (Eq. (5)) gives, with
rho' = d rho/dx_j = 0.1 pi cos(phi) (every j), rho'' = -0.1 pi^2 sin(phi) and
p' = (gam - 1)(2 rho - d/2) rho':
  S_rho = (d - 0.6) rho'
  S_m_k = (d - 0.6) rho' + p'                      (k = 1..d)
  S_e   = 2 rho rho' (d - 0.6) + d p' - d mu gam rho'' / Pr.
The semi-discrete system integrated is du/dt = r(u) + S(x, t), r the residual.
"""
import numpy as np


def mms_source(x, t, gam=1.4, mu=0.01, Pr=0.71):
    """x (d, ...) -> S (d + 2, ...)."""
    d = x.shape[0]
    phi = np.pi * (np.sum(x, axis=0) - 0.6 * t)
    rho = 2.0 + 0.1 * np.sin(phi)
    r1 = 0.1 * np.pi * np.cos(phi)
    r2 = -0.1 * np.pi ** 2 * np.sin(phi)
    p1 = (gam - 1.0) * (2.0 * rho - 0.5 * d) * r1
    s_rho = (d - 0.6) * r1
    s_m = s_rho + p1
    s_e = 2.0 * rho * r1 * (d - 0.6) + d * p1 - d * mu * gam * r2 / Pr
    return np.stack([s_rho] + [s_m] * d + [s_e])


def mms_source_nodes(mesh, t, **kw):
    """The source at the mesh nodes, (n_e, d+2, n_p)."""
    return np.ascontiguousarray(np.moveaxis(mms_source(np.moveaxis(mesh.x, 1, 0), t, **kw), 0, 1))
