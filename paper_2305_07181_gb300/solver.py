"""Convenience wrapper over the C ABI: one library context bound to one
operator and mesh.  Argument marshalling only -- numpy arrays for uploads,
torch CUDA float64 tensors (device memory and streams) for states.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import capi


class EsplitError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{capi.ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t: torch.Tensor):
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("state tensors must be contiguous float64 CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


@dataclass
class Params:
    gam: float = 1.4
    beta: float = 2.5
    R: float = 1.0
    mu: float = 0.0
    Pr: float = 0.71
    dissipation: bool = False
    viscous: bool = False
    heat_flux: bool = True
    scheme: str = "split"          # "split" | "hadamard" | "hybrid" | "hadamard_ir"
    precision: str = "fp64"        # "fp64" | "fp32_bulk" | "fp32" (include/esplit.h ESPLIT_FP*)

    def to_c(self) -> capi.esplit_params:
        sch = {"split": capi.ESPLIT_SCHEME_SPLIT, "hadamard": capi.ESPLIT_SCHEME_HADAMARD,
               "hybrid": capi.ESPLIT_SCHEME_HYBRID, "hadamard_ir": capi.ESPLIT_SCHEME_HADAMARD_IR}[self.scheme]
        prec = {"fp64": capi.ESPLIT_FP64, "fp32_bulk": capi.ESPLIT_FP32_BULK,
                "fp32": capi.ESPLIT_FP32}[self.precision]
        return capi.esplit_params(self.gam, self.beta, self.R, self.mu, self.Pr, int(self.dissipation),
                                  int(self.viscous), int(self.heat_flux), sch, prec)


class Solver:
    """Library context with an uploaded reference operator and mesh.

    ``op`` needs attributes d, n_p, n_fac, n_f, H, Q, facet_nodes, facet_w,
    ref_normals; ``mesh`` needs n_e, J, Lam, nu, pair, hmin (numpy arrays in
    the layouts of include/esplit.h)."""

    def __init__(self, op, mesh, params: Params | None = None, device: int = 0):
        self.device = device
        rc, self.ctx = capi.esplit_create(op.d, device)
        if rc:
            raise EsplitError(rc, "esplit_create failed")
        self.n_e, self.n_p, self.n_c = mesh.n_e, op.n_p, op.d + 2
        self.shape = (self.n_e, self.n_c, self.n_p)
        H = np.ascontiguousarray(op.H, dtype=np.float64)
        Q = np.ascontiguousarray(op.Q, dtype=np.float64)
        fnodes = np.ascontiguousarray(op.facet_nodes, dtype=np.int32)
        fw = np.ascontiguousarray(op.facet_w, dtype=np.float64)
        rn = np.ascontiguousarray(op.ref_normals, dtype=np.float64)
        self._check(capi.esplit_upload_operator(self.ctx, op.n_p, op.n_fac, op.n_f, _ptr(H), _ptr(Q), _ptr(fnodes),
                                                _ptr(fw), _ptr(rn)))
        J = np.ascontiguousarray(mesh.J, dtype=np.float64)
        Lam = np.ascontiguousarray(mesh.Lam, dtype=np.float64)
        nu = np.ascontiguousarray(mesh.nu, dtype=np.float64)
        pair = np.ascontiguousarray(mesh.pair, dtype=np.int32)
        hmin = np.ascontiguousarray(mesh.hmin, dtype=np.float64)
        self._check(capi.esplit_upload_mesh(self.ctx, mesh.n_e, _ptr(J), _ptr(Lam), _ptr(nu), _ptr(pair),
                                            _ptr(hmin)))
        self.params = params or Params()
        self.set_params(self.params)

    # -- lifecycle ---------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None):
            capi.esplit_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc:
            raise EsplitError(rc, capi.esplit_last_error(self.ctx))
        return rc

    # -- configuration -------------------------------------------------------
    def set_params(self, params: Params):
        self.params = params
        self._check(capi.esplit_set_params(self.ctx, params.to_c()))

    def set_hybrid_flags(self, flags):
        f = np.ascontiguousarray(np.asarray(flags, dtype=np.uint8))
        self._check(capi.esplit_set_hybrid_flags(self.ctx, _ptr(f), self.n_e))

    def set_boundary_states(self, slots, states):
        """Exterior states (n_b, n_c) of the mesh's boundary facet slots
        (flat indices element * n_slot + slot)."""
        sl = np.ascontiguousarray(np.asarray(slots, dtype=np.int32))
        st = np.ascontiguousarray(np.asarray(states, dtype=np.float64))
        self._check(capi.esplit_set_boundary_states(self.ctx, len(sl), _ptr(sl), _ptr(st)))

    def detect_hybrid(self, u: torch.Tensor, threshold: float = 1.1, stream=None) -> int:
        rc, n = capi.esplit_detect_hybrid(self.ctx, _dptr(u), float(threshold), _stream(stream))
        self._check(rc)
        return n

    def hybrid_flags(self) -> np.ndarray:
        f = np.empty(self.n_e, dtype=np.uint8)
        self._check(capi.esplit_get_hybrid_flags(self.ctx, _ptr(f)))
        return f

    # -- evaluation ------------------------------------------------------------
    def empty(self):
        return torch.empty(self.shape, dtype=torch.float64, device=f"cuda:{self.device}")

    def to_device(self, u):
        return torch.as_tensor(np.ascontiguousarray(u, dtype=np.float64)).to(f"cuda:{self.device}")

    def residual(self, u: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        out = self.empty() if out is None else out
        self._check(capi.esplit_residual(self.ctx, _dptr(u), _dptr(out), _stream(stream)))
        return out

    def residual_host(self, u_host: np.ndarray, out: np.ndarray | None = None, stream=None) -> np.ndarray:
        if out is None:
            out = np.empty(self.shape, dtype=np.float64)
        if not (u_host.flags.c_contiguous and out.flags.c_contiguous):
            raise ValueError("host buffers must be C-contiguous float64")
        self._check(capi.esplit_residual_host(self.ctx, _ptr(u_host), _ptr(out), _stream(stream)))
        return out

    def entropy(self, u: torch.Tensor, stream=None) -> float:
        rc, v = capi.esplit_entropy(self.ctx, _dptr(u), _stream(stream))
        self._check(rc)
        return v

    def entropy_rate(self, u: torch.Tensor, r: torch.Tensor, stream=None) -> float:
        rc, v = capi.esplit_entropy_rate(self.ctx, _dptr(u), _dptr(r), _stream(stream))
        self._check(rc)
        return v

    def rrk_step(self, u: torch.Tensor, dt: float, stream=None):
        rc, g, info = capi.esplit_rrk_step(self.ctx, _dptr(u), float(dt), _stream(stream))
        self._check(rc)
        return g, info

    def rrk_steps(self, u: torch.Tensor, dt: float, n_steps: int, stream=None):
        """n_steps relaxation RK4 steps in place, launched as a recorded CUDA
        graph per step; returns (list of g, info of the last step).  On a
        failing step raises EsplitError with ``n_done`` (completed steps) and
        ``g`` (their g values) attached; u then holds the state after them."""
        rc, g, info, done = capi.esplit_rrk_steps(self.ctx, _dptr(u), float(dt), int(n_steps), _stream(stream))
        if rc:
            err = EsplitError(rc, capi.esplit_last_error(self.ctx))
            err.n_done, err.g = done, g
            raise err
        return g, info

    def rrk_step_host(self, u_host: np.ndarray, dt: float, stream=None):
        if not (u_host.flags.c_contiguous and u_host.dtype == np.float64):
            raise ValueError("host state must be C-contiguous float64")
        rc, g, info = capi.esplit_rrk_step_host(self.ctx, _ptr(u_host), float(dt), _stream(stream))
        self._check(rc)
        return g, info

    def entropy_grad(self, u: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        out = self.empty() if out is None else out
        self._check(capi.esplit_entropy_grad(self.ctx, _dptr(u), _dptr(out), _stream(stream)))
        return out

    def rrk_step_vjp(self, u: torch.Tensor, dt: float, ubar_next: torch.Tensor, out: torch.Tensor | None = None,
                     stream=None):
        out = self.empty() if out is None else out
        rc, g = capi.esplit_rrk_step_vjp(self.ctx, _dptr(u), float(dt), _dptr(ubar_next), _dptr(out),
                                         _stream(stream))
        self._check(rc)
        return out, g

    def profile(self, on: bool = True):
        self._check(capi.esplit_profile_enable(self.ctx, on))

    def profile_read(self):
        rc, d = capi.esplit_profile_read(self.ctx)
        self._check(rc)
        return d

    def residual_vjp(self, u: torch.Tensor, cot: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        out = self.empty() if out is None else out
        self._check(capi.esplit_residual_vjp(self.ctx, _dptr(u), _dptr(cot), _dptr(out), _stream(stream)))
        return out

    def status(self) -> int:
        return capi.esplit_get_status(self.ctx)

    def launch_count(self) -> int:
        return capi.esplit_launch_count(self.ctx)
