"""ctypes binding of the C ABI in include/esplit.h (argument marshalling only).

Every function here has the name of the C entry point it calls.  The shared
library is built in-tree by ``paper_2305_07181_gb300.build``; importing this
module without it raises ImportError -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libesplit.so")

ESPLIT_OK = 0
ESPLIT_ERR_ARG = -1
ESPLIT_ERR_CUDA = -2
ESPLIT_ERR_MESH = -3
ESPLIT_ERR_NONPHYSICAL = -4
ESPLIT_ERR_RRK_NO_ROOT = -5
ESPLIT_ERR_UNSUPPORTED = -6
ESPLIT_ERR_STATE = -7

ESPLIT_FP64 = 0
ESPLIT_FP32_BULK = 1
ESPLIT_FP32 = 2
ESPLIT_SCHEME_SPLIT = 0
ESPLIT_SCHEME_HADAMARD = 1
ESPLIT_SCHEME_HYBRID = 2
ESPLIT_SCHEME_HADAMARD_IR = 3

ERROR_NAMES = {0: "OK", -1: "ERR_ARG", -2: "ERR_CUDA", -3: "ERR_MESH", -4: "ERR_NONPHYSICAL",
               -5: "ERR_RRK_NO_ROOT", -6: "ERR_UNSUPPORTED", -7: "ERR_STATE"}


class esplit_params(ctypes.Structure):
    _fields_ = [("gam", ctypes.c_double), ("beta", ctypes.c_double), ("R", ctypes.c_double),
                ("mu", ctypes.c_double), ("Pr", ctypes.c_double), ("dissipation", ctypes.c_int),
                ("viscous", ctypes.c_int), ("heat_flux", ctypes.c_int), ("scheme", ctypes.c_int),
                ("precision", ctypes.c_int)]


class esplit_stepinfo(ctypes.Structure):
    _fields_ = [("g", ctypes.c_double), ("estimate", ctypes.c_double), ("S_before", ctypes.c_double),
                ("S_after", ctypes.c_double), ("iterations", ctypes.c_int), ("status", ctypes.c_int),
                ("stage_rate", ctypes.c_double * 4)]


_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.c_int

_SIGNATURES = {
    "esplit_version": (_I, []),
    "esplit_math_eval": (_I, [_I, _P, _P, ctypes.c_size_t, _P]),
    "esplit_measure_fp64": (_I, [_I, _I, _D, _D]),
    "esplit_create": (_I, [ctypes.POINTER(_P), _I, _I]),
    "esplit_destroy": (None, [_P]),
    "esplit_upload_operator": (_I, [_P, _I, _I, _I, _P, _P, _P, _P, _P]),
    "esplit_upload_mesh": (_I, [_P, _I, _P, _P, _P, _P, _P]),
    "esplit_set_params": (_I, [_P, ctypes.POINTER(esplit_params)]),
    "esplit_get_params": (_I, [_P, ctypes.POINTER(esplit_params)]),
    "esplit_set_hybrid_flags": (_I, [_P, _P, _I]),
    "esplit_set_boundary_states": (_I, [_P, _I, _P, _P]),
    "esplit_detect_hybrid": (_I, [_P, _P, ctypes.c_double, ctypes.POINTER(ctypes.c_int), _P]),
    "esplit_get_hybrid_flags": (_I, [_P, _P]),
    "esplit_residual": (_I, [_P, _P, _P, _P]),
    "esplit_residual_noalloc": (_I, [_P, _P, _P, _P]),
    "esplit_residual_host": (_I, [_P, _P, _P, _P]),
    "esplit_entropy": (_I, [_P, _P, _D, _P]),
    "esplit_entropy_rate": (_I, [_P, _P, _P, _D, _P]),
    "esplit_rrk_step": (_I, [_P, _P, ctypes.c_double, _D, ctypes.POINTER(esplit_stepinfo), _P]),
    "esplit_rrk_step_host": (_I, [_P, _P, ctypes.c_double, _D, ctypes.POINTER(esplit_stepinfo), _P]),
    "esplit_rrk_steps": (_I, [_P, _P, ctypes.c_double, ctypes.c_int, _D, ctypes.POINTER(esplit_stepinfo),
                              ctypes.POINTER(ctypes.c_int), _P]),
    "esplit_residual_vjp": (_I, [_P, _P, _P, _P, _P]),
    "esplit_entropy_grad": (_I, [_P, _P, _P, _P]),
    "esplit_rrk_step_vjp": (_I, [_P, _P, ctypes.c_double, _P, _P, _D, _P]),
    "esplit_profile_enable": (_I, [_P, _I]),
    "esplit_profile_read": (_I, [_P, _D, ctypes.POINTER(ctypes.c_longlong), _I]),
    "esplit_get_status": (_I, [_P]),
    "esplit_last_error": (ctypes.c_char_p, [_P]),
    "esplit_launch_count": (ctypes.c_longlong, [_P]),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} is missing "
                          "(run `python -m paper_2305_07181_gb300.build`)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def exported_names():
    return list(_SIGNATURES)


# thin wrappers with the C names -------------------------------------------------

def esplit_version() -> int:
    return lib.esplit_version()


def esplit_create(dim: int, device: int = 0):
    h = _P()
    rc = lib.esplit_create(ctypes.byref(h), dim, device)
    return rc, h


def esplit_destroy(ctx) -> None:
    lib.esplit_destroy(ctx)


def esplit_upload_operator(ctx, n_p, n_fac, n_f, H_ref, Q_ref, facet_nodes, facet_w, ref_normals) -> int:
    return lib.esplit_upload_operator(ctx, n_p, n_fac, n_f, H_ref, Q_ref, facet_nodes, facet_w, ref_normals)


def esplit_upload_mesh(ctx, n_e, J, Lam, nu, pair, hmin) -> int:
    return lib.esplit_upload_mesh(ctx, n_e, J, Lam, nu, pair, hmin)


def esplit_set_params(ctx, prm: esplit_params) -> int:
    return lib.esplit_set_params(ctx, ctypes.byref(prm))


def esplit_get_params(ctx):
    prm = esplit_params()
    rc = lib.esplit_get_params(ctx, ctypes.byref(prm))
    return rc, prm


def esplit_set_hybrid_flags(ctx, flags_ptr, n_e) -> int:
    return lib.esplit_set_hybrid_flags(ctx, flags_ptr, n_e)


def esplit_set_boundary_states(ctx, n_b, slots_ptr, states_ptr) -> int:
    return lib.esplit_set_boundary_states(ctx, n_b, slots_ptr, states_ptr)


def esplit_detect_hybrid(ctx, u_ptr, threshold, stream=None):
    n = ctypes.c_int()
    rc = lib.esplit_detect_hybrid(ctx, u_ptr, threshold, ctypes.byref(n), stream)
    return rc, n.value


def esplit_get_hybrid_flags(ctx, flags_ptr) -> int:
    return lib.esplit_get_hybrid_flags(ctx, flags_ptr)


def esplit_residual(ctx, u_ptr, r_ptr, stream=None) -> int:
    return lib.esplit_residual(ctx, u_ptr, r_ptr, stream)


def esplit_residual_noalloc(ctx, u_ptr, r_ptr, stream=None) -> int:
    """Residual whose facet scratch is the library's static device array (no
    allocation of any kind); see include/esplit.h for the size limit and the
    rule that calls overlapping on the GPU race on that array."""
    return lib.esplit_residual_noalloc(ctx, u_ptr, r_ptr, stream)


def esplit_residual_host(ctx, u_ptr, r_ptr, stream=None) -> int:
    return lib.esplit_residual_host(ctx, u_ptr, r_ptr, stream)


def esplit_entropy(ctx, u_ptr, stream=None):
    out = ctypes.c_double()
    rc = lib.esplit_entropy(ctx, u_ptr, ctypes.byref(out), stream)
    return rc, out.value


def esplit_entropy_rate(ctx, u_ptr, r_ptr, stream=None):
    out = ctypes.c_double()
    rc = lib.esplit_entropy_rate(ctx, u_ptr, r_ptr, ctypes.byref(out), stream)
    return rc, out.value


def esplit_rrk_step(ctx, u_ptr, dt, stream=None):
    g = ctypes.c_double()
    info = esplit_stepinfo()
    rc = lib.esplit_rrk_step(ctx, u_ptr, dt, ctypes.byref(g), ctypes.byref(info), stream)
    return rc, g.value, info


def esplit_rrk_steps(ctx, u_ptr, dt, n_steps, stream=None):
    g = (ctypes.c_double * max(n_steps, 1))()
    info = esplit_stepinfo()
    done = ctypes.c_int()
    rc = lib.esplit_rrk_steps(ctx, u_ptr, dt, n_steps, g, ctypes.byref(info), ctypes.byref(done), stream)
    return rc, list(g)[:done.value], info, done.value


def esplit_rrk_step_host(ctx, u_host_ptr, dt, stream=None):
    g = ctypes.c_double()
    info = esplit_stepinfo()
    rc = lib.esplit_rrk_step_host(ctx, u_host_ptr, dt, ctypes.byref(g), ctypes.byref(info), stream)
    return rc, g.value, info


def esplit_entropy_grad(ctx, u_ptr, grad_ptr, stream=None) -> int:
    return lib.esplit_entropy_grad(ctx, u_ptr, grad_ptr, stream)


def esplit_rrk_step_vjp(ctx, u_ptr, dt, ubar_next_ptr, ubar_ptr, stream=None):
    g = ctypes.c_double()
    rc = lib.esplit_rrk_step_vjp(ctx, u_ptr, dt, ubar_next_ptr, ubar_ptr, ctypes.byref(g), stream)
    return rc, g.value


PROFILE_GROUPS = ("face", "split_volume", "hadamard_volume", "entropy_reduce", "root_solve", "stage_update",
                  "viscous")


def esplit_profile_enable(ctx, on: bool) -> int:
    return lib.esplit_profile_enable(ctx, int(bool(on)))


def esplit_profile_read(ctx):
    n = len(PROFILE_GROUPS)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_longlong * n)()
    rc = lib.esplit_profile_read(ctx, ms, cnt, n)
    return rc, {g: (ms[i], cnt[i]) for i, g in enumerate(PROFILE_GROUPS)}


def esplit_residual_vjp(ctx, u_ptr, cot_ptr, grad_ptr, stream=None) -> int:
    return lib.esplit_residual_vjp(ctx, u_ptr, cot_ptr, grad_ptr, stream)


def esplit_get_status(ctx) -> int:
    return lib.esplit_get_status(ctx)


def esplit_last_error(ctx) -> str:
    s = lib.esplit_last_error(ctx)
    return s.decode() if s else ""


def esplit_launch_count(ctx) -> int:
    return lib.esplit_launch_count(ctx)


def esplit_measure_fp64(device: int = 0, mode: int = 0):
    """(rc, rate, ms per timed launch): FLOP/s of float64 FMA chains (mode 0),
    float64 tensor-core MMA chains (1), both interleaved (2), float32 FMA
    chains (3); operations per second of float64 divide (4), the library's
    log (5) and exp (6), the CUDA library's log (7) and exp (8), a
    float64 -> float32 -> float64 round trip with an FMA (9); FLOP/s of the
    warp-level bf16 tensor-core MMA (10)."""
    f, ms = ctypes.c_double(), ctypes.c_double()
    rc = lib.esplit_measure_fp64(device, mode, ctypes.byref(f), ctypes.byref(ms))
    return rc, f.value, ms.value


def esplit_math_eval(fn, x_ptr, y_ptr, n, stream=None) -> int:
    return lib.esplit_math_eval(fn, x_ptr, y_ptr, n, stream)
