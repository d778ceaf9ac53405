"""Accuracy of the table-driven float64 log, log1p, exp and expm1 the kernels
use (Tang's methods, fmath.cuh), through esplit_math_eval, against the host's
libm (numpy; correctly rounded to within 1 ulp) and next to the CUDA math
library's own versions, over random arguments spanning the ranges the
residual kernels see and beyond."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2305_07181_gb300 as es
    return es


def _eval(lib, fn, x):
    xd = torch.as_tensor(x, dtype=torch.float64, device="cuda")
    yd = torch.empty_like(xd)
    rc = lib.capi.esplit_math_eval(fn, ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(yd.data_ptr()), xd.numel(),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def _ulps(a, b):
    return np.abs(a - b) / np.spacing(np.abs(b))


def _args(kind, n=400000, seed=0):
    rng = np.random.default_rng(seed)
    if kind == "log":
        return np.concatenate([np.exp(rng.uniform(-700, 700, n)), 1.0 + rng.uniform(-1e-3, 1e-3, n // 4),
                               rng.uniform(0.5, 2.0, n // 4), [1.0, 2.0, 0.5, 1e-300, 1e300]])
    if kind == "log1p":
        return np.concatenate([rng.uniform(-0.9, 3.0, n), rng.uniform(-1e-4, 1e-4, n // 4),
                               rng.uniform(-1e-12, 1e-12, n // 8), [0.0, -0.5, 1e-300]])
    if kind == "exp":
        return np.concatenate([rng.uniform(-700, 700, n), rng.uniform(-1, 1, n // 4), rng.uniform(-1e-6, 1e-6, n // 8),
                               [0.0, 1.0, -1.0, 707.9, -707.9]])
    return np.concatenate([rng.uniform(-5, 5, n), rng.uniform(-0.05, 0.05, n // 4), rng.uniform(-1e-8, 1e-8, n // 8),
                           [0.0, 1e-300, -1e-300]])


@pytest.mark.parametrize("fn,name,ref,bound", [(0, "log", np.log, 2.0), (1, "log1p", np.log1p, 2.0),
                                               (2, "exp", np.exp, 2.0), (3, "expm1", np.expm1, 2.0)])
def test_table_driven_functions(lib, fn, name, ref, bound):
    x = _args(name)
    y = _eval(lib, fn, x)
    yc = _eval(lib, fn + 4, x)
    yr = ref(x)
    u_own = _ulps(y, yr)
    u_cuda = _ulps(yc, yr)
    print(f"{name}: max ulp own {u_own.max():.2f}, CUDA library {u_cuda.max():.2f}, "
          f"mean own {u_own.mean():.3f}")
    assert u_own.max() <= bound


def test_special_arguments_defer_to_library(lib):
    x = np.array([0.0, -1.0, np.inf, np.nan, 5e-324])
    for fn in (0, 4):
        y = _eval(lib, fn, x)
        assert y[0] == -np.inf and np.isnan(y[1]) and y[2] == np.inf and np.isnan(y[3])
    e = _eval(lib, 2, np.array([-np.inf, np.inf, 800.0, -800.0, np.nan]))
    assert e[0] == 0.0 and e[1] == np.inf and e[2] == np.inf and e[3] == 0.0 and np.isnan(e[4])
