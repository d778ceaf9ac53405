"""esplit_residual_noalloc: the residual for callers that must not allocate
device memory while they run (their device memory is owned by a pool
allocator of their own, or their loop cannot absorb the synchronisation that
cudaMalloc/cudaFree can cause).  Its facet scratch is a static device array
of the library, so this file is collected last: if it fails, a run that stops
at the first failure has already run every other test.  It must pass both
alone in a fresh process and after the other tests."""
import ctypes

import numpy as np
import pytest
import torch

from esplit_inputs import tri_operator, periodic_tri_mesh, states

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the FP64 parity tolerance of the other GPU tests


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2305_07181_gb300 as es
    return es


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("p,scheme", [(2, "split"), (3, "hybrid"), (4, "hadamard")])
def test_noalloc_matches_residual_twice(lib, p, scheme):
    op = tri_operator(p)
    m = periodic_tri_mesh(op, 9, 10.0, 0.05)
    s = lib.Solver(op, m, lib.Params(scheme=scheme, dissipation=True))
    if scheme == "hybrid":
        s.set_hybrid_flags(np.random.default_rng(1).integers(0, 2, m.n_e))
    ref = s.empty()
    for call in range(2):  # two calls in a row, on different states
        u = s.to_device(states.add_uniform_noise(states.isentropic_vortex(m), 1e-3, 100 + call))
        s.residual(u, ref)
        out = torch.full_like(ref, float("nan"))
        rc = lib.capi.esplit_residual_noalloc(s.ctx, _ptr(u), _ptr(out), _stream())
        assert rc == 0, lib.capi.esplit_last_error(s.ctx)
        torch.cuda.synchronize()
        num = (out - ref).abs().amax(dim=(0, 2))
        den = ref.abs().amax(dim=(0, 2))
        assert float((num / den).max()) <= TOL
    assert s.status() == 0
    s.close()


def test_noalloc_rejects_meshes_beyond_its_scratch(lib):
    op = tri_operator(4)           # n_c * n_slot = 4 * 15 = 60 doubles per element
    m = periodic_tri_mesh(op, 192, 10.0, 0.05)   # 73,728 elements -> 4.4e6 > 2^21
    s = lib.Solver(op, m, lib.Params())
    u = s.to_device(states.isentropic_vortex(m))
    out = s.empty()
    rc = lib.capi.esplit_residual_noalloc(s.ctx, _ptr(u), _ptr(out), _stream())
    assert rc == lib.capi.ESPLIT_ERR_ARG
    msg = lib.capi.esplit_last_error(s.ctx)
    assert "2097152" in msg and "4423680" in msg
    s.close()


def test_noalloc_viscous_matches_residual(lib):
    """With the viscous terms on, the no-allocation call uses the viscous
    scratch the context allocated when they were switched on."""
    op = tri_operator(2)
    m = periodic_tri_mesh(op, 5, 10.0, 0.05)
    s = lib.Solver(op, m, lib.Params(mu=0.05, viscous=True, dissipation=True))
    u = s.to_device(states.random_positive_state(m.n_e, 2, op.n_p, seed=70))
    ref = s.residual(u)
    out = torch.full_like(ref, float("nan"))
    rc = lib.capi.esplit_residual_noalloc(s.ctx, _ptr(u), _ptr(out), _stream())
    assert rc == 0, lib.capi.esplit_last_error(s.ctx)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    s.close()


def test_noalloc_fp32_bulk_matches_residual(lib):
    """FP32-bulk precision: the no-allocation call (facet kernel first, the
    uncached float32 split variant) against esplit_residual (the cached
    order) at the FP32-bulk bound of the parity tests, on two calls."""
    op = tri_operator(3)
    m = periodic_tri_mesh(op, 9, 10.0, 0.05)
    s = lib.Solver(op, m, lib.Params(dissipation=True, precision="fp32_bulk"))
    ref = s.empty()
    for call in range(2):
        u = s.to_device(states.add_uniform_noise(states.isentropic_vortex(m), 1e-3, 110 + call))
        s.residual(u, ref)
        out = torch.full_like(ref, float("nan"))
        rc = lib.capi.esplit_residual_noalloc(s.ctx, _ptr(u), _ptr(out), _stream())
        assert rc == 0, lib.capi.esplit_last_error(s.ctx)
        torch.cuda.synchronize()
        num = (out - ref).abs().amax(dim=(0, 2))
        den = ref.abs().amax(dim=(0, 2))
        assert float((num / den).max()) <= 1e-11
    s.close()


def test_noalloc_fp32_matches_residual(lib):
    """Float32 precision: the no-allocation call runs the same kernels in the
    same order as esplit_residual, with its float32 facet scratch in the
    static array: equal results, on two calls."""
    op = tri_operator(3)
    m = periodic_tri_mesh(op, 9, 10.0, 0.05)
    s = lib.Solver(op, m, lib.Params(dissipation=True, precision="fp32"))
    ref = s.empty()
    for call in range(2):
        u = s.to_device(states.add_uniform_noise(states.isentropic_vortex(m), 1e-3, 130 + call))
        s.residual(u, ref)
        out = torch.full_like(ref, float("nan"))
        rc = lib.capi.esplit_residual_noalloc(s.ctx, _ptr(u), _ptr(out), _stream())
        assert rc == 0, lib.capi.esplit_last_error(s.ctx)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    s.close()


def test_noalloc_allocates_nothing(lib):
    """After a first call (which looks up the static array and loads the
    kernels it launches), further calls leave the device's free memory and
    PyTorch's allocator untouched, and with kernel timing enabled on the
    context they record no timing (timing would create CUDA events)."""
    op = tri_operator(2)
    m = periodic_tri_mesh(op, 9, 10.0, 0.05)
    s = lib.Solver(op, m, lib.Params(dissipation=True))
    u = s.to_device(states.add_uniform_noise(states.isentropic_vortex(m), 1e-3, 120))
    out = s.empty()
    rc = lib.capi.esplit_residual_noalloc(s.ctx, _ptr(u), _ptr(out), _stream())
    assert rc == 0, lib.capi.esplit_last_error(s.ctx)
    s.profile(True)
    s.profile_read()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        rc = lib.capi.esplit_residual_noalloc(s.ctx, _ptr(u), _ptr(out), _stream())
        assert rc == 0, lib.capi.esplit_last_error(s.ctx)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0
    assert all(v[1] == 0 for v in s.profile_read().values())
    # the context's own residual still records its timing
    s.residual(u, out)
    assert any(v[1] > 0 for v in s.profile_read().values())
    s.profile(False)
    s.close()
