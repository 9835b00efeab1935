"""radon_fwd_noalloc: the forward transform for callers that cannot allocate.

Some callers cannot call cudaMalloc when they run: their host framework has
reserved the whole device for its own pool, or the deployment must keep a
fixed device footprint, or the loop cannot take the device-wide
synchronisation that cudaMalloc/cudaFree can cause. radon_fwd_noalloc serves
them with its work memory in a static device array of the library. These
checks call it through the C ABI and compare it with radon_fwd, the regular
entry point, on two calls in a row (the second sees the first call's leftovers
in the shared array). This file is collected last on purpose.
"""
import ctypes

import pytest
import torch

import synth
from parity import assert_parity   # the bounds of the other GPU parity tests

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_07651_gb300 import _lib
    return _lib


def _plan(lib, geo, **kw):
    L = lib.load()
    d = lib.RadonDesc()
    lib.check(L.radon_desc_init(ctypes.byref(d), geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx,
                                geo.qmin, geo.qmax))
    d.device = torch.cuda.current_device()
    for k, v in kw.items():
        setattr(d, k, v)
    h = ctypes.c_void_p()
    lib.check(L.radon_plan_create_ex(ctypes.byref(h), ctypes.byref(d)))
    return h


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_forward_matches_regular_forward_twice(lib):
    L = lib.load()
    geo = synth.Geometry(300, 96, 280, 72, 0.005, 0.02, 0.2, 0.7)
    plan = _plan(lib, geo, n_qsplit=2)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    try:
        for tag in (51, 52):
            f = torch.tensor(synth.band_limited_gather(geo, tag, n_events=6, nu=10.0),
                             dtype=torch.float32, device="cuda")
            g_ref = torch.empty((geo.Nq, geo.Ntau), dtype=torch.float32, device="cuda")
            g = torch.full((geo.Nq, geo.Ntau), float("nan"), dtype=torch.float32, device="cuda")
            lib.check(L.radon_fwd(plan, _ptr(f), _ptr(g_ref), stream))
            lib.check(L.radon_fwd_noalloc(plan, _ptr(f), _ptr(g), stream))
            torch.cuda.synchronize()
            assert_parity(g.double().cpu().numpy(), g_ref.double().cpu().numpy(), what=f"no-alloc call {tag}")
    finally:
        L.radon_plan_destroy(plan)


def test_noalloc_forward_with_quintic_splines(lib):
    """The six-tap kernels through the static work area as well."""
    L = lib.load()
    geo = synth.Geometry(256, 96, 200, 64, 0.004, 0.02, 0.2, 0.7)
    plan = _plan(lib, geo, spline_order=5)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    try:
        f = torch.tensor(synth.band_limited_gather(geo, 53, n_events=6, nu=10.0), dtype=torch.float32, device="cuda")
        g_ref = torch.empty((geo.Nq, geo.Ntau), dtype=torch.float32, device="cuda")
        g = torch.full((geo.Nq, geo.Ntau), float("nan"), dtype=torch.float32, device="cuda")
        lib.check(L.radon_fwd(plan, _ptr(f), _ptr(g_ref), stream))
        lib.check(L.radon_fwd_noalloc(plan, _ptr(f), _ptr(g), stream))
        torch.cuda.synchronize()
        assert_parity(g.double().cpu().numpy(), g_ref.double().cpu().numpy(), what="quintic no-alloc")
    finally:
        L.radon_plan_destroy(plan)


def test_noalloc_rejects_plans_beyond_the_static_area(lib):
    L = lib.load()
    geo = synth.Geometry(2048, 2048, 2048, 2048, 2.0 / 2047, 2.0 / 2047, 0.2, 0.7)
    plan = _plan(lib, geo)
    try:
        f = torch.zeros((geo.Nx, geo.Nt), dtype=torch.float32, device="cuda")
        g = torch.zeros((geo.Nq, geo.Ntau), dtype=torch.float32, device="cuda")
        st = L.radon_fwd_noalloc(plan, _ptr(f), _ptr(g), None)
        assert st == 4  # RADON_ERR_UNSUPPORTED
        assert "bytes" in L.radon_last_error().decode()
        assert L.radon_fwd_noalloc(None, _ptr(f), _ptr(g), None) == 1
    finally:
        L.radon_plan_destroy(plan)
