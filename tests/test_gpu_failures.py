"""Failure paths on the GPU, made on the host (nothing faults the device):

* the allocation-failure hook (RADON_FAIL_ALLOC_AT=n) makes the n-th device
  allocation of a plan or batch creation fail: the call returns
  RADON_ERR_OOM, releases what it had allocated, and the context and later
  plans work;
* a lattice whose output-interpolation profiles fit the opt-in shared-memory
  limit but not once the kernel's own static shared arrays are counted is
  refused at plan creation (RADON_ERR_UNSUPPORTED), not at the first
  transform.
"""
import ctypes
import os

import numpy as np
import pytest
import torch

import synth
from oracle.logpolar import Desc, LogPolar
from parity import assert_parity

pytestmark = pytest.mark.gpu

OOM, UNSUPPORTED = 2, 4


@pytest.fixture(scope="module")
def hr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1604_07651_gb300 as hr
    return hr


@pytest.fixture
def fail_at(monkeypatch):
    def arm(n):
        monkeypatch.setenv("RADON_FAIL_ALLOC_AT", str(n))
    yield arm
    monkeypatch.delenv("RADON_FAIL_ALLOC_AT", raising=False)


GEO = synth.Geometry(256, 96, 200, 64, 0.004, 0.02, 0.2, 0.7)


def _plan(hr):
    return hr.Plan(GEO.Nt, GEO.Nx, GEO.Ntau, GEO.Nq, GEO.dt, GEO.dx, GEO.qmin, GEO.qmax,
                   sigma=1.25, omega_c=0.35, tsplit=(0.25, 0.5))


def test_allocation_failure_hook_reports_oom_and_leaks_nothing(hr, fail_at):
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    hits = 0
    for n in (1, 2, 3, 7, 15, 40, 100000):
        fail_at(n)
        try:
            p = _plan(hr)
        except hr.RadonError as e:
            assert e.status == OOM, e
            assert "cudaMalloc" in str(e)
            hits += 1
        else:
            assert n == 100000          # more allocations asked for than a plan makes
            p.close()
    assert hits == 6
    torch.cuda.synchronize()
    assert free0 - torch.cuda.mem_get_info()[0] < 8 << 20   # the failed creations released their memory
    # disarmed: a plan works and matches the oracle
    os.environ.pop("RADON_FAIL_ALLOC_AT", None)
    p = _plan(hr)
    f = synth.band_limited_gather(GEO, 81, n_events=5, nu=10.0)
    ref = LogPolar(Desc(GEO.Nt, GEO.Nx, GEO.Ntau, GEO.Nq, GEO.dt, GEO.dx, GEO.qmin, GEO.qmax,
                        sigma=1.25, omega_c=0.35, tsplits=(0.25, 0.5))).forward(f)
    assert_parity(p.forward(torch.tensor(f, dtype=torch.float32, device="cuda")).cpu().numpy(), ref,
                  what="after failed creations")
    p.close()


def test_allocation_failure_hook_in_batch_creation(hr, fail_at):
    geos = synth.batch_geometries(6)
    dicts = [dict(Nt=g.Nt, Nx=g.Nx, Ntau=g.Ntau, Nq=g.Nq, dt=g.dt, dx=g.dx, qmin=g.qmin, qmax=g.qmax)
             for g in geos]
    for n in (1, 9, 60):
        fail_at(n)
        with pytest.raises(hr.RadonError) as ei:
            hr.Batch(dicts)
        assert ei.value.status == OOM
    os.environ.pop("RADON_FAIL_ALLOC_AT", None)
    b = hr.Batch(dicts)
    f = b.pack([torch.tensor(synth.batch_gather(g, i), dtype=torch.float32) for i, g in enumerate(geos)])
    assert torch.isfinite(b.forward(f)).all()
    b.close()


def test_profiles_beyond_shared_memory_refused_at_creation(hr):
    """9 time pieces on a 512^2 gather with slownesses up to 3 s/km: the
    oversampling is chosen (host-only geometry) so that the nine rho profiles
    of an output column take just under the opt-in shared memory per block,
    inside the interpolation kernel's static shared arrays (a few hundred
    bytes): the plan must be refused at creation."""
    from paper_1604_07651_gb300 import _lib
    L = _lib.load()
    optin = torch.cuda.get_device_properties(0).shared_memory_per_block_optin
    ts = [0.7 / 1.6 ** k for k in range(8)][::-1]
    N = 512

    def desc(sigma):
        d = _lib.RadonDesc()
        _lib.check(L.radon_desc_init(ctypes.byref(d), N, N, N, N, 2.0 / (N - 1), 2.0 / (N - 1), 0.0, 3.0))
        d.sigma = sigma
        d.n_tsplit = len(ts)
        for i, v in enumerate(ts):
            d.tsplit[i] = v
        d.device = torch.cuda.current_device()
        return d

    found = None
    for sigma in np.arange(8.0, 12.0, 0.01):
        d = desc(float(sigma))
        n = ctypes.c_int(0)
        infos = (_lib.RadonPieceInfo * 16)()
        if L.radon_geometry(ctypes.byref(d), ctypes.byref(n), infos, 16) != 0:
            continue
        pieces = [infos[i] for i in range(n.value)]
        need = len(pieces) * max(p.Nrho for p in pieces) * 4
        if optin - 256 < need <= optin:
            assert max(p.Prho for p in pieces) <= 12288 and max(p.Ptheta for p in pieces) <= 6144
            found = d
            break
        if need > optin:
            break
    assert found is not None, "no geometry in the margin"
    h = ctypes.c_void_p()
    st = L.radon_plan_create_ex(ctypes.byref(h), ctypes.byref(found))
    assert st == UNSUPPORTED, (st, L.radon_last_error())
    assert b"profiles" in L.radon_last_error()
    assert not h.value
