"""GPU parity on unequally spaced offsets and slownesses
(``radon_plan_create_grid`` / ``radon_batch_create_grid``, Section 4):

* lattice geometry identical to the FP64 log-polar oracle on the same grids;
* forward and adjoint against that oracle, relative L2 <= 1e-5, for jittered
  offsets with a near-offset gap and slownesses denser towards qmin, with
  several time and slowness pieces and a ragged size;
* the regular grids passed as lists give the regular plan's results;
* a 1024x1024 gather on jittered offsets against the FP64 direct sum on the
  same offsets (sampled outputs, 1e-2);
* a batch of gathers on their own offsets against single plans;
* the Radon-domain mute on given slownesses against the oracle, exactly;
* bad grids are refused with an error and the context stays usable.
"""
import dataclasses

import numpy as np
import pytest
import torch

import synth
from parity import assert_parity
from oracle import direct as odirect
from oracle import solvers
from oracle.logpolar import Desc, LogPolar

pytestmark = pytest.mark.gpu



def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def hr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1604_07651_gb300 as hr
    return hr


def _cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _pair(hr, geo, sigma=1.25, omega_c=0.35, tsplit=(0.25, 0.5), nq=1):
    plan = hr.Plan(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax,
                   sigma=sigma, omega_c=omega_c, tsplit=tsplit, n_qsplit=nq,
                   x=geo.offsets, q=geo.slownesses)
    desc = Desc(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax,
                sigma=sigma, omega_c=omega_c, tsplits=tuple(tsplit), n_qsplit=nq,
                x=geo.offsets, q_values=geo.slownesses)
    return plan, desc


CASES = {
    "jitter_256x96": (synth.irregular_geometry(256, 96, 256, 64, 0.004, 1.6, 0.2, 0.7, 11,
                                               jitter=0.4, near=0.1, q_power=1.5), {}),
    "ragged_333x150_pieces": (synth.irregular_geometry(333, 150, 301, 77, 0.006, 2.0, 0.15, 0.65, 12,
                                                       jitter=0.3, near=0.05, q_power=1.3),
                              dict(tsplit=(0.3, 0.6), nq=2)),
    "offsets_only_sigma2": (dataclasses.replace(synth.irregular_geometry(300, 120, 300, 120, 0.006, 1.8, 0.2,
                                                                         0.7, 13, jitter=0.45), slownesses=None),
                            dict(sigma=2.0, omega_c=0.25, tsplit=(0.3, 0.6))),
}


@pytest.mark.parametrize("name", list(CASES))
def test_geometry_matches_oracle_on_given_grids(hr, name):
    geo, kw = CASES[name]
    plan, desc = _pair(hr, geo, **kw)
    lp = LogPolar(desc)
    gpu = {(p["jt_lo"], p["l_lo"]): p for p in plan.pieces()}
    assert len(gpu) == len(lp.parts)
    for part in lp.parts:
        p = gpu[(part.jt_lo, part.l_lo)]
        for k in ("jt_hi", "l_hi", "Ntheta", "Nrho", "k1max", "k2max"):
            assert p[k] == getattr(part, k), k
        for k in ("alpha", "beta", "a", "O1", "O2", "a_r", "r_max", "dtheta", "drho", "theta_m"):
            assert abs(p[k] - getattr(part, k)) <= 1e-12 * max(1.0, abs(getattr(part, k))), k


@pytest.mark.parametrize("name", list(CASES))
def test_forward_and_adjoint_match_oracle_on_given_grids(hr, name):
    geo, kw = CASES[name]
    plan, desc = _pair(hr, geo, **kw)
    lp = LogPolar(desc)
    f = synth.band_limited_gather(geo, 71, n_events=6, nu=10.0)
    g = synth.random_radon_image(geo, 72)
    assert_parity(plan.forward(_cuda(f)).cpu().numpy(), lp.forward(f), what=name + " forward")
    assert_parity(plan.adjoint(_cuda(g)).cpu().numpy(), lp.adjoint(g), what=name + " adjoint")


def test_regular_grids_given_as_lists(hr):
    geo = synth.Geometry(256, 64, 256, 64, 0.004, 1.6 / 63, 0.2, 0.7)
    reg = hr.Plan(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax)
    lst = hr.Plan(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax,
                  x=list(geo.x()), q=list(geo.q()))
    assert [(p["Ntheta"], p["Nrho"]) for p in reg.pieces()] == [(p["Ntheta"], p["Nrho"]) for p in lst.pieces()]
    f = synth.band_limited_gather(geo, 73, n_events=6, nu=10.0)
    g = synth.random_radon_image(geo, 74)
    a, b = reg.forward(_cuda(f)).cpu().numpy(), lst.forward(_cuda(f)).cpu().numpy()
    assert _rel(b, a) < 1e-6
    a, b = reg.adjoint(_cuda(g)).cpu().numpy(), lst.adjoint(_cuda(g)).cpu().numpy()
    assert _rel(b, a) < 1e-6


def test_jittered_1024_against_direct_sum(hr):
    """Section 5's accuracy on 40 % jittered offsets with a 100 m near-offset
    gap and uneven slownesses: 4096 sampled outputs and gather points against
    the FP64 direct sum on the same offsets."""
    N = 1024
    geo = synth.irregular_geometry(N, N, N, N, 2.0 / (N - 1), 2.0, 0.2, 0.7, 14,
                                   jitter=0.4, near=0.1, q_power=1.5)
    f = synth.band_limited_gather(geo, 75, n_events=24, nu=15.0)
    plan = hr.Plan(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax,
                   x=geo.offsets, q=geo.slownesses)
    g = plan.forward(_cuda(f)).cpu().numpy()
    rng = np.random.default_rng(76)
    ii, li = rng.integers(0, N, 4096), rng.integers(0, N, 4096)
    ref = odirect.fwd_x_points(f, geo.dt, geo.x(), geo.tau(), geo.q(), ii, li)
    assert _rel(g[li, ii], ref) < 1e-2
    gs = synth.smooth_radon_image(geo, 77)
    fa = plan.adjoint(_cuda(gs)).cpu().numpy()
    jj, kk = rng.integers(0, N, 4096), rng.integers(0, N, 4096)
    ref = odirect.adj_x_points(gs, geo.dt, geo.x(), 0.0, geo.dtau, geo.q(), jj, kk)
    assert _rel(fa[kk, jj], ref) < 1e-2


def test_batch_on_given_grids_matches_single_plans(hr):
    geos = [synth.irregular_geometry(256, 64 + 16 * i, 200, 48 + 8 * i, 0.004, 1.2 + 0.2 * i, 0.2, 0.7,
                                     20 + i, jitter=0.35, near=0.05 * i, q_power=1.0 + 0.3 * i)
            for i in range(3)]
    spec = [dict(Nt=g.Nt, Nx=g.Nx, Ntau=g.Ntau, Nq=g.Nq, dt=g.dt, dx=g.dx, qmin=g.qmin, qmax=g.qmax,
                 x=g.offsets, q=g.slownesses) for g in geos]
    spec[1].pop("q")                                    # offsets only for one gather
    batch = hr.Batch(spec)
    fs = [synth.band_limited_gather(g, 80 + i, n_events=5, nu=10.0) for i, g in enumerate(geos)]
    imgs = batch.unpack_images(batch.forward(batch.pack([_cuda(f) for f in fs])))
    gs = [synth.random_radon_image(g, 90 + i) for i, g in enumerate(geos)]
    gp = torch.cat([_cuda(g).reshape(-1) for g in gs])
    adjs = batch.unpack_gathers(batch.adjoint(gp))
    for i, (g, f) in enumerate(zip(geos, fs)):
        plan = hr.Plan(g.Nt, g.Nx, g.Ntau, g.Nq, g.dt, g.dx, g.qmin, g.qmax, x=g.offsets,
                       q=None if i == 1 else g.slownesses)
        assert _rel(imgs[i].cpu().numpy(), plan.forward(_cuda(f)).cpu().numpy()) < 1e-6
        assert _rel(adjs[i].cpu().numpy(), plan.adjoint(_cuda(gs[i])).cpu().numpy()) < 1e-6


def test_mute_on_given_slownesses_matches_oracle(hr):
    geo, _ = CASES["jitter_256x96"]
    plan, _ = _pair(hr, geo)
    g = np.random.default_rng(78).standard_normal((geo.Nq, geo.Ntau))
    for keep in ("below", "above"):
        out = plan.mute(_cuda(g), 0.4523, 0.0371, keep=keep).cpu().numpy()
        ref = solvers.mute(g.astype(np.float32), geo.tau(), geo.q(), 0.4523, 0.0371, keep)
        np.testing.assert_array_equal(out, ref.astype(np.float32))


def test_bad_grids_are_refused(hr):
    geo = synth.Geometry(64, 16, 64, 8, 0.004, 0.05, 0.2, 0.7)
    x = list(geo.x())
    bad_x = [x[:3] + [x[1]] + x[4:], [-0.01] + x[1:], x[:8] + [float("nan")] + x[9:]]
    for bx in bad_x:
        with pytest.raises(hr.RadonError):
            hr.Plan(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax, x=bx)
    q = list(geo.q())
    with pytest.raises(hr.RadonError):
        hr.Plan(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax, q=q[::-1])
    with pytest.raises(ValueError):
        hr.Plan(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax, x=x[:-1])
    plan = hr.Plan(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax, x=x, q=q)
    f = synth.band_limited_gather(geo, 79, n_events=3, nu=10.0)
    assert np.isfinite(plan.forward(_cuda(f)).cpu().numpy()).all()
