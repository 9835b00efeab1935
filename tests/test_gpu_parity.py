"""GPU parity: the CUDA log-polar path (through the C ABI) against the oracle.

* against the FP64 log-polar oracle on the same lattices: relative L2 <= 1e-5,
  every element within 1e-5 of the result's peak and every output column /
  gather trace within 1e-4 of its own norm (tests/parity.py), forward and
  adjoint, up to the full 2048x2048 benchmark workload; lattice geometry
  identical;
* against the FP64 direct summation over hyperbolas: relative L2 <= 1e-2 on
  band-limited data (Section 5), also at 2048x2048 on sampled outputs;
* inner-product test (Eq. (16)) to the paper's FP32 level, 1e-5;
* the GPU direct-summation comparator against the oracle's direct sum.
"""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import direct as odirect
from parity import assert_parity
from oracle.logpolar import Desc, LogPolar

pytestmark = pytest.mark.gpu


METHOD_TOL = 1e-2    # log-polar vs direct summation, band-limited data


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def hr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1604_07651_gb300 as hr
    return hr


def _pair(hr, geo, sigma=1.25, omega_c=0.35, tsplit=(0.25, 0.5), nq=1, tau0=0.0, dtau=0.0, rows_per_band=None):
    plan = hr.Plan(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax,
                   tau0=tau0, dtau=dtau, sigma=sigma, omega_c=omega_c, tsplit=tsplit, n_qsplit=nq,
                   rows_per_band=rows_per_band)
    desc = Desc(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax,
                tau0=tau0, dtau=dtau, sigma=sigma, omega_c=omega_c, tsplits=tuple(tsplit),
                n_qsplit=nq)
    return plan, desc


def _default_pair(hr, geo, **kw):
    """A plan with the library's default method parameters and the FP64
    oracle descriptor of the same lattices (from the plan's resolved
    descriptor)."""
    plan = hr.Plan(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax, **kw)
    d = plan.desc
    desc = Desc(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax, tau0=d.tau0, dtau=d.dtau,
                sigma=d.sigma, omega_c=d.omega_c, tsplits=tuple(d.tsplit[i] for i in range(d.n_tsplit)),
                n_qsplit=d.n_qsplit)
    return plan, desc


def _cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


CASES = {
    # name: (geometry, method kwargs)
    "small_gather_256x64": (synth.Geometry(256, 64, 256, 64, 0.004, 1.6 / 63, 0.2, 0.7), {}),
    "square_256": (synth.Geometry(256, 256, 256, 256, 2.0 / 255, 2.0 / 255, 0.2, 0.7), {}),
    "ragged_333x150": (synth.Geometry(333, 150, 301, 77, 0.006, 0.013, 0.15, 0.65),
                       dict(tsplit=(0.3, 0.6), nq=2)),
    "qmin0_no_split": (synth.Geometry(200, 90, 180, 50, 0.005, 0.02, 0.0, 0.6), dict(tsplit=())),
    "sigma2_wc025": (synth.Geometry(300, 120, 300, 120, 0.006, 0.015, 0.2, 0.7),
                     dict(sigma=2.0, omega_c=0.25, tsplit=(0.3, 0.6))),
    "tau0_offset": (synth.Geometry(256, 96, 200, 64, 0.004, 0.02, 0.2, 0.7),
                    dict(tau0=0.2, dtau=0.004)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_geometry_matches_oracle(hr, name):
    geo, kw = CASES[name]
    plan, desc = _pair(hr, geo, **kw)
    lp = LogPolar(desc)
    gpu = {(p["jt_lo"], p["l_lo"]): p for p in plan.pieces()}
    assert len(gpu) == len(lp.parts)
    for part in lp.parts:
        p = gpu[(part.jt_lo, part.l_lo)]
        for k in ("jt_hi", "l_hi", "Ntheta", "Nrho", "k1max", "k2max"):
            assert p[k] == getattr(part, k), k
        assert p["Ptheta"] == part.P_theta and p["Prho"] == part.P_rho
        for k in ("alpha", "beta", "a", "O1", "O2", "a_r", "r_max", "dtheta", "drho", "theta_m"):
            assert abs(p[k] - getattr(part, k)) <= 1e-12 * max(1.0, abs(getattr(part, k))), k


@pytest.mark.parametrize("name", list(CASES))
def test_forward_and_adjoint_match_logpolar_oracle(hr, name):
    geo, kw = CASES[name]
    plan, desc = _pair(hr, geo, **kw)
    lp = LogPolar(desc)
    f = synth.band_limited_gather(geo, 31, n_events=6, nu=10.0)
    g_ref = lp.forward(f)
    g = plan.forward(_cuda(f)).cpu().numpy()
    assert_parity(g, g_ref, what=name + " forward")
    gg = synth.random_radon_image(geo, 32)
    f_ref = lp.adjoint(gg)
    fa = plan.adjoint(_cuda(gg)).cpu().numpy()
    assert_parity(fa, f_ref, what=name + " adjoint")


def test_dot_test_fp32(hr):
    """Eq. (16) in FP32: the paper reports O(1e-5)."""
    geo = synth.Geometry(512, 256, 512, 256, 2.0 / 511, 2.0 / 255, 0.2, 0.7)
    plan, _ = _pair(hr, geo, tsplit=(0.3, 0.6), nq=2)
    rng = np.random.default_rng(9)
    f = _cuda(rng.standard_normal((geo.Nx, geo.Nt)))
    g = _cuda(rng.standard_normal((geo.Nq, geo.Ntau)))
    lhs = torch.sum(plan.forward(f).double() * g.double()).item()
    rhs = torch.sum(f.double() * plan.adjoint(g).double()).item()
    assert abs(lhs - rhs) / abs(lhs) < 1e-5


def test_matches_direct_sum_band_limited_512(hr, oracle_direct):
    """Default method parameters, band-limited 512^2 gather, every output."""
    geo, f = synth.sweep_gather(512, noise=0.0, nu_range=(8.0, 12.0))
    plan, _ = _default_pair(hr, geo)
    g_or = oracle_direct.fwd(f, geo.dt, geo.dx, geo.tau(), geo.q())
    g = plan.forward(_cuda(f)).cpu().numpy()
    assert _rel(g, g_or) < METHOD_TOL


def test_full_size_2048_sampled_against_direct_sum(hr, oracle_direct):
    """The benchmark workload (2048^2 gather, 32 Ricker events 20-40 Hz, 5 %
    noise, default method parameters): forward on 4096 sampled outputs and
    adjoint on 4096 sampled gather points against the FP64 direct sum."""
    geo, f = synth.sweep_gather(2048, noise=0.05)
    plan, _ = _default_pair(hr, geo)
    rng = np.random.default_rng(2048)
    ii = rng.integers(0, geo.Ntau, 4096)
    li = rng.integers(0, geo.Nq, 4096)
    g = plan.forward(_cuda(f)).cpu().numpy()
    ref = odirect.fwd_points(f, geo.dt, geo.dx, geo.tau(), geo.q(), ii, li)
    assert _rel(g[li, ii], ref) < METHOD_TOL
    # adjoint of a band-limited Radon image (Gaussian blobs in tau and q)
    gg = synth.smooth_radon_image(geo, 77)
    fa = plan.adjoint(_cuda(gg)).cpu().numpy()
    jj = rng.integers(0, geo.Nt, 4096)
    kk = rng.integers(0, geo.Nx, 4096)
    refa = odirect.adj_points(gg, geo.Nt, geo.Nx, geo.dt, geo.dx, 0.0, geo.dtau, geo.q(), jj, kk)
    assert _rel(fa[kk, jj], refa) < METHOD_TOL


def test_large_4096_sampled_against_direct_sum(hr, oracle_direct):
    """Large single gather (4096^2, 64 Ricker primaries plus their multiples,
    default method parameters; FFT lengths up to 6144): forward on 4096
    random outputs and adjoint on 4096 random gather points against the FP64
    direct sum, O(N) per point."""
    geo, f = synth.large_gather(4096)
    plan, _ = _default_pair(hr, geo)
    assert max(max(p["Ptheta"], p["Prho"]) for p in plan.pieces()) > 4096
    rng = np.random.default_rng(4096)
    ii = rng.integers(0, geo.Ntau, 4096)
    li = rng.integers(0, geo.Nq, 4096)
    g = plan.forward(_cuda(f)).cpu().numpy()
    ref = odirect.fwd_points(f, geo.dt, geo.dx, geo.tau(), geo.q(), ii, li)
    assert _rel(g[li, ii], ref) < METHOD_TOL
    gg = synth.smooth_radon_image(geo, 78)
    fa = plan.adjoint(_cuda(gg)).cpu().numpy()
    jj = rng.integers(0, geo.Nt, 4096)
    kk = rng.integers(0, geo.Nx, 4096)
    refa = odirect.adj_points(gg, geo.Nt, geo.Nx, geo.dt, geo.dx, 0.0, geo.dtau, geo.q(), jj, kk)
    assert _rel(fa[kk, jj], refa) < METHOD_TOL
    plan.close()


def test_full_size_2048_against_logpolar_oracle(hr):
    """The benchmark workload and plan (2048^2 gather, default method), every
    output, against the FP64 log-polar oracle on the same lattices: the
    forward of the benchmark gather, and the adjoint of a random Radon image
    and of a band-limited one (Gaussian blobs in tau and q). Default method
    parameters and rows per band tuned at plan creation, as the benchmark
    plans it."""
    geo, f = synth.sweep_gather(2048, noise=0.05)
    plan, desc = _default_pair(hr, geo, rows_per_band=0)
    lp = LogPolar(desc)
    assert_parity(plan.forward(_cuda(f)).cpu().numpy(), lp.forward(f), what="2048 forward")
    for name, gg in (("random", synth.random_radon_image(geo, 33)), ("blobs", synth.smooth_radon_image(geo, 77))):
        assert_parity(plan.adjoint(_cuda(gg)).cpu().numpy(), lp.adjoint(gg), what="2048 adjoint " + name)
    plan.close()


# Geometries whose lattices take each radix plan of the 9 * 2^a FFT lengths:
# (dimension, length): Nt = Ntau, Nx = Nq, dt, dx, qmin, qmax, method
RADIX9 = {
    ("rho", 144): (128, 128, 0.004, 1.6 / 127, 0.2, 0.7, {}),                       # half length 72 = 8 x 9
    ("rho", 288): (192, 128, 0.004, 1.6 / 127, 0.2, 0.7, {}),                       # 144 = 16 x 9
    ("rho", 576): (320, 256, 0.004, 1.6 / 255, 0.2, 0.7, {}),                       # 288 = 16 x 2 x 9
    ("rho", 1152): (768, 384, 0.002, 2.0 / 383, 0.2, 0.7, {}),                      # 576 = 16 x 4 x 9
    ("theta", 144): (128, 32, 0.004, 1.6 / 31, 0.2, 0.7, dict(nq=2)),               # 16 x 9
    ("theta", 288): (128, 128, 0.004, 1.6 / 127, 0.2, 0.7, dict(nq=2)),             # 16 x 2 x 9
    ("theta", 576): (128, 160, 0.004, 1.6 / 159, 0.2, 0.7, dict(nq=2)),             # 16 x 4 x 9
    ("theta", 1152): (768, 768, 0.002, 2.0 / 767, 0.1, 0.9, dict(sigma=2.0, omega_c=0.25)),   # 16 x 8 x 9
    ("theta", 2304): (1024, 1024, 0.002, 2.0 / 1023, 0.1, 0.7, dict(sigma=2.0, omega_c=0.25)),  # 16 x 16 x 9
}


@pytest.mark.parametrize("key", list(RADIX9))
def test_radix9_fft_lengths_match_oracle(hr, key):
    """Every radix plan of the 9 * 2^a lengths (column FFT of that length, or
    row FFT with that half length) against the FP64 oracle, forward and
    adjoint; the row length 2304 (half 1152 = 16 x 8 x 9) is the 2048x2048
    workload's."""
    dim, length = key
    Nt, Nx, dt, dx, qmin, qmax, kw = RADIX9[key]
    geo = synth.Geometry(Nt, Nx, Nt, Nx, dt, dx, qmin, qmax)
    plan, desc = _pair(hr, geo, **kw)
    assert length in [p["Ptheta" if dim == "theta" else "Prho"] for p in plan.pieces()]
    lp = LogPolar(desc)
    f = synth.band_limited_gather(geo, 95, n_events=6, nu=10.0)
    g = synth.random_radon_image(geo, 96)
    assert_parity(plan.forward(_cuda(f)).cpu().numpy(), lp.forward(f), what=f"{key} forward")
    assert_parity(plan.adjoint(_cuda(g)).cpu().numpy(), lp.adjoint(g), what=f"{key} adjoint")
    plan.close()


def test_direct_sum_kernel_matches_oracle(hr, oracle_direct):
    geo, f = synth.single_gather(1)
    g = hr.direct_forward(_cuda(f), geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax).cpu().numpy()
    g_or = oracle_direct.fwd(f, geo.dt, geo.dx, geo.tau(), geo.q())
    assert _rel(g, g_or) < 1e-4
    gg = synth.random_radon_image(geo, 4)
    fa = hr.direct_adjoint(_cuda(gg), geo.Nt, geo.Nx, geo.dt, geo.dx, geo.qmin, geo.qmax).cpu().numpy()
    f_or = oracle_direct.adj(gg, geo.Nt, geo.Nx, geo.dt, geo.dx, 0.0, geo.dtau, geo.q())
    assert _rel(fa, f_or) < 1e-4


def test_autograd_backward_is_adjoint_and_fd(hr):
    geo = synth.Geometry(128, 64, 128, 48, 0.008, 0.03, 0.2, 0.7)
    plan, _ = _pair(hr, geo)
    f = _cuda(synth.band_limited_gather(geo, 5)).requires_grad_(True)
    w = _cuda(synth.random_radon_image(geo, 6))
    loss = torch.sum(hr.radon(f, plan) * w)
    loss.backward()
    np.testing.assert_allclose(f.grad.cpu().numpy(), plan.adjoint(w).cpu().numpy(), rtol=0, atol=1e-6)
    # finite difference along a random direction (the operator is linear, so
    # the FD quotient is exact up to FP32 rounding)
    v = _cuda(np.random.default_rng(1).standard_normal((geo.Nx, geo.Nt)))
    eps = 1e-2
    with torch.no_grad():
        lp = torch.sum(plan.forward(f + eps * v).double() * w.double())
        lm = torch.sum(plan.forward(f - eps * v).double() * w.double())
    fd = ((lp - lm) / (2 * eps)).item()
    an = torch.sum(f.grad.double() * v.double()).item()
    assert abs(fd - an) / abs(an) < 1e-3


def test_errors_are_reported_not_fatal(hr):
    geo = synth.Geometry(64, 32, 64, 16, 0.01, 0.05, 0.2, 0.7)
    plan, _ = _pair(hr, geo)
    with pytest.raises(ValueError):
        plan.forward(torch.zeros((geo.Nx, geo.Nt + 1), device="cuda"))
    from paper_1604_07651_gb300 import _lib
    L = _lib.load()
    assert L.radon_fwd(plan._handle, None, None, None) == 1
    with pytest.raises(hr.RadonError):
        hr.Plan(64, 32, 64, 16, 0.01, 0.05, 0.5, 0.2)
    # the context is still usable afterwards
    out = plan.forward(torch.zeros((geo.Nx, geo.Nt), device="cuda"))
    assert float(out.abs().max()) == 0.0


def test_edge_cases(hr, oracle_direct):
    """Smallest gathers, a single slowness column, zero input."""
    geo = synth.Geometry(8, 4, 8, 3, 0.1, 0.1, 0.2, 0.7)
    plan, desc = _pair(hr, geo, tsplit=())
    f = np.random.default_rng(3).standard_normal((geo.Nx, geo.Nt))
    g_ref = LogPolar(desc).forward(f)
    assert_parity(plan.forward(_cuda(f)).cpu().numpy(), g_ref, what="8x4 forward")
    geo1 = synth.Geometry(64, 32, 64, 1, 0.01, 0.03, 0.4, 0.4)
    plan1, desc1 = _pair(hr, geo1, tsplit=())
    f1 = synth.band_limited_gather(geo1, 8)
    assert_parity(plan1.forward(_cuda(f1)).cpu().numpy(), LogPolar(desc1).forward(f1), what="one column forward")
    z = plan1.forward(torch.zeros((geo1.Nx, geo1.Nt), device="cuda"))
    assert float(z.abs().max()) == 0.0


def test_fixed_point_scale_range(hr):
    """The gridding and the adjoint column profiles accumulate in fixed point scaled
    by the input's own maximum: the transforms stay linear (to FP32 rounding)
    across the whole float range, and a spike well above the rest of the
    data does not wipe out the small values beside it."""
    geo = synth.Geometry(256, 96, 200, 64, 0.004, 0.02, 0.2, 0.7)
    plan, desc = _pair(hr, geo)
    ref = LogPolar(desc)
    f = synth.band_limited_gather(geo, 51, n_events=5, nu=10.0)
    g = synth.random_radon_image(geo, 52)
    fwd1 = plan.forward(_cuda(f)).cpu().numpy().astype(np.float64)
    adj1 = plan.adjoint(_cuda(g)).cpu().numpy().astype(np.float64)
    for c in (2.0 ** -80, 1e-20, 3e15, 2.0 ** 90):
        assert _rel(plan.forward(_cuda(f * c)).cpu().numpy() / c, fwd1) < 1e-6, c
        assert _rel(plan.adjoint(_cuda(g * c)).cpu().numpy() / c, adj1) < 1e-6, c
    # a spike 1e3 times the data (FP32 FFT round-off of the spike alone is
    # ~1e-5 of the rest): the transform of the rest keeps that accuracy
    spike = np.zeros_like(f)
    spike[40, 100] = 1e3 * np.abs(f).max()
    fs = plan.forward(_cuda(f + spike)).cpu().numpy() - plan.forward(_cuda(spike)).cpu().numpy()
    assert _rel(fs, ref.forward(f)) < 1e-4
    gsp = np.zeros_like(g)
    gsp[10, 50] = 1e3 * np.abs(g).max()
    ad = plan.adjoint(_cuda(g + gsp)).cpu().numpy() - plan.adjoint(_cuda(gsp)).cpu().numpy()
    assert _rel(ad, ref.adjoint(g)) < 1e-4


def test_non_finite_input_gives_non_finite_output(hr):
    """A NaN or infinite sample poisons its pieces (as the FFTs would) instead
    of being dropped or faulting; the next call on clean data is exact."""
    geo = synth.Geometry(128, 64, 128, 32, 0.004, 0.02, 0.2, 0.7)
    plan, desc = _pair(hr, geo)
    f = synth.band_limited_gather(geo, 61, n_events=4, nu=10.0)
    for bad in (np.nan, np.inf):
        fb = f.copy()
        fb[30, 70] = bad
        assert not np.isfinite(plan.forward(_cuda(fb)).cpu().numpy()).all()
        g = synth.random_radon_image(geo, 62)
        g[5, 60] = bad
        assert not np.isfinite(plan.adjoint(_cuda(g)).cpu().numpy()).all()
    assert_parity(plan.forward(_cuda(f)).cpu().numpy(), LogPolar(desc).forward(f), what="clean after non-finite")


def test_rows_per_band_choices_and_tuner(hr):
    """Every rows-per-band value, and the plan-time tuner (0), give the same
    transforms: the value only splits the row-FFT work among CTAs."""
    geo = synth.Geometry(300, 120, 280, 100, 0.005, 0.015, 0.2, 0.7)
    f = synth.band_limited_gather(geo, 71, n_events=5, nu=10.0)
    g_in = synth.random_radon_image(geo, 72)
    outs = {}
    for R in (0, 1, 2, 3, 4, 5, 6):
        plan = hr.Plan(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax, rows_per_band=R)
        assert 1 <= plan.desc.rows_per_band <= 6
        if R:
            assert plan.desc.rows_per_band == R
        outs[R] = (plan.forward(_cuda(f)).cpu().numpy(), plan.adjoint(_cuda(g_in)).cpu().numpy())
        plan.close()
    for R in (0, 1, 2, 4, 5, 6):
        assert _rel(outs[R][0], outs[3][0].astype(np.float64)) < 1e-6
        assert _rel(outs[R][1], outs[3][1].astype(np.float64)) < 1e-6


def test_forward_and_adjoint_are_bitwise_reproducible(hr):
    """No floating-point atomics anywhere: repeated transforms of the same
    input give the same bits. The 2048^2 benchmark plan has gridding tiles
    cut into several work units (the dense small-t samples), whose partial
    tiles are summed in a fixed order; other launches run in between so that
    the units are scheduled differently."""
    geo, f = synth.sweep_gather(2048, noise=0.05)
    plan, _ = _default_pair(hr, geo, rows_per_band=0)
    ft = _cuda(f)
    gg = _cuda(synth.smooth_radon_image(geo, 77))
    g0, a0 = plan.forward(ft), plan.adjoint(gg)
    noise = torch.empty(1 << 24, device="cuda")
    for i in range(3):
        noise.normal_()                       # unrelated work between the calls
        assert torch.equal(plan.forward(ft), g0), i
        assert torch.equal(plan.adjoint(gg), a0), i
    plan.close()
    geos = synth.batch_geometries(8)
    b = hr.Batch([dict(Nt=g.Nt, Nx=g.Nx, Ntau=g.Ntau, Nq=g.Nq, dt=g.dt, dx=g.dx, qmin=g.qmin, qmax=g.qmax)
                  for g in geos])
    fb = b.pack([torch.tensor(synth.batch_gather(g, i), dtype=torch.float32) for i, g in enumerate(geos)])
    r0 = b.forward(fb).clone()
    for _ in range(3):
        noise.normal_()
        assert torch.equal(b.forward(fb), r0)
    b.close()
