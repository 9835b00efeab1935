"""The quintic B-spline option (Section 7's higher-order kernel; six taps per
axis, three guard cells) on the GPU, through the C ABI, against the FP64
log-polar oracle with order=5 on the same lattices: forward and adjoint
element by element (tests/parity.py bounds) on small, ragged, multi-piece and
full 2048^2 workloads and on given offsets and slownesses, the closed-form
line integral of a Gaussian blob more accurately than the cubic path, the
FP32 inner-product test, batches of quintic gathers (FP32 and BF16 input),
and the refusal of a batch that mixes orders."""
import numpy as np
import pytest
import torch

from oracle import closed_forms as cf
import synth
from oracle.logpolar import Desc, LogPolar
from parity import assert_parity

pytestmark = pytest.mark.gpu

UNSUPPORTED = 4


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


def _pair(hr, geo, order=5, **kw):
    """A plan of the given B-spline order and the oracle descriptor of the
    same lattices (method parameters from the plan's resolved descriptor)."""
    plan = hr.Plan(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax,
                   spline_order=order, **kw)
    d = plan.desc
    assert d.spline_order == order
    desc = Desc(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax, tau0=d.tau0, dtau=d.dtau,
                sigma=d.sigma, omega_c=d.omega_c, tsplits=tuple(d.tsplit[i] for i in range(d.n_tsplit)),
                n_qsplit=d.n_qsplit, order=order)
    return plan, desc


CASES = {
    "small_gather_256x64": (synth.Geometry(256, 64, 256, 64, 0.004, 1.6 / 63, 0.2, 0.7), {}),
    "ragged_333x150_two_q_pieces": (synth.Geometry(333, 150, 301, 77, 0.006, 0.013, 0.15, 0.65),
                                    dict(tsplit=(0.3, 0.6), n_qsplit=2)),
    "qmin0_no_split": (synth.Geometry(200, 90, 180, 50, 0.005, 0.02, 0.0, 0.6), dict(tsplit=())),
    "sigma2_wc025": (synth.Geometry(300, 120, 300, 120, 0.006, 0.015, 0.2, 0.7),
                     dict(sigma=2.0, omega_c=0.25, tsplit=(0.3, 0.6))),
    "tau0_offset": (synth.Geometry(256, 96, 200, 64, 0.004, 0.02, 0.2, 0.7), dict(tau0=0.2, dtau=0.004)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_quintic_forward_and_adjoint_match_oracle(hr, name):
    geo, kw = CASES[name]
    plan, desc = _pair(hr, geo, **kw)
    lp = LogPolar(desc)
    gpu = {(p["jt_lo"], p["l_lo"]): p for p in plan.pieces()}
    for part in lp.parts:       # three guard cells: the oracle's lattices
        p = gpu[(part.jt_lo, part.l_lo)]
        assert (p["Ntheta"], p["Nrho"], p["Ptheta"], p["Prho"]) == (part.Ntheta, part.Nrho, part.P_theta,
                                                                     part.P_rho)
        assert part.Ntheta == part.n_theta + 7
    f = synth.band_limited_gather(geo, 41, n_events=6, nu=10.0)
    assert_parity(plan.forward(_cuda(f)).cpu().numpy(), lp.forward(f), what=name + " quintic forward")
    gg = synth.random_radon_image(geo, 42)
    assert_parity(plan.adjoint(_cuda(gg)).cpu().numpy(), lp.adjoint(gg), what=name + " quintic adjoint")
    plan.close()


def test_quintic_full_size_2048_against_oracle(hr):
    """The 2048^2 benchmark gather with quintic B-splines and the default
    method parameters, every output, forward and adjoint."""
    geo, f = synth.sweep_gather(2048, noise=0.05)
    plan, desc = _pair(hr, geo)
    lp = LogPolar(desc)
    assert_parity(plan.forward(_cuda(f)).cpu().numpy(), lp.forward(f), what="2048 quintic forward")
    gg = synth.smooth_radon_image(geo, 77)
    assert_parity(plan.adjoint(_cuda(gg)).cpu().numpy(), lp.adjoint(gg), what="2048 quintic adjoint")
    plan.close()


def test_quintic_blob_line_integral_beats_cubic(hr):
    """Gaussian blob in (s, y) whose line integrals have a closed form: on
    the same lattices (sigma 2, omega_c 0.25) the quintic path comes closer
    to the exact Radon transform than the cubic one."""
    N = 256
    geo = synth.Geometry(N, N, N, N, 2.0 / (N - 1), 2.0 / (N - 1), 0.2, 0.7)
    c1, c2, w = 0.45, 0.35, 0.06
    f = cf.blob_sy_gather(geo.t(), geo.x(), geo.T, geo.X, c1, c2, w)
    g_ex = cf.blob_sy_radon(geo.tau(), geo.q(), geo.T, geo.X, c1, c2, w)
    errs = {}
    for order in (3, 5):
        plan, _ = _pair(hr, geo, order=order, sigma=2.0, omega_c=0.25, tsplit=(0.3, 0.6))
        errs[order] = _rel(plan.forward(_cuda(f)).cpu().numpy(), g_ex)
        plan.close()
    assert errs[5] < 2e-5 and errs[5] < 0.5 * errs[3], errs


def test_quintic_dot_test_fp32(hr):
    geo = synth.Geometry(512, 256, 512, 256, 2.0 / 511, 2.0 / 255, 0.2, 0.7)
    plan, _ = _pair(hr, geo, tsplit=(0.3, 0.6), n_qsplit=2)
    rng = np.random.default_rng(19)
    f = _cuda(rng.standard_normal((geo.Nx, geo.Nt)))
    g = _cuda(rng.standard_normal((geo.Nq, geo.Ntau)))
    lhs = torch.sum(plan.forward(f).double() * g.double()).item()
    rhs = torch.sum(f.double() * plan.adjoint(g).double()).item()
    assert abs(lhs - rhs) / abs(lhs) < 1e-5
    plan.close()


def _geo_dict(geo, **kw):
    return dict(Nt=geo.Nt, Nx=geo.Nx, Ntau=geo.Ntau, Nq=geo.Nq, dt=geo.dt, dx=geo.dx, qmin=geo.qmin,
                qmax=geo.qmax, **kw)


def test_quintic_batch_against_oracle_and_mixed_orders_refused(hr):
    geos = [synth.Geometry(300, 64, 280, 48, 0.004, 0.025, 0.2, 0.7),
            synth.Geometry(520, 90, 520, 90, 0.004, 0.025, 0.2, 0.7),
            synth.Geometry(180, 120, 200, 60, 0.004, 0.025, 0.15, 0.65)]
    gathers = [synth.batch_gather(g, 300 + i) for i, g in enumerate(geos)]
    batch = hr.Batch([_geo_dict(g, spline_order=5) for g in geos])
    imgs = batch.unpack_images(batch.forward(batch.pack([torch.tensor(x, dtype=torch.float32) for x in gathers])))
    gimg = [synth.random_radon_image(g, 400 + i) for i, g in enumerate(geos)]
    fa = batch.unpack_gathers(batch.adjoint(torch.cat([torch.tensor(x, dtype=torch.float32).reshape(-1)
                                                       for x in gimg]).cuda()))
    for i, (geo, x, a, gi, fi) in enumerate(zip(geos, gathers, imgs, gimg, fa)):
        d = batch.plan_desc(i)
        assert d.spline_order == 5
        lp = LogPolar(Desc(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax,
                           sigma=d.sigma, omega_c=d.omega_c, tsplits=tuple(d.tsplit[k] for k in range(d.n_tsplit)),
                           n_qsplit=d.n_qsplit, order=5))
        assert_parity(a.cpu().numpy(), lp.forward(x), what="quintic batch forward")
        assert_parity(fi.cpu().numpy(), lp.adjoint(gi), what="quintic batch adjoint")
    batch.close()
    with pytest.raises(hr.RadonError) as ei:
        hr.Batch([_geo_dict(geos[0], spline_order=5), _geo_dict(geos[1])])
    assert ei.value.status == UNSUPPORTED and "order" in str(ei.value)


def test_quintic_on_given_grids_matches_oracle(hr):
    """Jittered offsets with a near-offset gap and slownesses denser towards
    qmin (radon_plan_create_grid), two slowness pieces, quintic B-splines."""
    geo = synth.irregular_geometry(256, 96, 256, 64, 0.004, 1.6, 0.2, 0.7, 11, jitter=0.4, near=0.1, q_power=1.5)
    plan = hr.Plan(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax, n_qsplit=2,
                   x=geo.offsets, q=geo.slownesses, spline_order=5)
    d = plan.desc
    lp = LogPolar(Desc(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax, sigma=d.sigma,
                       omega_c=d.omega_c, tsplits=tuple(d.tsplit[i] for i in range(d.n_tsplit)), n_qsplit=2,
                       x=geo.offsets, q_values=geo.slownesses, order=5))
    f = synth.band_limited_gather(geo, 61, n_events=6, nu=10.0)
    assert_parity(plan.forward(_cuda(f)).cpu().numpy(), lp.forward(f), what="quintic given grids forward")
    gg = synth.random_radon_image(geo, 62)
    assert_parity(plan.adjoint(_cuda(gg)).cpu().numpy(), lp.adjoint(gg), what="quintic given grids adjoint")
    plan.close()


def test_quintic_bf16_batch_against_oracle_on_rounded_input(hr):
    geos = [synth.Geometry(300, 64, 280, 48, 0.004, 0.025, 0.2, 0.7),
            synth.Geometry(180, 120, 200, 60, 0.004, 0.025, 0.15, 0.65)]
    gathers = [synth.batch_gather(g, 500 + i) for i, g in enumerate(geos)]
    batch = hr.Batch([_geo_dict(g, spline_order=5) for g in geos])
    fb = batch.pack([torch.tensor(x, dtype=torch.float32) for x in gathers], dtype=torch.bfloat16)
    imgs = batch.unpack_images(batch.forward(fb))
    for i, (geo, x, a) in enumerate(zip(geos, gathers, imgs)):
        d = batch.plan_desc(i)
        lp = LogPolar(Desc(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax,
                           sigma=d.sigma, omega_c=d.omega_c, tsplits=tuple(d.tsplit[k] for k in range(d.n_tsplit)),
                           n_qsplit=d.n_qsplit, order=5))
        xb = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
        assert_parity(a.cpu().numpy(), lp.forward(xb), what="quintic BF16 batch forward")
    batch.close()


def test_quintic_bitwise_reproducible(hr):
    """Split gridding tiles merge in a fixed order with six taps as well."""
    geo, f = synth.sweep_gather(1024, noise=0.05)
    plan, _ = _pair(hr, geo)
    x = _cuda(f)
    g0 = plan.forward(x)
    gg = _cuda(synth.random_radon_image(geo, 5))
    a0 = plan.adjoint(gg)
    for _ in range(3):
        assert torch.equal(plan.forward(x), g0)
        assert torch.equal(plan.adjoint(gg), a0)
    plan.close()
