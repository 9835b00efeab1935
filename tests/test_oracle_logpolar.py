"""Pins of the FP64 log-polar oracle (Sections 2-4).

The log-polar method is an approximation, so the oracle is checked against
what the mathematics fixes independently of it: the geometry conditions the
paper states (corners on the sector, Section 2.1), the exact line distance
behind P2 S (Eq. (9)-(10)), closed forms of zeta_hat, a closed-form line
integral of a Gaussian in (s, y) (Eq. (3)-(4)), the exact transpose
(Eq. (16)), and agreement with the direct sum on band-limited data
(Section 5). Planted mistakes in the oracle must break at least one pin.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

import synth
import oracle.logpolar as LP
from oracle import closed_forms as cf
from oracle.logpolar import Desc, LogPolar


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("alpha,beta", [(0.25, 0.42), (0.6, 0.9), (0.1, 0.05), (0.8, 1.4), (0.785, 0.3), (0.0005, 0.001)])
def test_square_in_sector_corners(alpha, beta):
    """Corners (0,0), (1,1) on the edges at -beta/2, +beta/2; corner (1,0)
    on the unit arc; the whole square inside the sector (Section 2.1)."""
    a, O1, O2 = LP.square_in_sector(alpha, beta)
    part = type("P", (), dict(alpha=alpha, a=a, O1=O1, O2=O2))
    u1, u2 = LP.map_T(part, np.array([0.0, 1.0, 1.0, 0.0]), np.array([0.0, 0.0, 1.0, 1.0]))
    ang = np.arctan2(u2, u1)
    r = np.hypot(u1, u2)
    assert abs(ang[0] + beta / 2) < 1e-13
    assert abs(ang[2] - beta / 2) < 1e-13
    assert abs(r[1] - 1.0) < 1e-13
    assert np.all(np.abs(ang) <= beta / 2 + 1e-13)
    assert np.all(r <= 1.0 + 1e-13)
    # the square of side a: edges of length a
    assert abs(math.hypot(u1[1] - u1[0], u2[1] - u2[0]) - a) < 1e-14


def test_line_distance_is_p2_s():
    """e^rho of ``radon_points`` equals the distance from the origin of the
    image under T of the line s = tau^2 + q^2 y, computed from two points."""
    d = Desc(64, 32, 50, 20, 0.01, 0.03, 0.2, 0.7)
    part = LP.plan(d)[0]
    ll, ii, xth, xrh, valid, scale = LP.radon_points(d, part)
    taub = d.tau()[ii] / d.T
    qb = d.q()[ll] * d.X / d.T
    p1 = LP.map_T(part, taub ** 2, np.zeros_like(taub))
    p2 = LP.map_T(part, taub ** 2 + qb ** 2, np.ones_like(taub))
    dx_, dy_ = p2[0] - p1[0], p2[1] - p1[1]
    dist = np.abs(p1[0] * dy_ - p1[1] * dx_) / np.hypot(dx_, dy_)
    e = np.exp(xrh * part.drho + part.rho0)
    np.testing.assert_allclose(e[valid], dist[valid], rtol=1e-13)
    # theta is the normal angle: n_theta . p = e^rho at both points of the line
    th = xth * part.dtheta + part.theta0
    for p in (p1, p2):
        np.testing.assert_allclose((np.cos(th) * p[0] + np.sin(th) * p[1])[valid], e[valid], rtol=1e-12)


def test_inner_radius_is_minimum_distance():
    """a_r is the smallest n_theta . u over the data region and |theta| <= beta/2."""
    d = Desc(128, 64, 64, 32, 0.008, 0.025, 0.2, 0.7, tsplits=(0.4,))
    for part in LP.plan(d):
        s = np.linspace(part.s0, part.s1, 200)
        y = np.linspace(0.0, 1.0, 200)
        S, Y = np.meshgrid(s, y)
        keep = S >= part.c_min + part.k2 * Y
        u1, u2 = LP.map_T(part, S[keep], Y[keep])
        dmin = min(float(np.min(u1 * math.cos(t) + u2 * math.sin(t)))
                   for t in np.linspace(-part.beta / 2, part.beta / 2, 41))
        assert part.a_r <= dmin + 1e-12
        assert dmin - part.a_r < 2e-3
        assert part.r_max >= float(np.max(np.hypot(u1, u2))) - 1e-12


def test_lattice_spacing_follows_eq18():
    """The lattice spacing is the Eq. (18) spacing divided by sigma, or finer."""
    for sigma in (1.0, 2.0):
        d = Desc(200, 80, 100, 40, 0.004, 0.02, 0.2, 0.7, sigma=sigma, tsplits=(0.5,))
        for part in LP.plan(d):
            assert part.dtheta <= part.dphi_rule / sigma * (1 + 1e-12)
            assert part.drho <= part.deta_rule / sigma * (1 + 1e-12)
            assert part.dtheta > part.dphi_rule / sigma * 0.5
            assert part.P_theta >= part.Ntheta + math.ceil(part.theta_m / part.dtheta - 1e-9)
            assert part.P_rho >= part.Nrho + math.ceil(-math.log(math.cos(part.theta_m)) / part.drho - 1e-9)


def test_b3_partition_of_unity_and_transform():
    x = np.linspace(-3, 3, 1001)
    s = sum(LP.b3(x - k) for k in range(-5, 6))
    np.testing.assert_allclose(s, 1.0, atol=1e-14)
    for w in (0.0, 0.13, 0.37, 0.5):
        val = quad(lambda t: LP.b3(np.array(t)) * math.cos(2 * math.pi * w * t), -2, 2,
                   points=[-1, 0, 1], epsabs=1e-15)[0]
        assert abs(val - LP.b3_hat(w)) < 1e-13


def test_zeta_hat_closed_form_symmetry_and_quadrature():
    tm = 0.52
    dc = LP.zeta_hat(tm, [0.0], [0.0])[0, 0]
    assert abs(dc - cf.zeta_hat_dc(tm)) < 1e-14
    w1 = np.array([-7.3, 7.3, 60.1])
    w2 = np.array([-120.0, 120.0])
    z = LP.zeta_hat(tm, w1, w2)
    np.testing.assert_allclose(z[0], z[1], atol=1e-14)           # even in w1
    np.testing.assert_allclose(z[:, 0], np.conj(z[:, 1]), atol=1e-14)  # real zeta
    for a, b in [(60.1, 120.0), (7.3, -120.0)]:
        re = quad(lambda t: math.cos(2 * math.pi * (t * a + b * math.log(math.cos(t)))) / math.cos(t),
                  -tm, tm, limit=4000, epsabs=1e-15, epsrel=1e-13)[0]
        im = quad(lambda t: -math.sin(2 * math.pi * (t * a + b * math.log(math.cos(t)))) / math.cos(t),
                  -tm, tm, limit=4000, epsabs=1e-15, epsrel=1e-13)[0]
        zz = LP.zeta_hat(tm, [a], [b])[0, 0]
        assert abs(zz - (re + 1j * im)) < 1e-12


BLOBS = [(0.5, 0.4, 0.1), (0.3, 0.5, 0.08), (0.7, 0.6, 0.09)]


@pytest.mark.parametrize("tsplits,nq", [((), 1), ((0.5,), 1), ((0.3, 0.6), 2)])
def test_blob_line_integral_closed_form(tsplits, nq):
    """C4: a Gaussian blob in (s, y) has a closed-form line integral; this
    pins the log-polar steps, their constants and the output scale
    2 X cos(psi) / a, bypassing the interpolation error in t."""
    N = 256
    geo = synth.Geometry(N, N, N, N, 2.0 / (N - 1), 2.0 / (N - 1), 0.2, 0.7)
    d = Desc(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax,
             sigma=2.0, omega_c=0.25, tsplits=tsplits, n_qsplit=nq)
    lp = LogPolar(d)
    for c1, c2, w in BLOBS:
        f = cf.blob_sy_gather(geo.t(), geo.x(), geo.T, geo.X, c1, c2, w)
        g = lp.forward(f)
        g_ex = cf.blob_sy_radon(geo.tau(), geo.q(), geo.T, geo.X, c1, c2, w)
        assert _rel(g, g_ex) < 5e-5, (c1, c2, w)


@pytest.mark.parametrize("tsplits,nq", [((), 1), ((0.3, 0.6), 2)])
def test_adjoint_is_exact_transpose(tsplits, nq):
    """Eq. (16) to FP64 rounding, for several pieces."""
    geo, f = synth.single_gather(1)
    d = Desc(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax,
             tsplits=tsplits, n_qsplit=nq)
    lp = LogPolar(d)
    g = synth.random_radon_image(geo, 3)
    lhs = float(np.sum(lp.forward(f) * g))
    rhs = float(np.sum(f * lp.adjoint(g)))
    assert abs(lhs - rhs) / abs(lhs) < 1e-12


def test_agrees_with_direct_sum_band_limited(oracle_direct):
    """Section 5: log-polar vs direct summation over hyperbolas on band-limited
    events (512x512, 12 Hz Ricker) to 1e-2 relative L2."""
    N = 512
    geo = synth.Geometry(N, N, N, N, 2.0 / (N - 1), 2.0 / (N - 1), 0.2, 0.7)
    f = synth.band_limited_gather(geo, 21, n_events=10, nu=12.0)
    g_or = oracle_direct.fwd(f, geo.dt, geo.dx, geo.tau(), geo.q())
    d = Desc(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax,
             sigma=2.0, omega_c=0.25, tsplits=(0.3, 0.6))
    g = LogPolar(d).forward(f)
    assert _rel(g, g_or) < 1e-2


# ---- planted mistakes: each must break a pin ------------------------------

def _blob_error(monkeypatch=None):
    N = 128
    geo = synth.Geometry(N, N, N, N, 2.0 / (N - 1), 2.0 / (N - 1), 0.2, 0.7)
    d = Desc(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax)
    c1, c2, w = BLOBS[0]
    f = cf.blob_sy_gather(geo.t(), geo.x(), geo.T, geo.X, c1, c2, w)
    g = LogPolar(d).forward(f)
    return _rel(g, cf.blob_sy_radon(geo.tau(), geo.q(), geo.T, geo.X, c1, c2, w))


def test_unplanted_blob_error_small():
    assert _blob_error() < 2e-5


def test_mutant_printed_O1_caught(monkeypatch):
    """The printed first component of O (with tan(beta)) fails the corner pin."""
    orig = LP.square_in_sector

    def mutant(alpha, beta):
        a, O1, O2 = orig(alpha, beta)
        return a, a * math.sin(alpha + math.pi / 4) * math.tan(beta) / math.sqrt(2.0), O2

    monkeypatch.setattr(LP, "square_in_sector", mutant)
    with pytest.raises(AssertionError):
        test_square_in_sector_corners(0.25, 0.42)


def test_mutant_output_scale_caught(monkeypatch):
    """Dropping cos(psi) from the output scale breaks the blob closed form."""
    orig = LP.radon_points

    def mutant(desc, part):
        ll, ii, xth, xrh, valid, scale = orig(desc, part)
        qb = desc.q()[ll] * desc.X / desc.T
        return ll, ii, xth, xrh, valid, scale / np.cos(np.arctan(qb * qb))

    monkeypatch.setattr(LP, "radon_points", mutant)
    assert _blob_error() > 1e-2


def test_mutant_single_deconvolution_caught(monkeypatch):
    """Dividing by the B-spline symbol once instead of twice breaks C4."""
    orig = LP.bspline_hat
    monkeypatch.setattr(LP, "bspline_hat", lambda order, w: np.sqrt(orig(order, w)))
    assert _blob_error() > 1e-3


def test_mutant_angle_sign_caught(monkeypatch):
    """The printed sign of P2's angle (theta = -alpha + psi) breaks C4."""
    orig = LP.radon_points

    def mutant(desc, part):
        ll, ii, xth, xrh, valid, scale = orig(desc, part)
        th = xth * part.dtheta + part.theta0
        th2 = np.clip(-th, -part.beta / 2, part.beta / 2)
        return ll, ii, (th2 - part.theta0) / part.dtheta, xrh, valid, scale

    monkeypatch.setattr(LP, "radon_points", mutant)
    assert _blob_error() > 1e-2


def test_lattice_spacing_rule_by_brute_force():
    """Eq. (18) by brute force, independent of the oracle's vectorised rule:
    every pair of neighbouring samples (t_j, x_k)-(t_j + dt, x_k) and
    (t_j, x_k)-(t_j, x_k + dx) of the time piece on an 8 x 16 gather, mapped
    one by one through (s, y) = (t^2, x^2) (rescaled), the rotation and
    scaling of the square in the sector, u = a R(alpha) (s - 1/2, y - 1/2) + O,
    and the log-polar angle and log-radius of u. The largest differences are
    the rule's spacings; on this geometry the t-neighbours decide the angle
    spacing and the x-neighbours the log-radius spacing (so dropping either
    direction, or swapping the axes, changes the rule and fails)."""
    for tsplits in ((), (0.5,)):
        d = Desc(8, 16, 8, 16, 0.05, 0.2, 0.2, 0.7, sigma=1.0, tsplits=tsplits)
        n_t, n_x = d.Nt - 1, d.Nx - 1
        for part in LP.plan(d):
            ca, sa = math.cos(part.alpha), math.sin(part.alpha)

            def lp(j, k):
                s = (j / n_t) ** 2 - 0.5
                y = (k / n_x) ** 2 - 0.5
                u1 = part.a * (ca * s - sa * y) + part.O1
                u2 = part.a * (sa * s + ca * y) + part.O2
                return math.atan2(u2, u1), 0.5 * math.log(u1 * u1 + u2 * u2)

            by_t = [0.0, 0.0]
            by_x = [0.0, 0.0]
            for j in range(part.jt_lo, part.jt_hi + 1):
                for k in range(d.Nx):
                    p0 = lp(j, k)
                    if j + 1 <= part.jt_hi:
                        p1 = lp(j + 1, k)
                        by_t = [max(by_t[0], abs(p1[0] - p0[0])), max(by_t[1], abs(p1[1] - p0[1]))]
                    if k + 1 < d.Nx:
                        p1 = lp(j, k + 1)
                        by_x = [max(by_x[0], abs(p1[0] - p0[0])), max(by_x[1], abs(p1[1] - p0[1]))]
            dphi, deta = max(by_t[0], by_x[0]), max(by_t[1], by_x[1])
            assert abs(part.dphi_rule - dphi) <= 1e-12 * dphi, (part.dphi_rule, dphi)
            assert abs(part.deta_rule - deta) <= 1e-12 * deta, (part.deta_rule, deta)
            if not tsplits:
                # both neighbour directions matter here: each decides one spacing
                assert by_t[0] > by_x[0] * 1.01 and by_x[1] > by_t[1] * 1.01, (by_t, by_x)


# ---- the quintic B-spline option (Section 7: higher-order kernels) --------

def test_b5_from_convolutions_partition_of_unity_and_transform():
    """B5 against two things that do not use its truncated-power formula:
    the convolution B3 * box * box evaluated numerically, and the transform
    sinc^6 by quadrature; plus the partition of unity."""
    h = 1e-3
    t = np.arange(-4.0, 4.0 + h / 2, h)
    box = np.where(np.abs(t) < 0.5 - h / 4, 1.0, np.where(np.abs(t) < 0.5 + h / 4, 0.5, 0.0))   # trapezoid edges
    conv = np.convolve(np.convolve(LP.b3(t), box, mode="same") * h, box, mode="same") * h
    np.testing.assert_allclose(conv, LP.b5(t), atol=2e-6)
    x = np.linspace(-4, 4, 1001)
    np.testing.assert_allclose(sum(LP.b5(x - k) for k in range(-8, 9)), 1.0, atol=1e-14)
    for w in (0.0, 0.11, 0.29, 0.5):
        val = quad(lambda u: LP.b5(np.array(u)) * math.cos(2 * math.pi * w * u), -3, 3,
                   points=[-2, -1, 0, 1, 2], epsabs=1e-15)[0]
        assert abs(val - LP.bspline_hat(5, w)) < 1e-13


@pytest.mark.parametrize("tsplits,nq", [((), 1), ((0.3, 0.6), 2)])
def test_quintic_blob_line_integral_and_transpose(tsplits, nq):
    """C4 with the quintic kernel: the Gaussian blob's closed-form line
    integral to 1e-5 (cubic: 5e-5), and the exact transpose to 1e-12."""
    N = 256
    geo = synth.Geometry(N, N, N, N, 2.0 / (N - 1), 2.0 / (N - 1), 0.2, 0.7)
    d = Desc(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax,
             sigma=2.0, omega_c=0.25, tsplits=tsplits, n_qsplit=nq, order=5)
    lp = LogPolar(d)
    assert all(p.Ntheta == p.n_theta + 7 and p.Nrho == p.n_rho + 7 for p in lp.parts)   # 3 guard cells
    for c1, c2, w in BLOBS:
        f = cf.blob_sy_gather(geo.t(), geo.x(), geo.T, geo.X, c1, c2, w)
        g_ex = cf.blob_sy_radon(geo.tau(), geo.q(), geo.T, geo.X, c1, c2, w)
        assert _rel(lp.forward(f), g_ex) < 1e-5, (c1, c2, w)
    rng = np.random.default_rng(55)
    f = rng.standard_normal((geo.Nx, geo.Nt))
    g = rng.standard_normal((geo.Nq, geo.Ntau))
    lhs, rhs = float(np.sum(lp.forward(f) * g)), float(np.sum(f * lp.adjoint(g)))
    assert abs(lhs - rhs) / abs(lhs) < 1e-12


def test_quintic_agrees_with_direct_sum_band_limited(oracle_direct):
    N = 512
    geo = synth.Geometry(N, N, N, N, 2.0 / (N - 1), 2.0 / (N - 1), 0.2, 0.7)
    f = synth.band_limited_gather(geo, 21, n_events=10, nu=12.0)
    g_or = oracle_direct.fwd(f, geo.dt, geo.dx, geo.tau(), geo.q())
    d = Desc(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax,
             sigma=2.0, omega_c=0.25, tsplits=(0.3, 0.6), order=5)
    assert _rel(LogPolar(d).forward(f), g_or) < 1e-2


def test_mutant_quintic_with_cubic_symbol_caught(monkeypatch):
    """Deconvolving the quintic gridding by the cubic symbol sinc^4 breaks C4."""
    monkeypatch.setattr(LP, "bspline_hat", lambda order, w: np.sinc(w) ** 4)
    N = 128
    geo = synth.Geometry(N, N, N, N, 2.0 / (N - 1), 2.0 / (N - 1), 0.2, 0.7)
    d = Desc(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax, order=5)
    c1, c2, w = BLOBS[0]
    f = cf.blob_sy_gather(geo.t(), geo.x(), geo.T, geo.X, c1, c2, w)
    g_ex = cf.blob_sy_radon(geo.tau(), geo.q(), geo.T, geo.X, c1, c2, w)
    assert _rel(LogPolar(d).forward(f), g_ex) > 1e-4
