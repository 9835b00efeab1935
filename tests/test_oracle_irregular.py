"""Pins of the oracles on unequally spaced offsets and slownesses (Section 4:
the log-polar method carries over to unequally spaced grids), no GPU.

* direct sum on given offsets: equal to the regular sum when the offsets are
  the regular grid; converges to the closed form of a Gaussian gather as the
  jittered offsets are refined (trapezoid rule, second order); its adjoint is
  the transpose;
* log-polar method on given offsets and slownesses: the Gaussian blob of
  Eq. (2) against its closed-form line integral, exact transpose, agreement
  with the direct sum on band-limited events; planted mistakes in the offset
  weights or positions break the blob pin.
"""
import numpy as np
import pytest

import synth
from oracle import closed_forms as cf
from oracle.logpolar import Desc, LogPolar


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _desc(geo, **kw):
    return Desc(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax,
                x=geo.offsets, q_values=geo.slownesses, **kw)


def test_direct_on_regular_offsets_is_the_regular_sum(oracle_direct):
    geo = synth.Geometry(60, 17, 50, 5, 0.01, 0.05, 0.1, 0.5)
    rng = np.random.default_rng(11)
    f = rng.standard_normal((geo.Nx, geo.Nt))
    g = rng.standard_normal((geo.Nq, geo.Ntau))
    x = np.arange(geo.Nx) * geo.dx
    np.testing.assert_allclose(oracle_direct.fwd_x(f, geo.dt, x, geo.tau(), geo.q()),
                               oracle_direct.fwd(f, geo.dt, geo.dx, geo.tau(), geo.q()), rtol=0, atol=1e-13)
    np.testing.assert_allclose(oracle_direct.adj_x(g, geo.Nt, geo.dt, x, 0.0, geo.dtau, geo.q()),
                               oracle_direct.adj(g, geo.Nt, geo.Nx, geo.dt, geo.dx, 0.0, geo.dtau, geo.q()),
                               rtol=0, atol=1e-13)


def test_direct_on_jittered_offsets_converges_to_closed_form(oracle_direct):
    """f = exp(-30 t^2 - 25 x^2), fine in t so that the x quadrature
    dominates: the error falls by more than 2.5 per halving of the offset
    spacing (second order on jittered nodes) and is below 3e-5 at 128
    traces; equal weights on the same jittered offsets stay first order."""
    tau = np.linspace(0.15, 0.6, 40)
    errs, errs_equal = [], []
    for Nx in (16, 32, 64, 128):
        geo = synth.irregular_geometry(800, Nx, 40, 7, 1.0 / 799, 1.0, 0.0, 0.9, 1)
        f = synth.gaussian_gather(geo, 30.0, 25.0)
        exact = cf.gaussian_tx(tau, geo.q(), 30.0, 25.0, geo.T, geo.X)
        errs.append(_rel(oracle_direct.fwd_x(f, geo.dt, geo.x(), tau, geo.q()), exact))
        errs_equal.append(_rel(oracle_direct.fwd(f, geo.dt, geo.dx, tau, geo.q()), exact))
    for a, b in zip(errs, errs[1:]):
        assert a / b > 2.5, errs
    assert errs[-1] < 3e-5
    assert errs_equal[-1] > 10 * errs[-1]


def test_direct_on_given_offsets_adjoint_is_transpose(oracle_direct):
    geo = synth.irregular_geometry(120, 33, 100, 17, 0.01, 1.2, 0.1, 0.6, 2, near=0.15, q_power=1.5)
    f = synth.band_limited_gather(geo, 41, n_events=4, nu=10.0)
    g = synth.random_radon_image(geo, 42)
    lhs = float(np.sum(oracle_direct.fwd_x(f, geo.dt, geo.x(), geo.tau(), geo.q()) * g))
    rhs = float(np.sum(f * oracle_direct.adj_x(g, geo.Nt, geo.dt, geo.x(), 0.0, geo.dtau, geo.q())))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


BLOBS = [(0.5, 0.4, 0.1), (0.3, 0.5, 0.08), (0.7, 0.6, 0.09)]
BLOB_TOL = 8e-4   # jittered-trapezoid error 1e-4 .. 2.5e-4 at 256 traces


def _blob_errors(geo, desc):
    lp = LogPolar(desc)
    out = []
    for c1, c2, w in BLOBS:
        f = cf.blob_sy_gather(geo.t(), geo.x(), geo.T, geo.X, c1, c2, w)
        out.append(_rel(lp.forward(f), cf.blob_sy_radon(geo.tau(), geo.q(), geo.T, geo.X, c1, c2, w)))
    return out


@pytest.fixture(scope="module")
def blob_geo():
    N = 256
    return synth.irregular_geometry(N, N, N, N, 2.0 / (N - 1), 2.0, 0.2, 0.7, 1, jitter=0.4, q_power=1.6)


def test_log_polar_blob_closed_form_on_given_grids(blob_geo):
    """C4 on jittered offsets and slownesses denser towards qmin."""
    errs = _blob_errors(blob_geo, _desc(blob_geo, sigma=2.0, omega_c=0.25))
    assert max(errs) < BLOB_TOL, errs


def test_log_polar_on_given_grids_adjoint_is_transpose():
    geo = synth.irregular_geometry(128, 48, 96, 40, 0.008, 1.5, 0.2, 0.7, 3, near=0.1, q_power=1.4)
    lp = LogPolar(_desc(geo, sigma=1.25, omega_c=0.35, tsplits=(0.25, 0.5), n_qsplit=2))
    f = synth.band_limited_gather(geo, 43, n_events=5, nu=10.0)
    g = synth.random_radon_image(geo, 44)
    lhs = float(np.sum(lp.forward(f) * g))
    rhs = float(np.sum(f * lp.adjoint(g)))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_log_polar_agrees_with_direct_sum_on_given_grids(oracle_direct):
    """Section 5's comparison on unequal grids (near-offset gap, 40 % jitter,
    uneven slownesses): at the regular-grid level (1.7e-3 forward, 2.0e-3
    adjoint), which the lattice spacing over the mean offset spacing keeps
    (the largest gap would give 2.6e-2)."""
    N = 384
    geo = synth.irregular_geometry(N, N, N, N, 2.0 / (N - 1), 2.0, 0.2, 0.7, 4, near=0.1, q_power=1.5)
    f = synth.band_limited_gather(geo, 45, n_events=10, nu=12.0)
    lp = LogPolar(_desc(geo, sigma=2.0, omega_c=0.25, tsplits=(0.3, 0.6)))
    g_or = oracle_direct.fwd_x(f, geo.dt, geo.x(), geo.tau(), geo.q())
    assert _rel(lp.forward(f), g_or) < 5e-3
    g = synth.smooth_radon_image(geo, 46)
    f_or = oracle_direct.adj_x(g, geo.Nt, geo.dt, geo.x(), 0.0, geo.dtau, geo.q())
    assert _rel(lp.adjoint(g), f_or) < 5e-3


def test_mutant_equal_offset_weights_caught(blob_geo, monkeypatch):
    def equal(self):
        k = np.arange(self.Nx)
        return np.where((k == 0) | (k == self.Nx - 1), 0.5, 1.0)
    monkeypatch.setattr(Desc, "x_weights", equal)
    assert max(_blob_errors(blob_geo, _desc(blob_geo, sigma=2.0, omega_c=0.25))) > BLOB_TOL


def test_mutant_regular_offset_positions_caught(blob_geo, monkeypatch):
    monkeypatch.setattr(Desc, "xb", lambda self: np.arange(self.Nx) / (self.Nx - 1))
    assert max(_blob_errors(blob_geo, _desc(blob_geo, sigma=2.0, omega_c=0.25))) > BLOB_TOL


def test_descriptor_rejects_bad_grids():
    with pytest.raises(ValueError):
        Desc(8, 4, 8, 3, 0.01, 0.1, 0.2, 0.6, x=(0.0, 0.2, 0.1, 0.3))
    with pytest.raises(ValueError):
        Desc(8, 4, 8, 3, 0.01, 0.1, 0.2, 0.6, x=(0.0, 0.1, 0.2))
    with pytest.raises(ValueError):
        Desc(8, 4, 8, 3, 0.01, 0.1, 0.2, 0.6, q_values=(0.2, 0.2, 0.6))


def test_irregular_geometry_generator():
    """The input recipe: inner offsets jittered within half a spacing (so
    strictly increasing), the end offsets fixed; slownesses from qmin to qmax,
    denser towards qmin for q_power > 1."""
    import synth
    geo = synth.irregular_geometry(100, 257, 90, 65, 0.004, 2.0, 0.2, 0.7, 5, jitter=0.45, near=0.1, q_power=1.6)
    x, q = geo.x(), geo.q()
    h = (2.0 - 0.1) / 256
    assert x.shape == (257,) and np.all(np.diff(x) > 0)
    assert x[0] == 0.1 and x[-1] == 2.0 and geo.X == 2.0
    assert np.max(np.abs(x - (0.1 + np.arange(257) * h))) <= 0.45 * h + 1e-12
    assert q.shape == (65,) and np.all(np.diff(q) > 0) and q[0] == 0.2 and abs(q[-1] - 0.7) < 1e-12
    assert np.diff(q)[0] < np.diff(q)[-1]
    again = synth.irregular_geometry(100, 257, 90, 65, 0.004, 2.0, 0.2, 0.7, 5, jitter=0.45, near=0.1, q_power=1.6)
    assert again == geo                                  # seeded
