"""Pins of the FP64 direct-summation oracle (Eq. (1), (3); Section 5).

Each check ties the oracle to something other than itself: a closed form of
Eq. (1), an exact special case, an invariant of the hyperbolic integral, or
brute force.
"""
import math

import numpy as np
import pytest

import synth
from oracle import closed_forms as cf


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_gaussian_closed_form_small_gather(oracle_direct):
    """C1: f = exp(-25 t^2 - 10 x^2) on the 256x64 gather (dt = 4 ms, 1.6 km)."""
    geo = synth.Geometry(256, 64, 256, 64, 0.004, 1.6 / 63, 0.2, 0.7)
    f = synth.gaussian_gather(geo, 25.0, 10.0)
    g = oracle_direct.fwd(f, geo.dt, geo.dx, geo.tau(), geo.q())
    g_ex = cf.gaussian_tx(geo.tau(), geo.q(), 25.0, 10.0, geo.T, geo.X)
    assert _rel(g, g_ex) < 1e-6


def test_gaussian_converges_with_refinement(oracle_direct):
    """Away from t = 0 the error of the cubic-in-t sum against the exact
    integral falls by about 2^3 each time dt halves (Keys is third order)."""
    errs = []
    for Nt in (100, 200, 400):
        geo = synth.Geometry(Nt, 64, 40, 7, 1.0 / (Nt - 1), 1.0 / 63, 0.0, 0.9)
        f = synth.gaussian_gather(geo, 30.0, 25.0)
        tau = np.linspace(0.15, 0.6, 40)
        g = oracle_direct.fwd(f, geo.dt, geo.dx, tau, geo.q())
        g_ex = cf.gaussian_tx(tau, geo.q(), 30.0, 25.0, geo.T, geo.X)
        errs.append(_rel(g, g_ex))
    assert errs[0] / errs[1] > 7.0 and errs[1] / errs[2] > 7.0
    assert errs[2] < 1e-7


def test_zero_slowness_is_trapezoid_sum(oracle_direct):
    """C3: at q = 0 and tau on the t-grid the cubic interpolation is exact,
    so R_h f(t_j, 0) = 2 * trapezoid over x of f(t_j, .)."""
    geo = synth.Geometry(40, 17, 40, 3, 0.01, 0.05, 0.0, 0.4)
    rng = np.random.default_rng(3)
    f = rng.standard_normal((geo.Nx, geo.Nt))
    g = oracle_direct.fwd(f, geo.dt, geo.dx, geo.t(), np.array([0.0]))
    w = np.ones(geo.Nx)
    w[0] = w[-1] = 0.5
    expect = 2.0 * geo.dx * (w[:, None] * f).sum(axis=0)
    np.testing.assert_allclose(g[0], expect, rtol=0, atol=1e-13)


def test_event_invariant(oracle_direct):
    """C2: f = h(t^2 - q0^2 x^2) gives R_h f(tau, q0) = 2 X h(tau^2) while the
    hyperbola stays inside the rectangle (catches q vs q^2 and factor-2 slips)."""
    Nt, Nx = 400, 60
    dt, dx = 0.005, 0.03
    q0 = 0.5
    T, X = (Nt - 1) * dt, (Nx - 1) * dx
    h = lambda u: np.exp(-((u - 0.8) / 0.15) ** 2)
    t = np.arange(Nt) * dt
    x = np.arange(Nx) * dx
    f = h(t[None, :] ** 2 - (q0 * x[:, None]) ** 2)
    tau = np.linspace(0.5, 1.2, 30)
    assert math.sqrt(tau[-1] ** 2 + (q0 * X) ** 2) < T
    g = oracle_direct.fwd(f, dt, dx, tau, np.array([q0]))[0]
    expect = cf.event_on_slowness(tau, q0, X, h)
    assert _rel(g, expect) < 2e-4


def test_adjoint_dot_identity(oracle_direct):
    """Eq. (16): <R f, g> = <f, R* g> to FP64 rounding."""
    geo = synth.Geometry(96, 24, 80, 20, 0.01, 0.04, 0.1, 0.9)
    rng = np.random.default_rng(7)
    f = rng.standard_normal((geo.Nx, geo.Nt))
    g = rng.standard_normal((geo.Nq, geo.Ntau))
    Rf = oracle_direct.fwd(f, geo.dt, geo.dx, geo.tau(), geo.q())
    Rg = oracle_direct.adj(g, geo.Nt, geo.Nx, geo.dt, geo.dx, 0.0, geo.dtau, geo.q())
    lhs, rhs = float(np.sum(Rf * g)), float(np.sum(f * Rg))
    assert abs(lhs - rhs) / abs(lhs) < 1e-12


def test_adjoint_matches_brute_force_and_matrix_transpose(oracle_direct):
    """The tau-range shortcut of the adjoint equals the sum over every (i, l),
    and the adjoint's matrix is the transpose of the forward's (tiny grid)."""
    geo = synth.Geometry(16, 8, 12, 5, 0.02, 0.05, 0.2, 0.8)
    rng = np.random.default_rng(11)
    g = rng.standard_normal((geo.Nq, geo.Ntau))
    fa = oracle_direct.adj(g, geo.Nt, geo.Nx, geo.dt, geo.dx, 0.0, geo.dtau, geo.q())
    fb = oracle_direct.adj_brute(g, geo.Nt, geo.Nx, geo.dt, geo.dx, geo.tau(), geo.q())
    np.testing.assert_allclose(fa, fb, rtol=0, atol=1e-14)
    n_in, n_out = geo.Nx * geo.Nt, geo.Nq * geo.Ntau
    A = np.zeros((n_out, n_in))
    for c in range(n_in):
        e = np.zeros(n_in)
        e[c] = 1.0
        A[:, c] = oracle_direct.fwd(e.reshape(geo.Nx, geo.Nt), geo.dt, geo.dx,
                                    geo.tau(), geo.q()).ravel()
    B = np.zeros((n_in, n_out))
    for c in range(n_out):
        e = np.zeros(n_out)
        e[c] = 1.0
        B[:, c] = oracle_direct.adj(e.reshape(geo.Nq, geo.Ntau), geo.Nt, geo.Nx, geo.dt,
                                    geo.dx, 0.0, geo.dtau, geo.q()).ravel()
    np.testing.assert_allclose(B, A.T, rtol=0, atol=1e-15)


def test_sampled_points_equal_full(oracle_direct):
    geo, f = synth.single_gather(1)
    g = oracle_direct.fwd(f, geo.dt, geo.dx, geo.tau(), geo.q())
    rng = np.random.default_rng(5)
    ii = rng.integers(0, geo.Ntau, 200)
    li = rng.integers(0, geo.Nq, 200)
    gp = oracle_direct.fwd_points(f, geo.dt, geo.dx, geo.tau(), geo.q(), ii, li)
    np.testing.assert_array_equal(gp, g[li, ii])
    gg = synth.random_radon_image(geo, 9)
    fa = oracle_direct.adj(gg, geo.Nt, geo.Nx, geo.dt, geo.dx, 0.0, geo.dtau, geo.q())
    jj = rng.integers(0, geo.Nt, 200)
    kk = rng.integers(0, geo.Nx, 200)
    fp = oracle_direct.adj_points(gg, geo.Nt, geo.Nx, geo.dt, geo.dx, 0.0, geo.dtau, geo.q(), jj, kk)
    np.testing.assert_array_equal(fp, fa[kk, jj])
