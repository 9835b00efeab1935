"""Pins of the FP64 sparse-inversion oracle (oracle/solvers.py), no GPU.

* the soft threshold of Section 3 on hand values;
* the iteration's fixed point is the minimiser of
  ||chi_S A g - f||^2 + mu ||g||_1: checked against an independent solver
  (cyclic coordinate descent, written here) on explicit matrices, with and
  without a trace mask, for the paper's iteration and for FISTA;
* the power iteration against the largest singular value from an SVD;
* on the oracle's log-polar operator: the objective never increases along the
  paper's iteration, and torch's gradient check of the operator (forward with
  the adjoint as its backward, FP64, a 128 x 32 gather);
* the Radon-domain mute on hand values and the limits of the multiple
  attenuation (border above or below every slowness).
"""
import numpy as np
import pytest

import synth
from oracle import solvers
from oracle.logpolar import Desc, LogPolar


def test_soft_threshold_hand_values():
    v = np.array([-3.0, -1.0, -0.5, 0.0, 0.99, 1.0, 1.5, 3.0])
    # threshold mu / 2 = 1
    np.testing.assert_array_equal(solvers.soft_threshold(v, 2.0), [-2.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.5, 2.0])
    np.testing.assert_array_equal(solvers.soft_threshold(v, 0.0), v)


def _lasso_cd(B, f, mu, sweeps=20000, tol=1e-15):
    """min ||B g - f||^2 + mu ||g||_1 by cyclic coordinate descent: each
    coordinate minimised exactly, g_i = S(b_i . r_i, at mu/2) / ||b_i||^2."""
    g = np.zeros(B.shape[1])
    r = f - B @ g
    nrm = np.sum(B * B, axis=0)
    for _ in range(sweeps):
        change = 0.0
        for i in range(B.shape[1]):
            if nrm[i] == 0.0:
                continue
            z = B[:, i] @ r + nrm[i] * g[i]
            gi = np.sign(z) * max(abs(z) - mu / 2, 0.0) / nrm[i]
            if gi != g[i]:
                r -= B[:, i] * (gi - g[i])
                change = max(change, abs(gi - g[i]))
                g[i] = gi
        if change < tol:
            break
    return g


def _problem(seed, m=40, n=30, missing=False):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((m, n))                      # "adjoint": image (n) -> data (m)
    g_true = np.zeros(n)
    g_true[rng.choice(n, 5, replace=False)] = rng.standard_normal(5) * 3
    f = B @ g_true + 0.05 * rng.standard_normal(m)
    mask = None
    if missing:
        mask = (rng.random(m) > 0.4).astype(float)
        f = f * mask
    return B, f, mask


@pytest.mark.parametrize("missing", [False, True])
@pytest.mark.parametrize("accelerate", [False, True])
def test_iteration_reaches_the_lasso_minimiser(missing, accelerate):
    B, f, mask = _problem(7, missing=missing)
    mu = 1.5
    # data [m] seen as [m][1] so that the mask applies per row, as per trace
    fwd = lambda r: B.T @ r[:, 0]
    adj = lambda g: (B @ g)[:, None]
    c2 = 0.9 / np.linalg.norm(B, 2) ** 2
    g = solvers.ista(fwd, adj, f[:, None], mu, c2, 30000 if not accelerate else 3000,
                     mask=mask, accelerate=accelerate)
    Bm = B if mask is None else B * mask[:, None]
    g_cd = _lasso_cd(Bm, f, mu)
    np.testing.assert_allclose(g, g_cd, rtol=0, atol=1e-8)
    assert np.count_nonzero(g_cd) < B.shape[1]            # the l1 term is active


def test_power_iteration_matches_svd():
    B, _, _ = _problem(3)
    fwd = lambda r: B.T @ r
    adj = lambda g: B @ g
    lam = solvers.power_norm2(fwd, adj, np.random.default_rng(0).standard_normal(B.shape[1]), 400)
    assert abs(lam - np.linalg.norm(B, 2) ** 2) < 1e-9 * lam


@pytest.fixture(scope="module")
def small_logpolar():
    geo = synth.Geometry(128, 32, 96, 24, 0.008, 0.05, 0.2, 0.7)
    desc = Desc(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax,
                sigma=1.25, omega_c=0.35, tsplits=())
    return geo, LogPolar(desc)


def test_objective_never_increases_on_the_log_polar_operator(small_logpolar):
    geo, lp = small_logpolar
    f = synth.band_limited_gather(geo, 31, n_events=4, nu=8.0)
    mask = (np.random.default_rng(5).random(geo.Nx) > 0.4).astype(float)
    f = f * mask[:, None]
    lam = solvers.power_norm2(lp.forward, lp.adjoint, np.ones((geo.Nq, geo.Ntau)), 40)
    c2 = 0.9 / lam
    mu = 0.05 * np.abs(lp.forward(f)).max()
    g = np.zeros((geo.Nq, geo.Ntau))
    prev = solvers.objective(lp.forward, lp.adjoint, f, g, mu, mask)
    for _ in range(8):
        g = solvers.ista(lp.forward, lp.adjoint, f, mu, c2, 1, g0=g, mask=mask)
        cur = solvers.objective(lp.forward, lp.adjoint, f, g, mu, mask)
        assert cur <= prev * (1 + 1e-12)
        prev = cur
    assert prev < solvers.objective(lp.forward, lp.adjoint, f, np.zeros_like(g), mu, mask)


def test_fp64_gradient_check_of_the_operator(small_logpolar):
    """The differentiation pattern in FP64: an autograd function whose backward
    is the adjoint passes torch's finite-difference gradient check."""
    torch = pytest.importorskip("torch")
    geo, lp = small_logpolar

    class Op(torch.autograd.Function):
        @staticmethod
        def forward(ctx, f):
            return torch.from_numpy(lp.forward(f.detach().numpy()))

        @staticmethod
        def backward(ctx, gg):
            return torch.from_numpy(lp.adjoint(gg.detach().numpy()))

    f = torch.from_numpy(np.random.default_rng(9).standard_normal((geo.Nx, geo.Nt))).requires_grad_(True)
    assert torch.autograd.gradcheck(Op.apply, (f,), eps=1e-6, atol=1e-7, rtol=1e-6, fast_mode=True)


def test_mute_hand_values():
    tau = np.array([0.0, 1.0, 2.0])
    q = np.array([0.1, 0.3, 0.5])
    g = np.arange(9, dtype=float).reshape(3, 3) + 1.0
    # line q = 0.2 + 0.1 tau: q=0.1 below everywhere, q=0.3 above at tau 0 only, q=0.5 above everywhere
    np.testing.assert_array_equal(solvers.mute(g, tau, q, 0.2, 0.1, "below"), [[1, 2, 3], [0, 5, 6], [0, 0, 0]])
    np.testing.assert_array_equal(solvers.mute(g, tau, q, 0.2, 0.1, "above"), [[0, 0, 0], [4, 0, 0], [7, 8, 9]])


def test_demultiple_limits(small_logpolar):
    """A border above every slowness leaves the gather untouched; a border
    below every slowness subtracts the whole sparse model (f - R* g)."""
    geo, lp = small_logpolar
    f = synth.band_limited_gather(geo, 33, n_events=4, nu=8.0)
    lam = solvers.power_norm2(lp.forward, lp.adjoint, np.ones((geo.Nq, geo.Ntau)), 30)
    c2, mu = 0.9 / lam, 0.05 * np.abs(lp.forward(f)).max()
    fo, g = solvers.demultiple(lp.forward, lp.adjoint, f, geo.tau(), geo.q(), 10.0, 0.0, 5, c2, mu)
    np.testing.assert_array_equal(fo, f)
    fo, g = solvers.demultiple(lp.forward, lp.adjoint, f, geo.tau(), geo.q(), -10.0, 0.0, 5, c2, mu)
    np.testing.assert_allclose(fo, f - lp.adjoint(g), rtol=0, atol=1e-12)
