"""Stage-level pins of the GPU path (through the C ABI) against the FP64
oracle's own stages, below the end-to-end parity tests:

* the sample lattice positions of every piece (the FP64 maps P1 T of
  Eq. (10)/(14), stored as first tap and FP32 fraction) within 1e-6 cells
  of the oracle's, and the gridding weights of Eq. (14)-(15) within 1e-6,
  on exactly the samples the oracle grids;
* the convolved lattice Q of Eq. (16)-(17) after a forward, and the lattice
  the adjoint gridding reads after an adjoint, element by element (the
  parity bounds of tests/parity.py) for every piece, cubic and quintic;
* the operator on a 16x8 -> 16x8 geometry assembled column by column: the
  adjoint's matrix is the forward's transpose to 1e-6 of its largest entry,
  and both match the oracle's matrices element by element.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import logpolar as LP
from oracle.logpolar import Desc, LogPolar
from parity import assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1604_07651_gb300 as hr
    return hr


def _cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


GEO = synth.Geometry(333, 150, 301, 77, 0.006, 0.013, 0.15, 0.65)
METHOD = dict(sigma=1.25, omega_c=0.35, tsplit=(0.3, 0.6), n_qsplit=2)


def _pair(hr, geo, order=3, **kw):
    plan = hr.Plan(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax, spline_order=order, **kw)
    d = plan.desc
    desc = Desc(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax, tau0=d.tau0, dtau=d.dtau,
                sigma=d.sigma, omega_c=d.omega_c, tsplits=tuple(d.tsplit[i] for i in range(d.n_tsplit)),
                n_qsplit=d.n_qsplit, order=order)
    return plan, LogPolar(desc)


def _piece_index(plan, lp):
    """Plan piece index of every oracle sub-problem (matched by its ranges)."""
    idx = {(p["jt_lo"], p["l_lo"]): i for i, p in enumerate(plan.pieces())}
    return [idx[(part.jt_lo, part.l_lo)] for part in lp.parts]


@pytest.mark.parametrize("order", [3, 5])
def test_sample_positions_and_weights_match_oracle(hr, order):
    plan, lp = _pair(hr, GEO, order, **METHOD)
    for part, pi, (jj, kk, xth, xrh, wfac) in zip(lp.parts, _piece_index(plan, lp), lp.dpts):
        th, rh, w = plan.piece_samples(pi)
        jl = jj - part.jt_lo
        gridded = wfac != 0
        assert np.all(w[kk[gridded], jl[gridded]] != 0)
        mask = np.zeros(w.shape, bool)
        mask[kk, jl] = True
        assert not np.any(w[~mask] != 0)                # nothing outside the oracle's samples
        sel = (kk[gridded], jl[gridded])
        assert np.max(np.abs(th[sel] - xth[gridded])) <= 1e-6
        assert np.max(np.abs(rh[sel] - xrh[gridded])) <= 1e-6
        ref = wfac[gridded] / (part.dtheta * part.drho)
        assert np.max(np.abs(w[sel] - ref) / np.abs(ref)) <= 1e-6
    plan.close()


@pytest.mark.parametrize("order", [3, 5])
def test_convolved_lattices_match_oracle_stages(hr, order):
    plan, lp = _pair(hr, GEO, order, **METHOD)
    f = synth.band_limited_gather(GEO, 51, n_events=6, nu=10.0)
    plan.forward(_cuda(f))
    for p, pi in enumerate(_piece_index(plan, lp)):
        _, Q = lp.stages_forward(f, p)
        assert_parity(plan.piece_lattice(pi), Q, what=f"piece {p} forward lattice")
    gg = synth.random_radon_image(GEO, 52)
    plan.adjoint(_cuda(gg))
    for p, pi in enumerate(_piece_index(plan, lp)):
        part, K = lp.parts[p], lp.K[p]
        ll, ii, yth, yrh, valid, scale = lp.rpts[p]
        Qt = LP.interp_adj(part, gg[ll, ii], yth, yrh, valid, scale)
        G = LP.conv(part, Qt, K, adjoint=True)
        assert_parity(plan.piece_lattice(pi), G, what=f"piece {p} adjoint lattice")
    plan.close()


def test_operator_matrix_16x8_is_transposed_by_the_adjoint(hr):
    geo = synth.Geometry(16, 8, 16, 8, 0.02, 0.1, 0.2, 0.7)
    plan, lp = _pair(hr, geo, tsplit=())
    n_in, n_out = geo.Nx * geo.Nt, geo.Nq * geo.Ntau
    A = np.zeros((n_out, n_in))
    A_or = np.zeros((n_out, n_in))
    for c in range(n_in):
        e = np.zeros(n_in)
        e[c] = 1.0
        A[:, c] = plan.forward(_cuda(e.reshape(geo.Nx, geo.Nt))).cpu().numpy().ravel()
        A_or[:, c] = lp.forward(e.reshape(geo.Nx, geo.Nt)).ravel()
    B = np.zeros((n_in, n_out))
    B_or = np.zeros((n_in, n_out))
    for r in range(n_out):
        e = np.zeros(n_out)
        e[r] = 1.0
        B[:, r] = plan.adjoint(_cuda(e.reshape(geo.Nq, geo.Ntau))).cpu().numpy().ravel()
        B_or[:, r] = lp.adjoint(e.reshape(geo.Nq, geo.Ntau)).ravel()
    amax = np.abs(A).max()
    assert amax > 0
    assert np.abs(B - A.T).max() <= 1e-6 * amax
    assert np.abs(B_or - A_or.T).max() <= 1e-12 * amax          # the oracle's exact transpose
    assert np.abs(A - A_or).max() <= 1e-5 * amax
    assert np.abs(B - B_or).max() <= 1e-5 * amax
    plan.close()
