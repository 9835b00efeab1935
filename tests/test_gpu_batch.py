"""Batches of uneven gathers (radon_batch_* through the C ABI): every gather
of a batch gives the result of its own plan, matches the FP64 log-polar
oracle on the same lattices, BF16 input matches the oracle on the rounded
input, and the batch replays from a CUDA graph."""
import numpy as np
import pytest
import torch

import synth
from oracle.logpolar import Desc, LogPolar
from parity import assert_parity

pytestmark = pytest.mark.gpu



def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def hr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1604_07651_gb300 as hr
    return hr


def _geo_dict(geo):
    return dict(Nt=geo.Nt, Nx=geo.Nx, Ntau=geo.Ntau, Nq=geo.Nq, dt=geo.dt, dx=geo.dx,
                qmin=geo.qmin, qmax=geo.qmax)


@pytest.fixture(scope="module")
def uneven(hr):
    geos = synth.batch_geometries(10)
    gathers = [synth.batch_gather(g, i) for i, g in enumerate(geos)]
    batch = hr.Batch([_geo_dict(g) for g in geos])
    return geos, gathers, batch


def test_batch_equals_single_plans(hr, uneven):
    geos, gathers, batch = uneven
    f = batch.pack([torch.tensor(x, dtype=torch.float32) for x in gathers])
    g = batch.forward(f)
    imgs = batch.unpack_images(g)
    fa = batch.unpack_gathers(batch.adjoint(g))
    for geo, x, gi, fai in zip(geos, gathers, imgs, fa):
        plan = hr.Plan(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax)
        gs = plan.forward(torch.tensor(x, dtype=torch.float32, device="cuda"))
        assert _rel(gi.cpu().numpy(), gs.cpu().numpy().astype(np.float64)) < 1e-6
        fs = plan.adjoint(gi.contiguous())
        assert _rel(fai.cpu().numpy(), fs.cpu().numpy().astype(np.float64)) < 1e-6
        plan.close()


def _small_batch():
    geos = [synth.Geometry(300, 64, 280, 48, 0.004, 0.025, 0.2, 0.7),
            synth.Geometry(520, 90, 520, 90, 0.004, 0.025, 0.2, 0.7),
            synth.Geometry(180, 120, 200, 60, 0.004, 0.025, 0.15, 0.65)]
    return geos, [synth.batch_gather(g, 100 + i) for i, g in enumerate(geos)]


def _oracle(geo, d):
    """The FP64 log-polar oracle with the method parameters of the library's
    resolved descriptor d (the batch's own plan of this gather)."""
    return LogPolar(Desc(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax,
                         sigma=d.sigma, omega_c=d.omega_c, tsplits=tuple(d.tsplit[i] for i in range(d.n_tsplit)),
                         n_qsplit=d.n_qsplit))


def test_batch_against_oracle_fp32_and_bf16(hr):
    geos, gathers = _small_batch()
    batch = hr.Batch([_geo_dict(g) for g in geos])
    f32 = batch.pack([torch.tensor(x, dtype=torch.float32) for x in gathers])
    g32 = batch.unpack_images(batch.forward(f32))
    fb = batch.pack([torch.tensor(x, dtype=torch.float32) for x in gathers], dtype=torch.bfloat16)
    gb = batch.unpack_images(batch.forward(fb))
    gimg = [synth.random_radon_image(g, 200 + i) for i, g in enumerate(geos)]
    fa = batch.unpack_gathers(batch.adjoint(torch.cat([torch.tensor(x, dtype=torch.float32).reshape(-1)
                                                       for x in gimg]).cuda()))
    for i, (geo, x, a, b, gi, fi) in enumerate(zip(geos, gathers, g32, gb, gimg, fa)):
        lp = _oracle(geo, batch.plan_desc(i))
        assert_parity(a.cpu().numpy(), lp.forward(x), what="batch FP32 forward")
        xb = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
        ref_b = lp.forward(xb)
        assert_parity(b.cpu().numpy(), ref_b, what="batch BF16 forward")   # same input as the kernel sees
        assert _rel(b.cpu().numpy(), lp.forward(x)) < 1e-2      # BF16 storage error of the input
        assert_parity(fi.cpu().numpy(), lp.adjoint(gi), what="batch adjoint")
    batch.close()


def test_batch_replays_from_a_cuda_graph(hr, uneven):
    geos, gathers, batch = uneven
    f = batch.pack([torch.tensor(x, dtype=torch.float32) for x in gathers])
    g = torch.empty(batch.g_offsets[-1], dtype=torch.float32, device="cuda")
    fa = torch.empty(batch.f_offsets[-1], dtype=torch.float32, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        batch.forward(f, out=g)          # warm-up (sets kernel attributes) outside capture
        batch.adjoint(g, out=fa)
    torch.cuda.current_stream().wait_stream(s)
    ref_g, ref_f = g.clone(), fa.clone()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        batch.forward(f, out=g)
        batch.adjoint(g, out=fa)
    g.zero_()
    fa.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert _rel(g.cpu().numpy(), ref_g.cpu().numpy().astype(np.float64)) < 1e-6
    assert _rel(fa.cpu().numpy(), ref_f.cpu().numpy().astype(np.float64)) < 1e-6


def test_batch_rows_per_band_tuning(hr, uneven):
    """The batch-wide rows-per-band tuner (every descriptor asks for 0) picks a
    feasible value and changes the work split only, not the results."""
    geos, gathers, batch = uneven
    tuned = hr.Batch([dict(_geo_dict(g), rows_per_band=0) for g in geos])
    f = batch.pack([torch.tensor(x, dtype=torch.float32) for x in gathers])
    g_ref = batch.forward(f)
    g = tuned.forward(f)
    assert _rel(g.cpu().numpy(), g_ref.cpu().numpy().astype(np.float64)) < 1e-6
    fa = tuned.adjoint(g_ref)
    fa_ref = batch.adjoint(g_ref)
    assert _rel(fa.cpu().numpy(), fa_ref.cpu().numpy().astype(np.float64)) < 1e-6
    tuned.close()
