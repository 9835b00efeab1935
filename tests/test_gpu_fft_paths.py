"""Every compile-time FFT pass schedule of the GPU path against the FP64
log-polar oracle: the column pass and the row transforms of the lengths
R0 * 256 (radices R0, 16, 16) are compiled per R0, so each R0 a plan can
produce gets a geometry whose lattices take it (found on the host with
radon_geometry), forward and adjoint element by element (tests/parity.py).
The 2048^2 benchmark plans (column R0 9 and 10, rows 4 and 6) are in
test_gpu_parity.py."""
import numpy as np
import pytest
import torch

import synth
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


# name: (Nt = Ntau, Nx = Nq, X (km), qmax, sigma), T = 2 s, qmin 0.2, omega_c 0.4
CASES = {
    "rows_R0_2": (768, 48, 1.0, 0.7, 2.0),        # row half length 512
    "rows_R0_3": (1536, 48, 1.0, 0.5, 2.0),       # 768
    "rows_R0_5": (2048, 128, 1.0, 0.5, 2.5),      # 1280
    "rows_R0_8": (2048, 128, 1.0, 0.7, 3.0),      # 2048
    "cols_R0_5": (512, 1024, 1.0, 0.5, 1.1),      # column length 1280
    "cols_R0_6": (512, 512, 1.0, 0.5, 2.5),       # 1536
    "cols_R0_8": (512, 1024, 1.0, 0.5, 1.5),      # 2048
    "cols_R0_12": (512, 1024, 1.0, 0.5, 2.5),     # 3072
    "rows_R0_10": (2048, 384, 2.0, 0.7, 3.0),     # 2560
    "rows_R0_12": (2048, 512, 2.0, 0.7, 3.0),     # 3072
}


def _r0(n):
    q = n // 256
    return q if n == 256 * q else None


@pytest.mark.parametrize("name", list(CASES))
def test_compiled_fft_lengths_match_oracle(hr, name):
    Nt, Nx, X, qmax, sigma = CASES[name]
    geo = synth.Geometry(Nt, Nx, Nt, Nx, 2.0 / (Nt - 1), X / (Nx - 1), 0.2, qmax)
    plan = hr.Plan(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax, sigma=sigma,
                   omega_c=0.4, tsplit=(0.25, 0.5))
    kind, want = name.split("_R0_")[0], int(name.split("_R0_")[1])
    pieces = plan.pieces()
    lengths = [p["Ptheta"] for p in pieces] if kind == "cols" else [p["Prho"] // 2 for p in pieces]
    assert want in [_r0(n) for n in lengths], lengths       # the geometry takes the length it names
    lp = LogPolar(Desc(geo.Nt, geo.Nx, geo.Ntau, geo.Nq, geo.dt, geo.dx, geo.qmin, geo.qmax, sigma=sigma,
                       omega_c=0.4, tsplits=(0.25, 0.5)))
    f = synth.band_limited_gather(geo, 91, n_events=6, nu=10.0)
    assert_parity(plan.forward(_cuda(f)).cpu().numpy(), lp.forward(f), what=name + " forward")
    gg = synth.random_radon_image(geo, 92)
    assert_parity(plan.adjoint(_cuda(gg)).cpu().numpy(), lp.adjoint(gg), what=name + " adjoint")
    plan.close()
