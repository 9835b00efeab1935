"""The library's FP64 host geometry (C++, through radon_geometry) equals the
oracle's (numpy) for every sub-problem, without a GPU: identical lattice
sizes, FFT sizes and frequency rectangles, floats to 1e-12."""
import ctypes

import pytest

from oracle.logpolar import Desc, plan as oracle_plan

CASES = [
    dict(Nt=256, Nx=64, Ntau=256, Nq=64, dt=0.004, dx=1.6 / 63, qmin=0.2, qmax=0.7),
    dict(Nt=2048, Nx=2048, Ntau=2048, Nq=2048, dt=2.0 / 2047, dx=2.0 / 2047, qmin=0.2, qmax=0.7),
    dict(Nt=333, Nx=150, Ntau=301, Nq=77, dt=0.006, dx=0.013, qmin=0.15, qmax=0.65,
         tsplits=(0.3, 0.6), n_qsplit=2),
    dict(Nt=200, Nx=90, Ntau=180, Nq=50, dt=0.005, dx=0.02, qmin=0.0, qmax=0.6, tsplits=()),
    dict(Nt=300, Nx=120, Ntau=300, Nq=120, dt=0.006, dx=0.015, qmin=0.2, qmax=0.7, sigma=2.0,
         omega_c=0.25, tsplits=(0.3, 0.6)),
    dict(Nt=256, Nx=96, Ntau=200, Nq=64, dt=0.004, dx=0.02, qmin=0.2, qmax=0.7, tau0=0.2,
         dtau=0.004),
    dict(Nt=64, Nx=32, Ntau=64, Nq=1, dt=0.01, dx=0.03, qmin=0.4, qmax=0.4, tsplits=()),
    dict(Nt=8, Nx=4, Ntau=8, Nq=3, dt=0.1, dx=0.1, qmin=0.2, qmax=0.7, tsplits=()),
    dict(Nt=1500, Nx=300, Ntau=1500, Nq=300, dt=0.004, dx=0.025, qmin=0.2, qmax=0.7,
         tsplits=(0.1, 0.25, 0.5), n_qsplit=3),
]


def _lib_geometry(c):
    from paper_1604_07651_gb300 import _lib
    L = _lib.load()
    d = _lib.RadonDesc()
    L.radon_desc_init(ctypes.byref(d), c["Nt"], c["Nx"], c["Ntau"], c["Nq"], c["dt"], c["dx"],
                      c["qmin"], c["qmax"])
    d.sigma = c.get("sigma", 2.0)
    d.omega_c = c.get("omega_c", 0.25)
    d.tau0 = c.get("tau0", 0.0)
    d.dtau = c.get("dtau", 0.0)
    ts = c.get("tsplits", ())
    d.n_tsplit = len(ts)
    for i, v in enumerate(ts):
        d.tsplit[i] = v
    d.n_qsplit = c.get("n_qsplit", 1)
    n = ctypes.c_int()
    infos = (_lib.RadonPieceInfo * 64)()
    _lib.check(L.radon_geometry(ctypes.byref(d), ctypes.byref(n), infos, 64))
    return [{k: getattr(infos[i], k) for k, _ in _lib.RadonPieceInfo._fields_} for i in range(n.value)]


@pytest.mark.parametrize("c", CASES, ids=[f"case{i}" for i in range(len(CASES))])
def test_host_geometry_equals_oracle(c):
    desc = Desc(c["Nt"], c["Nx"], c["Ntau"], c["Nq"], c["dt"], c["dx"], c["qmin"], c["qmax"],
                tau0=c.get("tau0", 0.0), dtau=c.get("dtau", 0.0), sigma=c.get("sigma", 2.0),
                omega_c=c.get("omega_c", 0.25), tsplits=c.get("tsplits", ()),
                n_qsplit=c.get("n_qsplit", 1))
    parts = oracle_plan(desc)
    lib = {(p["jt_lo"], p["l_lo"]): p for p in _lib_geometry(c)}
    assert len(lib) == len(parts)
    for part in parts:
        p = lib[(part.jt_lo, part.l_lo)]
        for k in ("jt_hi", "l_hi", "Ntheta", "Nrho", "k1max", "k2max"):
            assert p[k] == getattr(part, k), k
        assert (p["Ptheta"], p["Prho"]) == (part.P_theta, part.P_rho)
        for k in ("alpha", "beta", "a", "O1", "O2", "a_r", "r_max", "dphi_rule", "deta_rule",
                  "dtheta", "drho", "theta0", "rho0", "theta_m"):
            ref = getattr(part, k)
            assert abs(p[k] - ref) <= 1e-12 * max(1.0, abs(ref)), (k, p[k], ref)
