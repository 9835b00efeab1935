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
    # lattices taking 9 * 2^a FFT lengths: rho 144, rho 1152, theta 2304
    dict(Nt=128, Nx=128, Ntau=128, Nq=128, dt=0.004, dx=1.6 / 127, qmin=0.2, qmax=0.7, sigma=1.25,
         omega_c=0.35, tsplits=(0.25, 0.5)),
    dict(Nt=768, Nx=384, Ntau=768, Nq=384, dt=0.002, dx=2.0 / 383, qmin=0.2, qmax=0.7, sigma=1.25,
         omega_c=0.35, tsplits=(0.25, 0.5)),
    dict(Nt=1024, Nx=1024, Ntau=1024, Nq=1024, dt=0.002, dx=2.0 / 1023, qmin=0.1, qmax=0.7,
         tsplits=(0.25, 0.5)),
    # quintic B-splines: three guard cells per side
    dict(Nt=256, Nx=96, Ntau=200, Nq=64, dt=0.004, dx=0.02, qmin=0.2, qmax=0.7, sigma=1.1,
         omega_c=0.4, tsplits=(0.25, 0.5), order=5),
    dict(Nt=2048, Nx=2048, Ntau=2048, Nq=2048, dt=2.0 / 2047, dx=2.0 / 2047, qmin=0.2, qmax=0.7,
         sigma=1.1, omega_c=0.4, tsplits=(0.25, 0.5), order=5),
]


def _lib_geometry(c, x=None, q=None):
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
    d.spline_order = c.get("order", 3)
    n = ctypes.c_int()
    infos = (_lib.RadonPieceInfo * 64)()
    arr = lambda v: None if v is None else (ctypes.c_double * len(v))(*v)
    _lib.check(L.radon_geometry_grid(ctypes.byref(d), arr(x), arr(q), ctypes.byref(n), infos, 64))
    return [{k: getattr(infos[i], k) for k, _ in _lib.RadonPieceInfo._fields_} for i in range(n.value)]


def _given_grid_cases():
    import synth
    out = []
    for args, kw, method in [
        ((256, 96, 256, 64, 0.004, 1.6, 0.2, 0.7, 11), dict(jitter=0.4, near=0.1, q_power=1.5), {}),
        ((333, 150, 301, 77, 0.006, 2.0, 0.15, 0.65, 12), dict(jitter=0.3, near=0.05, q_power=1.3),
         dict(tsplits=(0.3, 0.6), n_qsplit=2)),
        ((2048, 2048, 2048, 2048, 2.0 / 2047, 2.0, 0.2, 0.7, 14), dict(jitter=0.4, near=0.1, q_power=1.5),
         dict(sigma=1.25, omega_c=0.35, tsplits=(0.25, 0.5))),
    ]:
        geo = synth.irregular_geometry(*args, **kw)
        c = dict(Nt=geo.Nt, Nx=geo.Nx, Ntau=geo.Ntau, Nq=geo.Nq, dt=geo.dt, dx=geo.dx, qmin=geo.qmin,
                 qmax=geo.qmax, **method)
        out.append((c, geo.offsets, geo.slownesses))
    return out


def _check(c, x=None, q=None):
    desc = Desc(c["Nt"], c["Nx"], c["Ntau"], c["Nq"], c["dt"], c["dx"], c["qmin"], c["qmax"],
                tau0=c.get("tau0", 0.0), dtau=c.get("dtau", 0.0), sigma=c.get("sigma", 2.0),
                omega_c=c.get("omega_c", 0.25), tsplits=c.get("tsplits", ()),
                n_qsplit=c.get("n_qsplit", 1), x=x, q_values=q, order=c.get("order", 3))
    parts = oracle_plan(desc)
    lib = {(p["jt_lo"], p["l_lo"]): p for p in _lib_geometry(c, x, q)}
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


@pytest.mark.parametrize("c", CASES, ids=[f"case{i}" for i in range(len(CASES))])
def test_host_geometry_equals_oracle(c):
    _check(c)


@pytest.mark.parametrize("i", range(3))
def test_host_geometry_on_given_grids_equals_oracle(i):
    """Unequal offsets and slownesses (radon_geometry_grid): the same lattices
    as the oracle, whose spacing rule runs over equally spaced offsets of the
    same range."""
    c, x, q = _given_grid_cases()[i]
    _check(c, x, q)


def test_host_geometry_quintic_on_given_grids_equals_oracle():
    """Quintic B-splines (three guard cells) on unequal offsets and
    slownesses, two slowness pieces."""
    c, x, q = _given_grid_cases()[1]
    _check(dict(c, order=5), x, q)
