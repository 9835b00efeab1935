"""Seeded synthetic CMP gathers and Radon-domain images.

This module only draws inputs. It holds none of the transform's arithmetic,
so both the oracle and the CUDA path may use it.

Layouts follow the library: a gather is ``f[Nx][Nt]`` (time fastest), a
Radon image is ``g[Nq][Ntau]`` (intercept time fastest). Everything is
float64; callers cast.

Events are hyperbolic reflections ``t = sqrt(tau0^2 + q0^2 x^2)`` carrying a
Ricker wavelet ``r(t) = (1 - 2 pi^2 nu^2 t^2) exp(-pi^2 nu^2 t^2)`` (the
CMP-gather model of the paper's Section 1 and Section 5 tests).
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = [
    "Geometry", "ricker", "rng_for", "hyperbolic_gather", "gaussian_gather",
    "random_radon_image", "single_gather", "sweep_gather", "large_gather", "missing_trace_gather",
    "batch_gather", "primaries_multiples",
    "band_limited_gather", "batch_geometries", "irregular_geometry",
]


@dataclasses.dataclass(frozen=True)
class Geometry:
    """Sampling of one gather and of its Radon image (physical units).

    ``offsets`` / ``slownesses``, when given, replace the regular offset grid
    ``k dx`` / slowness grid (unequally spaced geometries); X is then the
    largest offset."""
    Nt: int
    Nx: int
    Ntau: int
    Nq: int
    dt: float
    dx: float
    qmin: float
    qmax: float
    offsets: tuple | None = None
    slownesses: tuple | None = None

    @property
    def T(self) -> float:
        return (self.Nt - 1) * self.dt

    @property
    def X(self) -> float:
        if self.offsets is not None:
            return float(self.offsets[-1])
        return (self.Nx - 1) * self.dx

    @property
    def dtau(self) -> float:
        return self.T / (self.Ntau - 1)

    def t(self) -> np.ndarray:
        return np.arange(self.Nt) * self.dt

    def x(self) -> np.ndarray:
        if self.offsets is not None:
            return np.asarray(self.offsets, dtype=np.float64)
        return np.arange(self.Nx) * self.dx

    def tau(self) -> np.ndarray:
        return np.arange(self.Ntau) * self.dtau

    def q(self) -> np.ndarray:
        if self.slownesses is not None:
            return np.asarray(self.slownesses, dtype=np.float64)
        if self.Nq == 1:
            return np.array([self.qmin])
        return self.qmin + np.arange(self.Nq) * (self.qmax - self.qmin) / (self.Nq - 1)


def rng_for(tag: int) -> np.random.Generator:
    """PCG64 stream seeded by ``1604 + tag`` (one tag per workload)."""
    return np.random.Generator(np.random.PCG64(1604 + int(tag)))


def ricker(t: np.ndarray, nu: float) -> np.ndarray:
    a = (np.pi * nu * t) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def hyperbolic_gather(geo: Geometry, tau0, q0, nu, amp) -> np.ndarray:
    """Sum of Ricker events on hyperbolas ``t = sqrt(tau0^2 + q0^2 x^2)``."""
    t = geo.t()[None, :]
    x = geo.x()[:, None]
    f = np.zeros((geo.Nx, geo.Nt))
    for tz, qz, fz, az in zip(np.atleast_1d(tau0), np.atleast_1d(q0),
                              np.atleast_1d(nu), np.atleast_1d(amp)):
        arr = np.sqrt(tz * tz + (qz * x) ** 2)
        f += az * ricker(t - arr, fz)
    return f


def gaussian_gather(geo: Geometry, a: float, b: float) -> np.ndarray:
    """``exp(-a t^2 - b x^2)`` sampled on the gather grid."""
    t = geo.t()[None, :]
    x = geo.x()[:, None]
    return np.exp(-a * t * t - b * x * x)


def random_radon_image(geo: Geometry, tag: int) -> np.ndarray:
    """Smooth random Radon-domain image (for adjoint and dot tests)."""
    rng = rng_for(tag)
    g = rng.standard_normal((geo.Nq, geo.Ntau))
    # light smoothing along tau keeps it band-limited (3-tap binomial, twice)
    for _ in range(2):
        g[:, 1:-1] = 0.25 * g[:, :-2] + 0.5 * g[:, 1:-1] + 0.25 * g[:, 2:]
    return g


def smooth_radon_image(geo: Geometry, tag: int, n_blobs: int = 24,
                       width_samples: float = 6.0) -> np.ndarray:
    """Band-limited Radon-domain image: Gaussian blobs of about
    ``width_samples`` samples in tau and q at random positions and signs."""
    rng = rng_for(tag)
    i = np.arange(geo.Ntau)[None, :]
    l = np.arange(geo.Nq)[:, None]
    sc = max(1.0, geo.Ntau / 256.0)
    g = np.zeros((geo.Nq, geo.Ntau))
    for _ in range(n_blobs):
        ci, cl = rng.uniform(0.05, 0.95) * geo.Ntau, rng.uniform(0.0, 1.0) * geo.Nq
        wi, wl = width_samples * sc, width_samples * max(1.0, geo.Nq / 256.0)
        g += rng.standard_normal() * np.exp(-((i - ci) / wi) ** 2 - ((l - cl) / wl) ** 2)
    return g


def single_gather(tag: int = 1, nu: float = 25.0) -> tuple[Geometry, np.ndarray]:
    """Small gather: Nt=256 (dt=4 ms), Nx=64 offsets on [0,1.6] km,
    Ntau=256, Nq=64 on q in [0.2,0.7] s/km, 8 Ricker events,
    tau0~U[0.1,0.9] s, q0~U[0.25,0.65] s/km, amplitude N(0,1)."""
    geo = Geometry(256, 64, 256, 64, 0.004, 1.6 / 63, 0.2, 0.7)
    rng = rng_for(tag)
    n = 8
    tau0 = rng.uniform(0.1, 0.9, n)
    q0 = rng.uniform(0.25, 0.65, n)
    amp = rng.standard_normal(n)
    return geo, hyperbolic_gather(geo, tau0, q0, np.full(n, nu), amp)


def sweep_gather(N: int, tag: int = 2, n_events: int = 32,
                 noise: float = 0.05, T: float = 2.0, X: float = 2.0,
                 nu_range=(20.0, 40.0)) -> tuple[Geometry, np.ndarray]:
    """Square gather N=Nt=Nx=Ntau=Nq on t in [0,T] s, x in [0,X] km,
    q in [0.2,0.7] s/km; ``n_events`` Ricker events with
    tau0~U[0.1,0.9T], q0~U[0.25,0.65], nu~U[nu_range], A~N(0,1),
    plus Gaussian noise of ``noise`` times the clean RMS."""
    geo = Geometry(N, N, N, N, T / (N - 1), X / (N - 1), 0.2, 0.7)
    rng = rng_for(tag * 100003 + N)
    tau0 = rng.uniform(0.1, 0.9 * T, n_events)
    q0 = rng.uniform(0.25, 0.65, n_events)
    nu = rng.uniform(nu_range[0], nu_range[1], n_events)
    amp = rng.standard_normal(n_events)
    f = hyperbolic_gather(geo, tau0, q0, nu, amp)
    if noise > 0:
        rms = float(np.sqrt(np.mean(f * f)))
        f = f + noise * rms * rng.standard_normal(f.shape)
    return geo, f


def band_limited_gather(geo: Geometry, tag: int, n_events: int = 8,
                        nu: float = 12.0) -> np.ndarray:
    """Events with a low-frequency Ricker on any geometry (no noise)."""
    rng = rng_for(tag)
    T = geo.T
    tau0 = rng.uniform(0.1 * T, 0.85 * T, n_events)
    q0 = rng.uniform(0.25, 0.65, n_events)
    amp = rng.standard_normal(n_events)
    return hyperbolic_gather(geo, tau0, q0, np.full(n_events, nu), amp)


def large_gather(N: int = 4096, tag: int = 5, n_events: int = 64,
                 T: float = 2.0, X: float = 2.0) -> tuple[Geometry, np.ndarray]:
    """Large square gather: n_events Ricker primaries (20-40 Hz) and their
    first multiples (events at 2*tau0 with the same q0, half amplitude,
    opposite sign)."""
    geo = Geometry(N, N, N, N, T / (N - 1), X / (N - 1), 0.2, 0.7)
    rng = rng_for(tag * 100003 + N)
    npri = n_events
    tau0 = rng.uniform(0.1, 0.45 * T, npri)
    q0 = rng.uniform(0.25, 0.65, npri)
    nu = rng.uniform(20.0, 40.0, npri)
    amp = rng.standard_normal(npri)
    f = hyperbolic_gather(geo, tau0, q0, nu, amp)
    f += hyperbolic_gather(geo, 2 * tau0, q0, nu, -0.5 * amp)
    return geo, f


def missing_trace_gather(tag: int = 3, Nt: int = 1024, Nx: int = 256, n_events: int = 20,
                         missing: float = 0.4) -> tuple[Geometry, np.ndarray, np.ndarray]:
    """Trace-interpolation workload: Nt samples at dt = 2 ms, Nx offsets on
    [0, 2] km, Ntau = Nt, Nq = Nx on q in [0.2, 0.7] s/km; n_events Ricker
    hyperbolas (tau0 ~ U[0.1, 1.8] s, q0 ~ U[0.25, 0.65], 15-30 Hz,
    A ~ N(0, 1)). Returns the geometry, the complete gather and the trace
    mask (1 recorded, 0 missing; a `missing` fraction of the traces, chosen
    at random)."""
    geo = Geometry(Nt, Nx, Nt, Nx, 0.002, 2.0 / (Nx - 1), 0.2, 0.7)
    rng = rng_for(tag * 1000 + 7)
    tau0 = rng.uniform(0.1, 1.8, n_events)
    q0 = rng.uniform(0.25, 0.65, n_events)
    nu = rng.uniform(15.0, 30.0, n_events)
    amp = rng.standard_normal(n_events)
    f = hyperbolic_gather(geo, tau0, q0, nu, amp)
    mask = np.ones(Nx)
    mask[rng.choice(Nx, int(round(missing * Nx)), replace=False)] = 0.0
    return geo, f, mask


def primaries_multiples(geo: Geometry, tag: int = 6, n_events: int = 8) -> tuple[np.ndarray, np.ndarray]:
    """Gather of n_events primaries (q0 ~ U[0.25, 0.40] s/km) and as many
    slower multiples (q0 ~ U[0.50, 0.65] s/km), tau0 ~ U[0.1, 0.8 T],
    10-20 Hz Ricker wavelets, A ~ N(0, 1): the two separate by moveout in
    the Radon domain along q = 0.45 s/km. Returns (gather, primaries only)."""
    rng = rng_for(6000 + tag)
    T = (geo.Nt - 1) * geo.dt
    prim = hyperbolic_gather(geo, rng.uniform(0.1, 0.8 * T, n_events), rng.uniform(0.25, 0.40, n_events),
                             rng.uniform(10.0, 20.0, n_events), rng.standard_normal(n_events))
    mult = hyperbolic_gather(geo, rng.uniform(0.1, 0.8 * T, n_events), rng.uniform(0.50, 0.65, n_events),
                             rng.uniform(10.0, 20.0, n_events), rng.standard_normal(n_events))
    return prim + mult, prim


def batch_gather(geo: Geometry, tag: int) -> np.ndarray:
    """One gather of the uneven batch: 10-40 Ricker hyperbolas (tau0 ~
    U[0.1, 0.9 T] s, q0 ~ U[0.25, 0.65] s/km, 10-25 Hz, A ~ N(0, 1))."""
    rng = rng_for(4000 + tag)
    n = int(rng.integers(10, 41))
    T = (geo.Nt - 1) * geo.dt
    return hyperbolic_gather(geo, rng.uniform(0.1, 0.9 * T, n), rng.uniform(0.25, 0.65, n),
                             rng.uniform(10.0, 25.0, n), rng.standard_normal(n))


def batch_geometries(n: int, tag: int = 4) -> list[Geometry]:
    """Uneven batch: Nt~U{500..3000} (dt=4 ms), Nx~U{60..480} (dx=25 m),
    Nq=Nx, Ntau=Nt, q in [0.2,0.7] s/km."""
    rng = rng_for(tag)
    out = []
    for _ in range(n):
        Nt = int(rng.integers(500, 3001))
        Nx = int(rng.integers(60, 481))
        out.append(Geometry(Nt, Nx, Nt, Nx, 0.004, 0.025, 0.2, 0.7))
    return out


def irregular_geometry(Nt: int, Nx: int, Ntau: int, Nq: int, dt: float, X: float,
                       qmin: float, qmax: float, tag: int, jitter: float = 0.4,
                       near: float = 0.0, q_power: float = 1.0) -> Geometry:
    """Unequally spaced offsets and slownesses.

    Offsets: Nx regular nodes on [near, X], the inner ones moved by
    U(-jitter, jitter) of the node spacing (jitter < 1/2 keeps them strictly
    increasing; the end nodes stay). Slownesses: qmin + (qmax - qmin) u^q_power
    on a regular u grid in [0, 1] (denser towards qmin for q_power > 1).
    ``dx`` holds the mean offset spacing."""
    rng = rng_for(700 + tag)
    h = (X - near) / (Nx - 1)
    x = near + np.arange(Nx) * h
    x[1:-1] += rng.uniform(-jitter, jitter, Nx - 2) * h
    u = np.linspace(0.0, 1.0, Nq) if Nq > 1 else np.zeros(1)
    q = qmin + (qmax - qmin) * u ** q_power
    return Geometry(Nt, Nx, Ntau, Nq, dt, h, qmin, qmax, tuple(float(v) for v in x),
                    tuple(float(v) for v in q))
