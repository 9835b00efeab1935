"""Sparse Radon inversion, FP64, plain numpy (test infrastructure).

The paper's iteration (Section 3, equations (iters) and (itersmd), after
Daubechies, Defrise and De Mol 2004, Theorem 3.1) for

    min_g  || chi_S R_h* g - f ||_2^2 + mu || g ||_1

is   g^n = S_{c^2 mu}( g^{n-1} + c^2 R_h (f - chi_S R_h* g^{n-1}) ),
with the soft threshold S_mu(v) = v + mu/2 (v <= -mu/2), 0 (|v| < mu/2),
v - mu/2 (v >= mu/2) and c ||R_h|| < 1. The accelerated variant moves the
gradient step to the extrapolated point of Beck and Teboulle (FISTA):
y^n = g^n + ((t_{n-1} - 1)/t_n)(g^n - g^{n-1}), t_n = (1 + sqrt(1 + 4 t_{n-1}^2))/2,
t_0 = 1, y^0 = g^0.

The operators are passed in as callables: ``fwd`` is R_h (data -> image) and
``adj`` is R_h* (image -> data); the oracle's own ``LogPolar`` or ``direct``
transforms, or explicit matrices in the tests.
"""
from __future__ import annotations

import numpy as np


def soft_threshold(v, mu: float):
    """S_mu of Section 3: shrink towards zero by mu / 2, zero inside."""
    v = np.asarray(v, dtype=np.float64)
    out = np.zeros_like(v)
    out[v >= mu / 2] = v[v >= mu / 2] - mu / 2
    out[v <= -mu / 2] = v[v <= -mu / 2] + mu / 2
    return out


def objective(fwd, adj, f, g, mu: float, mask=None) -> float:
    """|| chi_S R_h* g - f ||^2 + mu ||g||_1 (the functional the iteration minimises)."""
    r = adj(g)
    if mask is not None:
        r = r * np.asarray(mask, dtype=np.float64)[:, None]
    return float(np.sum((r - f) ** 2) + mu * np.sum(np.abs(g)))


def ista(fwd, adj, f, mu: float, c2: float, iters: int, g0=None, mask=None, accelerate: bool = False):
    """``iters`` iterations of the paper's soft-thresholding iteration
    (missing-data form when ``mask`` [Nx] is given; f must then be zero on
    the missing traces), or of its accelerated form."""
    f = np.asarray(f, dtype=np.float64)
    m = None if mask is None else np.asarray(mask, dtype=np.float64)[:, None]
    g = np.zeros_like(fwd(np.zeros_like(f))) if g0 is None else np.array(g0, dtype=np.float64)
    y = g.copy()
    t = 1.0
    for _ in range(iters):
        a = adj(y)
        if m is not None:
            a = a * m
        g_new = soft_threshold(y + c2 * fwd(f - a), c2 * mu)
        if accelerate:
            tn = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
            y = g_new + ((t - 1.0) / tn) * (g_new - g)
            t = tn
        else:
            y = g_new
        g = g_new
    return g


def power_norm2(fwd, adj, v0, iters: int) -> float:
    """||R_h R_h* v|| after ``iters`` normalised power steps from v0: the
    estimate of ||R_h||^2 (largest eigenvalue of R_h R_h*)."""
    v = np.asarray(v0, dtype=np.float64)
    v = v / np.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        z = fwd(adj(v))
        lam = float(np.linalg.norm(z))
        v = z / lam
    return lam


def mute(g, tau, q, q0: float, slope: float, keep: str = "below"):
    """The Radon-domain mute of the multiple attenuation (Section 6): zero
    the outputs (tau_i, q_l) of g[l][i] above the line q = q0 + slope * tau
    (keep="below": the primaries) or on or below it (keep="above": the
    multiples)."""
    g = np.array(g, dtype=np.float64)
    above = np.asarray(q, dtype=np.float64)[:, None] > q0 + slope * np.asarray(tau, dtype=np.float64)[None, :]
    g[above if keep == "below" else ~above] = 0.0
    return g


def demultiple(fwd, adj, f, tau, q, q0: float, slope: float, iters: int, c2: float, mu: float,
               accelerate: bool = False):
    """Multiple attenuation as the paper describes it: sparse Radon image by
    the soft-thresholding iteration, the multiples' part of it (beyond the
    border line) taken back to (t, x) and subtracted from the gather.
    Returns (f - multiples, sparse image)."""
    g = ista(fwd, adj, f, mu, c2, iters, accelerate=accelerate)
    return np.asarray(f, dtype=np.float64) - adj(mute(g, tau, q, q0, slope, keep="above")), g
