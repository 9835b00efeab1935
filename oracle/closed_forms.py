"""Oracle (test infrastructure only): exact values of the hyperbolic Radon
transform, Eq. (1), for inputs where the integral has a closed form.

Only tests/, ``__graft_entry__.smoke()`` and bench.py's ``cpu_baseline`` leg
may import this module.
"""
from __future__ import annotations

import math
import numpy as np
from scipy.special import erf


def gaussian_tx(tau, q, a, b, T, X):
    """R_h f for f = exp(-a t^2 - b x^2) on [0,T]x[0,X], zero outside (Eq. (11)).

    From Eq. (3): 2 int_0^{x*} exp(-a (tau^2 + q^2 x^2) - b x^2) dx with
    x* = min(X, sqrt(T^2 - tau^2)/q) (the hyperbola leaves the rectangle at
    t = T), i.e. exp(-a tau^2) sqrt(pi/c) erf(sqrt(c) x*), c = a q^2 + b.
    """
    tau = np.asarray(tau, dtype=np.float64)[None, :]
    q = np.asarray(q, dtype=np.float64)[:, None]
    c = a * q * q + b
    with np.errstate(divide="ignore", invalid="ignore"):
        xs = np.where(q > 0, np.sqrt(np.maximum(T * T - tau * tau, 0.0)) / np.where(q > 0, q, 1.0), X)
    xs = np.minimum(xs, X)
    xs = np.where(tau <= T, xs, 0.0)
    return np.exp(-a * tau * tau) * np.sqrt(np.pi / c) * erf(np.sqrt(c) * xs)


def blob_sy_gather(t, x, T, X, c1, c2, w):
    """Gather whose folded, squared form (Eq. (2)) is a Gaussian blob in (s, y):

        f~(s, y) = exp(-((s - c1)^2 + (y - c2)^2) / w^2),  s = (t/T)^2, y = (x/X)^2,

    i.e. f(t, x) = 2 (x/X) f~((t/T)^2, (x/X)^2)  (the 1/(2 sqrt y) of Eq. (2)
    inverted, in the rescaled variables of Eq. (12)).
    """
    tb2 = (np.asarray(t)[None, :] / T) ** 2
    xb = np.asarray(x)[:, None] / X
    return 2.0 * xb * np.exp(-((tb2 - c1) ** 2 + (xb * xb - c2) ** 2) / (w * w))


def blob_sy_radon(tau, q, T, X, c1, c2, w):
    """Exact R_h of ``blob_sy_gather`` while the blob lies inside the unit
    square: Eq. (12) and (3) give R_h f(tau, q) = 2 X int f~(tb^2 + qb^2 y, y) dy
    with tb = tau/T, qb = qX/T, and the Gaussian line integral is
    sqrt(pi) w exp(-d^2/w^2) / sqrt(1 + qb^4), d the distance from (c1, c2)
    to the line s = tb^2 + qb^2 y."""
    tb2 = (np.asarray(tau, dtype=np.float64)[None, :] / T) ** 2
    qb2 = (np.asarray(q, dtype=np.float64)[:, None] * X / T) ** 2
    nrm = np.sqrt(1.0 + qb2 * qb2)
    d = (c1 - qb2 * c2 - tb2) / nrm
    return 2.0 * X * math.sqrt(math.pi) * w * np.exp(-(d * d) / (w * w)) / nrm


def event_on_slowness(tau, q0, X, h):
    """Invariant of Eq. (1): for f = h(t^2 - q0^2 x^2) and a hyperbola that stays
    inside the rectangle, R_h f(tau, q0) = 2 X h(tau^2)."""
    return 2.0 * X * h(np.asarray(tau, dtype=np.float64) ** 2)


def zeta_hat_dc(theta_m):
    """zeta_hat(0, 0) = int_{-theta_m}^{theta_m} sec = 2 ln(sec + tan)."""
    return 2.0 * math.log(1.0 / math.cos(theta_m) + math.tan(theta_m))
