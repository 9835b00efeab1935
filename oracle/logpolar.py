"""Oracle (test infrastructure only): FP64 log-polar hyperbolic Radon transform.

Only tests/, ``__graft_entry__.smoke()`` and bench.py's ``cpu_baseline`` leg
may import this module. It shares no code with the CUDA library.

It carries out the paper's method step by step, in the paper's order and
notation, in plain numpy float64 (numpy's FFT is the only library step):

1. Rescaling to the unit rectangle, Eq. (12)-(13): ``tb = t/T``,
   ``xb = x/X``, ``taub = tau/T``, ``qb = q X / T``.
2. Fold and squaring ``(s, y) = (tb^2, xb^2)`` with the ``1/(2 sqrt y)``
   weight, Eq. (2)-(3); the integral becomes a straight-line Radon
   transform, Eq. (4).
3. Splitting of the time integral, Eq. (19), and of the slowness range
   (Section 5): each (t-piece, q-piece) is an independent sub-problem; a
   slowness piece gets its own map T, a time piece its own lattice.
4. Per sub-problem: ``beta``, ``alpha`` (Section 2.1), square side ``a``
   and centre ``O`` (Section 2.1, the displayed formulas after Eq. (7); the
   first component of O is read as derived from the corner conditions, see
   ``square_in_sector``), the map T of Eq. (8), the log-polar coordinates
   P1 of Eq. (10), the mute triangle ``s < k^2 y`` and the inner radius
   ``a_r`` (Section 2.1).
5. Log-polar sample spacing, Eq. (18).
6. Gridding with cubic B-splines, Eq. (14)-(15): every sample
   ``f(t_j, x_k)`` is smeared onto the log-polar lattice with weight
   ``f/(2x) e^eta J`` times the trapezoid weights, where the Jacobian
   ``J = 4 tb xb a^2 e^{-2 eta}`` cancels the ``1/(2x)``.
7. Convolution with ``zeta(theta, rho) = delta(cos theta - e^rho)``,
   Eq. (6)-(7), by zero-padded FFT, divided twice by the B-spline symbol
   and restricted to the frequency rectangle L, Eq. (14), (16)-(17).
8. Cubic B-spline interpolation at ``(phi, eta) = P2 S (tau^2, q^2)``,
   Eq. (9)-(10), (17), times the line-measure factor (see ``forward``).

The adjoint, Eq. (20), is the exact transpose of every discrete step, in
reverse order.

Readings where the paper is silent, garbled or inconsistent are stated at
each function.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Sequence

import numpy as np

# --------------------------------------------------------------------------
# Descriptor and partitions
# --------------------------------------------------------------------------


@dataclasses.dataclass(frozen=True)
class Desc:
    """Problem and method parameters (physical units).

    Output grid: ``tau_i = tau0 + i*dtau`` (``dtau`` defaults to
    ``(Nt-1) dt / (Ntau-1)``), ``q_l = qmin + l (qmax-qmin)/(Nq-1)``.
    ``sigma`` divides the spacing of Eq. (18); ``omega_c`` is the half-width
    of the frequency rectangle L in cycles per lattice cell; ``tsplits`` are
    the split points of Eq. (19) as fractions of T; ``n_qsplit`` is the
    number of slowness pieces.

    Unequally spaced grids (Section 4: the method carries over to them):
    ``x`` lists the Nx offsets (km, strictly increasing, x_0 >= 0; X is the
    largest) in place of ``k dx``, and ``q_values`` the Nq slownesses (s/km,
    strictly increasing, >= 0) in place of the regular q grid. Time and
    intercept time stay regular.

    ``order`` is the degree of the B-spline of the gridding, the
    deconvolution and the interpolation (Eq. (14)-(17)): 3 (cubic, the
    paper's) or 5 (quintic, the higher-order kernel Section 7 proposes);
    the lattice keeps (order + 1) / 2 guard cells per side.
    """
    Nt: int
    Nx: int
    Ntau: int
    Nq: int
    dt: float
    dx: float
    qmin: float
    qmax: float
    tau0: float = 0.0
    dtau: float = 0.0
    sigma: float = 2.0
    omega_c: float = 0.25
    tsplits: tuple = ()
    n_qsplit: int = 1
    x: tuple | None = None
    q_values: tuple | None = None
    order: int = 3

    def __post_init__(self):
        if self.order not in (3, 5):
            raise ValueError("order: the B-spline degree, 3 (cubic) or 5 (quintic)")
        if self.x is not None:
            x = np.asarray(self.x, dtype=np.float64)
            if x.shape != (self.Nx,) or self.Nx < 2 or x[0] < 0 or not np.all(np.diff(x) > 0):
                raise ValueError("x: need Nx strictly increasing offsets >= 0")
        if self.q_values is not None:
            q = np.asarray(self.q_values, dtype=np.float64)
            if q.shape != (self.Nq,) or q[0] < 0 or not np.all(np.diff(q) > 0):
                raise ValueError("q_values: need Nq strictly increasing slownesses >= 0")

    @property
    def T(self):
        return (self.Nt - 1) * self.dt

    @property
    def X(self):
        if self.x is not None:
            return float(self.x[-1])
        return (self.Nx - 1) * self.dx

    def xb(self):
        """Rescaled offsets x_k / X of Eq. (12)."""
        if self.x is None:
            return np.arange(self.Nx) / (self.Nx - 1)
        return np.asarray(self.x, dtype=np.float64) / self.X

    def xb_spacing(self):
        """Rescaled offsets the lattice spacing of Eq. (18) is taken over:
        the offsets themselves on a regular grid; on given offsets, equally
        spaced ones over the same range [x_0, X]. Reading (Section 4 only
        treats regular sampling): the gridding treats the samples as a
        quadrature, so the lattice has to resolve the band of the data, which
        the mean spacing sets; the largest gap would coarsen the lattice and
        raise the error tenfold at 40 % jitter."""
        if self.x is None:
            return self.xb()
        x0 = float(self.x[0])
        return (x0 + np.arange(self.Nx) * ((self.X - x0) / (self.Nx - 1))) / self.X

    def x_weights(self):
        """Trapezoid weights of the offsets in units of the mean rescaled
        spacing 1/(Nx-1): 1/2 at the ends and 1 inside on a regular grid;
        (xb_{k+1} - xb_{k-1}) / 2 times (Nx-1) inside and the half gaps at the
        ends on given offsets."""
        n_x = self.Nx - 1
        if self.x is None:
            k = np.arange(self.Nx)
            return np.where((k == 0) | (k == n_x), 0.5, 1.0)
        xb = self.xb()
        w = np.empty(self.Nx)
        w[0] = 0.5 * (xb[1] - xb[0])
        w[-1] = 0.5 * (xb[-1] - xb[-2])
        w[1:-1] = 0.5 * (xb[2:] - xb[:-2])
        return w * n_x

    @property
    def dtau_eff(self):
        return self.dtau if self.dtau > 0 else self.T / (self.Ntau - 1)

    def tau(self):
        return self.tau0 + np.arange(self.Ntau) * self.dtau_eff

    def q(self):
        if self.q_values is not None:
            return np.asarray(self.q_values, dtype=np.float64)
        if self.Nq == 1:
            return np.array([self.qmin], dtype=np.float64)
        return self.qmin + np.arange(self.Nq) * ((self.qmax - self.qmin) / (self.Nq - 1))


BETA_MIN = 1e-3  # smallest angular opening of a sub-problem (one-column pieces)
T_OVERLAP = 1.25  # half-width ratio of the time-partition transition bands


@dataclasses.dataclass
class Partition:
    tpiece: int
    jt_lo: int
    jt_hi: int
    l_lo: int
    l_hi: int
    s0: float
    s1: float
    m_lo: float
    m_hi: float
    alpha: float
    beta: float
    a: float
    O1: float
    O2: float
    c_min: float
    k2: float
    a_r: float
    r_max: float
    dphi_rule: float
    deta_rule: float
    n_theta: int
    n_rho: int
    dtheta: float
    drho: float
    theta0: float
    rho0: float
    Ntheta: int
    Nrho: int
    theta_m: float
    P_theta: int
    P_rho: int
    k1max: int
    k2max: int
    jfirst: np.ndarray  # per trace k: first gridded sample index (mute)
    order: int = 3      # B-spline degree (Desc.order)


def fft_size(n: int) -> int:
    """Smallest size >= n of the form 2^a, 3*2^a, 5*2^a (a >= 0) or 9*2^a
    (1 <= a <= 8). Reading: the paper fixes no FFT length beyond the padding
    the kernel window needs; any length at or above it gives the same linear
    convolution, and the frequency rectangle L is fixed in cycles per cell."""
    best = None
    p = 1
    while p < 2 * n + 2:
        for c in (p, 3 * p, 5 * p) + ((9 * p,) if 2 <= p <= 256 else ()):
            if c >= n and (best is None or c < best):
                best = c
        p *= 2
    return best


def t_window_edge(tb, b: float, r: float):
    """Rising edge of the time partition at split point b: 0 for tb <= b/r,
    1 for tb >= b r, raised cosine in log(tb) in between."""
    tb = np.asarray(tb, dtype=np.float64)
    with np.errstate(divide="ignore"):
        u = np.log(np.maximum(tb, 1e-300) / b) / math.log(r)
    u = np.clip(u, -1.0, 1.0)
    return 0.5 * (1.0 + np.sin(0.5 * math.pi * u))


def t_pieces(desc: Desc) -> list[tuple[int, int, int]]:
    """Time pieces of Eq. (19): (first sample, last sample, piece index).

    Reading: Eq. (19) cuts the time integral at t = a. A hard cut makes the
    data of each piece jump along the line s = a^2, which is nearly parallel
    to the integration lines s = tau^2 + q^2 y, and the band-limited B-spline
    representation cannot carry such a jump. The cut is therefore made with a
    smooth partition of unity: piece p carries the window
    psi_p = h_p - h_{p+1}, h_p the raised-cosine edge of ``t_window_edge``
    at split point b_p (h_0 = 1, h_n = 0), over [b_p / r, b_{p+1} r] with
    r = ``T_OVERLAP``. The windows sum to one, so the pieces add up to the
    whole integral exactly. Split points closer than the overlap band allows
    are dropped.
    """
    n = desc.Nt - 1
    r = T_OVERLAP
    bs = []
    for b in sorted(desc.tsplits):
        if not (0.0 < b < 1.0):
            continue
        if b * r >= 1.0:
            continue
        if bs and b / r < bs[-1] * r:
            continue
        bs.append(float(b))
    out = []
    edges = [None] + bs + [None]
    for p in range(len(edges) - 1):
        lo = 0 if edges[p] is None else int(math.ceil(edges[p] / r * n - 1e-9))
        hi = n if edges[p + 1] is None else int(math.floor(edges[p + 1] * r * n + 1e-9))
        out.append((lo, hi, p))
    return out


def t_window(desc: Desc, p: int, tb):
    """Window psi_p(tb) of time piece p (see ``t_pieces``)."""
    r = T_OVERLAP
    bs = []
    for b in sorted(desc.tsplits):
        if not (0.0 < b < 1.0) or b * r >= 1.0 or (bs and b / r < bs[-1] * r):
            continue
        bs.append(float(b))
    lo = np.ones_like(np.asarray(tb, dtype=np.float64)) if p == 0 else t_window_edge(tb, bs[p - 1], r)
    hi = np.zeros_like(lo) if p == len(bs) else t_window_edge(tb, bs[p], r)
    return lo - hi


def q_pieces(desc: Desc) -> list[tuple[int, int]]:
    """Column ranges of the slowness pieces (Section 5: slowness splitting).

    Reading: the angular range ``arctan(qb^2)`` is cut into ``n_qsplit``
    equal parts; a column belongs to the part its angle falls in; empty
    parts are dropped.
    """
    qb = desc.q() * desc.X / desc.T
    psi = np.arctan(qb * qb)
    n = max(1, int(desc.n_qsplit))
    if n == 1 or desc.Nq < 2:
        return [(0, desc.Nq - 1)]
    lo, hi = float(psi[0]), float(psi[-1])
    bounds = [lo + (hi - lo) * p / n for p in range(1, n)]
    piece = np.zeros(desc.Nq, dtype=np.int64)
    for bnd in bounds:
        piece += (psi >= bnd).astype(np.int64)
    out = []
    for p in range(n):
        idx = np.nonzero(piece == p)[0]
        if idx.size:
            out.append((int(idx[0]), int(idx[-1])))
    return out


def square_in_sector(alpha: float, beta: float) -> tuple[float, float, float]:
    """Side ``a`` and centre ``O`` of the square placed in the sector
    ``|angle| <= beta/2``, radius 1 (Section 2.1, after Eq. (7)).

    ``a`` is as printed. The printed ``O`` is garbled (``O = O(...)``, and
    its first component has ``tan(beta)``); the reading used here follows
    from the stated corner conditions: the corners (0,0) and (1,1) of the
    square lie on the two sector edges, which gives
    ``O1 = a sin(alpha+pi/4) / (sqrt 2 tan(beta/2))`` and
    ``O2 = a cos(alpha+pi/4) tan(beta/2) / sqrt 2`` (the second as printed).
    """
    s2a, sb, cb = math.sin(2 * alpha), math.sin(beta), math.cos(beta)
    a = sb / math.sqrt(s2a * sb + cb * (s2a + sb) + 1.0)
    th = math.tan(beta / 2)
    O1 = a * math.sin(alpha + math.pi / 4) / (math.sqrt(2.0) * th)
    O2 = a * math.cos(alpha + math.pi / 4) * th / math.sqrt(2.0)
    return a, O1, O2


def map_T(part: Partition, s, y):
    """Transformation T of Eq. (8): rotate by alpha, scale by a, shift by O."""
    ca, sa = math.cos(part.alpha), math.sin(part.alpha)
    ds, dy = np.asarray(s) - 0.5, np.asarray(y) - 0.5
    u1 = part.a * (ca * ds - sa * dy) + part.O1
    u2 = part.a * (sa * ds + ca * dy) + part.O2
    return u1, u2


def map_P1(u1, u2):
    """P1 of Eq. (10): angle phi and log-radius eta.

    Reading: the printed component order of P1 is (log r, angle); the names
    (phi, eta) of Eq. (14)-(15) are used as (angle, log-radius), which is
    the order the B-spline ``B3(theta - phi, rho - eta)`` needs.
    """
    return np.arctan2(u2, u1), 0.5 * np.log(u1 * u1 + u2 * u2)


def _clip_region(s0: float, s1: float, c: float, m: float) -> np.ndarray:
    """Vertices of {(s,y) in [s0,s1]x[0,1] : s >= c + m y} (convex polygon)."""
    rect = [(s0, 0.0), (s1, 0.0), (s1, 1.0), (s0, 1.0)]
    val = lambda p: p[0] - c - m * p[1]
    out = []
    for i in range(4):
        p, r = rect[i], rect[(i + 1) % 4]
        vp, vr = val(p), val(r)
        if vp >= 0:
            out.append(p)
        if (vp >= 0) != (vr >= 0):
            t = vp / (vp - vr)
            out.append((p[0] + t * (r[0] - p[0]), p[1] + t * (r[1] - p[1])))
    return np.array(out, dtype=np.float64)


def make_partition(desc: Desc, jt: tuple[int, int, int], lq: tuple[int, int]) -> Partition:
    """Geometry of one sub-problem, all in FP64.

    Reading of Eq. (19): the time pieces are not rescaled. Every piece of a
    slowness range shares that range's map T (alpha, beta, a, O); the piece
    only carries its own samples (through its window) and its own lattice,
    whose spacing follows Eq. (18) over the piece's samples ("samples in
    theta, rho ... become more dense" for small t) and whose rho-range spans
    the piece's data region.
    """
    n_t, n_x = desc.Nt - 1, desc.Nx - 1
    T, X = desc.T, desc.X
    j0, j1, tp = jt
    l0, l1 = lq
    s0 = (j0 / n_t) ** 2
    s1 = (j1 / n_t) ** 2
    qb = desc.q() * X / T
    m_lo = float(qb[l0] ** 2)
    m_hi = float(qb[l1] ** 2)
    psi_lo, psi_hi = math.atan(m_lo), math.atan(m_hi)
    # beta and alpha of Section 2.1, with a floor on beta for one-column pieces
    # (kept at psi_lo >= 0: the square lies inside the sector only then)
    if psi_hi - psi_lo < BETA_MIN:
        mid = max(0.5 * (psi_lo + psi_hi), 0.5 * BETA_MIN)
        psi_lo, psi_hi = mid - 0.5 * BETA_MIN, mid + 0.5 * BETA_MIN
    beta = psi_hi - psi_lo
    alpha = 0.5 * (psi_hi + psi_lo)
    a, O1, O2 = square_in_sector(alpha, beta)

    # Mute (Section 2.1): no output line (tau >= tau_min, q >= q_min) reaches
    # s < c_min + k^2 y with c_min = taub_min^2 and k = the smallest slowness of
    # the whole problem, so that triangle is left out. Reading: k is the
    # global q_min in every slowness piece, not the piece's own lower end;
    # cutting a piece's data along its own lowest-slowness line would make the
    # data jump along lines parallel to that piece's integration lines.
    taub_min = desc.tau0 / T
    c_min = taub_min * taub_min
    k2 = float(qb[0] ** 2)
    xb2 = desc.xb() ** 2
    tb2 = (np.arange(j0, j1 + 1) / n_t) ** 2
    jfirst = np.empty(desc.Nx, dtype=np.int64)
    for k in range(desc.Nx):
        ok = np.nonzero(tb2 >= c_min + k2 * xb2[k])[0]
        jfirst[k] = j0 + int(ok[0]) if ok.size else j1 + 1

    part = Partition(tp, j0, j1, l0, l1, s0, s1, m_lo, m_hi, alpha, beta, a, O1, O2,
                     c_min, k2, 0.0, 0.0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, jfirst, desc.order)
    # Data region of the piece: [s0, s1] x [0, 1] minus the muted triangle.
    poly = _clip_region(s0, s1, c_min, k2)
    u1, u2 = map_T(part, poly[:, 0], poly[:, 1])
    # Inner radius a_r (Section 2.1): smallest distance from the origin of a
    # line with normal angle in [-beta/2, beta/2] meeting the data region
    # (linear in u, so attained at a vertex and an extreme angle); the outer
    # radius is the largest |u| over the region (at most 1).
    part.a_r = min(float(np.min(u1 * math.cos(th) + u2 * math.sin(th)))
                   for th in (-beta / 2, beta / 2))
    part.r_max = float(np.max(np.sqrt(u1 * u1 + u2 * u2)))

    # Sample spacing of Eq. (18), over all samples of the time piece (on
    # given offsets: over equally spaced offsets of the same range).
    U1, U2 = map_T(part, tb2[None, :], (desc.xb_spacing() ** 2)[:, None])
    phi, eta = map_P1(U1, U2)
    dphi = max(float(np.max(np.abs(np.diff(phi, axis=1)))) if phi.shape[1] > 1 else 0.0,
               float(np.max(np.abs(np.diff(phi, axis=0)))) if phi.shape[0] > 1 else 0.0)
    deta = max(float(np.max(np.abs(np.diff(eta, axis=1)))) if eta.shape[1] > 1 else 0.0,
               float(np.max(np.abs(np.diff(eta, axis=0)))) if eta.shape[0] > 1 else 0.0)
    part.dphi_rule, part.deta_rule = dphi, deta

    # Lattice: spacing of Eq. (18) divided by sigma, (order + 1) / 2 guard
    # cells per side (the taps of a position reach that far beyond it), over
    # [-beta/2, beta/2] x [log a_r, log r_max].
    n_theta = max(1, int(math.ceil(desc.sigma * beta / dphi - 1e-9)))
    L_rho = math.log(part.r_max) - math.log(part.a_r)
    n_rho = max(1, int(math.ceil(desc.sigma * L_rho / deta - 1e-9)))
    dtheta = beta / n_theta
    drho = L_rho / n_rho
    part.n_theta, part.n_rho = n_theta, n_rho
    part.dtheta, part.drho = dtheta, drho
    g = guard_cells(desc.order)
    part.theta0 = -beta / 2 - g * dtheta
    part.rho0 = math.log(part.a_r) - g * drho
    part.Ntheta, part.Nrho = n_theta + 2 * g + 1, n_rho + 2 * g + 1

    # Kernel window and zero padding (Section 2.1, after Eq. (7)): the
    # convolution only ever pairs lattice points whose theta-difference is at
    # most the lattice width and whose rho-difference is at least -(Nrho-1) drho.
    theta_m = min((part.Ntheta - 1) * dtheta,
                  math.acos(math.exp(-(part.Nrho - 1) * drho)))
    part.theta_m = theta_m
    Ka = int(math.ceil(theta_m / dtheta - 1e-9))
    Kr = int(math.ceil(-math.log(math.cos(theta_m)) / drho - 1e-9))
    part.P_theta = fft_size(part.Ntheta + Ka)
    part.P_rho = fft_size(part.Nrho + Kr)
    part.k1max = min(int(math.floor(desc.omega_c * part.P_theta)), part.P_theta // 2 - 1)
    part.k2max = min(int(math.floor(desc.omega_c * part.P_rho)), part.P_rho // 2 - 1)
    return part


def plan(desc: Desc) -> list[Partition]:
    """All sub-problems, t-pieces outer, q-pieces inner."""
    if desc.Nt < 2 or desc.Nx < 2 or desc.Ntau < 2 or desc.Nq < 1:
        raise ValueError("need Nt, Nx, Ntau >= 2 and Nq >= 1")
    return [make_partition(desc, jt, lq) for jt in t_pieces(desc) for lq in q_pieces(desc)]


# --------------------------------------------------------------------------
# B-splines and the kernel spectrum
# --------------------------------------------------------------------------


def b3(x):
    """Centred cubic cardinal B-spline, support (-2, 2)."""
    ax = np.abs(x)
    return np.where(ax < 1.0, 2.0 / 3.0 - ax * ax + 0.5 * ax ** 3,
                    np.where(ax < 2.0, (2.0 - ax) ** 3 / 6.0, 0.0))


def b3_hat(w):
    """Fourier transform of B3 at frequency w (cycles per cell): sinc^4."""
    return np.sinc(w) ** 4


def b5(x):
    """Centred quintic cardinal B-spline, support (-3, 3), from its
    definition as the 6-fold convolution of the unit box: the truncated
    powers (3-|x|)^5 - 6 (2-|x|)^5 + 15 (1-|x|)^5, each term only where its
    base is positive, over 5! = 120."""
    ax = np.abs(np.asarray(x, dtype=np.float64))
    tp = lambda u: np.where(u > 0.0, u, 0.0) ** 5
    return (tp(3.0 - ax) - 6.0 * tp(2.0 - ax) + 15.0 * tp(1.0 - ax)) / 120.0


def bspline(order: int, x):
    """The centred cardinal B-spline of degree 3 or 5."""
    return b3(x) if order == 3 else b5(x)


def bspline_hat(order: int, w):
    """Its Fourier transform at frequency w (cycles per cell): sinc^(order+1)."""
    return np.sinc(w) ** (order + 1)


def guard_cells(order: int) -> int:
    """Guard cells per lattice side: (order + 1) / 2, the reach of the taps."""
    return (order + 1) // 2


def gl_nodes(theta_m: float, cycles: float, nodes_per_panel: int = 20, extra_panels: int = 4):
    """Composite Gauss-Legendre rule on [0, theta_m] with at least one panel
    per oscillation of the integrand."""
    x, wq = np.polynomial.legendre.leggauss(nodes_per_panel)
    npan = int(math.ceil(cycles)) + extra_panels
    edges = np.linspace(0.0, theta_m, npan + 1)
    h = 0.5 * (edges[1:] - edges[:-1])
    c = 0.5 * (edges[1:] + edges[:-1])
    th = (c[:, None] + h[:, None] * x[None, :]).ravel()
    wt = (h[:, None] * wq[None, :]).ravel()
    return th, wt


def zeta_hat(theta_m: float, w1, w2):
    """Continuous Fourier transform of zeta(theta, rho) = delta(cos theta - e^rho)
    truncated to |theta| <= theta_m (Section 2.1, Eq. (6)-(7)):

        zeta_hat(w1, w2) = int_{-theta_m}^{theta_m}
                           exp(-2 pi i (theta w1 + w2 log cos theta)) / cos theta  d theta

    (the rho-integral of the delta contributes 1/cos theta at rho = log cos theta).
    The integrand is even in theta, so the integral is twice the one over
    [0, theta_m] with cos(2 pi theta w1); it is evaluated for every (w1, w2)
    pair of the given vectors with one composite Gauss-Legendre rule, written
    as a matrix product: cos(2 pi theta_n w1)^T  @  (wt_n e^{-2 pi i w2 log cos theta_n} / cos theta_n).
    Returns an array [len(w1)][len(w2)].
    """
    w1 = np.atleast_1d(np.asarray(w1, dtype=np.float64))
    w2 = np.atleast_1d(np.asarray(w2, dtype=np.float64))
    cycles = (float(np.max(np.abs(w1))) * theta_m
              + float(np.max(np.abs(w2))) * abs(math.log(math.cos(theta_m))))
    th, wt = gl_nodes(theta_m, cycles)
    ct = np.cos(th)
    lc = np.log(ct)
    A = np.cos(2 * np.pi * np.outer(w1, th))             # [k1][n]
    out = np.empty((w1.size, w2.size), dtype=np.complex128)
    step = max(1, int(2e7 // max(th.size, 1)))
    for c0 in range(0, w2.size, step):
        ww = w2[c0:c0 + step]
        B = (wt / ct)[:, None] * np.exp(-2j * np.pi * np.outer(lc, ww))  # [n][k2]
        out[:, c0:c0 + step] = 2.0 * (A @ B.real + 1j * (A @ B.imag))
    return out


def kernel_spectrum(part: Partition) -> np.ndarray:
    """K = chi_L * zeta_hat / (B_hat_theta B_hat_rho)^2 on the rfft2 grid
    [P_theta][P_rho//2 + 1] (Eq. (14), (16)-(17)).

    Reading: ``F B3`` is the continuous transform sinc^4 of the B-spline in
    cell units (the USFFT convention the paper cites; sinc^6 for the quintic
    B-spline of ``Desc.order`` = 5); L is the rectangle
    |k1|/P_theta <= omega_c, k2/P_rho <= omega_c; the Nyquist bins are always
    outside L.
    """
    Pt, Pr = part.P_theta, part.P_rho
    K = np.zeros((Pt, Pr // 2 + 1), dtype=np.complex128)
    k1 = np.arange(0, part.k1max + 1)
    k2 = np.arange(0, part.k2max + 1)
    z = zeta_hat(part.theta_m, k1 / (Pt * part.dtheta), k2 / (Pr * part.drho))
    den = (bspline_hat(part.order, k1 / Pt)[:, None] * bspline_hat(part.order, k2 / Pr)[None, :]) ** 2
    Kh = z / den
    K[:part.k1max + 1, :part.k2max + 1] = Kh
    K[Pt - part.k1max:, :part.k2max + 1] = Kh[:0:-1]  # even in k1
    return K


def kernel_half(part: Partition) -> np.ndarray:
    """The stored half of K: rows k1 = 0..k1max, columns k2 = 0..k2max."""
    K = kernel_spectrum(part)
    return K[:part.k1max + 1, :part.k2max + 1]


# --------------------------------------------------------------------------
# Coordinates and weights
# --------------------------------------------------------------------------


def data_points(desc: Desc, part: Partition):
    """Gridded samples of one sub-problem: indices, lattice positions and weights.

    Weight of sample (j, k) (Eq. (14)-(15), trapezoid in x, rectangle in t):

        W = f(t_j, x_k) * 2 a^2 tb_j e^{-eta} * psi_p(tb_j) * w_k * dtb * dxb

    which is f/(2 xb) * e^eta * J * dtb dxb / S with J = 4 tb xb a^2 e^{-2 eta}
    (the xb cancels, as the paper notes after Eq. (14)); psi_p is the window
    of the time piece.
    Reading: rectangle weights in t (matching the interpolating cubic in t of
    the reference direct sum) and trapezoid weights in x (end traces 1/2; on
    given offsets, the trapezoid weights of those offsets, Desc.x_weights).
    """
    n_t, n_x = desc.Nt - 1, desc.Nx - 1
    jj, kk = [], []
    for k in range(desc.Nx):
        j = np.arange(part.jfirst[k], part.jt_hi + 1)
        jj.append(j)
        kk.append(np.full(j.size, k))
    jj = np.concatenate(jj) if jj else np.zeros(0, np.int64)
    kk = np.concatenate(kk) if kk else np.zeros(0, np.int64)
    tb = jj / n_t
    xb = desc.xb()[kk]
    u1, u2 = map_T(part, tb * tb, xb * xb)
    phi, eta = map_P1(u1, u2)
    wk = desc.x_weights()[kk]
    wt = t_window(desc, part.tpiece, tb)
    wfac = 2.0 * part.a ** 2 * tb * wt * np.exp(-eta) * wk / (n_t * n_x)
    xth = (phi - part.theta0) / part.dtheta
    xrh = (eta - part.rho0) / part.drho
    return jj, kk, xth, xrh, wfac


def radon_points(desc: Desc, part: Partition):
    """Outputs of one sub-problem: (column, row) indices, lattice positions,
    validity and output scale.

    Line of output (tau, q) in (s, y): s = c + m y with c = taub^2 and
    m = qb^2. Its normal angle is theta = alpha - psi,
    psi = arctan m (Section 2.1), and its distance from the origin after T is

        e^rho = a cos(psi) (c - 1/2 + m/2) + O1 cos theta + O2 sin theta,

    which is P2 S(tau^2, q^2) of Eq. (9)-(10). Reading: the angle of P2 is
    taken as +theta (the printed minus sign applies to the unrotated frame),
    and rho is the log of S's first component times cos theta.

    Output scale (Eq. (17) 'up to a scaling factor'): the line integral in
    the u-plane equals a * sqrt(1 + m^2) times the delta-integral of Eq. (4)
    in (s, y), and Eq. (12) contributes the factor X of the rescaling and the
    2 of the fold, so R_h f = 2 X cos(psi) / a * (line integral in u).
    Lines with e^rho outside [a_r, r_max] miss the piece's data region and
    give zero.
    """
    T, X = desc.T, desc.X
    taub = desc.tau() / T
    qb = desc.q()[part.l_lo:part.l_hi + 1] * X / T
    ll = np.repeat(np.arange(part.l_lo, part.l_hi + 1), desc.Ntau)
    ii = np.tile(np.arange(desc.Ntau), part.l_hi - part.l_lo + 1)
    m = np.repeat(qb * qb, desc.Ntau)
    c = np.tile(taub * taub, qb.size)
    psi = np.arctan(m)
    theta = part.alpha - psi
    e = (part.a * np.cos(psi) * (c - 0.5 + 0.5 * m)
         + part.O1 * np.cos(theta) + part.O2 * np.sin(theta))
    valid = (e >= part.a_r) & (e <= part.r_max)
    rho = np.log(np.where(valid, e, 1.0))
    xth = (theta - part.theta0) / part.dtheta
    xrh = (rho - part.rho0) / part.drho
    scale = 2.0 * X * np.cos(psi) / part.a
    return ll, ii, xth, xrh, valid, scale


# --------------------------------------------------------------------------
# The discrete steps and their transposes
# --------------------------------------------------------------------------


def _taps(x, order: int = 3):
    """The order + 1 lattice points whose B-spline reaches position x: first
    tap floor(x) - (order - 1) / 2, and each tap's weight."""
    i0 = np.floor(x).astype(np.int64) - (order - 1) // 2
    return i0, [bspline(order, x - i0 - d) for d in range(order + 1)]


def grid_fwd(part: Partition, xth, xrh, w) -> np.ndarray:
    """Smearing, Eq. (15): G[m][n] = sum_s W_s B(.)B(.) / (dtheta drho)."""
    G = np.zeros((part.Ntheta, part.Nrho))
    m0, wt = _taps(xth, part.order)
    n0, wr = _taps(xrh, part.order)
    sc = w / (part.dtheta * part.drho)
    for a in range(part.order + 1):
        for b in range(part.order + 1):
            np.add.at(G, (m0 + a, n0 + b), sc * wt[a] * wr[b])
    return G


def grid_adj(part: Partition, G, xth, xrh) -> np.ndarray:
    """Transpose of ``grid_fwd`` (per-sample sums; weights applied by caller)."""
    m0, wt = _taps(xth, part.order)
    n0, wr = _taps(xrh, part.order)
    acc = np.zeros(xth.shape)
    for a in range(part.order + 1):
        for b in range(part.order + 1):
            acc += G[m0 + a, n0 + b] * wt[a] * wr[b]
    return acc / (part.dtheta * part.drho)


def conv(part: Partition, G, K, adjoint=False) -> np.ndarray:
    """Finite convolution of Eq. (7) by zero-padded FFT (Eq. (16)-(17)):
    Q = IFFT2(FFT2(G) K) on the lattice; the transpose uses conj(K)."""
    pad = np.zeros((part.P_theta, part.P_rho))
    pad[:part.Ntheta, :part.Nrho] = G
    spec = np.fft.rfft2(pad)
    spec *= np.conj(K) if adjoint else K
    out = np.fft.irfft2(spec, s=(part.P_theta, part.P_rho))
    return out[:part.Ntheta, :part.Nrho]


def interp_fwd(part: Partition, Q, xth, xrh, valid, scale) -> np.ndarray:
    """B-spline interpolation of Eq. (17) at the output coordinates (lines
    that miss the piece take a dummy in-range position and give 0)."""
    g = guard_cells(part.order)
    m0, wt = _taps(xth, part.order)
    xr = np.where(valid, xrh, float(g))
    n0, wr = _taps(xr, part.order)
    acc = np.zeros(xth.shape)
    for a in range(part.order + 1):
        for b in range(part.order + 1):
            acc += Q[m0 + a, n0 + b] * wt[a] * wr[b]
    return np.where(valid, scale * acc, 0.0)


def interp_adj(part: Partition, vals, xth, xrh, valid, scale) -> np.ndarray:
    """Transpose of ``interp_fwd``."""
    Q = np.zeros((part.Ntheta, part.Nrho))
    g = guard_cells(part.order)
    m0, wt = _taps(xth, part.order)
    xr = np.where(valid, xrh, float(g))
    n0, wr = _taps(xr, part.order)
    v = np.where(valid, scale * vals, 0.0)
    for a in range(part.order + 1):
        for b in range(part.order + 1):
            np.add.at(Q, (m0 + a, n0 + b), v * wt[a] * wr[b])
    return Q


class LogPolar:
    """FP64 log-polar hyperbolic Radon operator pair for one descriptor."""

    def __init__(self, desc: Desc):
        self.desc = desc
        self.parts = plan(desc)
        self.K = [kernel_spectrum(p) for p in self.parts]
        self.dpts = [data_points(desc, p) for p in self.parts]
        self.rpts = [radon_points(desc, p) for p in self.parts]

    def forward(self, f) -> np.ndarray:
        """``f[Nx][Nt]`` -> ``g[Nq][Ntau]`` (Eq. (6)-(17)); t-pieces add."""
        d = self.desc
        f = np.asarray(f, dtype=np.float64)
        g = np.zeros((d.Nq, d.Ntau))
        for part, K, (jj, kk, xth, xrh, wfac), (ll, ii, yth, yrh, valid, scale) in zip(
                self.parts, self.K, self.dpts, self.rpts):
            G = grid_fwd(part, xth, xrh, f[kk, jj] * wfac)
            Q = conv(part, G, K)
            np.add.at(g, (ll, ii), interp_fwd(part, Q, yth, yrh, valid, scale))
        return g

    def adjoint(self, g) -> np.ndarray:
        """``g[Nq][Ntau]`` -> ``f[Nx][Nt]``: transpose of ``forward`` (Eq. (20))."""
        d = self.desc
        g = np.asarray(g, dtype=np.float64)
        f = np.zeros((d.Nx, d.Nt))
        for part, K, (jj, kk, xth, xrh, wfac), (ll, ii, yth, yrh, valid, scale) in zip(
                self.parts, self.K, self.dpts, self.rpts):
            Q = interp_adj(part, g[ll, ii], yth, yrh, valid, scale)
            G = conv(part, Q, K, adjoint=True)
            np.add.at(f, (kk, jj), wfac * grid_adj(part, G, xth, xrh))
        return f

    # -- intermediate stages, for stage-by-stage comparisons ---------------
    def stages_forward(self, f, p: int = 0):
        part, K = self.parts[p], self.K[p]
        jj, kk, xth, xrh, wfac = self.dpts[p]
        G = grid_fwd(part, xth, xrh, np.asarray(f, np.float64)[kk, jj] * wfac)
        Q = conv(part, G, K)
        return G, Q

    def info(self) -> list[dict]:
        out = []
        for p in self.parts:
            dct = {k: getattr(p, k) for k in Partition.__dataclass_fields__ if k != "jfirst"}
            out.append(dct)
        return out
