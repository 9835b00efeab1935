"""hradon: fast hyperbolic Radon transform (log-polar method) on sm_103a.

Thin Python binding of the C ABI in ``include/hradon.h``. Every step of the
transform runs in the library's CUDA kernels; PyTorch only provides device
memory, streams and autograd. There is no CPU fallback: without a CUDA device
or without the built library every call raises.

    plan = Plan(Nt, Nx, Ntau, Nq, dt, dx, qmin, qmax)      # geometry, kernel spectra
    g = plan.forward(f)        # f: cuda float32 [Nx][Nt]  ->  g: [Nq][Ntau]
    f2 = plan.adjoint(g)       # exact transpose (Eq. (16))
    g = radon(f, plan)         # autograd op: backward is the adjoint
    g = plan.ista(f, mu, mask=m)   # sparse inversion / trace interpolation (FISTA)
"""
from __future__ import annotations

import ctypes
from typing import Sequence

import numpy as np
import torch

from . import _lib
from ._lib import RadonError, RadonDesc, RadonPieceInfo

__all__ = ["Plan", "Batch", "radon", "radon_adjoint", "radon_adj", "direct_forward", "direct_adjoint", "RadonError",
           "HRadon", "default_method"]


def _stream_ptr(device: torch.device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _check_tensor(t: torch.Tensor, shape, name: str, device: torch.device):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.device != device or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float32 tensor on {device}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


def default_method() -> dict:
    """The library's default method parameters (``radon_desc_init``; host
    only, no device needed): ``sigma``, ``omega_c`` and the time splits
    ``tsplit`` (fractions of T)."""
    lib = _lib.load()
    d = RadonDesc()
    _lib.check(lib.radon_desc_init(ctypes.byref(d), 2, 2, 2, 1, 1.0, 1.0, 0.0, 1.0))
    return {"sigma": d.sigma, "omega_c": d.omega_c, "tsplit": tuple(d.tsplit[i] for i in range(d.n_tsplit))}


class Plan:
    """Plan of the log-polar hyperbolic Radon transform for one geometry.

    Parameters mirror ``radon_desc``: gather ``Nt`` x ``Nx`` samples at
    ``dt``, ``dx``; image ``Ntau`` x ``Nq`` with ``tau_i = tau0 + i*dtau``
    (``dtau=0``: ``(Nt-1) dt/(Ntau-1)``) and ``q`` evenly on
    ``[qmin, qmax]``; method parameters ``sigma``, ``omega_c``, ``tsplit``
    (split points of Eq. (19) as fractions of T), ``n_qsplit``;
    ``rows_per_band`` (1..6, or 0 to time them at plan creation; the plan's
    ``desc.rows_per_band`` reports the value in use); ``spline_order`` 3
    (cubic B-splines, the default) or 5 (quintic). Unequally spaced grids
    (``radon_plan_create_grid``): ``x`` gives the Nx offsets (km) in place of
    ``k*dx``, ``q`` the Nq slownesses (s/km) in place of the regular grid.
    """

    def __init__(self, Nt: int, Nx: int, Ntau: int, Nq: int, dt: float, dx: float,
                 qmin: float = 0.0, qmax: float = 1.0, *, tau0: float = 0.0, dtau: float = 0.0,
                 sigma: float | None = None, omega_c: float | None = None,
                 tsplit: Sequence[float] | None = None, n_qsplit: int = 1,
                 rows_per_band: int | None = None, device: int | torch.device | None = None,
                 x: Sequence[float] | None = None, q: Sequence[float] | None = None,
                 spline_order: int | None = None):
        lib = _lib.load()
        d = RadonDesc()
        _lib.check(lib.radon_desc_init(ctypes.byref(d), Nt, Nx, Ntau, Nq, dt, dx, qmin, qmax))
        d.tau0, d.dtau, d.n_qsplit = tau0, dtau, n_qsplit
        if sigma is not None:
            d.sigma = sigma
        if omega_c is not None:
            d.omega_c = omega_c
        if tsplit is not None:
            ts = list(tsplit)
            if len(ts) > _lib.MAX_TSPLIT:
                raise ValueError(f"at most {_lib.MAX_TSPLIT} time splits")
            d.n_tsplit = len(ts)
            for i, v in enumerate(ts):
                d.tsplit[i] = v
        if rows_per_band is not None:
            d.rows_per_band = rows_per_band
        if spline_order is not None:
            d.spline_order = spline_order
        if device is None:
            dev = torch.cuda.current_device()
        else:
            dev = torch.device(device).index if not isinstance(device, int) else device
            dev = 0 if dev is None else dev
        d.device = dev
        self.device = torch.device("cuda", dev)
        self._handle = ctypes.c_void_p()
        xa, qa = _grid_array(x, Nx, "x"), _grid_array(q, Nq, "q")
        _lib.check(lib.radon_plan_create_grid(ctypes.byref(self._handle), ctypes.byref(d), xa, qa))
        out = RadonDesc()
        _lib.check(lib.radon_plan_desc(self._handle, ctypes.byref(out)))
        self.desc = out
        self.Nt, self.Nx, self.Ntau, self.Nq = Nt, Nx, Ntau, Nq

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_handle", None) is not None and self._handle.value:
            _lib.load().radon_plan_destroy(self._handle)
            self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- info ---------------------------------------------------------------
    def pieces(self) -> list[dict]:
        lib = _lib.load()
        n = ctypes.c_int()
        _lib.check(lib.radon_plan_num_pieces(self._handle, ctypes.byref(n)))
        out = []
        for p in range(n.value):
            info = RadonPieceInfo()
            _lib.check(lib.radon_plan_piece_info(self._handle, p, ctypes.byref(info)))
            out.append({name: getattr(info, name) for name, _ in RadonPieceInfo._fields_})
        return out

    def piece_lattice(self, piece: int) -> np.ndarray:
        """Lattice [Ntheta][Nrho] of sub-problem `piece` as the last forward
        (convolved lattice) or adjoint (lattice the adjoint gridding reads)
        left it; synchronises the device (``radon_plan_piece_lattice``)."""
        info = self.pieces()[piece]
        out = np.empty((info["Ntheta"], info["Nrho"]), np.float32)
        _lib.check(_lib.load().radon_plan_piece_lattice(self._handle, piece, out.ctypes.data, out.size))
        return out

    def piece_samples(self, piece: int) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
        """Lattice positions (theta, rho, in cells) and gridding weights of the
        gather samples of sub-problem `piece`, each [Nx][jt_hi - jt_lo + 1];
        weight 0 marks a sample the piece does not grid
        (``radon_plan_piece_samples``)."""
        info = self.pieces()[piece]
        shape = (self.desc.Nx, info["jt_hi"] - info["jt_lo"] + 1)
        th, rh = np.empty(shape), np.empty(shape)
        w = np.empty(shape, np.float32)
        _lib.check(_lib.load().radon_plan_piece_samples(self._handle, piece, th.ctypes.data, rh.ctypes.data,
                                                        w.ctypes.data, w.size))
        return th, rh, w

    def device_bytes(self) -> int:
        v = ctypes.c_size_t()
        _lib.check(_lib.load().radon_plan_device_bytes(self._handle, ctypes.byref(v)))
        return v.value

    def set_profiling(self, enable: bool = True):
        _lib.check(_lib.load().radon_plan_set_profiling(self._handle, int(bool(enable))))

    def profile_read(self) -> dict:
        """Per-stage kernel time (ms), launches and algorithmic bytes since the
        last read (synchronises the recorded events)."""
        n = _lib.NSTAGES
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_longlong * n)()
        by = (ctypes.c_double * n)()
        _lib.check(_lib.load().radon_plan_profile_read(self._handle, ms, cnt, by))
        return {name: {"ms": ms[i], "launches": cnt[i], "bytes": by[i]}
                for i, name in enumerate(_lib.STAGE_NAMES)}

    # -- transforms ---------------------------------------------------------
    def forward(self, f: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """g = R_h f on the current stream. f: [Nx][Nt] float32 on the plan's device."""
        _check_tensor(f, (self.Nx, self.Nt), "f", self.device)
        if out is None:
            out = torch.empty((self.Nq, self.Ntau), dtype=torch.float32, device=self.device)
        _check_tensor(out, (self.Nq, self.Ntau), "out", self.device)
        _lib.check(_lib.load().radon_fwd(self._handle, ctypes.c_void_p(f.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), _stream_ptr(self.device)))
        return out

    def adjoint(self, g: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """f = R_h* g on the current stream. g: [Nq][Ntau] float32 on the plan's device."""
        _check_tensor(g, (self.Nq, self.Ntau), "g", self.device)
        if out is None:
            out = torch.empty((self.Nx, self.Nt), dtype=torch.float32, device=self.device)
        _check_tensor(out, (self.Nx, self.Nt), "out", self.device)
        _lib.check(_lib.load().radon_adj(self._handle, ctypes.c_void_p(g.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), _stream_ptr(self.device)))
        return out


    # -- sparse inversion (Section 3) ----------------------------------------
    def _work(self, fn_name: str) -> torch.Tensor:
        v = ctypes.c_size_t()
        _lib.check(getattr(_lib.load(), fn_name)(self._handle, ctypes.byref(v)))
        # torch's caching allocator returns blocks aligned to at least 512 bytes
        return torch.empty(max(1, v.value), dtype=torch.uint8, device=self.device)

    def opnorm(self, iters: int = 30, v0: torch.Tensor | None = None, seed: int = 0) -> float:
        """Estimate of ||R_h||^2 by the power iteration on R_h R_h*
        (``radon_opnorm``). ``v0`` defaults to a seeded Gaussian image."""
        if v0 is None:
            gen = torch.Generator(device="cpu").manual_seed(seed)
            v0 = torch.randn((self.Nq, self.Ntau), generator=gen).to(self.device)
        _check_tensor(v0, (self.Nq, self.Ntau), "v0", self.device)
        work = self._work("radon_opnorm_work_bytes")
        out = torch.zeros(1, dtype=torch.float32, device=self.device)
        _lib.check(_lib.load().radon_opnorm(self._handle, ctypes.c_void_p(v0.data_ptr()), int(iters),
                                            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(work.data_ptr()),
                                            work.numel(), _stream_ptr(self.device)))
        return float(out.item())

    def ista(self, f: torch.Tensor, mu: float, iters: int = 50, *, mask: torch.Tensor | None = None,
             g0: torch.Tensor | None = None, step: float | None = None, accelerate: bool = True,
             out: torch.Tensor | None = None) -> torch.Tensor:
        """Sparse Radon image of ``f`` by soft thresholding (``radon_ista``):
        ``iters`` iterations of the paper's ISTA (``accelerate=False``) or of
        FISTA. ``mask`` [Nx] marks recorded traces (missing-data form);
        ``step`` is c^2 (default 0.95 / ||R_h||^2 from ``opnorm``)."""
        _check_tensor(f, (self.Nx, self.Nt), "f", self.device)
        if mask is not None:
            _check_tensor(mask, (self.Nx,), "mask", self.device)
        if step is None:
            step = 0.95 / self.opnorm()
        if out is None:
            out = torch.zeros((self.Nq, self.Ntau), dtype=torch.float32, device=self.device)
        _check_tensor(out, (self.Nq, self.Ntau), "out", self.device)
        if g0 is not None:
            _check_tensor(g0, (self.Nq, self.Ntau), "g0", self.device)
            out.copy_(g0)
        work = self._work("radon_ista_work_bytes")
        _lib.check(_lib.load().radon_ista(
            self._handle, ctypes.c_void_p(f.data_ptr()),
            ctypes.c_void_p(mask.data_ptr() if mask is not None else None), ctypes.c_void_p(out.data_ptr()),
            int(iters), float(step), float(mu), int(bool(accelerate)), ctypes.c_void_p(work.data_ptr()),
            work.numel(), _stream_ptr(self.device)))
        return out


    def mute(self, g: torch.Tensor, q0: float, slope: float, keep: str = "below",
             out: torch.Tensor | None = None) -> torch.Tensor:
        """Radon-domain mute along the line q = q0 + slope * tau: keep the
        part below it (primaries) or above it (multiples)."""
        _check_tensor(g, (self.Nq, self.Ntau), "g", self.device)
        if out is None:
            out = torch.empty_like(g)
        _check_tensor(out, (self.Nq, self.Ntau), "out", self.device)
        side = {"below": 0, "above": 1}[keep]
        _lib.check(_lib.load().radon_mute(self._handle, ctypes.c_void_p(g.data_ptr()),
                                          ctypes.c_void_p(out.data_ptr()), float(q0), float(slope), side,
                                          _stream_ptr(self.device)))
        return out

    def demultiple(self, f: torch.Tensor, q0: float, slope: float, mu: float, iters: int = 30, *,
                   step: float | None = None, accelerate: bool = False):
        """Multiple attenuation: returns (f minus the multiples, sparse image).
        The multiples are the part of the sparse Radon image above the line
        q = q0 + slope * tau, taken back with the adjoint."""
        _check_tensor(f, (self.Nx, self.Nt), "f", self.device)
        if step is None:
            step = 0.95 / self.opnorm()
        g = torch.zeros((self.Nq, self.Ntau), dtype=torch.float32, device=self.device)
        f_out = torch.empty_like(f)
        work = self._work("radon_demultiple_work_bytes")
        _lib.check(_lib.load().radon_demultiple(
            self._handle, ctypes.c_void_p(f.data_ptr()), float(q0), float(slope), int(iters), float(step),
            float(mu), int(bool(accelerate)), ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(f_out.data_ptr()),
            ctypes.c_void_p(work.data_ptr()), work.numel(), _stream_ptr(self.device)))
        return f_out, g


def _grid_array(v, n, name):
    """A given offset / slowness list as a C double array (None: regular)."""
    if v is None:
        return None
    vals = [float(a) for a in v]
    if len(vals) != n:
        raise ValueError(f"{name} has {len(vals)} values, expected {n}")
    return (ctypes.c_double * n)(*vals)


def _desc(Nt, Nx, Ntau, Nq, dt, dx, qmin, qmax, tau0=0.0, dtau=0.0, sigma=None, omega_c=None,
          tsplit=None, n_qsplit=1, rows_per_band=None, device=0, spline_order=None) -> RadonDesc:
    d = RadonDesc()
    _lib.check(_lib.load().radon_desc_init(ctypes.byref(d), Nt, Nx, Ntau, Nq, dt, dx, qmin, qmax))
    d.tau0, d.dtau, d.n_qsplit, d.device = tau0, dtau, n_qsplit, device
    if sigma is not None:
        d.sigma = sigma
    if omega_c is not None:
        d.omega_c = omega_c
    if tsplit is not None:
        ts = list(tsplit)
        if len(ts) > _lib.MAX_TSPLIT:
            raise ValueError(f"at most {_lib.MAX_TSPLIT} time splits")
        d.n_tsplit = len(ts)
        for i, v in enumerate(ts):
            d.tsplit[i] = v
    if rows_per_band is not None:
        d.rows_per_band = rows_per_band
    if spline_order is not None:
        d.spline_order = spline_order
    return d


class Batch:
    """Many gathers of different sizes transformed together: every stage of
    the transform is one launch over all of them (``radon_batch_*``).

    ``geometries``: a list of dicts with the ``Plan`` arguments (``Nt``,
    ``Nx``, ``Ntau``, ``Nq``, ``dt``, ``dx``, ``qmin``, ``qmax`` and
    optionally ``tau0``, ``dtau``, ``sigma``, ``omega_c``, ``tsplit``,
    ``n_qsplit``, ``rows_per_band``, ``spline_order`` (one value for the
    whole batch); 0 in every ``rows_per_band`` times the feasible
    values over the whole batch; ``x`` / ``q``: given offsets / slownesses as
    in ``Plan``). Data are packed back to back (``f_offsets``,
    ``g_offsets``): gather i is ``f[f_offsets[i]:f_offsets[i+1]]`` viewed as
    [Nx][Nt]; ``forward`` accepts float32 or bfloat16 gathers."""

    def __init__(self, geometries: Sequence[dict], device: int | None = None):
        lib = _lib.load()
        dev = torch.cuda.current_device() if device is None else int(device)
        self.device = torch.device("cuda", dev)
        n = len(geometries)
        base = [{k: v for k, v in g.items() if k not in ("x", "q")} for g in geometries]
        arr = (RadonDesc * n)(*[_desc(device=dev, **g) for g in base])
        xs = [_grid_array(g.get("x"), g["Nx"], "x") for g in geometries]
        qs = [_grid_array(g.get("q"), g["Nq"], "q") for g in geometries]
        dp = ctypes.POINTER(ctypes.c_double)
        xp = (dp * n)(*[ctypes.cast(a, dp) if a is not None else dp() for a in xs])
        qp = (dp * n)(*[ctypes.cast(a, dp) if a is not None else dp() for a in qs])
        self._handle = ctypes.c_void_p()
        _lib.check(lib.radon_batch_create_grid(ctypes.byref(self._handle), n, arr, xp, qp))
        fo = (ctypes.c_longlong * (n + 1))()
        go = (ctypes.c_longlong * (n + 1))()
        _lib.check(lib.radon_batch_layout(self._handle, None, fo, go))
        self.f_offsets = list(fo)
        self.g_offsets = list(go)
        self.shapes = [((g["Nx"], g["Nt"]), (g["Nq"], g["Ntau"])) for g in geometries]

    def close(self):
        if getattr(self, "_handle", None) is not None and self._handle.value:
            _lib.load().radon_batch_destroy(self._handle)
            self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def plan_desc(self, i: int) -> RadonDesc:
        """The resolved descriptor of gather i's plan (``radon_batch_plan``)."""
        d = RadonDesc()
        _lib.check(_lib.load().radon_batch_plan(self._handle, i, ctypes.byref(d)))
        return d

    def pack(self, gathers: Sequence[torch.Tensor], dtype=torch.float32) -> torch.Tensor:
        """The packed gather buffer of the batch's layout."""
        out = torch.empty(self.f_offsets[-1], dtype=dtype, device=self.device)
        for i, t in enumerate(gathers):
            out[self.f_offsets[i]:self.f_offsets[i + 1]].copy_(t.reshape(-1))
        return out

    def unpack_images(self, g: torch.Tensor) -> list[torch.Tensor]:
        return [g[self.g_offsets[i]:self.g_offsets[i + 1]].view(*self.shapes[i][1])
                for i in range(len(self.shapes))]

    def unpack_gathers(self, f: torch.Tensor) -> list[torch.Tensor]:
        return [f[self.f_offsets[i]:self.f_offsets[i + 1]].view(*self.shapes[i][0])
                for i in range(len(self.shapes))]

    def forward(self, f: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        if f.device != self.device or not f.is_contiguous() or f.numel() != self.f_offsets[-1]:
            raise ValueError("f must be the contiguous packed gather buffer on the batch's device")
        if f.dtype == torch.float32:
            kind = 0
        elif f.dtype == torch.bfloat16:
            kind = 1
        else:
            raise ValueError("f must be float32 or bfloat16")
        if out is None:
            out = torch.empty(self.g_offsets[-1], dtype=torch.float32, device=self.device)
        if out.numel() != self.g_offsets[-1] or out.dtype != torch.float32 or not out.is_contiguous():
            raise ValueError("out must be the contiguous packed float32 image buffer")
        _lib.check(_lib.load().radon_batch_fwd(self._handle, ctypes.c_void_p(f.data_ptr()), kind,
                                               ctypes.c_void_p(out.data_ptr()), _stream_ptr(self.device)))
        return out

    def adjoint(self, g: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        if (g.device != self.device or not g.is_contiguous() or g.numel() != self.g_offsets[-1]
                or g.dtype != torch.float32):
            raise ValueError("g must be the contiguous packed float32 image buffer on the batch's device")
        if out is None:
            out = torch.empty(self.f_offsets[-1], dtype=torch.float32, device=self.device)
        if out.numel() != self.f_offsets[-1] or out.dtype != torch.float32 or not out.is_contiguous():
            raise ValueError("out must be the contiguous packed float32 gather buffer")
        _lib.check(_lib.load().radon_batch_adj(self._handle, ctypes.c_void_p(g.data_ptr()),
                                               ctypes.c_void_p(out.data_ptr()), _stream_ptr(self.device)))
        return out


class HRadon(torch.autograd.Function):
    """Autograd op of the linear operator R_h: the backward of the forward
    transform is the adjoint transform (Eq. (16)); nothing is saved."""

    @staticmethod
    def forward(ctx, f, plan):
        ctx.plan = plan
        return plan.forward(f.contiguous())

    @staticmethod
    def backward(ctx, grad_g):
        return ctx.plan.adjoint(grad_g.contiguous()), None


class HRadonAdjoint(torch.autograd.Function):
    @staticmethod
    def forward(ctx, g, plan):
        ctx.plan = plan
        return plan.adjoint(g.contiguous())

    @staticmethod
    def backward(ctx, grad_f):
        return ctx.plan.forward(grad_f.contiguous()), None


def radon(f: torch.Tensor, plan: Plan) -> torch.Tensor:
    """Differentiable forward transform."""
    return HRadon.apply(f, plan)


def radon_adjoint(g: torch.Tensor, plan: Plan) -> torch.Tensor:
    """Differentiable adjoint transform."""
    return HRadonAdjoint.apply(g, plan)


radon_adj = radon_adjoint   # the C ABI's name


def direct_forward(f: torch.Tensor, Ntau: int, Nq: int, dt: float, dx: float, qmin: float,
                   qmax: float, tau0: float = 0.0, dtau: float = 0.0) -> torch.Tensor:
    """Direct summation over hyperbolas on the GPU (the O(N^3) comparator)."""
    Nx, Nt = f.shape
    dtau = dtau if dtau > 0 else (Nt - 1) * dt / (Ntau - 1)
    dq = (qmax - qmin) / (Nq - 1) if Nq > 1 else 0.0
    _check_tensor(f, (Nx, Nt), "f", f.device)
    g = torch.empty((Nq, Ntau), dtype=torch.float32, device=f.device)
    _lib.check(_lib.load().radon_direct_fwd(ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                                            Nt, Nx, Ntau, Nq, dt, dx, tau0, dtau, qmin, dq,
                                            _stream_ptr(f.device)))
    return g


def direct_adjoint(g: torch.Tensor, Nt: int, Nx: int, dt: float, dx: float, qmin: float,
                   qmax: float, tau0: float = 0.0, dtau: float = 0.0) -> torch.Tensor:
    """Transpose of ``direct_forward``."""
    Nq, Ntau = g.shape
    dtau = dtau if dtau > 0 else (Nt - 1) * dt / (Ntau - 1)
    dq = (qmax - qmin) / (Nq - 1) if Nq > 1 else 0.0
    _check_tensor(g, (Nq, Ntau), "g", g.device)
    f = torch.empty((Nx, Nt), dtype=torch.float32, device=g.device)
    _lib.check(_lib.load().radon_direct_adj(ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(f.data_ptr()),
                                            Nt, Nx, Ntau, Nq, dt, dx, tau0, dtau, qmin, dq,
                                            _stream_ptr(g.device)))
    return f
