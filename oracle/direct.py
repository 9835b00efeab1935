"""Oracle (test infrastructure only): ctypes binding of ``direct.c``.

Only tests/, ``__graft_entry__.smoke()`` and bench.py's ``cpu_baseline`` leg
may import this module. The FP64 direct summation over hyperbolas it wraps
is the paper's reference method (Section 5: direct summation of Eq. (3)
with cubic interpolation in time); see ``direct.c`` for the formulas.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "direct.c")
_LIB = os.path.join(_HERE, "liboracle_direct.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile ``direct.c`` with gcc (OpenMP) into ``liboracle_direct.so``."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c99",
                        _SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i, d = ctypes.c_int, ctypes.c_double
        lib.oracle_direct_fwd.argtypes = [_dp, i, i, d, d, _dp, i, _dp, i, _dp]
        lib.oracle_direct_fwd_points.argtypes = [_dp, i, i, d, d, _dp, _dp, _ip, _ip, i, _dp]
        lib.oracle_direct_adj.argtypes = [_dp, i, i, d, d, d, d, i, _dp, i, _dp]
        lib.oracle_direct_adj_points.argtypes = [_dp, i, i, d, d, d, d, i, _dp, i, _ip, _ip, i, _dp]
        lib.oracle_direct_adj_brute.argtypes = [_dp, i, i, d, d, _dp, i, _dp, i, _dp]
        lib.oracle_direct_fwd_x.argtypes = [_dp, i, i, d, _dp, _dp, i, _dp, i, _dp]
        lib.oracle_direct_fwd_x_points.argtypes = [_dp, i, i, d, _dp, _dp, _dp, _ip, _ip, i, _dp]
        lib.oracle_direct_adj_x.argtypes = [_dp, i, i, d, _dp, d, d, i, _dp, i, _dp]
        lib.oracle_direct_adj_x_points.argtypes = [_dp, i, d, _dp, d, d, i, _dp, i, _ip, _ip, i, _dp]
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_set_threads.argtypes = [i]
        _lib = lib
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_ip)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_threads(n: int) -> None:
    """Threads of the following calls (the host's cores by default)."""
    _load().oracle_set_threads(int(n))


def fwd(f, dt, dx, tau, q):
    """Full forward: ``f[Nx][Nt]`` -> ``g[Nq][Ntau]``."""
    lib = _load()
    f, fp = _d(f)
    tau, tp = _d(tau)
    q, qp = _d(q)
    Nx, Nt = f.shape
    g = np.zeros((q.size, tau.size))
    lib.oracle_direct_fwd(fp, Nt, Nx, dt, dx, tp, tau.size, qp, q.size, g.ctypes.data_as(_dp))
    return g


def fwd_points(f, dt, dx, tau, q, ii, li):
    """Forward at sampled outputs ``g[li[p], ii[p]]``."""
    lib = _load()
    f, fp = _d(f)
    tau, tp = _d(tau)
    q, qp = _d(q)
    ii, iip = _i(ii)
    li, lip = _i(li)
    Nx, Nt = f.shape
    out = np.zeros(ii.size)
    lib.oracle_direct_fwd_points(fp, Nt, Nx, dt, dx, tp, qp, iip, lip, ii.size,
                                 out.ctypes.data_as(_dp))
    return out


def adj(g, Nt, Nx, dt, dx, tau0, dtau, q):
    """Full adjoint: ``g[Nq][Ntau]`` -> ``f[Nx][Nt]`` on tau_i = tau0 + i dtau."""
    lib = _load()
    g, gp = _d(g)
    q, qp = _d(q)
    Nq, Ntau = g.shape
    f = np.zeros((Nx, Nt))
    lib.oracle_direct_adj(gp, Nt, Nx, dt, dx, tau0, dtau, Ntau, qp, Nq, f.ctypes.data_as(_dp))
    return f


def adj_points(g, Nt, Nx, dt, dx, tau0, dtau, q, jj, kk):
    """Adjoint at sampled gather points ``f[kk[p], jj[p]]``."""
    lib = _load()
    g, gp = _d(g)
    q, qp = _d(q)
    jj, jp = _i(jj)
    kk, kp = _i(kk)
    Nq, Ntau = g.shape
    out = np.zeros(jj.size)
    lib.oracle_direct_adj_points(gp, Nt, Nx, dt, dx, tau0, dtau, Ntau, qp, Nq, jp, kp,
                                 jj.size, out.ctypes.data_as(_dp))
    return out


def adj_brute(g, Nt, Nx, dt, dx, tau, q):
    """Adjoint by brute force over every (i, l); tiny grids only."""
    lib = _load()
    g, gp = _d(g)
    tau, tp = _d(tau)
    q, qp = _d(q)
    Nq, Ntau = g.shape
    f = np.zeros((Nx, Nt))
    lib.oracle_direct_adj_brute(gp, Nt, Nx, dt, dx, tp, Ntau, qp, Nq, f.ctypes.data_as(_dp))
    return f


# ---- unequally spaced offsets (trapezoid weights on the given offsets) ----

def _offsets(x, Nx):
    x = np.ascontiguousarray(x, dtype=np.float64)
    if x.shape != (Nx,) or Nx < 2 or not np.all(np.diff(x) > 0):
        raise ValueError("need Nx >= 2 strictly increasing offsets")
    return x, x.ctypes.data_as(_dp)


def fwd_x(f, dt, x, tau, q):
    """Forward on offsets ``x[Nx]`` (km): ``f[Nx][Nt]`` -> ``g[Nq][Ntau]``."""
    lib = _load()
    f, fp = _d(f)
    Nx, Nt = f.shape
    x, xp = _offsets(x, Nx)
    tau, tp = _d(tau)
    q, qp = _d(q)
    g = np.zeros((q.size, tau.size))
    lib.oracle_direct_fwd_x(fp, Nt, Nx, dt, xp, tp, tau.size, qp, q.size, g.ctypes.data_as(_dp))
    return g


def fwd_x_points(f, dt, x, tau, q, ii, li):
    """Forward on offsets ``x`` at sampled outputs ``g[li[p], ii[p]]``."""
    lib = _load()
    f, fp = _d(f)
    Nx, Nt = f.shape
    x, xp = _offsets(x, Nx)
    tau, tp = _d(tau)
    q, qp = _d(q)
    ii, iip = _i(ii)
    li, lip = _i(li)
    out = np.zeros(ii.size)
    lib.oracle_direct_fwd_x_points(fp, Nt, Nx, dt, xp, tp, qp, iip, lip, ii.size, out.ctypes.data_as(_dp))
    return out


def adj_x(g, Nt, dt, x, tau0, dtau, q):
    """Adjoint on offsets ``x[Nx]``: ``g[Nq][Ntau]`` -> ``f[Nx][Nt]``."""
    lib = _load()
    g, gp = _d(g)
    x = np.asarray(x, dtype=np.float64)
    Nx = x.size
    x, xp = _offsets(x, Nx)
    q, qp = _d(q)
    Nq, Ntau = g.shape
    f = np.zeros((Nx, Nt))
    lib.oracle_direct_adj_x(gp, Nt, Nx, dt, xp, tau0, dtau, Ntau, qp, Nq, f.ctypes.data_as(_dp))
    return f


def adj_x_points(g, dt, x, tau0, dtau, q, jj, kk):
    """Adjoint on offsets ``x`` at sampled gather points ``f[kk[p], jj[p]]``."""
    lib = _load()
    g, gp = _d(g)
    x = np.asarray(x, dtype=np.float64)
    x, xp = _offsets(x, x.size)
    q, qp = _d(q)
    jj, jp = _i(jj)
    kk, kp = _i(kk)
    Nq, Ntau = g.shape
    out = np.zeros(jj.size)
    lib.oracle_direct_adj_x_points(gp, x.size, dt, xp, tau0, dtau, Ntau, qp, Nq, jp, kp, jj.size,
                                   out.ctypes.data_as(_dp))
    return out
