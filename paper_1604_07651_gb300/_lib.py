"""ctypes declarations of the C ABI in include/hradon.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

from . import build as _build

MAX_TSPLIT = 8
NSTAGES = 10
STAGE_NAMES = ["grid_fwd", "rows_r2c_fwd", "colconv_fwd", "rows_c2r_fwd", "interp_fwd",
               "bandrows_rowfft_adj", "colconv_adj", "rows_c2r_adj", "gather_adj", "profiles_adj"]
_c_int, _c_double, _vp = ctypes.c_int, ctypes.c_double, ctypes.c_void_p


class RadonDesc(ctypes.Structure):
    _fields_ = [("Nt", _c_int), ("Nx", _c_int), ("Ntau", _c_int), ("Nq", _c_int),
                ("dt", _c_double), ("dx", _c_double), ("qmin", _c_double), ("qmax", _c_double),
                ("tau0", _c_double), ("dtau", _c_double), ("sigma", _c_double),
                ("omega_c", _c_double), ("n_tsplit", _c_int),
                ("tsplit", _c_double * MAX_TSPLIT), ("n_qsplit", _c_int), ("device", _c_int),
                ("rows_per_band", _c_int), ("spline_order", _c_int)]


class RadonPieceInfo(ctypes.Structure):
    _fields_ = [("jt_lo", _c_int), ("jt_hi", _c_int), ("l_lo", _c_int), ("l_hi", _c_int),
                ("alpha", _c_double), ("beta", _c_double), ("a", _c_double), ("O1", _c_double),
                ("O2", _c_double), ("a_r", _c_double), ("r_max", _c_double),
                ("dphi_rule", _c_double), ("deta_rule", _c_double), ("dtheta", _c_double),
                ("drho", _c_double), ("theta0", _c_double), ("rho0", _c_double),
                ("Ntheta", _c_int), ("Nrho", _c_int), ("Ptheta", _c_int), ("Prho", _c_int),
                ("k1max", _c_int), ("k2max", _c_int), ("theta_m", _c_double),
                ("grid_tiles", _c_int), ("grid_units", _c_int), ("grid_split_tiles", _c_int),
                ("grid_max_tile_chunks", _c_int)]


# every symbol include/hradon.h declares, with its ctypes signature
SIGNATURES = {
    "radon_desc_init": (_c_int, [ctypes.POINTER(RadonDesc), _c_int, _c_int, _c_int, _c_int,
                                 _c_double, _c_double, _c_double, _c_double]),
    "radon_plan_create": (_c_int, [ctypes.POINTER(_vp), _c_int, _c_int, _c_int, _c_int,
                                   _c_double, _c_double, _c_double]),
    "radon_plan_create_ex": (_c_int, [ctypes.POINTER(_vp), ctypes.POINTER(RadonDesc)]),
    "radon_plan_create_grid": (_c_int, [ctypes.POINTER(_vp), ctypes.POINTER(RadonDesc),
                                        ctypes.POINTER(_c_double), ctypes.POINTER(_c_double)]),
    "radon_plan_destroy": (_c_int, [_vp]),
    "radon_fwd": (_c_int, [_vp, _vp, _vp, _vp]),
    "radon_adj": (_c_int, [_vp, _vp, _vp, _vp]),
    "radon_plan_num_pieces": (_c_int, [_vp, ctypes.POINTER(_c_int)]),
    "radon_plan_piece_info": (_c_int, [_vp, _c_int, ctypes.POINTER(RadonPieceInfo)]),
    "radon_plan_desc": (_c_int, [_vp, ctypes.POINTER(RadonDesc)]),
    "radon_geometry": (_c_int, [ctypes.POINTER(RadonDesc), ctypes.POINTER(_c_int),
                                ctypes.POINTER(RadonPieceInfo), _c_int]),
    "radon_geometry_grid": (_c_int, [ctypes.POINTER(RadonDesc), ctypes.POINTER(_c_double),
                                     ctypes.POINTER(_c_double), ctypes.POINTER(_c_int),
                                     ctypes.POINTER(RadonPieceInfo), _c_int]),
    "radon_plan_device_bytes": (_c_int, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "radon_plan_piece_lattice": (_c_int, [_vp, _c_int, _vp, ctypes.c_size_t]),
    "radon_plan_piece_samples": (_c_int, [_vp, _c_int, _vp, _vp, _vp, ctypes.c_size_t]),
    "radon_batch_create": (_c_int, [ctypes.POINTER(_vp), _c_int, ctypes.POINTER(RadonDesc)]),
    "radon_batch_create_grid": (_c_int, [ctypes.POINTER(_vp), _c_int, ctypes.POINTER(RadonDesc),
                                         ctypes.POINTER(ctypes.POINTER(_c_double)),
                                         ctypes.POINTER(ctypes.POINTER(_c_double))]),
    "radon_batch_destroy": (_c_int, [_vp]),
    "radon_batch_layout": (_c_int, [_vp, ctypes.POINTER(_c_int), ctypes.POINTER(ctypes.c_longlong),
                                    ctypes.POINTER(ctypes.c_longlong)]),
    "radon_batch_plan": (_c_int, [_vp, _c_int, ctypes.POINTER(RadonDesc)]),
    "radon_batch_fwd": (_c_int, [_vp, _vp, _c_int, _vp, _vp]),
    "radon_batch_adj": (_c_int, [_vp, _vp, _vp, _vp]),
    "radon_ista_work_bytes": (_c_int, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "radon_ista": (_c_int, [_vp, _vp, _vp, _vp, _c_int, ctypes.c_float, ctypes.c_float, _c_int, _vp,
                            ctypes.c_size_t, _vp]),
    "radon_opnorm_work_bytes": (_c_int, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "radon_mute": (_c_int, [_vp, _vp, _vp, _c_double, _c_double, _c_int, _vp]),
    "radon_demultiple_work_bytes": (_c_int, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "radon_demultiple": (_c_int, [_vp, _vp, _c_double, _c_double, _c_int, ctypes.c_float, ctypes.c_float,
                                  _c_int, _vp, _vp, _vp, ctypes.c_size_t, _vp]),
    "radon_opnorm": (_c_int, [_vp, _vp, _c_int, _vp, _vp, ctypes.c_size_t, _vp]),
    "radon_direct_fwd": (_c_int, [_vp, _vp, _c_int, _c_int, _c_int, _c_int, _c_double,
                                  _c_double, _c_double, _c_double, _c_double, _c_double, _vp]),
    "radon_direct_adj": (_c_int, [_vp, _vp, _c_int, _c_int, _c_int, _c_int, _c_double,
                                  _c_double, _c_double, _c_double, _c_double, _c_double, _vp]),
    "radon_plan_set_profiling": (_c_int, [_vp, _c_int]),
    "radon_plan_profile_read": (_c_int, [_vp, ctypes.POINTER(_c_double), ctypes.POINTER(ctypes.c_longlong),
                                         ctypes.POINTER(_c_double)]),
    "radon_fwd_noalloc": (_c_int, [_vp, _vp, _vp, _vp]),
    "radon_last_error": (ctypes.c_char_p, []),
    "radon_version": (ctypes.c_char_p, []),
}

STATUS = {0: "RADON_OK", 1: "RADON_ERR_INVALID_ARG", 2: "RADON_ERR_OOM", 3: "RADON_ERR_CUDA",
          4: "RADON_ERR_UNSUPPORTED"}

_lib = None


class RadonError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def load(build_if_missing: bool = True):
    """Load ``libhradon.so`` (building it in-tree first if it is missing or stale).
    Raises if the library cannot be built or loaded: there is no fallback."""
    global _lib
    if _lib is None:
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"{_build.LIB} is missing; run paper_1604_07651_gb300.build.build()")
        lib = ctypes.CDLL(_build.LIB)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(status: int):
    if status != 0:
        raise RadonError(status, load().radon_last_error().decode())
