"""The C-ABI library builds, loads, and exports every symbol include/hradon.h
declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hradon.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(radon_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1604_07651_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("radon_plan_create", "radon_fwd", "radon_adj", "radon_plan_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_1604_07651_gb300 import _lib
    assert set(declared_functions()) == set(_lib.SIGNATURES)


def test_host_side_argument_checks(lib):
    """Invalid descriptors are rejected on the host with a message, before any
    device work (these paths need no GPU)."""
    from paper_1604_07651_gb300 import _lib
    L = _lib.load()
    assert L.radon_version().decode().startswith("hradon")
    d = _lib.RadonDesc()
    assert L.radon_desc_init(ctypes.byref(d), 256, 64, 256, 64, 0.004, 0.025, 0.2, 0.7) == 0
    # the binding's struct matches the header's layout up to the last field
    assert (d.device, d.rows_per_band, d.n_qsplit, d.n_tsplit, d.spline_order) == (-1, 3, 1, 2, 3)
    h = ctypes.c_void_p()
    for field, value in [("Nt", 1), ("dt", 0.0), ("qmin", -1.0), ("omega_c", 0.6), ("sigma", 0.0),
                         ("n_qsplit", 0), ("n_tsplit", 9), ("rows_per_band", 7), ("rows_per_band", -1),
                         ("spline_order", 4), ("spline_order", 1), ("spline_order", 0)]:
        bad = _lib.RadonDesc.from_buffer_copy(d)
        setattr(bad, field, value)
        assert L.radon_plan_create_ex(ctypes.byref(h), ctypes.byref(bad)) == 1, field
        assert L.radon_last_error().decode()
        assert not h.value
    assert L.radon_plan_create_ex(ctypes.byref(h), None) == 1
    # given offsets / slownesses: checked on the host as well
    x = [0.025 * k for k in range(64)]
    q = [0.2 + 0.5 * l / 63 for l in range(64)]
    arr = lambda v: (ctypes.c_double * len(v))(*v)
    for bx, bq in [(x[:5] + [x[3]] + x[6:], None), ([-0.01] + x[1:], None), (x[:9] + [float("inf")] + x[10:], None),
                   (None, q[::-1]), (None, [q[0]] + q[:-1])]:
        rc = L.radon_plan_create_grid(ctypes.byref(h), ctypes.byref(d), arr(bx) if bx else None,
                                      arr(bq) if bq else None)
        assert rc == 1 and not h.value and L.radon_last_error().decode()
    one = _lib.RadonDesc.from_buffer_copy(d)
    one.Nx = 1
    assert L.radon_plan_create_grid(ctypes.byref(h), ctypes.byref(one), arr([0.5]), None) == 1
    assert L.radon_plan_destroy(None) == 0
    assert L.radon_fwd(None, None, None, None) == 1
    assert L.radon_adj(None, None, None, None) == 1
    assert L.radon_direct_fwd(None, None, 4, 4, 4, 4, 1.0, 1.0, 0.0, 1.0, 0.0, 0.1, None) == 1
    # a batch must share one B-spline order: refused before any device work
    pair = (_lib.RadonDesc * 2)(_lib.RadonDesc.from_buffer_copy(d), _lib.RadonDesc.from_buffer_copy(d))
    pair[1].spline_order = 5
    b = ctypes.c_void_p()
    assert L.radon_batch_create(ctypes.byref(b), 2, pair) == 4 and not b.value
    assert "order" in L.radon_last_error().decode()
