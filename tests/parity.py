"""Parity check of a CUDA result against its FP64 reference, element by element.

Three bounds, all of which must hold (out, ref: arrays of the same shape):

* relative L2 over the whole array <= tol (1e-5: FP32 against the FP64 oracle
  on the same lattices);
* every element: |out - ref| <= ELEM_C * tol * max|ref|. The FP32 FFTs spread
  their rounding error over the whole lattice, so an element's error scales
  with the array's peak, not with its own value; ELEM_C = 1 leaves about an
  order of magnitude over the largest element errors measured on the GPU
  (a few 1e-7 of the peak) while any wrong tap, seam or band of a size that
  matters shows up;
* every row (an output column [Nq][Ntau] of an image, a trace [Nx][Nt] of a
  gather) whose norm is at least ROW_FLOOR of the root-mean-square row norm:
  relative L2 of the row <= ROW_TOL. This catches a wrong band of outputs
  where the image is small (a row with 1e-2 of the typical energy still has
  to be right to 1e-4 of its own norm).

On failure the message gives the worst element's index, value and reference.
"""
from __future__ import annotations

import numpy as np

PARITY_TOL = 1e-5
ELEM_C = 1.0
ROW_TOL = 1e-4
ROW_FLOOR = 1e-2


def parity_stats(out, ref) -> dict:
    out = np.asarray(out, np.float64)
    ref = np.asarray(ref, np.float64)
    assert out.shape == ref.shape, (out.shape, ref.shape)
    err = out - ref
    nref = float(np.linalg.norm(ref))
    amax = float(np.abs(ref).max()) if ref.size else 0.0
    st = {"rel_l2": float(np.linalg.norm(err)) / nref if nref > 0 else float(np.linalg.norm(err)),
          "finite": bool(np.all(np.isfinite(out)))}
    if err.size:
        k = np.unravel_index(int(np.argmax(np.abs(err))), err.shape)
        st.update(worst_index=tuple(int(i) for i in k), worst_out=float(out[k]), worst_ref=float(ref[k]),
                  elem_rel=float(abs(err[k])) / amax if amax > 0 else float(abs(err[k])))
    else:
        st.update(worst_index=None, worst_out=0.0, worst_ref=0.0, elem_rel=0.0)
    st["row_rel_max"] = 0.0
    st["worst_row"] = None
    if ref.ndim == 2 and ref.shape[0] > 0 and nref > 0:
        rn = np.linalg.norm(ref, axis=1)
        en = np.linalg.norm(err, axis=1)
        rms = nref / np.sqrt(ref.shape[0])
        sel = np.nonzero(rn >= ROW_FLOOR * rms)[0]
        if sel.size:
            rr = en[sel] / rn[sel]
            i = int(np.argmax(rr))
            st["row_rel_max"] = float(rr[i])
            st["worst_row"] = int(sel[i])
    return st


def assert_parity(out, ref, tol: float = PARITY_TOL, what: str = "", c: float = ELEM_C,
                  row_tol: float = ROW_TOL) -> dict:
    """Assert the three bounds above; returns the statistics."""
    st = parity_stats(out, ref)
    msg = (f"{what}: rel L2 {st['rel_l2']:.3e} (<= {tol:g}), max|err|/max|ref| {st['elem_rel']:.3e} "
           f"(<= {c * tol:g}) at {st['worst_index']} (out {st['worst_out']:.6g}, ref {st['worst_ref']:.6g}), "
           f"worst row {st['worst_row']} rel L2 {st['row_rel_max']:.3e} (<= {row_tol:g})")
    assert st["finite"], what + ": non-finite output"
    assert st["rel_l2"] <= tol, msg
    assert st["elem_rel"] <= c * tol, msg
    assert st["row_rel_max"] <= row_tol, msg
    return st
