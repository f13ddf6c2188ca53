"""Element-wise comparison of a GPU result with the oracle's.

Every element must satisfy

    |gpu_j - oracle_j| <= tol * max(|oracle_j|, floor * max_k |oracle_k|),

that is, a relative error of at most tol where the oracle's value is not small
(at least `floor` of the largest), and an absolute error of at most
tol * floor * max|oracle| elsewhere. A norm-wise check alone would let a few
elements (an edge column, the last tile of a CTA, one slice of a batch) drift
far beyond tol and still pass. The norm-wise relative error is printed beside
the worst element, for the record.

Tolerances used by the tests: 1e-10 for FP64 iterates, 1e-4 for FP32 and
2e-3 for results of reduced-precision (BF16/FP16) values against exact FP64.
"""
from __future__ import annotations

import numpy as np


def close(got, ref, tol: float, what: str = "", floor: float = 0.1) -> float:
    """Assert the element-wise bound above; return the worst element's error / bound ratio."""
    got = np.asarray(got, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    assert got.shape == ref.shape, (what, got.shape, ref.shape)
    assert np.all(np.isfinite(got)), f"{what}: non-finite GPU values"
    scale = float(np.abs(ref).max()) if ref.size else 0.0
    err = np.abs(got - ref)
    if scale == 0.0:
        assert err.size == 0 or err.max() == 0.0, f"{what}: oracle is all zero, GPU max |value| {err.max():.3e}"
        return 0.0
    bound = tol * np.maximum(np.abs(ref), floor * scale)
    ratio = err / bound
    k = int(np.argmax(ratio))
    norm = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    msg = (f"{what}: worst element {k} of {ref.size}: gpu {got[k]:.9e} oracle {ref[k]:.9e} |d| {err[k]:.3e} "
           f"bound {bound[k]:.3e} (ratio {ratio[k]:.3f}); norm-wise relative {norm:.3e}")
    print(msg)
    assert ratio[k] <= 1.0, msg
    return float(ratio[k])


def close_scalar(got: float, ref: float, tol: float, what: str = "") -> None:
    """Relative check of one scalar (rho, a norm)."""
    d = abs(got - ref)
    assert d <= tol * abs(ref) or (ref == 0.0 and got == 0.0), f"{what}: {got!r} vs {ref!r} (|d| {d:.3e}, tol {tol})"


def close_norm(got, ref, tol: float, what: str = "") -> float:
    """Norm-wise relative check, with the worst element printed beside it.

    Used only for the storage error of BF16/FP16 matrix values against the
    exact FP64 matrix: that error is the format's (an 8-bit mantissa rounds
    each entry by up to 2^-9 of its row's scale), not the kernel's, and the
    2e-3 tolerance for reduced-precision values bounds it norm-wise. The
    kernel itself is checked element by element against the oracle run on
    the stored values.
    """
    got = np.asarray(got, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    assert np.all(np.isfinite(got)), f"{what}: non-finite GPU values"
    norm = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    err = np.abs(got - ref)
    k = int(np.argmax(err))
    scale = float(np.abs(ref).max())
    msg = (f"{what}: norm-wise relative {norm:.3e} (tol {tol}); worst element {k}: |d| {err[k]:.3e} = "
           f"{err[k] / scale:.3e} of max|oracle|")
    print(msg)
    assert norm <= tol, msg
    return norm
