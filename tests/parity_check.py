"""Element-by-element comparison used by every GPU parity test.

``close(a, ref)`` returns the larger of two relative errors of ``a`` against
``ref``:

  * the largest entry error against the largest reference entry,
    max_i |a_i - ref_i| / max_i |ref_i|, which bounds every single value, so an
    error confined to a few entries (one face's rows, one cell) cannot hide in
    a norm over many correct ones;
  * the 2-norm error, ||a - ref||_2 / ||ref||_2.

A test asserts ``close(a, ref) <= tol`` with the tolerance of its precision:
1e-12 for FP64 operator-level results, 1e-5 for FP32, and the looser bounds
stated at whole-cycle and whole-solve comparisons.
"""
import numpy as np


def _np(x):
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    return np.asarray(x, dtype=np.float64).ravel()


def max_rel(a, ref):
    """max_i |a_i - ref_i| / max_i |ref_i| (inf if a holds a non-finite value)."""
    a, ref = _np(a), _np(ref)
    if not np.all(np.isfinite(a)):
        return float("inf")
    return float(np.max(np.abs(a - ref)) / max(np.max(np.abs(ref)), 1e-300)) if a.size else 0.0


def norm_rel(a, ref):
    """||a - ref||_2 / ||ref||_2 (inf if a holds a non-finite value)."""
    a, ref = _np(a), _np(ref)
    if not np.all(np.isfinite(a)):
        return float("inf")
    return float(np.linalg.norm(a - ref) / max(np.linalg.norm(ref), 1e-300)) if a.size else 0.0


def close(a, ref):
    """The larger of the element-wise and the 2-norm relative error."""
    return max(max_rel(a, ref), norm_rel(a, ref))
