"""Parity checks shared by the GPU tests.

Every comparison of a GPU result with the oracle (or with another GPU path)
checks two things at the same tolerance `tol`:

* the relative 2-norm  ||got - ref||_2 / ||ref||_2 <= tol, and
* element by element   max_i |got_i - ref_i| <= tol * max_i |ref_i|.

The 2-norm alone dilutes an error confined to a few entries (a band of grid
nodes next to the boundary, a handful of points) by sqrt(size / k); the
element-wise bound does not, so an indexing slip that touches only the nodes
near Gamma still fails.
"""
import numpy as np


def _flat(x):
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    return np.asarray(x, dtype=np.float64).reshape(-1)


def parity_errors(got, ref):
    """(relative 2-norm error, max-abs error / max |ref|)."""
    g, r = _flat(got), _flat(ref)
    if g.shape != r.shape:
        raise AssertionError(f"shape {g.shape} != {r.shape}")
    d = g - r
    rn = max(float(np.linalg.norm(r)), 1e-300)
    rm = max(float(np.max(np.abs(r))) if r.size else 0.0, 1e-300)
    emax = float(np.max(np.abs(d))) if d.size else 0.0
    return float(np.linalg.norm(d)) / rn, emax / rm


def assert_parity(got, ref, tol, what=""):
    g = _flat(got)
    assert np.all(np.isfinite(g)), f"{what}: non-finite output"
    e2, einf = parity_errors(g, ref)
    assert e2 <= tol and einf <= tol, (
        f"{what}: rel 2-norm {e2:.3e}, max-abs/max|ref| {einf:.3e}, tol {tol:g}")
