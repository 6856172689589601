"""Error metrics of the parity tests that cannot pass on NaN or infinity.

Python's built-in ``max`` keeps its first argument when a comparison is false,
so ``max(0.0, nan)`` is ``0.0``: a running maximum that starts at zero would
let an output that is NaN everywhere through as "error 0".  Every helper here
first asserts that what it compares is finite, and the running maximum takes a
NaN (``not (x <= worst)`` is true for NaN) and keeps it from then on.
"""
from __future__ import annotations

import numpy as np


def _np(x):
    if hasattr(x, "detach"):                      # a torch tensor
        x = x.detach().cpu().double().numpy()
    return np.asarray(x)


def assert_finite(x, what="output"):
    """Assert that every entry of ``x`` (numpy array or torch tensor) is finite."""
    a = _np(x)
    bad = ~np.isfinite(a)
    assert not bad.any(), f"{what}: {int(bad.sum())} of {a.size} values are not finite"
    return a


def rel_l2_field(got, ref):
    """||got - ref|| / ||ref|| over a whole array, after finiteness checks."""
    got = assert_finite(got, "result")
    ref = assert_finite(ref, "reference")
    return float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300))


def rel_l2(got, ref):
    """Relative L2 error per component of [3][...] fields; the largest of the
    three (NaN-propagating ``np.max``), after finiteness checks."""
    got = assert_finite(got, "result")
    ref = assert_finite(ref, "reference")
    e = [np.linalg.norm(got[c] - ref[c]) / max(np.linalg.norm(ref[c]), 1e-300)
         for c in range(got.shape[0])]
    return float(np.max(e))


def max_abs_rel(got, ref, scale=None):
    """max |got - ref| / scale (scale defaults to max |ref|), after finiteness checks."""
    got = assert_finite(got, "result")
    ref = assert_finite(ref, "reference")
    sc = float(np.abs(ref).max()) if scale is None else float(scale)
    return float(np.abs(got - ref).max() / max(sc, 1e-300))


class Worst:
    """Running maximum of error values that keeps NaN once it has seen one."""

    def __init__(self, start: float = 0.0):
        self.value = float(start)

    def update(self, x) -> float:
        x = float(x)
        if self.value != self.value:              # NaN already seen: keep it
            return self.value
        if not (x <= self.value):                 # true for a larger x and for NaN
            self.value = x
        return self.value

    def __float__(self):
        return self.value

    def __lt__(self, other):
        return self.value < other

    def __le__(self, other):
        return self.value <= other

    def __repr__(self):
        return f"Worst({self.value!r})"
