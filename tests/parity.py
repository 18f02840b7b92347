"""Parity bars shared by the GPU tests (FP32 CUDA path vs the FP64 oracle).

Every comparison asserts two things on the same arrays:
* the relative L2 error ||got - ref|| / ||ref|| <= tol (the bar of the
  float32 path after nt steps);
* a per-element bound max |got - ref| <= PEAK * tol * max |ref|, so that one
  wrong value (a sponge corner, a far-face receiver, a tile seam) cannot hide
  under the global norm.  PEAK = 2: float32 rounding is not spread evenly over
  the field, and the worst element of a correct run reaches 1.34 tol of the
  largest magnitude (SO16, 400 steps, 56 x 52 x 48) while its relative L2
  error stays below tol.
"""
import numpy as np

TOL = 1e-5
PEAK = 2.0


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (n if n > 0 else 1.0)


def max_rel(a, b):
    """max |a - b| / max |b| (0 / 0 = 0)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    s = np.abs(b).max() if b.size else 0.0
    e = np.abs(a - b).max() if a.size else 0.0
    return e / s if s > 0 else e


def assert_close(got, ref, tol=TOL, what=""):
    """Both bars: relative L2 <= tol and every element within PEAK * tol of
    the largest reference magnitude."""
    r, m = rel_l2(got, ref), max_rel(got, ref)
    assert r <= tol, "%s: rel-L2 %.3e > %.1e" % (what, r, tol)
    assert m <= PEAK * tol, "%s: max |error| / max |ref| %.3e > %.1e" % (what, m, PEAK * tol)
    return r, m
