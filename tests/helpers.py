"""Comparison helpers for the parity tests (numpy only: they also run on the GPU machine)."""
from __future__ import annotations

import numpy as np

TOL = {1: 1e-13, 2: 1e-28, 4: 1e-58}   # relative error bounds, complex double / DD / QD


def _two_sum(a, b):
    s = a + b
    bb = s - a
    e = (a - (s - bb)) + (b - bb)
    return s, e


def limb_diff(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """(sum of A's limbs) - (sum of B's limbs) along the last axis, formed exactly as a
    floating-point expansion (vectorised grow-expansion) and then rounded to double."""
    terms = [A[..., j] for j in range(A.shape[-1])] + [-B[..., j] for j in range(B.shape[-1])]
    h: list[np.ndarray] = []
    for t in terms:
        q = t
        nh = []
        for comp in h:
            q, e = _two_sum(q, comp)
            nh.append(e)
        nh.append(q)
        h = nh
    out = np.zeros_like(A[..., 0])
    for comp in h:   # smallest first
        out = out + comp
    return out


def cabs_diff(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """|A - B| for complex values stored as [..., 2, L] limbs."""
    dr = limb_diff(A[..., 0, :], B[..., 0, :])
    di = limb_diff(A[..., 1, :], B[..., 1, :])
    return np.hypot(dr, di)


def cabs(A: np.ndarray) -> np.ndarray:
    return np.hypot(A[..., 0, :].sum(-1), A[..., 1, :].sum(-1))


def rel_err_per_point(got: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """max |got - ref| / max |ref| over all entries of each point (axis 0 = point)."""
    d = cabs_diff(got, ref).reshape(got.shape[0], -1).max(axis=1)
    m = cabs(ref).reshape(ref.shape[0], -1).max(axis=1)
    return d / np.maximum(m, 1e-300)


def digits(err: np.ndarray) -> float:
    """Correct decimal places implied by a relative error (the paper's "quality")."""
    e = float(np.max(err))
    return float("inf") if e == 0 else -np.log10(e)
