"""Lattice geometry and the nearest-neighbour shift (FP64 checker).

QDP++ evaluates data-parallel expressions site by site over the whole
lattice (Sec. 1, Sec. 4 of the paper); the one non-local primitive of such an
expression is the periodic nearest-neighbour shift.  Its direction follows
QDP++: ``shift(f, +1, mu)`` is the field whose value at x is f(x + mu_hat).
"""
from __future__ import annotations

import numpy as np


def axis_of(mu: int) -> int:
    """Numpy axis of lattice direction mu in a canonical site array (x0 last)."""
    if not 0 <= mu <= 3:
        raise ValueError(f"direction {mu} outside 0..3")
    return 3 - mu


def shift(f: np.ndarray, sign: int, mu: int) -> np.ndarray:
    """Periodic shift: out(x) = f(x + sign * mu_hat).

    ``f`` has the four site axes first.  ``np.roll(f, -1, axis)`` moves the
    entry at x+1 to x, which is exactly out(x) = f(x + mu_hat).
    """
    if sign not in (+1, -1):
        raise ValueError("sign must be +1 or -1")
    return np.roll(f, -sign, axis=axis_of(mu))


def spatial_dirs(j_decay: int) -> tuple[int, int, int]:
    """The three directions other than ``j_decay``, in increasing order."""
    return tuple(mu for mu in range(4) if mu != j_decay)


def coords(dims) -> np.ndarray:
    """Integer coordinates, shape ``(L3, L2, L1, L0, 4)``; entry [..., mu] = x_mu."""
    L0, L1, L2, L3 = dims
    x3, x2, x1, x0 = np.meshgrid(np.arange(L3), np.arange(L2), np.arange(L1), np.arange(L0),
                                 indexing="ij")
    return np.stack([x0, x1, x2, x3], axis=-1)
