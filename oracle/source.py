"""Source creation (FP64 checker).

"Source creation" is the first stage of each Chroma measurement the paper
times (Sec. 5).  The point source at x0 is the LatticePropagator whose twelve
spin-colour columns are unit vectors at one site:
S(x)[s c][s' c'] = delta_{x, x0} delta_{s s'} delta_{c c'}.
"""
from __future__ import annotations

import numpy as np


def point_propagator(dims, x0=(0, 0, 0, 0)) -> np.ndarray:
    L0, L1, L2, L3 = dims
    S = np.zeros((L3, L2, L1, L0, 4, 3, 4, 3), dtype=np.complex128)
    site = (x0[3], x0[2], x0[1], x0[0])
    for s in range(4):
        for c in range(3):
            S[site + (s, c, s, c)] = 1.0
    return S


def point_fermion(dims, x0=(0, 0, 0, 0), spin: int = 0, color: int = 0) -> np.ndarray:
    """Point LatticeFermion: a unit entry at (x0, spin, color)."""
    L0, L1, L2, L3 = dims
    f = np.zeros((L3, L2, L1, L0, 4, 3), dtype=np.complex128)
    f[(x0[3], x0[2], x0[1], x0[0], spin, color)] = 1.0
    return f
