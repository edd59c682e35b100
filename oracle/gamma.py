"""Dirac gamma matrices (FP64 checker).

The paper computes the "hadron spectrum (mesonic and baryonic)" (Sec. 5) in
Chroma on top of QDP++, whose spin basis is the DeGrand-Rossi chiral basis.
The paper does not print it; this module writes it out.  gamma_1..gamma_4 are
Hermitian, satisfy the Euclidean Clifford algebra and gamma_5 =
gamma_1 gamma_2 gamma_3 gamma_4 = diag(1, 1, -1, -1).

The sixteen basis elements are numbered as in QDP++:
Gamma(n) = gamma_1^{n_0} gamma_2^{n_1} gamma_3^{n_2} gamma_4^{n_3} where
n = n_0 + 2 n_1 + 4 n_2 + 8 n_3, so Gamma(15) = gamma_5.
The charge-conjugation matrix is C = gamma_2 gamma_4.
"""
from __future__ import annotations

import numpy as np

I = 1j


def _m(rows) -> np.ndarray:
    return np.array(rows, dtype=np.complex128)


GAMMA1 = _m([[0, 0, 0, I], [0, 0, I, 0], [0, -I, 0, 0], [-I, 0, 0, 0]])
GAMMA2 = _m([[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]])
GAMMA3 = _m([[0, 0, I, 0], [0, 0, 0, -I], [-I, 0, 0, 0], [0, I, 0, 0]])
GAMMA4 = _m([[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]])
GAMMAS = (GAMMA1, GAMMA2, GAMMA3, GAMMA4)


def Gamma(n: int) -> np.ndarray:
    """Basis element Gamma(n) = gamma_1^{n_0} gamma_2^{n_1} gamma_3^{n_2} gamma_4^{n_3}."""
    if not 0 <= n <= 15:
        raise ValueError(f"gamma index {n} outside 0..15")
    g = np.eye(4, dtype=np.complex128)
    for bit in range(4):
        if (n >> bit) & 1:
            g = g @ GAMMAS[bit]
    return g


GAMMA5 = Gamma(15)
C = GAMMA2 @ GAMMA4
