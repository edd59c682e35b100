"""Gauge-covariant Gaussian (Wuppertal) smearing (FP64 checker).

The paper's source smearing (SRC) and sink smearing (SNK) stages (Sec. 5,
Fig. 4) apply this operator; the paper names the stages but does not print
the operator.  One iteration is the covariant nearest-neighbour hop over the
three directions other than ``j_decay``:

    psi'(x) = psi(x) + kappa * sum_{i != j_decay} [ U_i(x) psi(x + i_hat)
                                                    + U_i(x - i_hat)^dag psi(x - i_hat) ]

and the smeared field is N such iterations, psi_N = (1 + kappa H)^N psi_0.

Readings taken where the paper is silent:

* multiplicative iteration (each step acts on the previous step's result),
  not the Jacobi form psi_{k+1} = psi_0 + kappa H psi_k;
* no normalisation factor such as 1/(1 + 6 kappa);
* the hop acts on colour only: every spin component and every source column
  of a propagator is smeared as an independent colour vector.

``psi`` has the four site axes first, then spin, then colour, then any
trailing axes (the source spin/colour of a propagator).
"""
from __future__ import annotations

import numpy as np

from .geometry import axis_of, shift, spatial_dirs


def _as_colour_columns(psi: np.ndarray) -> tuple[np.ndarray, tuple]:
    """View psi as (..sites.., spin, colour, R) with R = product of trailing axes."""
    if psi.ndim < 6 or psi.shape[4] != 4 or psi.shape[5] != 3:
        raise ValueError(f"expected (..sites.., 4, 3, ...), got {psi.shape}")
    trailing = psi.shape[6:]
    r = int(np.prod(trailing)) if trailing else 1
    return psi.reshape(psi.shape[:6] + (r,)), trailing


def hop(U: np.ndarray, psi: np.ndarray, j_decay: int = 3) -> np.ndarray:
    """H psi = sum_{i != j_decay} [U_i(x) psi(x+i) + U_i(x-i)^dag psi(x-i)].

    ``U`` has shape (4, ..sites.., 3, 3); ``psi`` is in colour-column form.
    Colour matrices act on the colour axis through broadcast matmul.
    """
    out = np.zeros_like(psi)
    for mu in spatial_dirs(j_decay):
        Umu = U[mu][..., None, :, :]                      # (..sites.., 1, 3, 3)
        fwd = shift(psi, +1, mu)                          # psi(x + mu)
        out += Umu @ fwd
        U_back = shift(U[mu], -1, mu)[..., None, :, :]    # U_mu(x - mu)
        bwd = shift(psi, -1, mu)                          # psi(x - mu)
        out += np.conj(np.swapaxes(U_back, -1, -2)) @ bwd
    return out


def gauss_smear(U: np.ndarray, psi: np.ndarray, kappa: float, n_iter: int,
                j_decay: int = 3) -> np.ndarray:
    """Return (1 + kappa H)^N psi for a fermion or propagator field."""
    if U.shape[0] != 4 or U.shape[-2:] != (3, 3) or U.shape[1:5] != psi.shape[:4]:
        raise ValueError("links and field disagree on the lattice")
    if n_iter < 0:
        raise ValueError("negative iteration count")
    axis_of(j_decay)
    cur, trailing = _as_colour_columns(np.asarray(psi, dtype=np.complex128))
    for _ in range(n_iter):
        cur = cur + kappa * hop(U, cur, j_decay)
    return cur.reshape(cur.shape[:6] + trailing)
