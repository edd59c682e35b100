"""Hadron-spectrum contractions (FP64 checker).

The paper's HAD stage computes the "hadron spectrum (mesonic and baryonic)"
(Sec. 5, Fig. 4) without printing the contractions.  The mesonic two-point
function written out here is the standard one:

    C(t, p) = sum_{x : x_{j_decay} = t} exp(-i p.(x - x0))
              tr[ Gamma_snk S1(x) Gamma_src^dag gamma_5 S2(x)^dag gamma_5 ]

with the trace over spin and colour, S(x) the 12x12 propagator at x
(row = sink spin/colour, column = source spin/colour), and
p = 2 pi (n_1/L_1, n_2/L_2, n_3/L_3) over the three directions other than
``j_decay`` in increasing order.

Readings taken where the paper is silent:

* the source vertex enters as Gamma_src^dag (not gamma_4 Gamma^dag gamma_4);
* "the 16 mesons" are the channels Gamma_snk = Gamma_src = Gamma(n), n = 0..15;
* x is measured from the source origin x0 for the momentum phase; output
  timeslices are indexed by the absolute coordinate t = x_{j_decay}.
"""
from __future__ import annotations

import numpy as np

from .gamma import GAMMA5, Gamma
from .geometry import axis_of, coords, spatial_dirs

_I3 = np.eye(3, dtype=np.complex128)


def _spin_colour(g: np.ndarray) -> np.ndarray:
    """A 4x4 spin matrix as the 12x12 matrix g (x) 1_colour, index s*3 + c."""
    return np.kron(g, _I3)


def meson_site(S1: np.ndarray, S2: np.ndarray, g_snk: int, g_src: int) -> np.ndarray:
    """Site trace c(x) = tr[Gamma_snk S1 Gamma_src^dag g5 S2^dag g5], shape (..sites..).

    By cyclicity of the trace this is tr[X S2^dag] with
    X = (g5 Gamma_snk) S1 (Gamma_src^dag g5), i.e. sum_ij X_ij conj(S2_ij).
    """
    sites = S1.shape[:4]
    m1 = S1.reshape(sites + (12, 12))
    m2 = S2.reshape(sites + (12, 12))
    left = _spin_colour(GAMMA5 @ Gamma(g_snk))
    right = _spin_colour(Gamma(g_src).conj().T @ GAMMA5)
    X = left @ m1 @ right
    return np.sum(X * np.conj(m2), axis=(-2, -1))


def momentum_phases(dims, moms, j_decay: int = 3, origin=(0, 0, 0, 0)) -> np.ndarray:
    """exp(-i p.(x - x0)) per site and momentum, shape (n_mom, ..sites..)."""
    x = coords(dims)
    sd = spatial_dirs(j_decay)
    out = []
    for n in moms:
        arg = np.zeros(x.shape[:4])
        for k, mu in enumerate(sd):
            arg += n[k] * (x[..., mu] - origin[mu]) / dims[mu]
        out.append(np.exp(-2j * np.pi * arg))
    return np.array(out)


def timeslice_sum(site_values: np.ndarray, j_decay: int = 3) -> np.ndarray:
    """Sum a site field over each timeslice of direction j_decay, shape (Nt,)."""
    ax = axis_of(j_decay)
    moved = np.moveaxis(site_values, ax, 0)
    return moved.reshape(moved.shape[0], -1).sum(axis=1)


def meson_2pt(S1: np.ndarray, S2: np.ndarray, channels, moms=((0, 0, 0),), j_decay: int = 3,
              origin=(0, 0, 0, 0)) -> np.ndarray:
    """Correlators for channels [(g_snk, g_src), ...], shape (n_chan, n_mom, Nt) complex128."""
    if S1.shape != S2.shape or S1.shape[4:] != (4, 3, 4, 3):
        raise ValueError("propagators must both have shape (..sites.., 4, 3, 4, 3)")
    L3, L2, L1, L0 = S1.shape[:4]
    dims = (L0, L1, L2, L3)
    phases = momentum_phases(dims, moms, j_decay, origin)
    out = np.empty((len(channels), len(moms), dims[j_decay]), dtype=np.complex128)
    for j, (g_snk, g_src) in enumerate(channels):
        c = meson_site(S1, S2, g_snk, g_src)
        for k in range(len(moms)):
            out[j, k] = timeslice_sum(c * phases[k], j_decay)
    return out


SIXTEEN_MESONS = tuple((n, n) for n in range(16))
