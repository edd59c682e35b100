"""Seeded synthetic lattice fields in the canonical host layout.

Canonical layout (shared by every consumer of these arrays):

* a lattice has extents ``dims = (L0, L1, L2, L3)``; site ``(x0, x1, x2, x3)``
  has lexicographic index ``x0 + L0*(x1 + L1*(x2 + L2*x3))`` (x0 fastest), so a
  numpy array over sites has axes ``(L3, L2, L1, L0)``;
* gauge links: ``(4, L3, L2, L1, L0, 3, 3)`` complex, ``U[mu][site][a][b]``;
* propagator: ``(L3, L2, L1, L0, 4, 3, 4, 3)`` complex,
  ``S[site][s][c][s'][c']`` (sink spin/colour first, then source);
* fermion: ``(L3, L2, L1, L0, 4, 3)`` complex;
* colour matrix: ``(L3, L2, L1, L0, 3, 3)`` complex.

Every generator takes an optional ``x3_range=(lo, hi)``: only the slices
``lo <= x3 < hi`` are produced, bit-identical to the same slices of the full
field, because every random number is keyed by its global site index.

These are inputs only.  Nothing here smears, shifts or contracts.
"""
from __future__ import annotations

import numpy as np

from . import rng

# Gell-Mann matrices lambda_1..lambda_8 (Gell-Mann, 1962), used to draw
# random traceless Hermitian generators H = sum_a h_a lambda_a / 2.
_GELL_MANN = np.zeros((8, 3, 3), dtype=np.complex128)
_GELL_MANN[0][0, 1] = _GELL_MANN[0][1, 0] = 1
_GELL_MANN[1][0, 1], _GELL_MANN[1][1, 0] = -1j, 1j
_GELL_MANN[2][0, 0], _GELL_MANN[2][1, 1] = 1, -1
_GELL_MANN[3][0, 2] = _GELL_MANN[3][2, 0] = 1
_GELL_MANN[4][0, 2], _GELL_MANN[4][2, 0] = -1j, 1j
_GELL_MANN[5][1, 2] = _GELL_MANN[5][2, 1] = 1
_GELL_MANN[6][1, 2], _GELL_MANN[6][2, 1] = -1j, 1j
_GELL_MANN[7] = np.diag([1, 1, -2]) / np.sqrt(3)


def site_shape(dims) -> tuple[int, int, int, int]:
    L0, L1, L2, L3 = dims
    return (L3, L2, L1, L0)


def _slice_sites(dims, x3_range):
    """Global site indices of the requested x3 slices, in canonical order."""
    L0, L1, L2, L3 = dims
    lo, hi = (0, L3) if x3_range is None else x3_range
    if not (0 <= lo <= hi <= L3):
        raise ValueError(f"x3_range {x3_range} outside 0..{L3}")
    v3 = L0 * L1 * L2
    return np.arange(lo * v3, hi * v3, dtype=np.uint64), (hi - lo, L2, L1, L0)


def haar_su3_from_key(key, counter_base: np.ndarray) -> np.ndarray:
    """Haar-random SU(3) matrices, one per entry of ``counter_base``.

    Gram-Schmidt (QR) of a complex Gaussian 3x3 with the diagonal of R made
    real positive gives a Haar U(3) matrix (Mezzadri, Notices AMS 54 (2007));
    dividing by the principal cube root of its determinant puts it in SU(3).
    Matrix m uses counters ``9*counter_base[m] + k`` for its 9 entries.
    """
    cb = np.asarray(counter_base, dtype=np.uint64)
    k = cb[:, None] * np.uint64(9) + np.arange(9, dtype=np.uint64)[None, :]
    z = rng.complex_normal(key, k).reshape(-1, 3, 3)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    q = q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(q)
    return q * np.exp(-1j * np.angle(det) / 3.0)[:, None, None]


def near_unit_su3_from_key(key, counter_base: np.ndarray, eps: float) -> np.ndarray:
    """SU(3) matrices exp(i*eps*H), H = sum_a h_a lambda_a/2, h_a ~ N(0,1).

    The exponential is taken through the Hermitian eigendecomposition
    H = V diag(w) V^dag, so exp(i eps H) = V diag(exp(i eps w)) V^dag.
    Matrix m uses counters ``8*counter_base[m] + a`` (a = 0..7), each a
    Box-Muller pair of which the first normal is kept.
    """
    cb = np.asarray(counter_base, dtype=np.uint64)
    k = cb[:, None] * np.uint64(8) + np.arange(8, dtype=np.uint64)[None, :]
    h, _ = rng.normal_pairs(key, k)
    H = np.einsum("ma,aij->mij", h, _GELL_MANN) * 0.5
    w, v = np.linalg.eigh(H)
    return np.einsum("mij,mj,mkj->mik", v, np.exp(1j * eps * w), v.conj())


def gauge_field(dims, seed: int, field_id: int = 1, kind: str = "haar", eps: float = 0.3,
                x3_range=None) -> np.ndarray:
    """Gauge links U_mu(x), shape ``(4, nx3, L2, L1, L0, 3, 3)``.

    ``kind`` is ``"haar"`` (Haar-random SU(3)), ``"near_unit"``
    (exp(i eps H)) or ``"unit"`` (all links the identity).
    Link (mu, site) draws from counter base ``mu * V + site``.
    """
    sites, shp = _slice_sites(dims, x3_range)
    V = int(np.prod(dims))
    out = np.empty((4,) + shp + (3, 3), dtype=np.complex128)
    key = rng.stream_key(seed, field_id)
    for mu in range(4):
        base = np.uint64(mu * V) + sites
        if kind == "haar":
            m = haar_su3_from_key(key, base)
        elif kind == "near_unit":
            m = near_unit_su3_from_key(key, base, eps)
        elif kind == "unit":
            m = np.broadcast_to(np.eye(3, dtype=np.complex128), (len(sites), 3, 3))
        else:
            raise ValueError(f"unknown link kind {kind!r}")
        out[mu] = m.reshape(shp + (3, 3))
    return out


def gauge_transform(dims, seed: int, field_id: int = 7, x3_range=None) -> np.ndarray:
    """Haar-random SU(3) g(x) per site, shape ``(nx3, L2, L1, L0, 3, 3)``."""
    sites, shp = _slice_sites(dims, x3_range)
    g = haar_su3_from_key(rng.stream_key(seed, field_id), sites)
    return g.reshape(shp + (3, 3))


def periodic_distance(dims, x0, x3_range=None) -> np.ndarray:
    """Euclidean minimal-image distance |x - x0| on the periodic 4-torus."""
    L0, L1, L2, L3 = dims
    lo, hi = (0, L3) if x3_range is None else x3_range
    comps = []
    for mu, (L, rng_mu) in enumerate(zip(dims, (range(L0), range(L1), range(L2), range(lo, hi)))):
        d = np.abs(np.asarray(list(rng_mu)) - x0[mu]) % L
        comps.append(np.minimum(d, L - d).astype(np.float64))
    d0, d1, d2, d3 = comps
    r2 = (d3[:, None, None, None] ** 2 + d2[None, :, None, None] ** 2
          + d1[None, None, :, None] ** 2 + d0[None, None, None, :] ** 2)
    return np.sqrt(r2)


def propagator(dims, seed: int, field_id: int = 2, x0=(0, 0, 0, 0), envelope: float | None = 0.5,
               x3_range=None) -> np.ndarray:
    """Synthetic LatticePropagator, shape ``(nx3, L2, L1, L0, 4, 3, 4, 3)``.

    Entries are complex Gaussians (E|z|^2 = 1) times ``exp(-envelope * |x - x0|)``
    with the minimal-image distance; ``envelope=None`` leaves them unscaled.
    Entry (site, k) with k = 0..143 in canonical order uses counter
    ``144 * site + k``.
    """
    sites, shp = _slice_sites(dims, x3_range)
    k = sites[:, None] * np.uint64(144) + np.arange(144, dtype=np.uint64)[None, :]
    z = rng.complex_normal(rng.stream_key(seed, field_id), k).reshape(shp + (4, 3, 4, 3))
    if envelope is not None:
        w = np.exp(-envelope * periodic_distance(dims, x0, x3_range))
        z *= w[..., None, None, None, None]
    return z


def fermion(dims, seed: int, field_id: int = 3, x3_range=None) -> np.ndarray:
    """Gaussian LatticeFermion, shape ``(nx3, L2, L1, L0, 4, 3)``; counter ``12*site + k``."""
    sites, shp = _slice_sites(dims, x3_range)
    k = sites[:, None] * np.uint64(12) + np.arange(12, dtype=np.uint64)[None, :]
    return rng.complex_normal(rng.stream_key(seed, field_id), k).reshape(shp + (4, 3))


def round_to_f32(a: np.ndarray) -> np.ndarray:
    """Round a complex128 field to complex64 (RNE) and widen it back.

    Both the GPU path (which stores the complex64 values) and the FP64
    checker consume exactly these values, so parity measures arithmetic only.
    """
    return a.astype(np.complex64).astype(np.complex128)
