"""The FP64 checker spread over the host's cores (test infrastructure).

Each function computes an exact slice of a checker result, so a spawned
process pool can work on them side by side and the caller assembles them:
Gaussian smearing acts on colour only and never couples timeslices, so each
source column (s', c') of a propagator on one timeslice smears on its own;
the meson and baryon contractions are site-local, so channels and slabs of
sites split freely.  Large arrays travel as .npy files (memory-mapped by the
workers) rather than through the pool's pipes.

Start the pool with the "spawn" method (``pool()``): a child forked from a
process that has initialised CUDA can hang.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

from oracle import baryon, hadron, smear


def pool(n: int | None = None):
    """A spawned process pool with one worker per host core (or n)."""
    return mp.get_context("spawn").Pool(n or os.cpu_count() or 1)


def smear_column(U_path: str, col: np.ndarray, kappa: float, n_iter: int) -> np.ndarray:
    """(1 + kappa H)^N of one source column (shape (..sites.., 4, 3)) on the links in U_path."""
    U = np.load(U_path, mmap_mode="r")
    return smear.gauss_smear(np.asarray(U), col, kappa, n_iter, 3)


def smear_propagator(p, U_path: str, P: np.ndarray, kappa: float, n_iter: int) -> list:
    """Submit the 12 source columns of propagator P (..sites.., 4, 3, 4, 3) to pool p;
    returns the async results in column order (s' * 3 + c')."""
    return [p.apply_async(smear_column, (U_path, np.ascontiguousarray(P[..., sp, cp]), kappa, n_iter))
            for sp in range(4) for cp in range(3)]


def gather_propagator(results) -> np.ndarray:
    """Reassemble the columns submitted by smear_propagator."""
    cols = [r.get() for r in results]
    return np.stack(cols, axis=-1).reshape(cols[0].shape + (4, 3))


def meson_channels(path_a: str, path_b: str, channels, moms) -> tuple[np.ndarray, np.ndarray]:
    """Projected correlators (n_chan, n_mom, Nt) of S_a, S_b and, per channel and t,
    A(t) = sum_x |c(x)| (the scale of the momentum sums)."""
    Sa = np.asarray(np.load(path_a, mmap_mode="r"))
    Sb = np.asarray(np.load(path_b, mmap_mode="r"))
    C = hadron.meson_2pt(Sa, Sb, channels, moms, j_decay=3)
    A = np.stack([hadron.timeslice_sum(np.abs(hadron.meson_site(Sa, Sb, a, b)), 3) for a, b in channels])
    return C, A


def nucleon_slab(path_a: str, path_b: str, z0: int, z1: int, parity: int = +1) -> np.ndarray:
    """Nucleon site values (u = S_a, d = S_b) on the sites with x2 in [z0, z1)."""
    Sa = np.asarray(np.load(path_a, mmap_mode="r")[:, z0:z1])
    Sb = np.asarray(np.load(path_b, mmap_mode="r")[:, z0:z1])
    return baryon.baryon_site(Sa, Sb, kind="nucleon", parity=parity)


def timeslice_chain(U_path: str, P_path: str, t: int, kappa: float, n_iter: int, channels, keep_field: bool):
    """Smear timeslice t of the propagator in P_path on the links in U_path
    (complex64 canonical arrays, widened to FP64) and contract the meson
    channels at p = 0; returns (C_t per channel, the smeared timeslice or None)."""
    U = np.load(U_path, mmap_mode="r")
    P = np.load(P_path, mmap_mode="r")
    Ut = np.asarray(U[:, t:t + 1]).astype(np.complex128)
    Pt = np.asarray(P[t:t + 1]).astype(np.complex128)
    S = smear.gauss_smear(Ut, Pt, kappa, n_iter, 3)
    C = hadron.meson_2pt(S, S, channels)[:, 0, 0]
    return C, (S if keep_field else None)
