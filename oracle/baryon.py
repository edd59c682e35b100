"""Baryon two-point functions by explicit Wick contraction (FP64 checker).

The paper's hadron-spectrum stage is "mesonic and baryonic" (Sec. 5); it
prints no contraction.  This module writes the baryon correlators as the
Wick contraction of the interpolating operators, with every term's sign taken
from the Grassmann ordering, not typed in:

* nucleon (uud): chi_alpha = eps_abc (u_a^T C g5 d_b) u_c,alpha;
* Delta++ (uuu): chi_alpha = eps_abc (u_a^T C g_k u_b) u_c,alpha, k = 3;

with C = gamma_2 gamma_4 and the conjugate operator
chibar_alpha' = eps_a'b'c' ubar_c',alpha' (qbar_b' Gbar qbar_a'^T),
Gbar = gamma_4 G^dag gamma_4, whose Grassmann order is (c', b', a').  The
correlator is

    C(t, p) = sum_{x in t} exp(-i p.(x - x0)) sum_{alpha alpha'} P_{alpha' alpha}
              < chi_alpha(x) chibar_alpha'(x0) >

with the parity projector P = (1 + parity * gamma_4) / 2 and
< q_{i s}(x) qbar_{j s'}(x0) > = S^{ij}_{s s'}(x) the propagator (colour i, j;
spin s, s').  Overall sign and normalisation are a convention: the fully
nested pairing (each quark with the antiquark in the mirrored position) has
sign +1.

Readings taken where the paper is silent: the Cg5 nucleon and the Cg_3 Delta
interpolators above, no spin-3/2 projection of the Delta, no
normalisation; p and the origin as for the mesons.
"""
from __future__ import annotations

import itertools

import numpy as np

from .gamma import C, GAMMA4, GAMMA5, GAMMAS
from .hadron import momentum_phases, timeslice_sum

EPS = np.zeros((3, 3, 3))
for _a, _b, _c in itertools.permutations(range(3)):
    EPS[_a, _b, _c] = np.linalg.det(np.eye(3)[[_a, _b, _c]])


def bar(G: np.ndarray) -> np.ndarray:
    """Gbar = gamma_4 G^dag gamma_4."""
    return GAMMA4 @ G.conj().T @ GAMMA4


def diquark_matrix(kind: str) -> np.ndarray:
    if kind == "nucleon":
        return C @ GAMMA5
    if kind == "delta":
        return C @ GAMMAS[2]      # gamma_3
    raise ValueError(f"unknown baryon {kind!r}")


def permutation_sign(order) -> int:
    """Sign of a permutation given as a sequence of distinct integers (inversion count)."""
    inv = sum(1 for i in range(len(order)) for j in range(i + 1, len(order)) if order[i] > order[j])
    return -1 if inv % 2 else 1


def pairings(sink_flavours, source_flavours):
    """All flavour-conserving pairings of sink quarks with source antiquarks.

    Fields are numbered in Grassmann order: sink quarks 0..2, then source
    antiquarks 3..5.  A pairing maps sink quark i to source antiquark
    pair[i].  Its sign is that of the permutation bringing the string into
    adjacent (quark, antiquark) pairs, q_0 qbar_pair[0] q_1 qbar_pair[1] ...
    """
    n = len(sink_flavours)
    out = []
    for perm in itertools.permutations(range(n)):
        if all(sink_flavours[i] == source_flavours[perm[i]] for i in range(n)):
            order = []
            for i in range(n):
                order += [i, n + perm[i]]
            out.append((perm, permutation_sign(order)))
    return out


def _operators(kind: str):
    """Sink (colour a, b, c / spin rho, sigma, alpha) and source (c', b', a' order) flavours."""
    if kind == "nucleon":
        return ("u", "d", "u"), ("u", "d", "u")
    return ("u", "u", "u"), ("u", "u", "u")


def baryon_site(Su: np.ndarray, Sd: np.ndarray, kind: str = "nucleon", parity: int = +1) -> np.ndarray:
    """sum_{alpha alpha'} P_{alpha'alpha} <chi_alpha(x) chibar_alpha'(x0)> at every site.

    S arrays have shape (..sites.., 4, 3, 4, 3) = [s, c, s', c'].  The sink
    string is q1_{a rho} q2_{b sigma} q3_{c alpha} with weight
    eps_abc G_{rho sigma}; the source string is qbar3_{c' alpha'}
    qbar2_{b' sigma'} qbar1_{a' rho'} with weight eps_a'b'c' Gbar_{sigma' rho'}.
    Each pairing contributes sign * S(q_i, qbar_pair(i)) products, summed over
    all colour and spin indices by einsum.
    """
    G = diquark_matrix(kind)
    Gb = bar(G)
    P = 0.5 * (np.eye(4) + parity * GAMMA4)
    sink_fl, src_fl = _operators(kind)
    # source antiquarks in Grassmann order: index 0 -> (c', alpha'), 1 -> (b', sigma'), 2 -> (a', rho')
    prop = {"u": Su, "d": Sd}
    # index letters: sink a b c (colour), r s A (spin rho sigma alpha); source x y z = c' b' a' colours,
    # B S R = alpha' sigma' rho' spins
    sink_idx = [("a", "r"), ("b", "s"), ("c", "A")]
    src_idx = [("x", "B"), ("y", "S"), ("z", "R")]
    total = 0
    for perm, sign in pairings(sink_fl, src_fl):
        ops = []
        subs = []
        for i in range(3):
            ci, si = sink_idx[i]
            cj, sj = src_idx[perm[i]]
            ops.append(prop[sink_fl[i]])
            subs.append(f"...{si}{ci}{sj}{cj}")
        expr = ",".join(subs) + ",abc,zyx,rs,SR,BA->..."
        term = np.einsum(expr, *ops, EPS, EPS, G, Gb, P, optimize=True)
        total = total + sign * term
    return total


def baryon_2pt(Su: np.ndarray, Sd: np.ndarray, kind: str = "nucleon", parity: int = +1, moms=((0, 0, 0),),
               j_decay: int = 3, origin=(0, 0, 0, 0)) -> np.ndarray:
    """Correlator, shape (n_mom, Nt) complex128."""
    if Su.shape != Sd.shape or Su.shape[4:] != (4, 3, 4, 3):
        raise ValueError("propagators must both have shape (..sites.., 4, 3, 4, 3)")
    L3, L2, L1, L0 = Su.shape[:4]
    dims = (L0, L1, L2, L3)
    c = baryon_site(Su, Sd, kind, parity)
    phases = momentum_phases(dims, moms, j_decay, origin)
    return np.array([timeslice_sum(c * phases[k], j_decay) for k in range(len(moms))])
