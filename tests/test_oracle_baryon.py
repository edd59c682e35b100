"""Pins of the FP64 baryon contractions (CPU only)."""
import itertools

import numpy as np
import pytest

from oracle import baryon
from oracle.gamma import GAMMA4
from synth import fields


def test_wick_signs_from_grassmann_order():
    nuc = baryon.pairings(("u", "d", "u"), ("u", "d", "u"))
    assert sorted(perm for perm, _ in nuc) == [(0, 1, 2), (2, 1, 0)]
    signs = dict(nuc)
    assert signs[(2, 1, 0)] == +1            # fully nested pairing
    assert signs[(0, 1, 2)] == -1            # u-quark exchange
    delta = baryon.pairings(("u", "u", "u"), ("u", "u", "u"))
    assert len(delta) == 6 and sum(s for _, s in delta) == 0


def test_wick_sum_is_a_determinant():
    """For one flavour the signed sum over pairings of prod S(q_i, qbar_pi(i)) is,
    up to the sign of the nested reference, det of the 3x3 matrix S(q_i, qbar_j)."""
    rng = np.random.default_rng(3)
    for _ in range(5):
        M = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
        wick = sum(sign * np.prod([M[i, perm[i]] for i in range(3)])
                   for perm, sign in baryon.pairings(("u",) * 3, ("u",) * 3))
        assert np.isclose(wick, -np.linalg.det(M))


@pytest.mark.parametrize("kind", ["nucleon", "delta"])
def test_baryon_gauge_invariance(kind):
    dims = (2, 3, 2, 3)
    Su = fields.propagator(dims, 7, field_id=81, envelope=None)
    Sd = fields.propagator(dims, 7, field_id=82, envelope=None)
    g = fields.gauge_transform(dims, 7)
    x0 = (1, 2, 0, 1)
    g0 = g[x0[3], x0[2], x0[1], x0[0]]

    def transform(S):
        return np.einsum("tzyxab,tzyxsbrc,dc->tzyxsard", g, S, g0.conj())

    a = baryon.baryon_2pt(Su, Sd, kind, +1, ((0, 0, 0), (1, 0, 1)))
    b = baryon.baryon_2pt(transform(Su), transform(Sd), kind, +1, ((0, 0, 0), (1, 0, 1)))
    assert np.allclose(a, b, atol=1e-12 * np.abs(a).max())
    if kind == "delta":
        return  # three identical quarks antisymmetrise any colour tensor back to epsilon
    # and a colour mistake (a cyclic-only tensor instead of epsilon) is not invariant
    saved = baryon.EPS.copy()
    try:
        baryon.EPS[...] = 0
        for i in range(3):
            baryon.EPS[i, (i + 1) % 3, (i + 2) % 3] = 1
        c = baryon.baryon_site(transform(Su), transform(Sd), kind)
        d = baryon.baryon_site(Su, Sd, kind)
        assert not np.allclose(c, d)
    finally:
        baryon.EPS[...] = saved


@pytest.mark.parametrize("kind", ["nucleon", "delta"])
def test_static_quarks_have_positive_parity(kind):
    """Forward static quarks, S = delta_ij (1 + g4)/2: the negative-parity
    projection vanishes exactly, the positive one does not."""
    dims = (2, 2, 2, 2)
    Pp = 0.5 * (np.eye(4) + GAMMA4)
    S1 = np.einsum("st,ab->satb", Pp, np.eye(3))
    S = np.broadcast_to(S1, fields.site_shape(dims) + S1.shape).copy()
    neg = baryon.baryon_site(S, S, kind, -1)
    pos = baryon.baryon_site(S, S, kind, +1)
    assert np.all(np.abs(neg) < 1e-14)
    assert np.all(np.abs(pos) > 1e-3)


def test_parity_projectors_add_up():
    """P+ + P- = 1: the two projections sum to the unprojected spin trace."""
    dims = (2, 2, 2, 2)
    Su = fields.propagator(dims, 9, field_id=83, envelope=None)
    Sd = fields.propagator(dims, 9, field_id=84, envelope=None)
    for kind in ("nucleon", "delta"):
        plus = baryon.baryon_site(Su, Sd, kind, +1)
        minus = baryon.baryon_site(Su, Sd, kind, -1)
        saved = GAMMA4.copy()
        # unprojected: P = 1 -> parity 0 gives P = 1/2, so twice that
        both = 2 * baryon.baryon_site(Su, Sd, kind, 0)
        assert np.allclose(plus + minus, both)
        assert np.array_equal(GAMMA4, saved)


def _brute_site(Su, Sd, kind, parity):
    """Loop-and-determinant evaluation at one site (independent of the einsum engine)."""
    G = baryon.diquark_matrix(kind)
    Gb = baryon.bar(G)
    P = 0.5 * (np.eye(4) + parity * GAMMA4)
    eps = [(p, baryon.EPS[p]) for p in itertools.permutations(range(3))]
    total = 0j
    spins = list(itertools.product(range(4), repeat=6))
    for (a, b, c), e1 in eps:
        for (ap, bp, cp), e2 in eps:
            Ms, ws = [], []
            for r, s, al, rp, sp, alp in spins:
                w = e1 * e2 * G[r, s] * Gb[sp, rp] * P[alp, al]
                if w == 0:
                    continue
                sink = [(r, a), (s, b), (al, c)]
                src = [(alp, cp), (sp, bp), (rp, ap)]      # Grassmann order c', b', a'
                if kind == "delta":
                    M = np.array([[Su[si, ci, sj, cj] for (sj, cj) in src] for (si, ci) in sink])
                    Ms.append(-M)                              # nested reference sign
                else:
                    u = [[Su[sink[i][0], sink[i][1], src[j][0], src[j][1]] for j in (2, 0)] for i in (0, 2)]
                    d = Sd[sink[1][0], sink[1][1], src[1][0], src[1][1]]
                    Ms.append(np.array([[d * u[0][0], d * u[0][1]], [u[1][0], u[1][1]]]))
                ws.append(w)
            if ws:
                dets = np.linalg.det(np.array(Ms)) if kind == "nucleon" else -np.linalg.det(-np.array(Ms))
                total += np.sum(np.array(ws) * dets)
    return total


@pytest.mark.parametrize("kind,parity", [("nucleon", 1), ("delta", 1), ("nucleon", -1)])
def test_baryon_engine_matches_loop_determinant(kind, parity):
    dims = (1, 1, 1, 1)
    Su = fields.propagator(dims, 11, field_id=85, envelope=None)
    Sd = fields.propagator(dims, 11, field_id=86, envelope=None)
    engine = baryon.baryon_site(Su, Sd, kind, parity)[0, 0, 0, 0]
    brute = _brute_site(Su[0, 0, 0, 0], Sd[0, 0, 0, 0], kind, parity)
    assert np.isclose(engine, brute, rtol=1e-10)
