"""Pins of the FP64 checker against what the mathematics fixes (CPU only).

None of these re-uses the checker's own formula: they test closed forms,
algebraic identities, invariances and brute-force sums written separately.
"""
import itertools

import numpy as np
import pytest

from oracle import gamma, geometry, hadron, smear, source
from synth import fields

# ---------------------------------------------------------------------------
# Gamma basis


def test_gamma_clifford_and_hermiticity():
    for mu in range(4):
        g = gamma.GAMMAS[mu]
        assert np.array_equal(g, g.conj().T)
        for nu in range(4):
            anti = g @ gamma.GAMMAS[nu] + gamma.GAMMAS[nu] @ g
            assert np.array_equal(anti, 2.0 * (mu == nu) * np.eye(4))


def test_gamma5_is_diag_and_basis_is_signed_permutations():
    assert np.array_equal(gamma.GAMMA5, np.diag([1, 1, -1, -1]).astype(complex))
    assert np.array_equal(gamma.GAMMA5,
                          gamma.GAMMA1 @ gamma.GAMMA2 @ gamma.GAMMA3 @ gamma.GAMMA4)
    units = {1, -1, 1j, -1j}
    for n in range(16):
        g = gamma.Gamma(n)
        for row in g:
            nz = row[row != 0]
            assert len(nz) == 1 and complex(nz[0]) in units
    # orthogonality tr(Gamma_m^dag Gamma_n) = 4 delta_mn: the 16 are a basis
    gram = np.array([[np.trace(gamma.Gamma(m).conj().T @ gamma.Gamma(n)) for n in range(16)]
                     for m in range(16)])
    assert np.allclose(gram, 4 * np.eye(16))


def test_charge_conjugation():
    C = gamma.C
    Cinv = np.linalg.inv(C)
    for g in gamma.GAMMAS:
        assert np.allclose(C @ g @ Cinv, -g.T)
    assert np.allclose(C.T, -C)
    assert np.allclose(Cinv, C.T)


# ---------------------------------------------------------------------------
# shift


def test_shift_against_index_loop():
    dims = (3, 4, 5, 2)
    rng = np.random.default_rng(0)
    f = rng.normal(size=fields.site_shape(dims) + (2,))
    L0, L1, L2, L3 = dims
    for mu in range(4):
        for sign in (+1, -1):
            out = geometry.shift(f, sign, mu)
            for x0, x1, x2, x3 in itertools.product(range(L0), range(L1), range(L2), range(L3)):
                y = [x0, x1, x2, x3]
                y[mu] = (y[mu] + sign) % dims[mu]
                assert np.array_equal(out[x3, x2, x1, x0], f[y[3], y[2], y[1], y[0]])


def test_shift_identities():
    dims = (4, 3, 2, 5)
    f = np.random.default_rng(1).normal(size=fields.site_shape(dims) + (3,))
    for mu in range(4):
        assert np.array_equal(geometry.shift(geometry.shift(f, +1, mu), -1, mu), f)
        g = f
        for _ in range(dims[mu]):
            g = geometry.shift(g, +1, mu)
        assert np.array_equal(g, f)


# ---------------------------------------------------------------------------
# Smearing


def _plane_wave_factor(kappa, n_vec, dims, j_decay):
    return 1.0 + 2.0 * kappa * sum(np.cos(2 * np.pi * n_vec[mu] / dims[mu])
                                   for mu in range(4) if mu != j_decay)


@pytest.mark.parametrize("j_decay", [3, 1])
def test_smear_free_plane_wave(j_decay):
    """At U = 1 a plane wave is an eigenvector: factor (1 + 2 kappa sum cos p_i)^N."""
    dims = (4, 6, 3, 5)
    kappa, N = 0.17, 6
    U = fields.gauge_field(dims, 0, kind="unit")
    x = geometry.coords(dims)
    v = np.random.default_rng(2).normal(size=(4, 3, 4, 3)) + 0j
    for n_vec in [(1, 0, 0, 0), (0, 2, 1, 3), (3, 5, 2, 4), (2, 3, 1, 0)]:
        ph = np.exp(2j * np.pi * sum(n_vec[mu] * x[..., mu] / dims[mu] for mu in range(4)))
        psi = ph[..., None, None, None, None] * v
        out = smear.gauss_smear(U, psi, kappa, N, j_decay)
        expect = _plane_wave_factor(kappa, n_vec, dims, j_decay) ** N * psi
        # rounding scales with the intermediate norms, bounded by (1 + 6 kappa)^N |psi|
        tol = 1e-13 * (1 + 6 * kappa) ** N * np.abs(psi).max()
        assert np.allclose(out, expect, rtol=0, atol=tol)


def _free_point_profile(dims3, kappa, N, r):
    """f(r) = V3^-1 sum_p exp(i p.r) (1 + 2 kappa sum_i cos p_i)^N, written as a sum."""
    V3 = int(np.prod(dims3))
    total = 0.0 + 0.0j
    for n in itertools.product(*(range(L) for L in dims3)):
        p = [2 * np.pi * n[i] / dims3[i] for i in range(3)]
        F = 1 + 2 * kappa * sum(np.cos(pi) for pi in p)
        total += np.exp(1j * sum(p[i] * r[i] for i in range(3))) * F ** N
    return total / V3


def test_smear_free_point_source_closed_form():
    dims = (4, 3, 5, 3)
    kappa, N, x0 = 0.23, 4, (1, 2, 0, 1)
    U = fields.gauge_field(dims, 0, kind="unit")
    S = smear.gauss_smear(U, source.point_propagator(dims, x0), kappa, N)
    eye = np.eye(12).reshape(4, 3, 4, 3)
    for x1, x2, x0_ in itertools.product(range(dims[1]), range(dims[2]), range(dims[0])):
        r = ((x0_ - x0[0]) % dims[0], (x1 - x0[1]) % dims[1], (x2 - x0[2]) % dims[2])
        f = _free_point_profile(dims[:3], kappa, N, r)
        assert np.allclose(S[x0[3], x2, x1, x0_], f * eye, atol=1e-12)
    other = [t for t in range(dims[3]) if t != x0[3]]
    assert np.all(S[other] == 0)


def _dense_hop(U, dims, j_decay):
    """(3V x 3V) hop matrix from explicit coordinate loops (adds, never dedups)."""
    L0, L1, L2, L3 = dims
    V = L0 * L1 * L2 * L3

    def idx(x):
        return x[0] + L0 * (x[1] + L1 * (x[2] + L2 * x[3]))

    H = np.zeros((3 * V, 3 * V), dtype=complex)
    for x in itertools.product(range(L0), range(L1), range(L2), range(L3)):
        i = idx(x)
        for mu in range(4):
            if mu == j_decay:
                continue
            y = list(x)
            y[mu] = (x[mu] + 1) % dims[mu]
            z = list(x)
            z[mu] = (x[mu] - 1) % dims[mu]
            Ux = U[mu, x[3], x[2], x[1], x[0]]
            Uz = U[mu, z[3], z[2], z[1], z[0]]
            H[3 * i:3 * i + 3, 3 * idx(y):3 * idx(y) + 3] += Ux
            H[3 * i:3 * i + 3, 3 * idx(z):3 * idx(z) + 3] += Uz.conj().T
    return H


@pytest.mark.parametrize("dims,j_decay", [((2, 2, 2, 4), 3), ((3, 3, 3, 4), 3), ((2, 3, 2, 3), 0)])
def test_smear_brute_force_dense(dims, j_decay):
    kappa, N = 0.21, 5
    U = fields.gauge_field(dims, 5, kind="haar")
    psi = fields.fermion(dims, 5)
    H = _dense_hop(U, dims, j_decay)
    V = int(np.prod(dims))
    # canonical (..sites.., spin, colour) -> vector index (site, colour) per spin
    vec = psi.reshape(V, 4, 3).transpose(1, 0, 2).reshape(4, 3 * V).T
    M = np.eye(3 * V) + kappa * H
    for _ in range(N):
        vec = M @ vec
    expect = vec.T.reshape(4, V, 3).transpose(1, 0, 2).reshape(psi.shape)
    out = smear.gauss_smear(U, psi, kappa, N, j_decay)
    assert np.allclose(out, expect, rtol=1e-13, atol=1e-13 * np.abs(expect).max())


def _gauge_links(U, g):
    """U^g_mu(x) = g(x) U_mu(x) g(x + mu)^dag."""
    out = np.empty_like(U)
    for mu in range(4):
        g_fwd = geometry.shift(g, +1, mu)
        out[mu] = g @ U[mu] @ np.conj(np.swapaxes(g_fwd, -1, -2))
    return out


def test_smear_gauge_covariance():
    dims = (4, 3, 5, 4)
    U = fields.gauge_field(dims, 11, kind="haar")
    g = fields.gauge_transform(dims, 11)
    S = fields.propagator(dims, 11, envelope=None)
    kappa, N = 0.3, 3
    Ug = _gauge_links(U, g)
    Sg = np.einsum("tzyxab,tzyxsbrc->tzyxsarc", g, S)
    lhs = smear.gauss_smear(Ug, Sg, kappa, N)
    rhs = np.einsum("tzyxab,tzyxsbrc->tzyxsarc", g, smear.gauss_smear(U, S, kappa, N))
    assert np.allclose(lhs, rhs, atol=1e-12 * np.abs(rhs).max())
    # and a plausible mistake (U instead of U^dag on the backward hop) is not covariant
    assert not np.allclose(smear.gauss_smear(U, S, kappa, N),
                           smear.gauss_smear(U.conj(), S, kappa, N))


# ---------------------------------------------------------------------------
# Mesons


def test_pion_is_sum_of_squares():
    dims = (3, 4, 2, 5)
    S = fields.propagator(dims, 3)
    C = hadron.meson_2pt(S, S, [(15, 15)])[0, 0]
    expect = np.sum(np.abs(S) ** 2, axis=(1, 2, 3, 4, 5, 6, 7))
    # each |z|^2 is real up to one rounding (numpy may fuse the complex product)
    assert np.all(np.abs(C.imag) <= 1e-14 * C.real)
    assert np.all(C.real > 0)
    assert np.allclose(C.real, expect, rtol=1e-14)


def test_meson_completeness_sum_rule():
    """sum_n tr[G_n S1 G_n^dag g5 S2^dag g5] = 4 sum_ab tr_s(S1^ab) conj(tr_s(S2^ab))."""
    dims = (2, 3, 2, 4)
    S1 = fields.propagator(dims, 4, field_id=21, envelope=None)
    S2 = fields.propagator(dims, 4, field_id=22, envelope=None)
    tot = sum(hadron.meson_site(S1, S2, n, n) for n in range(16))
    tr1 = np.einsum("tzyxsasb->tzyxab", S1)
    tr2 = np.einsum("tzyxsasb->tzyxab", S2)
    expect = 4 * np.sum(tr1 * np.conj(tr2), axis=(-2, -1))
    assert np.allclose(tot, expect, atol=1e-12 * np.abs(expect).max())


def test_meson_factorised_spin_colour():
    """For S1 = G_a (x) A and S2 = G_b (x) B the site trace factorises."""
    dims = (2, 2, 2, 2)
    rng = np.random.default_rng(9)
    A = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
    B = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
    for a, b, snk, src in [(3, 5, 7, 7), (15, 0, 15, 15), (1, 14, 2, 11), (6, 9, 12, 4)]:
        # S[s c s' c'] = G[s s'] A[c c']
        s1 = np.einsum("ij,ab->iajb", gamma.Gamma(a), A)
        s2 = np.einsum("ij,ab->iajb", gamma.Gamma(b), B)
        S1 = np.broadcast_to(s1, fields.site_shape(dims) + s1.shape)
        S2 = np.broadcast_to(s2, fields.site_shape(dims) + s2.shape)
        c = hadron.meson_site(S1, S2, snk, src)
        g5 = gamma.GAMMA5
        spin = np.trace(gamma.Gamma(snk) @ gamma.Gamma(a) @ gamma.Gamma(src).conj().T
                        @ g5 @ gamma.Gamma(b).conj().T @ g5)
        colour = np.trace(A @ B.conj().T)
        assert np.allclose(c, spin * colour)


def test_meson_gauge_invariance():
    dims = (3, 2, 4, 3)
    S1 = fields.propagator(dims, 5, field_id=31)
    S2 = fields.propagator(dims, 5, field_id=32)
    g = fields.gauge_transform(dims, 5)
    x0 = (1, 0, 2, 1)
    g0 = g[x0[3], x0[2], x0[1], x0[0]]

    def transform(S):
        return np.einsum("tzyxab,tzyxsbrc,dc->tzyxsard", g, S, g0.conj())

    ch = hadron.SIXTEEN_MESONS + ((3, 12), (5, 10))
    moms = ((0, 0, 0), (1, 0, 1), (2, 1, 3))
    a = hadron.meson_2pt(S1, S2, ch, moms)
    b = hadron.meson_2pt(transform(S1), transform(S2), ch, moms)
    assert np.allclose(a, b, atol=1e-12 * np.abs(a).max())


def test_free_point_source_mesons_parseval():
    """At U = 1 the smeared point source is f(x) 1_12: every channel is 12 sum f^2,
    and by Parseval the pion at t0 is (12/V3) sum_p F(p)^{2N}, zero elsewhere."""
    dims = (4, 4, 3, 4)
    kappa, N = 0.25, 5
    U = fields.gauge_field(dims, 0, kind="unit")
    S = smear.gauss_smear(U, source.point_propagator(dims), kappa, N)
    C = hadron.meson_2pt(S, S, hadron.SIXTEEN_MESONS)[:, 0, :]
    V3 = dims[0] * dims[1] * dims[2]
    parseval = 0.0
    for n in itertools.product(*(range(L) for L in dims[:3])):
        F = 1 + 2 * kappa * sum(np.cos(2 * np.pi * n[i] / dims[i]) for i in range(3))
        parseval += F ** (2 * N)
    parseval *= 12.0 / V3
    assert np.allclose(C[:, 0], parseval, rtol=1e-12)
    assert np.all(C[:, 1:] == 0)


def test_momentum_projection_equals_fft():
    dims = (4, 3, 5, 2)
    S1 = fields.propagator(dims, 6, field_id=41, envelope=None)
    S2 = fields.propagator(dims, 6, field_id=42, envelope=None)
    moms = list(itertools.product(range(dims[0]), range(dims[1]), range(dims[2])))
    C = hadron.meson_2pt(S1, S2, [(5, 9)], moms)[0]          # (n_mom, Nt)
    c = hadron.meson_site(S1, S2, 5, 9)                      # (t, z, y, x)
    F = np.fft.fftn(c, axes=(1, 2, 3))                       # index [t, kz, ky, kx]
    for k, (nx, ny, nz) in enumerate(moms):
        assert np.allclose(C[k], F[:, nz, ny, nx], atol=1e-12 * np.abs(F).max())
    # p = 0 is the plain timeslice sum
    assert np.allclose(C[moms.index((0, 0, 0))], c.sum(axis=(1, 2, 3)))


def test_pion_reflection_symmetry():
    dims = (4, 4, 4, 3)
    S = fields.propagator(dims, 8, envelope=0.3)
    moms = ((1, 0, 0), (-1, 0, 0), (1, 2, -1), (-1, -2, 1))
    C = hadron.meson_2pt(S, S, [(15, 15)], moms)[0]
    assert np.allclose(C[1], np.conj(C[0]))
    assert np.allclose(C[3], np.conj(C[2]))
