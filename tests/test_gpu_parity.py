"""CUDA path against the FP64 checker, element by element, through the C ABI.

Every input is seeded synthetic data rounded to complex64 (or bfloat16 for
BF16 storage) on the host; the checker consumes the same rounded values.
"""
import numpy as np
import pytest
import torch

from oracle import geometry, hadron, smear, source
from synth import configs, fields
from tests.parity_util import TOL_BF16, TOL_F32, corr_err, field_err, to_bf16_complex

pytestmark = pytest.mark.gpu


def dev():
    return torch.device("cuda:0")


def upload(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def make_field(q, lat, kind, prec, canon):
    return q.Field(lat, kind, prec, device=dev()).import_(upload(canon.astype(np.complex64)))


def export(f) -> np.ndarray:
    return f.export().cpu().numpy()


# ---------------------------------------------------------------------------
# field setup


@pytest.mark.parametrize("kind", ["gauge", "propagator", "fermion", "colour"])
def test_import_export_roundtrip(qdpg_gpu, kind):
    q = qdpg_gpu
    dims = (3, 5, 2, 4)
    lat = q.Lattice(dims, 3)
    rng = np.random.default_rng(1)
    K = {"gauge": q.GAUGE, "propagator": q.PROPAGATOR, "fermion": q.FERMION, "colour": q.COLOR_MATRIX}[kind]
    shp = lat.canonical_shape(K)
    a = fields.round_to_f32(rng.normal(size=shp) + 1j * rng.normal(size=shp))
    assert np.array_equal(export(make_field(q, lat, K, q.F32, a)), a)
    assert np.array_equal(export(make_field(q, lat, K, q.BF16, a)), to_bf16_complex(a))
    # a complex128 canonical buffer gives the same storage as the complex64 one
    f64 = q.Field(lat, K, q.F32, device=dev()).import_(upload(a))
    assert np.array_equal(export(f64), a)


def test_reconstruct12_links(qdpg_gpu):
    q = qdpg_gpu
    dims = (4, 3, 5, 2)
    lat = q.Lattice(dims, 3)
    U = fields.round_to_f32(fields.gauge_field(dims, 3, kind="haar"))
    r = export(make_field(q, lat, q.GAUGE, q.F32_R12, U))
    assert np.array_equal(r[..., :2, :], U[..., :2, :])         # rows 0, 1 stored exactly
    assert np.abs(r[..., 2, :] - U[..., 2, :]).max() < 1e-6      # row 2 = (row0 x row1)^*
    rb = export(make_field(q, lat, q.GAUGE, q.BF16_R12, U))
    assert np.array_equal(rb[..., :2, :], to_bf16_complex(U[..., :2, :]))
    assert np.abs(rb[..., 2, :] - U[..., 2, :]).max() < 2e-2


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_point_source_exact(qdpg_gpu, prec):
    q = qdpg_gpu
    dims = (4, 3, 5, 6)
    lat = q.Lattice(dims, 3)
    p = q.PREC_NAMES[prec]
    x0 = (3, 1, 4, 2)
    S = q.point_source(q.Field(lat, q.PROPAGATOR, p, device=dev()), x0)
    assert np.array_equal(export(S), source.point_propagator(dims, x0))
    F = q.point_source(q.Field(lat, q.FERMION, p, device=dev()), x0, spin_color=7)
    assert np.array_equal(export(F), source.point_fermion(dims, x0, spin=2, color=1))


# ---------------------------------------------------------------------------
# shift


@pytest.mark.parametrize("dims,jd", [((3, 4, 5, 6), 3), ((4, 3, 2, 5), 1), ((2, 1, 3, 4), 0)])
def test_shift_bit_exact(qdpg_gpu, dims, jd):
    q = qdpg_gpu
    lat = q.Lattice(dims, jd)
    F = fields.round_to_f32(fields.fermion(dims, 2))
    P = to_bf16_complex(fields.round_to_f32(fields.propagator(dims, 2, envelope=None)))
    U = fields.round_to_f32(fields.gauge_field(dims, 2, kind="haar"))
    cases = [(q.FERMION, q.F32, F), (q.PROPAGATOR, q.BF16, P), (q.GAUGE, q.F32, U)]
    for kind, prec, canon in cases:
        src = make_field(q, lat, kind, prec, canon)
        dst = src.like()
        for mu in range(4):
            for sign in (+1, -1):
                q.shift(dst, src, sign, mu)
                got = export(dst)
                if kind == q.GAUGE:
                    expect = np.stack([geometry.shift(canon[m], sign, mu) for m in range(4)])
                else:
                    expect = geometry.shift(canon, sign, mu)
                assert np.array_equal(got, expect), (kind, prec, mu, sign)
    # shift(+mu) then shift(-mu) is the identity, bit for bit
    src = make_field(q, lat, q.FERMION, q.F32, F)
    a, b = src.like(), src.like()
    q.shift(a, src, +1, 2)
    q.shift(b, a, -1, 2)
    assert np.array_equal(export(b), F)


# ---------------------------------------------------------------------------
# Gaussian smearing

SMEAR_CASES = [
    # dims, lattice j_decay, smear j_decay, kind, links, kappa, N, pass scratch
    ((4, 4, 4, 8), 3, 3, "prop", "haar", 0.25, 5, True),
    ((6, 5, 3, 4), 3, 3, "prop", "near_unit", 0.21, 4, False),     # V3 = 90: ragged block
    ((2, 2, 2, 4), 3, 3, "ferm", "haar", 0.3, 6, True),            # L = 2: x+i == x-i
    ((1, 3, 2, 4), 3, 3, "ferm", "haar", 0.2, 3, True),            # L = 1: x+i == x
    ((5, 4, 3, 6), 1, 1, "prop", "haar", 0.17, 3, True),           # other decay direction
    ((5, 4, 3, 6), 3, 0, "ferm", "haar", 0.17, 4, True),           # smear across timeslices
    ((12, 12, 12, 4), 3, 3, "prop", "near_unit", 0.21, 9, True),   # several blocks per timeslice
]


@pytest.mark.parametrize("case", SMEAR_CASES, ids=lambda c: f"{c[0]}-jd{c[1]}{c[2]}-{c[3]}-N{c[6]}")
def test_smear_f32_vs_oracle(qdpg_gpu, case):
    q = qdpg_gpu
    dims, jd_lat, jd, kind, links, kappa, N, with_scratch = case
    lat = q.Lattice(dims, jd_lat)
    U = fields.round_to_f32(fields.gauge_field(dims, 4, kind=links))
    if kind == "prop":
        psi = fields.round_to_f32(fields.propagator(dims, 4, envelope=0.3))
        K = q.PROPAGATOR
    else:
        psi = fields.round_to_f32(fields.fermion(dims, 4))
        K = q.FERMION
    Uf = make_field(q, lat, q.GAUGE, q.F32, U)
    f = make_field(q, lat, K, q.F32, psi)
    q.gauss_smear(Uf, f, kappa, N, jd, scratch=f.like() if with_scratch else None)
    ref = smear.gauss_smear(U, psi, kappa, N, jd)
    assert field_err(export(f), ref) <= TOL_F32


def test_smear_zero_and_one_iteration(qdpg_gpu):
    q = qdpg_gpu
    dims = (4, 3, 5, 2)
    lat = q.Lattice(dims, 3)
    U = fields.round_to_f32(fields.gauge_field(dims, 6, kind="haar"))
    psi = fields.round_to_f32(fields.propagator(dims, 6, envelope=None))
    Uf = make_field(q, lat, q.GAUGE, q.F32, U)
    f = make_field(q, lat, q.PROPAGATOR, q.F32, psi)
    q.gauss_smear(Uf, f, 0.3, 0)
    assert np.array_equal(export(f), psi)
    q.gauss_smear(Uf, f, 0.3, 1, scratch=f.like())
    assert field_err(export(f), smear.gauss_smear(U, psi, 0.3, 1)) <= TOL_F32


@pytest.mark.parametrize("links", ["f32_r12", "bf16_r12", "bf16"])
def test_smear_compressed_links(qdpg_gpu, links):
    q = qdpg_gpu
    dims = (6, 4, 4, 4)
    lat = q.Lattice(dims, 3)
    U = fields.round_to_f32(fields.gauge_field(dims, 8, kind="near_unit"))
    psi = fields.round_to_f32(fields.propagator(dims, 8, envelope=0.3))
    Uf = make_field(q, lat, q.GAUGE, q.PREC_NAMES[links], U)
    f = make_field(q, lat, q.PROPAGATOR, q.F32, psi)
    q.gauss_smear(Uf, f, 0.21, 6, scratch=f.like())
    err = field_err(export(f), smear.gauss_smear(U, psi, 0.21, 6))
    assert err <= (TOL_F32 if links == "f32_r12" else TOL_BF16)


def test_smear_bf16_storage(qdpg_gpu):
    q = qdpg_gpu
    dims = (8, 8, 8, 4)
    lat = q.Lattice(dims, 3)
    U = fields.round_to_f32(fields.gauge_field(dims, 9, kind="near_unit"))
    psi = fields.round_to_f32(fields.propagator(dims, 9, envelope=0.5))
    Uf = make_field(q, lat, q.GAUGE, q.BF16_R12, U)
    f = make_field(q, lat, q.PROPAGATOR, q.BF16, psi)
    q.gauss_smear(Uf, f, 0.21, 20, scratch=f.like())
    err = field_err(export(f), smear.gauss_smear(U, psi, 0.21, 20))
    assert err <= TOL_BF16


# ---------------------------------------------------------------------------
# mesons


@pytest.mark.parametrize("dims", [(4, 4, 4, 8), (5, 3, 7, 6)])
def test_sixteen_mesons_vs_oracle(qdpg_gpu, dims):
    q = qdpg_gpu
    lat = q.Lattice(dims, 3)
    S1 = fields.round_to_f32(fields.propagator(dims, 10, field_id=51, envelope=0.4))
    S2 = fields.round_to_f32(fields.propagator(dims, 10, field_id=52, envelope=0.4))
    f1 = make_field(q, lat, q.PROPAGATOR, q.F32, S1)
    f2 = make_field(q, lat, q.PROPAGATOR, q.F32, S2)
    C = q.meson_2pt(f1, f2, q.SIXTEEN_MESONS).cpu().numpy()
    assert corr_err(C, hadron.meson_2pt(S1, S2, hadron.SIXTEEN_MESONS)) <= TOL_F32
    C11 = q.meson_2pt(f1, f1, q.SIXTEEN_MESONS).cpu().numpy()
    assert corr_err(C11, hadron.meson_2pt(S1, S1, hadron.SIXTEEN_MESONS)) <= TOL_F32


def test_all_256_gamma_pairs_and_momenta(qdpg_gpu):
    q = qdpg_gpu
    dims = (4, 3, 5, 3)
    lat = q.Lattice(dims, 3)
    S1 = fields.round_to_f32(fields.propagator(dims, 11, field_id=61, envelope=None))
    S2 = fields.round_to_f32(fields.propagator(dims, 11, field_id=62, envelope=None))
    f1 = make_field(q, lat, q.PROPAGATOR, q.F32, S1)
    f2 = make_field(q, lat, q.PROPAGATOR, q.F32, S2)
    chans = [(a, b) for a in range(16) for b in range(16)]          # 16 mask pairs, many passes
    moms = [(0, 0, 0), (1, 0, 0), (-1, 2, 0), (0, -1, -2), (3, 1, 4)]
    origin = (2, 1, 3, 0)
    C = q.meson_2pt(f1, f2, chans, moms, origin=origin).cpu().numpy()
    ref = hadron.meson_2pt(S1, S2, chans, moms, origin=origin)
    assert corr_err(C, ref) <= TOL_F32


def test_mesons_bf16_storage_and_decay_direction(qdpg_gpu):
    q = qdpg_gpu
    dims = (4, 6, 3, 5)
    lat = q.Lattice(dims, 1)                                         # t along direction 1
    S = to_bf16_complex(fields.round_to_f32(fields.propagator(dims, 12, envelope=0.3)))
    f = make_field(q, lat, q.PROPAGATOR, q.BF16, S)
    moms = [(0, 0, 0), (1, 1, -1)]
    C = q.meson_2pt(f, f, q.SIXTEEN_MESONS, moms).cpu().numpy()
    ref = hadron.meson_2pt(S, S, hadron.SIXTEEN_MESONS, moms, j_decay=1)
    assert corr_err(C, ref) <= TOL_F32


# ---------------------------------------------------------------------------
# whole chains


def test_chain_4x8_matches_stored_values(qdpg_gpu):
    import os

    q = qdpg_gpu
    w = configs.CHAIN_4x8
    lat = q.Lattice(w.dims, w.j_decay)
    U = fields.round_to_f32(fields.gauge_field(w.dims, w.seed, kind=w.links))
    Uf = make_field(q, lat, q.GAUGE, q.F32, U)
    S = q.point_source(q.Field(lat, q.PROPAGATOR, q.F32, device=dev()))
    q.gauss_smear(Uf, S, w.kappa, w.n_smear, w.j_decay, scratch=S.like())
    C = q.meson_2pt(S, S, q.SIXTEEN_MESONS).cpu().numpy()[:, 0, :]
    data = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "chain_4x8_mesons.txt"))
    stored = (data[:, 2] + 1j * data[:, 3]).reshape(16, w.Nt)
    assert corr_err(C[:, None, :], stored[:, None, :]) <= TOL_F32


def _sublattice(w, t):
    """Single-timeslice lattice (L3 = 1) holding timeslice t of the workload."""
    return (w.dims[0], w.dims[1], w.dims[2], 1), (t, t + 1)


@pytest.mark.slow
def test_mesons_16x32_full_size_sampled_timeslices(qdpg_gpu):
    """The 16^3x32 workload end to end on the GPU (the benchmark's launch
    configuration); the checker recomputes sampled timeslices exactly, since
    smearing and contractions never couple timeslices."""
    q = qdpg_gpu
    w = configs.MESONS_16x32
    lat = q.Lattice(w.dims, w.j_decay)
    U = fields.round_to_f32(fields.gauge_field(w.dims, w.seed, kind=w.links, eps=w.eps))
    P = fields.round_to_f32(fields.propagator(w.dims, w.seed))
    Uf = make_field(q, lat, q.GAUGE, q.F32, U)
    src = q.point_source(q.Field(lat, q.PROPAGATOR, q.F32, device=dev()))
    snk = make_field(q, lat, q.PROPAGATOR, q.F32, P)
    scratch = snk.like()
    q.gauss_smear(Uf, src, w.kappa, w.n_smear, w.j_decay, scratch=scratch)
    q.gauss_smear(Uf, snk, w.kappa, w.n_smear, w.j_decay, scratch=scratch)
    C = q.meson_2pt(snk, snk, q.SIXTEEN_MESONS).cpu().numpy()[:, 0, :]
    src_h = export(src)
    snk_h = snk.export()
    assert np.all(src_h[1:] == 0)                                    # smearing never leaves t = 0
    sampled = (0, 17, 31)
    C_ref = []
    for t in sampled:
        sub, rng_t = _sublattice(w, t)
        Ut = U[:, t:t + 1]
        ref = smear.gauss_smear(Ut, P[t:t + 1], w.kappa, w.n_smear, 3)
        got = snk_h[t:t + 1].cpu().numpy()
        assert field_err(got, ref) <= TOL_F32, t
        C_ref.append(hadron.meson_2pt(ref, ref, hadron.SIXTEEN_MESONS)[:, 0, 0])
        if t == 0:
            s_ref = smear.gauss_smear(Ut, source.point_propagator(sub), w.kappa, w.n_smear, 3)
            assert field_err(src_h[0:1], s_ref) <= TOL_F32
    # the correlator norm runs over t for each channel: here over the sampled t
    C_ref = np.stack(C_ref, axis=-1)                                 # (16, n_sampled)
    assert corr_err(C[:, None, list(sampled)], C_ref[:, None, :]) <= TOL_F32


# ---------------------------------------------------------------------------
# growth beyond the FP32 range of the contractions: power-of-two rescaling


@pytest.mark.parametrize("prec,tol", [("f32", TOL_F32), ("bf16", TOL_BF16)])
def test_smearing_growth_rescaled_exactly(qdpg_gpu, prec, tol):
    """kappa = 0.3, N = 60: the field grows by ~2^85 and its meson site
    values (~2^170) would overflow FP32; the smearing rescales by exact
    powers of two (the field's exp) and the contractions apply them to the
    FP64 sums, so field and correlators still match the checker."""
    q = qdpg_gpu
    dims = (8, 8, 8, 4)
    lat = q.Lattice(dims, 3)
    U = fields.round_to_f32(fields.gauge_field(dims, 61, kind="near_unit"))
    P = fields.round_to_f32(fields.propagator(dims, 62))
    P_in = to_bf16_complex(P) if prec == "bf16" else P
    Uf = make_field(q, lat, q.GAUGE, q.F32, U)
    S = make_field(q, lat, q.PROPAGATOR, q.PREC_NAMES[prec], P_in)
    q.gauss_smear(Uf, S, 0.3, 60, 3, scratch=S.like())
    got = export(S)
    ref = smear.gauss_smear(U, P_in, 0.3, 60, 3)
    assert np.isfinite(got).all() and np.abs(ref).max() > 2.0 ** 70
    assert field_err(got, ref) <= tol
    C = q.meson_2pt(S, S, q.SIXTEEN_MESONS).cpu().numpy()
    assert np.isfinite(C).all()
    # the contraction of the field as stored (exact to FP32 site arithmetic)
    assert corr_err(C, hadron.meson_2pt(got, got, hadron.SIXTEEN_MESONS)) <= TOL_F32
    if prec == "f32":
        assert corr_err(C, hadron.meson_2pt(ref, ref, hadron.SIXTEEN_MESONS)) <= TOL_F32
