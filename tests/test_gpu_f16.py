"""Float16 storage with the tensor-core smearing hop, against the FP64 checker.

Propagators are stored as float16 pairs times a per-field power of two
(the scale record), links as float16 (full or reconstruct-12); all
arithmetic is FP32.  Storage rounding is exact and checked bit for bit;
smearing and contractions are checked against the checker on the same
FP32-rounded inputs within the reduced-precision tolerance.
"""
import numpy as np
import pytest
import torch

from oracle import geometry, hadron, smear, source
from synth import fields
from tests.parity_util import TOL_BF16, corr_err, field_err, field_err_t, proj_err

pytestmark = pytest.mark.gpu

# Reduced-precision storage: the same bound as for bfloat16.
TOL_F16 = TOL_BF16


def dev():
    return torch.device("cuda:0")


def upload(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def export(f):
    return f.export().cpu().numpy()


def f16_expected(a: np.ndarray) -> np.ndarray:
    """The stored-and-exported value of complex64 data: scale exponent
    e = frexp(max |re|,|im|) - 14, then float16 round-to-nearest-even of
    value * 2^-e, times 2^e."""
    m = float(max(np.abs(a.real).max(), np.abs(a.imag).max()))
    e = np.frexp(m)[1] - 14 if m > 0 else 0
    t = torch.from_numpy(np.ascontiguousarray(a.astype(np.complex64)))
    re = torch.ldexp(t.real, torch.tensor(-float(e))).to(torch.float16).to(torch.float64)
    im = torch.ldexp(t.imag, torch.tensor(-float(e))).to(torch.float16).to(torch.float64)
    return np.ldexp(re.numpy(), e) + 1j * np.ldexp(im.numpy(), e)


def to_f16_complex(a: np.ndarray) -> np.ndarray:
    t = torch.from_numpy(np.ascontiguousarray(a.astype(np.complex64)))
    return t.real.to(torch.float16).double().numpy() + 1j * t.imag.to(torch.float16).double().numpy()


@pytest.mark.parametrize("scale", [1e-3, 1.0, 3e6])
def test_f16_propagator_import_export_exact(qdpg_gpu, scale):
    q = qdpg_gpu
    dims = (4, 3, 5, 2)
    lat = q.Lattice(dims, 3)
    rng = np.random.default_rng(7)
    shp = lat.canonical_shape(q.PROPAGATOR)
    a = fields.round_to_f32(scale * (rng.normal(size=shp) + 1j * rng.normal(size=shp)))
    P = q.Field(lat, q.PROPAGATOR, q.F16, device=dev()).import_(upload(a.astype(np.complex64)))
    assert np.array_equal(export(P), f16_expected(a))


def test_f16_links_exact_and_reconstructed(qdpg_gpu):
    q = qdpg_gpu
    dims = (4, 3, 4, 2)
    lat = q.Lattice(dims, 3)
    U = fields.round_to_f32(fields.gauge_field(dims, 5, kind="haar"))
    full = export(q.Field(lat, q.GAUGE, q.F16, device=dev()).import_(upload(U.astype(np.complex64))))
    assert np.array_equal(full, to_f16_complex(U))
    r12 = export(q.Field(lat, q.GAUGE, q.F16_R12, device=dev()).import_(upload(U.astype(np.complex64))))
    assert np.array_equal(r12[..., :2, :], to_f16_complex(U[..., :2, :]))
    assert np.abs(r12[..., 2, :] - U[..., 2, :]).max() < 3e-3


def test_f16_point_source_and_shift_exact(qdpg_gpu):
    q = qdpg_gpu
    dims = (4, 3, 5, 6)
    lat = q.Lattice(dims, 3)
    x0 = (3, 1, 4, 2)
    S = q.point_source(q.Field(lat, q.PROPAGATOR, q.F16, device=dev()), x0)
    assert np.array_equal(export(S), source.point_propagator(dims, x0))
    rng = np.random.default_rng(3)
    shp = lat.canonical_shape(q.PROPAGATOR)
    a = fields.round_to_f32(100.0 * (rng.normal(size=shp) + 1j * rng.normal(size=shp)))
    P = q.Field(lat, q.PROPAGATOR, q.F16, device=dev()).import_(upload(a.astype(np.complex64)))
    base = export(P)
    for mu in range(4):
        for sign in (1, -1):
            D = q.shift(P.like(), P, sign, mu)
            assert np.array_equal(export(D), geometry.shift(base, sign, mu)), (mu, sign)


# (dims, j_decay, kappa, N, link precision, propagator): lattices covering
# whole-plane tiles, halo tiles (Lx = 12, 16, 24, 48) and a non-default decay
# direction; growth up to 2^90 over the iterations exercises the rescaling.
SMEAR_CASES = [
    ((4, 4, 4, 8), 3, 0.25, 5, "f16", "point"),
    ((8, 8, 8, 4), 3, 0.30, 12, "f16_r12", "synthetic"),
    ((12, 12, 6, 2), 3, 0.21, 9, "f16", "synthetic"),
    ((16, 16, 4, 2), 3, 0.21, 10, "f16_r12", "synthetic"),
    ((24, 6, 4, 2), 3, 0.15, 7, "f16", "synthetic"),
    ((48, 2, 3, 2), 3, 0.20, 6, "f16_r12", "synthetic"),
    ((8, 6, 8, 4), 1, 0.22, 8, "f16", "synthetic"),
    ((8, 8, 4, 2), 3, 0.30, 60, "f16_r12", "synthetic"),
]


def _smear_inputs(dims, jd, prop):
    U = fields.round_to_f32(fields.gauge_field(dims, 11, kind="haar"))
    if prop == "point":
        P = source.point_propagator(dims)
    else:
        P = fields.round_to_f32(fields.propagator(dims, 12))
    return U, P


@pytest.mark.parametrize("dims,jd,kappa,n_iter,lprec,prop", SMEAR_CASES)
def test_f16_smear_matches_checker(qdpg_gpu, dims, jd, kappa, n_iter, lprec, prop):
    q = qdpg_gpu
    lat = q.Lattice(dims, jd)
    U, P = _smear_inputs(dims, jd, prop)
    Uf = q.Field(lat, q.GAUGE, q.PREC_NAMES[lprec], device=dev()).import_(upload(U.astype(np.complex64)))
    S = q.Field(lat, q.PROPAGATOR, q.F16, device=dev()).import_(upload(P.astype(np.complex64)))
    q.gauss_smear(Uf, S, kappa, n_iter, jd, scratch=S.like())
    got = export(S)
    q.device_status()
    ref = smear.gauss_smear(U, P, kappa, n_iter, jd)
    err = field_err(got, ref)
    err_t = field_err_t(got, ref, 3 - jd)
    assert np.isfinite(got).all()
    assert err <= TOL_F16 and err_t <= TOL_F16, (err, err_t)
    # float16 has 11 significant bits; the observed error is far inside the bound
    assert err <= 5e-3, err


def test_f16_smear_without_scratch_and_repeated_calls(qdpg_gpu):
    """The library allocates the ping-pong buffer when none is given, and a
    second call continues from the first call's scale."""
    q = qdpg_gpu
    dims, jd = (8, 8, 8, 4), 3
    lat = q.Lattice(dims, jd)
    U, P = _smear_inputs(dims, jd, "synthetic")
    Uf = q.Field(lat, q.GAUGE, q.F16, device=dev()).import_(upload(U.astype(np.complex64)))
    S = q.Field(lat, q.PROPAGATOR, q.F16, device=dev()).import_(upload(P.astype(np.complex64)))
    q.gauss_smear(Uf, S, 0.27, 7, jd)
    q.gauss_smear(Uf, S, 0.27, 8, jd, scratch=S.like())
    ref = smear.gauss_smear(U, P, 0.27, 15, jd)
    assert field_err(export(S), ref) <= 5e-3


def test_f16_mesons_match_checker(qdpg_gpu):
    q = qdpg_gpu
    dims, jd = (8, 8, 8, 4), 3
    lat = q.Lattice(dims, jd)
    U, P = _smear_inputs(dims, jd, "synthetic")
    Uf = q.Field(lat, q.GAUGE, q.F16_R12, device=dev()).import_(upload(U.astype(np.complex64)))
    S = q.Field(lat, q.PROPAGATOR, q.F16, device=dev()).import_(upload(P.astype(np.complex64)))
    q.gauss_smear(Uf, S, 0.25, 20, jd, scratch=S.like())
    moms = q.momenta_up_to(2)
    C = q.meson_2pt(S, S, q.SIXTEEN_MESONS, moms=moms, origin=(1, 2, 3, 0)).cpu().numpy()
    ref = smear.gauss_smear(U, P, 0.25, 20, jd)
    C_ref = hadron.meson_2pt(ref, ref, hadron.SIXTEEN_MESONS, moms=moms, origin=(1, 2, 3, 0))
    assert corr_err(C, C_ref) <= TOL_F16
    # site values carry the scale too: their zero-momentum timeslice sums agree
    sites = q.meson_sites(S, S, q.SIXTEEN_MESONS).cpu().numpy().astype(np.complex128)
    k0 = moms.index((0, 0, 0))
    assert corr_err(sites.sum(axis=-1), C_ref[:, k0, :]) <= TOL_F16


@pytest.mark.parametrize("kind,parity", [(0, 1), (0, -1), (1, 1)])
def test_f16_baryons_match_checker(qdpg_gpu, kind, parity):
    from oracle import baryon

    q = qdpg_gpu
    dims, jd = (4, 4, 4, 4), 3
    lat = q.Lattice(dims, jd)
    U = fields.round_to_f32(fields.gauge_field(dims, 21, kind="haar"))
    Pu = fields.round_to_f32(fields.propagator(dims, 22))
    Pd = fields.round_to_f32(fields.propagator(dims, 23))
    Uf = q.Field(lat, q.GAUGE, q.F16, device=dev()).import_(upload(U.astype(np.complex64)))
    Su = q.Field(lat, q.PROPAGATOR, q.F16, device=dev()).import_(upload(Pu.astype(np.complex64)))
    Sd = q.Field(lat, q.PROPAGATOR, q.F16, device=dev()).import_(upload(Pd.astype(np.complex64)))
    q.gauss_smear(Uf, Su, 0.2, 6, jd, scratch=Su.like())
    q.gauss_smear(Uf, Sd, 0.2, 9, jd, scratch=Sd.like())
    ru = smear.gauss_smear(U, Pu, 0.2, 6, jd)
    rd = smear.gauss_smear(U, Pd, 0.2, 9, jd)
    moms = [(0, 0, 0), (1, 0, 0), (0, -1, 1)]
    if kind == 0:
        C = q.baryon_2pt(Su, Sd, kind=0, parity=parity, moms=moms).cpu().numpy()
        C_ref = baryon.baryon_2pt(ru, rd, kind="nucleon", parity=parity, moms=moms)
    else:
        C = q.baryon_2pt(Su, None, kind=1, parity=parity, moms=moms).cpu().numpy()
        C_ref = baryon.baryon_2pt(ru, ru, kind="delta", parity=parity, moms=moms)
    assert corr_err(C, C_ref) <= TOL_F16


def test_f16_rejects_unserved_lattice(qdpg_gpu):
    q = qdpg_gpu
    dims = (5, 4, 4, 2)  # first spatial extent not a multiple of 4
    lat = q.Lattice(dims, 3)
    Uf = q.Field(lat, q.GAUGE, q.F16, device=dev())
    S = q.Field(lat, q.PROPAGATOR, q.F16, device=dev())
    with pytest.raises(q.QdpgError) as ei:
        q.gauss_smear(Uf, S, 0.2, 2, 3, scratch=S.like())
    assert ei.value.status == -7


@pytest.mark.parametrize("dims,moms", [((8, 8, 8, 4), ((0, 0, 0),)), ((12, 6, 5, 2), ((0, 0, 0), (1, 0, 0))),
                                       ((8, 8, 4, 2), "eight")])
def test_f16_self_pair_orbit_form_agrees_with_global_reads(qdpg_gpu, dims, moms):
    """A float16 self pair runs the orbit kernel (the staged float16 site
    blocks converted once into FP32 rows per site); the global-read form
    reads the same stored numbers: the two agree to FP32 rounding, with the
    reducing sums (p = 0, two momenta) and with site values for the
    projection (eight momenta), including a ragged last block (V3 = 360)."""
    q = qdpg_gpu
    lat = q.Lattice(dims, 3)
    P = fields.round_to_f32(fields.propagator(dims, 44, envelope=0.4))
    S = q.Field(lat, q.PROPAGATOR, q.F16, device=dev()).import_(upload(P.astype(np.complex64)))
    mlist = q.momenta_up_to(2)[:8] if moms == "eight" else list(moms)
    outs = []
    for form in (0, 2):
        q.debug_set(q.DEBUG_MESON_FORM, form)
        try:
            outs.append(q.meson_2pt(S, S, q.SIXTEEN_MESONS, moms=mlist).cpu().numpy())
            q.device_status()
        finally:
            q.debug_set(q.DEBUG_MESON_FORM, 0)
    Sx = export(S)
    ref = hadron.meson_2pt(Sx, Sx, hadron.SIXTEEN_MESONS, moms=mlist)
    # per channel, the sum over each timeslice of the site values' magnitudes
    # (the scale a cancelling p != 0 sum is accurate to in FP32)
    A = np.stack([np.abs(hadron.meson_site(Sx, Sx, a, b)).sum(axis=(1, 2, 3)) for a, b in hadron.SIXTEEN_MESONS])
    for C in outs:
        assert proj_err(C, ref, A[:, None, :]) <= 1e-5
    k0 = [i for i, m in enumerate(mlist) if tuple(m) == (0, 0, 0)]
    if k0:
        assert corr_err(outs[0][:, k0[0], :], ref[:, k0[0], :]) <= 1e-5
