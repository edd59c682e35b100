"""Site values and the tensor-core momentum projection against the FP64 checker."""
import numpy as np
import pytest
import torch

from oracle import baryon, hadron
from synth import fields
from tests.parity_util import TOL_F32, corr_err, proj_err

pytestmark = pytest.mark.gpu


def _prop(q, lat, canon):
    return q.Field(lat, q.PROPAGATOR, q.F32, device="cuda:0").import_(
        torch.from_numpy(canon.astype(np.complex64)).to("cuda:0"))


def _dft(site_vals, dims, moms, origin=(0, 0, 0, 0)):
    """FP64 projection of (n, Nt, Lz, Ly, Lx) site values with the checker's phases."""
    ph = hadron.momentum_phases(dims, moms, 3, origin)          # (n_mom, t, z, y, x)
    return np.einsum("jtzyx,mtzyx->jmt", site_vals, ph)


@pytest.mark.parametrize("dims,n_chan", [((4, 4, 4, 8), 3), ((5, 3, 7, 6), 5), ((16, 16, 12, 2), 70)])
def test_projection_of_random_site_values(qdpg_gpu, dims, n_chan):
    q = qdpg_gpu
    lat = q.Lattice(dims, 3)
    rng = np.random.default_rng(4)
    shp = (n_chan, dims[3], dims[2], dims[1], dims[0])
    vals = (rng.normal(size=shp) + 1j * rng.normal(size=shp)).astype(np.complex64)
    moms = q.momenta_up_to(4)
    origin = (1, 2, 0, 0)
    sites = torch.from_numpy(vals.reshape(n_chan, dims[3], -1)).to("cuda:0")
    C = q.momentum_project(lat, sites, moms, origin=origin).cpu().numpy()
    q.device_status()
    ref = _dft(vals.astype(np.complex128), dims, moms, origin)
    assert corr_err(C, ref) <= TOL_F32


def test_meson_site_values(qdpg_gpu):
    q = qdpg_gpu
    dims = (4, 3, 5, 3)
    lat = q.Lattice(dims, 3)
    S1 = fields.round_to_f32(fields.propagator(dims, 30, field_id=101, envelope=None))
    S2 = fields.round_to_f32(fields.propagator(dims, 30, field_id=102, envelope=None))
    chans = [(15, 15), (3, 12), (7, 7)]
    got = q.meson_sites(_prop(q, lat, S1), _prop(q, lat, S2), chans).cpu().numpy()
    for j, (a, b) in enumerate(chans):
        ref = hadron.meson_site(S1, S2, a, b).reshape(dims[3], -1)
        assert np.linalg.norm(got[j] - ref) <= TOL_F32 * np.linalg.norm(ref)


def test_mesons_and_baryons_at_33_momenta(qdpg_gpu):
    q = qdpg_gpu
    dims = (6, 6, 6, 4)
    lat = q.Lattice(dims, 3)
    S1 = fields.round_to_f32(fields.propagator(dims, 31, field_id=103, envelope=0.3))
    S2 = fields.round_to_f32(fields.propagator(dims, 31, field_id=104, envelope=0.3))
    f1, f2 = _prop(q, lat, S1), _prop(q, lat, S2)
    moms = q.momenta_up_to(4)
    C = q.momentum_project(lat, q.meson_sites(f1, f2, q.SIXTEEN_MESONS), moms).cpu().numpy()
    ref = hadron.meson_2pt(S1, S2, hadron.SIXTEEN_MESONS, moms)
    assert corr_err(C, ref) <= TOL_F32
    for kind, K in (("nucleon", q.NUCLEON), ("delta", q.DELTA)):
        sv = q.baryon_sites(f1, f2, K, +1)
        Cb = q.momentum_project(lat, sv.reshape(1, dims[3], -1), moms).cpu().numpy()
        refb = baryon.baryon_2pt(S1, S2, kind, +1, moms)
        assert corr_err(Cb, refb[None]) <= TOL_F32, kind


def test_meson_and_baryon_2pt_many_momenta_on_tensor_cores(qdpg_gpu):
    """meson_2pt / baryon_2pt with 8 or more momenta project on the tensor
    cores internally; with an origin, a 33-momentum set, and a smeared
    field rescaled by powers of two (kappa = 0.3, N = 40) whose cube exceeds
    the FP32 range of the contractions, they match the checker."""
    from oracle import smear

    q = qdpg_gpu
    dims = (6, 6, 6, 4)
    lat = q.Lattice(dims, 3)
    U = fields.round_to_f32(fields.gauge_field(dims, 32, kind="near_unit"))
    P1 = fields.round_to_f32(fields.propagator(dims, 33, envelope=0.3))
    P2 = fields.round_to_f32(fields.propagator(dims, 34, envelope=0.3))
    Uf = q.Field(lat, q.GAUGE, q.F32, device="cuda:0").import_(torch.from_numpy(U.astype(np.complex64)).to("cuda:0"))
    f1, f2 = _prop(q, lat, P1), _prop(q, lat, P2)
    q.gauss_smear(Uf, f1, 0.3, 40, 3, scratch=f1.like())
    S1 = smear.gauss_smear(U, P1, 0.3, 40, 3)
    assert np.abs(S1).max() > 2.0 ** 50          # the Delta's three factors of S1 exceed the FP32 range
    moms, origin = q.momenta_up_to(4), (1, 0, 2, 3)
    C = q.meson_2pt(f1, f2, q.SIXTEEN_MESONS, moms, origin=origin).cpu().numpy()
    ref = hadron.meson_2pt(S1, P2, hadron.SIXTEEN_MESONS, moms, origin=origin)
    assert np.isfinite(C).all()
    # smeared fields are smooth: errors relative to sum_x |c(x)| per t (proj_err)
    A = np.stack([np.abs(hadron.meson_site(S1, P2, a, b)).sum(axis=(1, 2, 3)) for a, b in hadron.SIXTEEN_MESONS])
    assert proj_err(C, ref, A) <= TOL_F32
    assert corr_err(C[:, :1], ref[:, :1]) <= TOL_F32          # zero momentum: no cancellation
    for kind, K in (("nucleon", q.NUCLEON), ("delta", q.DELTA)):
        Sd = P2 if kind == "nucleon" else S1
        Cb = q.baryon_2pt(f1, f2 if kind == "nucleon" else None, K, -1, moms, origin=origin).cpu().numpy()
        refb = baryon.baryon_2pt(S1, Sd, kind, -1, moms, origin=origin)
        Ab = np.abs(baryon.baryon_site(S1, Sd, kind, -1)).sum(axis=(1, 2, 3))
        assert np.isfinite(Cb).all()
        assert proj_err(Cb[None], refb[None], Ab[None]) <= TOL_F32, kind
