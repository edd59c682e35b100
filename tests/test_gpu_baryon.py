"""Baryon contractions on the GPU against the FP64 Wick-contraction checker."""
import numpy as np
import pytest
import torch

from oracle import baryon
from synth import fields
from tests.parity_util import TOL_F32, corr_err, to_bf16_complex

pytestmark = pytest.mark.gpu


def _field(q, lat, prec, canon):
    return q.Field(lat, q.PROPAGATOR, prec, device="cuda:0").import_(
        torch.from_numpy(canon.astype(np.complex64)).to("cuda:0"))


@pytest.mark.parametrize("kind,parity", [("nucleon", 1), ("nucleon", -1), ("delta", 1), ("delta", -1)])
def test_baryons_vs_oracle(qdpg_gpu, kind, parity):
    q = qdpg_gpu
    dims = (5, 3, 7, 3)                     # V3 = 105: a partial block of 32 sites
    lat = q.Lattice(dims, 3)
    Su = fields.round_to_f32(fields.propagator(dims, 20, field_id=91, envelope=0.3))
    Sd = fields.round_to_f32(fields.propagator(dims, 20, field_id=92, envelope=0.3))
    fu, fd = _field(q, lat, q.F32, Su), _field(q, lat, q.F32, Sd)
    moms = [(0, 0, 0), (1, 0, 0), (-1, 1, 2)]
    origin = (2, 1, 3, 0)
    K = q.NUCLEON if kind == "nucleon" else q.DELTA
    C = q.baryon_2pt(fu, fd if kind == "nucleon" else None, K, parity, moms, origin=origin).cpu().numpy()
    ref = baryon.baryon_2pt(Su, Sd, kind, parity, moms, origin=origin)
    assert corr_err(C[None], ref[None]) <= TOL_F32


def test_baryons_bf16_and_other_decay_direction(qdpg_gpu):
    q = qdpg_gpu
    dims = (4, 5, 4, 3)
    lat = q.Lattice(dims, 1)
    Su = to_bf16_complex(fields.round_to_f32(fields.propagator(dims, 21, field_id=93, envelope=0.3)))
    Sd = to_bf16_complex(fields.round_to_f32(fields.propagator(dims, 21, field_id=94, envelope=0.3)))
    fu, fd = _field(q, lat, q.BF16, Su), _field(q, lat, q.BF16, Sd)
    for kind, K in (("nucleon", q.NUCLEON), ("delta", q.DELTA)):
        C = q.baryon_2pt(fu, fd, K, +1, [(0, 0, 0), (0, 1, 1)]).cpu().numpy()
        ref = baryon.baryon_2pt(Su, Sd, kind, +1, [(0, 0, 0), (0, 1, 1)], j_decay=1)
        assert corr_err(C[None], ref[None]) <= TOL_F32, kind
