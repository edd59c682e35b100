"""All pairs of a set of propagators in one pass (qdpg_meson_2pt_multi)
against the pairwise entry point and the FP64 checker: three propagators
(one smeared far enough to be rescaled by its power-of-two scale record),
the sixteen mesons at zero momentum and at the 33 momenta with |n|^2 <= 4,
FP32, BF16 and float16 storage, a lattice whose timeslice volume is not a multiple
of the kernel's 4-site blocks, and a timeslice batch smaller than the
lattice (a tiny site-value budget is not settable, so a long Nt stands in:
the batches are exercised by the 48^3x96 workload in the bench)."""
import numpy as np
import pytest
import torch

from oracle import hadron, smear
from synth import fields
from tests.parity_util import TOL_BF16, TOL_F32, corr_err, proj_err

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _props(q, dims, prec):
    lat = q.Lattice(dims, 3)
    U64 = fields.round_to_f32(fields.gauge_field(dims, 41, kind="haar"))
    lp = q.F16 if prec == "f16" else q.F32
    U = q.Field(lat, q.GAUGE, lp, device=DEV).import_(torch.from_numpy(U64.astype(np.complex64)).to(DEV))
    out, ref = [], []
    for i, (kappa, n) in enumerate(((0.2, 3), (0.15, 1), (0.3, 60))):
        P64 = fields.round_to_f32(fields.propagator(dims, 41, field_id=10 + i, envelope=0.3))
        f = q.Field(lat, q.PROPAGATOR, q.PREC_NAMES[prec], device=DEV).import_(
            torch.from_numpy(P64.astype(np.complex64)).to(DEV))
        q.gauss_smear(U, f, kappa, n, 3, scratch=f.like())
        out.append(f)
        ref.append(smear.gauss_smear(U64, P64, kappa, n, 3) if prec == "f32" else None)
    return lat, out, ref


@pytest.mark.parametrize("dims,prec,nmom", [((6, 5, 3, 4), "f32", 1), ((6, 5, 3, 4), "f32", 33),
                                            ((8, 4, 4, 3), "bf16", 1), ((4, 4, 4, 6), "f32", 8),
                                            ((8, 6, 5, 3), "f16", 33), ((4, 5, 3, 4), "f16", 1)])
def test_multi_equals_pairwise_and_checker(qdpg_gpu, dims, prec, nmom):
    q = qdpg_gpu
    lat, props, ref = _props(q, dims, prec)
    moms = [(0, 0, 0)] + [m for m in q.momenta_up_to(4) if m != (0, 0, 0)][:nmom - 1]
    C = q.meson_2pt_multi(props, q.SIXTEEN_MESONS, moms).cpu().numpy()
    torch.cuda.synchronize()
    q.device_status()
    n = len(props)
    for a in range(n):
        for b in range(n):
            pw = q.meson_2pt(props[a], props[b], q.SIXTEEN_MESONS, moms).cpu().numpy()
            scale = np.abs(pw).max()
            assert np.abs(C[a, b] - pw).max() <= 1e-5 * scale, (a, b)
            if prec == "f32":
                r = hadron.meson_2pt(ref[a], ref[b], hadron.SIXTEEN_MESONS, moms, j_decay=3)
                A = np.stack([hadron.timeslice_sum(np.abs(hadron.meson_site(ref[a], ref[b], x, y)), 3)
                              for x, y in hadron.SIXTEEN_MESONS])
                k0 = moms.index((0, 0, 0))
                assert corr_err(C[a, b][:, k0:k0 + 1], r[:, k0:k0 + 1]) <= TOL_F32, (a, b)
                assert proj_err(C[a, b], r, A) <= TOL_F32, (a, b)
            else:
                assert corr_err(C[a, b], pw) <= TOL_BF16


def test_multi_rejects_unequal_masks_and_bad_sets(qdpg_gpu):
    q = qdpg_gpu
    lat, props, _ = _props(q, (4, 4, 4, 2), "f32")
    with pytest.raises(q.QdpgError) as ei:
        q.meson_2pt_multi(props, [(1, 4)])       # gamma_1 (mask 3) with gamma_3 (mask 2)
    assert ei.value.status == -7
    with pytest.raises(q.QdpgError):
        q.meson_2pt_multi(props * 3, q.SIXTEEN_MESONS)     # 9 > 8 propagators
