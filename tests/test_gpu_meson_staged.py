"""The three forms of the F32/BF16 meson contraction against each other and
against the FP64 checker: the orbit kernel (the default where every
channel's two masks are equal, as for the sixteen mesons: a thread keeps one
orbit of spin blocks in registers), the kernel that stages S2 in shared
memory (channels with unequal masks), and the one reading both propagators
from global memory.  Channel sets with and without unequal masks; zero and nonzero
momenta, site values, S1 = S2 and S1 != S2, a ragged last block (V3 not a
multiple of the block's 64 sites) and another decay direction.  The two
kernels split the sixteen weighted terms of a channel value differently,
so they agree to FP32 rounding, not bit for bit."""
import numpy as np
import pytest
import torch

from oracle import hadron
from synth import fields
from tests.parity_util import TOL_F32, corr_err

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _prop(q, lat, seed, prec):
    P = fields.round_to_f32(fields.propagator(lat.dims, seed, envelope=0.3))
    return P, q.Field(lat, q.PROPAGATOR, q.PREC_NAMES[prec], device=DEV).import_(torch.from_numpy(P.astype(np.complex64)).to(DEV))


def _forms(q, fn):
    """The default kernel's result and those of the staged (1) and global-read (2) forms."""
    out = []
    for form in (0, 1, 2):
        q.debug_set(q.DEBUG_MESON_FORM, form)
        try:
            out.append(fn().cpu().numpy())
        finally:
            q.debug_set(q.DEBUG_MESON_FORM, 0)
    torch.cuda.synchronize()
    q.device_status()
    return out


CASES = [((8, 8, 8, 4), 3, "f32", True, ((0, 0, 0),)),
         ((6, 5, 7, 3), 3, "f32", False, ((0, 0, 0), (1, 0, 0), (0, -1, 2))),
         ((8, 4, 6, 4), 1, "f32", True, ((0, 0, 0), (1, 1, 0))),
         ((16, 16, 16, 2), 3, "bf16", False, ((0, 0, 0),)),
         ((12, 12, 6, 2), 3, "f32", False, tuple(m for m in [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (-1, 0, 0),
                                                             (0, -1, 0), (0, 0, -1), (1, 1, 1)]))]


@pytest.mark.parametrize("dims,jd,prec,same,moms", CASES)
def test_staged_meson_matches_unstaged_and_checker(qdpg_gpu, dims, jd, prec, same, moms):
    q = qdpg_gpu
    lat = q.Lattice(dims, jd)
    P1, S1 = _prop(q, lat, 3, prec)
    P2, S2 = (P1, S1) if same else _prop(q, lat, 4, prec)
    chans = q.SIXTEEN_MESONS + ((1, 2), (5, 11), (15, 0)) if not same else q.SIXTEEN_MESONS
    a, b, c = _forms(q, lambda: q.meson_2pt(S1, S2, chans, moms))
    assert corr_err(a, c) <= 1e-6 and corr_err(b, c) <= 1e-6
    if prec == "f32":
        ref = hadron.meson_2pt(P1, P2, chans, moms, j_decay=jd)
        assert corr_err(a, ref) <= TOL_F32 if len(moms) < 8 else np.abs(a - ref).max() <= 1e-5 * np.abs(ref).max()


def test_staged_meson_site_values(qdpg_gpu):
    q = qdpg_gpu
    lat = q.Lattice((6, 5, 7, 3), 3)
    P1, S1 = _prop(q, lat, 5, "f32")
    P2, S2 = _prop(q, lat, 6, "f32")
    chans = q.SIXTEEN_MESONS
    a, b, c = _forms(q, lambda: q.meson_sites(S1, S2, chans))
    assert np.abs(a - c).max() <= 1e-6 * np.abs(c).max() and np.abs(b - c).max() <= 1e-6 * np.abs(c).max()
    ref = np.stack([hadron.meson_site(P1, P2, x, y) for x, y in chans])       # (16, t, z, y, x)
    ref = ref.reshape(16, lat.Nt, lat.V3)
    assert np.abs(a - ref).max() <= 1e-6 * np.abs(ref).max()
