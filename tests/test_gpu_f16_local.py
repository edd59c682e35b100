"""One float16 tensor-core hop, checked site by site against the FP64 checker.

A global or per-timeslice norm dilutes an error confined to a few
low-amplitude sites (a wrong halo row or link far from the source).  This
test removes that blind spot for the float16 hop: for a single iteration
the inputs of both sides are the same float16 numbers (the stored
propagator and links, exported exactly), the products of float16 inputs
are exact and the sums FP32, so every output component of the device
differs from the checker's by at most the float16 rounding of the output
(half an ulp, 2^-11 of the component) plus the FP32 rounding of the sum,
bounded by a small multiple of the local magnitude L(x) (the largest
component of psi at x and its six spatial neighbours).  Inputs carry the
exp(-|x - x0|) envelope, so magnitudes span several decades and a
mistake at a faint site exceeds its bound by orders of magnitude.

Lattices cover halo tiles with the y halo wrapping at both ends, a
whole-plane tile, first extents 8, 12, 16, 24 and 48, and several tiles per
plane; reconstruct-12 links (row 2 rebuilt in FP32 and rounded to float16
inside the hop) get a bound one link rounding looser.  The batch path's
float16 jobs run the same multi-job kernel and are checked bit for bit
against this entry point by the batch tests.
"""
import numpy as np
import pytest
import torch

from oracle import geometry, smear
from synth import fields

pytestmark = pytest.mark.gpu

CASES = [
    ((16, 16, 4, 2), "f16"),      # Lx 16: four 4-row halo tiles per plane, y halo wraps at both ends
    ((8, 8, 8, 4), "f16"),        # whole-plane tiles (no halo)
    ((12, 10, 6, 2), "f16"),      # Lx 12: two 5-row tiles per plane
    ((24, 6, 4, 2), "f16"),       # Lx 24: three 2-row tiles per plane
    ((48, 2, 3, 2), "f16"),       # Lx 48: one-row tiles, three planes
    ((16, 8, 4, 2), "f16_r12"),   # reconstruct-12 links
]


def _local_magnitude(psi: np.ndarray, j_decay: int) -> np.ndarray:
    """L(x): the largest |component| of psi over x and its six spatial neighbours."""
    m = np.abs(psi).reshape(psi.shape[:4] + (-1,)).max(axis=-1)
    L = m.copy()
    for mu in geometry.spatial_dirs(j_decay):
        for sign in (1, -1):
            L = np.maximum(L, geometry.shift(m, sign, mu))
    return L


@pytest.mark.parametrize("dims,lprec", CASES)
def test_f16_one_hop_site_by_site(qdpg_gpu, dims, lprec):
    q = qdpg_gpu
    dev = torch.device("cuda:0")
    jd, kappa = 3, 0.21
    lat = q.Lattice(dims, jd)
    U = fields.round_to_f32(fields.gauge_field(dims, 31, kind="haar"))
    P = fields.round_to_f32(fields.propagator(dims, 32, x0=(1, 1, 1, 0), envelope=1.0))
    Uf = q.Field(lat, q.GAUGE, q.PREC_NAMES[lprec], device=dev).import_(
        torch.from_numpy(U.astype(np.complex64)).to(dev))
    S = q.Field(lat, q.PROPAGATOR, q.F16, device=dev).import_(torch.from_numpy(P.astype(np.complex64)).to(dev))
    # the float16 numbers the hop reads (links: rows as stored; reconstruct-12
    # row 2 as the library rebuilds it)
    U16 = Uf.export().cpu().numpy().astype(np.complex128)
    P16 = S.export().cpu().numpy().astype(np.complex128)
    q.gauss_smear(Uf, S, kappa, 1, jd, scratch=S.like())
    got = S.export().cpu().numpy().astype(np.complex128)
    q.device_status()
    ref = smear.gauss_smear(U16, P16, kappa, 1, jd)

    L = _local_magnitude(P16, jd)[..., None, None, None, None]
    link_slack = 2.0 ** -16 if lprec == "f16" else 2.0 ** -9 * kappa   # FP32 sums; or one rounding of row 2
    floor = 2.0 ** -36 * np.abs(ref).max()
    for part in (np.real, np.imag):
        err = np.abs(part(got) - part(ref))
        bound = 2.0 ** -11 * np.abs(part(ref)) + link_slack * L + floor
        worst = np.unravel_index(np.argmax(err / bound), err.shape)
        assert (err <= bound).all(), (worst, err[worst], bound[worst])
    # the test has teeth: the faintest sites are far below the largest values
    assert L.min() < 1e-2 * L.max()
