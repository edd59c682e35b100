"""Seeded input generators and the stored checker values (CPU only)."""
import os

import numpy as np

from oracle import hadron, smear, source
from synth import configs, fields, rng

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _su3_errors(m):
    m = m.reshape(-1, 3, 3)
    unit = np.abs(m @ np.conj(np.swapaxes(m, -1, -2)) - np.eye(3)).max()
    det = np.abs(np.linalg.det(m) - 1).max()
    return unit, det


def test_links_are_su3_and_sliceable():
    dims = (4, 3, 2, 6)
    for kind in ("haar", "near_unit"):
        U = fields.gauge_field(dims, 123, kind=kind)
        assert max(_su3_errors(U)) < 1e-13
        part = fields.gauge_field(dims, 123, kind=kind, x3_range=(2, 5))
        assert np.array_equal(part, U[:, 2:5])
    near = fields.gauge_field(dims, 5, kind="near_unit", eps=0.3)
    haar = fields.gauge_field(dims, 5, kind="haar")
    # near-unit links sit close to 1, Haar links do not (E tr U = 0 under Haar)
    assert np.abs(np.trace(near, axis1=-2, axis2=-1)).mean() > 2.5
    assert np.abs(np.trace(haar, axis1=-2, axis2=-1).mean()) < 0.5


def test_propagator_sliceable_and_enveloped():
    dims = (4, 4, 4, 6)
    S = fields.propagator(dims, 9)
    assert np.array_equal(fields.propagator(dims, 9, x3_range=(1, 3)), S[1:3])
    d = fields.periodic_distance(dims, (0, 0, 0, 0))
    assert d[0, 0, 0, 0] == 0 and d[3, 0, 0, 0] == 3 and d[0, 0, 0, 3] == 1
    near = np.abs(S[0, 0, 0, 0]).mean()
    far = np.abs(S[3, 2, 2, 2]).mean()
    assert near > 10 * far


def test_rng_uniform_and_normal_moments():
    key = rng.stream_key(1, 2)
    u = rng.uniform(key, np.arange(200000))
    assert 0 < u.min() and u.max() <= 1 and abs(u.mean() - 0.5) < 3e-3
    a, b = rng.normal_pairs(key, np.arange(100000))
    for z in (a, b):
        assert abs(z.mean()) < 0.02 and abs(z.var() - 1) < 0.02
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.02


def test_golden_chain_4x8_mesons():
    """The checker still reproduces its stored values for the 4^3x8 chain."""
    data = np.loadtxt(os.path.join(GOLDEN, "chain_4x8_mesons.txt"))
    w = configs.CHAIN_4x8
    U = fields.round_to_f32(fields.gauge_field(w.dims, w.seed, kind=w.links))
    S = smear.gauss_smear(U, source.point_propagator(w.dims), w.kappa, w.n_smear, w.j_decay)
    C = hadron.meson_2pt(S, S, hadron.SIXTEEN_MESONS)[:, 0, :]
    stored = (data[:, 2] + 1j * data[:, 3]).reshape(16, w.Nt)
    assert np.allclose(C, stored, rtol=1e-12, atol=1e-12 * np.abs(stored).max())
