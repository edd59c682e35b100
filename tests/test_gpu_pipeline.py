"""The pipelined (bulk-copy) smearing kernel: agreement with the simple
kernel, and its bounded waits running out without hanging or faulting."""
import numpy as np
import pytest
import torch

from oracle import smear
from synth import fields
from tests.parity_util import TOL_F32, field_err

pytestmark = pytest.mark.gpu


def _field(q, lat, kind, prec, canon):
    return q.Field(lat, kind, prec, device="cuda:0").import_(torch.from_numpy(canon.astype(np.complex64)).to("cuda:0"))


@pytest.mark.parametrize("dims,prec,sites,lprec", [
    ((16, 16, 16, 4), "f32", 0, "f32"), ((8, 12, 6, 3), "f32", 0, "f32"),
    ((24, 24, 8, 2), "f32", 0, "f32"), ((24, 24, 4, 2), "f32", 288, "f32"),
    ((48, 12, 3, 2), "bf16", 288, "f32"), ((8, 8, 8, 4), "bf16", 0, "f32"),
    ((12, 6, 4, 2), "bf16", 0, "f32"), ((16, 16, 2, 3), "f32", 0, "f32"),
    ((16, 8, 1, 2), "f32", 0, "f32"), ((16, 16, 3, 2), "bf16", 0, "f32"),
    # every fixed halo-tile shape (row-major stages from tensor-map copies)
    ((16, 16, 4, 2), "f32", 128, "f32"), ((48, 12, 3, 2), "f32", 288, "f32"),
    ((24, 16, 2, 2), "f32", 96, "f32"), ((48, 8, 3, 2), "f32", 96, "f32"),
    ((24, 24, 3, 2), "f32", 192, "f32"), ((48, 12, 2, 2), "f32", 192, "f32"),
    ((24, 24, 2, 2), "f32", 288, "f32_r12"), ((16, 16, 4, 2), "bf16", 128, "bf16_r12"),
    ((48, 12, 3, 2), "bf16", 288, "bf16")])
def test_pipelined_equals_simple_kernel(qdpg_gpu, dims, prec, sites, lprec):
    """sites: most sites per tile (0 = default); 288 gives 12-row tiles at
    Lx = 24 and 6-row tiles at Lx = 48.  Whole-plane tiles with Lz = 1, 2, 3
    cover the staging of planes z-1, z, z+1 in one, two or three copies;
    halo tiles at the first, last and inner rows cover the y-halo runs,
    and every fixed halo shape (Lx 16, 24, 48) its row-major stages."""
    q = qdpg_gpu
    q.debug_set(q.TUNE_TILE_CONSUMERS, sites)
    try:
        _pipelined_vs_simple(q, dims, prec, lprec)
    finally:
        q.debug_set(q.TUNE_TILE_CONSUMERS, 0)


def _pipelined_vs_simple(q, dims, prec, lprec="f32"):
    lat = q.Lattice(dims, 3)
    U = fields.round_to_f32(fields.gauge_field(dims, 31, kind="haar"))
    psi = fields.round_to_f32(fields.propagator(dims, 31, envelope=0.3))
    p = q.PREC_NAMES[prec]
    Uf = _field(q, lat, q.GAUGE, q.PREC_NAMES[lprec], U)
    a = _field(q, lat, q.PROPAGATOR, p, psi)
    b = _field(q, lat, q.PROPAGATOR, p, psi)
    q.gauss_smear(Uf, a, 0.2, 3, scratch=a.like())                # pipelined kernel
    q.debug_set(q.DEBUG_FORCE_SIMPLE_HOP, 1)
    try:
        q.gauss_smear(Uf, b, 0.2, 3, scratch=b.like())            # one-thread-per-site kernel
    finally:
        q.debug_set(q.DEBUG_FORCE_SIMPLE_HOP, 0)
    q.device_status()
    ea, eb = a.export().cpu().numpy(), b.export().cpu().numpy()
    assert np.array_equal(ea, eb)
    if prec == "f32" and lprec == "f32":
        assert field_err(ea, smear.gauss_smear(U, psi, 0.2, 3)) <= TOL_F32


def test_pipeline_wait_runs_out_and_reports(qdpg_gpu):
    """Drop the copies of one pipeline stage: every wait for it gives up after
    2 ms, the kernel records the timeout and returns; the context stays usable."""
    q = qdpg_gpu
    dims = (8, 8, 8, 2)
    lat = q.Lattice(dims, 3)
    U = fields.round_to_f32(fields.gauge_field(dims, 33, kind="haar"))
    psi = fields.round_to_f32(fields.propagator(dims, 33, envelope=None))
    Uf = _field(q, lat, q.GAUGE, q.F32, U)
    f = _field(q, lat, q.PROPAGATOR, q.F32, psi)
    q.device_status()                                   # clean before
    q.debug_set(q.DEBUG_WAIT_TIMEOUT_NS, 2_000_000)
    q.debug_set(q.DEBUG_DROP_STAGE, 5)
    try:
        q.gauss_smear(Uf, f, 0.2, 1, scratch=f.like())
        with pytest.raises(q.QdpgError) as err:
            q.device_status()
        assert err.value.status == -6
    finally:
        q.debug_set(q.DEBUG_DROP_STAGE, -1)
        q.debug_set(q.DEBUG_WAIT_TIMEOUT_NS, 1_000_000_000)
    q.device_status()                                   # the flag was cleared
    g = _field(q, lat, q.PROPAGATOR, q.F32, psi)
    q.gauss_smear(Uf, g, 0.2, 2, scratch=g.like())
    q.device_status()
    assert field_err(g.export().cpu().numpy(), smear.gauss_smear(U, psi, 0.2, 2)) <= TOL_F32


def test_autotuner_picks_a_config_and_keeps_parity(qdpg_gpu, tmp_path):
    q = qdpg_gpu
    dims = (16, 16, 8, 2)
    lat = q.Lattice(dims, 3)
    U = fields.round_to_f32(fields.gauge_field(dims, 35, kind="near_unit"))
    psi = fields.round_to_f32(fields.propagator(dims, 35, envelope=0.3))
    Uf = _field(q, lat, q.GAUGE, q.F32, U)
    f = _field(q, lat, q.PROPAGATOR, q.F32, psi)
    sites, grid_mode, us = q.tune_smear(Uf, f, f.like(), reps=2)
    assert 32 <= sites <= 288 and grid_mode in (0, 1) and us > 0
    # psi is only read by the tuner
    assert np.array_equal(f.export().cpu().numpy(), psi)
    q.gauss_smear(Uf, f, 0.2, 4, scratch=f.like())
    q.device_status()
    assert field_err(f.export().cpu().numpy(), smear.gauss_smear(U, psi, 0.2, 4)) <= TOL_F32
    path = str(tmp_path / "tune.txt")
    q.tune_save(path)
    q.tune_load(path)
    text = open(path).read()
    assert f"16 16 8 2 3 {q.F32} {q.F32} {sites} {grid_mode}" in text


@pytest.mark.parametrize("prec,dims,sites", [("f32", (16, 16, 6, 2), 0), ("bf16", (16, 16, 6, 2), 0),
                                             ("f32", (24, 24, 4, 2), 288), ("f32", (48, 12, 3, 2), 96)])
def test_tensor_map_and_bulk_staging_agree(qdpg_gpu, prec, dims, sites):
    """Whole-plane tiles stage interior planes with one tensor-map copy per
    stage, halo tiles of a fixed shape stage row-major with five; the
    bulk-copy staging of the same rows gives the same bits."""
    q = qdpg_gpu
    q.debug_set(q.TUNE_TILE_CONSUMERS, sites)
    lat = q.Lattice(dims, 3)
    U = fields.round_to_f32(fields.gauge_field(dims, 37, kind="haar"))
    psi = fields.round_to_f32(fields.propagator(dims, 37, envelope=0.3))
    p = q.PREC_NAMES[prec]
    Uf = _field(q, lat, q.GAUGE, q.F32, U)
    outs = []
    for off in (0, 1):
        q.debug_set(q.TUNE_TENSOR_COPY, off)
        try:
            f = _field(q, lat, q.PROPAGATOR, p, psi)
            q.gauss_smear(Uf, f, 0.2, 4, scratch=f.like())
            q.device_status()
            outs.append(f.export().cpu().numpy())
        finally:
            q.debug_set(q.TUNE_TENSOR_COPY, 0)
    q.debug_set(q.TUNE_TILE_CONSUMERS, 0)
    assert np.array_equal(outs[0], outs[1])
    if prec == "f32":
        assert field_err(outs[0], smear.gauss_smear(U, psi, 0.2, 4)) <= TOL_F32
