"""Host-buffer import and export through the C ABI (qdpg_field_import_host,
qdpg_field_export_host): canonical host data -> device field -> canonical
host data, in chunks of whole timeslices through the library's own staging
buffer.  Each precision must give the same device bits as the device-buffer
import and the same values back as the device-buffer export; FP32 storage
of complex64 input round-trips bit for bit.  Small chunk bounds force many
chunks (one timeslice per chunk, and ragged last chunks)."""
import numpy as np
import pytest
import torch

from synth import fields

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _canon(q, lat, kind, seed):
    dims = lat.dims
    if kind == q.GAUGE:
        return fields.round_to_f32(fields.gauge_field(dims, seed, kind="haar"))
    if kind == q.PROPAGATOR:
        return fields.round_to_f32(fields.propagator(dims, seed, envelope=0.3))
    return fields.round_to_f32(fields.fermion(dims, seed))


CASES = [
    # kind, precision, dims, j_decay, chunk bytes (0 = default)
    ("prop", "f32", (6, 4, 5, 7), 3, 1),
    ("prop", "f32", (6, 4, 5, 7), 3, 3 * 6 * 4 * 5 * 144 * 16),   # 3 timeslices per chunk, ragged last
    ("prop", "bf16", (8, 4, 4, 5), 3, 2 * 8 * 4 * 4 * 144 * 8),
    ("prop", "f16", (8, 4, 4, 6), 3, 1),
    ("prop", "f32", (4, 6, 3, 5), 1, 0),                            # decay direction 1: one chunk
    ("gauge", "f32", (4, 4, 6, 5), 3, 1),
    ("gauge", "f32_r12", (4, 4, 6, 5), 3, 2 * 4 * 4 * 6 * 36 * 16),
    ("gauge", "bf16_r12", (4, 4, 4, 4), 3, 0),
    ("gauge", "f16", (8, 4, 4, 3), 3, 1),
    ("ferm", "f32", (4, 4, 4, 9), 3, 1),
]


@pytest.mark.parametrize("kind,prec,dims,jd,chunk", CASES)
@pytest.mark.parametrize("ctype", ["c64", "c128"])
def test_host_import_export_matches_device_path(qdpg_gpu, kind, prec, dims, jd, chunk, ctype):
    q = qdpg_gpu
    K = {"prop": q.PROPAGATOR, "gauge": q.GAUGE, "ferm": q.FERMION}[kind]
    P = q.PREC_NAMES[prec]
    lat = q.Lattice(dims, jd)
    canon = _canon(q, lat, K, 17)
    host = canon.astype(np.complex64 if ctype == "c64" else np.complex128)
    q.debug_set(q.DEBUG_STAGE_BYTES, chunk)
    try:
        pinned = torch.from_numpy(host).pin_memory()
        a = q.Field(lat, K, P, device=DEV).import_host(pinned)
        b = q.Field(lat, K, P, device=DEV).import_(torch.from_numpy(host).to(DEV))
        back_host = a.export_host()
        back_dev = b.export()
        torch.cuda.synchronize()
    finally:
        q.debug_set(q.DEBUG_STAGE_BYTES, 0)
    q.device_status()
    # same device bits: the data, and the scale's exponent and bound at the
    # head of a propagator's or fermion's scale record
    nb = a.nbytes - (q.SCALE_RECORD_BYTES if K != q.GAUGE else 0)
    assert torch.equal(a.storage[:nb], b.storage[:nb])
    if K != q.GAUGE:
        assert torch.equal(a.storage[nb:nb + 8], b.storage[nb:nb + 8])
    assert torch.equal(back_host, back_dev.cpu())     # same values back
    if prec == "f32":
        assert np.array_equal(back_host.numpy(), canon)   # FP32-representable input: exact round trip


def test_host_import_pageable_memory(qdpg_gpu):
    q = qdpg_gpu
    lat = q.Lattice((4, 4, 4, 8), 3)
    canon = _canon(q, lat, q.PROPAGATOR, 5)
    a = q.Field(lat, q.PROPAGATOR, q.F32, device=DEV).import_host(canon.astype(np.complex64))  # pageable numpy
    out = torch.empty(lat.canonical_shape(q.PROPAGATOR), dtype=torch.complex128)             # pageable tensor
    a.export_host(out)
    torch.cuda.synchronize()
    assert np.array_equal(out.numpy(), canon)


def test_allocation_failures_return_nomem_and_recover(qdpg_gpu):
    """Every call that allocates a temporary reports QDPG_ERR_NOMEM when the
    allocation fails (forced by the host-side hook), launches nothing, and the
    same call succeeds once allocations work again."""
    q = qdpg_gpu
    dims = (4, 4, 4, 8)
    lat = q.Lattice(dims, 3)
    U = q.Field(lat, q.GAUGE, q.F32, device=DEV).import_(torch.from_numpy(_canon(q, lat, q.GAUGE, 3)).to(DEV))
    S = q.Field(lat, q.PROPAGATOR, q.F32, device=DEV).import_(
        torch.from_numpy(_canon(q, lat, q.PROPAGATOR, 4).astype(np.complex64)).to(DEV))
    moms = q.momenta_up_to(4)                       # 33 momenta: site values go to a temporary
    host = _canon(q, lat, q.PROPAGATOR, 4)
    calls = {
        "gauss_smear without scratch": lambda: q.gauss_smear(U, S, 0.2, 2, 3),
        "meson_2pt at 33 momenta": lambda: q.meson_2pt(S, S, q.SIXTEEN_MESONS, moms),
        "baryon_2pt at 33 momenta": lambda: q.baryon_2pt(S, S, q.NUCLEON, +1, moms),
        "field_import_host": lambda: q.Field(lat, q.PROPAGATOR, q.F32, device=DEV).import_host(host),
        "field_export_host": lambda: S.export_host(),
    }
    for name, call in calls.items():
        n0 = q.device_alloc_count()
        q.debug_set(q.DEBUG_FAIL_ALLOCS, 1)
        try:
            with pytest.raises(q.QdpgError) as ei:
                call()
        finally:
            q.debug_set(q.DEBUG_FAIL_ALLOCS, 0)
        assert ei.value.status == -5, (name, ei.value)
        assert "refused" in str(ei.value), name
        assert q.device_alloc_count() == n0, name
        call()                                       # allocations work again
        torch.cuda.synchronize()
        assert q.device_alloc_count() > n0, name
    q.device_status()
