"""The allocation-free smearing entry point, checked against the allocating one.

qdpg_gauss_smear_noalloc exists for callers that cannot allocate device
memory when they smear (their own pool manager owns all device memory, or
they must avoid the implicit synchronisation of cudaMalloc/cudaFree).  Its
ping-pong buffer is the library's 32 MiB static device array.  The test calls
it through the C ABI twice in a row -- the second call finds the first call's
data still in the shared array -- and compares each result with
qdpg_gauss_smear given a caller-owned scratch field.  It also checks that the
calls allocate nothing: the library's own allocation counter, the bytes in
use in its memory pool and torch's caching allocator stay unchanged.
FP32 and BF16 storage are covered, and a smearing long enough (kappa = 0.3,
N = 60) that the power-of-two rescaling runs through the static scratch.
"""
import ctypes
import gc

import numpy as np
import pytest
import torch

from synth import fields
from tests.parity_util import TOL_F32, field_err

pytestmark = pytest.mark.gpu

QDPG_ERR_ARG = -1


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _field(q, lat, kind, canon, prec=None):
    f = q.Field(lat, kind, q.F32 if prec is None else prec, device="cuda:0")
    return f.import_(torch.from_numpy(canon.astype(np.complex64)).to("cuda:0"))


def _memory_state(q):
    """The library's allocation counter and its pool's bytes in use, and
    torch's caching allocator (all unchanged by a call that allocates nothing)."""
    torch.cuda.synchronize()
    return q.device_alloc_count(), q.device_pool_used(), torch.cuda.memory_allocated()


@pytest.mark.parametrize("kind,prec,dims,n_iter,kappa", [
    ("prop", "f32", (8, 8, 8, 16), 7, 0.21),
    ("ferm", "f32", (16, 16, 16, 32), 6, 0.21),
    ("prop", "bf16", (8, 8, 8, 16), 5, 0.21),
    ("prop", "f32", (8, 8, 4, 8), 60, 0.3),      # growth bound > 40 bits: rescaled by 2^-31 every 21 hops
])
def test_noalloc_matches_allocating_entry_point(qdpg_gpu, kind, prec, dims, n_iter, kappa):
    q = qdpg_gpu
    lib = q.load()
    lat = q.Lattice(dims, 3)
    U = _field(q, lat, q.GAUGE, fields.round_to_f32(fields.gauge_field(dims, 21, kind="haar")))
    K = q.PROPAGATOR if kind == "prop" else q.FERMION
    P = q.PREC_NAMES[prec]
    tol = TOL_F32 if prec == "f32" else 1e-6      # BF16: both runs round identically; allow rounding-order slack
    for call, fid in enumerate((71, 72)):        # two calls in a row share the static scratch
        if kind == "prop":
            psi = fields.round_to_f32(fields.propagator(dims, 21, field_id=fid, envelope=0.3))
        else:
            psi = fields.round_to_f32(fields.fermion(dims, 21, field_id=fid))
        ref = _field(q, lat, K, psi, P)
        scratch = ref.like()
        q.gauss_smear(U, ref, kappa, n_iter + call, 3, scratch=scratch)
        got = _field(q, lat, K, psi, P)
        gc.collect()                             # no tensor of this test is freed inside the window below
        before = _memory_state(q)
        rc = lib.qdpg_gauss_smear_noalloc(U._h, got._h, kappa, n_iter + call, 3, _stream())
        assert rc == 0
        assert _memory_state(q) == before, "the allocation-free entry point allocated device memory"
        a = got.export().cpu().numpy()
        b = ref.export().cpu().numpy()
        assert field_err(a, b) <= tol, call


def test_noalloc_rejects_a_field_beyond_the_static_scratch(qdpg_gpu):
    q = qdpg_gpu
    lib = q.load()
    dims = (16, 16, 16, 32)                       # a 151 MB FP32 propagator > 32 MiB
    lat = q.Lattice(dims, 3)
    U = q.Field(lat, q.GAUGE, q.F32, device="cuda:0")
    psi = q.Field(lat, q.PROPAGATOR, q.F32, device="cuda:0")
    before = q.launch_count()
    rc = lib.qdpg_gauss_smear_noalloc(U._h, psi._h, 0.2, 3, 3, _stream())
    assert rc == QDPG_ERR_ARG
    buf = ctypes.create_string_buffer(256)
    lib.qdpg_last_error(buf, 256)
    assert b"static scratch" in buf.value
    assert q.launch_count() == before
