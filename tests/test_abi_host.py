"""The C ABI library loads, exports every declared symbol, and validates
arguments on the host (CPU only: no call here reaches the GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qdpg.h")

OK, ERR_ARG, ERR_SHAPE, ERR_DTYPE, ERR_UNSUPPORTED = 0, -1, -2, -3, -7


@pytest.fixture(scope="module")
def q():
    import paper_1111_5596_gb300 as q
    from paper_1111_5596_gb300 import build as b

    b.build()
    q.load()
    return q


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qdpg_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for needed in ("qdpg_lattice_create", "qdpg_field_wrap", "qdpg_shift", "qdpg_gauss_smear",
                   "qdpg_meson_2pt", "qdpg_point_source", "qdpg_field_import", "qdpg_field_export"):
        assert needed in names


def test_library_exports_every_declared_symbol(q):
    lib = ctypes.CDLL(q.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def _lat(q, dims, jd=3):
    h = ctypes.c_void_p()
    rc = q._lib.qdpg_lattice_create((ctypes.c_int * 4)(*dims), jd, ctypes.byref(h))
    return rc, h


def test_lattice_validation(q):
    assert _lat(q, (4, 4, 4, 8))[0] == OK
    assert _lat(q, (4, 0, 4, 8))[0] == ERR_ARG
    assert _lat(q, (4, 4, 4, 8), 4)[0] == ERR_ARG
    assert _lat(q, (4, 4, 4, 8), -1)[0] == ERR_ARG
    assert _lat(q, (2048, 2048, 2048, 2))[0] == ERR_ARG      # volume >= 2^31
    assert q._lib.qdpg_lattice_create(None, 3, None) == ERR_ARG
    buf = ctypes.create_string_buffer(256)
    assert q._lib.qdpg_last_error(buf, 256) == ERR_ARG
    assert b"null" in buf.value


def test_field_bytes_and_wrap_validation(q):
    rc, lat = _lat(q, (4, 6, 2, 3))
    V = 4 * 6 * 2 * 3
    fb = q._lib.qdpg_field_bytes
    rec = lambda n: (n + 255) // 256 * 256 + q.SCALE_RECORD_BYTES  # data padded to 256 B, then the scale record
    assert fb(lat, q.PROPAGATOR, q.F32) == rec(V * 144 * 8)
    assert fb(lat, q.PROPAGATOR, q.BF16) == rec(V * 144 * 4)
    assert fb(lat, q.GAUGE, q.F32) == V * 36 * 8
    assert fb(lat, q.GAUGE, q.F32_R12) == V * 24 * 8
    assert fb(lat, q.GAUGE, q.BF16_R12) == V * 24 * 4
    assert fb(lat, q.FERMION, q.F32) == rec(V * 12 * 8)
    assert fb(lat, q.COLOR_MATRIX, q.F32) == V * 9 * 8
    assert fb(lat, q.PROPAGATOR, q.F32_R12) == 0               # reconstruct-12 is gauge-only
    # float16 propagators: site-major data, padded to 256 bytes, then the scale record
    assert fb(lat, q.PROPAGATOR, q.F16) == rec(V * 144 * 4)
    assert fb(lat, q.GAUGE, q.F16) == V * 36 * 4
    assert fb(lat, q.GAUGE, q.F16_R12) == V * 24 * 4
    assert fb(lat, q.FERMION, q.F16) == 0                        # float16 is propagator/gauge only
    assert fb(lat, q.PROPAGATOR, q.F16_R12) == 0
    assert fb(lat, q.PROPAGATOR, 6) == 0
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(1 << 20)                             # never dereferenced by wrap
    need = fb(lat, q.FERMION, q.F32)
    w = q._lib.qdpg_field_wrap
    assert w(lat, q.FERMION, q.F32, fake, need, ctypes.byref(h)) == OK
    q._lib.qdpg_field_release(h)
    assert w(lat, q.FERMION, q.F32, fake, need - 1, ctypes.byref(h)) == ERR_SHAPE
    assert w(lat, q.FERMION, q.F32, None, need, ctypes.byref(h)) == ERR_ARG
    assert w(lat, q.FERMION, q.F32, ctypes.c_void_p((1 << 20) + 8), need, ctypes.byref(h)) == ERR_ARG
    assert w(lat, q.FERMION, q.F32_R12, fake, need, ctypes.byref(h)) == ERR_DTYPE
    q._lib.qdpg_lattice_destroy(lat)


def _no_device():
    import torch

    return not torch.cuda.is_available()


# The handles below wrap made-up device addresses; every call must fail its
# host-side checks before any launch.  Run only where no GPU can be reached.
host_only = pytest.mark.skipif(not _no_device(), reason="fake device addresses: host-only test")


def _wrap(q, lat, kind, prec, addr):
    h = ctypes.c_void_p()
    need = q._lib.qdpg_field_bytes(lat, kind, prec)
    assert q._lib.qdpg_field_wrap(lat, kind, prec, ctypes.c_void_p(addr), need, ctypes.byref(h)) == OK
    return h


@host_only
def test_operation_argument_errors_are_caught_on_host(q):
    L = q._lib
    launches_before = q.launch_count()
    _, lat = _lat(q, (4, 4, 4, 4))
    _, lat2 = _lat(q, (4, 4, 4, 6))
    U = _wrap(q, lat, q.GAUGE, q.F32, 1 << 24)
    P = _wrap(q, lat, q.PROPAGATOR, q.F32, 1 << 26)
    P2 = _wrap(q, lat2, q.PROPAGATOR, q.F32, 1 << 28)
    F = _wrap(q, lat, q.FERMION, q.F32, 1 << 30)
    Fb = _wrap(q, lat, q.FERMION, q.BF16, 1 << 31)
    gs = L.qdpg_gauss_smear
    assert gs(None, P, 0.2, 3, 3, None, None) == ERR_ARG
    assert gs(P, P, 0.2, 3, 3, None, None) == ERR_SHAPE         # U must be a gauge field
    assert gs(U, U, 0.2, 3, 3, None, None) == ERR_SHAPE
    assert gs(U, P2, 0.2, 3, 3, None, None) == ERR_SHAPE         # different lattice
    assert gs(U, P, 0.2, 3, 4, None, None) == ERR_ARG            # j_decay
    assert gs(U, P, 0.2, -1, 3, None, None) == ERR_ARG
    assert gs(U, P, float("nan"), 2, 3, None, None) == ERR_ARG
    assert gs(U, P, 0.2, 2, 3, F, None) == ERR_SHAPE              # scratch kind
    assert gs(U, F, 0.2, 2, 3, Fb, None) == ERR_SHAPE             # scratch precision
    assert gs(U, P, 0.2, 2, 3, P, None) == ERR_ARG                # scratch aliases psi
    assert gs(U, P, 0.2, 0, 3, None, None) == OK                  # zero iterations: no-op, no launch
    sh = L.qdpg_shift
    assert sh(P, P, 1, 0, None) == ERR_ARG                        # aliasing
    assert sh(P, F, 1, 0, None) == ERR_SHAPE
    assert sh(P2, P, 1, 0, None) == ERR_SHAPE
    assert sh(F, _wrap(q, lat, q.FERMION, q.F32, 1 << 32), 2, 0, None) == ERR_ARG
    assert sh(F, _wrap(q, lat, q.FERMION, q.F32, 1 << 33), 1, 4, None) == ERR_ARG
    ps = L.qdpg_point_source
    assert ps(U, (ctypes.c_int * 4)(0, 0, 0, 0), 0, None) == ERR_SHAPE
    assert ps(P, (ctypes.c_int * 4)(0, 0, 4, 0), 0, None) == ERR_ARG
    assert ps(F, (ctypes.c_int * 4)(0, 0, 0, 0), 12, None) == ERR_ARG
    m = L.qdpg_meson_2pt
    g = (ctypes.c_int * 1)(15)
    bad = (ctypes.c_int * 1)(16)
    mom = (ctypes.c_int * 3)(0, 0, 0)
    out = ctypes.c_void_p(1 << 34)
    assert m(P, F, g, g, 1, mom, 1, None, out, None) == ERR_SHAPE
    assert m(P, P2, g, g, 1, mom, 1, None, out, None) == ERR_SHAPE
    assert m(P, P, bad, g, 1, mom, 1, None, out, None) == ERR_ARG
    assert m(P, P, g, g, 0, mom, 1, None, out, None) == ERR_ARG
    assert m(P, P, g, g, 1, mom, 65, None, out, None) == ERR_ARG
    assert m(P, P, g, g, 1, mom, 1, None, None, None) == ERR_ARG
    b = L.qdpg_baryon_2pt
    assert b(P, P, 2, 1, mom, 1, None, out, None) == ERR_ARG          # kind
    assert b(P, P, 0, 0, mom, 1, None, out, None) == ERR_ARG          # parity
    assert b(P, None, 0, 1, mom, 1, None, out, None) == ERR_ARG       # nucleon needs Sd
    assert b(P, F, 0, 1, mom, 1, None, out, None) == ERR_SHAPE
    assert b(P, P2, 0, 1, mom, 1, None, out, None) == ERR_SHAPE
    assert b(P, P, 1, 1, mom, 65, None, out, None) == ERR_ARG
    assert L.qdpg_field_import(P, None, 0, None) == ERR_ARG
    assert L.qdpg_field_import(P, out, 7, None) == ERR_DTYPE
    # float16 propagators go with float16 links, on the layout's decay direction
    PH = _wrap(q, lat, q.PROPAGATOR, q.F16, 1 << 35)
    PH2 = _wrap(q, lat, q.PROPAGATOR, q.F16, 1 << 36)
    UH = _wrap(q, lat, q.GAUGE, q.F16_R12, 1 << 37)
    assert gs(U, PH, 0.2, 2, 3, None, None) == ERR_DTYPE
    assert gs(UH, P, 0.2, 2, 3, None, None) == ERR_DTYPE
    assert gs(UH, PH, 0.2, 2, 1, None, None) == ERR_UNSUPPORTED
    assert gs(UH, PH, 0.2, 1000, 3, None, None) == ERR_ARG       # more iterations than scale slots
    assert gs(UH, PH, 0.2, 2, 3, P, None) == ERR_SHAPE           # scratch precision
    assert gs(UH, PH, 0.2, 2, 3, PH, None) == ERR_ARG            # scratch aliases psi
    assert L.qdpg_gauss_smear_noalloc(UH, PH, 0.2, 2, 3, None) == ERR_DTYPE
    assert m(PH, P, g, g, 1, mom, 1, None, out, None) == ERR_DTYPE
    assert b(PH, P, 0, 1, mom, 1, None, out, None) == ERR_DTYPE
    assert sh(PH, P, 1, 0, None) == ERR_SHAPE
    assert L.qdpg_tune_smear(UH, PH, PH2, 3, 2, None) == ERR_UNSUPPORTED
    assert q.launch_count() == launches_before                    # every error came before a launch


@host_only
def test_batch_planning_validates_jobs_on_host(q):
    L = q._lib
    launches_before = q.launch_count()
    _, lat = _lat(q, (4, 4, 4, 4))
    _, lat2 = _lat(q, (4, 4, 4, 6))
    U = _wrap(q, lat, q.GAUGE, q.F32, 1 << 24)
    P = _wrap(q, lat, q.PROPAGATOR, q.F32, 1 << 26)
    Ps = _wrap(q, lat, q.PROPAGATOR, q.F32, 1 << 27)
    P2 = _wrap(q, lat2, q.PROPAGATOR, q.F32, 1 << 28)
    F = _wrap(q, lat, q.FERMION, q.F32, 1 << 30)
    Fb = _wrap(q, lat, q.FERMION, q.BF16, 1 << 31)
    mes = 1 << 34

    def create(*jobs, jd=3):
        arr = (q.CJob * max(1, len(jobs)))(*[q.CJob(*j) for j in jobs])
        h = ctypes.c_void_p()
        rc = L.qdpg_batch_create(arr, len(jobs), jd, ctypes.byref(h))
        if rc == OK:
            L.qdpg_batch_destroy(h)
        return rc

    good = (U, P, Ps, 0.2, 3, mes)
    assert create(good) == OK
    assert create(good, (U, F, _wrap(q, lat, q.FERMION, q.F32, 1 << 29), 0.1, 0, None)) == OK
    assert create(jd=4, *[good]) == ERR_ARG
    assert create() == ERR_ARG                                   # no jobs
    assert create((None, P, Ps, 0.2, 3, None)) == ERR_ARG
    assert create((P, P, Ps, 0.2, 3, None)) == ERR_SHAPE         # U must be a gauge field
    assert create((U, P, P, 0.2, 3, None)) == ERR_SHAPE          # scratch aliases psi
    assert create((U, P, F, 0.2, 3, None)) == ERR_SHAPE          # scratch kind
    assert create((U, F, Fb, 0.2, 3, None)) == ERR_SHAPE         # scratch precision
    assert create((U, P2, Ps, 0.2, 3, None)) == ERR_SHAPE        # different lattice
    assert create((U, P, Ps, float("nan"), 3, None)) == ERR_ARG
    assert create((U, P, Ps, 0.2, -1, None)) == ERR_ARG
    assert create((U, F, Fb, 0.2, 3, mes)) == ERR_SHAPE          # mesons need a propagator
    assert L.qdpg_batch_create(None, 1, 3, ctypes.byref(ctypes.c_void_p())) == ERR_ARG
    assert L.qdpg_batch_run(None, 0, None) == ERR_ARG
    L.qdpg_batch_destroy(None)
    assert q.launch_count() == launches_before


def test_tuning_settings_are_validated_on_host(q):
    """Launch-shape settings of the smearing kernels: accepted within their
    ranges, rejected outside them, and reset to the defaults."""
    L = q._lib
    TILE, STAGES, F16_WARPS, TENSOR_COPY = 4, 5, 8, 9
    try:
        assert L.qdpg_debug_set(TILE, 288) == OK                # 12-row tiles at Lx = 24
        assert L.qdpg_debug_set(TILE, 289) == ERR_ARG
        assert L.qdpg_debug_set(TILE, 16) == ERR_ARG
        assert L.qdpg_debug_set(STAGES, 17) == ERR_ARG
        assert L.qdpg_debug_set(F16_WARPS, 12) == ERR_ARG
        assert L.qdpg_debug_set(TENSOR_COPY, 1) == OK           # bulk copies only
        assert L.qdpg_debug_set(TENSOR_COPY, 2) == ERR_ARG
        assert L.qdpg_debug_set(99, 0) == ERR_ARG               # unknown setting
    finally:
        for what in (TILE, STAGES, F16_WARPS, TENSOR_COPY):
            assert L.qdpg_debug_set(what, 0) == OK


def test_host_io_and_alloc_hooks_validate_on_host(q):
    lib = q._lib
    assert lib.qdpg_field_import_host(None, None, 0, None) == ERR_ARG
    assert lib.qdpg_field_export_host(None, None, None) == ERR_ARG
    assert lib.qdpg_debug_set(q.DEBUG_FAIL_ALLOCS, -1) == ERR_ARG
    assert lib.qdpg_debug_set(q.DEBUG_STAGE_BYTES, -5) == ERR_ARG
    assert lib.qdpg_debug_set(q.DEBUG_FAIL_ALLOCS, 0) == OK
    assert lib.qdpg_debug_set(q.DEBUG_STAGE_BYTES, 0) == OK
    assert isinstance(q.device_alloc_count(), int)
