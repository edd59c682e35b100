"""Python binding of libqdpg: Gaussian smearing and hadron contractions on GB300.

Argument marshalling only: every operation runs in the CUDA kernels of
libqdpg.so, called through its C ABI (``include/qdpg.h``).  PyTorch provides
device memory and the current CUDA stream.  There is no CPU fallback: if the
library is missing, every call raises.

Names follow QDP++/Chroma: a :class:`Lattice` with a decay direction,
fields of kind GAUGE / PROPAGATOR / FERMION / COLOR_MATRIX, ``shift``,
``gauss_smear``, ``point_source`` and ``meson_2pt``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqdpg.so")

COLOR_MATRIX, GAUGE, FERMION, PROPAGATOR = 0, 1, 2, 3
F32, BF16, F32_R12, BF16_R12, F16, F16_R12 = 0, 1, 2, 3, 4, 5
CANON_F64, CANON_F32 = 0, 1
SCALE_RECORD_BYTES = 8192

PREC_NAMES = {"f32": F32, "bf16": BF16, "f32_r12": F32_R12, "bf16_r12": BF16_R12, "f16": F16, "f16_r12": F16_R12}

_lib = None


class QdpgError(RuntimeError):
    """A libqdpg call returned a non-zero status."""

    def __init__(self, status: int, message: str):
        super().__init__(f"qdpg status {status}: {message}")
        self.status = status


class CJob(ctypes.Structure):
    """Mirror of the C struct qdpg_job."""

    _fields_ = [("U", ctypes.c_void_p), ("psi", ctypes.c_void_p), ("scratch", ctypes.c_void_p),
                ("kappa", ctypes.c_double), ("n_iter", ctypes.c_int), ("mesons_out", ctypes.c_void_p)]


def load() -> ctypes.CDLL:
    """Load libqdpg.so (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libqdpg.so not built ({LIB_PATH}); run __graft_entry__.build() first")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    ip = ctypes.POINTER(ctypes.c_int)
    sig = {
        "qdpg_version": (i, []),
        "qdpg_launch_count": (ctypes.c_uint64, []),
        "qdpg_last_error": (i, [ctypes.c_char_p, sz]),
        "qdpg_lattice_create": (i, [ip, i, ctypes.POINTER(vp)]),
        "qdpg_lattice_destroy": (None, [vp]),
        "qdpg_field_bytes": (sz, [vp, i, i]),
        "qdpg_field_wrap": (i, [vp, i, i, vp, sz, ctypes.POINTER(vp)]),
        "qdpg_field_release": (None, [vp]),
        "qdpg_field_import": (i, [vp, vp, i, vp]),
        "qdpg_field_export": (i, [vp, vp, vp]),
        "qdpg_field_import_host": (i, [vp, vp, i, vp]),
        "qdpg_field_export_host": (i, [vp, vp, vp]),
        "qdpg_device_alloc_count": (ctypes.c_uint64, []),
        "qdpg_device_pool_used": (i, [ctypes.POINTER(ctypes.c_uint64)]),
        "qdpg_point_source": (i, [vp, ip, i, vp]),
        "qdpg_shift": (i, [vp, vp, i, i, vp]),
        "qdpg_gauss_smear": (i, [vp, vp, d, i, i, vp, vp]),
        "qdpg_gauss_smear_noalloc": (i, [vp, vp, d, i, i, vp]),
        "qdpg_meson_2pt": (i, [vp, vp, ip, ip, i, ip, i, ip, vp, vp]),
        "qdpg_meson_2pt_multi": (i, [ctypes.POINTER(vp), i, ip, ip, i, ip, i, ip, vp, vp]),
        "qdpg_baryon_2pt": (i, [vp, vp, i, i, ip, i, ip, vp, vp]),
        "qdpg_meson_sites": (i, [vp, vp, ip, ip, i, vp, vp]),
        "qdpg_baryon_sites": (i, [vp, vp, i, i, vp, vp]),
        "qdpg_momentum_project": (i, [vp, vp, i, ip, i, ip, vp, vp]),
        "qdpg_device_status": (i, [vp]),
        "qdpg_debug_set": (i, [i, ctypes.c_longlong]),
        "qdpg_tune_smear": (i, [vp, vp, vp, i, i, vp]),
        "qdpg_tune_query": (i, [vp, vp, ip, ip, ctypes.POINTER(ctypes.c_float)]),
        "qdpg_tune_save": (i, [ctypes.c_char_p]),
        "qdpg_tune_load": (i, [ctypes.c_char_p]),
        "qdpg_profile_enable": (i, [i]),
        "qdpg_profile_reset": (i, []),
        "qdpg_profile_query": (i, [ctypes.c_char_p, ctypes.POINTER(d), ctypes.POINTER(ctypes.c_uint64)]),
        "qdpg_batch_create": (i, [ctypes.POINTER(CJob), i, i, vp]),
        "qdpg_batch_run": (i, [vp, i, vp]),
        "qdpg_batch_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int):
    if status != 0:
        buf = ctypes.create_string_buffer(512)
        _lib.qdpg_last_error(buf, 512)
        raise QdpgError(status, buf.value.decode())


def _ints(vals):
    arr = (ctypes.c_int * len(vals))(*[int(v) for v in vals])
    return arr


def _stream(stream=None):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def launch_count() -> int:
    """Kernels libqdpg has launched in this process."""
    return int(load().qdpg_launch_count())


DEBUG_WAIT_TIMEOUT_NS, DEBUG_DROP_STAGE, DEBUG_FORCE_SIMPLE_HOP = 1, 2, 3
DEBUG_FAIL_ALLOCS, DEBUG_STAGE_BYTES, DEBUG_MESON_FORM = 11, 12, 13
TUNE_TILE_CONSUMERS, TUNE_STAGES, TUNE_GRID, TUNE_TENSOR_COPY = 4, 5, 7, 9


def device_alloc_count() -> int:
    """Device allocations libqdpg has made for its own temporaries in this process."""
    return int(load().qdpg_device_alloc_count())


def device_pool_used() -> int:
    """Bytes in use in libqdpg's own device memory pool on the current device."""
    v = ctypes.c_uint64()
    _check(load().qdpg_device_pool_used(ctypes.byref(v)))
    return int(v.value)


def device_status(stream=None):
    """Synchronise the stream and raise QdpgError(-6) if a kernel's bounded wait gave up."""
    _check(load().qdpg_device_status(_stream(stream)))


def debug_set(what: int, value: int):
    """Test hooks: wait time limit (ns), dropped pipeline stage, forced simple hop kernel."""
    _check(load().qdpg_debug_set(int(what), int(value)))


def profile_enable(on: bool = True):
    """Bracket every library kernel launch with CUDA events on its stream."""
    _check(load().qdpg_profile_enable(1 if on else 0))


def profile_reset():
    _check(load().qdpg_profile_reset())


def profile_query(name: str) -> tuple[float, int]:
    """(summed kernel time in ms, launches) of one kernel name since the last reset."""
    ms = ctypes.c_double()
    n = ctypes.c_uint64()
    _check(load().qdpg_profile_query(name.encode(), ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, int(n.value)


class Lattice:
    """Lattice extents ``dims = (L0, L1, L2, L3)`` (x0 fastest) and decay direction."""

    def __init__(self, dims, j_decay: int = 3):
        lib = load()
        self.dims = tuple(int(x) for x in dims)
        self.j_decay = int(j_decay)
        h = ctypes.c_void_p()
        _check(lib.qdpg_lattice_create(_ints(self.dims), self.j_decay, ctypes.byref(h)))
        self._h = h

    @property
    def Nt(self) -> int:
        return self.dims[self.j_decay]

    @property
    def V(self) -> int:
        return int(np.prod(self.dims))

    @property
    def V3(self) -> int:
        return self.V // self.Nt

    def field_bytes(self, kind: int, prec: int) -> int:
        return int(_lib.qdpg_field_bytes(self._h, kind, prec))

    def canonical_shape(self, kind: int) -> tuple:
        L0, L1, L2, L3 = self.dims
        sites = (L3, L2, L1, L0)
        return {COLOR_MATRIX: sites + (3, 3), GAUGE: (4,) + sites + (3, 3),
                FERMION: sites + (4, 3), PROPAGATOR: sites + (4, 3, 4, 3)}[kind]

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.qdpg_lattice_destroy(self._h)
            self._h = None


class Field:
    """A lattice-wide field in device layout, backed by a torch CUDA byte tensor."""

    def __init__(self, lattice: Lattice, kind: int, prec: int = F32, device=None, storage=None):
        import torch

        self.lattice, self.kind, self.prec = lattice, int(kind), int(prec)
        nbytes = lattice.field_bytes(self.kind, self.prec)
        if nbytes == 0:
            raise QdpgError(-3, f"precision {prec} is not valid for kind {kind}")
        if storage is None:
            storage = torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")
        if storage.numel() * storage.element_size() < nbytes or not storage.is_cuda:
            raise ValueError("storage must be a CUDA tensor of at least field_bytes bytes")
        self.storage = storage
        self.nbytes = nbytes
        h = ctypes.c_void_p()
        _check(_lib.qdpg_field_wrap(lattice._h, self.kind, self.prec, ctypes.c_void_p(storage.data_ptr()),
                                    nbytes, ctypes.byref(h)))
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.qdpg_field_release(self._h)
            self._h = None

    def import_(self, canonical, stream=None) -> "Field":
        """Fill from a canonical-layout complex tensor (complex128 or complex64) on this device."""
        import torch

        if not isinstance(canonical, torch.Tensor) or not canonical.is_cuda:
            raise ValueError("canonical data must be a CUDA tensor (copy it with .to('cuda') first)")
        if tuple(canonical.shape) != self.lattice.canonical_shape(self.kind):
            raise ValueError(f"canonical shape {tuple(canonical.shape)} != "
                             f"{self.lattice.canonical_shape(self.kind)}")
        if canonical.dtype == torch.complex128:
            ctype = CANON_F64
        elif canonical.dtype == torch.complex64:
            ctype = CANON_F32
        else:
            raise ValueError("canonical data must be complex128 or complex64")
        canonical = canonical.contiguous()
        _check(_lib.qdpg_field_import(self._h, ctypes.c_void_p(canonical.data_ptr()), ctype, _stream(stream)))
        self._keep = canonical  # stay alive until the stream has consumed it
        return self

    def export(self, stream=None):
        """Return the field as a canonical-layout complex128 CUDA tensor."""
        import torch

        out = torch.empty(self.lattice.canonical_shape(self.kind), dtype=torch.complex128,
                          device=self.storage.device)
        _check(_lib.qdpg_field_export(self._h, ctypes.c_void_p(out.data_ptr()), _stream(stream)))
        return out

    def import_host(self, canonical, stream=None) -> "Field":
        """Fill from a canonical-layout complex128/complex64 array in host memory
        (numpy array or CPU tensor; page-locked memory keeps the call
        asynchronous).  The library stages the data through its own device
        buffer; the host array is kept alive until the stream has passed."""
        import torch

        if isinstance(canonical, np.ndarray):
            canonical = torch.from_numpy(canonical)
        if not isinstance(canonical, torch.Tensor) or canonical.is_cuda:
            raise ValueError("canonical data must be a host (CPU) array")
        if tuple(canonical.shape) != self.lattice.canonical_shape(self.kind):
            raise ValueError(f"canonical shape {tuple(canonical.shape)} != "
                             f"{self.lattice.canonical_shape(self.kind)}")
        if canonical.dtype == torch.complex128:
            ctype = CANON_F64
        elif canonical.dtype == torch.complex64:
            ctype = CANON_F32
        else:
            raise ValueError("canonical data must be complex128 or complex64")
        canonical = canonical.contiguous()
        _check(_lib.qdpg_field_import_host(self._h, ctypes.c_void_p(canonical.data_ptr()), ctype, _stream(stream)))
        self._keep = canonical
        return self

    def export_host(self, out=None, stream=None):
        """Write the field to a canonical-layout complex128 CPU tensor (page-locked
        if ``out`` is not given).  Asynchronous: synchronise the stream before
        reading the result."""
        import torch

        shape = self.lattice.canonical_shape(self.kind)
        if out is None:
            out = torch.empty(shape, dtype=torch.complex128, pin_memory=True)
        if out.is_cuda or out.dtype != torch.complex128 or tuple(out.shape) != shape or not out.is_contiguous():
            raise ValueError("out must be a contiguous complex128 CPU tensor of the canonical shape")
        _check(_lib.qdpg_field_export_host(self._h, ctypes.c_void_p(out.data_ptr()), _stream(stream)))
        return out

    def like(self) -> "Field":
        return Field(self.lattice, self.kind, self.prec, device=self.storage.device)


def point_source(field: Field, x0=(0, 0, 0, 0), spin_color: int = 0, stream=None) -> Field:
    _check(_lib.qdpg_point_source(field._h, _ints(x0), int(spin_color), _stream(stream)))
    return field


def shift(dst: Field, src: Field, sign: int, mu: int, stream=None) -> Field:
    """dst(x) = src(x + sign * mu_hat)."""
    _check(_lib.qdpg_shift(dst._h, src._h, int(sign), int(mu), _stream(stream)))
    return dst


def gauss_smear(U: Field, psi: Field, kappa: float, n_iter: int, j_decay: int = 3, scratch: Field | None = None,
                stream=None) -> Field:
    """In-place Gaussian smearing of ``psi`` (n_iter covariant hops)."""
    _check(_lib.qdpg_gauss_smear(U._h, psi._h, float(kappa), int(n_iter), int(j_decay),
                                 scratch._h if scratch is not None else None, _stream(stream)))
    return psi


def gauss_smear_noalloc(U: Field, psi: Field, kappa: float, n_iter: int, j_decay: int = 3, stream=None) -> Field:
    """Gaussian smearing that allocates nothing: the library's 32 MiB static
    device scratch serves as the ping-pong buffer, so ``psi`` may be at most
    that size.  For callers that cannot allocate device memory when they
    smear.  Calls that overlap on the GPU share the scratch and race."""
    _check(_lib.qdpg_gauss_smear_noalloc(U._h, psi._h, float(kappa), int(n_iter), int(j_decay), _stream(stream)))
    return psi


def tune_smear(U: Field, psi: Field, scratch: Field, j_decay: int = 3, reps: int = 5, stream=None):
    """Time the pipelined smearing kernel's launch shapes on these fields and
    keep the fastest for later gauss_smear calls; returns (sites per tile,
    grid mode, microseconds per hop)."""
    _check(_lib.qdpg_tune_smear(U._h, psi._h, scratch._h, int(j_decay), int(reps), _stream(stream)))
    c, gm, us = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
    _check(_lib.qdpg_tune_query(U._h, psi._h, ctypes.byref(c), ctypes.byref(gm), ctypes.byref(us)))
    return c.value, gm.value, us.value


def tune_save(path: str):
    _check(load().qdpg_tune_save(path.encode()))


def tune_load(path: str):
    _check(load().qdpg_tune_load(path.encode()))


def meson_2pt(S1: Field, S2: Field, channels, moms=((0, 0, 0),), origin=None, out=None, stream=None):
    """Meson correlators, complex128 CUDA tensor of shape (n_chan, n_mom, Nt)."""
    import torch

    channels = list(channels)
    moms = [tuple(m) for m in moms]
    nt = S1.lattice.Nt
    if out is None:
        out = torch.empty((len(channels), len(moms), nt), dtype=torch.complex128, device=S1.storage.device)
    flat = [c for m in moms for c in m]
    _check(_lib.qdpg_meson_2pt(S1._h, S2._h, _ints([c[0] for c in channels]), _ints([c[1] for c in channels]),
                               len(channels), _ints(flat), len(moms),
                               _ints(origin) if origin is not None else None,
                               ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def meson_2pt_multi(props, channels, moms=((0, 0, 0),), origin=None, out=None, stream=None):
    """Meson correlators of every ordered pair of the propagators in one pass,
    complex128 CUDA tensor (n, n, n_chan, n_mom, Nt): out[a, b] is
    meson_2pt(props[a], props[b], ...)."""
    import torch

    props = list(props)
    channels = list(channels)
    moms = [tuple(m) for m in moms]
    n, nt = len(props), props[0].lattice.Nt
    if out is None:
        out = torch.empty((n, n, len(channels), len(moms), nt), dtype=torch.complex128, device=props[0].storage.device)
    handles = (ctypes.c_void_p * n)(*[p._h.value for p in props])
    flat = [c for m in moms for c in m]
    _check(_lib.qdpg_meson_2pt_multi(handles, n, _ints([c[0] for c in channels]), _ints([c[1] for c in channels]),
                                     len(channels), _ints(flat), len(moms),
                                     _ints(origin) if origin is not None else None,
                                     ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


NUCLEON, DELTA = 0, 1


def baryon_2pt(Su: Field, Sd: Field | None = None, kind: int = NUCLEON, parity: int = +1, moms=((0, 0, 0),),
               origin=None, out=None, stream=None):
    """Nucleon (kind 0, uud) or Delta++ (kind 1, uuu) correlator, complex128 CUDA tensor (n_mom, Nt)."""
    import torch

    moms = [tuple(m) for m in moms]
    if out is None:
        out = torch.empty((len(moms), Su.lattice.Nt), dtype=torch.complex128, device=Su.storage.device)
    flat = [c for m in moms for c in m]
    _check(_lib.qdpg_baryon_2pt(Su._h, Sd._h if Sd is not None else None, int(kind), int(parity), _ints(flat),
                                len(moms), _ints(origin) if origin is not None else None,
                                ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def meson_sites(S1: Field, S2: Field, channels, out=None, stream=None):
    """Site traces of the meson channels, complex64 CUDA tensor (n_chan, Nt, V3)."""
    import torch

    channels = list(channels)
    lat = S1.lattice
    if out is None:
        out = torch.empty((len(channels), lat.Nt, lat.V3), dtype=torch.complex64, device=S1.storage.device)
    _check(_lib.qdpg_meson_sites(S1._h, S2._h, _ints([c[0] for c in channels]), _ints([c[1] for c in channels]),
                                 len(channels), ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def baryon_sites(Su: Field, Sd: Field | None = None, kind: int = NUCLEON, parity: int = +1, out=None, stream=None):
    """Baryon site values, complex64 CUDA tensor (Nt, V3)."""
    import torch

    lat = Su.lattice
    if out is None:
        out = torch.empty((lat.Nt, lat.V3), dtype=torch.complex64, device=Su.storage.device)
    _check(_lib.qdpg_baryon_sites(Su._h, Sd._h if Sd is not None else None, int(kind), int(parity),
                                  ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def momentum_project(lattice: Lattice, sites, moms, origin=None, out=None, stream=None):
    """Project site values (n_chan, Nt, V3) complex64 onto momenta on the tensor
    cores; complex128 CUDA tensor (n_chan, n_mom, Nt)."""
    import torch

    if sites.dtype != torch.complex64 or not sites.is_cuda or not sites.is_contiguous():
        raise ValueError("sites must be a contiguous complex64 CUDA tensor")
    n_chan = sites.numel() // (lattice.Nt * lattice.V3)
    if n_chan * lattice.Nt * lattice.V3 != sites.numel():
        raise ValueError("sites size is not a multiple of Nt*V3")
    moms = [tuple(m) for m in moms]
    if out is None:
        out = torch.empty((n_chan, len(moms), lattice.Nt), dtype=torch.complex128, device=sites.device)
    flat = [c for m in moms for c in m]
    _check(_lib.qdpg_momentum_project(lattice._h, ctypes.c_void_p(sites.data_ptr()), n_chan, _ints(flat), len(moms),
                                      _ints(origin) if origin is not None else None,
                                      ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def momenta_up_to(n2max: int = 4):
    """Integer momenta (nx, ny, nz) with nx^2 + ny^2 + nz^2 <= n2max (33 for 4)."""
    r = int(n2max ** 0.5)
    return [(a, b, c) for a in range(-r, r + 1) for b in range(-r, r + 1) for c in range(-r, r + 1)
            if a * a + b * b + c * c <= n2max]


SIXTEEN_MESONS = tuple((n, n) for n in range(16))


class Batch:
    """Many independent smear (+ 16 zero-momentum mesons) jobs run together.

    ``jobs``: sequence of ``(U, psi, scratch, kappa, n_iter, mesons)`` with
    ``mesons`` a complex128 CUDA tensor of shape (16, Nt) or None.  Each run
    smears every psi in place and, where ``mesons`` is given, writes
    ``mesons[j, t]`` for channel Gamma(j) at sink and source."""

    def __init__(self, jobs, j_decay: int = 3):
        import torch

        lib = load()
        jobs = list(jobs)
        arr = (CJob * max(1, len(jobs)))()
        keep = []
        for k, (U, psi, scratch, kappa, n_iter, mes) in enumerate(jobs):
            if mes is not None:
                if not (isinstance(mes, torch.Tensor) and mes.is_cuda and mes.dtype == torch.complex128
                        and mes.is_contiguous() and tuple(mes.shape) == (16, psi.lattice.Nt)):
                    raise ValueError("mesons must be a contiguous complex128 CUDA tensor of shape (16, Nt)")
            arr[k] = CJob(U._h, psi._h, scratch._h, float(kappa), int(n_iter),
                          mes.data_ptr() if mes is not None else None)
            keep.append((U, psi, scratch, mes))
        h = ctypes.c_void_p()
        _check(lib.qdpg_batch_create(arr, len(jobs), int(j_decay), ctypes.byref(h)))
        self._h, self._keep = h, keep

    def run(self, use_graph: bool = False, stream=None):
        """Issue every job on the stream; with ``use_graph`` the first call also
        captures a CUDA graph that later calls launch."""
        _check(_lib.qdpg_batch_run(self._h, 1 if use_graph else 0, _stream(stream)))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.qdpg_batch_destroy(self._h)
            self._h = None
