"""Seeded synthetic inputs generated on the GPU with torch, for workloads too
large to synthesise on the host within a benchmark run (the 64-job batch
with sixteen 24^3x48 lattices, the 48^3x96 scale run).

Same recipes as ``synth.fields`` -- Haar-random SU(3) links (Gram-Schmidt
of a complex Gaussian matrix, phases fixed so that det = 1) or near-unit
links exp(i eps H) with H a Gaussian combination of the Gell-Mann
matrices (here through the matrix exponential), propagator
entries that are complex Gaussians with E|z|^2 = 1 times
exp(-envelope |x - x0|) with the minimal-image distance -- but drawn from
torch's Philox generator on the device, so the values differ from the host
streams.  Nothing here belongs to the method's arithmetic: these are inputs.
"""
from __future__ import annotations

import math

import torch


def _gen(seed: int, field_id: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed((int(seed) * 1000003 + int(field_id)) % (1 << 63))
    return g


def _complex_normal(shape, gen, device) -> torch.Tensor:
    """Complex Gaussians with E|z|^2 = 1 (complex64)."""
    z = torch.randn(tuple(shape) + (2,), generator=gen, device=device, dtype=torch.float32)
    return torch.view_as_complex(z * math.sqrt(0.5))


def haar_su3(n: int, gen, device) -> torch.Tensor:
    """n Haar-random SU(3) matrices, complex64, shape (n, 3, 3)."""
    z = _complex_normal((n, 3, 3), gen, device).to(torch.complex128)
    cols = []
    for j in range(3):
        v = z[:, :, j]
        for u in cols:
            v = v - (u.conj() * v).sum(-1, keepdim=True) * u
        v = v / torch.linalg.vector_norm(v, dim=-1, keepdim=True)
        cols.append(v)
    q = torch.stack(cols, dim=-1)                      # unitary, R with positive diagonal
    det = torch.linalg.det(q)
    q = q / torch.pow(det, 1.0 / 3.0)[:, None, None]   # principal cube root: det -> 1
    return q.to(torch.complex64)


def _gell_mann(device) -> torch.Tensor:
    """The eight Gell-Mann matrices, shape (8, 3, 3), complex128."""
    s3 = 1.0 / math.sqrt(3.0)
    m = torch.zeros((8, 3, 3), dtype=torch.complex128)
    m[0, 0, 1] = m[0, 1, 0] = 1
    m[1, 0, 1], m[1, 1, 0] = -1j, 1j
    m[2, 0, 0], m[2, 1, 1] = 1, -1
    m[3, 0, 2] = m[3, 2, 0] = 1
    m[4, 0, 2], m[4, 2, 0] = -1j, 1j
    m[5, 1, 2] = m[5, 2, 1] = 1
    m[6, 1, 2], m[6, 2, 1] = -1j, 1j
    m[7, 0, 0], m[7, 1, 1], m[7, 2, 2] = s3, s3, -2 * s3
    return m.to(device)


def near_unit_su3(n: int, gen, device, eps: float = 0.3) -> torch.Tensor:
    """n SU(3) matrices exp(i eps H), H = sum_a h_a lambda_a / 2 with
    h_a ~ N(0, 1), complex64, shape (n, 3, 3) (matrix exponential of the
    anti-Hermitian traceless i eps H)."""
    h = torch.randn((n, 8), generator=gen, device=device, dtype=torch.float64)
    H = torch.einsum("na,aij->nij", h.to(torch.complex128), _gell_mann(device)) * 0.5
    return torch.linalg.matrix_exp(1j * eps * H).to(torch.complex64)


def gauge_field(dims, seed: int, device, field_id: int = 1, kind: str = "haar", eps: float = 0.3) -> torch.Tensor:
    """Links of ``kind`` "haar" (Haar-random SU(3)) or "near_unit"
    (exp(i eps H)), canonical shape (4, L3, L2, L1, L0, 3, 3), complex64."""
    L0, L1, L2, L3 = dims
    V = L0 * L1 * L2 * L3
    g = _gen(seed, field_id, device)
    out = torch.empty((4, V, 3, 3), dtype=torch.complex64, device=device)
    chunk = 1 << 20
    for mu in range(4):
        for s in range(0, V, chunk):
            n = min(chunk, V - s)
            out[mu, s:s + n] = haar_su3(n, g, device) if kind == "haar" else near_unit_su3(n, g, device, eps)
    return out.reshape(4, L3, L2, L1, L0, 3, 3)


def propagator(dims, seed: int, device, field_id: int = 2, x0=(0, 0, 0, 0), envelope: float = 0.5) -> torch.Tensor:
    """Synthetic propagator, canonical shape (L3, L2, L1, L0, 4, 3, 4, 3), complex64."""
    L0, L1, L2, L3 = dims
    g = _gen(seed, field_id, device)
    z = _complex_normal((L3, L2, L1, L0, 144), g, device)
    comps = []
    for L, c in zip(dims, x0):
        d = (torch.arange(L, device=device) - c).remainder(L)
        comps.append(torch.minimum(d, L - d).to(torch.float32))
    d0, d1, d2, d3 = comps
    r = torch.sqrt(d3[:, None, None, None] ** 2 + d2[None, :, None, None] ** 2
                   + d1[None, None, :, None] ** 2 + d0[None, None, None, :] ** 2)
    z *= torch.exp(-envelope * r)[..., None]
    return z.reshape(L3, L2, L1, L0, 4, 3, 4, 3)
