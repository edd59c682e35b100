"""Batched smearing + mesons (many sources at once, Sec. 5) against the FP64
checker and against the one-job entry points, through the C ABI.

The batch mixes three lattices, FP32, BF16 and float16 storage,
propagators and a fermion, and iteration counts 0..9 (even and odd), so
that jobs leave the multi-job launches at different steps and the
multi-job pipelined kernel, the multi-job tensor-core kernel and the
per-job fallback all run.
"""
import numpy as np
import pytest
import torch

from oracle import hadron, smear
from synth import fields
from tests.parity_util import TOL_BF16, TOL_F32, corr_err, field_err, field_err_t, to_bf16_complex

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")

# (dims, kind, psi precision, link precision, kappa, n_iter, mesons)
JOBS = [
    ((8, 8, 8, 4), "prop", "f32", "f32", 0.21, 5, True),
    ((8, 8, 8, 4), "prop", "f32", "f32", 0.18, 8, True),
    ((8, 8, 8, 4), "prop", "f32", "f32", 0.25, 0, True),
    ((8, 8, 8, 4), "prop", "f32", "f32", 0.15, 3, False),
    ((6, 4, 8, 3), "prop", "f32", "f32", 0.20, 4, True),    # lattice of its own class
    ((8, 8, 8, 4), "prop", "bf16", "bf16_r12", 0.21, 7, True),
    ((8, 8, 8, 4), "ferm", "f32", "f32", 0.22, 6, False),   # one vector: per-job kernel
    ((8, 8, 8, 4), "prop", "f32", "f32", 0.30, 45, True),   # growth 2^67: rescaled by 2^-31 twice
    ((8, 8, 8, 4), "prop", "f16", "f16_r12", 0.27, 9, True),  # float16: tensor-core multi-job hop
    ((8, 8, 8, 4), "prop", "f16", "f16_r12", 0.19, 4, True),
    ((12, 12, 4, 2), "prop", "f16", "f16", 0.22, 6, True),
]


def _canon(dims, kind, seed, prec):
    a = (fields.propagator(dims, seed, envelope=0.4) if kind == "prop" else fields.fermion(dims, seed))
    a = fields.round_to_f32(a)
    return to_bf16_complex(a) if prec == "bf16" else a


def _setup(q):
    lats, gauges, rows = {}, {}, []
    for k, (dims, kind, prec, lprec, kappa, n, mes) in enumerate(JOBS):
        if dims not in lats:
            lats[dims] = q.Lattice(dims, 3)
            gauges[dims] = fields.round_to_f32(fields.gauge_field(dims, 40, kind="near_unit"))
        lat = lats[dims]
        U = gauges[dims]
        Uf = q.Field(lat, q.GAUGE, q.PREC_NAMES[lprec], device=DEV).import_(
            torch.from_numpy(U.astype(np.complex64)).to(DEV))
        K = q.PROPAGATOR if kind == "prop" else q.FERMION
        psi = _canon(dims, kind, 100 + k, prec)
        f = q.Field(lat, K, q.PREC_NAMES[prec], device=DEV)
        m = torch.zeros((16, lat.Nt), dtype=torch.complex128, device=DEV) if mes else None
        rows.append(dict(U=U, Uf=Uf, psi=psi, f=f, scratch=f.like(), mesons=m, kappa=kappa, n=n,
                         prec=prec, lprec=lprec, lat=lat))
    return rows


def _load(rows):
    for r in rows:
        r["f"].import_(torch.from_numpy(r["psi"].astype(np.complex64)).to(DEV))


def _batch(q, rows):
    return q.Batch([(r["Uf"], r["f"], r["scratch"], r["kappa"], r["n"], r["mesons"]) for r in rows], j_decay=3)


def test_batch_matches_oracle_and_single_job_path(qdpg_gpu):
    q = qdpg_gpu
    rows = _setup(q)
    _load(rows)
    b = _batch(q, rows)
    b.run()
    torch.cuda.synchronize()
    q.device_status()
    for r in rows:
        out = r["f"].export().cpu().numpy()
        ref = smear.gauss_smear(r["U"], r["psi"], r["kappa"], r["n"], 3)
        exact_links = r["lprec"] == "f32" and r["prec"] == "f32"
        tol = TOL_F32 if exact_links else TOL_BF16
        if r["n"] == 0:
            assert np.array_equal(out, r["psi"])
        else:
            assert field_err(out, ref) <= tol and field_err_t(out, ref) <= tol
        # the one-job entry point gives the same bits
        g = r["f"].like().import_(torch.from_numpy(r["psi"].astype(np.complex64)).to(DEV))
        q.gauss_smear(r["Uf"], g, r["kappa"], r["n"], 3, scratch=g.like())
        assert np.array_equal(g.export().cpu().numpy(), out)
        if r["mesons"] is not None:
            C = r["mesons"].cpu().numpy()[:, None, :]
            # the contraction of the smeared field as stored
            assert corr_err(C, hadron.meson_2pt(out, out, hadron.SIXTEEN_MESONS)) <= TOL_F32
            # and of the FP64 smeared field
            assert corr_err(C, hadron.meson_2pt(ref, ref, hadron.SIXTEEN_MESONS)) <= tol


def test_batch_graph_replays_the_same_work(qdpg_gpu):
    q = qdpg_gpu
    rows = _setup(q)
    b = _batch(q, rows)
    _load(rows)
    b.run()
    torch.cuda.synchronize()
    direct = [(r["f"].export().cpu().numpy(), None if r["mesons"] is None else r["mesons"].cpu().numpy())
              for r in rows]
    _load(rows)
    n0 = q.launch_count()
    b.run()
    torch.cuda.synchronize()
    per_run = q.launch_count() - n0
    assert per_run > 0
    for capture_call in (True, False):      # the first graph call runs directly, then captures
        _load(rows)
        for r in rows:
            if r["mesons"] is not None:
                r["mesons"].zero_()
        n1 = q.launch_count()
        b.run(use_graph=True)
        torch.cuda.synchronize()
        q.device_status()
        assert q.launch_count() - n1 == per_run
        for r, (f_ref, m_ref) in zip(rows, direct):
            assert np.array_equal(r["f"].export().cpu().numpy(), f_ref)
            if m_ref is not None:
                assert np.array_equal(r["mesons"].cpu().numpy(), m_ref)
