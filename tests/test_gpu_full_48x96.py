"""The 48^3x96 scale workload at full size, in the library's default launch
shapes: its strongest propagator, (kappa, N) = (0.30, 80), whose growth
(about 2^112) only the power-of-two scale records keep inside the FP32 and
float16 ranges, and its mildest, (0.15, 10); then the cross pair S_a S_b --
the sixteen mesons at the 33 momenta with |n|^2 <= 4 -- and the nucleon with
u = S_a, d = S_b at the same momenta.  FP32 storage (FP32 links) and
float16 storage (float16 reconstruct-12 links, tensor-core hop).

The inputs are the scale workload's own (near-unit links, synthetic
propagators 6 and 1 of its eight), drawn on the device by the seeded
generator; the FP64 checker recomputes two sampled timeslices exactly from
the same values (smearing and contractions never couple timeslices), spread
over the host cores.  Errors: smeared fields ||a - r|| / ||r|| per sampled
timeslice (export applies the scale record, so this compares the unscaled
values); correlators per (channel, momentum), plain over the sampled t at
p = 0 and relative to A(t) = sum_x |c(x)| over all momenta.
"""
import os
import tempfile

import numpy as np
import pytest
import torch

from synth import configs
from synth import device as synth_dev
from tests import oracle_pool
from tests.parity_util import TOL_BF16, TOL_F32, corr_err, field_err, field_err_t, proj_err

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

SAMPLED_T = (0, 61)
IA, IB = 6, 1          # the workload's propagators at (0.30, 80) and (0.15, 10)


def _gpu_arm(q, lat, w, U_can, Pa_can, Pb_can, link_prec, psi_prec, ka, kb, moms):
    dev = U_can.device
    U = q.Field(lat, q.GAUGE, link_prec, device=dev).import_(U_can)
    Sa = q.Field(lat, q.PROPAGATOR, psi_prec, device=dev).import_(Pa_can)
    Sb = q.Field(lat, q.PROPAGATOR, psi_prec, device=dev).import_(Pb_can)
    scratch = Sa.like()
    q.gauss_smear(U, Sa, ka[0], ka[1], w.j_decay, scratch=scratch)
    q.gauss_smear(U, Sb, kb[0], kb[1], w.j_decay, scratch=scratch)
    del scratch, U
    C = q.meson_2pt(Sa, Sb, q.SIXTEEN_MESONS, moms).cpu().numpy()
    N = q.baryon_2pt(Sa, Sb, q.NUCLEON, +1, moms).cpu().numpy()
    q.device_status()
    fields_t = []
    for S in (Sa, Sb):
        f = S.export()
        fields_t.append(np.concatenate([f[t:t + 1].cpu().numpy() for t in SAMPLED_T]))
        del f
        torch.cuda.empty_cache()
    del Sa, Sb
    torch.cuda.empty_cache()
    return fields_t, C, N


def test_48x96_rescaled_propagator_cross_pair_and_nucleon(qdpg_gpu):
    q = qdpg_gpu
    w = configs.SCALE_48x96
    kn = [pair for pair in w.extra["kappa_n"] for _ in ("src", "snk")]
    ka, kb = kn[IA], kn[IB]
    assert ka == (0.30, 80) and kb == (0.15, 10)
    moms = q.momenta_up_to(4)
    k0 = moms.index((0, 0, 0))
    pool = oracle_pool.pool()            # spawned: no CUDA state in the workers
    tmp = tempfile.mkdtemp(prefix="qdpg48_")
    try:
        dev = torch.device("cuda:0")
        lat = q.Lattice(w.dims, w.j_decay)
        U_can = synth_dev.gauge_field(w.dims, w.seed, dev, kind=w.links, eps=w.eps)
        Pa_can = synth_dev.propagator(w.dims, w.seed + 17 * IA, dev)
        Pb_can = synth_dev.propagator(w.dims, w.seed + 17 * IB, dev)
        # the checker's inputs: the same complex64 values on the sampled timeslices
        jobs = {}
        for t in SAMPLED_T:
            Up = os.path.join(tmp, f"U{t}.npy")
            np.save(Up, U_can[:, t:t + 1].cpu().numpy().astype(np.complex128))
            jobs[t] = (oracle_pool.smear_propagator(pool, Up, Pa_can[t:t + 1].cpu().numpy().astype(np.complex128),
                                                    *ka),
                       oracle_pool.smear_propagator(pool, Up, Pb_can[t:t + 1].cpu().numpy().astype(np.complex128),
                                                    *kb))
        arms = {
            "f32": _gpu_arm(q, lat, w, U_can, Pa_can, Pb_can, q.F32, q.F32, ka, kb, moms),
            "f16_r12": _gpu_arm(q, lat, w, U_can, Pa_can, Pb_can, q.F16_R12, q.F16, ka, kb, moms),
        }
        del U_can, Pa_can, Pb_can
        torch.cuda.empty_cache()
        # checker: smeared fields, then the contractions of the cross pair
        ref_a, ref_b, contr = [], [], {}
        for t in SAMPLED_T:
            Sa = oracle_pool.gather_propagator(jobs[t][0])
            Sb = oracle_pool.gather_propagator(jobs[t][1])
            ref_a.append(Sa)
            ref_b.append(Sb)
            pa, pb = os.path.join(tmp, f"Sa{t}.npy"), os.path.join(tmp, f"Sb{t}.npy")
            np.save(pa, Sa)
            np.save(pb, Sb)
            chans = list(q.SIXTEEN_MESONS)
            mes = [pool.apply_async(oracle_pool.meson_channels, (pa, pb, chans[i:i + 4], moms))
                   for i in range(0, 16, 4)]
            nuc = [pool.apply_async(oracle_pool.nucleon_slab, (pa, pb, z, z + 6)) for z in range(0, 48, 6)]
            contr[t] = (mes, nuc)
        ph = None
        rC, aC, rN, aN = [], [], [], []
        for t in SAMPLED_T:
            mes, nuc = contr[t]
            parts = [m.get() for m in mes]
            rC.append(np.concatenate([c for c, _ in parts])[..., 0])
            aC.append(np.concatenate([a for _, a in parts])[..., 0])
            cN = np.concatenate([n.get() for n in nuc], axis=1)          # (1, 48, 48, 48)
            if ph is None:
                from oracle import hadron
                ph = hadron.momentum_phases(w.dims[:3] + (1,), moms, 3)
            rN.append(np.array([(cN * ph[k]).sum() for k in range(len(moms))]))
            aN.append(np.abs(cN).sum())
    finally:
        pool.terminate()
        pool.join()
        for f in os.listdir(tmp):
            os.remove(os.path.join(tmp, f))
        os.rmdir(tmp)
    ref_fa, ref_fb = np.concatenate(ref_a), np.concatenate(ref_b)
    rC, aC = np.stack(rC, -1), np.stack(aC, -1)                        # (16, 33, 2), (16, 2)
    rN, aN = np.stack(rN, -1), np.array(aN)[None, None]                # (33, 2)
    ts = list(SAMPLED_T)
    err = {}
    for arm, (fl, C, N) in arms.items():
        C, N = C[..., ts], N[..., ts]
        e = {
            "field_a": field_err(fl[0], ref_fa), "field_a_per_t": field_err_t(fl[0], ref_fa),
            "field_b": field_err(fl[1], ref_fb), "field_b_per_t": field_err_t(fl[1], ref_fb),
            "meson_p0": corr_err(C[:, k0:k0 + 1], rC[:, k0:k0 + 1]),
            "meson_all_p": proj_err(C, rC, aC),
            "nucleon_p0": corr_err(N[None, k0:k0 + 1], rN[None, k0:k0 + 1]),
            "nucleon_all_p": proj_err(N[None], rN[None], aN[0]),
        }
        err[arm] = e
    print({a: {k: f"{v:.2e}" for k, v in e.items()} for a, e in err.items()})
    scale = np.abs(ref_fa).max()
    assert scale > 2.0 ** 100, scale          # the rescaled propagator really left the FP32 range of its square
    for k, v in err["f32"].items():
        assert v <= TOL_F32, (k, v)
    for k, v in err["f16_r12"].items():
        assert v <= TOL_BF16, (k, v)
