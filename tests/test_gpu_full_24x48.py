"""The 24^3x48 workload at full size, in the launch configuration the
library picks for it: near-unit links, a synthetic propagator smeared with
kappa = 0.21, N = 40, then the sixteen mesons, the nucleon and the Delta++
projected onto the 33 momenta with |n|^2 <= 4 (tensor-core projection).
Three storages on the same seeded inputs: FP32, BF16 propagator with BF16
reconstruct-12 links, and float16 propagator (with its power-of-two scale)
with float16 reconstruct-12 links on the tensor-core hop.

Smearing and contractions never couple timeslices, so the FP64 checker
recomputes sampled timeslices exactly from the same inputs (drawn on the
device by the seeded generator, copied back for the checker).  Errors:
fields ||a - r|| / ||r|| on the sampled timeslices; correlators per
(channel, momentum) over the sampled t, plain at p = 0 and relative to
A(t) = sum_x |c(x)| over all momenta (the projected sums of a smooth field
cancel strongly).  The Delta's checker (the slowest) runs on the first
sampled timeslice only.
"""
import numpy as np
import pytest
import torch

from oracle import baryon, hadron, smear
from synth import configs
from synth import device as synth_dev
from tests.parity_util import TOL_BF16, TOL_F32, corr_err, field_err, proj_err

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

SAMPLED_T = (0, 29)


def _gpu_arm(q, lat, w, U_can, P_can, link_prec, psi_prec, moms):
    dev = U_can.device
    U = q.Field(lat, q.GAUGE, link_prec, device=dev).import_(U_can)
    S = q.Field(lat, q.PROPAGATOR, psi_prec, device=dev).import_(P_can)
    q.gauss_smear(U, S, w.kappa, w.n_smear, w.j_decay, scratch=S.like())
    C = q.meson_2pt(S, S, q.SIXTEEN_MESONS, moms).cpu().numpy()
    N = q.baryon_2pt(S, S, q.NUCLEON, +1, moms).cpu().numpy()
    D = q.baryon_2pt(S, None, q.DELTA, +1, moms).cpu().numpy()
    q.device_status()
    fld = S.export()
    sampled = np.concatenate([fld[t:t + 1].cpu().numpy() for t in SAMPLED_T])
    del U, S, fld
    torch.cuda.empty_cache()
    return sampled, C, N, D


def _project(c, dims, moms):
    """The checker's momentum projection of site values c on one timeslice."""
    ph = hadron.momentum_phases(dims, moms, 3)
    return np.array([hadron.timeslice_sum(c * ph[k], 3) for k in range(len(moms))])[:, 0]


def _errors(got, ref, moms):
    """got/ref: (field on sampled t, mesons, nucleon, delta, scales)."""
    f, C, N, D = got
    rf, rC, rN, rD, aC, aN, aD = ref
    k0 = moms.index((0, 0, 0))
    ts = list(SAMPLED_T)
    C, N, D = C[..., ts], N[..., ts], D[..., ts[:1]]
    return {
        "field": field_err(f, rf),
        "meson_p0": corr_err(C[:, k0:k0 + 1], rC[:, k0:k0 + 1]),
        "meson_all_p": proj_err(C, rC, aC),
        "nucleon_p0": corr_err(N[k0:k0 + 1], rN[k0:k0 + 1]),
        "nucleon_all_p": proj_err(N, rN, aN),
        "delta_p0": corr_err(D[k0:k0 + 1], rD[k0:k0 + 1]),
        "delta_all_p": proj_err(D, rD, aD),
    }


def test_24x48_full_size_three_storages_sampled_timeslices(qdpg_gpu):
    q = qdpg_gpu
    w = configs.BF16_24x48
    dev = torch.device("cuda:0")
    lat = q.Lattice(w.dims, w.j_decay)
    moms = q.momenta_up_to(4)
    assert len(moms) == 33
    U_can = synth_dev.gauge_field(w.dims, w.seed, dev, kind=w.links, eps=w.eps)
    P_can = synth_dev.propagator(w.dims, w.seed, dev)
    arms = {
        "f32": _gpu_arm(q, lat, w, U_can, P_can, q.F32, q.F32, moms),
        "bf16_r12": _gpu_arm(q, lat, w, U_can, P_can, q.BF16_R12, q.BF16, moms),
        "f16_r12": _gpu_arm(q, lat, w, U_can, P_can, q.F16_R12, q.F16, moms),
    }
    # the checker on the sampled timeslices, from the same complex64 inputs
    rf, rC, rN, rD, aC, aN, aD = [], [], [], [], [], [], []
    dims_t = w.dims[:3] + (1,)
    for t in SAMPLED_T:
        Ut = U_can[:, t:t + 1].cpu().numpy().astype(np.complex128)
        Pt = P_can[t:t + 1].cpu().numpy().astype(np.complex128)
        S = smear.gauss_smear(Ut, Pt, w.kappa, w.n_smear, w.j_decay)
        rf.append(S)
        rC.append(hadron.meson_2pt(S, S, hadron.SIXTEEN_MESONS, moms, j_decay=w.j_decay)[..., 0])
        aC.append(np.stack([np.abs(hadron.meson_site(S, S, a, b)).sum() for a, b in hadron.SIXTEEN_MESONS]))
        cN = baryon.baryon_site(S, S, kind="nucleon", parity=+1)
        rN.append(_project(cN, dims_t, moms))
        aN.append(np.abs(cN).sum())
        if t == SAMPLED_T[0]:
            cD = baryon.baryon_site(S, S, kind="delta", parity=+1)
            rD.append(_project(cD, dims_t, moms))
            aD.append(np.abs(cD).sum())
    ref = (np.concatenate(rf), np.stack(rC, -1), np.stack(rN, -1), np.stack(rD, -1),
           np.stack(aC, -1), np.stack(aN, -1)[None], np.stack(aD, -1)[None])
    err = {arm: _errors(got, ref, moms) for arm, got in arms.items()}
    # reduced precision against FP32 on every timeslice (no checker needed)
    f32 = arms["f32"]
    k0 = moms.index((0, 0, 0))
    for arm in ("bf16_r12", "f16_r12"):
        err[arm]["meson_p0_vs_f32_all_t"] = corr_err(arms[arm][1][:, k0:k0 + 1], f32[1][:, k0:k0 + 1])
    print({a: {k: f"{v:.2e}" for k, v in e.items()} for a, e in err.items()})
    for k, v in err["f32"].items():
        assert v <= TOL_F32, (k, v)
    for arm in ("bf16_r12", "f16_r12"):
        for k, v in err[arm].items():
            assert v <= TOL_BF16, (arm, k, v)
    # float16 (11 significant bits) sits well inside the bound; BF16 (8 bits)
    # comes closest on the cancelling p = 0 meson channels (1.8e-2 measured)
    assert max(err["f16_r12"].values()) <= 5e-3
