"""The timeslice-slab partition of one lattice on two and three CPU ranks
(gloo): each rank smears and contracts only its own timeslices (the FP64
checker stands in for the per-slab computation here), the correlators are
gathered over the process group, and the gathered result equals the
one-rank computation on the whole lattice exactly and the checker's
values; slab boundaries are balanced and cover every timeslice once."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1111_5596_gb300 import tslab

DIMS, JD, KAPPA, N = (4, 4, 4, 6), 3, 0.2, 3


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _slab_correlators(t0, nt):
    """The path on the slab's timeslices [t0, t0 + nt): synthetic propagator
    and links of those timeslices, smeared, 16 mesons at two momenta."""
    import torch

    from oracle import hadron, smear
    from synth import fields

    sub = tslab.slab_dims(DIMS, JD, nt)
    U = fields.gauge_field(DIMS, 5, kind="haar", x3_range=(t0, t0 + nt)).reshape((4,) + tuple(reversed(sub)) + (3, 3))
    P = fields.propagator(DIMS, 5, x3_range=(t0, t0 + nt))
    S = smear.gauss_smear(U, P, KAPPA, N, JD)
    C = hadron.meson_2pt(S, S, hadron.SIXTEEN_MESONS, ((0, 0, 0), (1, 0, 0)), j_decay=JD)
    return torch.from_numpy(C)


def _rank(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    C = tslab.run_partitioned(DIMS, JD, world, rank, _slab_correlators)
    out.put((rank, C.numpy()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_partitioned_correlators_equal_whole_lattice(world):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((out.get(timeout=180) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    whole = _slab_correlators(0, DIMS[JD]).numpy()
    for rank, C in res:
        assert C.shape == whole.shape
        assert np.array_equal(C, whole), rank          # the same timeslice sums, gathered in order
    # and the checker on the whole lattice in one call agrees (it is the same arithmetic)
    from oracle import hadron, smear
    from synth import fields

    S = smear.gauss_smear(fields.gauge_field(DIMS, 5, kind="haar"), fields.propagator(DIMS, 5), KAPPA, N, JD)
    ref = hadron.meson_2pt(S, S, hadron.SIXTEEN_MESONS, ((0, 0, 0), (1, 0, 0)), j_decay=JD)
    assert np.abs(whole - ref).max() <= 1e-12 * np.abs(ref).max()


def test_slabs_cover_every_timeslice_once():
    for Nt in (1, 5, 6, 32, 96):
        for world in (1, 2, 3, 4, 8):
            if world > Nt:
                with pytest.raises(ValueError):
                    tslab.slab(Nt, world, 0)
                continue
            seen = []
            for r in range(world):
                t0, nt = tslab.slab(Nt, world, r)
                assert nt >= Nt // world and nt <= Nt // world + 1
                seen.extend(range(t0, t0 + nt))
            assert seen == list(range(Nt))
    assert tslab.slab_dims((4, 5, 6, 8), 3, 2) == (4, 5, 6, 2)
    assert tslab.slab_dims((4, 5, 6, 8), 1, 3) == (4, 3, 6, 8)


def test_single_rank_gather_is_identity():
    import torch

    x = torch.arange(12.0).reshape(2, 6)
    assert tslab.gather_timeslices(x, 6, 1, 0) is x
