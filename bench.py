#!/usr/bin/env python
"""Benchmark of the smearing + meson chain on GB300 (one JSON line on stdout).

One step is one pass of the whole path on the 16^3x32 workload (the shape of
the paper's run A, Fig. 4a), single precision storage:

  1. field setup: import the synthetic propagator (stand-in for the solver
     output, which is out of scope) from its canonical layout, and create the
     point source;
  2. SRC: Gaussian smearing of the point source, kappa = 0.21, N = 25;
  3. SNK: Gaussian smearing of the propagator, kappa = 0.21, N = 25;
  4. HAD: the sixteen meson correlators at zero momentum with FP64
     timeslice sums.

``value`` is the algorithmic bytes of a step (each field read and written
once per pass, links read once per smearing iteration) divided by the
device time per step, with inputs resident in HBM.  ``e2e`` is the same
quantity through the public API with the inputs copied from pinned host
memory and the correlators read back every step.

Two further workloads are measured once each and reported under
``components`` (``--no-batch``/``--no-scale`` skip them):

  * ``batch``: 64 smearing + meson jobs of uneven lattice, N and kappa, FP32
    one job at a time against batches replayed from CUDA graphs (FP32, BF16,
    and float16 storage on the tensor-core hop), with the reduced-precision
    correlator errors;
  * ``scale_48x96``: eight 48^3x96 propagators smeared at (kappa, N) up to
    (0.30, 80), all 8 x 8 meson pairs and the nucleon at 33 momenta, with
    FP32 and with float16 storage, checked against the FP64 checker on a
    sampled timeslice.

``--impl reference`` times the FP64 checker on the host cores on a bounded
sample of the same workload (one timeslice per step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "smear GB/s (%HBM peak), contraction sites/s; BF16 vs FP32 batched at tol"
CSRC = os.path.join(ROOT, "paper_1111_5596_gb300", "csrc")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.txt")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="minimum host time of the checker baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the launch-shape autotuning (default shapes; for profiling runs)")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the 64-job batched comparison (FP32 one job at a time vs batched FP32/BF16)")
    ap.add_argument("--batch-steps", type=int, default=5)
    ap.add_argument("--no-24x48", action="store_true", help="skip the 24^3x48 smearing-hop roofline component")
    ap.add_argument("--partition", choices=["replica", "tslab"], default="replica",
                    help="replica: every rank runs its own lattice (weak scaling); tslab: the ranks split one "
                         "lattice into timeslice slabs and gather the correlators (strong scaling)")
    ap.add_argument("--no-scale", action="store_true",
                    help="skip the 48^3x96 scale run (8 propagators, 64 meson pairs + nucleon at 33 momenta)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# workload bookkeeping (shared by both arms)


def workload():
    from synth import configs

    return configs.MESONS_16x32


def step_bytes(w, n_timeslices=None) -> dict:
    """Algorithmic bytes per step (FP32 storage) for all or some timeslices."""
    V = w.V3 * (w.Nt if n_timeslices is None else n_timeslices)
    prop = V * 144 * 8
    hop = V * (144 * 8 * 2 + 3 * 9 * 8)          # read psi, write psi, 3 spatial links
    b = {
        "import": 2 * prop,                      # canonical read + device-layout write
        "point_source": prop,                    # write
        "smear_src": w.n_smear * hop,
        "smear_snk": w.n_smear * hop,
        "mesons": prop,                          # S1 = S2: one read
    }
    b["total"] = sum(b.values())
    b["hop_per_launch"] = hop
    return b


# ---------------------------------------------------------------------------
# host FP64 checker arm


def run_checker_sample(w, t: int, U64, P64):
    """The FP64 checker on one timeslice of the step: SRC, SNK, 16 mesons."""
    from oracle import hadron, smear, source

    sub = (w.dims[0], w.dims[1], w.dims[2], 1)
    Ut = U64[:, t:t + 1]
    src = smear.gauss_smear(Ut, source.point_propagator(sub), w.kappa, w.n_smear, 3)
    snk = smear.gauss_smear(Ut, P64[t:t + 1], w.kappa, w.n_smear, 3)
    C = hadron.meson_2pt(snk, snk, hadron.SIXTEEN_MESONS)
    return src, snk, C


def checker_inputs(w, t0: int, t1: int):
    from synth import fields

    U = fields.round_to_f32(fields.gauge_field(w.dims, w.seed, kind=w.links, eps=w.eps, x3_range=(t0, t1)))
    U = U.reshape((4, t1 - t0) + U.shape[2:])
    P = fields.round_to_f32(fields.propagator(w.dims, w.seed, x3_range=(t0, t1)))
    return U, P


def _checker_timeslice(args):
    """One timeslice of the step through the FP64 checker (a pool task)."""
    w, t, Ut, Pt = args
    run_checker_sample(w, 0, Ut, Pt)
    return t


def checker_pool(n: int):
    """A spawned process pool of n workers, one numpy thread each (a child
    forked from a process that has initialised CUDA can hang)."""
    import multiprocessing as mp

    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    return mp.get_context("spawn").Pool(n)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def checker_timed(w, pool, n_workers: int, n_timeslices: int):
    """Wall time of n_timeslices whole timeslices of the step through the
    checker, spread over the pool (smearing and contractions never couple
    timeslices, so each timeslice is an exact, independent share)."""
    U, P = checker_inputs(w, 0, n_timeslices)
    tasks = [(w, t, U[:, t:t + 1], P[t:t + 1]) for t in range(n_timeslices)]
    t0 = time.perf_counter()
    done = pool.map(_checker_timeslice, tasks, chunksize=1)
    dt = time.perf_counter() - t0
    assert sorted(done) == list(range(n_timeslices))
    return dt


def cpu_baseline(w, min_seconds: float) -> dict:
    """The checker on the host cores over whole timeslices of the step: one
    timeslice per worker and round, the whole lattice when it fits the time
    (min_seconds of wall time is the floor of the sample)."""
    cores = min(host_cores(), w.Nt)
    pool = checker_pool(cores)
    try:
        pool.map(_checker_timeslice, [(w, 0) + checker_inputs(w, 0, 1)] * cores, chunksize=1)  # warm the workers
        n = cores
        dt = checker_timed(w, pool, cores, n)
        if dt < min_seconds and n < w.Nt:
            n = w.Nt
            dt = checker_timed(w, pool, cores, n)
    finally:
        pool.terminate()
        pool.join()
    b = step_bytes(w, n_timeslices=n)["total"]
    return {"value": b / dt / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} of {w.Nt} timeslices of the step (SRC + SNK smearing N={w.n_smear}, 16 mesons), "
                      f"numpy FP64, one timeslice per process on {cores} host cores, {dt:.1f} s wall"}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workload()
    cores = min(host_cores(), w.Nt)
    pool = checker_pool(cores)
    try:
        for _ in range(args.warmup):
            checker_timed(w, pool, cores, cores)
        dts = [checker_timed(w, pool, cores, cores) for _ in range(args.steps)]
    finally:
        pool.terminate()
        pool.join()
    dt = sum(dts) / len(dts)
    b = step_bytes(w, n_timeslices=cores)["total"]
    value = b / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_block(w),
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": cores, "kind": "oracle",
                         "sample": f"{cores} of {w.Nt} timeslices per step (SRC + SNK smearing N={w.n_smear}, "
                                   f"16 mesons), numpy FP64, one timeslice per process on {cores} host cores"},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_block(w) -> dict:
    L0, L1, L2, L3 = w.dims
    return {"workload": w.name, "lattice": f"{L0}x{L1}x{L2}x{L3}", "kappa": w.kappa, "n_smear": w.n_smear,
            "links": f"{w.links} SU(3) eps={w.eps}", "storage": "f32 propagator, f32 links",
            "stages": "import + point source + SRC smear + SNK smear + 16 mesons p=0",
            "l2": "inputs larger than L2 (151 MB propagator per field vs 129 MB L2)",
            "parallelism": "independent replica per GPU"}


# ---------------------------------------------------------------------------
# GPU arm


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index  # nvidia-smi --id: the GPU's UUID, else its index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": d["hbm_gbs"], "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def traffic_for(kernel: str):
    """ncu DRAM bytes per launch, if captured on the current kernel sources."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    with open(TRAFFIC_FILE) as f:
        for line in f:
            parts = line.split()
            if len(parts) != 4 or parts[0] != kernel:
                continue
            h = hashlib.sha256()
            for name in parts[2].split(","):
                with open(os.path.join(CSRC, name), "rb") as src:
                    h.update(src.read())
            return int(parts[1]) if h.hexdigest() == parts[3] else None
    return None


def batch_arms(q, dev, args) -> dict:
    """The 64 uneven smearing + meson jobs four ways on the same inputs:
    FP32 one job at a time (gauss_smear + meson_2pt per job), FP32 as one
    batch replayed from a CUDA graph, BF16 storage with BF16 reconstruct-12
    links as one batch from a graph, and float16 storage (per-field
    power-of-two scale) with float16 reconstruct-12 links on the tensor-core
    hop as one batch from a graph.  Each pass re-imports every propagator,
    smears it with its own (kappa, N) and contracts the 16 zero-momentum
    mesons.  Returns times, throughput and the reduced-precision errors
    against the FP32 results (which agree with the FP64 checker to 1e-5)."""
    import torch

    from synth import configs, device as synth_dev

    w = configs.BATCH_64
    jobs = configs.batch_jobs(w)
    lats, rows = {}, []
    for j in jobs:
        dims = j["dims"]
        if dims not in lats:
            lats[dims] = q.Lattice(dims, 3)
        lat = lats[dims]
        U_can = synth_dev.gauge_field(dims, j["seed"], dev)
        P_can = synth_dev.propagator(dims, j["seed"], dev)
        r = {"job": j, "lat": lat, "P": P_can,
             "U32": q.Field(lat, q.GAUGE, q.F32, device=dev).import_(U_can),
             "Ub": q.Field(lat, q.GAUGE, q.BF16_R12, device=dev).import_(U_can),
             "Uh": q.Field(lat, q.GAUGE, q.F16_R12, device=dev).import_(U_can),
             "Uf": q.Field(lat, q.GAUGE, q.F16, device=dev).import_(U_can)}
        del U_can
        for tag, prec in (("32", q.F32), ("b", q.BF16), ("h", q.F16), ("f", q.F16)):
            r["p" + tag] = q.Field(lat, q.PROPAGATOR, prec, device=dev)
            r["s" + tag] = r["p" + tag].like()
        r["m1"] = torch.zeros((16, 1, lat.Nt), dtype=torch.complex128, device=dev)
        for tag in ("32", "b", "h", "f"):
            r["m" + tag] = torch.zeros((16, lat.Nt), dtype=torch.complex128, device=dev)
        rows.append(r)
    # launch shapes per (lattice, precision) class, by the autotuner
    if not args.no_tune:
        seen = set()
        for r in rows:
            for tag, U in (("32", r["U32"]), ("b", r["Ub"])):
                key = (r["job"]["dims"], tag)
                if key not in seen:
                    seen.add(key)
                    q.tune_smear(U, r["p" + tag].import_(r["P"]), r["s" + tag], 3, reps=2)
    b32 = q.Batch([(r["U32"], r["p32"], r["s32"], r["job"]["kappa"], r["job"]["n_iter"], r["m32"]) for r in rows])
    bb = q.Batch([(r["Ub"], r["pb"], r["sb"], r["job"]["kappa"], r["job"]["n_iter"], r["mb"]) for r in rows])
    bh = q.Batch([(r["Uh"], r["ph"], r["sh"], r["job"]["kappa"], r["job"]["n_iter"], r["mh"]) for r in rows])
    bf = q.Batch([(r["Uf"], r["pf"], r["sf"], r["job"]["kappa"], r["job"]["n_iter"], r["mf"]) for r in rows])

    def single_fp32():
        for r in rows:
            j = r["job"]
            r["p32"].import_(r["P"])
            q.gauss_smear(r["U32"], r["p32"], j["kappa"], j["n_iter"], 3, scratch=r["s32"])
            q.meson_2pt(r["p32"], r["p32"], q.SIXTEEN_MESONS, out=r["m1"])

    def batched(bt, tag):
        for r in rows:
            r["p" + tag].import_(r["P"])
        bt.run(use_graph=True)

    def timed(fn):
        for _ in range(max(args.warmup, 3)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.batch_steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        q.device_status()
        return e0.elapsed_time(e1) / args.batch_steps

    t_single = timed(single_fp32)
    t_b32 = timed(lambda: batched(b32, "32"))
    t_bb = timed(lambda: batched(bb, "b"))
    t_bh = timed(lambda: batched(bh, "h"))
    t_bf = timed(lambda: batched(bf, "f"))

    # correlator error of the BF16 batch against FP32, per job: max over
    # channels of ||C_bf16(.) - C_f32(.)|| / ||C_f32(.)|| over t
    def corr_err(a, ref):
        d = torch.linalg.vector_norm(a - ref, dim=-1)
        n = torch.linalg.vector_norm(ref, dim=-1)
        n = torch.where(n > 1e-12 * n.max(), n, n.max())
        return float((d / n).max())

    errs = [corr_err(r["mb"], r["m32"]) for r in rows]
    errs_h = [corr_err(r["mh"], r["m32"]) for r in rows]
    errs_f = [corr_err(r["mf"], r["m32"]) for r in rows]
    # FP32 one at a time and FP32 batched run the same per-site arithmetic:
    # the smeared fields agree bit for bit (the correlators only to the
    # order of their FP64 atomic timeslice sums)
    single_fields = []
    for r in rows:
        j = r["job"]
        r["p32"].import_(r["P"])
        q.gauss_smear(r["U32"], r["p32"], j["kappa"], j["n_iter"], 3, scratch=r["s32"])
        q.meson_2pt(r["p32"], r["p32"], q.SIXTEEN_MESONS, out=r["m1"])
        single_fields.append(r["p32"].storage.clone())
    batched(b32, "32")
    torch.cuda.synchronize()
    same = all(torch.equal(f, r["p32"].storage) for f, r in zip(single_fields, rows))
    del single_fields
    mes_dev = max(corr_err(r["m1"][:, 0, :], r["m32"]) for r in rows)
    by_n, by_n_h = {}, {}
    for r, e, eh in zip(rows, errs, errs_h):
        band = "N<=25" if r["job"]["n_iter"] <= 25 else "N>25"
        by_n[band] = max(by_n.get(band, 0.0), e)
        by_n_h[band] = max(by_n_h.get(band, 0.0), eh)
    hop_sites = sum(r["job"]["n_iter"] * r["lat"].V for r in rows)
    sites = sum(r["lat"].V for r in rows)
    # FP32-equivalent algorithmic bytes of a pass: import, N hops, mesons
    bytes32 = sum(r["lat"].V * (2 * 1152 + r["job"]["n_iter"] * (2 * 1152 + 216) + 1152) for r in rows)
    return {
        "workload": w.name, "jobs": len(rows),
        "lattices": {f"{d[0]}^3x{d[3]}": sum(1 for r in rows if r["job"]["dims"] == d) for d in lats},
        "hop_sites_per_pass": hop_sites, "contraction_sites_per_pass": sites,
        "ms_per_pass": {"fp32_single": t_single, "fp32_batched_graph": t_b32, "bf16_batched_graph": t_bb,
                        "f16_tc_batched_graph": t_bh},
        "fp32_equiv_gbs": {"fp32_single": bytes32 / t_single / 1e6, "fp32_batched_graph": bytes32 / t_b32 / 1e6,
                           "bf16_batched_graph": bytes32 / t_bb / 1e6, "f16_tc_batched_graph": bytes32 / t_bh / 1e6},
        "speedup_f16_tc_batched_vs_fp32_single": t_single / t_bh,
        "f16_vs_fp32_corr_rel_err_max": max(errs_h), "f16_vs_fp32_corr_rel_err_max_by_n": by_n_h,
        "f16_tol": 2e-2, "f16_within_tol": max(errs_h) <= 2e-2,
        "f16_full_links": {"ms_per_pass": t_bf, "speedup_vs_fp32_single": t_single / t_bf,
                           "corr_rel_err_max": max(errs_f), "within_tol": max(errs_f) <= 2e-2,
                           "storage": "propagators float16 x scale, links float16 (all nine entries)"},
        "f16_storage": "propagators float16 x per-field power-of-two scale, links float16 reconstruct-12, "
                       "tensor-core hop (mma.sync m16n8k16, FP32 accumulation)",
        "speedup_bf16_batched_vs_fp32_single": t_single / t_bb,
        "speedup_fp32_batched_vs_fp32_single": t_single / t_b32,
        "bf16_vs_fp32_corr_rel_err_max": max(errs), "bf16_vs_fp32_corr_rel_err_max_by_n": by_n,
        "bf16_tol": 2e-2, "bf16_within_tol": max(errs) <= 2e-2,
        "f16_jobs_err": sorted([[r["job"]["dims"][0], r["job"]["n_iter"], round(e, 5)] for r, e in zip(rows, errs_h)],
                               key=lambda x: x[1]),
        "bf16_jobs_err": sorted([[r["job"]["dims"][0], r["job"]["n_iter"], round(e, 5)] for r, e in zip(rows, errs)],
                                key=lambda x: x[1]),
        "fp32_batched_fields_equal_single_bitwise": bool(same),
        "fp32_batched_vs_single_corr_rel_diff": mes_dev,
        "inputs": "device-generated seeded Haar SU(3) links and exp(-0.5|x|) Gaussian propagators per job",
    }


def scale_run(q, dev, args) -> dict:
    """The 48^3x96 scale workload, one pass per storage: eight synthetic
    propagators (device-generated, seeded), each smeared at its own
    (kappa, N) in {(0.15,10), (0.20,20), (0.25,40), (0.30,80)} x {source,
    sink}; then the sixteen mesons of all 8 x 8 propagator pairs and the
    nucleon (u = propagator 0, d = propagator 1), each projected to the 33
    momenta with |n|^2 <= 4, FP64 sums.  Once with FP32 propagators and
    links (rescaled by exact powers of two where the growth needs it), once
    with float16 propagators and float16 reconstruct-12 links on the
    tensor-core hop.  Reports times, the float16 correlator error against
    FP32, and the FP32 correlators of propagator 0 on timeslice 0 against
    the FP64 checker (exact for a sample: the path never couples
    timeslices)."""
    import numpy as np
    import torch

    from oracle import hadron, smear
    from synth import configs, device as synth_dev

    torch.cuda.empty_cache()  # the batch comparison's fields are gone; return their memory
    w = configs.SCALE_48x96
    lat = q.Lattice(w.dims, w.j_decay)
    kn = [pair for pair in w.extra["kappa_n"] for _ in ("src", "snk")]
    moms = q.momenta_up_to(4)
    V = lat.V
    res = {"workload": w.name, "lattice": "48x48x48x96", "links": f"{w.links} SU(3) eps={w.eps}",
           "props_kappa_n": kn, "n_mom": len(moms), "meson_pairs": len(kn) ** 2, "channels_per_pair": 16}

    def ev():
        return torch.cuda.Event(enable_timing=True)

    corr, sample = {}, {}
    for arm, up, pp, bpsi, blink in (("fp32", q.F32, q.F32, 1152, 216), ("f16_tc", q.F16_R12, q.F16, 576, 72)):
        U_can = synth_dev.gauge_field(w.dims, w.seed, dev, kind=w.links, eps=w.eps)
        U = q.Field(lat, q.GAUGE, up, device=dev).import_(U_can)
        if arm == "fp32":
            sample["U"] = U_can[:, :1].cpu().numpy()
        del U_can
        scratch = q.Field(lat, q.PROPAGATOR, pp, device=dev)
        props, t_smear = [], 0.0
        for i, (kappa, n) in enumerate(kn):
            P_can = synth_dev.propagator(w.dims, w.seed + 17 * i, dev)
            f = q.Field(lat, q.PROPAGATOR, pp, device=dev).import_(P_can)
            if arm == "fp32" and i in (IA, IB):
                sample[i] = P_can[:1].cpu().numpy()
            del P_can
            torch.cuda.synchronize()
            e0, e1 = ev(), ev()
            e0.record()
            q.gauss_smear(U, f, kappa, n, w.j_decay, scratch=scratch)
            e1.record()
            torch.cuda.synchronize()
            t_smear += e0.elapsed_time(e1)
            props.append(f)
        del scratch
        C = torch.empty((len(kn), len(kn), 16, len(moms), lat.Nt), dtype=torch.complex128, device=dev)
        e0, e1 = ev(), ev()
        e0.record()
        q.meson_2pt_multi(props, q.SIXTEEN_MESONS, moms, out=C)  # all 64 pairs: every propagator read once per site
        Cn = q.baryon_2pt(props[0], props[1], q.NUCLEON, +1, moms)
        e1.record()
        torch.cuda.synchronize()
        q.device_status()
        t_con = e0.elapsed_time(e1)
        corr[arm] = (C.cpu().numpy(), Cn.cpu().numpy())
        hops = sum(n for _, n in kn)
        res[arm] = {"smear_ms": t_smear, "contract_ms": t_con, "total_ms": t_smear + t_con, "hops": hops,
                    "contraction": "qdpg_meson_2pt_multi (8 propagators, 64 pairs in one pass)",
                    "smear_gbs": hops * V * (2 * bpsi + blink) / (t_smear * 1e-3) / 1e9,
                    "smear_fp32_equiv_gbs": hops * V * 2520 / (t_smear * 1e-3) / 1e9,
                    "finite": bool(np.isfinite(corr[arm][0]).all() and np.isfinite(corr[arm][1]).all())}
        del props, U, C, Cn
        torch.cuda.empty_cache()

    def corr_err(a, ref):
        d = np.linalg.norm(a - ref, axis=-1)
        nrm = np.linalg.norm(ref, axis=-1)
        nrm = np.where(nrm > 1e-12 * nrm.max(), nrm, nrm.max())
        return float((d / nrm).max())

    (C32, N32), (C16, N16) = corr["fp32"], corr["f16_tc"]
    res["speedup_f16_tc_vs_fp32"] = res["fp32"]["total_ms"] / res["f16_tc"]["total_ms"]
    res["f16_vs_fp32_meson_corr_rel_err_max"] = max(corr_err(C16[a, b], C32[a, b])
                                                    for a in range(len(kn)) for b in range(len(kn)))
    res["f16_vs_fp32_nucleon_corr_rel_err"] = corr_err(N16, N32)
    res["f16_tol"] = 2e-2
    # FP32 against the checker: the cross pair of the (0.30, 80) propagator
    # (rescaled by the scale records) and a (0.15, 10) one on timeslice 0, all
    # 16 mesons at 33 momenta; the checker's 24 source columns (each smears
    # alone: the operator acts on colour) are spread over the host cores
    t0 = time.perf_counter()
    (ka, na), (kb, nb) = kn[IA], kn[IB]
    U0 = sample["U"].astype(np.complex128)
    cores = host_cores()
    pool = checker_pool(min(cores, 24))
    try:
        cols = [pool.apply_async(_smear_column, (U0, np.ascontiguousarray(sample[i][..., sp, cp]).astype(np.complex128),
                                                 kk, nn))
                for i, kk, nn in ((IA, ka, na), (IB, kb, nb)) for sp in range(4) for cp in range(3)]
        got_cols = [c.get() for c in cols]
    finally:
        pool.terminate()
        pool.join()
    Sa = np.stack(got_cols[:12], axis=-1).reshape(got_cols[0].shape + (4, 3))
    Sb = np.stack(got_cols[12:], axis=-1).reshape(got_cols[0].shape + (4, 3))
    ref = hadron.meson_2pt(Sa, Sb, hadron.SIXTEEN_MESONS, moms, j_decay=w.j_decay)
    # scale of each momentum sum: A(t) = sum_x |c(x)| (a smooth field's p != 0
    # correlators cancel strongly; FP32 site values bound the error relative to A)
    A = np.stack([np.abs(hadron.meson_site(Sa, Sb, a, b)).sum(axis=(1, 2, 3)) for a, b in hadron.SIXTEEN_MESONS])
    got = C32[IA, IB][:, :, :1]
    k0 = moms.index((0, 0, 0))
    res["fp32_vs_checker"] = {
        "sample": f"cross pair S_a S_b, a = propagator {IA} (kappa {ka}, N {na}, rescaled by the scale record), "
                  f"b = propagator {IB} (kappa {kb}, N {nb}), timeslice 0, 16 mesons x 33 momenta",
        "p0_corr_rel_err": corr_err(got[:, k0:k0 + 1], ref[:, k0:k0 + 1]),
        "err_rel_to_abs_site_sum": float((np.abs(got - ref)[..., 0] / A).max()),
        "plain_corr_rel_err_all_p": corr_err(got, ref), "tol": 1e-5,
        "largest_smeared_value_log2": float(np.log2(np.abs(Sa).max())),
        "checker_s": time.perf_counter() - t0, "checker_cores": min(cores, 24)}
    return res


def _smear_column(U, col, kappa, n_iter):
    """One source column of a propagator timeslice through the FP64 checker (a pool task)."""
    from oracle import smear

    return smear.gauss_smear(U, col, kappa, n_iter, 3)


IA, IB = 6, 1   # the scale workload's propagators at (0.30, 80) and (0.15, 10)


def hop_24x48(q, dev, args) -> dict:
    """The smearing hop on the 24^3x48 lattice (the shape of the paper's run B,
    Fig. 4b), FP32 propagator and links, kappa = 0.21, in the tuned launch
    shape: mean per-launch time from CUDA events around each launch, and back
    to back (events around whole smearing calls), as a roofline block."""
    import torch

    from synth import configs, device as synth_dev

    w = configs.BF16_24x48
    lat = q.Lattice(w.dims, w.j_decay)
    U = q.Field(lat, q.GAUGE, q.F32, device=dev).import_(
        synth_dev.gauge_field(w.dims, w.seed, dev, kind=w.links, eps=w.eps))
    S = q.Field(lat, q.PROPAGATOR, q.F32, device=dev).import_(synth_dev.propagator(w.dims, w.seed, dev))
    scratch = S.like()
    tuned = (None, None, None) if args.no_tune else q.tune_smear(U, S, scratch, w.j_decay, reps=3)
    n_b2b = 26          # below the rescaling threshold at kappa = 0.21 (40 bits): hops only
    for _ in range(2):
        q.gauss_smear(U, S, w.kappa, n_b2b, w.j_decay, scratch=scratch)
    torch.cuda.synchronize()
    q.profile_reset()
    q.profile_enable(True)
    for _ in range(2):
        q.gauss_smear(U, S, w.kappa, n_b2b, w.j_decay, scratch=scratch)
    torch.cuda.synchronize()
    q.profile_enable(False)
    hop_ms, hop_n = q.profile_query("smear_hop")
    stream = torch.cuda.current_stream()
    ev = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        q.gauss_smear(U, S, w.kappa, n_b2b, w.j_decay, scratch=scratch)
        e1.record(stream)
        ev.append((e0, e1))
    torch.cuda.synchronize()
    q.device_status()
    b2b_s = min(a.elapsed_time(z) for a, z in ev) * 1e-3 / n_b2b
    avg_s = hop_ms * 1e-3 / hop_n
    per_launch = lat.V * (2 * 1152 + 216)
    peak = measured_peaks()
    return {"kernel": "smear_hop (FP32 propagator, 12 columns)", "lattice": "24x24x24x48", "bound": "hbm",
            "achieved": per_launch / avg_s / 1e9, "peak": peak["hbm_gbs"], "unit": "GB/s",
            "frac": per_launch / avg_s / 1e9 / peak["hbm_gbs"], "peak_source": peak["source"],
            "traffic": traffic_for("smear_hop_24x48"), "algorithmic_bytes_per_launch": per_launch,
            "avg_launch_us": avg_s * 1e6, "back_to_back_us": b2b_s * 1e6,
            "frac_back_to_back": per_launch / b2b_s / 1e9 / peak["hbm_gbs"], "launches": hop_n,
            "tuned_tile_sites": tuned[0], "tuned_grid_mode": tuned[1]}


def max_over_ranks(x: float, world: int, device) -> float:
    """Largest per-rank value (the slowest rank's time) on every rank."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank: float, seconds: float) -> float:
    """Units all ranks processed (each rank its own problem of the same size)
    divided by the slowest rank's time."""
    return world * units_per_rank / seconds


def gpu_arm(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1111_5596_gb300 as q
    from synth import configs, fields

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    q.load()

    base = workload()
    tslab_mode = args.partition == "tslab" and world > 1
    if tslab_mode:
        # one lattice split by timeslices: this rank's slab [t0, t0 + nt), same seeds on every rank
        from paper_1111_5596_gb300 import tslab

        w = base
        t0, nt = tslab.slab(w.Nt, world, rank)
        lat = q.Lattice(tslab.slab_dims(w.dims, w.j_decay, nt), w.j_decay)
        sub = lat.dims
        U_h = torch.from_numpy(fields.gauge_field(w.dims, w.seed, kind=w.links, eps=w.eps, x3_range=(t0, t0 + nt))
                               .reshape((4,) + tuple(reversed(sub)) + (3, 3)).astype(np.complex64))
        P_h = torch.from_numpy(fields.propagator(w.dims, w.seed, x3_range=(t0, t0 + nt)).astype(np.complex64))
    else:
        t0, nt = 0, base.Nt
        w = configs.Workload(base.name, base.dims, base.links, base.kappa, base.n_smear, base.prop, eps=base.eps,
                             seed=base.seed + 1000 * rank)          # independent problem per rank
        lat = q.Lattice(w.dims, w.j_decay)
        U_h = torch.from_numpy(fields.gauge_field(w.dims, w.seed, kind=w.links, eps=w.eps).astype(np.complex64))
        P_h = torch.from_numpy(fields.propagator(w.dims, w.seed).astype(np.complex64))
    U_h, P_h = U_h.pin_memory(), P_h.pin_memory()
    U_dev, P_dev = U_h.to(dev), P_h.to(dev)

    U = q.Field(lat, q.GAUGE, q.F32, device=dev).import_(U_dev)
    src = q.Field(lat, q.PROPAGATOR, q.F32, device=dev)
    snk = q.Field(lat, q.PROPAGATOR, q.F32, device=dev)
    scratch = q.Field(lat, q.PROPAGATOR, q.F32, device=dev)
    C = torch.empty((16, 1, lat.Nt), dtype=torch.complex128, device=dev)
    C_h = torch.empty((16, 1, w.Nt), dtype=torch.complex128).pin_memory()
    if tslab_mode and t0 != 0:
        src.storage.zero_()   # the point source (origin) lies on rank 0's slab; this slab's source is zero

    # launch shapes of the smearing kernel, picked by measurement before timing
    tuned = (None, None) if args.no_tune else q.tune_smear(U, snk.import_(P_dev), scratch, w.j_decay, reps=3)

    def source():
        if t0 == 0:
            q.point_source(src)

    def correlators():
        # the slabs' correlators gathered over the ranks (tslab); the whole lattice's otherwise
        return tslab.gather_timeslices(C, w.Nt, world, rank) if tslab_mode else C

    def step_device():
        snk.import_(P_dev)
        source()
        q.gauss_smear(U, src, w.kappa, w.n_smear, w.j_decay, scratch=scratch)
        q.gauss_smear(U, snk, w.kappa, w.n_smear, w.j_decay, scratch=scratch)
        q.meson_2pt(snk, snk, q.SIXTEEN_MESONS, out=C)
        return correlators()

    def barrier():
        if world > 1:
            dist.barrier()

    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        step_device()
    torch.cuda.synchronize()

    # ---- timed region: device-resident inputs ----
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except AttributeError:
        gpu_id = str(local)
    clocks = ClockSampler(gpu_id)
    clocks.start()
    launches0 = q.launch_count()
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step_device()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = q.launch_count() - launches0
    clk = clocks.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, world, dev)

    # Per-kernel durations from CUDA events around every launch, in a
    # separate pass of the same steps: the events between launches keep
    # consecutive hops from overlapping their set-up, so the step time above
    # is taken without them.
    q.profile_reset()
    q.profile_enable(True)
    for _ in range(args.steps):
        step_device()
    torch.cuda.synchronize()
    q.profile_enable(False)
    kern = {name: q.profile_query(name) for name in ("smear_hop", "meson_2pt", "field_import", "point_source")}

    # The same hops back to back (events around whole smearing calls only):
    # consecutive launches then overlap one hop's set-up with the previous
    # hop's tail (programmatic dependent launch), which the per-launch events
    # above prevent.
    # an even count of hops: an odd one ends with a copy of the ping-pong
    # buffer back into psi, which is not a hop
    n_even = w.n_smear - (w.n_smear & 1)
    b2b = []
    for _ in range(args.steps):
        snk.import_(P_dev)
        e_b0, e_b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e_b0.record(stream)
        q.gauss_smear(U, snk, w.kappa, n_even, w.j_decay, scratch=scratch)
        e_b1.record(stream)
        b2b.append((e_b0, e_b1))
    torch.cuda.synchronize()
    hop_b2b_s = sum(a.elapsed_time(z) for a, z in b2b) * 1e-3 / (args.steps * n_even)

    b = step_bytes(w)
    peaks = measured_peaks()
    # tslab: the ranks share one lattice (its bytes once); replicas: each rank's lattice counts
    value = (b["total"] / (ms * 1e-3) if tslab_mode else whole_job_rate(world, b["total"], ms * 1e-3)) / 1e9

    hop_ms, hop_n = kern["smear_hop"]
    hop_avg_s = hop_ms / hop_n * 1e-3
    b["hop_per_launch"] = lat.V * (144 * 8 * 2 + 3 * 9 * 8)   # this rank's lattice (a slab under tslab)
    achieved = b["hop_per_launch"] / hop_avg_s / 1e9
    mes_ms, mes_n = kern["meson_2pt"]
    smear_s = hop_ms * 1e-3 / args.steps
    roofline = {"kernel": "smear_hop (FP32 propagator, 12 columns)", "bound": "hbm", "achieved": achieved,
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                "peak_source": peaks["source"], "traffic": traffic_for("smear_hop"),
                "algorithmic_bytes_per_launch": b["hop_per_launch"], "avg_launch_us": hop_avg_s * 1e6,
                "back_to_back_us": hop_b2b_s * 1e6,
                "frac_back_to_back": b["hop_per_launch"] / hop_b2b_s / 1e9 / peaks["hbm_gbs"],
                "launches": hop_n, "tuned_tile_sites": tuned[0], "tuned_grid_mode": tuned[1]}
    b_rank = step_bytes(w, n_timeslices=lat.Nt)   # this rank's share (its slab under tslab)
    components = {
        "smear_gbs_kernel": (b_rank["smear_src"] + b_rank["smear_snk"]) / smear_s / 1e9,
        "smear_hbm_frac": achieved / peaks["hbm_gbs"],
        "contraction_sites_per_s": lat.V / (mes_ms / mes_n * 1e-3),
        "contraction_gbs": b_rank["mesons"] / (mes_ms / mes_n * 1e-3) / 1e9,
        "kernel_ms_per_step": {k: v[0] / args.steps for k, v in kern.items()},
    }

    # ---- end to end through the public API, host buffers ----
    e2e = None
    if not args.no_e2e:
        copy_stream = torch.cuda.Stream(dev)
        P_done = torch.cuda.Event()

        def step_e2e():
            # host buffers through the library's own staging: the links first;
            # the propagator's import runs on a second stream while the
            # source, which does not need it, is smeared
            U.import_host(U_h)
            copy_stream.wait_stream(stream)
            snk.import_host(P_h, stream=copy_stream)
            P_done.record(copy_stream)
            source()
            q.gauss_smear(U, src, w.kappa, w.n_smear, w.j_decay, scratch=scratch)
            stream.wait_event(P_done)
            q.gauss_smear(U, snk, w.kappa, w.n_smear, w.j_decay, scratch=scratch)
            q.meson_2pt(snk, snk, q.SIXTEEN_MESONS, out=C)
            C_h.copy_(correlators(), non_blocking=True)
            stream.synchronize()
            return C_h

        for _ in range(args.warmup):
            step_e2e()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step_e2e()
        barrier()
        e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, world, dev)
        h2d = U_h.numel() * U_h.element_size() + P_h.numel() * P_h.element_size()
        e2e_rate = b["total"] / e2e_s if tslab_mode else whole_job_rate(world, b["total"], e2e_s)
        e2e = {"value": e2e_rate / 1e9, "unit": "GB/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": C_h.numel() * C_h.element_size(), "ms_per_step": e2e_s * 1e3,
               "path": "qdpg_field_import_host (page-locked canonical complex64) for links and propagator, "
                       "correlators read back every step"}

    if not args.no_24x48:
        components["hop_24x48"] = hop_24x48(q, dev, args)
        torch.cuda.empty_cache()

    batch = None
    if not args.no_batch:
        batch = batch_arms(q, dev, args)
        components["batch"] = batch

    if not args.no_scale and rank == 0:
        components["scale_48x96"] = scale_run(q, dev, args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, args.cpu_seconds)

    if rank == 0:
        highlights = {"hop_16x32_us_per_launch": roofline["avg_launch_us"], "hop_16x32_hbm_frac": roofline["frac"],
                      "hop_16x32_hbm_frac_back_to_back": roofline["frac_back_to_back"],
                      "meson_2pt_16x32_p0_us": mes_ms / mes_n * 1e3, "meson_2pt_gbs": components["contraction_gbs"]}
        if "hop_24x48" in components:
            highlights["hop_24x48_us_per_launch"] = components["hop_24x48"]["avg_launch_us"]
            highlights["hop_24x48_hbm_frac"] = components["hop_24x48"]["frac"]
        if batch:
            fl = batch.get("f16_full_links", {})
            highlights.update({
                "batch64_f16_vs_fp32_one_job": fl.get("speedup_vs_fp32_single"),
                "batch64_f16_r12_vs_fp32_one_job": batch.get("speedup_f16_tc_batched_vs_fp32_single"),
                "batch64_f16_corr_rel_err_max": fl.get("corr_rel_err_max"),
                "batch64_f16_within_2e-2": fl.get("within_tol")})
        sc48 = components.get("scale_48x96")
        if sc48:
            highlights.update({
                "scale48_f16_vs_fp32_end_to_end": sc48.get("speedup_f16_tc_vs_fp32"),
                "scale48_fp32_contract_ms": sc48.get("fp32", {}).get("contract_ms"),
                "scale48_f16_contract_ms": sc48.get("f16_tc", {}).get("contract_ms"),
                "scale48_fp32_vs_checker_p0_rel_err": sc48.get("fp32_vs_checker", {}).get("p0_corr_rel_err")})
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong" if tslab_mode else "weak",
            "vs_baseline": None, "dtype": "f32",
            "data": "synthetic: seeded near-unit SU(3) links (eps=0.3) and Gaussian propagator with "
                    "exp(-0.5|x|) envelope, complex64",
            "config": dict(config_block(w), **({"parallelism": f"tslab{world}: one lattice in timeslice slabs, "
                                                                  "correlators gathered (NCCL all_gather) every step"}
                                                 if tslab_mode else {})), "highlights": highlights, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clk, "components": components,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse_args()
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
