"""The seeded synthetic workloads, named by what they are.

Each one is shaped like a run of the paper (16^3x32 and 24^3x48 single
precision, Fig. 4) or a small/large variant of it.  Seeds are
``11115596 + index`` so every workload has its own streams.
"""
from __future__ import annotations

from dataclasses import dataclass, field

BASE_SEED = 11115596


@dataclass(frozen=True)
class Workload:
    name: str
    dims: tuple[int, int, int, int]
    links: str              # "haar" | "near_unit" | "unit"
    kappa: float
    n_smear: int
    prop: str               # "point" (point source only) | "synthetic"
    eps: float = 0.3
    seed: int = BASE_SEED
    j_decay: int = 3
    storage: tuple[str, ...] = ("f32",)
    extra: dict = field(default_factory=dict)

    @property
    def V(self) -> int:
        L0, L1, L2, L3 = self.dims
        return L0 * L1 * L2 * L3

    @property
    def V3(self) -> int:
        return self.V // self.dims[self.j_decay]

    @property
    def Nt(self) -> int:
        return self.dims[self.j_decay]


# Plain chain: point source, Haar links, pion at zero momentum.
CHAIN_4x8 = Workload("chain_4^3x8_haar_k0.25_n5", (4, 4, 4, 8), "haar", 0.25, 5, "point",
                     seed=BASE_SEED + 0)

# Run-A shape: near-unit links, SRC smear of a point source and SNK smear of a
# synthetic propagator, 16 mesons at zero momentum.
MESONS_16x32 = Workload("mesons_16^3x32_nearunit_k0.21_n25", (16, 16, 16, 32), "near_unit", 0.21, 25,
                        "synthetic", eps=0.3, seed=BASE_SEED + 1)

# Run-B shape: BF16 storage with reconstruct-12 links against FP32 storage.
BF16_24x48 = Workload("bf16r12_24^3x48_nearunit_k0.21_n40", (24, 24, 24, 48), "near_unit", 0.21, 40,
                      "synthetic", eps=0.3, seed=BASE_SEED + 2, storage=("f32", "bf16"))

# Batched uneven jobs.
BATCH_SIZES = ((8, 8, 8, 16), (12, 12, 12, 24), (16, 16, 16, 32), (24, 24, 24, 48))
BATCH_64 = Workload("batched_64jobs", (16, 16, 16, 32), "haar", 0.2, 25, "synthetic",
                    seed=BASE_SEED + 3, extra={"n_jobs": 64, "sizes": BATCH_SIZES,
                                               "n_range": (5, 50), "kappa_range": (0.15, 0.30)})

# Scale run: 48^3x96 with eight propagators at different (kappa, N).
SCALE_48x96 = Workload("scale_48^3x96_8props", (48, 48, 48, 96), "near_unit", 0.2, 20, "synthetic",
                       seed=BASE_SEED + 4, storage=("f32", "bf16"),
                       extra={"kappa_n": ((0.15, 10), (0.20, 20), (0.25, 40), (0.30, 80))})

ALL = (CHAIN_4x8, MESONS_16x32, BF16_24x48, BATCH_64, SCALE_48x96)


def batch_jobs(w: Workload = BATCH_64) -> list[dict]:
    """The jobs of a batched workload: lattice drawn uniformly from
    ``extra['sizes']``, N uniform in ``extra['n_range']`` (inclusive) and kappa
    uniform in ``extra['kappa_range']``, from the workload's seeded stream;
    each job gets its own seed for its fields."""
    import numpy as np

    from synth import rng

    n = w.extra["n_jobs"]
    sizes = w.extra["sizes"]
    n_lo, n_hi = w.extra["n_range"]
    k_lo, k_hi = w.extra["kappa_range"]
    key = rng.stream_key(w.seed, 90)
    u = rng.uniform(key, np.arange(3 * n, dtype=np.uint64)).reshape(n, 3)
    jobs = []
    for j in range(n):
        jobs.append({"dims": tuple(sizes[min(int(u[j, 0] * len(sizes)), len(sizes) - 1)]),
                     "n_iter": n_lo + min(int(u[j, 1] * (n_hi - n_lo + 1)), n_hi - n_lo),
                     "kappa": k_lo + (k_hi - k_lo) * float(u[j, 2]),
                     "seed": w.seed * 100 + j})
    return jobs
