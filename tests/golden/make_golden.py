"""Write the stored expected values under tests/golden/ from the FP64 checker only.

Run from the repository root:  python tests/golden/make_golden.py
Each file states the workload it was computed on; the inputs are the seeded
synthetic fields of ``synth`` rounded to complex64, as the GPU path sees them.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import hadron, smear, source  # noqa: E402
from synth import configs, fields  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def chain_4x8():
    w = configs.CHAIN_4x8
    U = fields.round_to_f32(fields.gauge_field(w.dims, w.seed, kind=w.links))
    S = smear.gauss_smear(U, source.point_propagator(w.dims), w.kappa, w.n_smear, w.j_decay)
    C = hadron.meson_2pt(S, S, hadron.SIXTEEN_MESONS)[:, 0, :]
    path = os.path.join(HERE, "chain_4x8_mesons.txt")
    with open(path, "w") as f:
        f.write(f"# workload {w.name}: Haar links (seed {w.seed}, field 1) rounded to complex64,\n")
        f.write("# point source at the origin, Gaussian smearing kappa=0.25 N=5 over x,y,z,\n")
        f.write("# 16 meson channels (Gamma_snk = Gamma_src = Gamma(n)) at p = 0.\n")
        f.write("# columns: n t Re(C) Im(C)   (computed by the FP64 checker, oracle/)\n")
        for n in range(16):
            for t in range(C.shape[1]):
                f.write(f"{n} {t} {C[n, t].real:.17e} {C[n, t].imag:.17e}\n")
    print("wrote", path)


if __name__ == "__main__":
    chain_4x8()
