"""FP64 CPU checker for the smearing and hadron-contraction path.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously
correct statement of what the CUDA library computes, written in numpy
complex128 from the definitions.  Only the test suite, the package smoke test
and the benchmark's CPU-baseline leg may import it; the library itself never
does, and it shares no code, table or helper with the CUDA path.

The paper (Winter, "Accelerating QDP++/Chroma on GPUs", Lattice 2011) names
the stages it moves off the host -- source creation, source smearing, sink
smearing and the hadron spectrum, mesonic and baryonic (Sec. 5, Fig. 4) --
but prints none of their formulas.  The definitions used here are the
standard lattice-QCD ones; every choice the paper leaves open is a stated
reading in the module that makes it.

Array layouts are the canonical host layouts of :mod:`synth.fields`
(sites on axes ``(L3, L2, L1, L0)``, x0 fastest).

Parity status: every function here is pinned by tests that do not re-use its
own formula (closed forms, invariants, brute force on tiny lattices, library
special cases); none is "parity unpinned".
"""
from . import gamma, geometry, hadron, smear, source  # noqa: F401
