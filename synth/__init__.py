"""Seeded synthetic inputs shared by the CUDA path and the FP64 checker.

This package holds random-number generation and input recipes only; it does
no smearing, shifting or contraction.
"""
from . import configs, fields, rng  # noqa: F401
