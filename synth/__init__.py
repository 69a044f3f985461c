"""Seeded synthetic inputs (knowledge bases, examples, hypothesis programs).

Shared by the oracle's tests and by the GPU path's tests and benchmark.  It
holds none of the evaluation method's arithmetic: it only draws and formats
inputs.
"""
from . import rng, programs, kb, hyps  # noqa: F401
