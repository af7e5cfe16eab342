"""Seeded synthetic input generators shared by the oracle and the GPU path.

This package holds no HiCR arithmetic: only SplitMix64 streams, slot fill
bytes, channel payload words and operation-table / trace builders.
"""
from . import splitmix, configs  # noqa: F401
