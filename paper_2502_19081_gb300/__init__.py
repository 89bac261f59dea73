"""Spatially mixed MD (force mixing of two local potentials) on one GB300.

The compute path lives in the CUDA library built from ``csrc/`` and is reached
through :mod:`paper_2502_19081_gb300.mix`; :mod:`paper_2502_19081_gb300.inputs`
builds seeded synthetic workloads.  Importing the package loads neither.
"""
__all__ = ["inputs", "mix"]
