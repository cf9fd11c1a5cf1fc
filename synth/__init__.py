"""Seeded synthetic inputs for XPCS correlation: speckle counts and q-masks.

This package is shared by the CPU oracle's tests and by the CUDA path's tests and
benchmark. It produces inputs only (photon-count frames, pixel-to-ring labels); it
holds none of the correlation arithmetic of the method itself.
"""
from .speckle import (  # noqa: F401
    pixel_radius,
    ring_qmap,
    sector_qmap,
    speckle_counts,
    speckle_counts_torch,
    rate_of_pixels,
)
