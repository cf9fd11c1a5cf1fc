"""CPU FP64/int64 oracle for XPCS two-time correlation on raw and compressed frames.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.
The CUDA library never calls it, links it or falls back to it; it shares no code,
constant or helper with the CUDA path.

Every function restates one definition of arXiv 2407.20356 ("Homomorphic data
compression for real time photon correlation analysis") in plain numpy: integer
sums and Grams in int64, everything else in float64.  Library primitives used as
steps: numpy matmul and ``numpy.linalg.eigh`` (LAPACK).
"""
from .xpcs_oracle import *  # noqa: F401,F403
