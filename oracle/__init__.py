"""FP64 CPU oracle for the inverse-free SVGP step (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The CUDA library neither imports nor links it,
and the two share no code.
"""
from . import dgp, rsvgp  # noqa: F401
