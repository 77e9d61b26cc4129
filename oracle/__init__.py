"""Plain FP64 CPU oracle of the mixTS-PIMD hot path (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package. The CUDA
library never calls it. The C source is compiled with ``-ffp-contract=off``.
"""
from .oracle import *  # noqa: F401,F403
from .oracle import build  # noqa: F401
