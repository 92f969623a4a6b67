"""FP64 CPU oracle for the matched-filter hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
library never calls it and shares no code with it.
"""
from .bege_oracle import *  # noqa: F401,F403
