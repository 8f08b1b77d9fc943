"""FP64 CPU oracle for generalized canonical purification.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference legs may import it.  The product
path (``paper_1512_07236_gb300``) never imports this package.
"""
from .gcp_oracle import *  # noqa: F401,F403
from . import gcp_oracle  # noqa: F401
