"""FP64 CPU oracle for the block epsilon-circulant all-at-once preconditioner.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import or run anything in this package.  The
GPU library never calls it, and it never calls the GPU library.
"""
from .bec_oracle import *  # noqa: F401,F403
