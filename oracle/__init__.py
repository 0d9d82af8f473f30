"""Oracle for the M-IHS hot path: plain, slow, obviously correct fp64 CPU code.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference legs of ``bench.py`` may import anything from here.  The
CUDA library never calls into this package and this package never calls into
the CUDA library; they share no code.
"""
from .mihs_oracle import *  # noqa: F401,F403
