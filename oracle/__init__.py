"""Plain FP64 CPU oracle of the MonoGS++ mapping step (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The CUDA library never calls it and
shares no code with it.
"""
from .gs_oracle import *  # noqa: F401,F403
