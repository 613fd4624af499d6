"""Plain FP64 CPU reference ("oracle") of the Super Smoother periodogram.

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it; the library never does.
"""
from .oracle import *  # noqa: F401,F403
