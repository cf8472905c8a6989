"""B300-native sampled-frame video analysis (Scanner's hist / shot / resize hot path).

``scn`` is the ctypes binding of ``libscn.so`` (C ABI in ``include/scn.h``);
``api`` adds small owning wrappers for tables, sequences and generated videos.
"""
from . import scn  # noqa: F401  (builds / loads libscn.so; raises if it cannot)
from .scn import *  # noqa: F401,F403
