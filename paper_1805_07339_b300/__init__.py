"""B300-native sampled-frame video analysis (Scanner's hist / shot / resize hot path).

``scn`` is the ctypes binding of ``libscn.so`` (C ABI in ``include/scn.h``).  It
is imported on first use of a library name (``paper_1805_07339_b300.scn_hist``,
``from paper_1805_07339_b300 import scn``), so that the seeds-and-sizes module
``workloads`` can be imported without building or loading the CUDA library.
Importing ``scn`` raises if ``libscn.so`` cannot be built or loaded: there is no
CPU path.
"""
import importlib


def __getattr__(name):
    if name.startswith("__"):
        raise AttributeError(name)
    scn = importlib.import_module(__name__ + ".scn")
    try:
        return getattr(scn, name)
    except AttributeError:
        raise AttributeError(f"module {__name__!r} has no attribute {name!r}") from None
