"""Compile libscn.so in-tree for sm_103a with nvcc (no JIT, no torch extension)."""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libscn.so")
# measurement-only library (the shared-memory reduction probe), outside libscn.so's C ABI
PROBE_SRC = os.path.join(CSRC, "measure", "scn_probe.cu")
PROBE_LIB = os.path.join(HERE, "libscn_probe.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr"]


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def deps() -> list[str]:
    return sources() + sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))) + \
        [os.path.join(ROOT, "include", "scn.h"), __file__]


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in deps())


def _compile(src: str, obj: str, extra: list[str], verbose: bool) -> None:
    cmd = [NVCC, *ARCH, *FLAGS, *extra, "-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    """Each source is compiled to its own object (in parallel; the sources are
    separate translation units either way), then one link makes libscn.so."""
    if not (force or stale()):
        return LIB
    from concurrent.futures import ThreadPoolExecutor
    extra = extra or []
    objdir = os.path.join(ROOT, "_build")
    os.makedirs(objdir, exist_ok=True)
    objs = [os.path.join(objdir, os.path.basename(src)[:-3] + ".o") for src in sources()]
    # an object is rebuilt when forced, or when its source, a header or this script is newer
    shared = [p for p in deps() if not p.endswith(".cu")]
    todo = [(src, obj) for src, obj in zip(sources(), objs)
            if force or extra or not os.path.exists(obj)
            or any(os.path.getmtime(p) > os.path.getmtime(obj) for p in [src, *shared])]
    with ThreadPoolExecutor(max_workers=max(1, min(len(objs), os.cpu_count() or 1))) as pool:
        for f in [pool.submit(_compile, src, obj, extra, verbose) for src, obj in todo]:
            f.result()
    cmd = [NVCC, *ARCH, "-shared", "-cudart", "shared", "-o", LIB + ".tmp", *objs]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


def build_probe(force: bool = False) -> str:
    """Compile the measurement probe into its own library (libscn_probe.so)."""
    hdrs = sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")))
    if not force and os.path.exists(PROBE_LIB) and all(
            os.path.getmtime(p) <= os.path.getmtime(PROBE_LIB) for p in [PROBE_SRC, __file__, *hdrs]):
        return PROBE_LIB
    cmd = [NVCC, *ARCH, *FLAGS, "-I", os.path.join(ROOT, "include"), "-shared", "-cudart", "shared",
           "-o", PROBE_LIB + ".tmp", PROBE_SRC]
    subprocess.check_call(cmd)
    os.replace(PROBE_LIB + ".tmp", PROBE_LIB)
    return PROBE_LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else None))
