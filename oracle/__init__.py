"""CPU oracle for the sampled-frame convert / histogram / shot-score / resize path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code with
the CUDA library in ``paper_1805_07339_b300``: the pixel arithmetic lives in the
plain C file ``orc.c`` (loaded here through ctypes), the sampling operator and the
proposal network's fp64 reference are written below and in ``cnn.py``.

Paper anchors (Scanner, Poms et al., ACM TOG 37(4) 2018):
  * videos are tables with one row per frame (Sec. 3, "Videos as logical tables");
  * sampling selects rows by stride, range or index list (Sec. 3.2,
    "Sampling/spacing operations"; the access patterns of Sec. 5.1.1);
  * a stencil op sees a constant-offset window of consecutive elements
    (Sec. 3.2, "Stencil operations") - the shot score is the two-element case;
  * HIST computes a per-frame colour histogram (Sec. 5.1.2); shot boundaries are
    found from histogram differences (Sec. 5.2, data mining).
The numeric readings (bins, BT.601 constants, threshold, resize convention,
generator) are listed in the design notes; each C routine states its definition.

Parity pins live in tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "orc.c")
_LIB = os.path.join(_HERE, "liborc.so")

SAMPLE_STRIDE, SAMPLE_RANGE, SAMPLE_GATHER, SAMPLE_KEYFRAME = 0, 1, 2, 3
KEYFRAME_INTERVAL = 104  # the paper's average keyframe distance (Sec. 5.1.1)


def build(force: bool = False) -> str:
    """Compile orc.c into liborc.so with gcc (no optimisation beyond -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", _LIB, _SRC,
                               "-lm", "-lpthread"])
    return _LIB


class GenParams(ctypes.Structure):
    _fields_ = [("master_seed", ctypes.c_uint64), ("video_id", ctypes.c_uint64),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("num_frames", ctypes.c_int64), ("num_shots", ctypes.c_int32),
                ("shot_mode", ctypes.c_int32)]


class Shot(ctypes.Structure):
    _fields_ = [("start", ctypes.c_int64), ("base", ctypes.c_int32 * 3),
                ("gx", ctypes.c_int32 * 3), ("gy", ctypes.c_int32 * 3)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        u64, i64, i32, p = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
        _lib.orc_sm.argtypes = [u64, u64]
        _lib.orc_sm.restype = u64
        _lib.orc_noise.argtypes = [u64, u64]
        _lib.orc_noise.restype = i32
        _lib.orc_gen_shots.argtypes = [ctypes.POINTER(GenParams), ctypes.POINTER(Shot), i64]
        _lib.orc_gen_shots.restype = i64
        _lib.orc_gen_frame.argtypes = [ctypes.POINTER(GenParams), ctypes.POINTER(Shot), i64, i64, p]
        _lib.orc_gen_frame.restype = None
        _lib.orc_yuv_to_rgb.argtypes = [i32, i32, i32, ctypes.POINTER(ctypes.c_int32)]
        _lib.orc_yuv_to_rgb.restype = None
        _lib.orc_yuv_to_rgb_array.argtypes = [p, i64, p]
        _lib.orc_yuv_to_rgb_array.restype = None
        _lib.orc_hist_frame.argtypes = [p, i32, i32, p]
        _lib.orc_hist_frame.restype = None
        _lib.orc_scores.argtypes = [p, i64, i64, p, p]
        _lib.orc_scores.restype = None
        _lib.orc_resize_norm_frame.argtypes = [p, i32, i32, i32, i32, p, p, p]
        _lib.orc_resize_norm_frame.restype = None
        _lib.orc_thumb_frame.argtypes = [p, i32, i32, p]
        _lib.orc_thumb_frame.restype = None
        _lib.orc_thumb_yuv_frame.argtypes = [p, i32, i32, p]
        _lib.orc_thumb_yuv_frame.restype = None
        _lib.orc_thumb_diff.argtypes = [p, p]
        _lib.orc_thumb_diff.restype = ctypes.c_double
        _lib.orc_thumb_diff_yuv.argtypes = [p, p]
        _lib.orc_thumb_diff_yuv.restype = ctypes.c_double
        _lib.orc_hist_batch.argtypes = [p, i64, i32, i32, p, i64, i32, p]
        _lib.orc_hist_batch.restype = None
        _lib.orc_gen_batch.argtypes = [ctypes.POINTER(GenParams), ctypes.POINTER(Shot), i64, p, i64,
                                       i64, i32, p]
        _lib.orc_gen_batch.restype = None
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


# --------------------------------------------------------------------------- generator
class Video:
    """Generator description of one synthetic video (shot table computed by the oracle)."""

    def __init__(self, master_seed: int, video_id: int, width: int, height: int,
                 num_frames: int, num_shots: int = 1, shot_mode: int = 0):
        self.params = GenParams(master_seed, video_id, width, height, num_frames, num_shots, shot_mode)
        self.width, self.height, self.num_frames = width, height, num_frames
        cap = num_frames if shot_mode == 1 else num_shots
        arr = (Shot * max(cap, 1))()
        n = lib().orc_gen_shots(ctypes.byref(self.params), arr, cap)
        if n < 0:
            raise ValueError("impossible shot table request")
        self._shots = arr
        self.num_shots_made = int(n)

    @property
    def frame_bytes(self) -> int:
        return self.width * self.height * 3 // 2

    def shots(self) -> list[dict]:
        return [dict(start=s.start, base=list(s.base), gx=list(s.gx), gy=list(s.gy))
                for s in self._shots[: self.num_shots_made]]

    def shot_starts(self) -> np.ndarray:
        return np.array([s.start for s in self._shots[: self.num_shots_made]], dtype=np.int64)

    def keyframes(self) -> np.ndarray:
        """Every KEYFRAME_INTERVAL-th frame plus every shot start, sorted, unique."""
        k = set(range(0, self.num_frames, KEYFRAME_INTERVAL)) | set(int(s) for s in self.shot_starts())
        return np.array(sorted(k), dtype=np.int64)

    def frame(self, f: int) -> np.ndarray:
        out = np.empty(self.frame_bytes, dtype=np.uint8)
        lib().orc_gen_frame(ctypes.byref(self.params), self._shots, self.num_shots_made, f, _ptr(out))
        return out

    def frames(self, idx, nthreads: int = 1) -> np.ndarray:
        idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
        out = np.empty((len(idx), self.frame_bytes), dtype=np.uint8)
        if len(idx):
            lib().orc_gen_batch(ctypes.byref(self.params), self._shots, self.num_shots_made,
                                _ptr(idx), len(idx), self.frame_bytes, nthreads, _ptr(out))
        return out


def sm(seed: int, i: int) -> int:
    return int(lib().orc_sm(seed & (2**64 - 1), i & (2**64 - 1)))


def noise(s_pix: int, q: int) -> int:
    return int(lib().orc_noise(s_pix, q))


# --------------------------------------------------------------------------- sampling
def sample(kind: int, num_frames: int, start: int = 0, stop: int = 0, step: int = 1,
           indices=None, keyframes=None) -> np.ndarray:
    """Sampling operator (Sec. 3.2): the sequence of table rows selected.

    STRIDE: start, start+step, ... < stop.  RANGE: [start, stop).  GATHER: the
    given list, in the given order (duplicates kept).  KEYFRAME: the table's
    keyframe list.  Every selected row must lie in [0, num_frames).
    """
    if kind == SAMPLE_STRIDE or kind == SAMPLE_RANGE:
        if kind == SAMPLE_RANGE:
            step = 1
        if step < 1 or start < 0 or stop > num_frames:
            raise ValueError("bad stride/range")
        return np.array(list(range(start, stop, step)), dtype=np.int64)
    if kind == SAMPLE_GATHER:
        out = np.array(list(indices), dtype=np.int64)
        if len(out) and (out.min() < 0 or out.max() >= num_frames):
            raise ValueError("gather index out of range")
        return out
    if kind == SAMPLE_KEYFRAME:
        return np.array(sorted(set(int(k) for k in keyframes)), dtype=np.int64)
    raise ValueError("unknown sampling kind")


# --------------------------------------------------------------------------- pixel math
def yuv_to_rgb(Y: int, U: int, V: int) -> tuple[int, int, int]:
    out = (ctypes.c_int32 * 3)()
    lib().orc_yuv_to_rgb(Y, U, V, out)
    return int(out[0]), int(out[1]), int(out[2])


def yuv_to_rgb_array(yuv: np.ndarray) -> np.ndarray:
    """[n][3] uint8 (Y, U, V) -> [n][3] uint8 (R, G, B)."""
    yuv = np.ascontiguousarray(yuv, dtype=np.uint8).reshape(-1, 3)
    out = np.empty_like(yuv)
    lib().orc_yuv_to_rgb_array(_ptr(yuv), len(yuv), _ptr(out))
    return out


def hist_frame(frame: np.ndarray, W: int, H: int) -> np.ndarray:
    frame = np.ascontiguousarray(frame, dtype=np.uint8)
    assert frame.size >= W * H * 3 // 2
    h = np.zeros(48, dtype=np.uint32)
    lib().orc_hist_frame(_ptr(frame), W, H, _ptr(h))
    return h.reshape(3, 16)


def hist_batch(frames: np.ndarray, W: int, H: int, idx=None, nthreads: int = 1) -> np.ndarray:
    """hist of frames[idx[k]] (or frames[k]) for a [T][frame_bytes] uint8 array."""
    frames = np.ascontiguousarray(frames, dtype=np.uint8)
    fb = frames.shape[1]
    if idx is None:
        n, ip = frames.shape[0], None
    else:
        idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
        n, ip = len(idx), _ptr(idx)
    h = np.zeros((n, 48), dtype=np.uint32)
    if n:
        lib().orc_hist_batch(_ptr(frames), fb, W, H, ip, n, nthreads, _ptr(h))
    return h.reshape(n, 3, 16)


def scores(hist: np.ndarray, pixel_count: int) -> tuple[np.ndarray, np.ndarray]:
    hist = np.ascontiguousarray(hist, dtype=np.uint32).reshape(-1, 48)
    n = hist.shape[0]
    s = np.zeros(n, dtype=np.uint32)
    f = np.zeros(n, dtype=np.uint8)
    if n:
        lib().orc_scores(_ptr(hist), n, pixel_count, _ptr(s), _ptr(f))
    return s, f


DEFAULT_MEAN = (0.485, 0.456, 0.406)
DEFAULT_STD = (0.229, 0.224, 0.225)


def resize_norm_frame(frame: np.ndarray, W: int, H: int, oh: int = 224, ow: int = 224,
                      mean=DEFAULT_MEAN, std=DEFAULT_STD) -> np.ndarray:
    frame = np.ascontiguousarray(frame, dtype=np.uint8)
    m = np.ascontiguousarray(np.asarray(mean, dtype=np.float64))
    s = np.ascontiguousarray(np.asarray(std, dtype=np.float64))
    out = np.empty((3, oh, ow), dtype=np.float64)
    lib().orc_resize_norm_frame(_ptr(frame), W, H, oh, ow, _ptr(m), _ptr(s), _ptr(out))
    return out


def thumb_frame(frame: np.ndarray, W: int, H: int) -> np.ndarray:
    frame = np.ascontiguousarray(frame, dtype=np.uint8)
    out = np.empty((36, 64), dtype=np.uint8)
    lib().orc_thumb_frame(_ptr(frame), W, H, _ptr(out))
    return out


def thumb_yuv_frame(frame: np.ndarray, W: int, H: int) -> np.ndarray:
    """[3][6][32]: Y at luma pixel (2 s c, 6 s r), and U, V of the chroma sample it uses."""
    frame = np.ascontiguousarray(frame, dtype=np.uint8)
    out = np.empty((3, 6, 32), dtype=np.uint8)
    lib().orc_thumb_yuv_frame(_ptr(frame), W, H, _ptr(out))
    return out


def thumb_diff(ta: np.ndarray, tb: np.ndarray) -> float:
    """Mean |luma thumbnail difference| (the luma gate between two frames)."""
    ta = np.ascontiguousarray(ta, dtype=np.uint8)
    tb = np.ascontiguousarray(tb, dtype=np.uint8)
    return float(lib().orc_thumb_diff(_ptr(ta), _ptr(tb)))


def thumb_diff_yuv(ya: np.ndarray, yb: np.ndarray) -> float:
    """Mean |dY| + mean |dU| + mean |dV| of two coarse YUV thumbnails (the luma + chroma gate)."""
    ya = np.ascontiguousarray(ya, dtype=np.uint8)
    yb = np.ascontiguousarray(yb, dtype=np.uint8)
    return float(lib().orc_thumb_diff_yuv(_ptr(ya), _ptr(yb)))
