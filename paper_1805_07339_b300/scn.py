"""ctypes binding of libscn.so (include/scn.h).  Argument marshalling only.

The functions keep the C names.  Device buffers are torch CUDA tensors passed
by pointer; streams default to torch's current stream.  Every compute step runs
in libscn's CUDA kernels; there is no CPU path here: if the library cannot be
built or loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

c_i32, c_i64, c_u64, c_vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p

SCN_OK, SCN_EINVAL, SCN_ERANGE, SCN_ENOMEM, SCN_ECUDA, SCN_ETIMEOUT, SCN_EUNSUPPORTED = range(7)
SCN_STRIDE, SCN_RANGE, SCN_GATHER, SCN_KEYFRAME = range(4)
SCN_F32, SCN_BF16 = 0, 1
SCN_FILL_VALUE, SCN_FILL_REPEAT = 0, 1


class ScnError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.scn_status_str(status).decode()
        if status == SCN_ECUDA:
            msg += f" (cudaError {_lib.scn_last_cuda_error()})"
        super().__init__(f"{where}: {msg} [{status}]")


class scn_gen_params(ctypes.Structure):
    _fields_ = [("master_seed", c_u64), ("video_id", c_u64), ("width", c_i32), ("height", c_i32),
                ("num_frames", c_i64), ("num_shots", c_i32), ("shot_mode", c_i32)]


class scn_shot(ctypes.Structure):
    _fields_ = [("start", c_i64), ("base", c_i32 * 3), ("gx", c_i32 * 3), ("gy", c_i32 * 3)]


class scn_table_desc(ctypes.Structure):
    _fields_ = [("width", c_i32), ("height", c_i32), ("num_frames", c_i64), ("frame_stride", c_i64),
                ("d_nv12", c_vp), ("h_rows", ctypes.POINTER(c_i64)), ("num_rows", c_i64),
                ("h_keyframes", ctypes.POINTER(c_i64)), ("num_keyframes", c_i64)]


class scn_sample_spec(ctypes.Structure):
    _fields_ = [("kind", c_i32), ("start", c_i64), ("stop", c_i64), ("step", c_i64),
                ("h_indices", ctypes.POINTER(c_i64)), ("n", c_i64)]


class scn_tune(ctypes.Structure):
    _fields_ = [("chunk_rows", c_i32), ("grid", c_i32), ("item_kpx", c_i32)]


# (name, restype, argtypes) of every exported symbol declared in include/scn.h
_P = ctypes.POINTER
SIGNATURES = [
    ("scn_status_str", ctypes.c_char_p, [c_i32]),
    ("scn_last_cuda_error", c_i32, []),
    ("scn_version", ctypes.c_char_p, []),
    ("scn_device_sm_count", c_i32, []),
    ("scn_gen_shots", c_i32, [_P(scn_gen_params), _P(scn_shot), c_i64, _P(c_i64)]),
    ("scn_video_create", c_i32, [_P(scn_gen_params), _P(c_vp)]),
    ("scn_video_destroy", c_i32, [c_vp]),
    ("scn_video_shots", c_i32, [c_vp, _P(scn_shot), c_i64, _P(c_i64)]),
    ("scn_video_keyframes", c_i32, [c_vp, _P(c_i64), c_i64, _P(c_i64)]),
    ("scn_generate", c_i32, [c_vp, c_vp, c_i64, c_i64, c_i64, c_vp]),
    ("scn_generate_frames", c_i32, [c_vp, c_vp, c_i64, c_vp, c_i64, c_vp]),
    ("scn_table_create", c_i32, [_P(scn_table_desc), _P(c_vp)]),
    ("scn_table_destroy", c_i32, [c_vp]),
    ("scn_sample_indices", c_i32, [c_vp, _P(scn_sample_spec), _P(c_i64), c_i64, _P(c_i64)]),
    ("scn_sample", c_i32, [c_vp, _P(scn_sample_spec), _P(c_vp)]),
    ("scn_seq_length", c_i32, [c_vp, _P(c_i64)]),
    ("scn_seq_destroy", c_i32, [c_vp]),
    ("scn_seq_sync_status", c_i32, [c_vp, c_vp]),
    ("scn_seq_set_wait_test", c_i32, [c_vp, c_u64, c_i32]),
    ("scn_cnn_set_wait_test", c_i32, [c_vp, c_u64, c_i32]),
    ("scn_seq_set_tune", c_i32, [c_vp, _P(scn_tune)]),
    ("scn_seq_get_tune", c_i32, [c_vp, _P(scn_tune)]),
    ("scn_hist", c_i32, [c_vp, c_vp, c_vp]),
    ("scn_shot_scores", c_i32, [c_vp, c_i64, c_i64, c_vp, c_vp, c_vp]),
    ("scn_hist_scores", c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp]),
    ("scn_hist_scores_noalloc", c_i32, [c_vp, c_i32, c_i32, c_i64, c_vp, c_i64, c_vp, c_vp, c_vp, c_vp]),
    ("scn_plan_create", c_i32, [_P(c_vp), c_i32, _P(c_vp), _P(c_vp), _P(c_vp), _P(scn_tune), _P(c_vp)]),
    ("scn_plan_destroy", c_i32, [c_vp]),
    ("scn_plan_set_tune", c_i32, [c_vp, _P(scn_tune)]),
    ("scn_plan_get_tune", c_i32, [c_vp, _P(scn_tune)]),
    ("scn_plan_info", c_i32, [c_vp, _P(c_i64), _P(c_i64), _P(c_i64), _P(c_i32)]),
    ("scn_plan_run", c_i32, [c_vp, c_vp]),
    ("scn_plan_capture_graph", c_i32, [c_vp, c_vp]),
    ("scn_plan_replay", c_i32, [c_vp, c_vp]),
    ("scn_plan_sync_status", c_i32, [c_vp, c_vp]),
    ("scn_plan_autotune", c_i32, [c_vp, c_i32, c_vp, _P(scn_tune), _P(ctypes.c_float)]),
    ("scn_cnn_num_params", c_i64, []),
    ("scn_cnn_create", c_i32, [c_i64, _P(c_vp)]),
    ("scn_cnn_destroy", c_i32, [c_vp]),
    ("scn_cnn_set_params", c_i32, [c_vp, _P(ctypes.c_float), c_i64]),
    ("scn_cnn_get_params", c_i32, [c_vp, _P(ctypes.c_float), c_i64]),
    ("scn_cnn_forward", c_i32, [c_vp, c_vp, c_vp, c_vp, c_i64, c_vp, c_vp]),
    ("scn_cnn_gradients", c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp, c_i64, ctypes.c_float, c_vp, c_vp, c_vp]),
    ("scn_cnn_train_step", c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp, c_i64, ctypes.c_float, ctypes.c_float, c_vp, c_vp]),
    ("scn_cnn_activation", c_i32, [c_vp, c_i32, _P(c_vp)]),
    ("scn_cnn_sync_status", c_i32, [c_vp, c_vp]),
    ("scn_gated_hist_scores", c_i32, [c_vp, c_vp, ctypes.c_float, c_vp, c_vp, c_vp, _P(c_i64), c_vp]),
    ("scn_proposal_hist_scores", c_i32, [c_vp, c_vp, ctypes.c_float, c_vp, c_vp, c_vp, c_vp, c_vp, _P(c_i64), c_vp]),
    ("scn_thumb_diff", c_i32, [c_vp, c_i64, c_vp, c_vp]),
    ("scn_cascade_hist_scores", c_i32, [c_vp, c_vp, ctypes.c_float, ctypes.c_float, c_vp, c_vp, c_vp, c_vp, c_vp,
                                        c_vp, c_vp, _P(c_i64), c_vp]),
    ("scn_thumb_diff_yuv", c_i32, [c_vp, c_i64, c_vp, c_vp]),
    ("scn_thumbs_yuv", c_i32, [c_vp, c_vp, c_vp, c_vp]),
    ("scn_resize_norm", c_i32, [c_vp, c_i32, c_i32, _P(ctypes.c_float), _P(ctypes.c_float), c_i32, c_vp, c_vp]),
    ("scn_thumbs", c_i32, [c_vp, c_vp, c_vp]),
    ("scn_resize_norm_both", c_i32, [c_vp, c_i32, c_i32, _P(ctypes.c_float), _P(ctypes.c_float), c_vp, c_vp, c_vp]),
    ("scn_space", c_i32, [c_vp, c_vp, c_i32, c_i32, c_vp, c_vp, c_vp]),
    ("scn_slice", c_i32, [c_vp, c_i64, c_vp, c_vp, c_vp]),
    ("scn_slice_middles", c_i32, [c_vp, c_vp, c_i64, c_vp, c_vp]),
    ("scn_shot_scores_sliced", c_i32, [c_vp, c_i64, c_i64, c_vp, c_vp, c_vp, c_vp]),
    ("scn_montage", c_i32, [c_vp, c_vp, c_i64, c_i32, c_i32, c_i32, c_vp, c_vp]),
    ("scn_window_scores", c_i32, [c_vp, c_i64, c_i64, c_i64, c_i32, c_i32, c_i64, c_vp, c_i64, c_i64, c_vp, c_vp, c_vp]),
    ("scn_bounded_state_scores", c_i32, [c_vp, c_i64, c_i64, c_i64, c_i64, c_i32, c_i64, c_i64, c_i64, c_i64, c_i64,
                                         c_vp, c_vp, c_vp, c_vp]),
]


def _load() -> ctypes.CDLL:
    path = _build.build()
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()
LIB_PATH = _build.LIB


def lib() -> ctypes.CDLL:
    return _lib


def _check(status: int, where: str) -> None:
    if status != SCN_OK:
        raise ScnError(status, where)


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _i64_array(values):
    """values (list, tuple or array of ints) as one contiguous int64 buffer:
    (pointer, count, owner); the owner must outlive the call that reads the pointer."""
    arr = np.ascontiguousarray(values, dtype=np.int64).reshape(-1)
    n = int(arr.size)
    if n == 0:
        arr = np.zeros(1, dtype=np.int64)
    return arr.ctypes.data_as(ctypes.POINTER(c_i64)), n, arr


def _ptr(t) -> int | None:
    if t is None:
        return None
    return t.data_ptr()


# --------------------------------------------------------------------------- thin wrappers
def scn_version() -> str:
    return _lib.scn_version().decode()


def scn_device_sm_count() -> int:
    return int(_lib.scn_device_sm_count())


def _shots_list(arr, n):
    return [dict(start=s.start, base=list(s.base), gx=list(s.gx), gy=list(s.gy)) for s in arr[:n]]


def scn_gen_shots(master_seed: int, video_id: int, width: int, height: int, num_frames: int,
                  num_shots: int = 1, shot_mode: int = 0) -> list[dict]:
    p = scn_gen_params(master_seed, video_id, width, height, num_frames, num_shots, shot_mode)
    n = c_i64()
    _check(_lib.scn_gen_shots(ctypes.byref(p), None, 0, ctypes.byref(n)), "scn_gen_shots")
    arr = (scn_shot * max(n.value, 1))()
    _check(_lib.scn_gen_shots(ctypes.byref(p), arr, n.value, ctypes.byref(n)), "scn_gen_shots")
    return _shots_list(arr, n.value)


def scn_video_create(master_seed: int, video_id: int, width: int, height: int, num_frames: int,
                     num_shots: int = 1, shot_mode: int = 0) -> int:
    p = scn_gen_params(master_seed, video_id, width, height, num_frames, num_shots, shot_mode)
    h = c_vp()
    _check(_lib.scn_video_create(ctypes.byref(p), ctypes.byref(h)), "scn_video_create")
    return h.value


def scn_video_destroy(v: int) -> None:
    _check(_lib.scn_video_destroy(v), "scn_video_destroy")


def scn_video_shots(v: int) -> list[dict]:
    n = c_i64()
    _check(_lib.scn_video_shots(v, None, 0, ctypes.byref(n)), "scn_video_shots")
    arr = (scn_shot * max(n.value, 1))()
    _check(_lib.scn_video_shots(v, arr, n.value, ctypes.byref(n)), "scn_video_shots")
    return _shots_list(arr, n.value)


def scn_video_keyframes(v: int) -> list[int]:
    n = c_i64()
    _check(_lib.scn_video_keyframes(v, None, 0, ctypes.byref(n)), "scn_video_keyframes")
    arr = (c_i64 * max(n.value, 1))()
    _check(_lib.scn_video_keyframes(v, arr, n.value, ctypes.byref(n)), "scn_video_keyframes")
    return list(arr[: n.value])


def scn_generate(v: int, out, first_frame: int, count: int, frame_stride: int, stream=None) -> None:
    _check(_lib.scn_generate(v, _ptr(out), first_frame, count, frame_stride, _stream(stream)), "scn_generate")


def scn_generate_frames(v: int, frames, out, frame_stride: int, stream=None) -> None:
    _check(_lib.scn_generate_frames(v, _ptr(frames), frames.numel(), _ptr(out), frame_stride, _stream(stream)),
           "scn_generate_frames")


def scn_table_create(nv12, width: int, height: int, num_frames: int, frame_stride: int | None = None,
                     rows=None, keyframes=None, d_nv12: int | None = None) -> int:
    """nv12: a CUDA uint8 tensor (or pass d_nv12 as a raw device address)."""
    if frame_stride is None:
        frame_stride = width * height * 3 // 2
    rows_arr, nrows, rows_keep = _i64_array(rows) if rows is not None else (None, 0, None)
    kf_arr, nkf, kf_keep = _i64_array(keyframes) if keyframes is not None else (None, 0, None)
    d = scn_table_desc(width, height, num_frames, frame_stride, d_nv12 if d_nv12 is not None else _ptr(nv12),
                       rows_arr, nrows, kf_arr, nkf)
    h = c_vp()
    _check(_lib.scn_table_create(ctypes.byref(d), ctypes.byref(h)), "scn_table_create")
    del rows_keep, kf_keep  # the library copied the lists
    return h.value


def scn_table_destroy(t: int) -> None:
    _check(_lib.scn_table_destroy(t), "scn_table_destroy")


def _spec(kind: int, start: int = 0, stop: int = 0, step: int = 1, indices=None):
    if indices is not None:
        arr, n, keep = _i64_array(indices)
    else:
        arr, n, keep = None, 0, None
    return scn_sample_spec(kind, start, stop, step, arr, n), keep


def scn_sample_indices(t: int, kind: int, start: int = 0, stop: int = 0, step: int = 1, indices=None) -> list[int]:
    sp, keep = _spec(kind, start, stop, step, indices)
    n = c_i64()
    _check(_lib.scn_sample_indices(t, ctypes.byref(sp), None, 0, ctypes.byref(n)), "scn_sample_indices")
    out = (c_i64 * max(n.value, 1))()
    _check(_lib.scn_sample_indices(t, ctypes.byref(sp), out, n.value, ctypes.byref(n)), "scn_sample_indices")
    del keep
    return list(out[: n.value])


def scn_sample(t: int, kind: int, start: int = 0, stop: int = 0, step: int = 1, indices=None) -> int:
    sp, keep = _spec(kind, start, stop, step, indices)
    h = c_vp()
    _check(_lib.scn_sample(t, ctypes.byref(sp), ctypes.byref(h)), "scn_sample")
    del keep
    return h.value


def scn_seq_length(s: int) -> int:
    n = c_i64()
    _check(_lib.scn_seq_length(s, ctypes.byref(n)), "scn_seq_length")
    return n.value


def scn_seq_destroy(s: int) -> None:
    _check(_lib.scn_seq_destroy(s), "scn_seq_destroy")


def scn_seq_sync_status(s: int, stream=None) -> int:
    return int(_lib.scn_seq_sync_status(s, _stream(stream)))


def scn_seq_set_wait_test(s: int, wait_limit_ns: int = 0, withhold_after: int = -1) -> None:
    """Test hook: bounded-wait limit of this sequence's hist launches (0: default)
    and, for withhold_after >= 0, chunks each producer hands out before withholding."""
    _check(_lib.scn_seq_set_wait_test(s, wait_limit_ns, withhold_after), "scn_seq_set_wait_test")


def scn_cnn_set_wait_test(c: int, wait_limit_ns: int = 0, withhold_batch: int = -1) -> None:
    """Test hook: bounded-wait limit of this network's inference launches (0: default)
    and, for withhold_batch >= 0, the batch whose input-built signal is withheld."""
    _check(_lib.scn_cnn_set_wait_test(c, wait_limit_ns, withhold_batch), "scn_cnn_set_wait_test")


def scn_seq_set_tune(s: int, chunk_rows: int = 0, grid: int = 0, item_kpx: int = 0) -> None:
    t = scn_tune(chunk_rows, grid, item_kpx)
    _check(_lib.scn_seq_set_tune(s, ctypes.byref(t)), "scn_seq_set_tune")


def scn_seq_get_tune(s: int) -> dict:
    t = scn_tune()
    _check(_lib.scn_seq_get_tune(s, ctypes.byref(t)), "scn_seq_get_tune")
    return dict(chunk_rows=t.chunk_rows, grid=t.grid, item_kpx=t.item_kpx)


def scn_hist(s: int, hist, stream=None) -> None:
    _check(_lib.scn_hist(s, _ptr(hist), _stream(stream)), "scn_hist")


def scn_hist_scores(s: int, hist, score, flag, stream=None) -> None:
    _check(_lib.scn_hist_scores(s, _ptr(hist), _ptr(score), _ptr(flag), _stream(stream)), "scn_hist_scores")


def scn_hist_scores_noalloc(nv12, width: int, height: int, frame_stride: int, slots, hist, score, flag,
                            stream=None) -> None:
    """Allocation-free hist+scores: slots is a device int32 tensor of frame slots."""
    _check(_lib.scn_hist_scores_noalloc(_ptr(nv12), width, height, frame_stride, _ptr(slots), slots.numel(),
                                        _ptr(hist), _ptr(score), _ptr(flag), _stream(stream)),
           "scn_hist_scores_noalloc")


def scn_shot_scores(hist, n: int, pixel_count: int, score, flag, stream=None) -> None:
    _check(_lib.scn_shot_scores(_ptr(hist), n, pixel_count, _ptr(score), _ptr(flag), _stream(stream)),
           "scn_shot_scores")


def scn_plan_create(seqs, hists, scores, flags, tune: dict | None = None) -> int:
    """seqs: sequence handles; hists/scores/flags: CUDA tensors (one per sequence)."""
    n = len(seqs)
    arr = lambda xs: (c_vp * n)(*[None if x is None else (x if isinstance(x, int) else x.data_ptr()) for x in xs])
    t = scn_tune(**tune) if tune else None
    h = c_vp()
    _check(_lib.scn_plan_create(arr(seqs), n, arr(hists), arr(scores), arr(flags),
                                ctypes.byref(t) if t is not None else None, ctypes.byref(h)), "scn_plan_create")
    return h.value


def scn_plan_destroy(p: int) -> None:
    _check(_lib.scn_plan_destroy(p), "scn_plan_destroy")


def scn_plan_set_tune(p: int, chunk_rows: int = 0, grid: int = 0, item_kpx: int = 0) -> None:
    t = scn_tune(chunk_rows, grid, item_kpx)
    _check(_lib.scn_plan_set_tune(p, ctypes.byref(t)), "scn_plan_set_tune")


def scn_plan_get_tune(p: int) -> dict:
    t = scn_tune()
    _check(_lib.scn_plan_get_tune(p, ctypes.byref(t)), "scn_plan_get_tune")
    return dict(chunk_rows=t.chunk_rows, grid=t.grid, item_kpx=t.item_kpx)


def scn_plan_info(p: int) -> dict:
    a, b, c, g = c_i64(), c_i64(), c_i64(), c_i32()
    _check(_lib.scn_plan_info(p, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(g)), "scn_plan_info")
    return dict(items=a.value, frames=b.value, nv12_bytes=c.value, grid=g.value)


def scn_plan_run(p: int, stream=None) -> None:
    _check(_lib.scn_plan_run(p, _stream(stream)), "scn_plan_run")


def scn_plan_capture_graph(p: int, stream=None) -> None:
    _check(_lib.scn_plan_capture_graph(p, _stream(stream)), "scn_plan_capture_graph")


def scn_plan_replay(p: int, stream=None) -> None:
    _check(_lib.scn_plan_replay(p, _stream(stream)), "scn_plan_replay")


def scn_plan_sync_status(p: int, stream=None) -> int:
    return int(_lib.scn_plan_sync_status(p, _stream(stream)))


def scn_plan_autotune(p: int, reps: int = 3, stream=None) -> tuple[dict, float]:
    t = scn_tune()
    ms = ctypes.c_float()
    _check(_lib.scn_plan_autotune(p, reps, _stream(stream), ctypes.byref(t), ctypes.byref(ms)), "scn_plan_autotune")
    return dict(chunk_rows=t.chunk_rows, grid=t.grid, item_kpx=t.item_kpx), float(ms.value)


def scn_cnn_num_params() -> int:
    return int(_lib.scn_cnn_num_params())


def scn_cnn_create(max_batch: int) -> int:
    h = c_vp()
    _check(_lib.scn_cnn_create(max_batch, ctypes.byref(h)), "scn_cnn_create")
    return h.value


def scn_cnn_destroy(c: int) -> None:
    _check(_lib.scn_cnn_destroy(c), "scn_cnn_destroy")


def scn_cnn_set_params(c: int, params) -> None:
    import numpy as np
    a = np.ascontiguousarray(params, dtype=np.float32)
    _check(_lib.scn_cnn_set_params(c, a.ctypes.data_as(_P(ctypes.c_float)), a.size), "scn_cnn_set_params")


def scn_cnn_get_params(c: int):
    import numpy as np
    a = np.empty(scn_cnn_num_params(), dtype=np.float32)
    _check(_lib.scn_cnn_get_params(c, a.ctypes.data_as(_P(ctypes.c_float)), a.size), "scn_cnn_get_params")
    return a


def scn_cnn_forward(c: int, thumbs, n: int, logits, prev=None, cur=None, stream=None) -> None:
    _check(_lib.scn_cnn_forward(c, _ptr(thumbs), _ptr(prev), _ptr(cur), n, _ptr(logits), _stream(stream)),
           "scn_cnn_forward")


def scn_cnn_gradients(c: int, thumbs, labels, batch: int, pos_weight: float, loss=None, grads=None, prev=None,
                      cur=None, stream=None) -> None:
    _check(_lib.scn_cnn_gradients(c, _ptr(thumbs), _ptr(prev), _ptr(cur), _ptr(labels), batch, pos_weight,
                                  _ptr(loss), _ptr(grads), _stream(stream)), "scn_cnn_gradients")


def scn_cnn_train_step(c: int, thumbs, labels, batch: int, pos_weight: float, lr: float, loss=None, prev=None,
                       cur=None, stream=None) -> None:
    _check(_lib.scn_cnn_train_step(c, _ptr(thumbs), _ptr(prev), _ptr(cur), _ptr(labels), batch, pos_weight, lr,
                                   _ptr(loss), _stream(stream)), "scn_cnn_train_step")


def scn_cnn_activation(c: int, layer: int) -> int:
    p = c_vp()
    _check(_lib.scn_cnn_activation(c, layer, ctypes.byref(p)), "scn_cnn_activation")
    return p.value


def scn_cnn_sync_status(c: int, stream=None) -> int:
    return int(_lib.scn_cnn_sync_status(c, _stream(stream)))


def scn_gated_hist_scores(s: int, gate, tau: float, proposed, score, flag, stream=None, count: bool = True):
    """Returns the number of proposals (the call then waits for the stream), or None with count=False
    (fully asynchronous)."""
    m = c_i64()
    _check(_lib.scn_gated_hist_scores(s, _ptr(gate), tau, _ptr(proposed), _ptr(score), _ptr(flag),
                                      ctypes.byref(m) if count else None, _stream(stream)), "scn_gated_hist_scores")
    return m.value if count else None


def scn_proposal_hist_scores(s: int, net: int, tau: float, thumbs, logits, proposed, score, flag, stream=None,
                             count: bool = True):
    """As scn_gated_hist_scores, gated by the network's logits."""
    m = c_i64()
    _check(_lib.scn_proposal_hist_scores(s, net, tau, _ptr(thumbs), _ptr(logits), _ptr(proposed), _ptr(score),
                                         _ptr(flag), ctypes.byref(m) if count else None, _stream(stream)),
           "scn_proposal_hist_scores")
    return m.value if count else None


def scn_cascade_hist_scores(s: int, net: int, tau_diff: float, tau_net: float, thumbs, yuv, diff, gate, proposed,
                            score, flag, stream=None, count: bool = True):
    """The luma + chroma difference gate over coarse YUV thumbnails as a prefilter, the
    network on what passes (luma thumbnails gathered for those pairs only), the exact
    kernel on pairs that pass both (see include/scn.h)."""
    m = c_i64()
    _check(_lib.scn_cascade_hist_scores(s, net, tau_diff, tau_net, _ptr(thumbs), _ptr(yuv), _ptr(diff), _ptr(gate),
                                        _ptr(proposed), _ptr(score), _ptr(flag), ctypes.byref(m) if count else None,
                                        _stream(stream)),
           "scn_cascade_hist_scores")
    return m.value if count else None


def scn_thumb_diff(thumbs, n: int, diff, stream=None) -> None:
    _check(_lib.scn_thumb_diff(_ptr(thumbs), n, _ptr(diff), _stream(stream)), "scn_thumb_diff")


def scn_thumb_diff_yuv(yuv, n: int, diff, stream=None) -> None:
    _check(_lib.scn_thumb_diff_yuv(_ptr(yuv), n, _ptr(diff), _stream(stream)), "scn_thumb_diff_yuv")


def scn_resize_norm(s: int, oh: int, ow: int, mean, std, dtype: int, out, stream=None) -> None:
    m = (ctypes.c_float * 3)(*[float(x) for x in mean])
    sd = (ctypes.c_float * 3)(*[float(x) for x in std])
    _check(_lib.scn_resize_norm(s, oh, ow, m, sd, dtype, _ptr(out), _stream(stream)), "scn_resize_norm")


def scn_resize_norm_both(s: int, oh: int, ow: int, mean, std, out_f32, out_bf16, stream=None) -> None:
    m = (ctypes.c_float * 3)(*[float(x) for x in mean])
    sd = (ctypes.c_float * 3)(*[float(x) for x in std])
    _check(_lib.scn_resize_norm_both(s, oh, ow, m, sd, _ptr(out_f32), _ptr(out_bf16), _stream(stream)),
           "scn_resize_norm_both")


def scn_thumbs(s: int, thumb, stream=None) -> None:
    _check(_lib.scn_thumbs(s, _ptr(thumb), _stream(stream)), "scn_thumbs")


def scn_thumbs_yuv(s: int, thumb, yuv, stream=None) -> None:
    """thumb: [n][36][64] luma thumbnails or None; yuv: [n][3][6][32] coarse YUV thumbnails or None."""
    _check(_lib.scn_thumbs_yuv(s, _ptr(thumb), _ptr(yuv), _stream(stream)), "scn_thumbs_yuv")


def scn_space(s: int, values, elem_bytes: int, out, fill_mode: int = SCN_FILL_VALUE, fill: bytes | None = None,
              stream=None) -> None:
    """values: CUDA tensor holding length(s) elements of elem_bytes bytes; out: CUDA tensor
    holding num_frames elements of the table."""
    buf = None
    if fill is not None:
        if len(fill) != elem_bytes:
            raise ValueError("fill must be elem_bytes long")
        buf = ctypes.create_string_buffer(bytes(fill), elem_bytes)
    _check(_lib.scn_space(s, _ptr(values), elem_bytes, fill_mode, buf, _ptr(out), _stream(stream)), "scn_space")


def scn_slice(flags, n: int, starts, count, stream=None) -> None:
    _check(_lib.scn_slice(_ptr(flags), n, _ptr(starts), _ptr(count), _stream(stream)), "scn_slice")


def scn_slice_middles(starts, count, n: int, mids, stream=None) -> None:
    _check(_lib.scn_slice_middles(_ptr(starts), _ptr(count), n, _ptr(mids), _stream(stream)), "scn_slice_middles")


def scn_shot_scores_sliced(hist, n: int, pixel_count: int, boundary, score, flag, stream=None) -> None:
    _check(_lib.scn_shot_scores_sliced(_ptr(hist), n, pixel_count, _ptr(boundary), _ptr(score), _ptr(flag),
                                       _stream(stream)), "scn_shot_scores_sliced")


def scn_montage(s: int, elems, m: int, cols: int, tile_w: int, tile_h: int, out, stream=None) -> None:
    _check(_lib.scn_montage(s, _ptr(elems), m, cols, tile_w, tile_h, _ptr(out), _stream(stream)), "scn_montage")


def scn_window_scores(hist, hist_first: int, hist_count: int, n: int, a: int, b: int, pixel_count: int, k0: int,
                      k1: int, score, flag, boundary=None, stream=None) -> None:
    """hist: CUDA tensor holding elements [hist_first, hist_first + hist_count) of the sequence."""
    _check(_lib.scn_window_scores(_ptr(hist), hist_first, hist_count, n, a, b, pixel_count, _ptr(boundary), k0, k1,
                                  _ptr(score), _ptr(flag), _stream(stream)), "scn_window_scores")


def scn_bounded_state_scores(hist, hist_first: int, hist_count: int, n: int, pixel_count: int, shift: int,
                             warmup: int, run_first: int, run_len: int, run_stride: int, runs: int, score, flag,
                             boundary=None, stream=None) -> None:
    """hist: CUDA tensor holding elements [hist_first, hist_first + hist_count); score/flag: one slot per
    output of each run (run r, element k -> r*run_len + k - run start)."""
    _check(_lib.scn_bounded_state_scores(_ptr(hist), hist_first, hist_count, n, pixel_count, shift, warmup,
                                         run_first, run_len, run_stride, runs, _ptr(boundary), _ptr(score),
                                         _ptr(flag), _stream(stream)), "scn_bounded_state_scores")

