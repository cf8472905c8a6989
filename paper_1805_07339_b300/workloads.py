"""Seeded synthetic workloads: sizes, seeds and raw random inputs.

Holds no arithmetic of the method (no conversion, binning, scoring or
resampling).  The CUDA path, the tests and the benchmark take their inputs from
here; video frames themselves come from each side's own generator.
"""
from __future__ import annotations

import numpy as np

MASTER_SEED = 20180805

# 1 synthetic 320x180 video, 240 frames, 8 shots, stride-1
TINY = dict(width=320, height=180, num_frames=240, num_shots=8)
# 1 synthetic 1920x1080 video, 7200 frames (22.4 GB of NV12), 60 shots
HD = dict(width=1920, height=1080, num_frames=7200, num_shots=60)
HD_GATHER = 1000          # gathered frames of the 1080p video
HD_STRIDE = 24            # sparse stride of the 1080p video
HD_GATHER_SEED = 1000     # numpy seed of the gather list


def random_nv12(seed: int, n: int, width: int, height: int) -> np.ndarray:
    """n frames of uniformly random bytes (exercises every clamp and bin)."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, 256, (n, width * height * 3 // 2), dtype=np.uint8)


def random_indices(seed: int, num_frames: int, m: int, distinct: bool = True) -> np.ndarray:
    """m frame numbers in [0, num_frames): distinct and sorted, or i.i.d. in draw order."""
    rng = np.random.default_rng(seed)
    if distinct:
        return np.sort(rng.choice(num_frames, size=m, replace=False)).astype(np.int64)
    return rng.integers(0, num_frames, m).astype(np.int64)


def hd_gather() -> np.ndarray:
    """The 1080p gather list: 1000 distinct sorted frames of 7200."""
    return random_indices(HD_GATHER_SEED, HD["num_frames"], HD_GATHER)


# Batched uneven workload: videos of four resolution classes, uniform lengths,
# and one of four sampling patterns each.
RESOLUTIONS = [(640, 360), (1280, 720), (1920, 1080), (3840, 2160)]
SAMPLINGS = ["stride1", "stride24", "range", "gather5"]
BATCH_SEED = 3


def batched_spec(nvideos: int = 64, min_len: int = 200, max_len: int = 3000, seed: int = BATCH_SEED,
                 resolutions=None) -> list[dict]:
    """Per video: id, width, height, frames, shots (one per 120 frames) and the
    sampled frame numbers (sorted for stride/range, in draw order for gather)."""
    rng = np.random.default_rng(seed)
    res = resolutions or RESOLUTIONS
    out = []
    for v in range(nvideos):
        W, H = res[int(rng.integers(0, len(res)))]
        T = int(rng.integers(min_len, max_len + 1))
        kind = SAMPLINGS[int(rng.integers(0, len(SAMPLINGS)))]
        if kind == "stride1":
            idx = np.arange(T)
        elif kind == "stride24":
            idx = np.arange(0, T, 24)
        elif kind == "range":
            a, b = sorted(int(x) for x in rng.choice(T + 1, size=2, replace=False))
            idx = np.arange(a, b)
        else:
            m = max(1, T // 20)
            idx = np.sort(rng.choice(T, size=m, replace=False))
        out.append(dict(video_id=1000 + v, width=W, height=H, num_frames=T, num_shots=max(1, T // 120),
                        sampling=kind, frames=idx.astype(np.int64)))
    return out


# News-archive-shaped stream: many 640x360 videos of log-uniform length with
# geometric shot lengths; each sampled at stride 24 plus a seeded 1% gather.
STREAM = dict(width=640, height=360, nvideos=2000, min_len=1800, max_len=54000, stride=24, gather_percent=1)
STREAM_SEED = 5
STREAM_ID0 = 200000  # video ids of the stream (disjoint from every other workload)


def stream_spec(nvideos: int = STREAM["nvideos"], seed: int = STREAM_SEED, min_len: int = STREAM["min_len"],
                max_len: int = STREAM["max_len"], id0: int = STREAM_ID0) -> list[dict]:
    """Per video: id, size, length (log-uniform in [min_len, max_len]), shot_mode 1
    (geometric shot lengths), the stride-24 frames and a sorted seeded 1% gather."""
    rng = np.random.default_rng(seed)
    W, H, step = STREAM["width"], STREAM["height"], STREAM["stride"]
    out = []
    for v in range(nvideos):
        T = int(round(float(np.exp(rng.uniform(np.log(min_len), np.log(max_len))))))
        m = max(1, (T * STREAM["gather_percent"] + 50) // 100)
        gather = np.sort(rng.choice(T, size=m, replace=False)).astype(np.int64)
        out.append(dict(video_id=id0 + v, width=W, height=H, num_frames=T, shot_mode=1,
                        stride=np.arange(0, T, step, dtype=np.int64), gather=gather))
    return out
