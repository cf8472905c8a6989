"""Sequence operations of the oracle: spacing, slicing, slice representatives,
sliced shot scores, montage.  TEST INFRASTRUCTURE ONLY (same rules as the
package: only tests/, the smoke check and the bench's CPU legs use it).

Definitions (Scanner, Poms et al. 2018):
  * spacing inverts sampling: the sampled results go back to their frames and
    the other frames receive "fill" elements (Sec. 3.2, sampling/spacing); the
    fill is a given element, or (the repeat reading) the nearest earlier
    sampled frame's result;
  * slicing partitions a sequence at boundaries so that stencils and state do
    not cross them (Sec. 3.2, slicing/unslicing); a boundary element starts a
    slice, and so does element 0;
  * a film summary shows one frame per shot (Sec. 5.2, montage); here the
    middle element of each slice, nearest-neighbour downsampled into a tile;
  * a stencil S[a, b] reads a window of elements around each output (Sec. 3.2);
  * a bounded-state op carries state from element to element, and before it
    produces element i it has processed at least the W elements before i (the
    warmup, Sec. 3.2); a run of outputs therefore starts W elements early and
    drops those outputs; dependency analysis treats the op as a stencil over
    (i - W .. i) (Sec. 4.2).
Pins: tests/test_oracle_seqops.py.
"""
from __future__ import annotations

import numpy as np

from . import scores as _scores
from . import yuv_to_rgb_array


def space(values: np.ndarray, frames, num_frames: int, repeat: bool = False, fill=None) -> np.ndarray:
    """values: [n, ...] results of the sampled elements; frames: the frame each element sampled."""
    values = np.asarray(values)
    elem = values.shape[1:]
    fill_v = np.zeros(elem, dtype=values.dtype) if fill is None else np.asarray(fill, dtype=values.dtype)
    have = [None] * num_frames
    for k, f in enumerate(frames):  # a later element sampling the same frame replaces an earlier one
        have[int(f)] = k
    out = np.empty((num_frames,) + elem, dtype=values.dtype)
    last = None
    for t in range(num_frames):
        if have[t] is not None:
            last = values[have[t]]
            out[t] = last
        elif repeat and last is not None:
            out[t] = last
        else:
            out[t] = fill_v
    return out


def slice_starts(flags) -> np.ndarray:
    """First element of every slice: k == 0 or flags[k] != 0, ascending."""
    flags = np.asarray(flags)
    return np.array([k for k in range(len(flags)) if k == 0 or flags[k] != 0], dtype=np.int64)


def slice_middles(starts, n: int) -> np.ndarray:
    ends = list(starts[1:]) + [n]
    return np.array([(s + e - 1) // 2 for s, e in zip(starts, ends)], dtype=np.int64)


def sliced_scores(hist: np.ndarray, boundary, pixel_count: int):
    """Shot scores whose stencil stops at slice starts (score 0 there)."""
    s, f = _scores(hist, pixel_count)
    s = s.copy()
    f = f.copy()
    for k in range(len(s)):
        if k == 0 or boundary[k] != 0:
            s[k] = 0
            f[k] = 0
    return s, f


def montage(frames: list, W: int, H: int, cols: int, tile_w: int, tile_h: int) -> np.ndarray:
    """frames: NV12 frames of the tiles in order (None = a black tile)."""
    m = len(frames)
    rows = (m + cols - 1) // cols
    out = np.zeros((rows * tile_h, cols * tile_w, 3), dtype=np.uint8)
    xs = [((2 * x + 1) * W) // (2 * tile_w) for x in range(tile_w)]
    ys = [((2 * y + 1) * H) // (2 * tile_h) for y in range(tile_h)]
    for i, fr in enumerate(frames):
        if fr is None:
            continue
        fr = np.asarray(fr, dtype=np.uint8)
        yuv = np.empty((tile_h, tile_w, 3), dtype=np.uint8)
        for ty, sy in enumerate(ys):
            for tx, sx in enumerate(xs):
                uv = W * H + (sy // 2) * W + (sx // 2) * 2
                yuv[ty, tx] = (fr[sy * W + sx], fr[uv], fr[uv + 1])
        r0, c0 = (i // cols) * tile_h, (i % cols) * tile_w
        out[r0:r0 + tile_h, c0:c0 + tile_w] = yuv_to_rgb_array(yuv.reshape(-1, 3)).reshape(tile_h, tile_w, 3)
    return out


def window_scores(hist: np.ndarray, a: int, b: int, pixel_count: int, boundary=None):
    """Stencil S[a, b] shot score (Sec. 3.2 stencils; a < 0 <= b): for element k,
    with P = -a frames before it and F = b + 1 frames from it,
      score[k] = sum over bins | F * sum_{j=a}^{-1} h[k+j] - P * sum_{j=0}^{b} h[k+j] |,
      flag[k] = 2 * score[k] > P * F * pixel_count,
    i.e. the L1 distance of the two windows' mean histograms, scaled by P * F to stay
    in integers.  An element whose window reaches outside the sequence, or contains a
    slice start after its first element (boundary[s] != 0 for k+a < s <= k+b), gets
    score 0 and flag 0.  a = -1, b = 0 is the plain two-frame shot score."""
    h = np.asarray(hist, dtype=np.int64).reshape(len(hist), -1)
    n = h.shape[0]
    P, F = -a, b + 1
    score = np.zeros(n, dtype=np.uint64)
    flag = np.zeros(n, dtype=np.uint8)
    for k in range(n):
        if k + a < 0 or k + b >= n:
            continue
        if boundary is not None and any(boundary[s] for s in range(k + a + 1, k + b + 1)):
            continue
        before = h[k + a:k].sum(axis=0)
        after = h[k:k + b + 1].sum(axis=0)
        sc = int(np.abs(F * before - P * after).sum())
        score[k] = sc
        flag[k] = 1 if 2 * sc > P * F * pixel_count else 0
    return score, flag


def stencil_inputs(k0: int, k1: int, a: int, b: int, n: int) -> tuple[int, int]:
    """Per-element dependency analysis of S[a, b] (Sec. 4.2): the input elements the
    outputs [k0, k1) read, clipped to the sequence."""
    return max(0, k0 + a), min(n, k1 + b)


def bounded_state_run(hist: np.ndarray, pixel_count: int, shift: int, j0: int, k0: int, k1: int, boundary=None):
    """One run of the bounded-state shot score: process elements j0 .. k1-1 in order,
    return the outputs of [k0, k1) as (score list, flag list).

    The state is a reference histogram m.  The first processed element, and an
    element where a slice starts (boundary != 0), set m to its own histogram and
    output (0, 0).  Every other element j outputs d = sum over bins |h[j] - m| and
    f = (2 d > pixel_count), then updates m to h[j] when f is set (a cut restarts
    the reference), else m + floor((h[j] - m) / 2**shift) (an exponential average
    of the shot so far).  shift = 0 makes m the previous histogram, i.e. the plain
    two-frame score."""
    h = np.asarray(hist, dtype=np.int64).reshape(len(hist), -1)
    m = None
    scores, flags = [], []
    for j in range(j0, k1):
        if m is None or (boundary is not None and boundary[j] != 0):
            m = h[j].copy()
            d, f = 0, 0
        else:
            d = int(np.abs(h[j] - m).sum())
            f = 1 if 2 * d > pixel_count else 0
            if f:
                m = h[j].copy()
            else:
                m = m + np.floor_divide(h[j] - m, 2 ** shift)
        if j >= k0:
            scores.append(d)
            flags.append(f)
    return scores, flags


def bounded_state_runs(first: int, length: int, stride: int, count: int, n: int) -> list[tuple[int, int]]:
    """Output runs of the pattern: run r covers [first + r*stride, first + r*stride + length)
    clipped to [0, n) (possibly empty)."""
    out = []
    for r in range(count):
        k0 = first + r * stride
        out.append((min(k0, n), min(k0 + length, n)))
    return out


def bounded_state_scores(hist: np.ndarray, pixel_count: int, shift: int, warmup: int, first: int, length: int,
                         stride: int, count: int, boundary=None):
    """Bounded-state shot scores over runs of outputs, each run processed on its own
    from W = warmup elements before its first output (clipped at element 0); output
    slot r*length + (k - run start) holds element k of run r.  Slots of elements
    past the sequence's end hold -1."""
    n = len(hist)
    score = np.full(count * length, -1, dtype=np.int64)
    flag = np.full(count * length, -1, dtype=np.int64)
    for r, (k0, k1) in enumerate(bounded_state_runs(first, length, stride, count, n)):
        if k1 <= k0:
            continue
        s, f = bounded_state_run(hist, pixel_count, shift, max(0, k0 - warmup), k0, k1, boundary)
        score[r * length:r * length + (k1 - k0)] = s
        flag[r * length:r * length + (k1 - k0)] = f
    return score, flag


def bounded_state_inputs(first: int, length: int, stride: int, count: int, warmup: int, n: int) -> list[int]:
    """The exact set of input elements the runs read (Sec. 4.2: a warmup of W is a
    stencil footprint i - W .. i), ascending."""
    need = set()
    for k0, k1 in bounded_state_runs(first, length, stride, count, n):
        if k1 > k0:
            need.update(range(max(0, k0 - warmup), k1))
    return sorted(need)
