"""Stencils and bounded-state ops over sharded sequences: per-element dependency
analysis, halos and warmup.

The paper runs a stencil op over a sequence split into tasks; each task reads
the extra elements its window needs (Sec. 3.2 stencils, Sec. 4.2 dependency
analysis).  Here a shard of outputs [k0, k1) of S[a, b] needs input elements
[k0 + a, k1 + b) clipped to the sequence; the computation itself runs in
libscn (scn_window_scores), which refuses a slice that does not cover that range.

A bounded-state op with warmup W (Sec. 3.2) reads i - W .. i for output i
(Sec. 4.2 treats it as that stencil); its runs of outputs are processed
independently, each from W elements before its first output
(scn_bounded_state_scores, one launch for all runs).
"""
from __future__ import annotations

from . import scn


def dependency_range(k0: int, k1: int, a: int, b: int, n: int) -> tuple[int, int]:
    """Input elements the outputs [k0, k1) of S[a, b] read, clipped to [0, n)."""
    return max(0, k0 + a), min(n, k1 + b)


def shards(n: int, parts: int) -> list[tuple[int, int]]:
    """parts contiguous output ranges covering [0, n)."""
    step = -(-n // max(parts, 1))
    return [(k, min(n, k + step)) for k in range(0, n, step)] if n else []


def window_scores_sharded(torch, hist, n: int, a: int, b: int, pixel_count: int, parts: int, boundary=None,
                          stream=None):
    """S[a, b] window scores of an n-element histogram sequence, computed shard by shard,
    each shard given only its dependency range (a copy, as another task or device would
    hold it).  Returns (score uint64 as int64 tensor, flag) for all n elements."""
    score = torch.empty(n, dtype=torch.int64, device="cuda")
    flag = torch.empty(n, dtype=torch.uint8, device="cuda")
    for k0, k1 in shards(n, parts):
        i0, i1 = dependency_range(k0, k1, a, b, n)
        part = hist[i0:i1].clone()  # only the shard's inputs, with its halo
        bpart = boundary[i0:i1].clone() if boundary is not None else None
        scn.scn_window_scores(part, i0, i1 - i0, n, a, b, pixel_count, k0, k1, score[k0:k1], flag[k0:k1],
                              boundary=bpart, stream=stream)
    return score, flag


def state_shards(n: int, parts: int) -> tuple[int, int, int, int]:
    """Run pattern (run_first, run_len, run_stride, runs) splitting outputs [0, n) into
    `parts` contiguous shards (the last one ragged)."""
    step = max(1, -(-n // max(parts, 1)))
    return 0, step, step, -(-n // step) if n else 0


def state_sparse(n: int, every: int, offset: int = 0) -> tuple[int, int, int, int]:
    """Run pattern producing only outputs offset, offset + every, ... (one output per run)."""
    return offset, 1, every, max(0, -(-(n - offset) // every))


def state_inputs(run_first: int, run_len: int, run_stride: int, runs: int, warmup: int,
                 n: int) -> list[tuple[int, int]]:
    """The exact input elements the runs read, as disjoint ascending intervals: run r
    with outputs [k0, k1) reads [max(0, k0 - warmup), k1) (Sec. 4.2)."""
    out: list[tuple[int, int]] = []
    for r in range(runs):
        k0 = run_first + r * run_stride
        if k0 >= n:
            break
        lo, hi = max(0, k0 - warmup), min(n, k0 + run_len)
        if out and lo <= out[-1][1]:
            out[-1] = (out[-1][0], max(out[-1][1], hi))
        else:
            out.append((lo, hi))
    return out


def state_input_fraction(run_first: int, run_len: int, run_stride: int, runs: int, warmup: int, n: int) -> float:
    """Share of the n elements that the runs read (sparse execution, Sec. 4.2)."""
    return sum(b - a for a, b in state_inputs(run_first, run_len, run_stride, runs, warmup, n)) / n if n else 0.0
