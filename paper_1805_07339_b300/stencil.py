"""Stencils over sharded sequences: per-element dependency analysis and halos.

The paper runs a stencil op over a sequence split into tasks; each task reads
the extra elements its window needs (Sec. 3.2 stencils, Sec. 4.2 dependency
analysis).  Here a shard of outputs [k0, k1) of S[a, b] needs input elements
[k0 + a, k1 + b) clipped to the sequence; the computation itself runs in
libscn (scn_window_scores), which refuses a slice that does not cover that range.
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
