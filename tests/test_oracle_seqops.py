"""Pins for the oracle's sequence operations: hand-worked cases, the identities
that tie spacing to sampling, brute-force partitions, and the montage against the
full-frame conversion (itself pinned by the BT.601 colour bars)."""
import numpy as np

import oracle
from oracle import seqops


def test_space_hand_example():
    # sampled frames 1, 4 (stride 3 from 1) of a 7-frame video
    v = np.array([[10], [20]])
    assert seqops.space(v, [1, 4], 7, fill=[-1])[:, 0].tolist() == [-1, 10, -1, -1, 20, -1, -1]
    assert seqops.space(v, [1, 4], 7, repeat=True, fill=[-1])[:, 0].tolist() == [-1, 10, 10, 10, 20, 20, 20]
    # a frame sampled twice: the later element wins
    assert seqops.space(np.array([[1], [2], [3]]), [5, 2, 5], 6)[:, 0].tolist() == [0, 0, 2, 0, 0, 3]


def test_space_inverts_sampling():
    rng = np.random.default_rng(3)
    for T, idx in [(50, np.arange(0, 50, 7)), (40, np.sort(rng.choice(40, 9, replace=False))),
                   (30, rng.integers(0, 30, 12))]:
        dense = rng.integers(0, 1000, (T, 3))
        sampled = dense[idx]
        out = seqops.space(sampled, idx, T, fill=[-5, -5, -5])
        # sampling the spaced sequence gives back what was sampled (last writer for repeats)
        last = {int(f): k for k, f in enumerate(idx)}
        for f, k in last.items():
            assert np.array_equal(out[f], sampled[k])
        # every other frame holds the fill
        assert np.sum(np.all(out == -5, axis=1)) == T - len(last)
        rep = seqops.space(sampled, idx, T, repeat=True, fill=[-5, -5, -5])
        first = min(last)
        assert np.all(rep[:first] == -5) and not np.any(np.all(rep[first:] == -5, axis=1))


def test_slices_partition_the_sequence():
    rng = np.random.default_rng(4)
    for n in (1, 2, 17, 300):
        flags = (rng.random(n) < 0.2).astype(np.uint8)
        st = seqops.slice_starts(flags)
        assert st[0] == 0 and np.all(np.diff(st) > 0)
        # brute force: every element belongs to exactly one slice, and a new one begins exactly at flags
        sid = np.cumsum([1 if (k == 0 or flags[k]) else 0 for k in range(n)]) - 1
        assert len(st) == sid[-1] + 1
        for i, s in enumerate(st):
            assert sid[s] == i and (s == 0 or sid[s - 1] == i - 1)
        mid = seqops.slice_middles(st, n)
        ends = np.append(st[1:], n)
        assert np.all((st <= mid) & (mid < ends)) and np.all(np.abs((mid - st) - (ends - 1 - mid)) <= 1)


def test_sliced_scores_reset_at_boundaries():
    rng = np.random.default_rng(5)
    hist = rng.integers(0, 1000, (20, 48)).astype(np.uint32)
    b = np.zeros(20, np.uint8)
    s0, f0 = oracle.scores(hist, 5000)
    s, f = seqops.sliced_scores(hist, b, 5000)
    assert np.array_equal(s, s0) and np.array_equal(f, f0)  # no slices: plain stencil
    b[[4, 11]] = 1
    s, f = seqops.sliced_scores(hist, b, 5000)
    assert s[4] == 0 and s[11] == 0 and f[4] == 0 and f[11] == 0
    keep = [k for k in range(20) if k not in (0, 4, 11)]
    assert np.array_equal(s[keep], s0[keep])


def test_montage_full_size_tile_is_the_converted_frame():
    rng = np.random.default_rng(6)
    W, H = 16, 8
    fr = rng.integers(0, 256, W * H * 3 // 2).astype(np.uint8)
    m = seqops.montage([fr], W, H, cols=1, tile_w=W, tile_h=H)
    # full-size tile: every pixel maps to itself, so the tile is the whole frame in RGB
    yuv = np.empty((H, W, 3), np.uint8)
    for y in range(H):
        for x in range(W):
            uv = W * H + (y // 2) * W + (x // 2) * 2
            yuv[y, x] = (fr[y * W + x], fr[uv], fr[uv + 1])
    assert np.array_equal(m, oracle.yuv_to_rgb_array(yuv.reshape(-1, 3)).reshape(H, W, 3))


def test_montage_layout_and_constant_frames():
    W, H = 32, 18
    grey = np.full(W * H * 3 // 2, 128, np.uint8)
    grey[:W * H] = 126  # Y = 126 -> (298*110 + 128) >> 8 = 128
    m = seqops.montage([grey, None, grey], W, H, cols=2, tile_w=5, tile_h=3)
    assert m.shape == (6, 10, 3)
    assert np.all(m[:3, :5] == 128) and np.all(m[:3, 5:] == 0) and np.all(m[3:, :5] == 128) and np.all(m[3:, 5:] == 0)
    assert oracle.yuv_to_rgb(126, 128, 128) == (128, 128, 128)


def test_window_scores_reduce_to_the_plain_score():
    rng = np.random.default_rng(10)
    hist = rng.integers(0, 900, (40, 48)).astype(np.uint32)
    s0, f0 = oracle.scores(hist, 7000)
    s, f = seqops.window_scores(hist, -1, 0, 7000)
    assert np.array_equal(s.astype(np.uint64), s0.astype(np.uint64)) and np.array_equal(f, f0)


def test_window_scores_hand_cases():
    # one bin, pixel_count 10: a cut between frames 3 and 4, and a one-frame flash at 8
    h = np.zeros((12, 1), np.int64)
    h[:4, 0] = 10
    h[4:, 0] = 0
    h[8, 0] = 10
    s, f = seqops.window_scores(h, -2, 1, 10)  # P = 2 before, F = 2 from k
    # k = 4: before = frames 2, 3 (20), after = frames 4, 5 (0): |2*20 - 2*0| = 40 > 2*2*10/2
    assert s[4] == 40 and f[4] == 1
    # k = 8 (the flash): before = 6, 7 (0), after = 8, 9 (10): |0 - 20| = 20, 2*20 = 40 = P*F*10: no flag
    assert s[8] == 20 and f[8] == 0
    # the plain score flags the flash twice (into it and out of it)
    _, fp = seqops.window_scores(h, -1, 0, 10)
    assert fp[8] == 1 and fp[9] == 1
    # windows outside the sequence: the first 2 and the last 1 elements
    assert s[0] == s[1] == s[11] == 0
    # a slice start inside the window (after its first element) zeroes the score: the windows of
    # k = 4, 5, 6 contain frame 5 after their first frame; k = 7's window starts at frame 5
    bnd = np.zeros(12, np.uint8)
    bnd[5] = 1
    sb, _ = seqops.window_scores(h, -2, 1, 10, boundary=bnd)
    assert sb[4] == 0 and sb[5] == 0 and sb[6] == 0
    assert sb[3] == s[3] and sb[7] == s[7] and sb[8] == s[8]


def test_window_scores_brute_force_and_dependency_ranges():
    rng = np.random.default_rng(11)
    for a, b in [(-1, 0), (-3, 0), (-2, 2), (-5, 4)]:
        hist = rng.integers(0, 50, (30, 4)).astype(np.int64)
        s, f = seqops.window_scores(hist, a, b, 100)
        for k in range(30):
            if k + a < 0 or k + b >= 30:
                assert s[k] == 0
                continue
            P, F = -a, b + 1
            mb = hist[k + a:k].sum(0) / P
            ma = hist[k:k + b + 1].sum(0) / F
            assert abs(s[k] - P * F * np.abs(mb - ma).sum()) < 1e-6
        # outputs [k0, k1) computed from only their dependency range give the same values
        for k0, k1 in [(0, 7), (7, 19), (19, 30)]:
            i0, i1 = seqops.stencil_inputs(k0, k1, a, b, 30)
            part = np.zeros_like(hist)
            part[i0:i1] = hist[i0:i1]  # everything outside the range erased
            sp, _ = seqops.window_scores(part, a, b, 100)
            assert np.array_equal(sp[k0:k1], s[k0:k1])
