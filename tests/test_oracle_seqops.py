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


def test_bounded_state_hand_example():
    # two bins, pixel_count 100, shift 1 (the reference moves half way to each frame, floor)
    h = np.zeros((5, 2), np.int64)
    h[:] = [[10, 0], [6, 4], [9, 1], [0, 60], [0, 61]]
    # serial: m = (10, 0); k=1: |6-10|+|4-0| = 8, m = (10-2, 0+2) = (8, 2);
    # k=2: |9-8|+|1-2| = 2, m = (8 + floor(1/2), 2 + floor(-1/2)) = (8, 1);
    # k=3: |0-8|+|60-1| = 67, 134 > 100: cut, m = (0, 60); k=4: |0|+|61-60| = 1
    s, f = seqops.bounded_state_scores(h, 100, 1, 0, 0, 5, 5, 1)
    assert s.tolist() == [0, 8, 2, 67, 1] and f.tolist() == [0, 0, 0, 1, 0]
    # runs of two outputs, warmup 1: run [2, 4) starts at 1 with m = (6, 4):
    # k=2: |9-6|+|1-4| = 6, m = (6 + floor(3/2), 4 + floor(-3/2)) = (7, 2); k=3: |0-7|+|60-2| = 65, a cut;
    # the ragged run [4, 5) starts at 3 with m = (0, 60): k=4 scores 1; slot 5 is past the end
    s, f = seqops.bounded_state_scores(h, 100, 1, 1, 0, 2, 2, 3)
    assert s.tolist() == [0, 8, 6, 65, 1, -1] and f.tolist() == [0, 0, 0, 1, 0, -1]
    # warmup 0: every run starts from its own first output, which scores 0; run [2, 4) has m = (9, 1)
    # at k=3: |0-9|+|60-1| = 68
    s, _ = seqops.bounded_state_scores(h, 100, 1, 0, 0, 2, 2, 3)
    assert s.tolist() == [0, 8, 0, 68, 0, -1]
    # a slice start at 2 restarts the state as a run start does: m = (9, 1), k=3: |0-9|+|60-1| = 68, a cut
    bnd = np.array([0, 0, 1, 0, 0], np.uint8)
    s, f = seqops.bounded_state_scores(h, 100, 1, 0, 0, 5, 5, 1, boundary=bnd)
    assert s.tolist() == [0, 8, 0, 68, 1] and f.tolist() == [0, 0, 0, 1, 0]
    # sparse outputs (every other element, warmup 2) read exactly the elements within 2 before each
    assert seqops.bounded_state_inputs(1, 1, 2, 2, 2, 5) == [0, 1, 2, 3]
    assert seqops.bounded_state_inputs(4, 1, 9, 3, 1, 5) == [3, 4]


def test_bounded_state_shift_zero_is_the_plain_score():
    rng = np.random.default_rng(12)
    hist = rng.integers(0, 900, (60, 48)).astype(np.uint32)
    s0, f0 = oracle.scores(hist, 20000)
    for warmup, length in [(1, 60), (1, 7), (3, 1), (60, 13)]:
        count = -(-60 // length)
        s, f = seqops.bounded_state_scores(hist, 20000, 0, warmup, 0, length, length, count)
        assert np.array_equal(s[:60], s0.astype(np.int64)) and np.array_equal(f[:60], f0.astype(np.int64))
    bnd = (rng.random(60) < 0.1).astype(np.uint8)
    sb, fb = seqops.sliced_scores(hist, bnd, 20000)
    s, f = seqops.bounded_state_scores(hist, 20000, 0, 1, 0, 60, 60, 1, boundary=bnd)
    assert np.array_equal(s, sb.astype(np.int64)) and np.array_equal(f, fb.astype(np.int64))


def test_bounded_state_runs_agree_with_serial_where_the_state_restarts():
    # Shot-like histograms: the state of a run equals the serial state from a slice start
    # on, so a run whose warmup reaches back to a slice start (or to element 0) gives the
    # serial outputs; with shift > 0 and no restart in reach they may differ.
    rng = np.random.default_rng(13)
    n = 90
    base = rng.integers(0, 400, (6, 48))
    shot = np.repeat(np.arange(6), 15)
    hist = (base[shot] + rng.integers(0, 60, (n, 48))).astype(np.int64)
    bnd = np.zeros(n, np.uint8)
    bnd[::15] = 1
    serial, sflag = seqops.bounded_state_scores(hist, 30000, 2, 0, 0, n, n, 1, boundary=bnd)
    for length, warmup in [(5, 15), (10, 14), (7, 20), (1, 15)]:
        count = -(-n // length)
        s, f = seqops.bounded_state_scores(hist, 30000, 2, warmup, 0, length, length, count, boundary=bnd)
        assert np.array_equal(s[:n], serial) and np.array_equal(f[:n], sflag)
    # no slice starts: warmup that reaches element 0 reproduces the serial run
    serial, _ = seqops.bounded_state_scores(hist, 30000, 2, 0, 0, n, n, 1)
    s, _ = seqops.bounded_state_scores(hist, 30000, 2, n, 0, 10, 10, 9)
    assert np.array_equal(s, serial)
    short, _ = seqops.bounded_state_scores(hist, 30000, 2, 1, 0, 10, 10, 9)
    assert not np.array_equal(short, serial)
