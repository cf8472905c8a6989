"""Pins for the oracle's synthetic-video generator (the stand-in for decoded frames).

The generator is the input side of every parity test, so it is pinned against
things other than itself: the published SplitMix64 outputs, the exact
Irwin-Hall distribution of the noise term, hand evaluation of single pixels,
and the structural rules of the shot table.
"""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
M64 = 2**64 - 1


def test_splitmix64_published_vectors(orc):
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "splitmix64_seed0.txt"))
            if ln.strip() and not ln.startswith("#")]
    for idx, hexval in rows:
        assert orc.sm(0, int(idx)) == int(hexval, 16)


def _mix(z):
    z ^= z >> 30
    z = (z * 0xBF58476D1CE4E5B9) & M64
    z ^= z >> 27
    z = (z * 0x94D049BB133111EB) & M64
    z ^= z >> 31
    return z


def _sm(s, i):
    return _mix((s + (i + 1) * 0x9E3779B97F4A7C15) & M64)


def test_noise_exact_irwin_hall_pmf(orc):
    # S = sum of 12 independent uniform bytes; noise = floor((S - 1514) / 32).
    pmf_s = np.ones(256) / 256.0
    one = np.ones(256) / 256.0
    for _ in range(11):
        pmf_s = np.convolve(pmf_s, one)
    S = np.arange(len(pmf_s))
    nvals = np.floor((S - 1514) / 32.0).astype(int)
    expect = {}
    for v, p in zip(nvals, pmf_s):
        expect[v] = expect.get(v, 0.0) + p
    seed = _sm(20180805, 7)
    N = 400_000
    samples = np.array([orc.noise(seed, q) for q in range(N)])
    assert samples.min() >= -48 and samples.max() <= 48
    assert abs(samples.mean()) < 0.05
    assert 7.9 <= samples.std() <= 8.1
    # chi-square over well-populated cells
    vals, counts = np.unique(samples, return_counts=True)
    chi2, dof = 0.0, 0
    for v, c in zip(vals, counts):
        e = expect.get(int(v), 0.0) * N
        if e >= 20:
            chi2 += (c - e) ** 2 / e
            dof += 1
    assert dof > 30
    assert chi2 < dof + 6 * np.sqrt(2 * dof)


def test_noise_hand_evaluated(orc):
    for s_pix, q in [(12345, 0), (_sm(1, 2), 987654321), (M64, 2**40 + 3)]:
        w0, w1 = _sm(s_pix, 2 * q), _sm(s_pix, 2 * q + 1)
        S = sum((w0 >> (8 * b)) & 255 for b in range(8)) + sum((w1 >> (8 * b)) & 255 for b in range(4))
        assert orc.noise(s_pix, q) == (S - 1530 + 16) // 32


def test_pixels_hand_evaluated(orc):
    seed, vid, W, H, T = 20180805, 3, 64, 36, 12
    v = orc.Video(seed, vid, W, H, T, num_shots=3)
    shots = v.shots()
    s_v = _sm(seed, vid)
    s_pix = _sm(s_v, 2)
    for f in (0, 5, 11):
        fr = v.frame(f)
        sh = [s for s in shots if s["start"] <= f][-1]
        dt = f - sh["start"]
        for (pl, xp, yp) in [(0, 0, 0), (0, 63, 35), (0, 17, 9), (1, 0, 0), (1, 31, 17), (2, 5, 11)]:
            Wp, Hp = (W, H) if pl == 0 else (W // 2, H // 2)
            x, y = (xp, yp) if pl == 0 else (2 * xp, 2 * yp)
            q = ((f * 3 + pl) * Hp + yp) * Wp + xp
            w0, w1 = _sm(s_pix, 2 * q), _sm(s_pix, 2 * q + 1)
            S = sum((w0 >> (8 * b)) & 255 for b in range(8)) + sum((w1 >> (8 * b)) & 255 for b in range(4))
            n = (S - 1514) // 32
            val = sh["base"][pl] + (sh["gx"][pl] * (x - dt)) // W + (sh["gy"][pl] * y) // H + n
            val = min(max(val, 16), 235 if pl == 0 else 240)
            if pl == 0:
                got = fr[yp * W + xp]
            else:
                got = fr[W * H + yp * W + 2 * xp + (pl - 1)]
            assert got == val, (f, pl, xp, yp)


def test_shot_table_uniform(orc):
    T, S = 7200, 60
    v = orc.Video(20180805, 0, 1920, 1080, T, num_shots=S)
    st = v.shot_starts()
    assert len(st) == S and st[0] == 0
    assert np.all(np.diff(st) > 0) and st[-1] <= T - 1
    # boundaries are the first S-1 distinct draws 1 + SM(s_shot, j) mod (T-1)
    s_shot = _sm(_sm(20180805, 0), 1)
    seen, j = [], 0
    while len(seen) < S - 1:
        b = 1 + _sm(s_shot, j) % (T - 1)
        j += 1
        if b not in seen:
            seen.append(b)
    assert list(st[1:]) == sorted(seen)
    shots = v.shots()
    for a, b in zip(shots, shots[1:]):
        dy = abs(a["base"][0] - b["base"][0])
        duv = abs(a["base"][1] - b["base"][1]) + abs(a["base"][2] - b["base"][2])
        assert not (dy < 48 and duv < 64)
    for s in shots:
        assert 16 <= s["base"][0] <= 235 and 16 <= s["base"][1] <= 240 and 16 <= s["base"][2] <= 240
        assert all(-32 <= g <= 32 for g in s["gx"] + s["gy"])


def test_shot_table_geometric(orc):
    T = 54000
    v = orc.Video(20180805, 11, 640, 360, T, shot_mode=1)
    st = v.shot_starts()
    L = np.diff(np.append(st, T))
    assert st[0] == 0 and np.all(L[:-1] >= 2) and np.all(L <= 300)
    # p = 1/64 geometric failures + 2, capped at 300: mean close to 2 + 63
    assert 55 < L[:-1].mean() < 75


def test_keyframes_rule(orc):
    v = orc.Video(20180805, 0, 320, 180, 240, num_shots=8)
    kf = v.keyframes()
    assert set(range(0, 240, 104)) <= set(kf.tolist())
    assert set(v.shot_starts().tolist()) <= set(kf.tolist())
    assert np.all(np.diff(kf) > 0)


def test_frame_statistics(orc):
    v = orc.Video(20180805, 0, 320, 180, 240, num_shots=8)
    shots = v.shots()
    W, H = 320, 180
    for f in (0, 100, 239):
        fr = v.frame(f)
        sh = [s for s in shots if s["start"] <= f][-1]
        y = fr[: W * H].astype(float)
        assert y.min() >= 16 and y.max() <= 235
        uv = fr[W * H:].reshape(H // 2, W)
        assert uv.min() >= 16 and uv.max() <= 240
        # with no clamping in play the plane mean is base + mean ramp
        if 60 <= sh["base"][0] <= 190:
            assert abs(y.mean() - sh["base"][0]) < 18


def test_frames_threaded_equal_serial(orc):
    v = orc.Video(5, 1, 320, 180, 40, num_shots=4)
    a = v.frames(range(40), nthreads=1)
    b = v.frames(range(40), nthreads=4)
    assert np.array_equal(a, b)
    assert np.array_equal(a[7], v.frame(7))
