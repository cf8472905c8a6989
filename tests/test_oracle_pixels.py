"""Pins for the oracle's BT.601 conversion, histogram, shot score, resize and thumbnails.

Each pin comes from outside the oracle: the standard colour bars, the
BT.601 matrix re-derived in floating point from Kr/Kb, brute force over tiny
frames, mass and L1 invariants, and the library bilinear interpolation.
"""
import os

import numpy as np
import pytest
import torch

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _bt601_float(Y, U, V):
    # BT.601: Kr = 0.299, Kb = 0.114; limited range 219 luma / 224 chroma levels.
    Kr, Kb = 0.299, 0.114
    Kg = 1 - Kr - Kb
    yl = (Y - 16) * 255.0 / 219.0
    cb = (U - 128) * 255.0 / 224.0
    cr = (V - 128) * 255.0 / 224.0
    R = yl + 2 * (1 - Kr) * cr
    G = yl - 2 * (1 - Kb) * Kb / Kg * cb - 2 * (1 - Kr) * Kr / Kg * cr
    B = yl + 2 * (1 - Kb) * cb
    return [np.clip(np.round(c), 0, 255) for c in (R, G, B)]


def test_colour_bars(orc):
    for ln in open(os.path.join(GOLDEN, "bt601_colour_bars.txt")):
        if not ln.strip() or ln.startswith("#"):
            continue
        name, *vals = ln.split()
        Y, U, V, R, G, B = map(int, vals)
        got = orc.yuv_to_rgb(Y, U, V)
        for g, e in zip(got, (R, G, B)):
            assert abs(g - e) <= 2, (name, got)


def test_black_white_exact(orc):
    assert orc.yuv_to_rgb(16, 128, 128) == (0, 0, 0)
    assert orc.yuv_to_rgb(235, 128, 128) == (255, 255, 255)


def test_conversion_within_one_level_of_float_matrix_exhaustive(orc):
    # every (Y, U, V) byte triple, one U value at a time
    Y, V = np.meshgrid(np.arange(256), np.arange(256), indexing="ij")
    Y, V = Y.ravel(), V.ravel()
    worst = 0
    for U in range(256):
        yuv = np.stack([Y, np.full_like(Y, U), V], axis=1).astype(np.uint8)
        got = orc.yuv_to_rgb_array(yuv).astype(np.int64)
        ref = _bt601_float(Y.astype(float), float(U), V.astype(float))
        for c in range(3):
            worst = max(worst, int(np.abs(got[:, c] - ref[c]).max()))
    assert worst <= 1


def _bt601_fixed_point_coefficients():
    """The five x256 integer coefficients of 8-bit BT.601 limited-range YCbCr -> RGB,
    derived from the standard's luma weights Kr = 0.299, Kb = 0.114 and the 219-level
    luma / 224-level chroma excursions: round(256 * matrix entry)."""
    Kr, Kb = 0.299, 0.114
    Kg = 1 - Kr - Kb
    sy, sc = 255.0 / 219.0, 255.0 / 224.0
    entries = {
        "Y": sy,                                # R, G, B from luma
        "R_Cr": 2 * (1 - Kr) * sc,               # R from Cr
        "G_Cb": 2 * (1 - Kb) * Kb / Kg * sc,     # G from Cb (subtracted)
        "G_Cr": 2 * (1 - Kr) * Kr / Kg * sc,     # G from Cr (subtracted)
        "B_Cb": 2 * (1 - Kb) * sc,               # B from Cb
    }
    return {k: int(np.floor(256 * v + 0.5)) for k, v in entries.items()}


def test_fixed_point_coefficients_from_kr_kb():
    c = _bt601_fixed_point_coefficients()
    # the values that every integer BT.601 implementation with x256 scaling uses
    assert c == {"Y": 298, "R_Cr": 409, "G_Cb": 100, "G_Cr": 208, "B_Cb": 516}


def test_conversion_exact_against_derived_fixed_point_exhaustive(orc):
    """Every (Y, U, V) byte triple: the oracle equals the fixed-point form built from
    the coefficients derived above, C = Y-16, D = U-128, E = V-128,
    value = clamp((coef . (C, D, E) + 128) >> 8, 0, 255) with an arithmetic shift."""
    c = _bt601_fixed_point_coefficients()
    Y, V = np.meshgrid(np.arange(256, dtype=np.int64), np.arange(256, dtype=np.int64), indexing="ij")
    Y, V = Y.ravel(), V.ravel()
    C, E = Y - 16, V - 128
    for U in range(256):
        D = U - 128
        yuv = np.stack([Y, np.full_like(Y, U), V], axis=1).astype(np.uint8)
        got = orc.yuv_to_rgb_array(yuv).astype(np.int64)
        R = np.clip((c["Y"] * C + c["R_Cr"] * E + 128) >> 8, 0, 255)
        G = np.clip((c["Y"] * C - c["G_Cb"] * D - c["G_Cr"] * E + 128) >> 8, 0, 255)
        B = np.clip((c["Y"] * C + c["B_Cb"] * D + 128) >> 8, 0, 255)
        assert np.array_equal(got[:, 0], R), U
        assert np.array_equal(got[:, 1], G), U
        assert np.array_equal(got[:, 2], B), U


def test_hist_identity_clamp_shift():
    # the kernel folds clamp(x >> 8, 0, 255) >> 4 into clamp(x >> 12, 0, 15)
    x = np.arange(-(1 << 20), 1 << 20, dtype=np.int64)
    a = np.clip(x >> 8, 0, 255) >> 4
    b = np.clip(x >> 12, 0, 15)
    assert np.array_equal(a, b)


def _brute_hist(orc, frame, W, H):
    h = np.zeros((3, 16), dtype=np.int64)
    for y in range(H):
        for x in range(W):
            Y = int(frame[y * W + x])
            U = int(frame[W * H + (y // 2) * W + 2 * (x // 2)])
            V = int(frame[W * H + (y // 2) * W + 2 * (x // 2) + 1])
            rgb = orc.yuv_to_rgb(Y, U, V)
            for c in range(3):
                h[c, rgb[c] // 16] += 1
    return h


@pytest.mark.parametrize("W,H", [(2, 2), (4, 2), (16, 8), (6, 4)])
def test_hist_brute_force_random_bytes(orc, W, H):
    rng = np.random.default_rng(W * 100 + H)
    for _ in range(5):
        fr = rng.integers(0, 256, W * H * 3 // 2, dtype=np.uint8)
        assert np.array_equal(orc.hist_frame(fr, W, H), _brute_hist(orc, fr, W, H))


def test_hist_mass_and_constant(orc):
    W, H = 320, 180
    v = orc.Video(20180805, 0, W, H, 240, num_shots=8)
    for f in (0, 77, 239):
        h = orc.hist_frame(v.frame(f), W, H)
        assert np.all(h.sum(axis=1) == W * H)
    fr = np.empty(W * H * 3 // 2, dtype=np.uint8)
    fr[: W * H] = 100
    fr[W * H:: 2] = 60
    fr[W * H + 1:: 2] = 200
    h = orc.hist_frame(fr, W, H)
    rgb = orc.yuv_to_rgb(100, 60, 200)
    for c in range(3):
        assert h[c, rgb[c] // 16] == W * H and np.count_nonzero(h[c]) == 1


def test_scores_invariants(orc):
    W, H = 32, 16
    P = W * H
    base = np.zeros((3, 16), dtype=np.uint32)
    base[:, 5] = P
    moved = base.copy()
    moved[1, 5] = 0
    moved[1, 9] = P
    half = base.copy()
    half[2, 5] = P // 2
    half[2, 6] = P - P // 2
    hists = np.stack([base, base, moved, base, half, half])
    s, f = orc.scores(hists, P)
    assert s.tolist() == [0, 0, 2 * P, 2 * P, P, 0]
    # flag: 2*score > P, i.e. score > P/2
    assert f.tolist() == [0, 0, 1, 1, 1, 0]
    # a score of exactly P/2 is not a boundary, one more is
    q = base.copy()
    q[0, 5] = P - P // 4
    q[0, 6] = P // 4
    s2, f2 = orc.scores(np.stack([base, q]), P)
    assert s2.tolist() == [0, P // 2] and f2.tolist() == [0, 0]
    q[0, 5] -= 1
    q[0, 6] += 1
    s3, f3 = orc.scores(np.stack([base, q]), P)
    assert s3.tolist() == [0, P // 2 + 2] and f3.tolist() == [0, 1]
    # symmetry and the 6*W*H bound on random histograms of equal mass
    rng = np.random.default_rng(3)
    for _ in range(20):
        a = rng.multinomial(P, np.ones(16) / 16, size=3).astype(np.uint32)
        b = rng.multinomial(P, np.ones(16) / 16, size=3).astype(np.uint32)
        sab, _ = orc.scores(np.stack([a, b]), P)
        sba, _ = orc.scores(np.stack([b, a]), P)
        assert sab[1] == sba[1] <= 6 * P
        assert sab[1] == int(np.abs(a.astype(np.int64) - b).sum())


def test_constant_shot_scores_zero(orc):
    # a shot with no ramp drift and no noise: frames are identical -> scores 0
    W, H = 64, 36
    fr = np.full(W * H * 3 // 2, 128, dtype=np.uint8)
    fr[: W * H] = np.arange(W * H) % 200 + 16
    hs = np.stack([orc.hist_frame(fr, W, H)] * 5)
    s, f = orc.scores(hs, W * H)
    assert s.tolist() == [0] * 5 and f.tolist() == [0] * 5


def _rgb_planes(orc, fr, W, H):
    Yp = fr[: W * H].reshape(H, W)
    uv = fr[W * H:].reshape(H // 2, W)
    U = np.repeat(np.repeat(uv[:, 0::2], 2, axis=0), 2, axis=1)
    V = np.repeat(np.repeat(uv[:, 1::2], 2, axis=0), 2, axis=1)
    yuv = np.stack([Yp.ravel(), U.ravel(), V.ravel()], axis=1)
    return orc.yuv_to_rgb_array(yuv).reshape(H, W, 3).transpose(2, 0, 1).astype(np.float64)


@pytest.mark.parametrize("W,H,oh,ow", [(320, 180, 224, 224), (64, 36, 224, 224), (1920, 1080, 224, 224),
                                       (640, 360, 17, 31), (16, 8, 3, 5)])
def test_resize_matches_library_bilinear(orc, W, H, oh, ow):
    rng = np.random.default_rng(W + H)
    fr = rng.integers(0, 256, W * H * 3 // 2, dtype=np.uint8)
    mean, std = (0.485, 0.456, 0.406), (0.229, 0.224, 0.225)
    got = orc.resize_norm_frame(fr, W, H, oh, ow, mean, std)
    rgb = torch.from_numpy(_rgb_planes(orc, fr, W, H))[None]
    ref = torch.nn.functional.interpolate(rgb, size=(oh, ow), mode="bilinear", align_corners=False,
                                          antialias=False)[0].numpy()
    ref = (ref / 255.0 - np.array(mean)[:, None, None]) / np.array(std)[:, None, None]
    assert np.abs(got - ref).max() < 1e-12


def test_resize_constant_image_exact(orc):
    W, H = 320, 180
    fr = np.empty(W * H * 3 // 2, dtype=np.uint8)
    fr[: W * H] = 90
    fr[W * H:: 2] = 140
    fr[W * H + 1:: 2] = 100
    rgb = orc.yuv_to_rgb(90, 140, 100)
    mean, std = (0.5, 0.25, 0.125), (0.5, 2.0, 0.25)
    got = orc.resize_norm_frame(fr, W, H, 224, 224, mean, std)
    for c in range(3):
        assert np.all(got[c] == (rgb[c] / 255.0 - mean[c]) / std[c])


def test_thumbnails(orc):
    for W, H in [(320, 180), (640, 360), (1920, 1080)]:
        rng = np.random.default_rng(W)
        fr = rng.integers(0, 256, W * H * 3 // 2, dtype=np.uint8)
        t = orc.thumb_frame(fr, W, H)
        s = W // 64
        assert s == H // 36
        Yp = fr[: W * H].reshape(H, W)
        assert np.array_equal(t, Yp[0: 36 * s: s, 0: 64 * s: s])


def test_coarse_yuv_thumbnails(orc):
    # Y at luma pixel (2 s c, 6 s r), U and V of the chroma sample (s c, 3 s r) that pixel uses
    for W, H in [(320, 180), (640, 360), (1920, 1080)]:
        rng = np.random.default_rng(W + 1)
        fr = rng.integers(0, 256, W * H * 3 // 2, dtype=np.uint8)
        yuv = orc.thumb_yuv_frame(fr, W, H)
        s = W // 64
        Yp = fr[: W * H].reshape(H, W)
        Up = fr[W * H:].reshape(H // 2, W)[:, 0::2]
        Vp = fr[W * H:].reshape(H // 2, W)[:, 1::2]
        assert np.array_equal(yuv[0], Yp[0: 36 * s: 6 * s, 0: 64 * s: 2 * s])
        assert np.array_equal(yuv[0], orc.thumb_frame(fr, W, H)[0::6, 0::2])
        assert np.array_equal(yuv[1], Up[0: 18 * s: 3 * s, 0: 32 * s: s])
        assert np.array_equal(yuv[2], Vp[0: 18 * s: 3 * s, 0: 32 * s: s])
        # and it is the chroma that the conversion uses at those luma pixels
        for r, c in [(0, 0), (5, 31), (3, 9)]:
            y, x = 6 * s * r, 2 * s * c
            assert yuv[1, r, c] == fr[W * H + (y >> 1) * W + 2 * (x >> 1)]
            assert yuv[2, r, c] == fr[W * H + (y >> 1) * W + 2 * (x >> 1) + 1]


def test_thumb_diff_hand_values(orc):
    a = np.zeros((36, 64), dtype=np.uint8)
    b = a.copy()
    b[0, :32] = 10          # 32 samples differ by 10: 320 / 2304
    b[35, 63] = 255         # and one by 255
    assert orc.thumb_diff(a, b) == (320 + 255) / 2304
    assert orc.thumb_diff(b, a) == orc.thumb_diff(a, b) and orc.thumb_diff(a, a) == 0.0
    ya = np.full((3, 6, 32), 128, dtype=np.uint8)
    yb = ya.copy()
    yb[0, 0, :] = 152       # 32 Y samples +24: 768 / 192 = 4
    yb[1] = 160             # every U sample +32: mean 32
    yb[2, :3] = 100         # half the V samples -28: mean 14
    assert orc.thumb_diff_yuv(ya, yb) == 4.0 + 32.0 + 14.0
    assert orc.thumb_diff_yuv(yb, ya) == orc.thumb_diff_yuv(ya, yb) and orc.thumb_diff_yuv(ya, ya) == 0.0
