"""Spacing, slicing, sliced scores and the per-shot montage on the GPU against
the oracle's definitions (bit-exact)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import seqops  # noqa: E402
from paper_1805_07339_b300.workloads import MASTER_SEED, TINY  # noqa: E402


@pytest.fixture(scope="module")
def scn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_07339_b300 import scn as s
    return s


@pytest.fixture(scope="module")
def tiny(scn, orc):
    W, H, T, S = TINY["width"], TINY["height"], TINY["num_frames"], TINY["num_shots"]
    fb = W * H * 3 // 2
    v = scn.scn_video_create(MASTER_SEED, 0, W, H, T, S)
    buf = torch.empty(T * fb, dtype=torch.uint8, device="cuda")
    scn.scn_generate(v, buf, 0, T, fb)
    t = scn.scn_table_create(buf, W, H, T)
    frames = orc.Video(MASTER_SEED, 0, W, H, T, S).frames(range(T), nthreads=8)
    yield dict(scn=scn, buf=buf, table=t, W=W, H=H, T=T, frames=frames)
    scn.scn_table_destroy(t)
    scn.scn_video_destroy(v)


def _hs(scn, seq, n):
    h = torch.empty((n, 48), dtype=torch.int32, device="cuda")
    s = torch.empty(n, dtype=torch.int32, device="cuda")
    f = torch.empty(n, dtype=torch.uint8, device="cuda")
    scn.scn_hist_scores(seq, h, s, f)
    return h, s, f


@pytest.mark.parametrize("kind", ["stride", "gather"])
def test_space_matches_oracle(tiny, kind):
    scn, T = tiny["scn"], tiny["T"]
    if kind == "stride":
        idx = np.arange(3, T, 24)
        seq = scn.scn_sample(tiny["table"], scn.SCN_STRIDE, 3, T, 24)
    else:  # unsorted, with repeats
        rng = np.random.default_rng(7)
        idx = rng.integers(0, T, 57)
        seq = scn.scn_sample(tiny["table"], scn.SCN_GATHER, indices=idx.tolist())
    try:
        n = len(idx)
        h, s, f = _hs(scn, seq, n)
        for vals, eb, fill in ((h, 192, bytes(range(192))), (s, 4, b"\xff\xff\xff\x7f"), (f, 1, b"\x07")):
            for mode in (scn.SCN_FILL_VALUE, scn.SCN_FILL_REPEAT):
                out = torch.empty((T,) + tuple(vals.shape[1:]), dtype=vals.dtype, device="cuda")
                scn.scn_space(seq, vals, eb, out, fill_mode=mode, fill=fill)
                fill_v = np.frombuffer(fill, dtype=vals.cpu().numpy().dtype).reshape(vals.shape[1:])
                ref = seqops.space(vals.cpu().numpy(), idx, T, repeat=mode == scn.SCN_FILL_REPEAT, fill=fill_v)
                assert np.array_equal(out.cpu().numpy(), ref), (eb, mode)
        # no fill given: zero bytes
        out = torch.full((T,), -1, dtype=torch.int32, device="cuda")
        scn.scn_space(seq, s, 4, out)
        assert np.array_equal(out.cpu().numpy(), seqops.space(s.cpu().numpy(), idx, T))
    finally:
        scn.scn_seq_destroy(seq)


@pytest.mark.parametrize("n", [0, 1, 2, 1000, 8193, 1_300_000])
def test_slice_matches_oracle(scn, n):
    rng = np.random.default_rng(n)
    flags = (rng.random(n) < 0.01).astype(np.uint8)
    d_flags = torch.from_numpy(flags).cuda()
    starts = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    count = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    scn.scn_slice(d_flags, n, starts, count)
    m = int(count.item())
    ref = np.flatnonzero(np.concatenate([[1], flags[1:]])) if n else np.zeros(0, np.int64)
    if n <= 8193:
        assert np.array_equal(ref, seqops.slice_starts(flags))
    assert m == len(ref) and np.array_equal(starts.cpu().numpy()[:m], ref)
    if n:
        mids = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        scn.scn_slice_middles(starts, count, n, mids)
        assert np.array_equal(mids.cpu().numpy()[:m], seqops.slice_middles(ref, n))
        assert np.all(mids.cpu().numpy()[m:] == -1)  # nothing written past the slices


def test_sliced_scores_match_oracle(scn):
    rng = np.random.default_rng(9)
    n, px = 3001, 320 * 180
    hist = rng.integers(0, 4000, (n, 48)).astype(np.uint32)
    b = (rng.random(n) < 0.05).astype(np.uint8)
    s = torch.empty(n, dtype=torch.int32, device="cuda")
    f = torch.empty(n, dtype=torch.uint8, device="cuda")
    scn.scn_shot_scores_sliced(torch.from_numpy(hist.view(np.int32)).cuda(), n, px, torch.from_numpy(b).cuda(), s, f)
    rs, rf = seqops.sliced_scores(hist, b, px)
    assert np.array_equal(s.cpu().numpy().view(np.uint32), rs) and np.array_equal(f.cpu().numpy(), rf)


def test_shot_montage_pipeline(tiny, orc):
    """Detect shots, slice at them, take each slice's middle frame, lay the frames out as a montage."""
    scn, W, H, T = tiny["scn"], tiny["W"], tiny["H"], tiny["T"]
    seq = scn.scn_sample(tiny["table"], scn.SCN_STRIDE, 0, T, 1)
    try:
        _, _, f = _hs(scn, seq, T)
        starts = torch.empty(T, dtype=torch.int32, device="cuda")
        count = torch.empty(1, dtype=torch.int64, device="cuda")
        scn.scn_slice(f, T, starts, count)
        mids = torch.empty(T, dtype=torch.int32, device="cuda")
        scn.scn_slice_middles(starts, count, T, mids)
        m = int(count.item())
        cols, tw, th = 4, 80, 45
        rows = (m + cols - 1) // cols
        out = torch.empty((rows * th, cols * tw, 3), dtype=torch.uint8, device="cuda")
        scn.scn_montage(seq, mids, m, cols, tw, th, out)
        # oracle pipeline on the oracle's own frames
        h = orc.hist_batch(tiny["frames"], W, H, nthreads=8)
        _, rf = orc.scores(h, W * H)
        rst = seqops.slice_starts(rf)
        rmid = seqops.slice_middles(rst, T)
        assert m == len(rst) and m >= 4
        ref = seqops.montage([tiny["frames"][k] for k in rmid], W, H, cols, tw, th)
        assert np.array_equal(out.cpu().numpy(), ref)
        # tiles whose element lies outside the sequence are black
        bad = torch.tensor([0, T, -1], dtype=torch.int32, device="cuda")
        out2 = torch.full((th, 3 * tw, 3), 9, dtype=torch.uint8, device="cuda")
        scn.scn_montage(seq, bad, 3, 3, tw, th, out2)
        o2 = out2.cpu().numpy()
        assert np.array_equal(o2[:, :tw], seqops.montage([tiny["frames"][0]], W, H, 1, tw, th))
        assert np.all(o2[:, tw:] == 0)
    finally:
        scn.scn_seq_destroy(seq)


def test_montage_random_bytes_and_odd_tiles(scn, orc):
    """Uniformly random NV12 (every clamp), tile sizes that do not divide the frame."""
    from paper_1805_07339_b300.workloads import random_nv12
    W, H = 64, 36
    fr = random_nv12(31, 5, W, H)
    buf = torch.from_numpy(fr.reshape(-1)).cuda()
    t = scn.scn_table_create(buf, W, H, 5)
    seq = scn.scn_sample(t, scn.SCN_STRIDE, 0, 5, 1)
    try:
        for tw, th, cols in ((64, 36, 2), (13, 7, 3), (100, 50, 5)):
            el = torch.tensor([4, 0, 2, 1, 3], dtype=torch.int32, device="cuda")
            rows = (5 + cols - 1) // cols
            out = torch.empty((rows * th, cols * tw, 3), dtype=torch.uint8, device="cuda")
            scn.scn_montage(seq, el, 5, cols, tw, th, out)
            ref = seqops.montage([fr[k] for k in (4, 0, 2, 1, 3)], W, H, cols, tw, th)
            assert np.array_equal(out.cpu().numpy(), ref), (tw, th)
    finally:
        scn.scn_seq_destroy(seq)
        scn.scn_table_destroy(t)


@pytest.mark.parametrize("a,b", [(-1, 0), (-2, 1), (-8, 3), (-64, 63)])
def test_window_scores_match_oracle(scn, a, b):
    rng = np.random.default_rng(-a * 100 + b)
    n, px = 1501, 320 * 180
    hist = rng.integers(0, 4000, (n, 48)).astype(np.uint32)
    bnd = (rng.random(n) < 0.03).astype(np.uint8)
    d_hist = torch.from_numpy(hist.view(np.int32)).cuda()
    for boundary in (None, bnd):
        s = torch.empty(n, dtype=torch.int64, device="cuda")
        f = torch.empty(n, dtype=torch.uint8, device="cuda")
        scn.scn_window_scores(d_hist, 0, n, n, a, b, px, 0, n, s, f,
                              boundary=None if boundary is None else torch.from_numpy(boundary).cuda())
        rs, rf = seqops.window_scores(hist, a, b, px, boundary=boundary)
        assert np.array_equal(s.cpu().numpy().view(np.uint64), rs) and np.array_equal(f.cpu().numpy(), rf)


def test_window_scores_plain_window_equals_shot_scores(tiny):
    scn, T, W, H = tiny["scn"], tiny["T"], tiny["W"], tiny["H"]
    seq = scn.scn_sample(tiny["table"], scn.SCN_STRIDE, 0, T, 1)
    try:
        h, s, f = _hs(scn, seq, T)
        ws = torch.empty(T, dtype=torch.int64, device="cuda")
        wf = torch.empty(T, dtype=torch.uint8, device="cuda")
        scn.scn_window_scores(h, 0, T, T, -1, 0, W * H, 0, T, ws, wf)
        assert np.array_equal(ws.cpu().numpy(), s.cpu().numpy().astype(np.int64))
        assert np.array_equal(wf.cpu().numpy(), f.cpu().numpy())
    finally:
        scn.scn_seq_destroy(seq)


def test_window_scores_sharded_with_halos(scn):
    """Shards that hold only their dependency range (outputs plus a -a / b element halo)
    give the unsharded result; a slice missing part of the range is refused."""
    from paper_1805_07339_b300 import stencil
    rng = np.random.default_rng(21)
    n, px, a, b = 2000, 640 * 360, -5, 3
    d_hist = torch.from_numpy(rng.integers(0, 9000, (n, 48)).astype(np.int32)).cuda()
    d_bnd = torch.from_numpy((rng.random(n) < 0.02).astype(np.uint8)).cuda()
    full_s = torch.empty(n, dtype=torch.int64, device="cuda")
    full_f = torch.empty(n, dtype=torch.uint8, device="cuda")
    scn.scn_window_scores(d_hist, 0, n, n, a, b, px, 0, n, full_s, full_f, boundary=d_bnd)
    for parts in (1, 3, 7, 64):
        s, f = stencil.window_scores_sharded(torch, d_hist, n, a, b, px, parts, boundary=d_bnd)
        assert torch.equal(s, full_s) and torch.equal(f, full_f), parts
    # outputs [100, 200) need elements [95, 203): a slice starting at 96 is one short
    s = torch.empty(100, dtype=torch.int64, device="cuda")
    f = torch.empty(100, dtype=torch.uint8, device="cuda")
    with pytest.raises(scn.ScnError):
        scn.scn_window_scores(d_hist[96:203].clone(), 96, 107, n, a, b, px, 100, 200, s, f)
    scn.scn_window_scores(d_hist[95:203].clone(), 95, 108, n, a, b, px, 100, 200, s, f,
                          boundary=d_bnd[95:203].clone())
    assert torch.equal(s, full_s[100:200]) and torch.equal(f, full_f[100:200])
    with pytest.raises(scn.ScnError):  # window wider than 64
        scn.scn_window_scores(d_hist, 0, n, n, -65, 0, px, 0, n, full_s, full_f)


def _shot_hists(rng, n, px):
    """Histograms with shot structure: per shot a random 16-bin distribution per channel,
    per frame a multinomial draw of px pixels from it (each channel sums to px)."""
    hist = np.empty((n, 48), np.int64)
    k = 0
    while k < n:
        L = min(n - k, int(rng.integers(3, 90)))
        for c in range(3):
            p = rng.dirichlet(np.full(16, 0.6))
            q = p * rng.uniform(0.85, 1.15, (L, 16))
            q /= q.sum(1, keepdims=True)
            hist[k:k + L, 16 * c:16 * c + 16] = [rng.multinomial(px, qq) for qq in q]
        k += L
    return hist


def _state_run(scn, d_hist, n, px, shift, warmup, pat, d_bnd=None, hist_first=0, hist_count=None):
    first, length, stride, runs = pat
    slots = runs * length
    s = torch.full((max(slots, 1),), -1, dtype=torch.int32, device="cuda")
    f = torch.full((max(slots, 1),), 255, dtype=torch.uint8, device="cuda")
    scn.scn_bounded_state_scores(d_hist, hist_first, n if hist_count is None else hist_count, n, px, shift, warmup,
                                 first, length, stride, runs, s, f, boundary=d_bnd)
    return s.cpu().numpy()[:slots].astype(np.int64) & 0xFFFFFFFF, f.cpu().numpy()[:slots]


@pytest.mark.parametrize("shift,warmup,pat", [
    (3, 0, (0, 1501, 1501, 1)),       # serial
    (3, 24, (0, 94, 94, 16)),         # shards, the last one ragged
    (2, 10, (0, 2, 2, 751)),          # 751 two-element shards
    (2, 24, (0, 1, 24, 63)),          # sparse: every 24th output
    (4, 3, (5, 7, 10, 150)),          # gaps between runs
    (0, 1, (0, 50, 50, 31)),          # shift 0: the plain score
    (30, 50, (11, 13, 13, 200)),      # runs past the end
])
@pytest.mark.parametrize("sliced", [False, True])
def test_bounded_state_scores_match_oracle(scn, shift, warmup, pat, sliced):
    rng = np.random.default_rng(shift * 1000 + warmup + 7 * sliced)
    n, px = 1501, 320 * 180
    hist = _shot_hists(rng, n, px)
    bnd = (rng.random(n) < 0.02).astype(np.uint8) if sliced else None
    d_hist = torch.from_numpy(hist.astype(np.int32)).cuda()
    d_bnd = torch.from_numpy(bnd).cuda() if sliced else None
    s, f = _state_run(scn, d_hist, n, px, shift, warmup, pat, d_bnd)
    rs, rf = seqops.bounded_state_scores(hist, px, shift, warmup, *pat, boundary=bnd)
    written = rs >= 0
    assert np.array_equal(s[written], rs[written]) and np.array_equal(f[written], rf[written])
    assert (s[~written] == 0xFFFFFFFF).all() and (f[~written] == 255).all()  # slots past n untouched
    if shift == 0:
        ps, pf = (seqops.sliced_scores(hist, bnd, px) if sliced else oracle_scores(hist, px))
        for r in range(pat[3]):
            k0 = pat[0] + r * pat[2]
            for k in range(k0, min(k0 + pat[1], n)):
                if k > 0 and (k > k0 or warmup > 0):
                    assert s[r * pat[1] + k - k0] == ps[k]


def oracle_scores(hist, px):
    import oracle
    return oracle.scores(hist.astype(np.uint32), px)


def test_bounded_state_scores_edges_and_resident_slices(scn):
    rng = np.random.default_rng(31)
    n, px = 400, 64 * 36
    hist = _shot_hists(rng, n, px)
    d_hist = torch.from_numpy(hist.astype(np.int32)).cuda()
    s0 = torch.zeros(4, dtype=torch.int32, device="cuda")
    f0 = torch.zeros(4, dtype=torch.uint8, device="cuda")
    # nothing to do: no runs, an empty sequence, runs that start past the end
    scn.scn_bounded_state_scores(d_hist, 0, n, n, px, 2, 5, 0, 4, 4, 0, s0, f0)
    scn.scn_bounded_state_scores(d_hist, 0, 0, 0, px, 2, 5, 0, 4, 4, 1, s0, f0)
    scn.scn_bounded_state_scores(d_hist, 0, n, n, px, 2, 5, n, 4, 4, 1, s0, f0)
    assert not s0.any()
    # one element: score 0, flag 0
    s, f = _state_run(scn, d_hist[:1].clone(), 1, px, 2, 5, (0, 1, 1, 1))
    assert s.tolist() == [0] and f.tolist() == [0]
    # outputs [100, 200) with warmup 8 need elements [92, 200): a resident slice from 92 works, from 93 not
    pat = (100, 100, 100, 1)
    rs, rf = seqops.bounded_state_scores(hist, px, 2, 8, *pat)
    s, f = _state_run(scn, d_hist[92:200].clone(), n, px, 2, 8, pat, hist_first=92, hist_count=108)
    assert np.array_equal(s, rs[:100]) and np.array_equal(f, rf[:100])
    with pytest.raises(scn.ScnError):
        _state_run(scn, d_hist[93:200].clone(), n, px, 2, 8, pat, hist_first=93, hist_count=107)
    with pytest.raises(scn.ScnError):
        _state_run(scn, d_hist[92:199].clone(), n, px, 2, 8, pat, hist_first=92, hist_count=107)
    for bad in [dict(shift=31), dict(shift=-1), dict(warmup=-1), dict(pat=(0, 0, 1, 1)), dict(pat=(0, 5, 4, 2)),
                dict(px=715827883)]:
        a = dict(shift=2, warmup=1, pat=(0, 10, 10, 1), px=px)
        a.update(bad)
        with pytest.raises(scn.ScnError):
            _state_run(scn, d_hist, n, a["px"], a["shift"], a["warmup"], a["pat"])


def test_bounded_state_scores_full_size_sharded(scn):
    """200,000 elements as 1,184 shards (8 per SM) with warmup 32, and the serial run: the
    serial run against the oracle in full, 40 sampled shards one by one; shards whose warmup
    reaches a slice start agree with the serial run."""
    from paper_1805_07339_b300 import stencil
    rng = np.random.default_rng(32)
    n, px = 200_000, 640 * 360
    hist = _shot_hists(rng, n, px)
    bnd = np.zeros(n, np.uint8)
    bnd[rng.choice(n, 400, replace=False)] = 1
    d_hist = torch.from_numpy(hist.astype(np.int32)).cuda()
    d_bnd = torch.from_numpy(bnd).cuda()
    serial, sflag = _state_run(scn, d_hist, n, px, 3, 0, (0, n, n, 1), d_bnd)
    rs, rf = seqops.bounded_state_scores(hist, px, 3, 0, 0, n, n, 1, boundary=bnd)
    assert np.array_equal(serial, rs) and np.array_equal(sflag, rf)
    pat = stencil.state_shards(n, 1184)
    s, f = _state_run(scn, d_hist, n, px, 3, 32, pat, d_bnd)
    first, length, stride, runs = pat
    for r in rng.choice(runs, 40, replace=False):
        k0 = first + r * stride
        k1 = min(k0 + length, n)
        es, ef = seqops.bounded_state_run(hist, px, 3, max(0, k0 - 32), k0, k1, boundary=bnd)
        assert s[r * length:r * length + k1 - k0].tolist() == es and f[r * length:r * length + k1 - k0].tolist() == ef
    for r in range(runs):
        k0 = first + r * stride
        if k0 == 0 or bnd[max(0, k0 - 32):k0 + 1].any():
            k1 = min(k0 + length, n)
            assert np.array_equal(s[r * length:r * length + k1 - k0], serial[k0:k1])
