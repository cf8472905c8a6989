"""GPU parity: libscn's kernels against the CPU oracle, through the C ABI.

Integer outputs (generator bytes, histograms, scores, flags, thumbnails) must be
bit-exact.  The FP32 resize must be within 1e-4 abs of the fp64 oracle; the BF16
resize must equal round-to-nearest-even of the kernel's own FP32 value and lie
within one BF16 ulp (plus the FP32 tolerance) of the fp64 oracle rounded to BF16.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from tests.inputs import HD, MASTER_SEED, TINY, hd_gather, random_indices, random_nv12  # noqa: E402

RESIZE_TOL = 1e-4
MEAN, STD = (0.485, 0.456, 0.406), (0.229, 0.224, 0.225)


@pytest.fixture(scope="module")
def scn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_07339_b300 import scn as s
    return s


class Dev:
    """A device-resident table over a uint8 CUDA tensor of frames."""

    def __init__(self, scn, frames_u8, W, H, T, rows=None, keyframes=None):
        self.scn, self.W, self.H, self.T = scn, W, H, T
        self.buf = frames_u8
        self.fb = W * H * 3 // 2
        self.table = scn.scn_table_create(self.buf, W, H, T, rows=rows, keyframes=keyframes)

    def seq(self, kind, **kw):
        return self.scn.scn_sample(self.table, kind, **kw)

    def hist_scores(self, seq, tune=None):
        scn = self.scn
        n = scn.scn_seq_length(seq)
        if tune:
            scn.scn_seq_set_tune(seq, **tune)
        h = torch.full((max(n, 1), 48), 0xDEAD, dtype=torch.int32, device="cuda")
        s = torch.full((max(n, 1),), 0xBEEF, dtype=torch.int32, device="cuda")
        f = torch.full((max(n, 1),), 7, dtype=torch.uint8, device="cuda")
        scn.scn_hist_scores(seq, h, s, f)
        assert scn.scn_seq_sync_status(seq) == scn.SCN_OK
        return (h[:n].cpu().numpy().view(np.uint32).reshape(n, 3, 16), s[:n].cpu().numpy().view(np.uint32),
                f[:n].cpu().numpy())

    def close(self):
        self.scn.scn_table_destroy(self.table)


def _video(scn, cfg, vid=0):
    return scn.scn_video_create(MASTER_SEED, vid, cfg["width"], cfg["height"], cfg["num_frames"], cfg["num_shots"])


def _generate(scn, v, W, H, T):
    fb = W * H * 3 // 2
    buf = torch.empty(T * fb, dtype=torch.uint8, device="cuda")
    scn.scn_generate(v, buf, 0, T, fb)
    torch.cuda.synchronize()
    return buf


# --------------------------------------------------------------------------- generator
def test_generator_bytes_tiny_all_frames(scn, orc):
    W, H, T = TINY["width"], TINY["height"], TINY["num_frames"]
    v = _video(scn, TINY)
    try:
        buf = _generate(scn, v, W, H, T)
        ref = orc.Video(MASTER_SEED, 0, W, H, T, TINY["num_shots"]).frames(range(T), nthreads=8)
        got = buf.cpu().numpy().reshape(T, -1)
        assert np.array_equal(got, ref)
    finally:
        scn.scn_video_destroy(v)


def test_generator_sparse_frames_hd_and_geometric(scn, orc):
    cases = [(HD, 0, 1), (dict(width=640, height=360, num_frames=54000, num_shots=0), 5, 1)]
    for cfg, vid, mode in cases:
        W, H, T = cfg["width"], cfg["height"], cfg["num_frames"]
        if cfg["num_shots"] == 0:
            v = scn.scn_video_create(MASTER_SEED, vid, W, H, T, 0, 1)
            oref = orc.Video(MASTER_SEED, vid, W, H, T, 0, 1)
        else:
            v = scn.scn_video_create(MASTER_SEED, vid, W, H, T, cfg["num_shots"])
            oref = orc.Video(MASTER_SEED, vid, W, H, T, cfg["num_shots"])
        try:
            frames = np.array([0, 1, T // 3, T // 2 + 1, T - 2, T - 1], dtype=np.int64)
            fb = W * H * 3 // 2
            out = torch.empty(len(frames) * fb, dtype=torch.uint8, device="cuda")
            scn.scn_generate_frames(v, torch.from_numpy(frames).cuda(), out, fb)
            got = out.cpu().numpy().reshape(len(frames), fb)
            assert np.array_equal(got, oref.frames(frames, nthreads=6))
        finally:
            scn.scn_video_destroy(v)


# --------------------------------------------------------------------------- hist + scores
def _oracle_hs(orc, frames_np, W, H, idx):
    h = orc.hist_batch(frames_np, W, H, idx=idx, nthreads=8)
    s, f = orc.scores(h, W * H)
    return h, s, f


def test_hist_scores_tiny_stride1_bit_exact(scn, orc):
    W, H, T = TINY["width"], TINY["height"], TINY["num_frames"]
    v = _video(scn, TINY)
    ref_frames = orc.Video(MASTER_SEED, 0, W, H, T, TINY["num_shots"]).frames(range(T), nthreads=8)
    dev = Dev(scn, _generate(scn, v, W, H, T), W, H, T)
    try:
        seq = dev.seq(scn.SCN_STRIDE, start=0, stop=T, step=1)
        h, s, f = dev.hist_scores(seq)
        rh, rs, rf = _oracle_hs(orc, ref_frames, W, H, np.arange(T))
        assert np.array_equal(h, rh)
        assert np.array_equal(s, rs)
        assert np.array_equal(f, rf)
        assert f.sum() >= 1  # the generator's shots are visible
        # hist-only entry point and the standalone score kernel agree
        h2 = torch.zeros((T, 48), dtype=torch.int32, device="cuda")
        scn.scn_hist(seq, h2)
        s2 = torch.zeros(T, dtype=torch.int32, device="cuda")
        f2 = torch.zeros(T, dtype=torch.uint8, device="cuda")
        scn.scn_shot_scores(h2, T, W * H, s2, f2)
        assert np.array_equal(h2.cpu().numpy().view(np.uint32).reshape(T, 3, 16), rh)
        assert np.array_equal(s2.cpu().numpy().view(np.uint32), rs)
        assert np.array_equal(f2.cpu().numpy(), rf)
        scn.scn_seq_destroy(seq)
    finally:
        dev.close()
        scn.scn_video_destroy(v)


@pytest.mark.parametrize("W,H,n", [(320, 180, 16), (1920, 1080, 3), (16, 2, 9), (48, 6, 5), (1936, 1090, 2),
                                   (3840, 2160, 2), (640, 360, 33)])
def test_hist_random_bytes_bit_exact(scn, orc, W, H, n):
    frames = random_nv12(W * 7 + H, n, W, H)
    buf = torch.from_numpy(frames.reshape(-1)).cuda()
    dev = Dev(scn, buf, W, H, n)
    try:
        order = random_indices(n, n, 2 * n, distinct=False)
        seq = dev.seq(scn.SCN_GATHER, indices=order.tolist())
        h, s, f = dev.hist_scores(seq)
        rh, rs, rf = _oracle_hs(orc, frames, W, H, order)
        assert np.array_equal(h, rh)
        assert np.array_equal(s, rs)
        assert np.array_equal(f, rf)
        scn.scn_seq_destroy(seq)
    finally:
        dev.close()


@pytest.mark.parametrize("W,H,n,grid", [(8192, 130, 6, 2), (1920, 1080, 5, 2), (2048, 1024, 9, 3), (1936, 1090, 4, 1),
                                        (4096, 2052, 3, 1)])
def test_split_tail_queue_bit_exact(scn, orc, W, H, n, grid):
    """Whole-frame queue items (frames above 1 Mpx) with the last `grid` frames queued in quarters
    (fewer when a frame has under four row pairs per part), on random bytes, with a gather order
    that repeats and jumps back: equal to the oracle; chunks of a few rows cut the tail items too."""
    frames = random_nv12(W + 3 * H, n, W, H)
    buf = torch.from_numpy(frames.reshape(-1)).cuda()
    dev = Dev(scn, buf, W, H, n)
    try:
        order = list(range(n)) + [0, n - 1, n - 1]
        rh, rs, rf = _oracle_hs(orc, frames, W, H, np.array(order))
        for chunk_rows in (0, 6):
            seq = dev.seq(scn.SCN_GATHER, indices=order)
            h, s, f = dev.hist_scores(seq, tune=dict(item_kpx=W * H // 1000 + 1, grid=grid, chunk_rows=chunk_rows))
            assert np.array_equal(h, rh) and np.array_equal(s, rs) and np.array_equal(f, rf), chunk_rows
            scn.scn_seq_destroy(seq)
    finally:
        dev.close()


@pytest.mark.parametrize("tune", [dict(grid=1), dict(grid=2), dict(grid=3, chunk_rows=6), dict(grid=7),
                                  dict(chunk_rows=2, grid=16), dict(grid=1000), dict(chunk_rows=4, grid=2),
                                  dict(chunk_rows=10)])
def test_hist_launch_shapes_agree(scn, orc, tune):
    W, H, n = 640, 360, 12
    frames = random_nv12(99, n, W, H)
    dev = Dev(scn, torch.from_numpy(frames.reshape(-1)).cuda(), W, H, n)
    try:
        seq = dev.seq(scn.SCN_RANGE, start=0, stop=n)
        h, s, f = dev.hist_scores(seq, tune=tune)
        rh, rs, rf = _oracle_hs(orc, frames, W, H, np.arange(n))
        assert np.array_equal(h, rh) and np.array_equal(s, rs) and np.array_equal(f, rf)
        # a second call on the same sequence (counters reset themselves)
        h2, s2, f2 = dev.hist_scores(seq)
        assert np.array_equal(h2, rh) and np.array_equal(s2, rs)
        scn.scn_seq_destroy(seq)
    finally:
        dev.close()


@pytest.mark.parametrize("W,H,n,tune", [
    (16, 2, 9, dict(item_kpx=1)),                       # 32-pixel frames, one item each
    (48, 6, 5, dict(item_kpx=1, chunk_rows=2)),
    (336, 200, 17, dict(item_kpx=20, chunk_rows=6)),    # frames split into items, items into chunks
    (640, 360, 40, dict(item_kpx=230)),                 # whole frames, more items than one CTA's regions
    (640, 360, 40, dict(item_kpx=50, grid=1)),          # one CTA: its five regions share the queue
    (640, 360, 40, dict(item_kpx=50, grid=3, chunk_rows=10)),
    (1280, 720, 7, dict(item_kpx=1000)),                # the largest frames counted by region streams
    (1280, 720, 7, dict(item_kpx=100, grid=2)),
])
def test_region_stream_kernel_bit_exact(scn, orc, W, H, n, tune):
    """Queue launches of frames up to 1 Mpx run the region-stream kernel (each
    4-warp table region counts whole items of its own): bit-exact against the
    oracle whatever the item, chunk and grid shapes, and again on a second call
    (the queue and the cross-CTA counters reset themselves)."""
    frames = random_nv12(W * 5 + H + n, n, W, H)
    dev = Dev(scn, torch.from_numpy(frames.reshape(-1)).cuda(), W, H, n)
    try:
        seq = dev.seq(scn.SCN_RANGE, start=0, stop=n)
        rh, rs, rf = _oracle_hs(orc, frames, W, H, np.arange(n))
        for _ in range(2):
            h, s, f = dev.hist_scores(seq, tune=tune)
            assert np.array_equal(h, rh) and np.array_equal(s, rs) and np.array_equal(f, rf)
        scn.scn_seq_destroy(seq)
    finally:
        dev.close()


def test_edge_cases(scn, orc):
    W, H, T = 64, 36, 6
    frames = random_nv12(5, T, W, H)
    dev = Dev(scn, torch.from_numpy(frames.reshape(-1)).cuda(), W, H, T, keyframes=[0, 4])
    try:
        empty = dev.seq(scn.SCN_STRIDE, start=3, stop=3, step=1)
        assert scn.scn_seq_length(empty) == 0
        h = torch.zeros(1, dtype=torch.int32, device="cuda")
        scn.scn_hist_scores(empty, h, h, torch.zeros(1, dtype=torch.uint8, device="cuda"))
        scn.scn_seq_destroy(empty)
        one = dev.seq(scn.SCN_GATHER, indices=[2])
        hh, s, f = dev.hist_scores(one)
        assert np.array_equal(hh, orc.hist_frame(frames[2], W, H)[None])
        assert s.tolist() == [0] and f.tolist() == [0]
        scn.scn_seq_destroy(one)
        dup = dev.seq(scn.SCN_GATHER, indices=[1, 1, 1, 5, 5])
        hh, s, f = dev.hist_scores(dup)
        assert s[1] == 0 and s[2] == 0 and s[4] == 0 and s[3] > 0
        scn.scn_seq_destroy(dup)
        kf = dev.seq(scn.SCN_KEYFRAME)
        hh, s, f = dev.hist_scores(kf)
        rh, rs, rf = _oracle_hs(orc, frames, W, H, np.array([0, 4]))
        assert np.array_equal(hh, rh) and np.array_equal(s, rs)
        scn.scn_seq_destroy(kf)
    finally:
        dev.close()


def test_sampling_invariance_and_sparse_table(scn, orc):
    # the same frame gives the same histogram whichever sampling reaches it, and
    # a table that stores only some rows (strided storage) gives the same answers
    W, H, T = 320, 180, 96
    v = scn.scn_video_create(MASTER_SEED, 3, W, H, T, 5)
    try:
        buf = _generate(scn, v, W, H, T)
        dev = Dev(scn, buf, W, H, T)
        s1 = dev.seq(scn.SCN_STRIDE, start=0, stop=T, step=1)
        s24 = dev.seq(scn.SCN_STRIDE, start=0, stop=T, step=24)
        g = dev.seq(scn.SCN_GATHER, indices=[72, 24, 48])
        h1, _, _ = dev.hist_scores(s1)
        h24, _, _ = dev.hist_scores(s24)
        hg, _, _ = dev.hist_scores(g)
        assert np.array_equal(h24, h1[0::24])
        assert np.array_equal(hg, h1[[72, 24, 48]])
        rows = list(range(0, T, 24))
        sparse = torch.empty(len(rows) * dev.fb, dtype=torch.uint8, device="cuda")
        scn.scn_generate_frames(v, torch.tensor(rows, dtype=torch.int64, device="cuda"), sparse, dev.fb)
        sdev = Dev(scn, sparse, W, H, T, rows=rows)
        ss = sdev.seq(scn.SCN_STRIDE, start=0, stop=T, step=24)
        hs, sc, fl = sdev.hist_scores(ss)
        assert np.array_equal(hs, h24)
        for q in (s1, s24, g, ss):
            scn.scn_seq_destroy(q)
        sdev.close()
        dev.close()
    finally:
        scn.scn_video_destroy(v)


@pytest.fixture(scope="module")
def hd_video(scn):
    """The full 1080p workload: 7200 frames (22.4 GB) generated on the device."""
    W, H, T = HD["width"], HD["height"], HD["num_frames"]
    v = _video(scn, HD)
    buf = _generate(scn, v, W, H, T)
    yield v, buf
    scn.scn_video_destroy(v)
    del buf
    torch.cuda.empty_cache()


def _oracle_hists(orc, ovid, frames, W, H, batch=48):
    """Oracle histograms of the given frame numbers (frames generated and
    histogrammed on the host in batches, so host memory stays small)."""
    import os
    nt = max(1, min(32, os.cpu_count() or 1))
    frames = np.asarray(frames, dtype=np.int64)
    out = np.empty((len(frames), 3, 16), dtype=np.uint32)
    for i in range(0, len(frames), batch):
        fr = ovid.frames(frames[i:i + batch], nthreads=nt)
        out[i:i + batch] = orc.hist_batch(fr, W, H, nthreads=nt)
    return out


def test_hd_full_size_parity(scn, orc, hd_video):
    """Full-size 1080p, the three sampling modes, default (bench) launch shape.
    Every element of the stride-24 (300) and gather (1000) sequences, and every
    24th element of the stride-1 sequence (with its predecessor for the score), is
    compared with the oracle; every element is also checked for histogram mass
    and for score consistency with its histograms."""
    v, buf = hd_video
    W, H, T = HD["width"], HD["height"], HD["num_frames"]
    dev = Dev(scn, buf, W, H, T)
    ovid = orc.Video(MASTER_SEED, 0, W, H, T, HD["num_shots"])
    gather = hd_gather()
    every24 = np.arange(24, T, 24)
    need = np.unique(np.concatenate([np.arange(0, T, 24), every24 - 1, gather]))
    rh_all = _oracle_hists(orc, ovid, need, W, H)
    ref = {int(f): rh_all[i] for i, f in enumerate(need)}
    try:
        for kind, kw, checked in [(scn.SCN_STRIDE, dict(start=0, stop=T, step=1), every24),
                                  (scn.SCN_STRIDE, dict(start=0, stop=T, step=24), None),
                                  (scn.SCN_GATHER, dict(indices=gather.tolist()), None)]:
            idx = np.array(scn.scn_sample_indices(dev.table, kind, **kw))
            seq = dev.seq(kind, **kw)
            h, s, f = dev.hist_scores(seq)
            n = len(idx)
            assert np.all(h.sum(axis=2) == W * H)
            hs = h.reshape(n, 48).astype(np.int64)
            l1 = np.abs(np.diff(hs, axis=0)).sum(axis=1)
            assert np.array_equal(s[1:], l1) and s[0] == 0
            assert np.array_equal(f, (2 * s.astype(np.int64) > W * H).astype(np.uint8))
            ks = np.arange(n) if checked is None else checked
            rh = np.stack([ref[int(idx[k])] for k in ks])
            assert np.array_equal(h[ks], rh)
            for k in ks[ks > 0]:
                rs, rf = orc.scores(np.stack([ref[int(idx[k - 1])], ref[int(idx[k])]]), W * H)
                assert s[k] == rs[1] and f[k] == rf[1], k
            assert s[0] == 0 and f[0] == 0
            scn.scn_seq_destroy(seq)
    finally:
        dev.close()


# flat single-colour frames: every pixel of a channel lands in one counter, the
# worst case for the kernel's 16-bit lane counters; the YUV triples reach every
# extreme of the unclamped ("extended") bins: R 30 / -14, G 27 / -11, B 33 / -18
FLAT_YUV = [(255, 255, 255), (0, 0, 0), (255, 0, 0), (0, 255, 255), (16, 240, 16), (235, 128, 128),
            (16, 128, 128), (255, 255, 0)]


def _flat_frames(W, H):
    out = np.empty((len(FLAT_YUV), W * H * 3 // 2), dtype=np.uint8)
    for i, (y, u, v) in enumerate(FLAT_YUV):
        out[i, :W * H] = y
        out[i, W * H::2] = u
        out[i, W * H + 1::2] = v
    return out


@pytest.mark.parametrize("W,H", [(1920, 1080), (3840, 2160)])
def test_flat_frames_all_work_assignments(scn, orc, W, H):
    frames = _flat_frames(W, H)
    n = len(frames)
    order = list(range(n)) + [n - 1, 0]  # ends with a repeat and a jump back
    rh = np.stack([orc.hist_frame(frames[i], W, H) for i in range(n)])
    rs, rf = orc.scores(rh[order], W * H)
    for c in range(3):  # one bin per channel, the whole frame in it
        assert np.all(rh[:, c].max(axis=1) == W * H)
    buf = torch.from_numpy(frames.reshape(-1)).cuda()
    dev = Dev(scn, buf, W, H, n)
    try:
        # default: contiguous row-pair ranges per CTA; then the work queue with items
        # of about a quarter frame and of whole frames (with two CTAs, the last two frames
        # are queued in quarters), and a one-CTA launch
        for tune in (None, dict(item_kpx=W * H // 4000), dict(item_kpx=W * H // 1000 + 1),
                     dict(item_kpx=W * H // 1000 + 1, grid=2), dict(grid=1)):
            seq = dev.seq(scn.SCN_GATHER, indices=order)
            h, s, f = dev.hist_scores(seq, tune=tune)
            assert np.array_equal(h, rh[order]), tune
            assert np.array_equal(s, rs) and np.array_equal(f, rf), tune
            scn.scn_seq_destroy(seq)
        # a batched plan over two sequences of the flat frames
        seqs = [dev.seq(scn.SCN_GATHER, indices=order), dev.seq(scn.SCN_RANGE, start=0, stop=n)]
        outs = [(torch.full((len(q), 48), -1, dtype=torch.int32, device="cuda"),
                 torch.full((len(q),), -1, dtype=torch.int32, device="cuda"),
                 torch.full((len(q),), 9, dtype=torch.uint8, device="cuda")) for q in (order, range(n))]
        p = scn.scn_plan_create(seqs, [o[0] for o in outs], [o[1] for o in outs], [o[2] for o in outs])
        scn.scn_plan_run(p)
        assert scn.scn_plan_sync_status(p) == scn.SCN_OK
        h0 = outs[0][0].cpu().numpy().view(np.uint32).reshape(-1, 3, 16)
        h1 = outs[1][0].cpu().numpy().view(np.uint32).reshape(-1, 3, 16)
        assert np.array_equal(h0, rh[order]) and np.array_equal(h1, rh)
        assert np.array_equal(outs[0][1].cpu().numpy().view(np.uint32), rs)
        assert np.array_equal(outs[0][2].cpu().numpy(), rf)
        scn.scn_plan_destroy(p)
        for q in seqs:
            scn.scn_seq_destroy(q)
    finally:
        dev.close()


# --------------------------------------------------------------------------- resize + thumbnails
def _bf16_rne(x: np.ndarray) -> np.ndarray:
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(torch.bfloat16).float().numpy()


@pytest.mark.parametrize("W,H,oh,ow,n", [(320, 180, 224, 224, 4), (1920, 1080, 224, 224, 2), (640, 360, 17, 31, 3),
                                         (64, 36, 224, 224, 2), (3840, 2160, 224, 224, 1)])
def test_resize_norm_parity(scn, orc, W, H, oh, ow, n):
    frames = random_nv12(W + oh, n, W, H)
    dev = Dev(scn, torch.from_numpy(frames.reshape(-1)).cuda(), W, H, n)
    try:
        seq = dev.seq(scn.SCN_RANGE, start=0, stop=n)
        o32 = torch.empty((n, 3, oh, ow), dtype=torch.float32, device="cuda")
        o16 = torch.empty((n, 3, oh, ow), dtype=torch.bfloat16, device="cuda")
        scn.scn_resize_norm(seq, oh, ow, MEAN, STD, scn.SCN_F32, o32)
        scn.scn_resize_norm(seq, oh, ow, MEAN, STD, scn.SCN_BF16, o16)
        g32 = o32.cpu().numpy()
        g16 = o16.float().cpu().numpy()
        for k in range(n):
            ref = orc.resize_norm_frame(frames[k], W, H, oh, ow, MEAN, STD)
            assert np.abs(g32[k] - ref).max() <= RESIZE_TOL
            assert np.array_equal(g16[k], _bf16_rne(g32[k]))
            r16 = _bf16_rne(ref)
            mag = np.maximum(np.abs(r16), 2.0 ** -120)
            ulp = 2.0 ** (np.floor(np.log2(mag)) - 7)
            # within one BF16 ulp of the rounded fp64 value, plus the FP32 tolerance
            # (near zero a BF16 ulp is finer than the FP32 error bound)
            assert np.all(np.abs(g16[k] - r16) <= ulp + RESIZE_TOL)
        scn.scn_seq_destroy(seq)
    finally:
        dev.close()


@pytest.mark.parametrize("W,H,oh,ow,n", [(320, 180, 224, 224, 3), (1920, 1080, 224, 224, 2), (64, 36, 7, 300, 2)])
def test_resize_norm_both_equals_single_calls(scn, orc, W, H, oh, ow, n):
    """One pass writing FP32 and BF16 gives exactly the two single-precision calls, and the FP32
    values stay within tolerance of the fp64 oracle."""
    frames = random_nv12(W + 7 * oh, n, W, H)
    dev = Dev(scn, torch.from_numpy(frames.reshape(-1)).cuda(), W, H, n)
    try:
        seq = dev.seq(scn.SCN_GATHER, indices=list(range(n))[::-1])
        a32 = torch.empty((n, 3, oh, ow), dtype=torch.float32, device="cuda")
        a16 = torch.empty((n, 3, oh, ow), dtype=torch.bfloat16, device="cuda")
        b32 = torch.full((n, 3, oh, ow), float("nan"), dtype=torch.float32, device="cuda")
        b16 = torch.full((n, 3, oh, ow), float("nan"), dtype=torch.bfloat16, device="cuda")
        scn.scn_resize_norm(seq, oh, ow, MEAN, STD, scn.SCN_F32, a32)
        scn.scn_resize_norm(seq, oh, ow, MEAN, STD, scn.SCN_BF16, a16)
        scn.scn_resize_norm_both(seq, oh, ow, MEAN, STD, b32, b16)
        assert torch.equal(a32, b32) and torch.equal(a16.view(torch.int16), b16.view(torch.int16))
        ref = orc.resize_norm_frame(frames[n - 1], W, H, oh, ow, MEAN, STD)
        assert np.abs(b32[0].cpu().numpy() - ref).max() <= RESIZE_TOL
        # a BF16 output one byte off its alignment is rejected before any launch
        odd = torch.empty(b16.numel() * 2 + 2, dtype=torch.uint8, device="cuda")[1:]
        with pytest.raises(scn.ScnError):
            scn.scn_resize_norm_both(seq, oh, ow, MEAN, STD, b32, odd)
        scn.scn_seq_destroy(seq)
    finally:
        dev.close()


def test_resize_generator_frames_tiny(scn, orc):
    W, H, T = TINY["width"], TINY["height"], TINY["num_frames"]
    v = _video(scn, TINY)
    try:
        dev = Dev(scn, _generate(scn, v, W, H, T), W, H, T)
        idx = [0, 100, 239]
        seq = dev.seq(scn.SCN_GATHER, indices=idx)
        out = torch.empty((3, 3, 224, 224), dtype=torch.float32, device="cuda")
        scn.scn_resize_norm(seq, 224, 224, MEAN, STD, scn.SCN_F32, out)
        ref_frames = orc.Video(MASTER_SEED, 0, W, H, T, TINY["num_shots"]).frames(idx)
        for k in range(3):
            ref = orc.resize_norm_frame(ref_frames[k], W, H, 224, 224, MEAN, STD)
            assert np.abs(out[k].cpu().numpy() - ref).max() <= RESIZE_TOL
        scn.scn_seq_destroy(seq)
        dev.close()
    finally:
        scn.scn_video_destroy(v)


@pytest.mark.parametrize("W,H", [(320, 180), (640, 360), (1920, 1080), (3840, 2160)])
def test_thumbs_parity(scn, orc, W, H):
    n = 3
    frames = random_nv12(W, n, W, H)
    dev = Dev(scn, torch.from_numpy(frames.reshape(-1)).cuda(), W, H, n)
    try:
        seq = dev.seq(scn.SCN_GATHER, indices=[2, 0, 1])
        out = torch.empty((n, 36, 64), dtype=torch.uint8, device="cuda")
        scn.scn_thumbs(seq, out)
        got = out.cpu().numpy()
        for j, k in enumerate([2, 0, 1]):
            assert np.array_equal(got[j], orc.thumb_frame(frames[k], W, H))
        # luma and coarse YUV thumbnails in one launch: the same luma, YUV equal to the oracle's
        out2 = torch.zeros((n, 36, 64), dtype=torch.uint8, device="cuda")
        yuv = torch.zeros((n, 3, 6, 32), dtype=torch.uint8, device="cuda")
        scn.scn_thumbs_yuv(seq, out2, yuv)
        assert torch.equal(out2, out)
        gy = yuv.cpu().numpy()
        for j, k in enumerate([2, 0, 1]):
            assert np.array_equal(gy[j], orc.thumb_yuv_frame(frames[k], W, H))
        # YUV only
        yuv2 = torch.zeros_like(yuv)
        scn.scn_thumbs_yuv(seq, None, yuv2)
        assert torch.equal(yuv2, yuv)
        scn.scn_seq_destroy(seq)
    finally:
        dev.close()


def test_mixed_calls_queued_back_to_back(scn):
    """Hist (contiguous ranges, region streams, whole-frame queue with its split tail), resize,
    thumbnails and a batched plan queued on one stream with no host wait between them (the
    kernels are launched as programmatic dependents of one another): every output equals the
    same call's made alone, with the device idle before and after it."""
    W, H = TINY["width"], TINY["height"]
    vt = _video(scn, TINY)
    bt = _generate(scn, vt, W, H, TINY["num_frames"])
    vh = _video(scn, HD)
    bh = _generate(scn, vh, HD["width"], HD["height"], 12)
    dt = Dev(scn, bt, W, H, TINY["num_frames"])
    dh = Dev(scn, bh, HD["width"], HD["height"], 12)
    qt = dt.seq(scn.SCN_STRIDE, start=0, stop=TINY["num_frames"], step=1)
    qt2 = dt.seq(scn.SCN_STRIDE, start=3, stop=TINY["num_frames"], step=2)
    scn.scn_seq_set_tune(qt2, item_kpx=20)  # queue of small items: region streams
    qh = dh.seq(scn.SCN_GATHER, indices=[0, 5, 5, 11, 2, 7, 1])
    qh2 = dh.seq(scn.SCN_STRIDE, start=0, stop=12, step=1)
    scn.scn_seq_set_tune(qh2, item_kpx=2100, grid=3)  # whole-frame queue, last 3 frames in quarters
    n = {q: scn.scn_seq_length(q) for q in (qt, qt2, qh, qh2)}
    plan_outs = [(torch.empty((n[q], 48), dtype=torch.int32, device="cuda"),
                  torch.empty(n[q], dtype=torch.int32, device="cuda"),
                  torch.empty(n[q], dtype=torch.uint8, device="cuda")) for q in (qt2, qh)]
    plan = scn.scn_plan_create([qt2, qh], [o[0] for o in plan_outs], [o[1] for o in plan_outs],
                               [o[2] for o in plan_outs])

    def hist(q):
        out = (torch.empty((n[q], 48), dtype=torch.int32, device="cuda"), torch.empty(n[q], dtype=torch.int32, device="cuda"),
               torch.empty(n[q], dtype=torch.uint8, device="cuda"))
        scn.scn_hist_scores(q, *out)
        return out

    def resize(q):
        f32 = torch.empty((n[q], 3, 224, 224), dtype=torch.float32, device="cuda")
        b16 = torch.empty((n[q], 3, 224, 224), dtype=torch.bfloat16, device="cuda")
        scn.scn_resize_norm_both(q, 224, 224, MEAN, STD, f32, b16)
        return f32, b16

    def thumbs(q):
        th = torch.empty((n[q], 36, 64), dtype=torch.uint8, device="cuda")
        yuv = torch.empty((n[q], 3, 6, 32), dtype=torch.uint8, device="cuda")
        scn.scn_thumbs_yuv(q, th, yuv)
        return th, yuv

    def run_plan():
        for o in plan_outs:
            for x in o:
                x.fill_(-1)
        scn.scn_plan_run(plan)
        return tuple(x.clone() for o in plan_outs for x in o)

    ops = [lambda: hist(qt), lambda: resize(qh), lambda: hist(qh2), lambda: thumbs(qt), lambda: hist(qh),
           run_plan, lambda: hist(qt2), lambda: resize(qt), lambda: hist(qh2), lambda: thumbs(qh)]
    try:
        alone = []
        for op in ops:
            torch.cuda.synchronize()
            alone.append([x.cpu() for x in op()])
            torch.cuda.synchronize()
        queued = [op() for op in ops]
        torch.cuda.synchronize()
        for i, (q, a) in enumerate(zip(queued, alone)):
            for x, y in zip(q, a):
                assert torch.equal(x.cpu(), y), i
        for q in (qt, qt2, qh, qh2):
            assert scn.scn_seq_sync_status(q) == scn.SCN_OK
        assert scn.scn_plan_sync_status(plan) == scn.SCN_OK
        # the whole-frame queue with a split tail and the plan agree with the plain launches
        h0, s0, f0 = alone[2]
        plain = dh.seq(scn.SCN_STRIDE, start=0, stop=12, step=1)
        h1, s1, f1 = dh.hist_scores(plain)
        scn.scn_seq_destroy(plain)
        assert np.array_equal(h0.numpy().view(np.uint32).reshape(-1, 3, 16), h1)
        assert np.array_equal(s0.numpy().view(np.uint32), s1) and np.array_equal(f0.numpy(), f1)
    finally:
        scn.scn_plan_destroy(plan)
        for q in (qt, qt2, qh, qh2):
            scn.scn_seq_destroy(q)
        dt.close()
        dh.close()
        scn.scn_video_destroy(vt)
        scn.scn_video_destroy(vh)


def test_argument_errors_before_launch(scn):
    W, H, n = 64, 36, 2
    buf = torch.zeros(n * W * H * 3 // 2, dtype=torch.uint8, device="cuda")
    dev = Dev(scn, buf, W, H, n)
    try:
        seq = dev.seq(scn.SCN_RANGE, start=0, stop=n)
        with pytest.raises(scn.ScnError):
            scn.scn_hist_scores(seq, None, None, None)
        odd = torch.zeros(100, dtype=torch.uint8, device="cuda")
        with pytest.raises(scn.ScnError):
            scn.scn_hist(seq, odd[1:])  # misaligned histogram pointer
        with pytest.raises(scn.ScnError):
            scn.scn_resize_norm(seq, 0, 224, MEAN, STD, scn.SCN_F32, odd)
        with pytest.raises(scn.ScnError):
            scn.scn_resize_norm(seq, 224, 224, MEAN, (0.2, 0.0, 0.2), scn.SCN_F32, odd)
        with pytest.raises(scn.ScnError):
            scn.scn_seq_set_tune(seq, chunk_rows=3)
        scn.scn_seq_destroy(seq)
    finally:
        dev.close()
