"""Batched plans: many uneven sequences in one persistent launch fed by a work
queue, CUDA-graph replay and the autotuner, against the CPU oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1805_07339_b300.workloads import MASTER_SEED, batched_spec  # noqa: E402


@pytest.fixture(scope="module")
def scn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_07339_b300 import scn as s
    return s


class Batch:
    """Generate only the sampled rows of every video (strided tables), one
    sequence per video, and one output triple per sequence."""

    def __init__(self, scn, spec):
        self.scn, self.spec = scn, spec
        self.videos, self.tables, self.seqs, self.outs, self.bufs = [], [], [], [], []
        for v in spec:
            W, H, T = v["width"], v["height"], v["num_frames"]
            fb = W * H * 3 // 2
            rows = np.unique(v["frames"])
            vid = scn.scn_video_create(MASTER_SEED, v["video_id"], W, H, T, v["num_shots"])
            buf = torch.empty(max(len(rows), 1) * fb, dtype=torch.uint8, device="cuda")
            if len(rows):
                scn.scn_generate_frames(vid, torch.from_numpy(rows).cuda(), buf, fb)
            t = scn.scn_table_create(buf, W, H, T, rows=rows.tolist())
            s = scn.scn_sample(t, scn.SCN_GATHER, indices=v["frames"].tolist())
            n = len(v["frames"])
            self.outs.append((torch.full((max(n, 1), 48), -1, dtype=torch.int32, device="cuda"),
                              torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda"),
                              torch.full((max(n, 1),), 9, dtype=torch.uint8, device="cuda")))
            self.videos.append(vid)
            self.tables.append(t)
            self.seqs.append(s)
            self.bufs.append(buf)
        torch.cuda.synchronize()

    def plan(self, tune=None):
        return self.scn.scn_plan_create(self.seqs, [o[0] for o in self.outs], [o[1] for o in self.outs],
                                        [o[2] for o in self.outs], tune)

    def results(self):
        torch.cuda.synchronize()
        res = []
        for v, (h, s, f) in zip(self.spec, self.outs):
            n = len(v["frames"])
            res.append((h[:n].cpu().numpy().view(np.uint32).reshape(n, 3, 16), s[:n].cpu().numpy().view(np.uint32),
                        f[:n].cpu().numpy()))
        return res

    def close(self):
        for s in self.seqs:
            self.scn.scn_seq_destroy(s)
        for t in self.tables:
            self.scn.scn_table_destroy(t)
        for v in self.videos:
            self.scn.scn_video_destroy(v)


def _oracle_check(orc, v, got, picks):
    """Elements `picks` of video v (and their predecessors) against the oracle."""
    W, H = v["width"], v["height"]
    ov = orc.Video(MASTER_SEED, v["video_id"], W, H, v["num_frames"], v["num_shots"])
    need = sorted(set(picks) | {p - 1 for p in picks if p > 0})
    frames = ov.frames(v["frames"][need], nthreads=8)
    rh = orc.hist_batch(frames, W, H, nthreads=8)
    pos = {k: i for i, k in enumerate(need)}
    h, s, f = got
    for k in picks:
        assert np.array_equal(h[k], rh[pos[k]]), (v["video_id"], k)
        if k > 0:
            rs, rf = orc.scores(np.stack([rh[pos[k - 1]], rh[pos[k]]]), W * H)
            assert s[k] == rs[1] and f[k] == rf[1]
        else:
            assert s[0] == 0 and f[0] == 0


def _properties(v, got):
    W, H = v["width"], v["height"]
    h, s, f = got
    n = len(v["frames"])
    if n == 0:
        return
    assert np.all(h.sum(axis=2) == W * H)
    l1 = np.abs(np.diff(h.reshape(n, 48).astype(np.int64), axis=0)).sum(axis=1)
    assert s[0] == 0 and np.array_equal(s[1:], l1)
    assert np.array_equal(f, (2 * s.astype(np.int64) > W * H).astype(np.uint8))


def test_plan_small_mixed_against_oracle(scn, orc):
    res = [(640, 360), (1280, 720), (1920, 1080), (3840, 2160)]
    spec = batched_spec(nvideos=10, min_len=24, max_len=90, seed=11, resolutions=res)
    b = Batch(scn, spec)
    try:
        p = b.plan()
        scn.scn_plan_run(p)
        assert scn.scn_plan_sync_status(p) == scn.SCN_OK
        got = b.results()
        for v, g in zip(spec, got):
            _properties(v, g)
            n = len(v["frames"])
            if n == 0:
                continue
            picks = list(range(n)) if v["width"] <= 1280 and n <= 40 else sorted({0, 1, n // 2, n - 1})
            _oracle_check(orc, v, g, picks)
        info = scn.scn_plan_info(p)
        assert info["frames"] == sum(len(v["frames"]) for v in spec)
        scn.scn_plan_destroy(p)
    finally:
        b.close()


def test_plan_of_small_frames_against_oracle(scn, orc):
    """A plan whose frames are all at most 1 Mpx runs the region-stream kernel
    (each table region counts whole items of its own); every element of every
    video against the oracle, twice (the plan's queue resets itself)."""
    res = [(320, 180), (640, 360), (1280, 720)]
    spec = batched_spec(nvideos=9, min_len=20, max_len=60, seed=23, resolutions=res)
    b = Batch(scn, spec)
    try:
        p = b.plan()
        for _ in range(2):
            scn.scn_plan_run(p)
            assert scn.scn_plan_sync_status(p) == scn.SCN_OK
            got = b.results()
            for v, g in zip(spec, got):
                _properties(v, g)
                n = len(v["frames"])
                if n:
                    _oracle_check(orc, v, g, list(range(n)))
        scn.scn_plan_destroy(p)
    finally:
        b.close()


def test_plan_matches_single_sequences_and_graph_replay(scn):
    spec = batched_spec(nvideos=16, min_len=40, max_len=160, seed=5)
    b = Batch(scn, spec)
    try:
        # reference: each sequence on its own through scn_hist_scores
        ref = []
        for v, s in zip(spec, b.seqs):
            n = len(v["frames"])
            h = torch.zeros((max(n, 1), 48), dtype=torch.int32, device="cuda")
            sc = torch.zeros(max(n, 1), dtype=torch.int32, device="cuda")
            fl = torch.zeros(max(n, 1), dtype=torch.uint8, device="cuda")
            scn.scn_hist_scores(s, h, sc, fl)
            ref.append((h[:n].cpu(), sc[:n].cpu(), fl[:n].cpu()))
        stream = torch.cuda.Stream()
        p = b.plan(dict(chunk_rows=0, grid=0, item_kpx=700))
        with torch.cuda.stream(stream):
            scn.scn_plan_capture_graph(p, stream)
            for rep in range(3):
                for o in b.outs:
                    for t in o:
                        t.fill_(-1)
                scn.scn_plan_replay(p, stream)
                stream.synchronize()
                for (h, sc, fl), (rh, rs, rf), v in zip(b.outs, ref, spec):
                    n = len(v["frames"])
                    assert torch.equal(h[:n].cpu(), rh) and torch.equal(sc[:n].cpu(), rs)
                    assert torch.equal(fl[:n].cpu(), rf)
        assert scn.scn_plan_sync_status(p, stream) == scn.SCN_OK
        scn.scn_plan_destroy(p)
    finally:
        b.close()


def test_plan_autotune_keeps_results(scn):
    spec = batched_spec(nvideos=8, min_len=30, max_len=120, seed=8)
    b = Batch(scn, spec)
    try:
        p = b.plan()
        scn.scn_plan_run(p)
        first = b.results()
        best, ms = scn.scn_plan_autotune(p, reps=1)
        assert ms > 0 and best["item_kpx"] > 0
        assert scn.scn_plan_get_tune(p) == best
        for o in b.outs:
            for t in o:
                t.fill_(-1)
        scn.scn_plan_run(p)
        for a, c in zip(first, b.results()):
            for x, y in zip(a, c):
                assert np.array_equal(x, y)
        scn.scn_plan_destroy(p)
    finally:
        b.close()


def test_plan_rejects_bad_arguments(scn):
    spec = batched_spec(nvideos=2, min_len=10, max_len=20, seed=1, resolutions=[(640, 360)])
    b = Batch(scn, spec)
    try:
        with pytest.raises(scn.ScnError):  # a sequence may appear once
            scn.scn_plan_create([b.seqs[0], b.seqs[0]], [b.outs[0][0]] * 2, [b.outs[0][1]] * 2, [b.outs[0][2]] * 2)
        with pytest.raises(scn.ScnError):
            scn.scn_plan_create(b.seqs, [None, None], [o[1] for o in b.outs], [o[2] for o in b.outs])
        p = b.plan()
        with pytest.raises(scn.ScnError):
            scn.scn_plan_replay(p)  # nothing captured yet
        with pytest.raises(scn.ScnError):
            scn.scn_plan_set_tune(p, chunk_rows=3)
        scn.scn_plan_destroy(p)
    finally:
        b.close()


def _picks(rng, n, m=32):
    """m distinct elements (all of them if fewer), always with the first and last."""
    if n <= m:
        return list(range(n))
    return sorted(set(rng.choice(np.arange(1, n - 1), size=m - 2, replace=False).tolist()) | {0, n - 1})


def test_plan_full_batched_workload(scn, orc):
    """The full 64-video batch (only sampled rows materialised, ~200 GB), one
    launch; every element checked for mass and score consistency, and at least
    32 elements per video (all of a shorter one) against the oracle."""
    spec = batched_spec()
    free, _ = torch.cuda.mem_get_info()
    need = sum(len(np.unique(v["frames"])) * v["width"] * v["height"] * 3 // 2 for v in spec)
    if need > 0.8 * free:
        pytest.skip(f"needs {need / 1e9:.0f} GB of device memory")
    b = Batch(scn, spec)
    try:
        p = b.plan()
        scn.scn_plan_run(p)
        assert scn.scn_plan_sync_status(p) == scn.SCN_OK
        got = b.results()
        rng = np.random.default_rng(0)
        for v, g in zip(spec, got):
            _properties(v, g)
            n = len(v["frames"])
            if n:
                picks = _picks(rng, n)
                assert len(picks) >= min(n, 32)
                _oracle_check(orc, v, g, picks)
        scn.scn_plan_destroy(p)
    finally:
        b.close()
        torch.cuda.empty_cache()
