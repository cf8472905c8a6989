"""News-archive-shaped stream: chunked on-device generation of sampled rows,
one batched plan per chunk; every video's stride-24 and gather sequences against
the oracle (small streams), and the full 2000-video stream checked by
properties that hold at any size plus oracle spot checks."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1805_07339_b300.workloads import MASTER_SEED, stream_spec  # noqa: E402


@pytest.fixture(scope="module")
def scn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_07339_b300 import scn as s
    return s


def _oracle_video(orc, v, seqs=("stride", "gather")):
    W, H, T = v["width"], v["height"], v["num_frames"]
    ov = orc.Video(MASTER_SEED, v["video_id"], W, H, T, 0, 1)
    out = {}
    for name in seqs:
        idx = v[name]
        frames = ov.frames(idx, nthreads=8)
        h = orc.hist_batch(frames, W, H, nthreads=8)
        sc, fl = orc.scores(h, W * H)
        out[name] = (h, sc, fl)
    return out


def test_small_stream_matches_oracle(scn, orc):
    from paper_1805_07339_b300 import stream
    spec = stream_spec(nvideos=9, seed=11, min_len=200, max_len=1400, id0=300000)
    # chunks just big enough for the largest video: several chunks, both buffers reused
    fb = spec[0]["width"] * spec[0]["height"] * 3 // 2
    chunk = max(len(stream.sampled_rows(v)) for v in spec) * fb
    assert len(stream.plan_chunks(spec, chunk)) >= 3
    res = stream.run_stream(torch, spec, chunk_bytes=chunk, keep_hist=range(len(spec)))
    assert res.chunks >= 3 and res.videos == len(spec)
    assert res.frames == sum(len(v["stride"]) + len(v["gather"]) for v in spec)
    for i, v in enumerate(spec):
        ref = _oracle_video(orc, v)
        hs, hg = res.hist[i]
        assert np.array_equal(hs.astype(np.int64), ref["stride"][0].reshape(-1, 48))
        assert np.array_equal(hg.astype(np.int64), ref["gather"][0].reshape(-1, 48))
        assert np.array_equal(res.stride[i][0], ref["stride"][1]) and np.array_equal(res.stride[i][1], ref["stride"][2])
        assert np.array_equal(res.gather[i][0], ref["gather"][1]) and np.array_equal(res.gather[i][1], ref["gather"][2])


def test_full_news_stream(scn, orc):
    """2000 videos of 1800-54000 frames (30.6 M frames logical, 542 GB of sampled rows in 4 GB chunks)."""
    from paper_1805_07339_b300 import stream
    spec = stream_spec()
    lens = np.array([v["num_frames"] for v in spec])
    spot = [int(np.argmin(lens)), int(np.argsort(lens)[len(lens) // 2]), len(spec) - 1]
    res = stream.run_stream(torch, spec, keep_hist=spot)
    W, H = spec[0]["width"], spec[0]["height"]
    assert res.videos == 2000 and res.chunks > 100
    for i in range(len(spec)):
        for sc, fl in (res.stride[i], res.gather[i]):
            assert sc[0] == 0
            assert np.array_equal(fl, (2 * sc.astype(np.int64) > W * H).astype(np.uint8))
            assert sc.max() <= 6 * W * H
    for i in spot:
        ref = _oracle_video(orc, spec[i])
        hs, hg = res.hist[i]
        assert np.array_equal(hs.astype(np.int64), ref["stride"][0].reshape(-1, 48))
        assert np.array_equal(hg.astype(np.int64), ref["gather"][0].reshape(-1, 48))
        assert np.array_equal(res.stride[i][0], ref["stride"][1])
    # geometric shots (mean ~65 frames): about a third of the stride-24 pairs cross a boundary
    frac = np.mean(np.concatenate([res.stride[i][1][1:] for i in range(len(spec))]))
    assert 0.2 < frac < 0.45, frac


def test_stream_proposal_model(scn):
    """A model trained on stride-24 pairs of stream-shaped videos (disjoint ids)
    finds the boundaries between sampled frames of the stream's first 100 videos."""
    from paper_1805_07339_b300 import proposal
    r = proposal.run_stream_proposal(torch, eval_spec=stream_spec(nvideos=100))
    assert r["pairs"] > 50000 and 0.2 < r["positives"] / r["pairs"] < 0.45
    assert r["recall"] >= 0.99 and r["precision"] >= 0.95, r
