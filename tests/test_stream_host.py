"""Host logic of the stream runner: the workload spec and the chunk plan (no GPU)."""
import numpy as np
import pytest

from paper_1805_07339_b300.workloads import STREAM, stream_spec


def test_stream_spec_shape():
    spec = stream_spec()
    assert len(spec) == STREAM["nvideos"]
    T = np.array([v["num_frames"] for v in spec])
    assert T.min() >= STREAM["min_len"] and T.max() <= STREAM["max_len"]
    # log-uniform: the median sits near the geometric mean of the bounds, the mean well above it
    gm = np.sqrt(STREAM["min_len"] * STREAM["max_len"])
    assert 0.8 * gm < np.median(T) < 1.25 * gm and T.mean() > 1.3 * gm
    ids = [v["video_id"] for v in spec]
    assert len(set(ids)) == len(ids)
    for v in spec[:200]:
        assert np.array_equal(v["stride"], np.arange(0, v["num_frames"], 24))
        g = v["gather"]
        assert len(g) == max(1, (v["num_frames"] + 50) // 100)
        assert np.all(np.diff(g) > 0) and g[0] >= 0 and g[-1] < v["num_frames"]
    assert stream_spec(nvideos=5)[3]["num_frames"] == spec[3]["num_frames"]  # prefix-stable


def test_plan_chunks():
    from paper_1805_07339_b300 import stream  # needs the library only for import, not a GPU
    spec = stream_spec(nvideos=60, seed=2, min_len=1800, max_len=54000)
    fb = 640 * 360 * 3 // 2
    need = [len(stream.sampled_rows(v)) * fb for v in spec]
    for limit in (max(need), 2 * max(need), 1 << 32):
        chunks = stream.plan_chunks(spec, limit)
        assert [i for c in chunks for i in c] == list(range(len(spec)))  # every video once, in order
        for c in chunks:
            assert sum(need[i] for i in c) <= limit
        for a, b in zip(chunks, chunks[1:]):  # greedy: the next video did not fit
            assert sum(need[i] for i in a) + need[b[0]] > limit
    with pytest.raises(ValueError):
        stream.plan_chunks(spec, max(need) - 1)
    v = spec[0]
    assert np.array_equal(stream.sampled_rows(v), np.union1d(v["stride"], v["gather"]))
