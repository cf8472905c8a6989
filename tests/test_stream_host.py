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


def test_state_run_patterns_and_input_sets():
    """The bounded-state run patterns and their input sets against the oracle's brute-force set."""
    from oracle import seqops
    from paper_1805_07339_b300 import stencil
    assert stencil.state_shards(10, 3) == (0, 4, 4, 3)
    assert stencil.state_shards(0, 3)[3] == 0
    assert stencil.state_sparse(100, 24) == (0, 1, 24, 5)
    assert stencil.state_sparse(100, 24, 5) == (5, 1, 24, 4)
    for n in (1, 7, 50, 301):
        for pat in (stencil.state_shards(n, 1), stencil.state_shards(n, 4), stencil.state_shards(n, 64),
                    stencil.state_sparse(n, 24), stencil.state_sparse(n, 5, 2), (3, 2, 7, 40)):
            for w in (0, 1, 3, 30):
                got = [i for a, b in stencil.state_inputs(*pat, w, n) for i in range(a, b)]
                assert got == seqops.bounded_state_inputs(*pat, w, n), (n, pat, w)
    # every 24th of 7200 outputs after 3 warmup elements: 4 inputs per output, 1 for output 0
    assert stencil.state_input_fraction(*stencil.state_sparse(7200, 24), 3, 7200) == (299 * 4 + 1) / 7200
