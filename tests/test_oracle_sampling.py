"""Pins for the oracle's sampling operator (Sec. 3.2, sampling operations; the
stride / range / gather / keyframe access patterns of Sec. 5.1.1), against lists
written out by hand."""
import numpy as np
import pytest


def test_stride_lists(orc):
    S = orc.SAMPLE_STRIDE
    assert orc.sample(S, 40, start=5, stop=30, step=7).tolist() == [5, 12, 19, 26]
    assert orc.sample(S, 10, start=0, stop=10, step=1).tolist() == [0, 1, 2, 3, 4, 5, 6, 7, 8, 9]
    assert orc.sample(S, 10, start=9, stop=10, step=4).tolist() == [9]
    assert orc.sample(S, 10, start=3, stop=3, step=2).tolist() == []
    # the 1080p stride-24 sequence: 0, 24, ..., 7176 (300 elements; 7200 is not a frame)
    s24 = orc.sample(S, 7200, start=0, stop=7200, step=24)
    assert len(s24) == 300 and s24[0] == 0 and s24[1] == 24 and s24[-1] == 7176
    assert set(np.diff(s24).tolist()) == {24}


def test_range_excludes_stop(orc):
    R = orc.SAMPLE_RANGE
    assert orc.sample(R, 10, start=3, stop=7).tolist() == [3, 4, 5, 6]
    assert orc.sample(R, 10, start=0, stop=1).tolist() == [0]
    assert orc.sample(R, 10, start=4, stop=4).tolist() == []
    # a range ignores any step it is given
    assert orc.sample(R, 10, start=2, stop=5, step=3).tolist() == [2, 3, 4]


def test_gather_keeps_order_and_duplicates(orc):
    G = orc.SAMPLE_GATHER
    assert orc.sample(G, 10, indices=[5, 2, 5, 9, 0]).tolist() == [5, 2, 5, 9, 0]
    assert orc.sample(G, 10, indices=[]).tolist() == []


def test_keyframes_sorted_unique(orc):
    K = orc.SAMPLE_KEYFRAME
    assert orc.sample(K, 300, keyframes=[208, 0, 104, 50, 104]).tolist() == [0, 50, 104, 208]


def test_out_of_range_rejected(orc):
    with pytest.raises(ValueError):
        orc.sample(orc.SAMPLE_STRIDE, 10, start=0, stop=11, step=1)
    with pytest.raises(ValueError):
        orc.sample(orc.SAMPLE_STRIDE, 10, start=-1, stop=5, step=1)
    with pytest.raises(ValueError):
        orc.sample(orc.SAMPLE_STRIDE, 10, start=0, stop=5, step=0)
    with pytest.raises(ValueError):
        orc.sample(orc.SAMPLE_GATHER, 10, indices=[0, 10])
    with pytest.raises(ValueError):
        orc.sample(orc.SAMPLE_GATHER, 10, indices=[-1])


def test_video_keyframes_merge_interval_and_shot_starts(orc):
    # every 104th frame plus every shot start, nothing else
    v = orc.Video(20180805, 0, 320, 180, 240, num_shots=8)
    starts = v.shot_starts().tolist()
    assert starts[0] == 0 and len(starts) == 8 and starts == sorted(starts)
    kf = v.keyframes().tolist()
    assert kf == sorted(set([0, 104, 208] + starts))
    # a video shorter than one interval: its shot starts only (frame 0 among them)
    w = orc.Video(20180805, 3, 64, 36, 50, num_shots=3)
    assert w.keyframes().tolist() == sorted(set([0] + w.shot_starts().tolist()))
