"""The allocation-free hist+score entry point against the regular one.

scn_hist_scores_noalloc exists for callers that may not allocate device
memory themselves (for example code running inside an allocator hook, or a
host that owns every device buffer and only hands out fixed regions).  It keeps
its scratch in a fixed array inside the library.  This file is collected last
on purpose, so a run that stops at the first failure has run everything else.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from tests.inputs import MASTER_SEED, TINY, random_indices, random_nv12  # noqa: E402


@pytest.fixture(scope="module")
def scn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_07339_b300 import scn as s
    return s


def _regular(scn, buf, W, H, T, idx):
    t = scn.scn_table_create(buf, W, H, T)
    seq = scn.scn_sample(t, scn.SCN_GATHER, indices=[int(i) for i in idx])
    n = len(idx)
    h = torch.zeros((n, 48), dtype=torch.int32, device="cuda")
    s = torch.zeros(n, dtype=torch.int32, device="cuda")
    f = torch.zeros(n, dtype=torch.uint8, device="cuda")
    scn.scn_hist_scores(seq, h, s, f)
    assert scn.scn_seq_sync_status(seq) == scn.SCN_OK
    scn.scn_seq_destroy(seq)
    scn.scn_table_destroy(t)
    return h.cpu(), s.cpu(), f.cpu()


def _noalloc(scn, buf, W, H, idx):
    n = len(idx)
    slots = torch.tensor([int(i) for i in idx], dtype=torch.int32, device="cuda")
    h = torch.full((n, 48), -1, dtype=torch.int32, device="cuda")
    s = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    f = torch.full((n,), 9, dtype=torch.uint8, device="cuda")
    scn.scn_hist_scores_noalloc(buf, W, H, W * H * 3 // 2, slots, h, s, f)
    torch.cuda.synchronize()
    return h.cpu(), s.cpu(), f.cpu()


def test_noalloc_matches_regular_entry_point_twice(scn):
    # call 1: generator frames, stride-1 order; call 2: random bytes at 1080p,
    # gathered with repeats (exercises the scratch left by call 1)
    W, H, T = TINY["width"], TINY["height"], TINY["num_frames"]
    fb = W * H * 3 // 2
    v = scn.scn_video_create(MASTER_SEED, 0, W, H, T, TINY["num_shots"])
    try:
        buf = torch.empty(T * fb, dtype=torch.uint8, device="cuda")
        scn.scn_generate(v, buf, 0, T, fb)
        idx1 = np.arange(T)
        a = _noalloc(scn, buf, W, H, idx1)
        b = _regular(scn, buf, W, H, T, idx1)
        for x, y in zip(a, b):
            assert torch.equal(x, y)
    finally:
        scn.scn_video_destroy(v)
    W2, H2, T2 = 1920, 1080, 4
    frames = torch.from_numpy(random_nv12(77, T2, W2, H2).reshape(-1)).cuda()
    idx2 = random_indices(3, T2, 9, distinct=False)
    a2 = _noalloc(scn, frames, W2, H2, idx2)
    b2 = _regular(scn, frames, W2, H2, T2, idx2)
    for x, y in zip(a2, b2):
        assert torch.equal(x, y)


def test_noalloc_whole_frame_queue_with_split_tail(scn):
    """Enough 1080p frames for a whole-frame queue (at least eight per CTA), whose last frames are
    queued in quarters through the partial accumulators of the library's fixed scratch: the same
    histograms, scores and flags as the regular entry point."""
    W, H, T = 1920, 1080, 1200
    v = scn.scn_video_create(MASTER_SEED, 3, W, H, T, 10)
    buf = torch.empty(T * W * H * 3 // 2, dtype=torch.uint8, device="cuda")
    try:
        scn.scn_generate(v, buf, 0, T, W * H * 3 // 2)
        idx = list(range(T))
        idx[600:610] = idx[600:610][::-1]  # a stretch out of order: its scores cross shots both ways
        a = _noalloc(scn, buf, W, H, idx)
        b = _regular(scn, buf, W, H, T, idx)
        for x, y in zip(a, b):
            assert torch.equal(x, y)
        assert int(a[0].sum()) == 3 * W * H * T
    finally:
        scn.scn_video_destroy(v)
        del buf
        torch.cuda.empty_cache()


def test_noalloc_limits(scn):
    buf = torch.zeros(64 * 36 * 3 // 2, dtype=torch.uint8, device="cuda")
    out = torch.zeros(16, dtype=torch.int32, device="cuda")
    flag = torch.zeros(16, dtype=torch.uint8, device="cuda")
    too_many = torch.zeros(16385, dtype=torch.int32, device="cuda")
    with pytest.raises(scn.ScnError) as e:
        scn.scn_hist_scores_noalloc(buf, 64, 36, 64 * 36 * 3 // 2, too_many, out, out, flag)
    assert e.value.status == scn.SCN_ERANGE
    empty = torch.zeros(0, dtype=torch.int32, device="cuda")
    scn.scn_hist_scores_noalloc(buf, 64, 36, 64 * 36 * 3 // 2, empty, out, out, flag)
