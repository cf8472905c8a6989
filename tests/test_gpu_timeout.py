"""The bounded device waits and the status word, exercised without faulting or
hanging the GPU: the fused kernel's producer withholds work (a test hook), every
consumer's bounded wait runs out after a short limit, the launch ends by itself
and scn_seq_sync_status reports SCN_ETIMEOUT.  The sync also zeroes the scratch
that the launch left part-way, so the next call on the same sequence is exact
against the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from tests.inputs import random_nv12  # noqa: E402

LIMIT_NS = 20_000_000  # 20 ms per wait in the launches that are made to time out


@pytest.fixture(scope="module")
def scn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_07339_b300 import scn as s
    return s


def _run(scn, seq, n):
    h = torch.full((n, 48), 0x5A5A, dtype=torch.int32, device="cuda")
    s = torch.full((n,), 0x5A5A, dtype=torch.int32, device="cuda")
    f = torch.full((n,), 9, dtype=torch.uint8, device="cuda")
    scn.scn_hist_scores(seq, h, s, f)
    st = scn.scn_seq_sync_status(seq)
    return st, h.cpu().numpy().view(np.uint32).reshape(n, 3, 16), s.cpu().numpy().view(np.uint32), f.cpu().numpy()


@pytest.mark.parametrize("W,H,T,tune,withhold", [
    (1920, 1080, 12, None, 0),               # row-pair ranges per table region, nothing handed out
    (1920, 1080, 12, None, 1),               # each region counts its range (frames split over CTAs), then waits
    # work queue: 240 items of 15 row pairs in chunks of 4 row pairs (4 chunks an item), at
    # most one item per table region
    (320, 180, 40, dict(item_kpx=10, chunk_rows=8), 2),
    (320, 180, 40, dict(item_kpx=10, chunk_rows=8), 3),
])
def test_withheld_work_times_out_and_the_next_call_is_exact(scn, orc, W, H, T, tune, withhold):
    frames = random_nv12(100 + withhold, T, W, H)
    buf = torch.from_numpy(frames.reshape(-1)).cuda()
    table = scn.scn_table_create(buf, W, H, T)
    seq = scn.scn_sample(table, scn.SCN_STRIDE, start=0, stop=T, step=1)
    try:
        if tune:
            scn.scn_seq_set_tune(seq, **tune)
        rh = orc.hist_batch(frames, W, H, nthreads=8)
        rs, rf = orc.scores(rh, W * H)
        # the hook rejects limits outside [100 us, 10 s]
        with pytest.raises(scn.ScnError):
            scn.scn_seq_set_wait_test(seq, 1000, withhold)
        scn.scn_seq_set_wait_test(seq, LIMIT_NS, withhold)
        for _ in range(2):  # twice: the reset must leave the scratch ready for any later launch
            st, _, _, _ = _run(scn, seq, T)
            assert st == scn.SCN_ETIMEOUT
        # the status word was cleared by the sync
        assert scn.scn_seq_sync_status(seq) == scn.SCN_OK
        scn.scn_seq_set_wait_test(seq, 0, -1)
        for _ in range(2):
            st, h, s, f = _run(scn, seq, T)
            assert st == scn.SCN_OK
            assert np.array_equal(h, rh)
            assert np.array_equal(s, rs) and np.array_equal(f, rf)
    finally:
        scn.scn_seq_destroy(seq)
        scn.scn_table_destroy(table)


def test_short_limit_without_withholding_is_exact(scn, orc):
    # a 10 ms limit is far above any wait of a normal launch: results stay exact
    W, H, T = 640, 360, 64
    frames = random_nv12(7, T, W, H)
    buf = torch.from_numpy(frames.reshape(-1)).cuda()
    table = scn.scn_table_create(buf, W, H, T)
    seq = scn.scn_sample(table, scn.SCN_STRIDE, start=0, stop=T, step=1)
    try:
        scn.scn_seq_set_wait_test(seq, 10_000_000, -1)
        st, h, s, f = _run(scn, seq, T)
        assert st == scn.SCN_OK
        rh = orc.hist_batch(frames, W, H, nthreads=8)
        rs, rf = orc.scores(rh, W * H)
        assert np.array_equal(h, rh) and np.array_equal(s, rs) and np.array_equal(f, rf)
    finally:
        scn.scn_seq_destroy(seq)
        scn.scn_table_destroy(table)


@pytest.mark.parametrize("pairs,withhold", [(600, 0), (600, 1), (7199, 3)])
def test_forward_withheld_batch_times_out_and_the_next_call_is_exact(scn, pairs, withhold):
    """The proposal network's inference kernel: its builder warps withhold the
    "input built" signal of one batch (a test hook), the bounded waits on it run
    out after 20 ms, the launch ends by itself and scn_cnn_sync_status reports
    SCN_ETIMEOUT; the next launch (nothing withheld) gives the logits of a launch
    made before, bit for bit."""
    from paper_1805_07339_b300.proposal import he_uniform
    g = torch.Generator(device="cpu").manual_seed(11 + withhold)
    th = torch.randint(0, 256, (pairs + 1, 36, 64), dtype=torch.uint8, generator=g).cuda()
    net = scn.scn_cnn_create(8)
    try:
        scn.scn_cnn_set_params(net, he_uniform(3))
        ref = torch.full((pairs,), float("nan"), dtype=torch.float32, device="cuda")
        scn.scn_cnn_forward(net, th, pairs, ref)
        assert scn.scn_cnn_sync_status(net) == scn.SCN_OK
        with pytest.raises(scn.ScnError):  # limits outside [100 us, 10 s] are refused
            scn.scn_cnn_set_wait_test(net, 1000, withhold)
        scn.scn_cnn_set_wait_test(net, LIMIT_NS, withhold)
        z = torch.full((pairs,), float("nan"), dtype=torch.float32, device="cuda")
        for _ in range(2):
            scn.scn_cnn_forward(net, th, pairs, z)
            assert scn.scn_cnn_sync_status(net) == scn.SCN_ETIMEOUT
        assert scn.scn_cnn_sync_status(net) == scn.SCN_OK  # the status word was cleared
        scn.scn_cnn_set_wait_test(net, 0, -1)
        z.fill_(float("nan"))
        scn.scn_cnn_forward(net, th, pairs, z)
        assert scn.scn_cnn_sync_status(net) == scn.SCN_OK
        assert torch.equal(z, ref)
    finally:
        scn.scn_cnn_destroy(net)
