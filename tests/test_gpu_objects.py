"""Object creation does not wait for kernels already running: a video, a table and
a sequence created while a long generation launch runs on another stream return
before that launch ends, and the sequence made that way gives the same results as
one made on an idle GPU."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from tests.inputs import MASTER_SEED  # noqa: E402


@pytest.fixture(scope="module")
def scn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_07339_b300 import scn as s
    return s


def test_creation_behind_a_running_kernel(scn):
    W, H = 1920, 1080
    fb = W * H * 3 // 2
    # a small table the new objects refer to (its frames generated up front)
    T0 = 24
    v0 = scn.scn_video_create(MASTER_SEED, 5, W, H, T0, 3)
    small = torch.empty(T0 * fb, dtype=torch.uint8, device="cuda")
    scn.scn_generate(v0, small, 0, T0, fb)
    t0 = scn.scn_table_create(small, W, H, T0)
    ref = scn.scn_sample(t0, scn.SCN_STRIDE, start=0, stop=T0, step=1)  # made on an idle GPU (also warms the pool)
    torch.cuda.synchronize()
    # a long launch on another stream: about 2000 1080p frames of generation
    T = 2000
    vbig = scn.scn_video_create(MASTER_SEED, 6, W, H, T, 10)
    big = torch.empty(T * fb, dtype=torch.uint8, device="cuda")
    st = torch.cuda.Stream()
    objs = []
    try:
        scn.scn_generate(vbig, big, 0, T, fb, stream=st)
        c0 = time.perf_counter()
        v1 = scn.scn_video_create(MASTER_SEED, 7, W, H, 100, 4)
        t1 = scn.scn_table_create(small, W, H, T0)
        s1 = scn.scn_sample(t1, scn.SCN_STRIDE, start=0, stop=T0, step=1)
        s2 = scn.scn_sample(t1, scn.SCN_GATHER, indices=[5, 3, 22, 3])
        c1 = time.perf_counter()
        objs = [("s", s1), ("s", s2), ("t", t1), ("v", v1)]
        still_running = not st.query()
        st.synchronize()
        assert still_running, f"creation took {1e3 * (c1 - c0):.2f} ms and the launch had ended"
        # results of the sequence created behind the running launch
        outs = []
        for s in (ref, s1):
            h = torch.empty((T0, 48), dtype=torch.int32, device="cuda")
            sc = torch.empty(T0, dtype=torch.int32, device="cuda")
            fl = torch.empty(T0, dtype=torch.uint8, device="cuda")
            scn.scn_hist_scores(s, h, sc, fl)
            outs.append((h, sc, fl))
        torch.cuda.synchronize()
        for a, b in zip(*outs):
            assert torch.equal(a, b)
        h2 = torch.empty((4, 48), dtype=torch.int32, device="cuda")
        scn.scn_hist(s2, h2)
        torch.cuda.synchronize()
        hr = outs[0][0].cpu().numpy()
        assert np.array_equal(h2.cpu().numpy(), hr[[5, 3, 22, 3]])
    finally:
        st.synchronize()
        for kind, o in objs:
            {"s": scn.scn_seq_destroy, "t": scn.scn_table_destroy, "v": scn.scn_video_destroy}[kind](o)
        scn.scn_seq_destroy(ref)
        scn.scn_table_destroy(t0)
        scn.scn_video_destroy(v0)
        scn.scn_video_destroy(vbig)
