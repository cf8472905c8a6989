"""The shared-memory reduction probe that the hist kernel's binding-unit roofline
is stated against: every CTA reports its cycles, and the rate it implies lies
between half a warp-wide reduction and one per SM clock (one conflict-free
wavefront per clock is the most shared memory can serve)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_07339_b300 import scn as s
    return s


@pytest.fixture(scope="module")
def bench():
    import bench as b  # the probe lives in the benchmark's measurement library
    return b


def test_probe_rate_is_plausible(scn, bench):
    sms = scn.scn_device_sm_count()
    cyc = torch.zeros(sms, dtype=torch.int64, device="cuda")
    iters = 2048
    bench.probe_shared_reductions(iters, sms, cyc)
    torch.cuda.synchronize()
    c = cyc.cpu().numpy()
    assert (c > 0).all()
    warps, reds = bench.probe_geometry()
    assert warps >= 4 and reds in (2, 3)
    rate = warps * 8 * iters / np.median(c)
    assert 0.5 <= rate <= 1.05, rate


def test_probe_rejects_bad_arguments(scn, bench):
    cyc = torch.zeros(4, dtype=torch.int64, device="cuda")
    for iters, grid in ((0, 1), (1 << 21, 1), (1, 0), (1, 70000)):
        with pytest.raises(RuntimeError):
            bench.probe_shared_reductions(iters, grid, cyc)
    with pytest.raises(RuntimeError):
        bench.probe_shared_reductions(8, 1, cyc.view(torch.uint8)[1:])
